// k_standard.cu -- the "standard" per-element encrypted matrix product (Section 5.2.3):
// Y_j = sum_f w[f][j] X_f + Delta [b_j]_t, with X_f holding feature f of individual i in
// slot i. Multiplying a ciphertext by an integer scalar is coefficient-wise, so the kernel
// streams the coefficient form of all f ciphertexts from HBM exactly once.
//
// Streaming: each CTA owns a 256-word tile of every ciphertext (2 KB of feature f's
// ciphertext per feature) and a range of features (split-K). One thread issues
// cp.async.bulk copies of 16 feature rows plus their 16-wide weight rows into a 3-stage
// shared-memory ring; completion is counted on one mbarrier per stage (bounded waits: a
// timeout sets the context's error word and the CTA drains its copies and returns).
// Arithmetic: each residue x < 2^bits is split at s = ceil(bits/2) so that w * half fits a
// signed 32 x 32 -> 64 multiply-add; the per-split signed 64-bit sums are reduced mod q by
// k_standard_finalize (exact while |w| f 2^max(s, bits-s) < 2^63).
#include <algorithm>

#include "bfv_internal.h"

namespace {

constexpr int kE = 256;                   // ciphertext words per tile = threads per CTA
constexpr int kF = 16;                    // features per pipeline stage
constexpr int kS = 3;                     // stages in flight
constexpr int kNY = 16;                   // classes per pass (weights packed 16 wide)
constexpr long long kWaitLimit = 1ll << 24;

struct StdSmem {
    u64 x[kS][kF][kE];
    int w[kS][kF][kNY];
    u64 full[kS];
};

__global__ void __launch_bounds__(kE, 2) k_standard_stream(const int *__restrict__ W16, const u64 *__restrict__ X,
                                                           size_t ctw, size_t F, size_t fper, int split_bits,
                                                           longlong2 *partial, int *err, u32 extra_tx,
                                                           long long wait_limit) {
    extern __shared__ __align__(128) unsigned char raw[];
    StdSmem &s = *reinterpret_cast<StdSmem *>(raw);
    const size_t ntiles = ctw / kE;
    const size_t tile = blockIdx.x % ntiles, split = blockIdx.x / ntiles;
    const size_t e0 = tile * kE;
    const size_t fa = split * fper, fb = std::min(F, fa + fper);
    const int nst = fa < fb ? (int)((fb - fa + kF - 1) / kF) : 0;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < kS; ++i) mbar_init(&s.full[i], 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int st) {
        const int slot = st % kS;
        const size_t f0 = fa + (size_t)st * kF;
        const int nf = (int)std::min((size_t)kF, fb - f0);
        // extra_tx (failure injection only) adds bytes that never arrive to the first stage
        mbar_expect_tx(&s.full[slot], (u32)nf * (kE * 8 + kNY * 4) + (st == 0 ? extra_tx : 0u));
        for (int ff = 0; ff < nf; ++ff) bulk_g2s(&s.x[slot][ff][0], X + (f0 + ff) * ctw + e0, kE * 8, &s.full[slot]);
        bulk_g2s(&s.w[slot][0][0], W16 + f0 * kNY, (u32)nf * kNY * 4, &s.full[slot]);
    };
    if (tid == 0)
        for (int st = 0; st < (nst < kS ? nst : kS); ++st) issue(st);

    long long lo[kNY], hi[kNY];
#pragma unroll
    for (int j = 0; j < kNY; ++j) { lo[j] = 0; hi[j] = 0; }
    const u64 lmask = (1ull << split_bits) - 1;
    for (int st = 0; st < nst; ++st) {
        const int slot = st % kS;
        const bool ok = mbar_wait(&s.full[slot], (u32)((st / kS) & 1), wait_limit);
        if (__syncthreads_or(!ok)) {
            // a copy did not complete in time: report, drain what is in flight, return
            if (tid == 0) {
                atomicOr(err, 1);
                for (int k = st; k < (nst < st + kS ? nst : st + kS); ++k)
                    mbar_wait(&s.full[k % kS], (u32)((k / kS) & 1), wait_limit);
            }
            __syncthreads();
            return;
        }
        const size_t f0 = fa + (size_t)st * kF;
        const int nf = (int)std::min((size_t)kF, fb - f0);
        for (int ff = 0; ff < nf; ++ff) {
            const u64 x = s.x[slot][ff][tid];
            const int xl = (int)(x & lmask), xh = (int)(x >> split_bits);
            const int4 *wv = reinterpret_cast<const int4 *>(&s.w[slot][ff][0]);
#pragma unroll
            for (int q4 = 0; q4 < kNY / 4; ++q4) {
                const int4 w4 = wv[q4];
                const int ws[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    lo[q4 * 4 + u] += (long long)ws[u] * xl;
                    hi[q4 * 4 + u] += (long long)ws[u] * xh;
                }
            }
        }
        __syncthreads();                               // the slot is free again
        if (tid == 0 && st + kS < nst) issue(st + kS);
    }
    longlong2 *out = partial + split * kNY * ctw + e0 + tid;
#pragma unroll
    for (int j = 0; j < kNY; ++j) out[(size_t)j * ctw] = make_longlong2(lo[j], hi[j]);
}

// Y[j0 + j][e] = (sum over splits of hi 2^s + lo) mod q + Delta [b]_t at coefficient 0 of c0.
__global__ void __launch_bounds__(256) k_standard_finalize(const ModTab *__restrict__ mods, int N, int L, size_t ctw,
                                                           int splits, int nj, int j0, int split_bits,
                                                           const longlong2 *__restrict__ partial,
                                                           const u64 *__restrict__ bias_delta, u64 *Y) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)nj * ctw) return;
    const int j = (int)(idx / ctw);
    const size_t e = idx % ctw;
    long long lo = 0, hi = 0;
    for (int sp = 0; sp < splits; ++sp) {
        const longlong2 v = partial[((size_t)sp * kNY + j) * ctw + e];
        lo += v.x;
        hi += v.y;
    }
    const int l = (int)((e / N) % L);
    const ModTab T = mods[l];
    const long long q = (long long)T.q;
    long long h = hi % q; if (h < 0) h += q;
    long long a = lo % q; if (a < 0) a += q;
    const u64 sh = (1ull << split_bits) % T.q;
    u64 v = add_mod(mul_barrett((u64)h, sh, T.q, T.mu, T.bits), (u64)a, T.q);
    if (e < (size_t)L * N && e % N == 0) v = add_mod(v, bias_delta[(size_t)(j0 + j) * L + l], T.q);
    Y[(size_t)(j0 + j) * ctw + e] = v;
}

}  // namespace

StandardPlan standard_plan(const bfv_ctx *c, const bfv_model *m) {
    StandardPlan p{};
    const size_t ctw = 2 * (size_t)c->L * c->N;
    p.ntiles = ctw / kE;
    const size_t target = (size_t)c->sms * 2 * 6;    // about six waves of two CTAs per SM
    size_t splits = std::max<size_t>(1, (target + p.ntiles - 1) / p.ntiles);
    splits = std::min<size_t>(splits, std::max<size_t>(1, (m->f + 4 * kF - 1) / (4 * kF)));
    p.fper = ((m->f + splits - 1) / splits + kF - 1) / kF * kF;
    p.splits = (m->f + p.fper - 1) / p.fper;
    p.ngroups = (m->nY + kNY - 1) / kNY;
    p.split_bits = (c->bits + 1) / 2;
    p.bytes = p.splits * kNY * ctw * sizeof(longlong2);
    return p;
}

size_t standard_smem_bytes() { return sizeof(StdSmem); }

int launch_standard(const bfv_ctx *c, const bfv_model *m, const u64 *X_ct, u64 *Y_ct, void *ws, const StandardPlan &pl,
                    cudaStream_t st) {
    ProfScope prof_(c, BFV_K_STANDARD, st);
    const size_t ctw = 2 * (size_t)c->L * c->N;
    cudaFuncSetAttribute(k_standard_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(StdSmem));
    longlong2 *partial = (longlong2 *)ws;
    for (size_t gi = 0; gi < pl.ngroups; ++gi) {
        const int j0 = (int)(gi * kNY), nj = (int)std::min<size_t>(kNY, m->nY - j0);
        k_standard_stream<<<(unsigned)(pl.ntiles * pl.splits), kE, sizeof(StdSmem), st>>>(
            m->w16 + gi * m->f * kNY, X_ct, ctw, m->f, pl.fper, pl.split_bits, partial, c->derr,
            (u32)c->inject_extra_tx, c->inject_extra_tx ? (1ll << 12) : kWaitLimit);
        const size_t n = (size_t)nj * ctw;
        k_standard_finalize<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c->dmods, c->N, c->L, ctw, (int)pl.splits, nj, j0,
                                                                         pl.split_bits, partial, m->bias_delta, Y_ct);
        count_launch(c, 2);
    }
    return cudaGetLastError() == cudaSuccess ? BFV_OK : BFV_ERR_CUDA;
}
