// k_standard.cu -- the "standard" per-element encrypted matrix product (Section 5.2.3):
// Y_j = sum_f w[f][j] X_f + Delta [b_j]_t, with X_f holding feature f of individual i in
// slot i. Scalar-times-ciphertext is coefficient-wise, so the kernel works directly on the
// coefficient form: one pass over all f ciphertexts (the HBM stream), |Y| accumulators per
// coefficient. Each 55-bit coefficient is split into two 27/28-bit halves so that
// w * half fits a 32x32 -> 64 signed multiply-add; the two signed 64-bit accumulators
// are reduced mod q once at the end (|w| f < 2^35 keeps them exact).
#include "bfv_internal.h"

namespace {

constexpr int kTF = 128;   // features per shared-memory weight tile

template <int NY>
__global__ void __launch_bounds__(256) k_standard(const ModTab *__restrict__ mods, int N, int L, size_t F, int nY,
                                                  int j0, const int64_t *__restrict__ W,
                                                  const u64 *__restrict__ bias_delta, const u64 *__restrict__ X,
                                                  u64 *Y) {
    __shared__ int wt[kTF][NY];
    const size_t ctw = 2 * (size_t)L * N;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    long long lo[NY], hi[NY];
#pragma unroll
    for (int j = 0; j < NY; ++j) { lo[j] = 0; hi[j] = 0; }
    const bool live = e < ctw;
    for (size_t f0 = 0; f0 < F; f0 += kTF) {
        const int nf = (int)((F - f0) < (size_t)kTF ? (F - f0) : (size_t)kTF);
        __syncthreads();
        for (int x = threadIdx.x; x < kTF * NY; x += blockDim.x) {
            const int ff = x / NY, j = x % NY;
            wt[ff][j] = (ff < nf && j0 + j < nY) ? (int)W[(f0 + ff) * nY + j0 + j] : 0;
        }
        __syncthreads();
        if (!live) continue;
        const u64 *xp = X + f0 * ctw + e;
        int ff = 0;
        for (; ff + 4 <= nf; ff += 4) {
            u64 xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = __ldcs(xp + (size_t)(ff + u) * ctw);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int xl = (int)(xv[u] & 0x7FFFFFFull), xh = (int)(xv[u] >> 27);
#pragma unroll
                for (int j = 0; j < NY; ++j) {
                    const int w = wt[ff + u][j];
                    lo[j] += (long long)w * xl;
                    hi[j] += (long long)w * xh;
                }
            }
        }
        for (; ff < nf; ++ff) {
            const u64 xv = __ldcs(xp + (size_t)ff * ctw);
            const int xl = (int)(xv & 0x7FFFFFFull), xh = (int)(xv >> 27);
#pragma unroll
            for (int j = 0; j < NY; ++j) {
                const int w = wt[ff][j];
                lo[j] += (long long)w * xl;
                hi[j] += (long long)w * xh;
            }
        }
    }
    if (!live) return;
    const int l = (int)((e / N) % L);
    const bool c0k0 = (e / N) < (size_t)L && (e % N) == 0;
    const ModTab T = mods[l];
    const long long q = (long long)T.q;
    const u64 s27 = (1ull << 27) % T.q;
#pragma unroll
    for (int j = 0; j < NY; ++j) {
        if (j0 + j >= nY) break;
        long long h = hi[j] % q; if (h < 0) h += q;
        long long a = lo[j] % q; if (a < 0) a += q;
        u64 v = add_mod(mul_barrett((u64)h, s27, T.q, T.mu, T.bits), (u64)a, T.q);
        if (c0k0) v = add_mod(v, bias_delta[(size_t)(j0 + j) * L + l], T.q);
        Y[(size_t)(j0 + j) * ctw + e] = v;
    }
}

}  // namespace

int launch_standard(const bfv_ctx *c, const bfv_model *m, const u64 *X_ct, u64 *Y_ct, cudaStream_t st) {
    ProfScope prof_(c, BFV_K_STANDARD, st);
    const size_t ctw = 2 * (size_t)c->L * c->N;
    const unsigned blocks = (unsigned)((ctw + 255) / 256);
    for (int j0 = 0; j0 < (int)m->nY; j0 += 16) {
        const int left = (int)m->nY - j0;
        if (left > 8)
            k_standard<16><<<blocks, 256, 0, st>>>(c->dmods, c->N, c->L, m->f, (int)m->nY, j0, m->w_int, m->bias_delta, X_ct, Y_ct);
        else if (left > 4)
            k_standard<8><<<blocks, 256, 0, st>>>(c->dmods, c->N, c->L, m->f, (int)m->nY, j0, m->w_int, m->bias_delta, X_ct, Y_ct);
        else if (left > 2)
            k_standard<4><<<blocks, 256, 0, st>>>(c->dmods, c->N, c->L, m->f, (int)m->nY, j0, m->w_int, m->bias_delta, X_ct, Y_ct);
        else
            k_standard<2><<<blocks, 256, 0, st>>>(c->dmods, c->N, c->L, m->f, (int)m->nY, j0, m->w_int, m->bias_delta, X_ct, Y_ct);
        count_launch(c);
        if (left > 16) continue;
        break;
    }
    return cudaGetLastError() == cudaSuccess ? BFV_OK : BFV_ERR_CUDA;
}
