// k_packed.cu -- the packed matrix product of Algorithm 1 (Section 4.2.3) with bias.
//
// Pairs g = i*|Y| + j (numbered request by request when several requests, each with its own
// model, share the product) are processed in chunks. Per chunk, in evaluation form:
//   inputs       the chunk's individuals' ciphertexts -> evaluation form
//   MAC          C[g] = sum_k X[i][k] (.) W[j][k]          (Algorithm 1: multiply and add_many)
//   log2 N times C[g] += rot_gal(C[g])                     (Algorithm 1: rotate and accumulate)
//       rot(c) = (sigma(c0) + u0', u1'), (u0', u1') = KS(sigma(c1)):
//       ks_prep     c1 limb l -> sigma -> inverse NTT -> digit d_l (coefficients)
//       ks_modup    for target limb j of QP and part h of the evaluation points:
//                   U_c[j] = sum_i NTT_j(d_i mod q_j) (.) key[i][c][j]; the first one or two
//                   Cooley-Tukey stages are folded into the load, so each CTA transforms
//                   only its part of the points; the two sums live in tensor memory. For
//                   j < L the permuted addend sigma(c0) enters as U_0[j] += P sigma(c0)[j]
//                   (ModDown multiplies by P^-1 and adds to c0, which gives c0 + sigma(c0)
//                   + KS(...)_0 exactly)
//       ks_moddown_p  inverse NTT of U_c[P], r = [U_c[P] + floor(P/2)]_P
//       ks_moddown  C_c[l] += (U_c[l] + NTT_l(floor(P/2) - r)) * P^-1
//   bias+mask    C0 += Delta b_j; C *= NTT(mask_g), mask_g one-hot at slot g mod N (Algorithm 1: mask)
//   compress     Yacc[g / N] += C[g]                       (Algorithm 1: compression)
// and finally Y = inverse NTT(Yacc).
//
// How each key-switching kernel splits a limb over CTAs (the schedule) is a run-time choice
// (bfv_packed_schedule): every schedule computes the same bits.
#include <algorithm>

#include "bfv_internal.h"

namespace {

template <class K> void set_smem(K kern, size_t bytes) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Pair p of a fused product belongs to request r with pair_start[r] <= p < pair_start[r+1];
// g = p - pair_start[r] is the pair index inside its request (i = g / |Y|, j = g mod |Y|).
__device__ __forceinline__ int req_of(const ReqTable &rt, size_t p) {
    int r = 0;
    while (r + 1 < rt.n && rt.pair_start[r + 1] <= p) ++r;
    return r;
}

// ------------------------------------------------------------------ MAC (Algorithm 1: multiply, add_many)
// C[g][c][l][p] = sum_k Xe[i][k][c][l][p] * We[j][k][l][p] with the model of the pair's
// request; grid.x = (g, c, l), grid.y = tile.
__global__ void __launch_bounds__(256) k_mac(const ModTab *__restrict__ mods, int N, int L, size_t g0,
                                             const ReqTable rt, const u64 *__restrict__ Xe, u64 *C) {
    const size_t x = blockIdx.x;
    const int l = (int)(x % L), c = (int)((x / L) % 2);
    const size_t gl = x / (2 * L), gp = g0 + gl;
    const int r = req_of(rt, gp);
    const size_t g = gp - rt.pair_start[r];
    const int K = (int)rt.K[r], nY = (int)rt.nY[r];
    const long long x0 = rt.xoff[r] + (long long)(g / nY) * K;
    const size_t j = g % nY;
    const shoup_t *__restrict__ We = rt.w[r];
    const u64 q = BFV_LD(&mods[l].q), q2 = 2 * q;
    const size_t ctw = 2 * (size_t)L * N;
    const int p0 = blockIdx.y * 1024 + threadIdx.x;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int p = p0 + e * 256;
        if (p >= N) break;
        u64 acc = 0;
        for (int k = 0; k < K; ++k) {
            const u64 xv = BFV_LD(Xe + (size_t)(x0 + k) * ctw + ((size_t)c * L + l) * N + p);
            const shoup_t w = BFV_LDG(We + ((j * K + k) * L + l) * (size_t)N + p);
            acc = red2(acc + mul_shoup(xv, w, q), q2);
        }
        BFV_ST(C + gl * ctw + ((size_t)c * L + l) * N + p, red1(acc, q));
    }
}

// ------------------------------------------------------------------ key switching

// Limb unit (g, l): digit D[g][l] = INTT(sigma(C1[g][l])). MODE 1 splits a limb of N = 16384
// over two 256-thread CTAs (a cluster; the last inverse stage reads the partner's half).
template <int LOGN, int MODE>
LIMB_KERNEL_M(LOGN, MODE) k_ks_prep(const ModTab *__restrict__ mods, int L, u32 gal, const u64 *__restrict__ C,
                                    u64 *D) {
    extern __shared__ u64 sm[];
    LIMB_INDEX_M(LOGN, MODE);
    constexpr int NT = Split<LOGN, MODE>::NT, S = Split<LOGN, MODE>::S;
    const int l = (int)(unit % L);
    const size_t g = unit / L;
    const ModTab T = BFV_LD(mods + l);
    const u64 *limb = C + ((g * 2 + 1) * L + l) * (size_t)N;
    u64 *dst = D + (g * L + l) * (size_t)N;
    // the permuted reads below touch the whole limb in random order: bring it into L2 with
    // coalesced line prefetches first (each CTA of the group a share of the lines)
    for (int i = threadIdx.x + h * NT; i < N / 16; i += S * NT)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(limb + 16 * i));
    limb_inverse<LOGN, MODE>(sm, T, h, [&](int p) { return BFV_LD(limb + auto_src(p, gal, LOGN)); },
                             [&](int p, u64 v) { BFV_ST(dst + p, v); });
}

// ModUp works on parts of H = N / SPLIT evaluation points of a target limb (SPLIT = 2 or 4):
// the first log2 SPLIT Cooley-Tukey stages are done in the load (each CTA reads SPLIT points of
// the digit per output point) and the key-product accumulators live in tensor memory, so that a
// part of up to 16,384 points and its transform fit one CTA (the shared memory holds the
// transform only).
template <int LOGN, int SPLIT> struct ModUpShape {
    static_assert(SPLIT == 2 || SPLIT == 4, "ModUp splits a limb in halves or quarters");
    static constexpr int LOGS = SPLIT == 4 ? 2 : 1;
    static constexpr int LOGH = LOGN - LOGS;
    static constexpr int H = 1 << LOGH;
    // halves: 256 threads where two CTAs fit an SM's shared memory (their barriers then
    // overlap); quarters: 128 threads (four CTAs per SM at N = 16384)
    static constexpr int NT = SPLIT == 2 ? (LOGH == 13 ? 256 : nt_for(LOGH)) : (LOGH >= 13 ? 256 : 128);
    static constexpr int PTS = H / NT;               // points per thread
    static constexpr unsigned COLS = H / 32;         // 4 cells per point over 128 lanes
    static constexpr int PER_SM = 512 / (int)COLS;   // CTAs whose accumulators fit one SM's tensor memory
    // resident CTAs per SM the registers are budgeted for (128 per thread): no more than the
    // tensor memory holds
    static constexpr int MINB = PER_SM < 512 / NT ? PER_SM : 512 / NT;
    static constexpr size_t need = sizeof(u64) * PadSize<H>::value + 16;   // + the TMEM base address
    // shared memory large enough that no more CTAs share an SM than its tensor memory holds
    // (a further CTA would only wait in tcgen05.alloc): 228 KB per SM, 1 KB reserved per CTA
    static constexpr size_t floor_ = (size_t)228 * 1024 / (PER_SM + 1) - 1024 + 16;
    static constexpr size_t smem = need > floor_ ? need : floor_;
    static_assert(PTS % 4 == 0 && COLS >= 32 && COLS <= 512 && (COLS & (COLS - 1)) == 0, "ModUp TMEM layout");
    static_assert(smem <= 227 * 1024, "ModUp shared memory");
};

// Accumulators in tensor memory: thread t of warp w owns the points p = t + e NT (e < PTS) and
// keeps them in lane 32 (w % 4) + t % 32, columns 4 PTS (w / 4) + 4 e + {0, 1, 2, 3} = (acc0 low,
// acc0 high, acc1 low, acc1 high). tacc is the warp's address of its first column.
// acc_c[p] += v(p) * key_c[p] (+ x0(p) for acc0 when EXTRA), four points per TMEM access, key
// loads issued first. The sums are not reduced: L products below 2q each plus an addend below
// 2q stay below 2 (L + 1) q <= 32q < 2^64 (reduced at the end).
template <int H, int NT, bool EXTRA, class Val>
__device__ __forceinline__ void key_mac(u32 tacc, const shoup_t *__restrict__ k0, const shoup_t *__restrict__ k1,
                                        u64 q, Val val) {
    constexpr int PTS = H / NT;
#pragma unroll 1
    for (int e0 = 0; e0 < PTS; e0 += 4) {
        u64 v[4], x0[4];
        shoup_t a[4], b[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int p = threadIdx.x + (e0 + e) * NT;
            a[e] = BFV_LDG(k0 + p);
            b[e] = BFV_LDG(k1 + p);
            val(p, v[e], x0[e]);
        }
        u32 r[16];
        tmem_ld16(tacc + 4u * e0, r);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            u64 s0 = (((u64)r[4 * e + 1] << 32) | r[4 * e]) + mul_shoup(v[e], a[e], q);
            if constexpr (EXTRA) s0 += x0[e];
            const u64 s1 = (((u64)r[4 * e + 3] << 32) | r[4 * e + 2]) + mul_shoup(v[e], b[e], q);
            r[4 * e] = (u32)s0;
            r[4 * e + 1] = (u32)(s0 >> 32);
            r[4 * e + 2] = (u32)s1;
            r[4 * e + 3] = (u32)(s1 >> 32);
        }
        tmem_st16(tacc + 4u * e0, r);
    }
    tmem_wait_st();
}

// grid.x = (g, j, h): U[g][c][j][h H + p] = sum_i NTT_j(D[g][i] mod q_j)[h H + p] * key[i][c][j],
// and for j < L also U[g][0][j] += P sigma(C0[g][j]). The digit of index j itself is
// sigma(C1[g][j]) in evaluation form already (a permuted read, shared with that of C0).
template <int LOGN, int SPLIT>
__global__ void __launch_bounds__(ModUpShape<LOGN, SPLIT>::NT, ModUpShape<LOGN, SPLIT>::MINB)
    k_ks_modup(const ModTab *__restrict__ mods, int L, u32 gal, const u64 *__restrict__ C, const u64 *__restrict__ D,
               const shoup_t *__restrict__ key, u64 *U) {
    extern __shared__ u64 sm[];
    using MS = ModUpShape<LOGN, SPLIT>;
    constexpr int N = 1 << LOGN, H = MS::H, NT = MS::NT, PTS = MS::PTS;
    u32 *tslot = (u32 *)(sm + PadSize<H>::value);
    const int nqp = L + 1;
    const int h = blockIdx.x % SPLIT, j = (blockIdx.x / SPLIT) % nqp;
    const size_t g = blockIdx.x / (SPLIT * nqp);
    const ModTab T = BFV_LD(mods + j);
    const u64 q = T.q;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tmem_alloc(tslot, MS::COLS);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const u32 tbase = *tslot;
    const u32 tacc = tbase + ((u32)(32 * (warp & 3)) << 16) + (u32)(4 * PTS * (warp >> 2));
    {
        u32 z[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) z[k] = 0;
#pragma unroll 1
        for (int e0 = 0; e0 < PTS; e0 += 4) tmem_st16(tacc + 4u * e0, z);
        tmem_wait_st();
    }
    const size_t keystride = (size_t)nqp * N;     // one (digit, component) block
#pragma unroll 1
    for (int i = 0; i < L; ++i) {
        const shoup_t *k0 = key + ((size_t)i * 2 + 0) * keystride + (size_t)j * N + (size_t)h * H;
        const shoup_t *k1 = key + ((size_t)i * 2 + 1) * keystride + (size_t)j * N + (size_t)h * H;
        if (i == j) {
            const u64 *c0 = C + ((g * 2 + 0) * L + j) * (size_t)N;
            const u64 *c1 = C + ((g * 2 + 1) * L + j) * (size_t)N;
            key_mac<H, NT, true>(tacc, k0, k1, q, [&](int p, u64 &v, u64 &x0) {
                const int src = auto_src(h * H + p, gal, LOGN);
                v = BFV_LD(c1 + src);
                x0 = mul_shoup(BFV_LD(c0 + src), T.pmod, T.pmodp, q);
            });
        } else {
            const u64 *d = D + (g * L + i) * (size_t)N;   // digit i < q_i < 2 q_j
            ntt_forward_lazy<MS::LOGH, NT, LOGN == 14 && SPLIT == 2>(   // outputs feed Shoup products only
                sm, T, MS::LOGS, h,
                [&](int p) {
                    u64 v[SPLIT];
#pragma unroll
                    for (int k = 0; k < SPLIT; ++k) v[k] = BFV_LD(d + p + k * H);
                    return fold_stages<MS::LOGS>(T, h, v);
                },
                [&](int p, u64 v) { sm[padi(p)] = v; });
            __syncthreads();
            key_mac<H, NT, false>(tacc, k0, k1, q, [&](int p, u64 &v, u64 &) { v = sm[padi(p)]; });
            __syncthreads();
        }
    }
    u64 *u0 = U + ((g * 2 + 0) * nqp + j) * (size_t)N + (size_t)h * H;
    u64 *u1 = U + ((g * 2 + 1) * nqp + j) * (size_t)N + (size_t)h * H;
#pragma unroll 1
    for (int e0 = 0; e0 < PTS; e0 += 4) {
        u32 r[16];
        tmem_ld16(tacc + 4u * e0, r);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int p = threadIdx.x + (e0 + e) * NT;
            const u64 s0 = ((u64)r[4 * e + 1] << 32) | r[4 * e], s1 = ((u64)r[4 * e + 3] << 32) | r[4 * e + 2];
            BFV_ST(u0 + p, red1(mul_shoup(s0, 1, T.onep, q), q));
            BFV_ST(u1 + p, red1(mul_shoup(s1, 1, T.onep, q), q));
        }
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (warp == 0) tmem_dealloc(tbase, MS::COLS);
}

// Limb unit (g, c): R[g][c] = [INTT_P(U[g][c][P]) + floor(P/2)]_P. MODE 1 (two 256-thread CTAs
// per limb at N = 16384) on small pair chunks.
template <int LOGN, int MODE>
LIMB_KERNEL_M(LOGN, MODE) k_ks_moddown_p(const ModTab *__restrict__ mods, int L, const u64 *__restrict__ U, u64 *R) {
    extern __shared__ u64 sm[];
    LIMB_INDEX_M(LOGN, MODE);
    const int nqp = L + 1;
    const size_t gc = unit;
    const ModTab T = BFV_LD(mods + L);
    const u64 *src = U + (gc * nqp + L) * (size_t)N;
    u64 *dst = R + gc * N;
    limb_inverse<LOGN, MODE>(sm, T, h, [&](int p) { return BFV_LD(src + p); },
                             [&](int p, u64 v) { BFV_ST(dst + p, add_mod(v, T.phalf, T.q)); });
}

// Limb unit (g, c, l): C[g][c][l] += (U[g][c][l] + NTT_l(floor(P/2) - r)) * P^-1. Split modes 1
// and 2: two 256-thread CTAs per limb at N = 16384 (the first stage folded into the loads).
template <int LOGN, int MODE>
LIMB_KERNEL_M(LOGN, MODE) k_ks_moddown(const ModTab *__restrict__ mods, int L, const u64 *__restrict__ U,
                                       const u64 *__restrict__ R, u64 *C) {
    extern __shared__ u64 sm[];
    LIMB_INDEX_M(LOGN, MODE);
    constexpr int NT = Split<LOGN, MODE>::NT;
    const int nqp = L + 1;
    const int l = (int)(unit % L), c = (int)((unit / L) % 2);
    const size_t g = unit / (2 * L);
    const ModTab T = BFV_LD(mods + l);
    const u64 *r = R + (g * 2 + c) * (size_t)N;
    limb_forward<LOGN, true, MODE, MODE == 2>(sm, T, h, [&](int p) { return T.phalf + (T.q - red1(BFV_LD(r + p), T.q)); },
                       [&](int p, u64 v) { sm[padi(p & (M - 1))] = v; });
    __syncthreads();
    const u64 *u = U + ((g * 2 + c) * nqp + l) * (size_t)N + (size_t)h * M;
    u64 *dst = C + ((g * 2 + c) * L + l) * (size_t)N + (size_t)h * M;
    static_assert(M % (4 * NT) == 0, "points per thread must be a multiple of 4");
#pragma unroll 1
    for (int p0 = threadIdx.x; p0 < M; p0 += 4 * NT) {
        u64 a[4], b[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) { a[e] = BFV_LD(u + p0 + e * NT); b[e] = BFV_LD(dst + p0 + e * NT); }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int p = p0 + e * NT;
            const u64 v = red1(mul_shoup(a[e] + sm[padi(p)], T.pinv, T.pinvp, T.q), T.q);
            BFV_ST(dst + p, add_mod(b[e], v, T.q));
        }
    }
}

// ------------------------------------------------------------------ bias + mask (Algorithm 1: mask)
// The one-hot plaintext at slot s has coefficient k = N^-1 omega^(-e k) mod t, e = e_s the
// exponent of the slot's evaluation point (3^(s mod N/2) mod 2N, negated for s >= N/2). Since
// omega^N = -1 it is the automorphism X -> X^f of the slot-0 mask (e = 1), f = e_s^-1 mod 2N, and
// in evaluation form an automorphism is a permutation of positions: mask_s[p] = mask_0[auto_src(p,
// f)]. The context keeps mask_0 per limb; a product's masks are gathered from it.

// Limb unit l: maskev[l] = NTT_l(centred lift of the slot-0 mask) in Shoup form.
template <int LOGN>
LIMB_KERNEL(LOGN) k_mask_base(const ModTab *__restrict__ mods, int tmod, const u32 *__restrict__ maskpow,
                              shoup_t *maskev) {
    extern __shared__ u64 sm[];
    LIMB_INDEX(LOGN);
    const int l = (int)unit;
    const ModTab T = BFV_LD(mods + l);
    const u64 t = BFV_LD(&mods[tmod].q), th = (t - 1) / 2;
    const u32 twoN = 2u * N;
    limb_forward<LOGN>(
        sm, T, h,
        [&](int p) {
            const u64 v = BFV_LD(maskpow + ((twoN - (u32)p) & (twoN - 1)));
            return v <= th ? v : T.q - (t - v);
        },
        [&](int p, u64 v) { BFV_ST(maskev + (size_t)l * N + p, make_shoup(v, T.q)); });
}

// grid.x = (g, l, part of kBmPts x 256 points): C[g][0][l] = (C[g][0][l] + Delta [b_j]_t) mask_s and
// C[g][1][l] *= mask_s for the pair's slot s = (g0 + g) mod N.
constexpr int kBmThreads = 256, kBmPts = 8;
template <int LOGN>
__global__ void __launch_bounds__(kBmThreads) k_bias_mask(const ModTab *__restrict__ mods, int L, size_t g0,
                                                          const ReqTable rt, const shoup_t *__restrict__ maskev,
                                                          u64 *C) {
    constexpr int N = 1 << LOGN, PART = kBmThreads * kBmPts, NPART = N / PART;
    const size_t x = blockIdx.x;
    const int part = (int)(x % NPART), l = (int)((x / NPART) % L);
    const size_t gl = x / ((size_t)NPART * L), gp = g0 + gl;
    const int r = req_of(rt, gp);
    const size_t g = gp - rt.pair_start[r];
    const int j = (int)(g % rt.nY[r]), s = (int)(g % N);
    const u64 q = BFV_LD(&mods[l].q);
    // f = e_s^-1 mod 2N: 3 has order N/2 mod 2N, so 3^-y = 3^(N/2 - y); negated with e_s
    const u32 twoN = 2u * N;
    u32 f = 1, base = 3;
    for (u32 y = (u32)((N / 2 - s % (N / 2)) % (N / 2)); y; y >>= 1) {
        if (y & 1) f = (f * base) & (twoN - 1);
        base = (base * base) & (twoN - 1);
    }
    if (s >= N / 2) f = twoN - f;
    const u64 bd = BFV_LD(rt.bias[r] + (size_t)j * L + l);
    const shoup_t *mk = maskev + (size_t)l * N;
    u64 *c0 = C + ((gl * 2 + 0) * L + l) * (size_t)N, *c1 = C + ((gl * 2 + 1) * L + l) * (size_t)N;
    u64 a[kBmPts], b[kBmPts];
    shoup_t m[kBmPts];
#pragma unroll
    for (int e = 0; e < kBmPts; ++e) {
        const int p = part * PART + e * kBmThreads + threadIdx.x;
        m[e] = BFV_LDG(mk + auto_src(p, f, LOGN));
        a[e] = BFV_LD(c0 + p);
        b[e] = BFV_LD(c1 + p);
    }
#pragma unroll
    for (int e = 0; e < kBmPts; ++e) {
        const int p = part * PART + e * kBmThreads + threadIdx.x;
        BFV_ST(c0 + p, red1(mul_shoup(add_mod(a[e], bd, q), m[e], q), q));
        BFV_ST(c1 + p, red1(mul_shoup(b[e], m[e], q), q));
    }
}

// ------------------------------------------------------------------ compression (Algorithm 1: compression)
// Yacc[e] += sum_{g in [ga, gb)} C[g - g0][e] for every element e of one output ciphertext.
__global__ void __launch_bounds__(256) k_compress(const ModTab *__restrict__ mods, int N, int L, size_t ga, size_t gb,
                                                  size_t g0, const u64 *__restrict__ C, u64 *Yacc) {
    const size_t ctw = 2 * (size_t)L * N;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ctw) return;
    const u64 q = BFV_LD(&mods[(e / N) % L].q);
    u64 acc = BFV_LD(Yacc + e);
    size_t g = ga;
    for (; g + 4 <= gb; g += 4) {
        const u64 a = BFV_LD(C + (g - g0) * ctw + e), b = BFV_LD(C + (g + 1 - g0) * ctw + e);
        const u64 c = BFV_LD(C + (g + 2 - g0) * ctw + e), d = BFV_LD(C + (g + 3 - g0) * ctw + e);
        acc = red1(acc + red1(a + b, q), q);
        acc = red1(acc + red1(c + d, q), q);
    }
    for (; g < gb; ++g) acc = red1(acc + BFV_LD(C + (g - g0) * ctw + e), q);
    BFV_ST(Yacc + e, acc);
}

// Pair state (evaluation form) -> coefficient form; limb unit x uses modulus x % L.
template <int LOGN>
LIMB_KERNEL(LOGN) k_intt_copy(const ModTab *__restrict__ mods, int L, const u64 *__restrict__ in, u64 *out) {
    extern __shared__ u64 sm[];
    LIMB_INDEX(LOGN);
    const size_t x = unit;
    const ModTab T = BFV_LD(mods + x % L);
    limb_inverse<LOGN>(sm, T, h, [&](int p) { return BFV_LD(in + x * N + p); },
                       [&](int p, u64 v) { BFV_ST(out + x * N + p, v); });
}

int last_err() { return cudaGetLastError() == cudaSuccess ? BFV_OK : BFV_ERR_CUDA; }

// One ModUp launch over ng pairs with limbs split in SPLIT parts.
template <int LOGN, int SPLIT>
void launch_modup(const bfv_ctx *c, size_t ng, u32 gal, const u64 *C, const u64 *D, const shoup_t *key, u64 *U,
                  cudaStream_t st) {
    using MS = ModUpShape<LOGN, SPLIT>;
    set_smem(k_ks_modup<LOGN, SPLIT>, MS::smem);
    k_ks_modup<LOGN, SPLIT><<<(unsigned)(ng * c->nqp * SPLIT), MS::NT, MS::smem, st>>>(c->dmods, c->L, gal, C, D, key, U);
}

// The four kernels of one key switch (rotation by gal) for the ng pairs of a chunk, each split
// as the schedule says. Splits of two CTAs per limb exist at N = 16384 only (at N = 32768 every
// limb already runs on a two-CTA cluster, smaller rings use one CTA per limb).
template <int LOGN>
void ks_step(const bfv_ctx *c, const bfv_packed_schedule &sc, size_t ng, u32 gal, const shoup_t *key, u64 *C, u64 *D,
             u64 *U, u64 *R, cudaStream_t st) {
    const int L = c->L;
    constexpr bool PAIRS = LOGN == 14;
    {
        ProfScope pr(c, BFV_K_KS_PREP, st);
        if constexpr (PAIRS) {
            if (sc.prep_split == 2) launch_limbs<LOGN, 1>(k_ks_prep<LOGN, 1>, ng * L, st, 0, c->dmods, L, gal, (const u64 *)C, D);
            else if (sc.prep_split == 3) launch_limbs<LOGN, 2>(k_ks_prep<LOGN, 2>, ng * L, st, 0, c->dmods, L, gal, (const u64 *)C, D);
            else launch_limbs<LOGN, 0>(k_ks_prep<LOGN, 0>, ng * L, st, 0, c->dmods, L, gal, (const u64 *)C, D);
        } else {
            launch_limbs<LOGN, 0>(k_ks_prep<LOGN, 0>, ng * L, st, 0, c->dmods, L, gal, (const u64 *)C, D);
        }
    }
    {
        ProfScope pr(c, BFV_K_KS_MODUP, st);
        if (sc.modup_split == 4) launch_modup<LOGN, 4>(c, ng, gal, C, D, key, U, st);
        else launch_modup<LOGN, 2>(c, ng, gal, C, D, key, U, st);
    }
    {
        // two limbs per pair leave most SMs idle on small chunks: by default split each over two
        // CTAs there (measured: 41 -> 33 us per launch at 16 pairs; slower on full chunks)
        ProfScope pr(c, BFV_K_KS_MODDOWN_P, st);
        const bool two = sc.moddown_p_split == 2 || (sc.moddown_p_split == 0 && ng * 2 < (size_t)2 * c->sms);
        if constexpr (PAIRS) {
            if (sc.moddown_p_split == 3)
                launch_limbs<LOGN, 3>(k_ks_moddown_p<LOGN, 3>, ng * 2, st, 0, c->dmods, L, (const u64 *)U, R);
            else if (sc.moddown_p_split == 4)
                launch_limbs<LOGN, 2>(k_ks_moddown_p<LOGN, 2>, ng * 2, st, 0, c->dmods, L, (const u64 *)U, R);
            else if (two) launch_limbs<LOGN, 1>(k_ks_moddown_p<LOGN, 1>, ng * 2, st, 0, c->dmods, L, (const u64 *)U, R);
            else launch_limbs<LOGN, 0>(k_ks_moddown_p<LOGN, 0>, ng * 2, st, 0, c->dmods, L, (const u64 *)U, R);
        } else {
            (void)two;
            launch_limbs<LOGN, 0>(k_ks_moddown_p<LOGN, 0>, ng * 2, st, 0, c->dmods, L, (const u64 *)U, R);
        }
    }
    {
        ProfScope pr(c, BFV_K_KS_MODDOWN, st);
        if constexpr (PAIRS) {
            if (sc.moddown_split == 1)
                launch_limbs<LOGN, 0>(k_ks_moddown<LOGN, 0>, ng * 2 * L, st, 0, c->dmods, L, (const u64 *)U, (const u64 *)R, C);
            else if (sc.moddown_split == 3)
                launch_limbs<LOGN, 2>(k_ks_moddown<LOGN, 2>, ng * 2 * L, st, 0, c->dmods, L, (const u64 *)U, (const u64 *)R, C);
            else launch_limbs<LOGN, 1>(k_ks_moddown<LOGN, 1>, ng * 2 * L, st, 0, c->dmods, L, (const u64 *)U, (const u64 *)R, C);
        } else {
            launch_limbs<LOGN, 0>(k_ks_moddown<LOGN, 0>, ng * 2 * L, st, 0, c->dmods, L, (const u64 *)U, (const u64 *)R, C);
        }
    }
    count_launch(c, 4);
}

template <int LOGN>
int run_packed(const bfv_ctx *c, const bfv_keys *k, int nreq, const u64 *const *X_ct, u64 *const *Y_ct, char *ws,
               const PackedPlan &pl, cudaStream_t st) {
    constexpr int N = 1 << LOGN;
    const int L = c->L, nqp = c->nqp;
    const size_t ctw = 2 * (size_t)L * N;
    u64 *Xe = (u64 *)(ws + pl.off_xntt), *Yacc = (u64 *)(ws + pl.off_yacc), *C = (u64 *)(ws + pl.off_state);
    u64 *D = (u64 *)(ws + pl.off_digits), *U = (u64 *)(ws + pl.off_u), *R = (u64 *)(ws + pl.off_r);

    int rc;
    if (cudaMemsetAsync(Yacc, 0, pl.nout * ctw * sizeof(u64), st) != cudaSuccess) return BFV_ERR_CUDA;
    const size_t keyblock = (size_t)L * 2 * nqp * N;   // one Galois element
    ReqTable rt = pl.rt;
    for (size_t g0 = 0; g0 < pl.npairs; g0 += pl.chunk) {
        const size_t ng = std::min(pl.chunk, pl.npairs - g0);
        // evaluation form of the inputs of the individuals this chunk's pairs use
        size_t off = 0;
        for (int r = 0; r < nreq; ++r) {
            size_t ia, ib;
            chunk_window(pl, r, g0, ng, ia, ib);
            if (ia == ib) continue;
            const size_t K = rt.K[r];
            if ((rc = launch_ntt_limbs(c, X_ct[r] + ia * K * ctw, Xe + off * ctw, (ib - ia) * K, true, st))) return rc;
            rt.xoff[r] = (long long)off - (long long)(ia * K);
            off += (ib - ia) * K;
        }
        { ProfScope pr(c, BFV_K_MAC, st);
        k_mac<<<dim3((unsigned)(ng * 2 * L), (unsigned)((N + 1023) / 1024)), 256, 0, st>>>(c->dmods, N, L, g0, rt, Xe, C); }
        count_launch(c);
        for (int s = 0; s < k->ng; ++s)
            ks_step<LOGN>(c, pl.sched, ng, (u32)c->galois[s], k->gk_eval + (size_t)s * keyblock, C, D, U, R, st);
        { ProfScope pr(c, BFV_K_BIAS_MASK, st);
        k_bias_mask<LOGN><<<(unsigned)(ng * L * (N / (kBmThreads * kBmPts))), kBmThreads, 0, st>>>(c->dmods, L, g0, rt,
                                                                                                c->dmaskev, C); }
        count_launch(c);
        // compression: the pairs of request r that land in its output o are one contiguous range
        for (int r = 0; r < nreq; ++r) {
            const size_t pa = pl.rt.pair_start[r], pb = pl.rt.pair_start[r + 1];
            if (pb <= g0 || pa >= g0 + ng) continue;
            for (size_t o = 0; pa + o * N < pb; ++o) {
                const size_t ga = std::max(g0, pa + o * N), gb = std::min({g0 + ng, pa + (o + 1) * N, pb});
                if (ga >= gb) continue;
                ProfScope pr(c, BFV_K_COMPRESS, st);
                k_compress<<<(unsigned)((ctw + 255) / 256), 256, 0, st>>>(c->dmods, N, L, ga, gb, g0, C,
                                                                          Yacc + (pl.ycts[r] + o) * ctw);
                count_launch(c);
            }
        }
        if ((rc = last_err())) return rc;
    }
    for (int r = 0; r < nreq; ++r)
        if ((rc = launch_ntt_limbs(c, Yacc + pl.ycts[r] * ctw, Y_ct[r], pl.nouts[r], false, st))) return rc;
    return BFV_OK;
}

}  // namespace

#ifdef BFV_BOUNDS
BFV_BOUNDS_UPLOAD_FN(bounds_upload_packed)
#endif

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

bfv_packed_schedule default_schedule() {
    bfv_packed_schedule s{};
    s.pair_chunk = 2048;
    s.prep_split = 1;
    s.modup_split = 2;
    s.moddown_p_split = 0;
    s.moddown_split = 2;
    return s;
}

bool schedule_ok(const bfv_packed_schedule &s) {
    return s.pair_chunk >= 1 && s.prep_split >= 1 && s.prep_split <= 3 &&
           (s.modup_split == 2 || s.modup_split == 4) && s.moddown_p_split <= 4 &&
           s.moddown_split >= 1 && s.moddown_split <= 3;
}

bfv_packed_schedule schedule_for(const bfv_ctx *c, size_t npairs, size_t chunk) {
    bfv_packed_schedule s = default_schedule();
    {
        std::lock_guard<std::mutex> g(c->tune_mu);
        auto it = c->tuned.find(npairs);
        if (it == c->tuned.end()) it = c->tuned.find(0);
        if (it != c->tuned.end()) s = it->second;
    }
    if (chunk) s.pair_chunk = chunk;
    return s;
}

PackedPlan packed_plan_models(const bfv_ctx *c, int nreq, const bfv_model *const *models, const size_t *nXs,
                              size_t chunk, const bfv_packed_schedule *sched) {
    PackedPlan p{};
    const size_t N = c->N, L = c->L, nqp = c->nqp;
    p.nreq = nreq;
    p.nY = models[0]->nY;
    p.K = models[0]->K;
    p.rt.n = nreq;
    size_t pairs = 0, outs = 0;
    for (int r = 0; r < nreq; ++r) {
        const bfv_model *m = models[r];
        p.nXs[r] = nXs[r];
        p.rt.pair_start[r] = pairs;
        p.rt.K[r] = (u32)m->K;
        p.rt.nY[r] = (u32)m->nY;
        p.rt.w[r] = m->w_eval;
        p.rt.bias[r] = m->bias_delta;
        p.ycts[r] = outs;
        const size_t np = nXs[r] * m->nY;
        p.nouts[r] = (np + N - 1) / N;
        pairs += np;
        outs += p.nouts[r];
    }
    p.rt.pair_start[nreq] = pairs;
    p.nX = nreq == 1 ? nXs[0] : 0;
    p.npairs = pairs;
    p.nout = outs;
    p.sched = sched ? *sched : schedule_for(c, p.npairs, chunk);
    p.chunk = std::max<size_t>(1, std::min<size_t>(p.sched.pair_chunk, p.npairs));
    p.sched.pair_chunk = p.chunk;
    for (size_t g0 = 0; g0 < p.npairs; g0 += p.chunk) {
        size_t cts = 0;
        for (int r = 0; r < nreq; ++r) {
            size_t ia, ib;
            chunk_window(p, r, g0, std::min(p.chunk, p.npairs - g0), ia, ib);
            cts += (ib - ia) * p.rt.K[r];
        }
        p.xcts_chunk = std::max(p.xcts_chunk, cts);
    }
    const size_t ctb = 2 * L * N * sizeof(u64);
    size_t off = 0;
    p.off_xntt = off; off += al256(p.xcts_chunk * ctb);
    p.off_yacc = off; off += al256(p.nout * ctb);
    p.off_state = off; off += al256(p.chunk * ctb);
    p.off_digits = off; off += al256(p.chunk * L * N * sizeof(u64));
    p.off_u = off; off += al256(p.chunk * 2 * nqp * N * sizeof(u64));
    p.off_r = off; off += al256(p.chunk * 2 * N * sizeof(u64));
    p.total = off;
    return p;
}

PackedPlan packed_plan_multi(const bfv_ctx *c, const bfv_model *m, int nreq, const size_t *nXs, size_t chunk,
                             const bfv_packed_schedule *sched) {
    const bfv_model *ms[kMaxReq];
    for (int r = 0; r < nreq; ++r) ms[r] = m;
    return packed_plan_models(c, nreq, ms, nXs, chunk, sched);
}

PackedPlan packed_plan(const bfv_ctx *c, const bfv_model *m, size_t nX, size_t chunk, const bfv_packed_schedule *sched) {
    return packed_plan_multi(c, m, 1, &nX, chunk, sched);
}

int launch_packed_multi(const bfv_ctx *c, const bfv_keys *k, int nreq, const u64 *const *X_ct, u64 *const *Y_ct,
                        void *ws, const PackedPlan &plan, cudaStream_t st) {
    switch (c->logN) {
        case 12: return run_packed<12>(c, k, nreq, X_ct, Y_ct, (char *)ws, plan, st);
        case 13: return run_packed<13>(c, k, nreq, X_ct, Y_ct, (char *)ws, plan, st);
        case 14: return run_packed<14>(c, k, nreq, X_ct, Y_ct, (char *)ws, plan, st);
        case 15: return run_packed<15>(c, k, nreq, X_ct, Y_ct, (char *)ws, plan, st);
        default: return BFV_ERR_BAD_PARAMS;
    }
}

int launch_packed(const bfv_ctx *c, const bfv_keys *k, const u64 *X_ct, u64 *Y_ct, void *ws, const PackedPlan &plan,
                  cudaStream_t st) {
    return launch_packed_multi(c, k, 1, &X_ct, &Y_ct, ws, plan, st);
}

int launch_mask_base(const bfv_ctx *c, cudaStream_t st) {
#define L_(LG) launch_limbs<LG>(k_mask_base<LG>, (size_t)c->L, st, 0, c->dmods, c->nqp, (const u32 *)c->dmaskpow, c->dmaskev)
    switch (c->logN) {
        case 12: L_(12); break;
        case 13: L_(13); break;
        case 14: L_(14); break;
        case 15: L_(15); break;
        default: return BFV_ERR_BAD_PARAMS;
    }
#undef L_
    return last_err();
}

int launch_pair_export(const bfv_ctx *c, const PackedPlan &plan, const void *ws, size_t slot, u64 *ct_out,
                       cudaStream_t st) {
    const size_t ctw = 2 * (size_t)c->L * c->N;
    const u64 *C = (const u64 *)((const char *)ws + plan.off_state) + slot * ctw;
#define L_(LG) launch_limbs<LG>(k_intt_copy<LG>, 2 * c->L, st, 0, c->dmods, c->L, C, ct_out)
    switch (c->logN) {
        case 12: L_(12); break;
        case 13: L_(13); break;
        case 14: L_(14); break;
        case 15: L_(15); break;
        default: return BFV_ERR_BAD_PARAMS;
    }
#undef L_
    count_launch(c);
    return last_err();
}
