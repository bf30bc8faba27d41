// bfv_device.cuh -- device-side modular arithmetic and the shared-memory negacyclic NTT.
//
// Residues are 64-bit words modulo primes below 2^59. Constant operands (twiddles, keys,
// encoded weights, P^-1) are multiplied with Shoup's method (a precomputed companion
// w' = floor(w 2^64 / q) turns the reduction into one high and two low 64-bit products);
// variable x variable products use Barrett reduction with mu = floor(2^(2b) / q).
// Both transforms use Cooley-Tukey butterflies with Harvey's lazy bounds (values in [0, 4q), or
// unreduced where only Shoup products consume them).
//
// NTT layout: forward transform of a (coefficient order) leaves at position p the value
// a(psi^(2 brev(p) + 1)) (bit-reversed evaluation order). The inverse transform takes that
// layout back to coefficients: a decimation-in-time cyclic transform with omega^-1 = psi^-2 on
// the bit-reversed input gives b_k = sum_m B_m omega^(-m k) in natural order, and a post-twist by
// N^-1 psi^-k gives a_k. Every evaluation-form array in the library (keys, encoded weights,
// ciphertexts in flight) uses this layout.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

typedef unsigned long long u64;
typedef unsigned int u32;

#define BFV_MAXP 16      // ciphertext primes + special prime
#define BFV_MAXMOD 17    // + the plaintext modulus t (index nqp)
#define BFV_MAXW 16      // 64-bit words of Q (and of t*Q) for exact decryption

// Per-modulus constants, resident in device memory (one entry per prime and one for t).
struct ModTab {
    u64 q, q2;              // q and 2q
    u64 ninv, ninvp;        // N^-1 mod q and its Shoup companion
    u64 mu;                 // Barrett constant floor(2^(2 bits) / q)
    int bits;               // bit length of q
    int pad_;
    u64 pinv, pinvp;        // P^-1 mod q and companion (ciphertext primes only)
    u64 pmod, pmodp;        // P mod q and companion (ciphertext primes only)
    u64 phalf;              // floor(P/2) mod q
    u64 delta, deltap;      // floor(Q/t) mod q and companion
    u64 r64, r64p;          // 2^64 mod q and companion
    u64 onep;               // floor(2^64 / q): Shoup companion of 1 (reduces any 64-bit word to [0, 2q))
    const ulonglong2 *fw;   // forward twiddles {psi^brev(k), Shoup companion}, k < N
    const ulonglong2 *dt;   // inverse twiddles: dt[h + j] = {omega^-(j N / 2h), companion}, h = 2^s, j < h
    const ulonglong2 *tw;   // inverse post-twist {N^-1 psi^-k, companion}, k < N
};

// ------------------------------------------------------------------ bounds-checked debug build
//
// Built with -DBFV_BOUNDS, every global-memory access of the library's kernels goes through
// BFV_LD / BFV_ST / BFV_LDG (and every bulk copy through BFV_RANGE_OK): the address range must
// lie inside one of the buffers the current call may touch (the context's tables, the keys, the
// models, the caller's inputs, outputs and workspace at the sizes the call implies). An access
// outside them is skipped (a load yields 0) and sets bit 1 (value 2) of the context's error word,
// so a wrong index shows up as an error code instead of a fault. The table is per translation
// unit and per process, uploaded in stream order before each call's launches (calls of a
// bounds-checked build must not overlap). The release build compiles the macros to plain accesses.
#ifdef BFV_BOUNDS
#define BFV_MAX_RANGES 512
struct BoundsTable {
    int n;
    int pad_;
    int *err;
    unsigned long long lo[BFV_MAX_RANGES], hi[BFV_MAX_RANGES];
};
static __device__ BoundsTable g_bounds;
__device__ __forceinline__ bool bfv_in_bounds(const void *p, unsigned long long bytes) {
    const unsigned long long a = (unsigned long long)p;
    const int n = g_bounds.n;
    for (int i = 0; i < n; ++i)
        if (a >= g_bounds.lo[i] && a + bytes <= g_bounds.hi[i]) return true;
    if (g_bounds.err) atomicOr(g_bounds.err, 2);
    return false;
}
template <class T> __device__ __forceinline__ T bfv_ld(const T *p) { return bfv_in_bounds(p, sizeof(T)) ? *p : T{}; }
template <class T> __device__ __forceinline__ T bfv_ldg(const T *p) { return bfv_in_bounds(p, sizeof(T)) ? __ldg(p) : T{}; }
template <class T> __device__ __forceinline__ T bfv_ldcs(const T *p) { return bfv_in_bounds(p, sizeof(T)) ? __ldcs(p) : T{}; }
template <class T, class V> __device__ __forceinline__ void bfv_st(T *p, V v) {
    if (bfv_in_bounds(p, sizeof(T))) *p = v;
}
#define BFV_LD(p) bfv_ld(p)
#define BFV_LDG(p) bfv_ldg(p)
#define BFV_LDCS(p) bfv_ldcs(p)
#define BFV_ST(p, v) bfv_st((p), (v))
#define BFV_RANGE_OK(p, bytes) bfv_in_bounds((p), (bytes))
// Host side: each translation unit with kernels uploads the table to its own copy.
#define BFV_BOUNDS_UPLOAD_FN(name)                                                          \
    cudaError_t name(const BoundsTable &t, cudaStream_t st) {                              \
        return cudaMemcpyToSymbolAsync(g_bounds, &t, sizeof t, 0, cudaMemcpyHostToDevice, st); \
    }
#else
#define BFV_LD(p) (*(p))
#define BFV_LDG(p) __ldg(p)
#define BFV_LDCS(p) __ldcs(p)
#define BFV_ST(p, v) (*(p) = (v))
#define BFV_RANGE_OK(p, bytes) true
#endif

// ------------------------------------------------------------------ modular arithmetic

__device__ __forceinline__ u64 mul_shoup(u64 x, u64 w, u64 wp, u64 q) {
    // x < 2^64, w < q, wp = floor(w 2^64 / q): result in [0, 2q)
    const u64 h = __umul64hi(x, wp);
    return x * w - h * q;
}
__device__ __forceinline__ u64 red2(u64 x, u64 q2) { return x >= q2 ? x - q2 : x; }
__device__ __forceinline__ u64 red1(u64 x, u64 q) { return x >= q ? x - q : x; }
__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) { return red1(a + b, q); }
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// a * b mod q for a, b < q (Barrett, q < 2^61, mu = floor(2^(2 bits) / q)).
__device__ __forceinline__ u64 mul_barrett(u64 a, u64 b, u64 q, u64 mu, int bits) {
    const u64 lo = a * b, hi = __umul64hi(a, b);
    // z >> (bits - 1), z = hi:lo < 2^(2 bits)
    const int s = bits - 1;
    const u64 z1 = (lo >> s) | (hi << (64 - s));
    // q_est = floor(z1 * mu / 2^(bits + 1)); z1 < 2^(bits+1), mu < 2^(bits+1)
    const u64 plo = z1 * mu, phi = __umul64hi(z1, mu);
    const int s2 = bits + 1;
    const u64 qe = (plo >> s2) | (phi << (64 - s2));
    u64 r = lo - qe * q;
    r = red1(r, q);
    r = red1(r, q);
    return red1(r, q);
}

// Shoup companion floor(w 2^64 / q) by long division (setup-time helper on the device).
__device__ __forceinline__ u64 shoup_companion(u64 w, u64 q) {
    u64 rem = w, quo = 0;
#pragma unroll 1
    for (int i = 0; i < 64; ++i) {
        rem <<= 1;
        quo <<= 1;
        if (rem >= q) { rem -= q; quo |= 1; }
    }
    return quo;
}

// ------------------------------------------------------------------ butterflies

__device__ __forceinline__ void ct_bfly(u64 &X, u64 &Y, u64 w, u64 wp, u64 q, u64 q2) {
    const u64 x = red2(X, q2);
    const u64 t = mul_shoup(Y, w, wp, q);
    X = x + t;
    Y = x - t + q2;
}
// Without the reduction of X: both outputs exceed the inputs' bound by less than 2q (t < 2q).
// The lazy forward runs at most 14 such stages after an entry below 4q (at N = 32768 the first
// stage is the reducing fold), the inverse at most 15 after an entry below 2q: both stay below
// 32q < 2^64 for the primes below 2^59 the library accepts. The outputs then meet only Shoup
// products (which take any 64-bit input) or the inverse's post-twist.
__device__ __forceinline__ void ct_bfly_lazy(u64 &X, u64 &Y, u64 w, u64 wp, u64 q, u64 q2) {
    const u64 t = mul_shoup(Y, w, wp, q);
    const u64 x = X;
    X = x + t;
    Y = x - t + q2;
}

// Shared-memory index with one pad word every 16 words (conflict-free strided groups).
__device__ __forceinline__ int padi(int p) { return p + (p >> 4); }
template <int M> struct PadSize { static constexpr int value = M + (M >> 4); };

// ------------------------------------------------------------------ radix-2^R register kernels

// Forward Cooley-Tukey stages s .. s+R-1 (global stage numbers) on a group of 2^R values
// x[r] = a[base + r * t_last]; gblock is the global block index at stage s.
template <int R, bool LAZY = false>
__device__ __forceinline__ void fwd_radix(u64 (&x)[1 << R], int s, int gblock, const ulonglong2 *__restrict__ fw,
                                          u64 q, u64 q2) {
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int half = 1 << (R - 1 - u);
#pragma unroll
        for (int k = 0; k < (1 << u); ++k) {
            const int ti = (1 << (s + u)) + (gblock << u) + k;
            const ulonglong2 w = BFV_LDG(fw + ti);
#pragma unroll
            for (int j = 0; j < half; ++j) {
                if constexpr (LAZY) ct_bfly_lazy(x[k * 2 * half + j], x[k * 2 * half + j + half], w.x, w.y, q, q2);
                else ct_bfly(x[k * 2 * half + j], x[k * 2 * half + j + half], w.x, w.y, q, q2);
            }
        }
    }
}

// Inverse (decimation-in-time) stages S .. S+R-1 on a group of 2^R values x[r] = a[base + r 2^S],
// off = base mod 2^S: at stage S+u the pair (r, r + 2^u) sits at distance h = 2^(S+u) and its
// twiddle is dt[h + j], j = off + (r mod 2^u) 2^S its position in the half-block. Lazy
// butterflies: each stage adds less than 2q to the bound.
template <int R>
__device__ __forceinline__ void inv_radix(u64 (&x)[1 << R], int S, int off, const ulonglong2 *__restrict__ dt, u64 q,
                                          u64 q2) {
#pragma unroll
    for (int u = 0; u < R; ++u) {
#pragma unroll
        for (int m = 0; m < (1 << u); ++m) {
            const ulonglong2 w = BFV_LDG(dt + (1 << (S + u)) + off + (m << S));
#pragma unroll
            for (int k = 0; k < (1 << (R - 1 - u)); ++k) {
                const int r = m + (k << (u + 1));
                ct_bfly_lazy(x[r], x[r + (1 << u)], w.x, w.y, q, q2);
            }
        }
    }
}

// Pass schedule: LOGM stages in ceil(LOGM/4) passes of radix 2^3 or 2^4, R<P> larger first (the
// inverse driver takes them in reverse order).
template <int LOGM> struct Sched {
    static constexpr int NP = (LOGM + 3) / 4;
    template <int P> struct R { static constexpr int value = LOGM / NP + (P < LOGM % NP ? 1 : 0); };
};

// ------------------------------------------------------------------ forward NTT driver
//
// Transforms a sub-array of M = 2^LOGM points: sub-array `hidx` of the full size-N
// transform after its first C stages (C = log2 N - LOGM). load(p) returns the input at local
// position p (for C > 0: the value after stage C-1, produced by the caller); store(p, v)
// receives the final value in [0, q). sm: shared buffer of PadSize<M> words. Values given by
// load must be < 4q. The driver ends without a barrier after the last store.
// LAZY: no reductions at all (ct_bfly_lazy); store receives values below (4 + 2 log2 N) q, for
// consumers that only multiply them by Shoup constants.

// ILP2: the two radix-8 groups a thread handles in a pass are interleaved.
template <int LOGM, int NT, int P, int S, bool LAZY, bool ILP2 = false, class Load, class Store>
__device__ __forceinline__ void fwd_passes(u64 *sm, const ModTab &T, int C, int hidx, Load &load, Store &store) {
    constexpr int NP = Sched<LOGM>::NP;
    constexpr int R = Sched<LOGM>::template R<P>::value;
    constexpr int M = 1 << LOGM;
    constexpr int TL = M >> (S + R);
    constexpr int G = M >> R;
    const u64 q = T.q, q2 = T.q2;
#pragma unroll (ILP2 && R == 3 && G >= 2 * NT ? 2 : 1)
    for (int g = threadIdx.x; g < G; g += NT) {
        const int block = g / TL, off = g % TL;
        const int base = block * (TL << R) + off;
        u64 x[1 << R];
#pragma unroll
        for (int r = 0; r < (1 << R); ++r) {
            if constexpr (P == 0) x[r] = load(base + r * TL);
            else x[r] = sm[padi(base + r * TL)];
        }
        fwd_radix<R, LAZY>(x, S + C, (hidx << S) + block, T.fw, q, q2);
#pragma unroll
        for (int r = 0; r < (1 << R); ++r) {
            if constexpr (P == NP - 1) store(base + r * TL, LAZY ? x[r] : red1(red2(x[r], q2), q));
            else sm[padi(base + r * TL)] = x[r];
        }
    }
    if constexpr (P < NP - 1) {
        __syncthreads();
        fwd_passes<LOGM, NT, P + 1, S + R, LAZY, ILP2>(sm, T, C, hidx, load, store);
    }
}

template <int LOGM, int NT, class Load, class Store>
__device__ __forceinline__ void ntt_forward(u64 *sm, const ModTab &T, int C, int hidx, Load load, Store store) {
    fwd_passes<LOGM, NT, 0, 0, false>(sm, T, C, hidx, load, store);
}
template <int LOGM, int NT, bool ILP2 = false, class Load, class Store>
__device__ __forceinline__ void ntt_forward_lazy(u64 *sm, const ModTab &T, int C, int hidx, Load load, Store store) {
    fwd_passes<LOGM, NT, 0, 0, true, ILP2>(sm, T, C, hidx, load, store);
}

// ------------------------------------------------------------------ inverse NTT driver
//
// The first LOGM decimation-in-time stages of the inverse transform on M = 2^LOGM consecutive
// evaluation positions (their butterflies never leave them; the twiddles depend only on the
// position inside a half-block, so any aligned sub-array runs the same code). Passes of radix
// 2^3 or 2^4, smaller first (the first pass's twiddles are the same for every group). load(p)
// must return values < 2q (local position p); store(p, v) receives local position p unreduced,
// below (2 + 2 LOGM) q. The driver ends without a barrier after the last store.
template <int LOGM, int NT, int P, int S, class Load, class Store>
__device__ __forceinline__ void inv_passes(u64 *sm, const ModTab &T, Load &load, Store &store) {
    constexpr int NP = Sched<LOGM>::NP;
    constexpr int R = Sched<LOGM>::template R<NP - 1 - P>::value;
    constexpr int M = 1 << LOGM;
    constexpr int TL = 1 << S;
    constexpr int G = M >> R;
    const u64 q = T.q, q2 = T.q2;
#pragma unroll 1
    for (int g = threadIdx.x; g < G; g += NT) {
        const int block = g >> S, off = g & (TL - 1);
        const int base = block * (TL << R) + off;
        u64 x[1 << R];
#pragma unroll
        for (int r = 0; r < (1 << R); ++r) {
            if constexpr (P == 0) x[r] = load(base + r * TL);
            else x[r] = sm[padi(base + r * TL)];
        }
        inv_radix<R>(x, S, off, T.dt, q, q2);
#pragma unroll
        for (int r = 0; r < (1 << R); ++r) {
            if constexpr (P == NP - 1) store(base + r * TL, x[r]);
            else sm[padi(base + r * TL)] = x[r];
        }
    }
    if constexpr (P < NP - 1) {
        __syncthreads();
        inv_passes<LOGM, NT, P + 1, S + R>(sm, T, load, store);
    }
}

// The whole inverse transform of 2^LOGN points in one CTA: store(k, v) receives coefficient k in
// [0, q) (the post-twist N^-1 psi^-k applied to values below (2 + 2 LOGN) q < 32q).
template <int LOGN, int NT, class Load, class Store>
__device__ __forceinline__ void ntt_inverse(u64 *sm, const ModTab &T, Load load, Store store) {
    auto st = [&](int k, u64 v) {
        const ulonglong2 w = BFV_LDG(T.tw + k);
        store(k, red1(mul_shoup(v, w.x, w.y, T.q), T.q));
    };
    inv_passes<LOGN, NT, 0, 0>(sm, T, load, st);
}

// ------------------------------------------------------------------ index maps

// Bit reversal of p over logn bits.
__device__ __forceinline__ int brev_n(int p, int logn) { return (int)(__brev((u32)p) >> (32 - logn)); }

// Evaluation-layout automorphism X -> X^g: sigma_g(a) at position p is a at position
// brev(((2 brev(p) + 1) g mod 2N - 1) / 2).
__device__ __forceinline__ int auto_src(int p, u32 g, int logn) {
    const u32 e = 2u * (u32)brev_n(p, logn) + 1u;
    const u32 e2 = (e * g) & ((2u << logn) - 1u);
    return brev_n((int)((e2 - 1u) >> 1), logn);
}

// ------------------------------------------------------------------ TMA bulk copies and mbarriers

__device__ __forceinline__ u32 smem_addr(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(u64 *bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Arrive on the barrier and add `bytes` to the transaction count it waits for.
__device__ __forceinline__ void mbar_expect_tx(u64 *bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(u64 *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Bounded wait for the phase with the given parity; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(u64 *bar, u32 parity, long long limit) {
    const u32 a = smem_addr(bar);
    for (long long i = 0; i < limit; ++i) {
        u32 ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
// The same wait with the hardware suspending the thread for up to `hint_ns` nanoseconds per poll
// until the phase completes (a waiting warp then takes no issue slots); at most `limit` polls.
__device__ __forceinline__ bool mbar_wait_sleep(u64 *bar, u32 parity, long long limit, u32 hint_ns) {
    const u32 a = smem_addr(bar);
    for (long long i = 0; i < limit; ++i) {
        u32 ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity), "r"(hint_ns)
            : "memory");
        if (ok) return true;
    }
    return false;
}
// One-dimensional bulk copy global -> shared (16-byte aligned addresses, size a multiple of
// 16), completion counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, u32 bytes, u64 *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// ------------------------------------------------------------------ limbs split over a CTA pair
//
// Threads per CTA for a transform of 2^logm points.
constexpr int nt_for(int logm) { return logm >= 13 ? 512 : (logm == 12 ? 256 : 128); }

// A limb of N = 32768 points (256 KB) is larger than one CTA's shared memory. Such a limb is
// handled by a cluster of S = 2 CTAs; CTA h (its rank in the cluster) owns the evaluation
// positions and the coefficients [h M, (h+1) M), M = N/2:
//  * forward: the first Cooley-Tukey stage (distance N/2) is done in the load -- each CTA
//    reads both halves of the input -- and CTA h runs the remaining stages on its half;
//  * inverse: CTA h runs the first log2 N - 1 decimation-in-time stages on its own half of the
//    evaluation points (their butterflies stay inside it); after a cluster barrier the last
//    stage (distance N/2) reads the partner's half from distributed shared memory and applies
//    the post-twist.
// For N <= 16384, S = 1 and these are the single-CTA transforms.
// MODE 1 also splits an N = 16384 limb over two CTAs of 256 threads (68 KB of shared memory
// each), three of which share an SM (80 registers each) so that one's barrier waits overlap the
// others' work; MODE 2 is the same split with two CTAs per SM (128 registers each); MODE 3 splits
// the limb over two CTAs of 512 threads (one per SM; for launches too small to fill the GPU, where
// a transform's latency matters more than its throughput).
template <int LOGN, int MODE = 0> struct Split {
    static constexpr bool PAIR16K = (MODE == 1 || MODE == 2 || MODE == 3) && LOGN == 14;
    static constexpr int S = (LOGN > 14 || PAIR16K) ? 2 : 1;
    static constexpr int LOGM = LOGN - (S == 2 ? 1 : 0);
    static constexpr int M = 1 << LOGM;
    static constexpr int NT = PAIR16K ? (MODE == 3 ? 512 : 256) : nt_for(LOGM);
    static constexpr int MINB = PAIR16K ? (MODE == 1 ? 3 : MODE == 2 ? 2 : 1) : 1;
};

__device__ __forceinline__ u32 cluster_rank() {
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// All threads of all CTAs of the cluster; orders shared-memory writes before the barrier
// with reads after it, across the cluster.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Shared-memory address of `p` in the CTA of cluster rank `rank`.
__device__ __forceinline__ u32 cluster_map(const void *p, u32 rank) {
    u32 r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ u64 ld_cluster(u32 addr) {
    u64 v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}

// The first C Cooley-Tukey stages of a size-N forward transform, restricted to the outputs
// that land in sub-array `hidx` of size N/2^C: v[k] = input at p + k N/2^C (< 4q); returns
// the stage-C value at local position p of the sub-array (< 4q).
template <int C>
__device__ __forceinline__ u64 fold_stages(const ModTab &T, int hidx, u64 (&v)[1 << C]) {
    const u64 q = T.q, q2 = T.q2;
#pragma unroll
    for (int s = 0; s < C; ++s) {
        const int half = 1 << (C - 1 - s);
        const int side = (hidx >> (C - 1 - s)) & 1;
        const ulonglong2 w = BFV_LDG(T.fw + (1 << s) + (hidx >> (C - s)));
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const u64 a = red2(v[k], q2), t = mul_shoup(v[k + half], w.x, w.y, q);
            v[k] = side ? a - t + q2 : a + t;
        }
    }
    return v[0];
}

// Forward transform of one limb by CTA h of its group: load(k) returns coefficient k (< 4q,
// any k < N); store(p, v) receives the evaluation positions p this CTA owns, in [0, q)
// (LAZY: below 32q, for Shoup-product consumers only).
// ILP2: the two radix-8 groups a thread handles in a pass are interleaved (more independent
// multiplications in flight; more registers).
template <int LOGN, bool LAZY = false, int MODE = 0, bool ILP2 = false, class Load, class Store>
__device__ __forceinline__ void limb_forward(u64 *sm, const ModTab &T, int h, Load load, Store store) {
    using SP = Split<LOGN, MODE>;
    if constexpr (SP::S == 1) {
        fwd_passes<LOGN, SP::NT, 0, 0, LAZY, ILP2>(sm, T, 0, 0, load, store);
    } else {
        auto ld = [&](int p) {
            u64 v[2] = {load(p), load(p + SP::M)};
            return fold_stages<1>(T, h, v);
        };
        auto st = [&](int p, u64 v) { store(h * SP::M + p, v); };
        fwd_passes<SP::LOGM, SP::NT, 0, 0, LAZY, ILP2>(sm, T, 1, h, ld, st);
    }
}

// Inverse transform of one limb by CTA h of its group: load(p) returns evaluation position p
// (< 2q) for the positions this CTA owns; store(k, v) receives the coefficients k it owns,
// in [0, q). With S = 2 every thread of the cluster must call it (two cluster barriers), and
// sm must not be written by the caller between the call and the caller's next barrier.
template <int LOGN, int MODE = 0, class Load, class Store>
__device__ __forceinline__ void limb_inverse(u64 *sm, const ModTab &T, int h, Load load, Store store) {
    using SP = Split<LOGN, MODE>;
    if constexpr (SP::S == 1) {
        ntt_inverse<LOGN, SP::NT>(sm, T, load, store);
    } else {
        constexpr int M = SP::M;
        auto ld = [&](int p) { return load(h * M + p); };
        auto st = [&](int p, u64 v) { sm[padi(p)] = v; };
        inv_passes<SP::LOGM, SP::NT, 0, 0>(sm, T, ld, st);
        __syncthreads();
        const u64 q = T.q, q2 = T.q2;
        // last stage (distance M, across the pair): u = x[p] on CTA 0, t = dt[M + p] x[M + p] on CTA 1
        if (h == 1) {
#pragma unroll 4
            for (int p = threadIdx.x; p < M; p += SP::NT) {
                const ulonglong2 w = BFV_LDG(T.dt + M + p);
                sm[padi(p)] = mul_shoup(sm[padi(p)], w.x, w.y, q);
            }
        }
        cluster_sync();
        const u32 peer = cluster_map(sm, (u32)(h ^ 1));
#pragma unroll 4
        for (int p = threadIdx.x; p < M; p += SP::NT) {
            const u64 own = sm[padi(p)], other = ld_cluster(peer + 8u * (u32)padi(p));
            const u64 x = h == 0 ? own + other : other - own + q2;   // u + t, or u - t (below 32q)
            const ulonglong2 w = BFV_LDG(T.tw + h * M + p);
            store(h * M + p, red1(mul_shoup(x, w.x, w.y, q), q));
        }
        cluster_sync();
    }
}

// ------------------------------------------------------------------ tensor memory (TMEM)
//
// 128 lanes x 512 columns of 32-bit cells per SM. A warp reaches the 32 lanes of its quarter
// (warp % 4); an address is (lane << 16) | column relative to the allocation's base.

// One whole warp: allocate ncols columns (a power of two >= 32) and write the base address to
// *slot; then give up the right to allocate again so that other CTAs may.
__device__ __forceinline__ void tmem_alloc(u32 *slot, u32 ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
// One whole warp, after every thread's last access (see tmem_fence_*).
__device__ __forceinline__ void tmem_dealloc(u32 base, u32 ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}
// Order TMEM accesses across a thread barrier: before_sync ... __syncthreads() ... after_sync.
__device__ __forceinline__ void tmem_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 16 consecutive columns of this thread's lane (warp-wide, lane field = the warp's quarter).
__device__ __forceinline__ void tmem_ld16(u32 addr, u32 (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr)
        : "memory");
}
__device__ __forceinline__ void tmem_st16(u32 addr, const u32 (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(addr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 8 consecutive columns of this thread's lane (warp-wide).
__device__ __forceinline__ void tmem_ld8(u32 addr, u32 (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr)
                 : "memory");
}

// ------------------------------------------------------------------ tensor-core MMA (tcgen05, kind::f16)
//
// Shared-memory matrix descriptor of an operand tile in the canonical K-major layout without
// swizzling: core matrices of 8 rows x 16 bytes (128 contiguous bytes, row r at byte 16 r);
// `lbo` = bytes between core matrices adjacent along K, `sbo` = bytes between core matrices
// adjacent along M (or N). Bits: start address >> 4 [0, 14), lbo >> 4 [16, 30), sbo >> 4
// [32, 46), the descriptor version 1 at bit 46, no base offset, no swizzle.
__device__ __forceinline__ u64 umma_desc_kmajor(const void *tile, u32 lbo, u32 sbo) {
    const u32 a = smem_addr(tile);
    return (u64)((a & 0x3FFFFu) >> 4) | ((u64)(lbo >> 4) << 16) | ((u64)(sbo >> 4) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16 with f16 A and B, f32 D, both operands K-major: D type
// at bits [4, 6) (1 = f32), A and B types at [7, 10) and [10, 13) (0 = f16), N >> 3 at [17, 23),
// M >> 4 at [24, 29).
__host__ __device__ constexpr u32 umma_idesc_f16_f32(int M, int N) {
    return (1u << 4) | ((u32)(N >> 3) << 17) | ((u32)(M >> 4) << 24);
}
// D[tmem] (+)= A[smem] x B[smem]^T for one K = 16 step; issued by one thread.
__device__ __forceinline__ void umma_f16(u32 d_tmem, u64 adesc, u64 bdesc, u32 idesc, bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((u32)accumulate)
        : "memory");
}
// The mbarrier receives one arrival when every MMA this thread issued before has completed
// (its shared-memory operands read, its tensor-memory results written).
__device__ __forceinline__ void umma_commit(u64 *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}
// Orders this thread's generic-proxy shared-memory writes before later async-proxy reads (the
// tensor cores' operand loads) that a barrier hands them to.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ------------------------------------------------------------------ ChaCha20 (RFC 8439)

__device__ __forceinline__ u32 rotl(u32 x, int n) { return __funnelshift_l(x, x, n); }
#define BFV_QR(a, b, c, d)                                  \
    a += b; d ^= a; d = rotl(d, 16); c += d; b ^= c; b = rotl(b, 12); \
    a += b; d ^= a; d = rotl(d, 8);  c += d; b ^= c; b = rotl(b, 7);

// Block `counter` of the stream keyed by the 64-bit seed (zero-extended to 256 bits) with
// nonce (n0, n1, n2); writes the 16 output words.
__device__ __forceinline__ void chacha20_block(u64 seed, u32 counter, u32 n0, u32 n1, u32 n2, u32 (&o)[16]) {
    const u32 s0 = 0x61707865u, s1 = 0x3320646eu, s2 = 0x79622d32u, s3 = 0x6b206574u;
    const u32 k0 = (u32)seed, k1 = (u32)(seed >> 32);
    u32 x0 = s0, x1 = s1, x2 = s2, x3 = s3, x4 = k0, x5 = k1, x6 = 0, x7 = 0, x8 = 0, x9 = 0, x10 = 0, x11 = 0,
        x12 = counter, x13 = n0, x14 = n1, x15 = n2;
#pragma unroll 1
    for (int r = 0; r < 10; ++r) {
        BFV_QR(x0, x4, x8, x12) BFV_QR(x1, x5, x9, x13) BFV_QR(x2, x6, x10, x14) BFV_QR(x3, x7, x11, x15)
        BFV_QR(x0, x5, x10, x15) BFV_QR(x1, x6, x11, x12) BFV_QR(x2, x7, x8, x13) BFV_QR(x3, x4, x9, x14)
    }
    o[0] = x0 + s0; o[1] = x1 + s1; o[2] = x2 + s2; o[3] = x3 + s3;
    o[4] = x4 + k0; o[5] = x5 + k1; o[6] = x6; o[7] = x7;
    o[8] = x8; o[9] = x9; o[10] = x10; o[11] = x11;
    o[12] = x12 + counter; o[13] = x13 + n0; o[14] = x14 + n1; o[15] = x15 + n2;
}
#undef BFV_QR

// Ternary value {-1, 0, 1} from one word: floor(3 w / 2^32) - 1.
__device__ __forceinline__ int ternary_of(u32 w) { return (int)(((u64)w * 3ull) >> 32) - 1; }

// Discrete Gaussian from a 64-bit draw and a sign word: magnitude = number of thresholds
// not above the draw; negative when the sign bit is set and the magnitude is non-zero.
__device__ __forceinline__ int gauss_of(u32 lo, u32 hi, u32 sgn, const u64 *cdt, int n) {
    const u64 r = (u64)lo | ((u64)hi << 32);
    int mag = 0;
    for (int k = 0; k < n; ++k) mag += (r >= BFV_LD(cdt + k)) ? 1 : 0;
    return (mag != 0 && (sgn & 1u)) ? -mag : mag;
}

// A constant operand and its Shoup companion, stored side by side.
typedef ulonglong2 shoup_t;
__device__ __forceinline__ shoup_t make_shoup(u64 w, u64 q) { return make_ulonglong2(w, shoup_companion(w, q)); }
__device__ __forceinline__ u64 mul_shoup(u64 x, shoup_t w, u64 q) { return mul_shoup(x, w.x, w.y, q); }

// Small signed integer lifted into [0, q).
__device__ __forceinline__ u64 lift_small(int v, u64 q) { return v >= 0 ? (u64)v : q - (u64)(-v); }
