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
        for (int ff = 0; ff < nf; ++ff)
            if (BFV_RANGE_OK(X + (f0 + ff) * ctw + e0, kE * 8))
                bulk_g2s(&s.x[slot][ff][0], X + (f0 + ff) * ctw + e0, kE * 8, &s.full[slot]);
        if (BFV_RANGE_OK(W16 + f0 * kNY, (u32)nf * kNY * 4))
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
    for (int j = 0; j < kNY; ++j) BFV_ST(out + (size_t)j * ctw, make_longlong2(lo[j], hi[j]));
}

// ------------------------------------------------------------------ int8 weights: byte planes + dp4a
//
// For |w| <= 127 the product is formed byte by byte: x = sum_k 2^(8k) x_k, and for four
// features at a time the bytes x_k of the four residues are packed into one 32-bit word
// (PRMT) and dotted with the four features' int8 weights by one dp4a (4 multiply-adds per
// instruction). Each thread keeps one int32 accumulator per (class, byte plane) for 8 of
// the 16 classes (two threads per ciphertext word); an accumulator grows by at most
// 4 * 255 * 127 per dp4a, so a split may hold up to 65,536 features. The planes are folded
// into (lo, hi) = (sum_{k<4} 2^(8k) acc_k, sum_{k>=4} 2^(8(k-4)) acc_k), i.e. split at 32 bits.

constexpr int kE8 = 128;                  // ciphertext words per CTA tile (two threads per word)
constexpr int kS8 = 4;                    // stages in flight

struct Std8Smem {
    u64 x[kS8][kF][kE8];
    int w[kS8][kF / 4][kNY];               // four features' int8 weights per int32, per class
    u64 full[kS8];                         // copies of a stage landed
    u64 empty[kS8];                        // every warp is done with a stage
};

__device__ __forceinline__ int dp4a_us(u32 a, int b, int c) {
    int d;
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ u32 prmt(u32 a, u32 b, u32 sel) {
    u32 d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}
// Byte planes 4q .. 4q+3 of four 32-bit halves a0..a3: plane k holds byte k of a0, a1, a2, a3.
__device__ __forceinline__ void planes4(u32 a0, u32 a1, u32 a2, u32 a3, u32 (&p)[4]) {
    const u32 t01 = prmt(a0, a1, 0x5140u), t23 = prmt(a2, a3, 0x5140u);   // bytes 0, 1
    const u32 u01 = prmt(a0, a1, 0x7362u), u23 = prmt(a2, a3, 0x7362u);   // bytes 2, 3
    p[0] = prmt(t01, t23, 0x5410u);
    p[1] = prmt(t01, t23, 0x7632u);
    p[2] = prmt(u01, u23, 0x5410u);
    p[3] = prmt(u01, u23, 0x7632u);
}

template <int NP>
__global__ void __launch_bounds__(2 * kE8 + 32, 2) k_standard_dp4a(const int *__restrict__ W4, const u64 *__restrict__ X,
                                                                   size_t ctw, size_t F, size_t fper,
                                                                   longlong2 *partial, int *err, u32 extra_tx,
                                                                   long long wait_limit) {
    extern __shared__ __align__(128) unsigned char raw[];
    Std8Smem &s = *reinterpret_cast<Std8Smem *>(raw);
    constexpr int kConsumers = 2 * kE8;                 // warps 0..7 compute, warp 8 copies
    const size_t ntiles = ctw / kE8;
    const size_t tile = blockIdx.x % ntiles, split = blockIdx.x / ntiles;
    const size_t e0 = tile * kE8;
    const size_t fa = split * fper, fb = std::min(F, fa + fper);
    const int nst = fa < fb ? (int)((fb - fa + kF - 1) / kF) : 0;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < kS8; ++i) {
            mbar_init(&s.full[i], 1);
            mbar_init(&s.empty[i], kConsumers / 32);
        }
        mbar_init_fence();
    }
    __syncthreads();
    bool failed = false;
    if (tid >= kConsumers) {
        // producer warp: lane 0 streams the stages, refilling a slot once every consumer warp let go
        if (tid == kConsumers) {
            int st = 0;
            for (; st < nst; ++st) {
                const int slot = st % kS8;
                if (st >= kS8 && !mbar_wait(&s.empty[slot], (u32)(((st - kS8) / kS8) & 1), wait_limit)) {
                    failed = true;
                    break;
                }
                const size_t f0 = fa + (size_t)st * kF;
                const int nf = (int)std::min((size_t)kF, fb - f0);
                const int ng = (nf + 3) / 4;
                mbar_expect_tx(&s.full[slot], (u32)nf * (kE8 * 8) + (u32)ng * kNY * 4 + (st == 0 ? extra_tx : 0u));
                for (int ff = 0; ff < nf; ++ff)
                    if (BFV_RANGE_OK(X + (f0 + ff) * ctw + e0, kE8 * 8))
                        bulk_g2s(&s.x[slot][ff][0], X + (f0 + ff) * ctw + e0, kE8 * 8, &s.full[slot]);
                if (BFV_RANGE_OK(W4 + (f0 / 4) * kNY, (u32)ng * kNY * 4))
                    bulk_g2s(&s.w[slot][0][0], W4 + (f0 / 4) * kNY, (u32)ng * kNY * 4, &s.full[slot]);
            }
            // drain: the last stages issued may still be landing
            for (int k = st > kS8 ? st - kS8 : 0; k < st; ++k) mbar_wait(&s.full[k % kS8], (u32)((k / kS8) & 1), wait_limit);
        }
    } else {
        const int ew = tid % kE8, jh = tid / kE8;          // word, class half
        int acc[8][NP];
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int k = 0; k < NP; ++k) acc[j][k] = 0;
        for (int st = 0; st < nst; ++st) {
            const int slot = st % kS8;
            if (!mbar_wait(&s.full[slot], (u32)((st / kS8) & 1), wait_limit)) {
                failed = true;
                break;
            }
            const size_t f0 = fa + (size_t)st * kF;
            const int nf = (int)std::min((size_t)kF, fb - f0);
            for (int g4 = 0; g4 < (nf + 3) / 4; ++g4) {
                u64 x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = (g4 * 4 + u < nf) ? s.x[slot][g4 * 4 + u][ew] : 0ull;
                u32 pl[8];
                {
                    u32 lo4[4], hi4[4];
                    planes4((u32)x[0], (u32)x[1], (u32)x[2], (u32)x[3], lo4);
                    planes4((u32)(x[0] >> 32), (u32)(x[1] >> 32), (u32)(x[2] >> 32), (u32)(x[3] >> 32), hi4);
#pragma unroll
                    for (int k = 0; k < 4; ++k) { pl[k] = lo4[k]; pl[4 + k] = hi4[k]; }
                }
                const int4 *wv = reinterpret_cast<const int4 *>(&s.w[slot][g4][jh * 8]);
                const int4 wa = wv[0], wb = wv[1];
                const int ws[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                for (int j = 0; j < 8; ++j)
#pragma unroll
                    for (int k = 0; k < NP; ++k) acc[j][k] = dp4a_us(pl[k], ws[j], acc[j][k]);
            }
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(&s.empty[slot]);
        }
        if (!failed) {
            longlong2 *out = partial + (split * kNY + jh * 8) * ctw + e0 + ew;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                long long lo = 0, hi = 0;
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    if (k < 4) lo += (long long)acc[j][k] * (1ll << (8 * k));
                    else hi += (long long)acc[j][k] * (1ll << (8 * (k - 4)));
                }
                BFV_ST(out + (size_t)j * ctw, make_longlong2(lo, hi));
            }
        }
    }
    // a bounded wait ran out somewhere: report it (the output of this launch is invalid)
    if (__syncthreads_or(failed) && tid == 0) atomicOr(err, 1);
}

// ------------------------------------------------------------------ int8 weights on the tensor cores
//
// The same byte-plane sums as a tensor-core contraction: for each byte plane b < NP,
// D_b[e][j] = sum_f byte_b(X_f[e]) w[f][j] with M = 128 ciphertext words (a tile), N = 16
// classes and K = features, as tcgen05.mma kind::f16 (A: the byte planes, B: the weights, both
// exact in f16; D: f32 in tensor memory). A plane holds 1024 + byte (the byte placed under the
// exponent bits of 1024 by byte permutes, plane_rows), and after each plane's MMA a
// second MMA with a constant tile of -1024 removes the offset, so D_b sums byte x weight exactly:
// every product and every partial sum is an integer below 2^24 in magnitude (a chunk of 256
// features sums to below 2^23, an offset MMA adds at most 16 x 1279 x 127 before the correction
// removes it). After each chunk the sums are moved into the (lo, hi) int64 split sums that the
// dp4a kernel forms (lo = sum_{b<4} 2^(8b) D_b, hi = sum_{b>=4} 2^(8(b-4)) D_b).
//
// Warps 0-7 convert: thread t owns word e = t % 128 of the tile and features 8 (t / 128) ..
// +7 of each 16-feature stage; it splits its eight residues into byte planes and writes one
// 16-byte row of each plane's A tile (canonical K-major layout). The same threads drain the
// accumulators of their TMEM lane (classes 8 (t / 128) .. +7). Warp 8 streams the raw
// ciphertext rows and the stage's f16 weight tile (already in the canonical B layout) with
// cp.async.bulk; warp 9 allocates the tensor memory and one of its threads issues the MMAs.
// Two accumulator sets alternate so that a chunk drains while the next one accumulates. Waiting
// threads sleep in the barrier (a suspend-time hint) rather than spin. Every wait is bounded: a wait that runs out sets the context's error word and the CTA winds down
// (its MMAs completed, its copies landed or timed out, its tensor memory freed).

constexpr int kTcE = 128;                 // ciphertext words per tile (MMA M)
constexpr int kTcChunk = 16;              // stages (16 features each) per f32 accumulation chunk
constexpr int kTcConv = 256;              // converter threads
constexpr int kTcThreads = kTcConv + 64;  // + the copy warp and the MMA warp
constexpr u32 kTcCols = 256;              // tensor-memory columns: 2 sets x 8 planes x 16 classes

template <int NP> struct TcSmem {
    static constexpr int SR = NP >= 8 ? 2 : 3;        // raw stages in flight
    static constexpr int SA = 2;                      // converted stages in flight
    u64 x[SR][kF][kTcE];                              // raw rows: feature ff of the stage, word e
    uint16_t w[SR][256];                              // the stage's f16 weights (canonical B tile)
    alignas(128) uint16_t a[SA][NP][kTcE * kF];       // byte planes (canonical A tiles, 4 KB each)
    alignas(128) uint16_t b[SA][256];                 // the weights of the converted stage
    alignas(128) uint16_t neg[kTcE * kF];             // a constant A tile of -1024 (the offset correction)
    u64 raw_full[SR], raw_empty[SR], a_full[SA], a_empty[SA], acc_full[2], acc_empty[2], done;
    u32 tmem_base;
};

// The A rows of all NP byte planes from eight residues v[0..7] (features 8 k8 .. +7 of word e):
// row b holds the f16 pairs (1024 + byte_b(v[2i]), 1024 + byte_b(v[2i+1])), i < 4. For each pair
// of residues and each 32-bit half, one PRMT interleaves the bytes of planes {0, 2} and one those
// of {1, 3} ([x_0, y_0, x_2, y_2], [x_1, y_1, x_3, y_3]); one PRMT per plane then places two of
// them under the exponent byte 0x64 of 1024 (three PRMTs per two f16 pairs).
template <int NP>
__device__ __forceinline__ void plane_rows(const u64 (&v)[8], uint4 (&row)[NP]) {
    constexpr u32 C64 = 0x64646464u;
    u32 o[NP][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            if (4 * half >= NP) continue;
            const u32 x = half ? (u32)(v[2 * i] >> 32) : (u32)v[2 * i];
            const u32 y = half ? (u32)(v[2 * i + 1] >> 32) : (u32)v[2 * i + 1];
            const u32 t02 = prmt(x, y, 0x6240u), t13 = prmt(x, y, 0x7351u);
            const int b0 = 4 * half;
            if (b0 + 0 < NP) o[b0 + 0][i] = prmt(t02, C64, 0x4140u);     // [x_0, 64, y_0, 64]
            if (b0 + 2 < NP) o[b0 + 2][i] = prmt(t02, C64, 0x4342u);     // [x_2, 64, y_2, 64]
            if (b0 + 1 < NP) o[b0 + 1][i] = prmt(t13, C64, 0x4140u);     // [x_1, 64, y_1, 64]
            if (b0 + 3 < NP) o[b0 + 3][i] = prmt(t13, C64, 0x4342u);     // [x_3, 64, y_3, 64]
        }
    }
#pragma unroll
    for (int b = 0; b < NP; ++b) row[b] = make_uint4(o[b][0], o[b][1], o[b][2], o[b][3]);
}

// A bounded wait by a whole warp with one outcome for all its lanes (the tensor-memory loads that
// follow are warp-collective, so no lane may leave the loop alone).
constexpr u32 kTcSleepNs = 20000;         // suspend-time hint of a poll
__device__ __forceinline__ bool warp_wait(u64 *bar, u32 parity, long long limit) {
    return __all_sync(0xffffffffu, mbar_wait_sleep(bar, parity, limit, kTcSleepNs));
}

template <int NP>
__global__ void __launch_bounds__(kTcThreads, 2) k_standard_tc(const uint16_t *__restrict__ Wtc,
                                                              const u64 *__restrict__ X, size_t ctw, size_t F,
                                                              size_t fper, longlong2 *partial, int *err,
                                                              u32 extra_tx, long long wait_limit) {
    extern __shared__ __align__(1024) unsigned char raw[];
    using SM = TcSmem<NP>;
    constexpr int SR = SM::SR, SA = SM::SA;
    SM &s = *reinterpret_cast<SM *>(raw);
    const size_t ntiles = ctw / kTcE;
    const size_t tile = blockIdx.x % ntiles, split = blockIdx.x / ntiles;
    const size_t e0 = tile * kTcE;
    const size_t fa = split * fper, fb = std::min(F, fa + fper);
    const int nst = fa < fb ? (int)((fb - fa + kF - 1) / kF) : 0;
    const int nchunks = (nst + kTcChunk - 1) / kTcChunk;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        for (int i = 0; i < SR; ++i) { mbar_init(&s.raw_full[i], 1); mbar_init(&s.raw_empty[i], kTcConv / 32); }
        for (int i = 0; i < SA; ++i) { mbar_init(&s.a_full[i], kTcConv / 32); mbar_init(&s.a_empty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&s.acc_full[i], 1); mbar_init(&s.acc_empty[i], kTcConv / 32); }
        mbar_init(&s.done, 1);
        mbar_init_fence();
    }
    for (int i = tid; i < kTcE * kF / 2; i += kTcThreads) reinterpret_cast<u32 *>(s.neg)[i] = 0xE400E400u;  // -1024
    fence_proxy_async_smem();
    if (warp == 9) tmem_alloc(&s.tmem_base, kTcCols);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const u32 tbase = s.tmem_base;
    bool failed = false;

    if (warp == 8) {
        // copy warp: lane 0 streams the stages, refilling a slot once every converter warp let go
        if (tid == kTcConv) {
            int st = 0;
            for (; st < nst; ++st) {
                const int slot = st % SR;
                if (st >= SR && !mbar_wait_sleep(&s.raw_empty[slot], (u32)(((st - SR) / SR) & 1), wait_limit, kTcSleepNs)) {
                    failed = true;
                    break;
                }
                const size_t f0 = fa + (size_t)st * kF;
                const int nf = (int)std::min((size_t)kF, fb - f0);
                mbar_expect_tx(&s.raw_full[slot], (u32)nf * (kTcE * 8) + 512u + (st == 0 ? extra_tx : 0u));
                for (int ff = 0; ff < nf; ++ff)
                    if (BFV_RANGE_OK(X + (f0 + ff) * ctw + e0, kTcE * 8))
                        bulk_g2s(&s.x[slot][ff][0], X + (f0 + ff) * ctw + e0, kTcE * 8, &s.raw_full[slot]);
                if (BFV_RANGE_OK(Wtc + (f0 / kF) * 256, 512u))
                    bulk_g2s(&s.w[slot][0], Wtc + (f0 / kF) * 256, 512u, &s.raw_full[slot]);
            }
            // the last stages issued may still be landing
            for (int k = st > SR ? st - SR : 0; k < st; ++k)
                mbar_wait_sleep(&s.raw_full[k % SR], (u32)((k / SR) & 1), wait_limit, kTcSleepNs);
        }
    } else if (warp == 9) {
        // MMA warp: one thread issues NP MMAs per stage into the chunk's accumulator set
        if ((tid & 31) == 0) {
            constexpr u32 idesc = umma_idesc_f16_f32(kTcE, 16);
            for (int st = 0; st < nst && !failed; ++st) {
                const int c = st / kTcChunk, k = st % kTcChunk, set = c & 1, as = st % SA;
                if (k == 0 && c >= 2) {
                    if (!mbar_wait_sleep(&s.acc_empty[set], (u32)(((c - 2) / 2) & 1), wait_limit, kTcSleepNs)) { failed = true; break; }
                    tmem_fence_after_sync();
                }
                if (!mbar_wait_sleep(&s.a_full[as], (u32)((st / SA) & 1), wait_limit, kTcSleepNs)) { failed = true; break; }
                tmem_fence_after_sync();
                const u64 bdesc = umma_desc_kmajor(&s.b[as][0], 128, 256), ndesc = umma_desc_kmajor(s.neg, 128, 256);
#pragma unroll
                for (int b = 0; b < NP; ++b) {
                    const u32 d = tbase + (u32)(set * 128 + b * 16);
                    umma_f16(d, umma_desc_kmajor(&s.a[as][b][0], 128, 256), bdesc, idesc, k > 0);
                    umma_f16(d, ndesc, bdesc, idesc, true);          // minus 1024 x the stage's weights
                }
                umma_commit(&s.a_empty[as]);
                if (k == kTcChunk - 1 || st == nst - 1) umma_commit(&s.acc_full[set]);
            }
            // every MMA issued has completed before the CTA frees its shared and tensor memory
            umma_commit(&s.done);
            mbar_wait_sleep(&s.done, 0, wait_limit, kTcSleepNs);
        }
    } else {
        // converters: byte planes in, accumulators out
        const int e = tid & (kTcE - 1), k8 = tid >> 7;
        const u32 lane_addr = tbase + ((u32)(32 * (warp & 3)) << 16);
        long long lo[8], hi[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) { lo[j] = 0; hi[j] = 0; }
        // Chunk c's sums drain one plane per converted stage (the MMA warp needs that set again
        // only 16 stages later), so the converters never stop for a whole drain.
        int drained = 0, dplane = -1;                  // chunks drained; plane of the drain in progress
        auto drain_plane = [&](int c, int b) -> bool {
            const int set = c & 1;
            if (b == 0) {
                if (!warp_wait(&s.acc_full[set], (u32)((c / 2) & 1), wait_limit)) return false;
                tmem_fence_after_sync();
            }
            u32 r[8];
            tmem_ld8(lane_addr + (u32)(set * 128 + b * 16 + k8 * 8), r);
            tmem_wait_ld();
            const int sh = 8 * (b & 3);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const long long v = (long long)__float2int_rn(__uint_as_float(r[j])) * (1ll << sh);
                if (b < 4) lo[j] += v;
                else hi[j] += v;
            }
            if (b == NP - 1) {
                tmem_fence_before_sync();
                __syncwarp();
                if ((tid & 31) == 0) mbar_arrive(&s.acc_empty[set]);
            }
            return true;
        };
        auto drain_step = [&]() -> bool {
            if (dplane < 0) return true;
            if (!drain_plane(drained, dplane)) return false;
            if (++dplane == NP) { dplane = -1; ++drained; }
            return true;
        };
        for (int st = 0; st < nst; ++st) {
            const int rs = st % SR, as = st % SA;
            if (!warp_wait(&s.raw_full[rs], (u32)((st / SR) & 1), wait_limit)) { failed = true; break; }
            if (st >= SA && !warp_wait(&s.a_empty[as], (u32)(((st - SA) / SA) & 1), wait_limit)) { failed = true; break; }
            u64 v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = s.x[rs][k8 * 8 + i][e];   // rows past the range: weights are 0
            uint4 rows[NP];
            plane_rows<NP>(v, rows);
#pragma unroll
            for (int b = 0; b < NP; ++b)
                *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(&s.a[as][b][0]) + (e >> 3) * 256 + k8 * 128 +
                                           (e & 7) * 16) = rows[b];
            if (k8 == 0) reinterpret_cast<u32 *>(&s.b[as][0])[e] = reinterpret_cast<const u32 *>(&s.w[rs][0])[e];
            fence_proxy_async_smem();
            __syncwarp();
            if ((tid & 31) == 0) {
                mbar_arrive(&s.raw_empty[rs]);
                mbar_arrive(&s.a_full[as]);
            }
            // a chunk whose last stage the MMA warp finished SA stages ago starts draining
            const int done_st = st - SA;
            if (done_st >= 0 && done_st % kTcChunk == kTcChunk - 1) dplane = 0;
            if (!drain_step()) { failed = true; break; }
        }
        while (!failed && (dplane >= 0 || drained < nchunks)) {
            if (dplane < 0) dplane = 0;
            if (!drain_step()) { failed = true; break; }
        }
        if (!failed) {
            longlong2 *out = partial + (split * kNY + k8 * 8) * ctw + e0 + e;
#pragma unroll
            for (int j = 0; j < 8; ++j) BFV_ST(out + (size_t)j * ctw, make_longlong2(lo[j], hi[j]));
        }
    }
    // a bounded wait ran out somewhere: report it (the output of this launch is invalid)
    if (__syncthreads_or(failed) && tid == 0) atomicOr(err, 1);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (warp == 9) tmem_dealloc(tbase, kTcCols);
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
        const longlong2 v = BFV_LD(partial + ((size_t)sp * kNY + j) * ctw + e);
        lo += v.x;
        hi += v.y;
    }
    const int l = (int)((e / N) % L);
    const ModTab T = BFV_LD(mods + l);
    const long long q = (long long)T.q;
    long long h = hi % q; if (h < 0) h += q;
    long long a = lo % q; if (a < 0) a += q;
    const u64 sh = (1ull << split_bits) % T.q;
    u64 v = add_mod(mul_barrett((u64)h, sh, T.q, T.mu, T.bits), (u64)a, T.q);
    if (e < (size_t)L * N && e % N == 0) v = add_mod(v, BFV_LD(bias_delta + (size_t)(j0 + j) * L + l), T.q);
    BFV_ST(Y + (size_t)(j0 + j) * ctw + e, v);
}

}  // namespace

#ifdef BFV_BOUNDS
BFV_BOUNDS_UPLOAD_FN(bounds_upload_standard)
#endif

StandardPlan standard_plan(const bfv_ctx *c, const bfv_model *m) {
    StandardPlan p{};
    const size_t ctw = 2 * (size_t)c->L * c->N;
    p.int8 = m->wmax <= 127 && c->bits <= 64;
    p.tc = p.int8 && c->std_kernel == 0;
    p.ntiles = ctw / (p.int8 ? kE8 : kE);
    const size_t target = (size_t)c->sms * 2 * 6;    // about six waves of two CTAs per SM
    size_t splits = std::max<size_t>(1, (target + p.ntiles - 1) / p.ntiles);
    splits = std::min<size_t>(splits, std::max<size_t>(1, (m->f + 4 * kF - 1) / (4 * kF)));
    if (p.int8 && !p.tc) splits = std::max<size_t>(splits, (m->f + 65535) / 65536);   // int32 plane accumulators
    p.fper = ((m->f + splits - 1) / splits + kF - 1) / kF * kF;
    p.splits = (m->f + p.fper - 1) / p.fper;
    p.ngroups = (m->nY + kNY - 1) / kNY;
    p.split_bits = p.int8 ? 32 : (c->bits + 1) / 2;
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
    const int np = (c->bits + 7) / 8;
    const long long limit = c->inject_extra_tx ? (1ll << 12) : kWaitLimit;
    for (size_t gi = 0; gi < pl.ngroups; ++gi) {
        const int j0 = (int)(gi * kNY), nj = (int)std::min<size_t>(kNY, m->nY - j0);
        const unsigned grid = (unsigned)(pl.ntiles * pl.splits);
        if (pl.tc) {
            const uint16_t *wtc = m->wtc + gi * ((m->f + kF - 1) / kF) * 256;
#define STDTC(NP)                                                                                                  \
    {                                                                                                              \
        cudaFuncSetAttribute(k_standard_tc<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem<NP>)); \
        k_standard_tc<NP><<<grid, kTcThreads, sizeof(TcSmem<NP>), st>>>(wtc, X_ct, ctw, m->f, pl.fper, partial,       \
                                                                       c->derr, (u32)c->inject_extra_tx, tc_limit); \
    }
            const long long tc_limit = c->inject_extra_tx ? (1ll << 7) : (1ll << 16);   // <= ~1.3 s of polls
            switch (np) {
                case 4: STDTC(4); break;
                case 5: STDTC(5); break;
                case 6: STDTC(6); break;
                case 7: STDTC(7); break;
                default: STDTC(8); break;
            }
#undef STDTC
        } else if (pl.int8) {
            const int *w4 = m->w4 + gi * ((m->f + 3) / 4) * kNY;
#define STD8(NP)                                                                                                   \
    {                                                                                                              \
        cudaFuncSetAttribute(k_standard_dp4a<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Std8Smem)); \
        k_standard_dp4a<NP><<<grid, 2 * kE8 + 32, sizeof(Std8Smem), st>>>(w4, X_ct, ctw, m->f, pl.fper, partial,    \
                                                                        c->derr,                                  \
                                                                        (u32)c->inject_extra_tx, limit);          \
    }
            switch (np) {
                case 4: STD8(4); break;
                case 5: STD8(5); break;
                case 6: STD8(6); break;
                case 7: STD8(7); break;
                default: STD8(8); break;
            }
#undef STD8
        } else {
            k_standard_stream<<<grid, kE, sizeof(StdSmem), st>>>(m->w16 + gi * m->f * kNY, X_ct, ctw, m->f, pl.fper,
                                                                pl.split_bits, partial, c->derr,
                                                                (u32)c->inject_extra_tx, limit);
        }
        const size_t n = (size_t)nj * ctw;
        k_standard_finalize<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c->dmods, c->N, c->L, ctw, (int)pl.splits, nj, j0,
                                                                         pl.split_bits, partial, m->bias_delta, Y_ct);
        count_launch(c, 2);
    }
    return cudaGetLastError() == cudaSuccess ? BFV_OK : BFV_ERR_CUDA;
}
