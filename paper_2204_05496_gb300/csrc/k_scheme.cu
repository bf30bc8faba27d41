// k_scheme.cu -- BFV scheme kernels: limb NTTs, batch encode/decode, key generation,
// public-key encryption and exact decryption, model (weight) encoding.
//
// Every per-limb kernel runs Split<LOGN>::S CTAs per limb (a cluster of two at N = 32768,
// one otherwise): `h` is the CTA's part of the limb, `unit` the limb's index in the grid.
#include "bfv_internal.h"

namespace {

constexpr int kSkPurpose = 1, kPkA = 2, kPkE = 3, kGkA = 4, kGkE = 5, kEnc = 6;

// uniform residue mod q from four ChaCha words taken as a 128-bit integer
__device__ __forceinline__ u64 uniform_of(const u32 *w, const ModTab &T) {
    const u64 lo = (u64)w[0] | ((u64)w[1] << 32), hi = (u64)w[2] | ((u64)w[3] << 32);
    const u64 h = red1(mul_shoup(hi % T.q, T.r64, T.r64p, T.q), T.q);
    return add_mod(h, lo % T.q, T.q);
}

// ------------------------------------------------------------------ limb transforms
// in/out: [nlimbs][N]; limb x uses modulus x % L. The forward transform needs in != out and
// leaves its values unreduced (below 32q): its outputs only enter Shoup products (k_mac).
template <int LOGN, bool FWD>
LIMB_KERNEL(LOGN) k_ntt_limbs(const ModTab *__restrict__ mods, int L, const u64 *in, u64 *out) {
    extern __shared__ u64 sm[];
    LIMB_INDEX(LOGN);
    const ModTab T = BFV_LD(mods + unit % L);
    const u64 *src = in + unit * N;
    u64 *dst = out + unit * N;
    if constexpr (FWD)
        limb_forward<LOGN, true>(sm, T, h, [&](int p) { return BFV_LD(src + p); }, [&](int p, u64 v) { BFV_ST(dst + p, v); });
    else
        limb_inverse<LOGN>(sm, T, h, [&](int p) { return BFV_LD(src + p); }, [&](int p, u64 v) { BFV_ST(dst + p, v); });
}

// Inverse transform of evaluation-form {value, companion} arrays [limb][N]; limb x uses
// modulus x % nmod; output [limb][N] coefficients.
template <int LOGN>
LIMB_KERNEL(LOGN) k_intt_pairs(const ModTab *__restrict__ mods, int nmod, const shoup_t *__restrict__ in, u64 *out) {
    extern __shared__ u64 sm[];
    LIMB_INDEX(LOGN);
    const ModTab T = BFV_LD(mods + unit % nmod);
    const shoup_t *src = in + unit * N;
    u64 *dst = out + unit * N;
    limb_inverse<LOGN>(sm, T, h, [&](int p) { return BFV_LD(&src[p].x); }, [&](int p, u64 v) { BFV_ST(dst + p, v); });
}

// ------------------------------------------------------------------ encode / decode (mod t)
// A plaintext's slots are scattered to their evaluation positions (slot_pos) in shared
// memory -- each CTA keeps the positions it owns -- then inverse-transformed mod t.

// slots [count][N] -> plaintext [count][N].
template <int LOGN>
LIMB_KERNEL(LOGN) k_encode(const ModTab *__restrict__ mods, int tmod, const u32 *__restrict__ slot_pos,
                           const int64_t *slots, u64 *pt) {
    extern __shared__ u64 sm[];
    LIMB_INDEX(LOGN);
    const ModTab T = BFV_LD(mods + tmod);
    const int64_t *src = slots + unit * N;
    const int64_t t = (int64_t)T.q;
    for (int l = threadIdx.x; l < N; l += Split<LOGN>::NT) {
        const u32 pos = BFV_LD(slot_pos + l);
        if ((int)(pos / M) != h) continue;
        int64_t v = BFV_LD(src + l) % t;
        if (v < 0) v += t;
        sm[padi(pos % M)] = (u64)v;
    }
    __syncthreads();
    u64 *dst = pt + unit * N;
    limb_inverse<LOGN>(sm, T, h, [&](int p) { return sm[padi(p & (M - 1))]; }, [&](int p, u64 v) { BFV_ST(dst + p, v); });
}

// Packed features: plaintext (i, k) slot s = X[i][k N + s] (0 past f).
template <int LOGN>
LIMB_KERNEL(LOGN) k_encode_features(const ModTab *__restrict__ mods, int tmod, const u32 *__restrict__ slot_pos,
                                    const uint8_t *__restrict__ X, size_t f, int K, u64 *pt) {
    extern __shared__ u64 sm[];
    LIMB_INDEX(LOGN);
    const ModTab T = BFV_LD(mods + tmod);
    const size_t i = unit / K, k = unit % K;
    const uint8_t *row = X + i * f;
    for (int s = threadIdx.x; s < N; s += Split<LOGN>::NT) {
        const u32 pos = BFV_LD(slot_pos + s);
        if ((int)(pos / M) != h) continue;
        const size_t col = k * N + s;
        const u64 v = col < f ? (u64)BFV_LD(row + col) : 0;
        sm[padi(pos % M)] = v < T.q ? v : v % T.q;
    }
    __syncthreads();
    u64 *dst = pt + unit * N;
    limb_inverse<LOGN>(sm, T, h, [&](int p) { return sm[padi(p & (M - 1))]; }, [&](int p, u64 v) { BFV_ST(dst + p, v); });
}

// Feature columns: plaintext f' slot i = X[i][f'] for i < nX.
template <int LOGN>
LIMB_KERNEL(LOGN) k_encode_columns(const ModTab *__restrict__ mods, int tmod, const u32 *__restrict__ slot_pos,
                                   const uint8_t *__restrict__ X, size_t nX, size_t f, u64 *pt) {
    extern __shared__ u64 sm[];
    LIMB_INDEX(LOGN);
    const ModTab T = BFV_LD(mods + tmod);
    const size_t col = unit;
    for (int s = threadIdx.x; s < N; s += Split<LOGN>::NT) {
        const u32 pos = BFV_LD(slot_pos + s);
        if ((int)(pos / M) != h) continue;
        const u64 v = (size_t)s < nX ? (u64)BFV_LD(X + s * f + col) : 0;
        sm[padi(pos % M)] = v < T.q ? v : v % T.q;
    }
    __syncthreads();
    u64 *dst = pt + col * N;
    limb_inverse<LOGN>(sm, T, h, [&](int p) { return sm[padi(p & (M - 1))]; }, [&](int p, u64 v) { BFV_ST(dst + p, v); });
}

template <int LOGN>
LIMB_KERNEL(LOGN) k_decode(const ModTab *__restrict__ mods, int tmod, const u32 *__restrict__ slot_pos, const u64 *pt,
                           int64_t *slots) {
    extern __shared__ u64 sm[];
    LIMB_INDEX(LOGN);
    const ModTab T = BFV_LD(mods + tmod);
    const u64 *src = pt + unit * N;
    limb_forward<LOGN>(sm, T, h, [&](int p) { return BFV_LD(src + p); }, [&](int p, u64 v) { sm[padi(p & (M - 1))] = v; });
    __syncthreads();
    int64_t *dst = slots + unit * N;
    for (int l = threadIdx.x; l < N; l += Split<LOGN>::NT) {
        const u32 pos = BFV_LD(slot_pos + l);
        if ((int)(pos / M) == h) BFV_ST(dst + l, (int64_t)sm[padi(pos % M)]);
    }
}

// ------------------------------------------------------------------ key generation

__global__ void k_keygen_sk(u64 seed, int N, int8_t *sk) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    u32 w[16];
    chacha20_block(seed, (u32)k, kSkPurpose, 0, 0, w);
    BFV_ST(sk + k, (int8_t)ternary_of(w[0]));
}

// Evaluation form of s for every modulus of QP: out [nqp][N] {value, companion}.
template <int LOGN>
LIMB_KERNEL(LOGN) k_keygen_sk_eval(const ModTab *__restrict__ mods, const int8_t *__restrict__ sk, shoup_t *out) {
    extern __shared__ u64 sm[];
    LIMB_INDEX(LOGN);
    const ModTab T = BFV_LD(mods + unit);
    shoup_t *dst = out + unit * N;
    limb_forward<LOGN>(sm, T, h, [&](int p) { return lift_small(BFV_LD(sk + p), T.q); },
                       [&](int p, u64 v) { BFV_ST(dst + p, make_shoup(v, T.q)); });
}

// Public key limb l: pk1 = a (uniform), pk0 = -(a s + e); out [2][L][N] {value, companion}.
template <int LOGN>
LIMB_KERNEL(LOGN) k_keygen_pk(const ModTab *__restrict__ mods, const u64 *__restrict__ cdt, int cdt_len, u64 seed,
                              int L, const shoup_t *__restrict__ sk_eval, shoup_t *pk) {
    extern __shared__ u64 sm[];
    LIMB_INDEX(LOGN);
    const int l = (int)unit;
    const ModTab T = BFV_LD(mods + l);
    shoup_t *pk0 = pk + (size_t)l * N, *pk1 = pk + ((size_t)L + l) * N;
    const shoup_t *s = sk_eval + (size_t)l * N;
    limb_forward<LOGN>(
        sm, T, h,
        [&](int p) { u32 w[16]; chacha20_block(seed, (u32)p, kPkA, 0, (u32)l, w); return uniform_of(w, T); },
        [&](int p, u64 v) {
            BFV_ST(pk1 + p, make_shoup(v, T.q));
            BFV_ST(&pk0[p].x, red1(mul_shoup(v, BFV_LD(s + p), T.q), T.q));   // a s, finished below
        });
    __syncthreads();
    limb_forward<LOGN>(
        sm, T, h,
        [&](int p) { u32 w[16]; chacha20_block(seed, (u32)p, kPkE, 0, 0, w); return lift_small(gauss_of(w[0], w[1], w[2], cdt, cdt_len), T.q); },
        [&](int p, u64 v) { BFV_ST(pk0 + p, make_shoup(sub_mod(0, add_mod(BFV_LD(&pk0[p].x), v, T.q), T.q), T.q)); });
}

// Galois key (element gi, digit i, limb j of QP):
//   k1 = a, k0 = -a s + e + [i == j] [P]_{q_j} sigma_g(s); out [ng][L][2][nqp][N] {value, companion}.
template <int LOGN>
LIMB_KERNEL(LOGN) k_keygen_galois(const ModTab *__restrict__ mods, const u64 *__restrict__ cdt, int cdt_len, u64 seed,
                                  int L, const u64 *__restrict__ gal, const shoup_t *__restrict__ sk_eval, shoup_t *gk) {
    extern __shared__ u64 sm[];
    LIMB_INDEX(LOGN);
    const int nqp = L + 1;
    const int j = (int)(unit % nqp), i = (int)((unit / nqp) % L), gi = (int)(unit / ((size_t)nqp * L));
    const ModTab T = BFV_LD(mods + j);
    const u32 obj = (u32)gi * 256u + (u32)i;
    const u32 g = (u32)BFV_LD(gal + gi);
    shoup_t *k0 = gk + ((((size_t)gi * L + i) * 2 + 0) * nqp + j) * N;
    shoup_t *k1 = gk + ((((size_t)gi * L + i) * 2 + 1) * nqp + j) * N;
    const shoup_t *s = sk_eval + (size_t)j * N;
    limb_forward<LOGN>(
        sm, T, h,
        [&](int p) { u32 w[16]; chacha20_block(seed, (u32)p, kGkA, obj, (u32)j, w); return uniform_of(w, T); },
        [&](int p, u64 v) {
            BFV_ST(k1 + p, make_shoup(v, T.q));
            BFV_ST(&k0[p].x, red1(mul_shoup(v, BFV_LD(s + p), T.q), T.q));
        });
    __syncthreads();
    const u64 pmod = BFV_LD(&mods[L].q) % T.q;
    limb_forward<LOGN>(
        sm, T, h,
        [&](int p) { u32 w[16]; chacha20_block(seed, (u32)p, kGkE, obj, 0, w); return lift_small(gauss_of(w[0], w[1], w[2], cdt, cdt_len), T.q); },
        [&](int p, u64 v) {
            u64 r = sub_mod(v, BFV_LD(&k0[p].x), T.q);
            if (i == j) r = add_mod(r, mul_barrett(pmod, BFV_LD(&s[auto_src(p, g, LOGN)].x), T.q, T.mu, T.bits), T.q);
            BFV_ST(k0 + p, make_shoup(r, T.q));
        });
}

// ------------------------------------------------------------------ encryption

// Randomness of ciphertext c (object obj0 + c): u, e1, e2 per coefficient -> ws [count][3][N] int8.
__global__ void k_enc_sample(const u64 *__restrict__ cdt, int cdt_len, u64 seed, u32 obj0, int N, size_t total,
                             int8_t *ws) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const size_t c = idx / N;
    const int k = (int)(idx % N);
    u32 w[16];
    chacha20_block(seed, (u32)k, kEnc, obj0 + (u32)c, 0, w);
    int8_t *dst = ws + c * 3 * N;
    BFV_ST(dst + k, (int8_t)ternary_of(w[0]));
    BFV_ST(dst + N + k, (int8_t)gauss_of(w[1], w[2], w[3], cdt, cdt_len));
    BFV_ST(dst + 2 * N + k, (int8_t)gauss_of(w[4], w[5], w[6], cdt, cdt_len));
}

// Limb unit (c, l): both components of ciphertext c on limb l from one transform of u:
// comp 0 -> pk0 u + e1 + Delta m, comp 1 -> pk1 u + e2. The product pk1 u waits in comp 1's
// output limb (evaluation form) while comp 0 is inverted; the second inverse reads it in its
// first pass and overwrites it only in its last. With two CTAs per limb (MODE 1 at N = 16384,
// every N = 32768 limb) CTA h owns evaluation positions and coefficients [h M, (h+1) M): it
// writes and re-reads only its own half of comp 1's limb, and each inverse ends with a cluster
// barrier after the partner's last read of its shared memory.
template <int LOGN, int MODE>
LIMB_KERNEL_M(LOGN, MODE) k_enc_main(const ModTab *__restrict__ mods, int L, const shoup_t *__restrict__ pk,
                                     const int8_t *__restrict__ rnd, const u64 *__restrict__ pt, u64 *ct) {
    extern __shared__ u64 sm[];
    LIMB_INDEX_M(LOGN, MODE);
    const int l = (int)(unit % L);
    const size_t c = unit / L;
    const ModTab T = BFV_LD(mods + l);
    const int8_t *u = rnd + c * 3 * N, *e1 = u + N, *e2 = u + 2 * (size_t)N;
    const shoup_t *k0 = pk + (size_t)l * N, *k1 = pk + ((size_t)L + l) * N;
    const u64 *m = pt + c * N;
    u64 *out0 = ct + ((c * 2 + 0) * L + l) * (size_t)N, *out1 = ct + ((c * 2 + 1) * L + l) * (size_t)N;
    constexpr int NT = Split<LOGN, MODE>::NT;
    limb_forward<LOGN, true, MODE, MODE == 2>(sm, T, h, [&](int p) { return lift_small(BFV_LD(u + p), T.q); },
                                              [&](int p, u64 v) { sm[padi(p & (M - 1))] = v; });
    __syncthreads();
    // the public-key products in a pass of their own, four points per thread with their key loads
    // issued together: pk0 u stays in shared memory, pk1 u waits in comp 1's output limb
    static_assert(M % (4 * NT) == 0, "points per thread must be a multiple of 4");
#pragma unroll 1
    for (int p0 = threadIdx.x; p0 < M; p0 += 4 * NT) {
        shoup_t a[4], b[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            a[e] = BFV_LD(k0 + h * M + p0 + e * NT);
            b[e] = BFV_LD(k1 + h * M + p0 + e * NT);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int p = p0 + e * NT;
            const u64 v = sm[padi(p)];
            sm[padi(p)] = mul_shoup(v, a[e], T.q);
            BFV_ST(out1 + h * M + p, mul_shoup(v, b[e], T.q));
        }
    }
    __syncthreads();
    limb_inverse<LOGN, MODE>(sm, T, h, [&](int p) { return sm[padi(p & (M - 1))]; }, [&](int p, u64 v) {
        const u64 r = add_mod(v, lift_small(BFV_LD(e1 + p), T.q), T.q);
        // plaintext coefficients lie in [0, t) with t < q; reduce other words only when needed
        const u64 mv = BFV_LD(m + p), mr = mv < T.q ? mv : mv % T.q;
        BFV_ST(out0 + p, add_mod(r, red1(mul_shoup(mr, T.delta, T.deltap, T.q), T.q), T.q));
    });
    __syncthreads();
    limb_inverse<LOGN, MODE>(sm, T, h, [&](int p) { return BFV_LD(out1 + p); },
                             [&](int p, u64 v) { BFV_ST(out1 + p, add_mod(v, lift_small(BFV_LD(e2 + p), T.q), T.q)); });
}

// ------------------------------------------------------------------ decryption

// Limb unit (c, l): x_l = [c0 + c1 s]_{q_l} -> ws [count][L][N].
template <int LOGN>
LIMB_KERNEL(LOGN) k_dec_inner(const ModTab *__restrict__ mods, int L, const shoup_t *__restrict__ sk_eval,
                              const u64 *__restrict__ ct, u64 *x) {
    extern __shared__ u64 sm[];
    LIMB_INDEX(LOGN);
    const int l = (int)(unit % L);
    const size_t c = unit / L;
    const ModTab T = BFV_LD(mods + l);
    const u64 *c0 = ct + (c * 2 * L + l) * (size_t)N, *c1 = ct + ((c * 2 + 1) * L + l) * (size_t)N;
    const shoup_t *s = sk_eval + (size_t)l * N;
    limb_forward<LOGN, true>(sm, T, h, [&](int p) { return BFV_LD(c1 + p); },
                       [&](int p, u64 v) { sm[padi(p & (M - 1))] = mul_shoup(v, BFV_LD(s + p), T.q); });
    __syncthreads();
    u64 *dst = x + (c * L + l) * (size_t)N;
    limb_inverse<LOGN>(sm, T, h, [&](int p) { return sm[padi(p & (M - 1))]; },
                       [&](int p, u64 v) { BFV_ST(dst + p, add_mod(v, BFV_LD(c0 + p), T.q)); });
}

// Residues v_0..v_{L-1} (v_i < q_i, overwritten) -> the integer x in [0, Q) with x = v_i mod q_i
// as W 64-bit words: Garner's mixed-radix digits, then Horner's rule from the top digit.
__device__ __forceinline__ void crt_words(const ModTab *__restrict__ mods, const DecConst *__restrict__ dc,
                                          u64 (&v)[BFV_MAXP], u64 (&w)[BFV_MAXW]) {
    const int L = dc->L, W = dc->W;
    for (int i = 0; i < L; ++i) {
        const u64 qi = BFV_LD(&mods[i].q);
        u64 a = v[i];
        for (int j = 0; j < i; ++j) {
            a = sub_mod(a, red1(v[j], qi), qi);
            a = red1(mul_shoup(a, dc->inv[j][i], dc->invp[j][i], qi), qi);
        }
        v[i] = a;
    }
    for (int i = 0; i < W; ++i) w[i] = 0;
    w[0] = v[L - 1];
    for (int i = L - 2; i >= 0; --i) {            // w = w * q_i + v_i
        const u64 qi = BFV_LD(&mods[i].q);
        u64 carry = v[i];
        for (int n = 0; n < W; ++n) {
            const u64 lo = w[n] * qi, hi = __umul64hi(w[n], qi);
            const u64 s = lo + carry;
            carry = hi + (s < lo ? 1 : 0);
            w[n] = s;
        }
    }
}

// m = floor((t x + floor(Q/2)) / Q) mod t per coefficient, x = CRT(x_0..x_{L-1}) in [0, Q):
// Garner mixed-radix digits, Horner to a multi-word integer, binary long division.
__global__ void k_dec_round(const ModTab *__restrict__ mods, const DecConst *__restrict__ dc, const u64 *__restrict__ x,
                            int N, size_t total, u64 *pt) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const size_t c = idx / N;
    const int k = (int)(idx % N);
    if (!BFV_RANGE_OK(dc, sizeof(DecConst))) return;
    const int L = dc->L, W = dc->W;
    u64 v[BFV_MAXP];
    for (int i = 0; i < L; ++i) v[i] = BFV_LD(x + (c * L + i) * (size_t)N + k);
    u64 w[BFV_MAXW];
    crt_words(mods, dc, v, w);
    {                                             // w = w * t + floor(Q/2)
        u64 carry = 0;
        for (int n = 0; n < W; ++n) {
            const u64 lo = w[n] * dc->t, hi = __umul64hi(w[n], dc->t);
            u64 s = lo + carry;
            u64 c1 = hi + (s < lo ? 1 : 0);
            const u64 s2 = s + dc->qhalf[n];
            c1 += (s2 < s ? 1 : 0);
            w[n] = s2;
            carry = c1;
        }
    }
    u64 m = 0;
    for (int b = dc->tbits - 1; b >= 0; --b) {    // quotient bits, high to low
        const u64 *qs = dc->qshift[b];
        int cmp = 0;
        for (int n = W - 1; n >= 0 && cmp == 0; --n) cmp = (w[n] > qs[n]) - (w[n] < qs[n]);
        if (cmp >= 0) {
            u64 borrow = 0;
            for (int n = 0; n < W; ++n) {
                const u64 a = w[n], bq = qs[n];
                const u64 d = a - bq - borrow;
                borrow = (a < bq) || (a == bq && borrow) ? 1 : 0;
                w[n] = d;
            }
            m |= 1ull << b;
        }
    }
    BFV_ST(pt + idx, m % dc->t);
}

// Invariant noise of coefficient k of ciphertext c: z = [t x]_Q centred in (-Q/2, Q/2], x = [c0 +
// c1 s]_Q from k_dec_inner (t x = t Delta m + t e = t e - (Q mod t) m mod Q, so z / Q is the noise v
// of (t/Q)(c0 + c1 s) = m + v mod t). bits[c] = max over the ciphertext's coefficients of the bit
// length of |z| (bits[] zeroed by the caller).
__global__ void k_noise_bits(const ModTab *__restrict__ mods, const DecConst *__restrict__ dc,
                             const u64 *__restrict__ x, int N, size_t total, int *bits) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const size_t c = idx / N;
    const int k = (int)(idx % N);
    if (!BFV_RANGE_OK(dc, sizeof(DecConst))) return;
    const int L = dc->L, W = dc->W;
    u64 v[BFV_MAXP];
    for (int i = 0; i < L; ++i) {                  // [t x]_{q_i}; t < q_i
        const ModTab T = BFV_LD(mods + i);
        v[i] = mul_barrett(BFV_LD(x + (c * L + i) * (size_t)N + k), dc->t, T.q, T.mu, T.bits);
    }
    u64 w[BFV_MAXW];
    crt_words(mods, dc, v, w);                     // y = [t x]_Q in [0, Q)
    int cmp = 0;
    for (int n = W - 1; n >= 0 && cmp == 0; --n) cmp = (w[n] > dc->qhalf[n]) - (w[n] < dc->qhalf[n]);
    if (cmp > 0) {
        // y > floor(Q/2): |z| = Q - y = floor(Q/2) - d with d = y - floor(Q/2) - 1 (Q is odd)
        u64 borrow = 1;
        for (int n = 0; n < W; ++n) {             // w = y - floor(Q/2) - 1
            const u64 a = w[n], b = dc->qhalf[n];
            const u64 d = a - b - borrow;
            borrow = (a < b) || (a == b && borrow) ? 1 : 0;
            w[n] = d;
        }
        borrow = 0;
        for (int n = 0; n < W; ++n) {             // w = floor(Q/2) - w
            const u64 a = dc->qhalf[n], b = w[n];
            const u64 d = a - b - borrow;
            borrow = (a < b) || (a == b && borrow) ? 1 : 0;
            w[n] = d;
        }
    }
    int b = 0;
    for (int n = W - 1; n >= 0; --n)
        if (w[n]) { b = 64 * n + 64 - __clzll((long long)w[n]); break; }
    if (b && BFV_RANGE_OK(bits + c, sizeof(int))) atomicMax(bits + c, b);
}

// ------------------------------------------------------------------ model weights
// plaintext (j, k) mod t -> centred lift into q_l -> evaluation form; out [nY*K][L][N] {value, companion}.
template <int LOGN>
LIMB_KERNEL(LOGN) k_model_weights(const ModTab *__restrict__ mods, int L, int tmod, const u64 *__restrict__ pt,
                                  shoup_t *out) {
    extern __shared__ u64 sm[];
    LIMB_INDEX(LOGN);
    const int l = (int)(unit % L);
    const size_t jk = unit / L;
    const ModTab T = BFV_LD(mods + l);
    const u64 t = BFV_LD(&mods[tmod].q), th = (t - 1) / 2;
    const u64 *src = pt + jk * N;
    shoup_t *dst = out + (jk * L + l) * (size_t)N;
    limb_forward<LOGN>(sm, T, h, [&](int p) { const u64 v = BFV_LD(src + p); return v <= th ? v : T.q - (t - v); },
                       [&](int p, u64 v) { BFV_ST(dst + p, make_shoup(v, T.q)); });
}

// ------------------------------------------------------------------ dispatch helper

#define DISPATCH_LOGN(c, FN)          \
    switch ((c)->logN) {               \
        case 12: FN(12); break;        \
        case 13: FN(13); break;        \
        case 14: FN(14); break;        \
        case 15: FN(15); break;        \
        default: return BFV_ERR_BAD_PARAMS; \
    }

int last_err() { return cudaGetLastError() == cudaSuccess ? BFV_OK : BFV_ERR_CUDA; }

}  // namespace

#ifdef BFV_BOUNDS
BFV_BOUNDS_UPLOAD_FN(bounds_upload_scheme)
#endif

// ====================================================================== launchers

int launch_ntt_limbs(const bfv_ctx *c, const u64 *in, u64 *out, size_t nct, bool forward, cudaStream_t st) {
    ProfScope prof_(c, BFV_K_NTT, st);
    const size_t nl = nct * 2 * c->L;
    if (!nl) return BFV_OK;
#define L_(LG) launch_limbs<LG>(forward ? k_ntt_limbs<LG, true> : k_ntt_limbs<LG, false>, nl, st, 0, c->dmods, c->L, in, out)
    DISPATCH_LOGN(c, L_)
#undef L_
    count_launch(c);
    return last_err();
}

int launch_encode(const bfv_ctx *c, const int64_t *slots, size_t count, u64 *pt, cudaStream_t st) {
    ProfScope prof_(c, BFV_K_ENCODE, st);
#define L_(LG) launch_limbs<LG>(k_encode<LG>, count, st, 0, c->dmods, c->nqp, c->dslot, slots, pt)
    DISPATCH_LOGN(c, L_)
#undef L_
    count_launch(c);
    return last_err();
}

int launch_decode(const bfv_ctx *c, const u64 *pt, size_t count, int64_t *slots, cudaStream_t st) {
    ProfScope prof_(c, BFV_K_ENCODE, st);
#define L_(LG) launch_limbs<LG>(k_decode<LG>, count, st, 0, c->dmods, c->nqp, c->dslot, pt, slots)
    DISPATCH_LOGN(c, L_)
#undef L_
    count_launch(c);
    return last_err();
}

int launch_encode_features(const bfv_ctx *c, const uint8_t *X, size_t nX, size_t f, u64 *pt, cudaStream_t st) {
    ProfScope prof_(c, BFV_K_ENCODE, st);
    const int K = (int)((f + c->N - 1) / c->N);
#define L_(LG) launch_limbs<LG>(k_encode_features<LG>, nX * K, st, 0, c->dmods, c->nqp, c->dslot, X, f, K, pt)
    DISPATCH_LOGN(c, L_)
#undef L_
    count_launch(c);
    return last_err();
}

int launch_encode_columns(const bfv_ctx *c, const uint8_t *X, size_t nX, size_t f, u64 *pt, cudaStream_t st) {
    ProfScope prof_(c, BFV_K_ENCODE, st);
#define L_(LG) launch_limbs<LG>(k_encode_columns<LG>, f, st, 0, c->dmods, c->nqp, c->dslot, X, nX, f, pt)
    DISPATCH_LOGN(c, L_)
#undef L_
    count_launch(c);
    return last_err();
}

int launch_keygen(const bfv_ctx *c, bfv_keys *k, u64 seed, cudaStream_t st) {
    u64 *dgal = nullptr;
    if (cudaMalloc(&dgal, sizeof(u64) * c->galois.size()) != cudaSuccess) return BFV_ERR_OOM;
    if (cudaMemcpyAsync(dgal, c->galois.data(), sizeof(u64) * c->galois.size(), cudaMemcpyHostToDevice, st) !=
        cudaSuccess) {
        cudaFree(dgal);
        return BFV_ERR_CUDA;
    }
    {
        BoundsCall bc(c);
        bc.keys(k);
        bc.add(dgal, sizeof(u64) * c->galois.size());
        const int brc = bc.upload(st);
        if (brc) { cudaFree(dgal); return brc; }
    }
    k_keygen_sk<<<(c->N + 255) / 256, 256, 0, st>>>(seed, c->N, k->sk);
#define L_(LG)                                                                                                  \
    {                                                                                                           \
        launch_limbs<LG>(k_keygen_sk_eval<LG>, c->nqp, st, 0, c->dmods, (const int8_t *)k->sk, k->sk_eval);     \
        launch_limbs<LG>(k_keygen_pk<LG>, c->L, st, 0, c->dmods, (const u64 *)c->dcdt, c->cdt_len, seed, c->L,  \
                         (const shoup_t *)k->sk_eval, k->pk_eval);                                              \
        launch_limbs<LG>(k_keygen_galois<LG>, (size_t)k->ng * c->L * c->nqp, st, 0, c->dmods, (const u64 *)c->dcdt, \
                         c->cdt_len, seed, c->L, (const u64 *)dgal, (const shoup_t *)k->sk_eval, k->gk_eval);   \
    }
    int rc = BFV_OK;
    switch (c->logN) {
        case 12: L_(12); break;
        case 13: L_(13); break;
        case 14: L_(14); break;
        case 15: L_(15); break;
        default: rc = BFV_ERR_BAD_PARAMS;
    }
#undef L_
    count_launch(c, 4);
    if (!rc) rc = last_err();
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = BFV_ERR_CUDA;
    cudaFree(dgal);
    return rc;
}

int launch_keys_export(const bfv_ctx *c, const bfv_keys *k, int8_t *sk, u64 *pk, u64 *gk, cudaStream_t st) {
    if (sk && cudaMemcpyAsync(sk, k->sk, c->N, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return BFV_ERR_CUDA;
    const size_t npk = 2 * c->L, ngk = (size_t)k->ng * c->L * 2 * c->nqp;
#define L_(LG)                                                                                                     \
    {                                                                                                              \
        if (pk) { launch_limbs<LG>(k_intt_pairs<LG>, npk, st, 0, c->dmods, c->L, (const shoup_t *)k->pk_eval, pk); count_launch(c); } \
        if (gk) { launch_limbs<LG>(k_intt_pairs<LG>, ngk, st, 0, c->dmods, c->nqp, (const shoup_t *)k->gk_eval, gk); count_launch(c); } \
    }
    DISPATCH_LOGN(c, L_)
#undef L_
    return last_err();
}

int launch_encrypt(const bfv_ctx *c, const bfv_keys *k, const u64 *pt, size_t count, u64 seed, uint32_t obj0, u64 *ct,
                   void *ws, cudaStream_t st) {
    ProfScope prof_(c, BFV_K_ENCRYPT, st);
    int8_t *rnd = (int8_t *)ws;
    const size_t total = count * c->N;
    if (!total) return BFV_OK;
    k_enc_sample<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(c->dcdt, c->cdt_len, seed, obj0, c->N, total, rnd);
#define L_(LG) launch_limbs<LG>(k_enc_main<LG, 0>, count * c->L, st, 0, c->dmods, c->L, (const shoup_t *)k->pk_eval, \
                                (const int8_t *)rnd, pt, ct)
    if (c->logN == 14 && c->enc_split == 2)
        launch_limbs<14, 2>(k_enc_main<14, 2>, count * c->L, st, 0, c->dmods, c->L, (const shoup_t *)k->pk_eval,
                            (const int8_t *)rnd, pt, ct);
    else if (c->logN == 14 && c->enc_split == 3)
        launch_limbs<14, 1>(k_enc_main<14, 1>, count * c->L, st, 0, c->dmods, c->L, (const shoup_t *)k->pk_eval,
                            (const int8_t *)rnd, pt, ct);
    else
        DISPATCH_LOGN(c, L_)
#undef L_
    count_launch(c, 2);
    return last_err();
}

int launch_decrypt(const bfv_ctx *c, const bfv_keys *k, const u64 *ct, size_t count, u64 *pt, void *ws, cudaStream_t st) {
    ProfScope prof_(c, BFV_K_DECRYPT, st);
    u64 *x = (u64 *)ws;
    const size_t total = count * c->N;
    if (!total) return BFV_OK;
#define L_(LG) launch_limbs<LG>(k_dec_inner<LG>, count * c->L, st, 0, c->dmods, c->L, (const shoup_t *)k->sk_eval, ct, x)
    DISPATCH_LOGN(c, L_)
#undef L_
    k_dec_round<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(c->dmods, c->ddec, x, c->N, total, pt);
    count_launch(c, 2);
    return last_err();
}

int launch_noise_bits(const bfv_ctx *c, const bfv_keys *k, const u64 *ct, size_t count, u64 *x, int *bits,
                      cudaStream_t st) {
    const size_t total = count * c->N;
    if (!total) return BFV_OK;
    if (cudaMemsetAsync(bits, 0, count * sizeof(int), st) != cudaSuccess) return BFV_ERR_CUDA;
#define L_(LG) launch_limbs<LG>(k_dec_inner<LG>, count * c->L, st, 0, c->dmods, c->L, (const shoup_t *)k->sk_eval, ct, x)
    DISPATCH_LOGN(c, L_)
#undef L_
    k_noise_bits<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(c->dmods, c->ddec, x, c->N, total, bits);
    count_launch(c, 2);
    return last_err();
}

int launch_model_weights(const bfv_ctx *c, bfv_model *m, const u64 *w_pt, cudaStream_t st) {
    const size_t n = m->nY * m->K * c->L;
#define L_(LG) launch_limbs<LG>(k_model_weights<LG>, n, st, 0, c->dmods, c->L, c->nqp, w_pt, m->w_eval)
    DISPATCH_LOGN(c, L_)
#undef L_
    count_launch(c);
    return last_err();
}

// ====================================================================== CRT plaintext pair
//
// Section 4.2.2: scores that need more precision than one plaintext modulus are computed under
// two coprime moduli t0, t1 and recombined by the client. Garner's form:
// x = r0 + t0 ((r1 - r0) t0^-1 mod t1) in [0, t0 t1), returned centred in (-t0 t1 / 2, t0 t1 / 2].

namespace {

__global__ void k_crt_combine(const int64_t *__restrict__ r0, const int64_t *__restrict__ r1, u64 t0, u64 t1,
                              u64 inv, size_t n, int64_t *out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t s0 = (int64_t)t0, s1 = (int64_t)t1;
    const u64 a = (u64)(((BFV_LD(r0 + i) % s0) + s0) % s0), b = (u64)(((BFV_LD(r1 + i) % s1) + s1) % s1);
    const u64 d = (b + t1 - a % t1) % t1;               // (r1 - r0) mod t1
    const u64 x = a + t0 * ((d * inv) % t1);            // < t0 t1 < 2^62
    const u64 T = t0 * t1;
    BFV_ST(out + i, x > T / 2 ? (int64_t)x - (int64_t)T : (int64_t)x);
}

}  // namespace

int launch_crt_combine(const int64_t *r0, u64 t0, const int64_t *r1, u64 t1, u64 inv, size_t n, int64_t *out,
                       cudaStream_t st) {
    if (!n) return BFV_OK;
    k_crt_combine<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(r0, r1, t0, t1, inv, n, out);
    return cudaGetLastError() == cudaSuccess ? BFV_OK : BFV_ERR_CUDA;
}

// ====================================================================== allocation-free decryption
//
// bfv_decrypt_noalloc: decryption whose scratch (the per-limb residues [c0 + c1 s]_{q_l})
// lives in a fixed device array owned by this file instead of a caller workspace, for
// callers that must not call cudaMalloc at all. Host code cannot pass the array's symbol to a
// kernel (on the host it names a stand-in, not device memory): its device address is resolved
// with cudaGetSymbolAddress when a context is created (bfv_setup, the context's device current)
// and kept in the context, so a context made after a device reset resolves it afresh.

namespace {

constexpr size_t kNoAllocScratchBytes = 4u << 20;   // 4 MiB, held by every device that loads the library
static __device__ __align__(256) u64 g_noalloc_scratch[kNoAllocScratchBytes / sizeof(u64)];

}  // namespace

int noalloc_scratch_address(u64 **out, size_t *bytes) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return BFV_ERR_CUDA;
    *out = (u64 *)p;
    *bytes = kNoAllocScratchBytes;
    return BFV_OK;
}

extern "C" int bfv_decrypt_noalloc(bfv_ctx *ctx, const bfv_keys *keys, const uint64_t *ct, size_t count, uint64_t *pt,
                                   uintptr_t stream) {
    if (!ctx || !keys || keys->ctx != ctx) return BFV_ERR_INVALID_ARG;
    if (!count) return BFV_OK;
    if (!ct || !pt) return BFV_ERR_INVALID_ARG;
    if (count > kNoAllocScratchBytes / ((size_t)ctx->L * ctx->N * sizeof(u64))) return BFV_ERR_OVER_BUDGET;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return BFV_ERR_CUDA;
    if (dev != ctx->device) return BFV_ERR_INVALID_ARG;
    u64 *x = ctx->noalloc_scratch;
    if (!x) return BFV_ERR_CUDA;
    const bfv_ctx *c = ctx;
    cudaStream_t st = (cudaStream_t)stream;
    BoundsCall bc(c);
    bc.keys(keys);
    bc.io(ct, sizeof(u64) * count * 2 * c->L * c->N);
    bc.io(pt, sizeof(u64) * count * c->N);
    BFV_BOUNDS_UPLOAD(bc, st);
    ProfScope prof_(c, BFV_K_DECRYPT, st);
    // every scratch word k_dec_round reads is written by k_dec_inner in the same call
#define L_(LG) launch_limbs<LG>(k_dec_inner<LG>, count * c->L, st, 0, c->dmods, c->L, (const shoup_t *)keys->sk_eval, \
                                (const u64 *)ct, x)
    DISPATCH_LOGN(c, L_)
#undef L_
    const size_t total = count * c->N;
    k_dec_round<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(c->dmods, c->ddec, x, c->N, total, (u64 *)pt);
    count_launch(c, 2);
    return last_err();
}

extern "C" int bfv_decrypt_noalloc_max_count(const bfv_ctx *ctx, size_t *count) {
    if (!ctx || !count) return BFV_ERR_INVALID_ARG;
    *count = kNoAllocScratchBytes / ((size_t)ctx->L * ctx->N * sizeof(u64));
    return BFV_OK;
}
