/*
 * bfv_oracle.c -- plain, slow CPU reference for BFV-encrypted logistic-regression
 * scoring ("Scalable privacy-preserving cancer type prediction with homomorphic
 * encryption", Sections 4.2.2-4.2.3, Algorithm 1, Appendix).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load this library. It shares no code, header, table or constant
 * generator with the CUDA library; parameters (primes, roots, CRT constants, the
 * Gaussian table) are computed by oracle/__init__.py with Python integers and passed in.
 *
 * Every polynomial here is kept in coefficient form, with residues in [0, q).
 * Products are plain (unsigned __int128) a*b % q. Ring multiplication uses a
 * textbook negacyclic NTT (twist by psi^k, then a radix-2 Cooley-Tukey DFT with the
 * root psi^2), which the tests pin against schoolbook negacyclic convolution.
 * Pairs (i, j) are independent (Section 4.2.3), so loops over pairs may run on
 * several OpenMP threads; every pair's arithmetic is exact, so the result does not
 * depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

#define OC_MAXP 40

/* Parameter block filled by the Python side (field order mirrored there). */
typedef struct {
    int32_t N;               /* ring degree = number of slots */
    int32_t L;               /* number of ciphertext primes; the special prime is index L */
    uint64_t q[OC_MAXP];     /* q[0..L-1] ciphertext primes, q[L] = special prime P */
    uint64_t psi[OC_MAXP];   /* a primitive 2N-th root of unity mod q[i] */
    uint64_t t;              /* plaintext modulus */
    uint64_t omega;          /* slot-map root: primitive 2N-th root of unity mod t */
    uint64_t delta[OC_MAXP]; /* floor(Q / t) mod q[i], Q = q[0]...q[L-1] */
    uint64_t p_mod[OC_MAXP]; /* P mod q[i] */
    uint64_t p_inv[OC_MAXP]; /* P^-1 mod q[i] */
    uint64_t p_half;         /* floor(P / 2) */
    uint64_t cdt[32];        /* Gaussian magnitude thresholds (see sample_gauss) */
    int32_t cdt_len;
    int32_t nthreads;        /* OpenMP threads for loops over independent items */
} oc_params;

/* ------------------------------------------------------------------ modular */

static inline uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }
static inline uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) { uint64_t s = a + b; return s >= q ? s - q : s; }
static inline uint64_t submod(uint64_t a, uint64_t b, uint64_t q) { return a >= b ? a - b : a + q - b; }
static uint64_t powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) { if (e & 1) r = mulmod(r, a, q); a = mulmod(a, a, q); e >>= 1; }
    return r;
}
/* integer v (any sign) reduced into [0, q) */
static inline uint64_t lift_signed(int64_t v, uint64_t q) {
    if (v >= 0) return (uint64_t)v % q;
    uint64_t m = (uint64_t)(-(v + 1)) % q;   /* -v - 1 >= 0 */
    return q - 1 - m;
}
/* plaintext value v in [0, t) -> centred representative in (-t/2, t/2], reduced mod q */
static inline uint64_t lift_centred(uint64_t v, uint64_t t, uint64_t q) {
    int64_t c = (v <= (t - 1) / 2) ? (int64_t)v : (int64_t)v - (int64_t)t;
    return lift_signed(c, q);
}

/* ------------------------------------------------------------------ NTT */

/* In-place cyclic DFT of length N over Z_q with root omega (omega^N = 1):
 * a[m] <- sum_k a[k] omega^(m k). Iterative radix-2 Cooley-Tukey with bit reversal. */
static void cyclic_dft(uint64_t *a, int N, uint64_t q, uint64_t omega) {
    for (int i = 1, j = 0; i < N; i++) {
        int bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t tmp = a[i]; a[i] = a[j]; a[j] = tmp; }
    }
    uint64_t *pw = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(N / 2 > 0 ? N / 2 : 1));
    pw[0] = 1;
    for (int k = 1; k < N / 2; k++) pw[k] = mulmod(pw[k - 1], omega, q);
    for (int len = 2; len <= N; len <<= 1) {
        int half = len >> 1, stride = N / len;
        for (int i = 0; i < N; i += len)
            for (int j = 0; j < half; j++) {
                uint64_t u = a[i + j];
                uint64_t v = mulmod(a[i + j + half], pw[j * stride], q);
                a[i + j] = addmod(u, v, q);
                a[i + j + half] = submod(u, v, q);
            }
    }
    free(pw);
}

/* Negacyclic transform: a[m] <- a(psi^(2m+1)) = sum_k a[k] psi^k (psi^2)^(m k). */
void oc_ntt_forward(uint64_t *a, int N, uint64_t q, uint64_t psi) {
    uint64_t w = 1;
    for (int k = 0; k < N; k++) { a[k] = mulmod(a[k], w, q); w = mulmod(w, psi, q); }
    cyclic_dft(a, N, q, mulmod(psi, psi, q));
}

/* Inverse of oc_ntt_forward. */
void oc_ntt_inverse(uint64_t *a, int N, uint64_t q, uint64_t psi) {
    uint64_t psi_inv = powmod(psi, 2 * (uint64_t)N - 1, q);
    cyclic_dft(a, N, q, mulmod(psi_inv, psi_inv, q));
    uint64_t w = powmod((uint64_t)N, q - 2, q);   /* N^-1 */
    for (int k = 0; k < N; k++) { a[k] = mulmod(a[k], w, q); w = mulmod(w, psi_inv, q); }
}

/* out = a * b in Z_q[X]/(X^N + 1); out may alias a or b. */
void oc_polymul(const uint64_t *a, const uint64_t *b, uint64_t *out, int N, uint64_t q, uint64_t psi) {
    uint64_t *fa = (uint64_t *)malloc(sizeof(uint64_t) * N), *fb = (uint64_t *)malloc(sizeof(uint64_t) * N);
    memcpy(fa, a, sizeof(uint64_t) * N); memcpy(fb, b, sizeof(uint64_t) * N);
    oc_ntt_forward(fa, N, q, psi); oc_ntt_forward(fb, N, q, psi);
    for (int k = 0; k < N; k++) fa[k] = mulmod(fa[k], fb[k], q);
    oc_ntt_inverse(fa, N, q, psi);
    memcpy(out, fa, sizeof(uint64_t) * N);
    free(fa); free(fb);
}

/* ------------------------------------------------------------------ ChaCha20 (RFC 8439, Section 2.3) */

static inline uint32_t rotl32(uint32_t x, int n) { return (x << n) | (x >> (32 - n)); }
#define QR(a, b, c, d) do { \
    a += b; d ^= a; d = rotl32(d, 16); c += d; b ^= c; b = rotl32(b, 12); \
    a += b; d ^= a; d = rotl32(d, 8);  c += d; b ^= c; b = rotl32(b, 7); } while (0)

/* Quarter round on four words (RFC 8439 Section 2.1), exposed for its test vector. */
void oc_chacha_quarter(uint32_t *w) { QR(w[0], w[1], w[2], w[3]); }

/* ChaCha20 block function: 256-bit key (8 words), 32-bit block counter, 96-bit nonce (3 words). */
void oc_chacha20_block(const uint32_t key[8], uint32_t counter, const uint32_t nonce[3], uint32_t out[16]) {
    uint32_t s[16], x[16];
    s[0] = 0x61707865u; s[1] = 0x3320646eu; s[2] = 0x79622d32u; s[3] = 0x6b206574u;
    for (int i = 0; i < 8; i++) s[4 + i] = key[i];
    s[12] = counter; s[13] = nonce[0]; s[14] = nonce[1]; s[15] = nonce[2];
    memcpy(x, s, sizeof s);
    for (int r = 0; r < 10; r++) {
        QR(x[0], x[4], x[8], x[12]); QR(x[1], x[5], x[9], x[13]);
        QR(x[2], x[6], x[10], x[14]); QR(x[3], x[7], x[11], x[15]);
        QR(x[0], x[5], x[10], x[15]); QR(x[1], x[6], x[11], x[12]);
        QR(x[2], x[7], x[8], x[13]); QR(x[3], x[4], x[9], x[14]);
    }
    for (int i = 0; i < 16; i++) out[i] = x[i] + s[i];
}

/* Sampling purposes: the first nonce word. */
enum { P_SK = 1, P_PK_A = 2, P_PK_E = 3, P_GK_A = 4, P_GK_E = 5, P_ENC = 6 };

/* Draw block `k` for (seed, purpose, object, limb): key = 64-bit seed zero-extended. */
static void draw(uint64_t seed, uint32_t purpose, uint32_t obj, uint32_t limb, uint32_t k, uint32_t out[16]) {
    uint32_t key[8] = {(uint32_t)seed, (uint32_t)(seed >> 32), 0, 0, 0, 0, 0, 0};
    uint32_t nonce[3] = {purpose, obj, limb};
    oc_chacha20_block(key, k, nonce, out);
}
/* ternary value in {-1, 0, 1} from one word (Lemire's multiply-shift onto [0, 3)) */
static inline int ternary_from(uint32_t w) { return (int)(((uint64_t)w * 3u) >> 32) - 1; }
/* discrete Gaussian: magnitude = number of thresholds <= the 64-bit draw; sign bit negates */
static inline int gauss_from(const oc_params *p, uint32_t lo, uint32_t hi, uint32_t sgn) {
    uint64_t r = (uint64_t)lo | ((uint64_t)hi << 32);
    int mag = 0;
    for (int k = 0; k < p->cdt_len; k++) if (r >= p->cdt[k]) mag++;
    return (mag != 0 && (sgn & 1u)) ? -mag : mag;
}
/* uniform residue mod q from four words taken as a 128-bit integer */
static inline uint64_t uniform_from(const uint32_t *w, uint64_t q) {
    u128 r = (u128)w[0] | ((u128)w[1] << 32) | ((u128)w[2] << 64) | ((u128)w[3] << 96);
    return (uint64_t)(r % q);
}

/* Exported sampler views used by the tests. */
void oc_sample_ternary(uint64_t seed, uint32_t purpose, uint32_t obj, int N, int8_t *out) {
    uint32_t b[16];
    for (int k = 0; k < N; k++) { draw(seed, purpose, obj, 0, (uint32_t)k, b); out[k] = (int8_t)ternary_from(b[0]); }
}
void oc_sample_gauss(const oc_params *p, uint64_t seed, uint32_t purpose, uint32_t obj, int N, int8_t *out) {
    uint32_t b[16];
    for (int k = 0; k < N; k++) { draw(seed, purpose, obj, 0, (uint32_t)k, b); out[k] = (int8_t)gauss_from(p, b[0], b[1], b[2]); }
}

/* Encryption randomness of ciphertext `obj`: block k gives u_k (word 0), e1_k (words 1-3) and
 * e2_k (words 4-6). */
void oc_sample_enc(const oc_params *p, uint64_t seed, uint32_t obj, int8_t *u, int8_t *e1, int8_t *e2) {
    uint32_t b[16];
    for (int k = 0; k < p->N; k++) {
        draw(seed, P_ENC, obj, 0, (uint32_t)k, b);
        u[k] = (int8_t)ternary_from(b[0]);
        e1[k] = (int8_t)gauss_from(p, b[1], b[2], b[3]);
        e2[k] = (int8_t)gauss_from(p, b[4], b[5], b[6]);
    }
}

/* Uniform residues mod q[limb] for (seed, purpose, obj, limb), N values. */
void oc_sample_uniform(const oc_params *p, uint64_t seed, uint32_t purpose, uint32_t obj, uint32_t limb, uint64_t *out) {
    uint32_t b[16];
    for (int k = 0; k < p->N; k++) { draw(seed, purpose, obj, limb, (uint32_t)k, b); out[k] = uniform_from(b, p->q[limb]); }
}

/* ------------------------------------------------------------------ automorphism */

/* out(X) = a(X^g) in Z_q[X]/(X^N+1), g odd: coefficient k moves to k*g mod 2N, negated past N. */
void oc_automorph(const uint64_t *a, uint64_t *out, int N, uint64_t q, uint64_t g) {
    uint64_t twoN = 2 * (uint64_t)N;
    for (int k = 0; k < N; k++) {
        uint64_t d = ((uint64_t)k * g) % twoN;
        if (d < (uint64_t)N) out[d] = a[k];
        else out[d - N] = a[k] ? q - a[k] : 0;
    }
}

/* Galois elements of the rotate-and-sum, in the order applied: the row swap 2N-1,
 * then 3^(N/4), 3^(N/8), ..., 3^1 mod 2N (left row rotations by N/4, ..., 1). */
int oc_galois_elements(int N, uint64_t *out) {
    uint64_t twoN = 2 * (uint64_t)N;
    int n = 0;
    out[n++] = twoN - 1;
    for (int s = N / 4; s >= 1; s >>= 1) out[n++] = powmod(3, (uint64_t)s, twoN);
    return n;
}

/* ------------------------------------------------------------------ encode / decode */

/* Evaluation exponent of slot l: row r = l / (N/2), column c = l mod N/2,
 * e = 3^c mod 2N for row 0 and 2N - 3^c for row 1. */
static void slot_exponents(int N, uint64_t *e) {
    uint64_t twoN = 2 * (uint64_t)N, g = 1;
    for (int c = 0; c < N / 2; c++) { e[c] = g; e[c + N / 2] = twoN - g; g = (g * 3) % twoN; }
}

/* Batch encode: polynomial m (coefficients mod t) with m(omega^e_l) = v_l for every slot l. */
void oc_encode(const oc_params *p, const int64_t *v, uint64_t *m) {
    int N = p->N;
    uint64_t *e = (uint64_t *)malloc(sizeof(uint64_t) * N);
    slot_exponents(N, e);
    /* oc_ntt_forward index j holds the value at omega^(2j+1) */
    for (int l = 0; l < N; l++) m[(e[l] - 1) / 2] = lift_signed(v[l], p->t);
    oc_ntt_inverse(m, N, p->t, p->omega);
    free(e);
}

/* Batch decode: v_l = m(omega^e_l), in [0, t). */
void oc_decode(const oc_params *p, const uint64_t *m, int64_t *v) {
    int N = p->N;
    uint64_t *e = (uint64_t *)malloc(sizeof(uint64_t) * N), *f = (uint64_t *)malloc(sizeof(uint64_t) * N);
    slot_exponents(N, e);
    memcpy(f, m, sizeof(uint64_t) * N);
    oc_ntt_forward(f, N, p->t, p->omega);
    for (int l = 0; l < N; l++) v[l] = (int64_t)f[(e[l] - 1) / 2];
    free(e); free(f);
}

/* ------------------------------------------------------------------ keys */

/* Secret key s (ternary, N values). */
void oc_keygen_sk(const oc_params *p, uint64_t seed, int8_t *s) { oc_sample_ternary(seed, P_SK, 0, p->N, s); }

/* Public key pk = ([-(a s + e)]_Q, a), coefficient form, layout [2][L][N]. */
void oc_keygen_pk(const oc_params *p, uint64_t seed, const int8_t *s, uint64_t *pk) {
    int N = p->N, L = p->L;
    int8_t *e = (int8_t *)malloc(N);
    oc_sample_gauss(p, seed, P_PK_E, 0, N, e);
    uint64_t *ls = (uint64_t *)malloc(sizeof(uint64_t) * N);
    uint32_t b[16];
    for (int l = 0; l < L; l++) {
        uint64_t q = p->q[l], *pk0 = pk + (size_t)l * N, *pk1 = pk + (size_t)(L + l) * N;
        for (int k = 0; k < N; k++) { draw(seed, P_PK_A, 0, (uint32_t)l, (uint32_t)k, b); pk1[k] = uniform_from(b, q); }
        for (int k = 0; k < N; k++) ls[k] = lift_signed(s[k], q);
        oc_polymul(pk1, ls, pk0, N, q, p->psi[l]);
        for (int k = 0; k < N; k++) pk0[k] = submod(0, addmod(pk0[k], lift_signed(e[k], q), q), q);
    }
    free(e); free(ls);
}

/* Galois (key-switching) keys for the elements g[0..ng-1], coefficient form,
 * layout [ng][L digits][2][L+1 limbs][N]:
 *   k0[i][j] = -a_i s + e_i + (j == i ? [P]_{q_j} sigma_g(s) : 0),  k1[i][j] = a_i  (mod q_j over QP). */
void oc_keygen_galois(const oc_params *p, uint64_t seed, const int8_t *s, const uint64_t *gel, int ng, uint64_t *gk) {
    int N = p->N, L = p->L, nqp = L + 1;
    size_t limb = (size_t)N, per_digit = 2 * (size_t)nqp * limb, per_g = (size_t)L * per_digit;
#pragma omp parallel for schedule(dynamic) num_threads(p->nthreads > 0 ? p->nthreads : 1)
    for (int w = 0; w < ng * L; w++) {
        int gi = w / L, i = w % L;
        uint32_t obj = (uint32_t)gi * 256u + (uint32_t)i, b[16];
        int8_t *e = (int8_t *)malloc(N);
        uint64_t *ls = (uint64_t *)malloc(sizeof(uint64_t) * N), *sg = (uint64_t *)malloc(sizeof(uint64_t) * N);
        oc_sample_gauss(p, seed, P_GK_E, obj, N, e);
        for (int j = 0; j < nqp; j++) {
            uint64_t q = p->q[j];
            uint64_t *k0 = gk + gi * per_g + i * per_digit + (size_t)j * limb;
            uint64_t *k1 = gk + gi * per_g + i * per_digit + (size_t)(nqp + j) * limb;
            for (int k = 0; k < N; k++) { draw(seed, P_GK_A, obj, (uint32_t)j, (uint32_t)k, b); k1[k] = uniform_from(b, q); }
            for (int k = 0; k < N; k++) ls[k] = lift_signed(s[k], q);
            oc_polymul(k1, ls, k0, N, q, p->psi[j]);
            for (int k = 0; k < N; k++) k0[k] = submod(lift_signed(e[k], q), k0[k], q);
            if (j == i) {
                oc_automorph(ls, sg, N, q, gel[gi]);
                uint64_t pm = p->p_mod[j];
                for (int k = 0; k < N; k++) k0[k] = addmod(k0[k], mulmod(pm, sg[k], q), q);
            }
        }
        free(e); free(ls); free(sg);
    }
}

/* Forward-transform every limb of a Galois key block (layout as above) in place, so the
 * key switch can multiply pointwise. */
void oc_galois_to_eval(const oc_params *p, uint64_t *gk, int ng) {
    int N = p->N, L = p->L, nqp = L + 1;
    int nlimbs = ng * L * 2 * nqp;
#pragma omp parallel for schedule(dynamic) num_threads(p->nthreads > 0 ? p->nthreads : 1)
    for (int w = 0; w < nlimbs; w++) {
        int j = w % nqp;
        oc_ntt_forward(gk + (size_t)w * N, N, p->q[j], p->psi[j]);
    }
}

/* ------------------------------------------------------------------ encrypt / decrypt */

/* c = ([pk0 u + e1 + Delta m]_Q, [pk1 u + e2]_Q) for plaintext m (coefficients in [0, t)),
 * randomness from block k of (seed, P_ENC, obj): word 0 -> u, words 1-3 -> e1, words 4-6 -> e2. */
static void encrypt_one(const oc_params *p, const uint64_t *pk, const uint64_t *m, uint64_t seed, uint32_t obj, uint64_t *ct) {
    int N = p->N, L = p->L;
    int8_t *u = (int8_t *)malloc(N), *e1 = (int8_t *)malloc(N), *e2 = (int8_t *)malloc(N);
    oc_sample_enc(p, seed, obj, u, e1, e2);
    uint64_t *lu = (uint64_t *)malloc(sizeof(uint64_t) * N);
    for (int l = 0; l < L; l++) {
        uint64_t q = p->q[l];
        uint64_t *c0 = ct + (size_t)l * N, *c1 = ct + (size_t)(L + l) * N;
        for (int k = 0; k < N; k++) lu[k] = lift_signed(u[k], q);
        oc_polymul(pk + (size_t)l * N, lu, c0, N, q, p->psi[l]);
        oc_polymul(pk + (size_t)(L + l) * N, lu, c1, N, q, p->psi[l]);
        for (int k = 0; k < N; k++) {
            c0[k] = addmod(addmod(c0[k], lift_signed(e1[k], q), q), mulmod(p->delta[l], m[k] % q, q), q);
            c1[k] = addmod(c1[k], lift_signed(e2[k], q), q);
        }
    }
    free(u); free(e1); free(e2); free(lu);
}

/* Encrypt `count` plaintexts ([count][N]) into [count][2][L][N]; ciphertext c uses object id obj0 + c. */
void oc_encrypt(const oc_params *p, const uint64_t *pk, const uint64_t *m, int count, uint64_t seed, uint32_t obj0, uint64_t *ct) {
    size_t N = (size_t)p->N, ctsz = 2 * (size_t)p->L * N;
#pragma omp parallel for schedule(dynamic) num_threads(p->nthreads > 0 ? p->nthreads : 1)
    for (int c = 0; c < count; c++) encrypt_one(p, pk, m + (size_t)c * N, seed, obj0 + (uint32_t)c, ct + (size_t)c * ctsz);
}

/* x = [c0 + c1 s]_{q_l} per limb ([count][L][N]); the exact scale-and-round is done with
 * Python integers by the caller. */
void oc_decrypt_inner(const oc_params *p, const int8_t *s, const uint64_t *ct, int count, uint64_t *x) {
    int N = p->N, L = p->L;
    size_t ctsz = 2 * (size_t)L * N;
#pragma omp parallel for schedule(dynamic) num_threads(p->nthreads > 0 ? p->nthreads : 1)
    for (int w = 0; w < count * L; w++) {
        int c = w / L, l = w % L;
        uint64_t q = p->q[l];
        uint64_t *ls = (uint64_t *)malloc(sizeof(uint64_t) * N), *out = x + ((size_t)c * L + l) * N;
        for (int k = 0; k < N; k++) ls[k] = lift_signed(s[k], q);
        oc_polymul(ct + c * ctsz + (size_t)(L + l) * N, ls, out, N, q, p->psi[l]);
        const uint64_t *c0 = ct + c * ctsz + (size_t)l * N;
        for (int k = 0; k < N; k++) out[k] = addmod(out[k], c0[k], q);
        free(ls);
    }
}

/* ------------------------------------------------------------------ key switching and rotation */

/* ModDown: U over QP (coefficient form, [L+1][N]) -> round(U / P) over Q ([L][N]):
 * out[j] = (U[j] + floor(P/2) - r) * P^-1 mod q_j with r = [U[P] + floor(P/2)]_P,
 * i.e. floor((U + floor(P/2)) / P) for the integer U whose residues are the limbs. */
void oc_moddown(const oc_params *p, const uint64_t *U, uint64_t *out) {
    int N = p->N, L = p->L;
    size_t limb = (size_t)N;
    uint64_t P = p->q[L];
    for (int k = 0; k < N; k++) {
        uint64_t r = addmod(U[(size_t)L * limb + k], p->p_half, P);
        for (int j = 0; j < L; j++) {
            uint64_t q = p->q[j];
            uint64_t v = submod(addmod(U[(size_t)j * limb + k], p->p_half % q, q), r % q, q);
            out[(size_t)j * limb + k] = mulmod(v, p->p_inv[j], q);
        }
    }
}

/* Key switch of d (coefficient form over Q, [L][N]) with an evaluation-form Galois key block
 * gkg ([L digits][2][L+1][N]). Digits d_i = [d]_{q_i}; (U0, U1) = sum_i d_i * key_i over QP;
 * then ModDown: out_c[j] = (U_c[j] + floor(P/2) - r) * P^-1 mod q_j with r = [U_c[P] + floor(P/2)]_P. */
void oc_keyswitch(const oc_params *p, const uint64_t *gkg, const uint64_t *d, uint64_t *out0, uint64_t *out1) {
    int N = p->N, L = p->L, nqp = L + 1;
    size_t limb = (size_t)N, per_digit = 2 * (size_t)nqp * limb;
    uint64_t *U0 = (uint64_t *)malloc(sizeof(uint64_t) * nqp * limb), *U1 = (uint64_t *)malloc(sizeof(uint64_t) * nqp * limb);
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * limb);
    for (int j = 0; j < nqp; j++) {
        uint64_t q = p->q[j];
        uint64_t *a0 = U0 + j * limb, *a1 = U1 + j * limb;
        memset(a0, 0, sizeof(uint64_t) * limb); memset(a1, 0, sizeof(uint64_t) * limb);
        for (int i = 0; i < L; i++) {
            for (int k = 0; k < N; k++) tmp[k] = d[(size_t)i * limb + k] % q;
            oc_ntt_forward(tmp, N, q, p->psi[j]);
            const uint64_t *k0 = gkg + i * per_digit + (size_t)j * limb, *k1 = gkg + i * per_digit + (size_t)(nqp + j) * limb;
            for (int k = 0; k < N; k++) { a0[k] = addmod(a0[k], mulmod(tmp[k], k0[k], q), q); a1[k] = addmod(a1[k], mulmod(tmp[k], k1[k], q), q); }
        }
        oc_ntt_inverse(a0, N, q, p->psi[j]);
        oc_ntt_inverse(a1, N, q, p->psi[j]);
    }
    oc_moddown(p, U0, out0);
    oc_moddown(p, U1, out1);
    free(U0); free(U1); free(tmp);
}

/* rot_g(c) = ([sigma_g(c0) + u0]_Q, u1) with (u0, u1) = KS_g(sigma_g(c1)); ct layout [2][L][N]. */
void oc_rotate(const oc_params *p, const uint64_t *gkg, uint64_t g, const uint64_t *ct, uint64_t *out) {
    int N = p->N, L = p->L;
    size_t limb = (size_t)N;
    uint64_t *d = (uint64_t *)malloc(sizeof(uint64_t) * L * limb), *u0 = (uint64_t *)malloc(sizeof(uint64_t) * L * limb);
    for (int l = 0; l < L; l++) oc_automorph(ct + (size_t)(L + l) * limb, d + l * limb, N, p->q[l], g);
    oc_keyswitch(p, gkg, d, u0, out + (size_t)L * limb);
    for (int l = 0; l < L; l++) {
        uint64_t q = p->q[l];
        oc_automorph(ct + l * limb, out + l * limb, N, q, g);
        for (int k = 0; k < N; k++) out[l * limb + k] = addmod(out[l * limb + k], u0[l * limb + k], q);
    }
    free(d); free(u0);
}

/* ------------------------------------------------------------------ Algorithm 1 */

/* Ciphertext-plaintext product: each limb times the centred lift of plaintext m (mod t). */
void oc_mul_plain(const oc_params *p, const uint64_t *ct, const uint64_t *m, uint64_t *out) {
    int N = p->N, L = p->L;
    uint64_t *lm = (uint64_t *)malloc(sizeof(uint64_t) * N);
    for (int l = 0; l < L; l++) {
        uint64_t q = p->q[l];
        for (int k = 0; k < N; k++) lm[k] = lift_centred(m[k], p->t, q);
        oc_polymul(ct + (size_t)l * N, lm, out + (size_t)l * N, N, q, p->psi[l]);
        oc_polymul(ct + (size_t)(L + l) * N, lm, out + (size_t)(L + l) * N, N, q, p->psi[l]);
    }
    free(lm);
}

static void add_ct(const oc_params *p, uint64_t *acc, const uint64_t *x) {
    int N = p->N, L = p->L;
    for (int c = 0; c < 2; c++)
        for (int l = 0; l < L; l++) {
            uint64_t q = p->q[l];
            uint64_t *a = acc + ((size_t)c * L + l) * N;
            const uint64_t *b = x + ((size_t)c * L + l) * N;
            for (int k = 0; k < N; k++) a[k] = addmod(a[k], b[k], q);
        }
}

/* One pair (i, j) of Algorithm 1 up to the end of the rotate-and-accumulate loop:
 * c = sum_k X[i][k] * W[j][k], then c += rot_g(c) for each Galois element in order.
 * x: [K][2][L][N] input ciphertexts, w: [K][N] plaintexts mod t, gkg: evaluation-form keys
 * for the ng elements in gel. Result in out ([2][L][N]). */
void oc_pair_rotsum(const oc_params *p, const uint64_t *gkg, const uint64_t *gel, int ng,
                    const uint64_t *x, const uint64_t *w, int K, uint64_t *out) {
    int N = p->N, L = p->L, nqp = L + 1;
    size_t ctsz = 2 * (size_t)L * N, gsz = (size_t)L * 2 * nqp * N;
    uint64_t *tau = (uint64_t *)malloc(sizeof(uint64_t) * ctsz), *r = (uint64_t *)malloc(sizeof(uint64_t) * ctsz);
    memset(out, 0, sizeof(uint64_t) * ctsz);
    for (int k = 0; k < K; k++) {                 /* multiplication, then add_many */
        oc_mul_plain(p, x + k * ctsz, w + (size_t)k * N, tau);
        add_ct(p, out, tau);
    }
    for (int s = 0; s < ng; s++) {                /* rotate and accumulate */
        oc_rotate(p, gkg + s * gsz, gel[s], out, r);
        add_ct(p, out, r);
    }
    free(tau); free(r);
}

/* Bias and masking of one pair: c0 += Delta [b]_t (a constant polynomial), then c *= mask,
 * mask = the plaintext whose only non-zero slot is slot `slot` (value 1). */
void oc_pair_bias_mask(const oc_params *p, uint64_t *ct, uint64_t bias_t, int slot) {
    int N = p->N, L = p->L;
    for (int l = 0; l < L; l++) ct[(size_t)l * N] = addmod(ct[(size_t)l * N], mulmod(p->delta[l], bias_t % p->q[l], p->q[l]), p->q[l]);
    int64_t *v = (int64_t *)calloc(N, sizeof(int64_t));
    uint64_t *mask = (uint64_t *)malloc(sizeof(uint64_t) * N);
    v[slot] = 1;
    oc_encode(p, v, mask);
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * 2 * L * N);
    oc_mul_plain(p, ct, mask, tmp);
    memcpy(ct, tmp, sizeof(uint64_t) * 2 * L * N);
    free(v); free(mask); free(tmp);
}

/* Packed scores (Algorithm 1 with bias): X [nX][K][2][L][N] ciphertexts, Wp [nY][K][N] plaintexts,
 * bias_t [nY] values in [0, t). Pair g = i*nY + j lands in slot g mod N of output g / N.
 * Y: [ceil(nX*nY/N)][2][L][N]. pairs_out (optional, may be NULL): [nX*nY][2][L][N] masked pair
 * ciphertexts before compression. */
void oc_lr_packed(const oc_params *p, const uint64_t *gkg, const uint64_t *gel, int ng,
                  const uint64_t *X, int nX, const uint64_t *Wp, const uint64_t *bias_t, int nY, int K,
                  uint64_t *Y, uint64_t *pairs_out) {
    int N = p->N, L = p->L;
    size_t ctsz = 2 * (size_t)L * N;
    int npairs = nX * nY, nout = (npairs + N - 1) / N;
    uint64_t *R0 = pairs_out ? pairs_out : (uint64_t *)malloc(sizeof(uint64_t) * ctsz * (size_t)npairs);
#pragma omp parallel for schedule(dynamic) num_threads(p->nthreads > 0 ? p->nthreads : 1)
    for (int g = 0; g < npairs; g++) {
        int i = g / nY, j = g % nY;
        uint64_t *c = R0 + (size_t)g * ctsz;
        oc_pair_rotsum(p, gkg, gel, ng, X + (size_t)i * K * ctsz, Wp + (size_t)j * K * N, K, c);
        oc_pair_bias_mask(p, c, bias_t[j], g % N);
    }
    memset(Y, 0, sizeof(uint64_t) * ctsz * (size_t)nout);    /* compression */
    for (int g = 0; g < npairs; g++) add_ct(p, Y + (size_t)(g / N) * ctsz, R0 + (size_t)g * ctsz);
    if (!pairs_out) free(R0);
}

/* Standard (per-element) scores: slot i of X[f] holds feature f of individual i; output j is
 * sum_f w[f][j] * X[f] + Delta [b_j]_t, the integer weight lifted into each q_l.
 * X [nF][2][L][N], W [nF][nY] row-major, Y [nY][2][L][N]. */
void oc_lr_standard(const oc_params *p, const uint64_t *X, int nF, const int64_t *W, const uint64_t *bias_t, int nY, uint64_t *Y) {
    int N = p->N, L = p->L;
    size_t ctsz = 2 * (size_t)L * N;
#pragma omp parallel for schedule(static) num_threads(p->nthreads > 0 ? p->nthreads : 1)
    for (int j = 0; j < nY; j++) {
        uint64_t *y = Y + (size_t)j * ctsz;
        memset(y, 0, sizeof(uint64_t) * ctsz);
        for (int f = 0; f < nF; f++)
            for (int c = 0; c < 2; c++)
                for (int l = 0; l < L; l++) {
                    uint64_t q = p->q[l], w = lift_signed(W[(size_t)f * nY + j], q);
                    const uint64_t *x = X + (size_t)f * ctsz + ((size_t)c * L + l) * N;
                    uint64_t *a = y + ((size_t)c * L + l) * N;
                    for (int k = 0; k < N; k++) a[k] = addmod(a[k], mulmod(w, x[k], q), q);
                }
        for (int l = 0; l < L; l++) y[(size_t)l * N] = addmod(y[(size_t)l * N], mulmod(p->delta[l], bias_t[j] % p->q[l], p->q[l]), p->q[l]);
    }
}

/* One output coefficient of the standard product from its inputs: sum_f w[f] * x[f] mod q. */
uint64_t oc_standard_coeff(const int64_t *w, const uint64_t *x, int nF, uint64_t q) {
    uint64_t a = 0;
    for (int f = 0; f < nF; f++) a = addmod(a, mulmod(lift_signed(w[f], q), x[f], q), q);
    return a;
}

/* Schoolbook negacyclic product (the definition), for pinning the NTT at small N. */
void oc_polymul_schoolbook(const uint64_t *a, const uint64_t *b, uint64_t *out, int N, uint64_t q) {
    for (int k = 0; k < N; k++) out[k] = 0;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            uint64_t v = mulmod(a[i], b[j], q);
            int d = i + j;
            if (d < N) out[d] = addmod(out[d], v, q);
            else out[d - N] = submod(out[d - N], v, q);
        }
}

int oc_abi_version(void) { return 1; }
int oc_max_primes(void) { return OC_MAXP; }
int oc_has_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
