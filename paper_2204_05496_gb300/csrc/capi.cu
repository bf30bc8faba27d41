// capi.cu -- C ABI entry points and host-side precomputation (primes, NTT tables,
// CRT/rounding constants, Gaussian thresholds). Kernels live in k_*.cu.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "bfv_internal.h"

typedef unsigned __int128 u128;

namespace {

// ------------------------------------------------------------------ number theory (host)

u64 mulmod_h(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
u64 powmod_h(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod_h(r, a, q);
        a = mulmod_h(a, a, q);
        e >>= 1;
    }
    return r;
}
u64 inv_h(u64 a, u64 q) { return powmod_h(a, q - 2, q); }  // q prime

// Deterministic Miller-Rabin for 64-bit n (bases 2..37 are exact below 3.3e24).
bool is_prime_h(u64 n) {
    static const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 b : bases)
        if (n % b == 0) return n == b;
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (u64 a : bases) {
        u64 x = powmod_h(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < s; ++i) {
            x = mulmod_h(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

int ilog2_h(u64 n) { int l = 0; while ((1ull << l) < n) ++l; return l; }
u64 brev_h(u64 x, int bits) {
    u64 r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1ull) << (bits - 1 - i);
    return r;
}
u64 shoup_h(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

// Primes below 2^bits that are 1 mod 2N, descending.
bool ntt_primes_h(int bits, u64 N, int count, std::vector<u64> &out) {
    out.clear();
    const u64 m = 2 * N;
    u64 q = (1ull << bits) - m + 1;
    while ((int)out.size() < count) {
        if (q < (1ull << (bits - 1))) return false;
        if (is_prime_h(q)) out.push_back(q);
        q -= m;
    }
    return true;
}

// A primitive 2N-th root of unity mod q: x^((q-1)/2N) for the first x >= 2 whose N-th power is -1.
u64 root_2n_h(u64 q, u64 N) {
    for (u64 x = 2;; ++x) {
        u64 r = powmod_h(x, (q - 1) / (2 * N), q);
        if (powmod_h(r, N, q) == q - 1) return r;
    }
}

// Smallest primitive root modulo the prime p.
u64 smallest_primitive_root_h(u64 p) {
    std::vector<u64> fs;
    u64 n = p - 1;
    for (u64 d = 2; d * d <= n; ++d)
        if (n % d == 0) { fs.push_back(d); while (n % d == 0) n /= d; }
    if (n > 1) fs.push_back(n);
    for (u64 g = 2;; ++g) {
        bool ok = true;
        for (u64 f : fs)
            if (powmod_h(g, (p - 1) / f, p) == 1) { ok = false; break; }
        if (ok) return g;
    }
}

// ------------------------------------------------------------------ multi-word integers (little-endian)

typedef std::vector<u64> MW;
void mw_mul_small(MW &a, u64 m) {
    u64 carry = 0;
    for (auto &w : a) {
        u128 v = (u128)w * m + carry;
        w = (u64)v;
        carry = (u64)(v >> 64);
    }
    if (carry) a.push_back(carry);
}
u64 mw_divmod_small(MW &a, u64 d) {  // a <- floor(a / d), returns remainder
    u128 rem = 0;
    for (int i = (int)a.size() - 1; i >= 0; --i) {
        u128 cur = (rem << 64) | a[i];
        a[i] = (u64)(cur / d);
        rem = cur % d;
    }
    while (a.size() > 1 && a.back() == 0) a.pop_back();
    return (u64)rem;
}
int mw_bits(const MW &a) {   // bit length
    for (size_t n = a.size(); n-- > 0;)
        if (a[n]) {
            int b = 0;
            for (u64 x = a[n]; x; x >>= 1) ++b;
            return (int)(64 * n) + b;
        }
    return 0;
}
u64 mw_mod_small(const MW &a, u64 d) {
    u128 rem = 0;
    for (int i = (int)a.size() - 1; i >= 0; --i) rem = ((rem << 64) | a[i]) % d;
    return (u64)rem;
}

// ------------------------------------------------------------------ Gaussian thresholds
// exp(-k^2 / (2 sigma^2)), sigma = num/den, in 120-bit binary fixed point with exact integer
// arithmetic: base = exp(-1 / (2 num^2)) by its Taylor series, raised to (k den)^2 by squaring.

const int FB = 120;
u128 fx_mul(u128 a, u128 b) {  // (a * b) >> FB, a, b < 2^124
    u64 a0 = (u64)a, a1 = (u64)(a >> 64), b0 = (u64)b, b1 = (u64)(b >> 64);
    u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
    // 256-bit sum: p11 << 128 + (p01 + p10) << 64 + p00
    u128 mid = p01 + p10;  // < 2^125, no overflow for our operand sizes
    u128 lo = p00 + (mid << 64);
    u128 carry = (lo < p00) ? 1 : 0;
    u128 hi = p11 + (mid >> 64) + carry;
    // shift right by FB = 120: result = hi << 8 | lo >> 120
    return (hi << (128 - FB)) | (lo >> FB);
}
u128 fx_pow(u128 b, u64 e) {
    u128 r = (u128)1 << FB;
    while (e) {
        if (e & 1) r = fx_mul(r, b);
        b = fx_mul(b, b);
        e >>= 1;
    }
    return r;
}
int gaussian_table_h(uint32_t num, uint32_t den, u64 *out) {
    if (num == 0 || den == 0) return -1;
    const int tail = (int)(6ull * num / den);
    if (tail < 1 || tail > 32) return -1;
    // base = exp(-x), x = 1 / (2 num^2): alternating series, positive and negative parts apart
    const u64 d = 2ull * num * num;
    u128 term = (u128)1 << FB, pos = term, neg = 0;
    for (int n = 1; n < 40 && term; ++n) {
        term = term / d / (u64)n;
        if (n & 1) neg += term; else pos += term;
    }
    const u128 base = pos - neg;
    std::vector<u128> rho(tail + 1);
    for (int k = 0; k <= tail; ++k) rho[k] = fx_pow(base, (u64)k * k * den * den);
    u128 Z = rho[0];
    for (int k = 1; k <= tail; ++k) Z += 2 * rho[k];
    u128 cum = 0;
    for (int k = 0; k < tail; ++k) {
        cum += (k == 0) ? rho[0] : 2 * rho[k];
        // floor(2^64 cum / Z) by binary long division
        u128 rem = cum;
        u64 q = 0;
        for (int i = 0; i < 64; ++i) {
            rem <<= 1;
            q <<= 1;
            if (rem >= Z) { rem -= Z; q |= 1; }
        }
        out[k] = q;
    }
    return tail;
}

// IEEE binary16 bits of an integer of magnitude below 2048 (exact: 11 significant bits).
uint16_t f16_of_small(int64_t v) {
    if (v == 0) return 0;
    const uint16_t sign = v < 0 ? 0x8000 : 0;
    uint32_t a = (uint32_t)(v < 0 ? -v : v);
    int e = 0;
    while ((a >> (e + 1)) != 0) ++e;                  // a in [2^e, 2^(e+1))
    const uint32_t mant = (a << (10 - e)) & 0x3FFu;   // the 10 bits below the leading one
    return (uint16_t)(sign | (uint32_t)(e + 15) << 10 | mant);
}

bool params_ok(const bfv_params *p) {
    if (!p) return false;
    if (p->N != 4096 && p->N != 8192 && p->N != 16384 && p->N != 32768) return false;
    if (p->L < 1 || p->L > BFV_MAXP - 1) return false;
    if (p->prime_bits < 30 || p->prime_bits > 59) return false;   // lazy transforms stay below 32q < 2^64
    if (p->t < 3 || p->t >= (1ull << 31) || (p->t - 1) % (2ull * p->N) != 0 || !is_prime_h(p->t)) return false;
    if (p->sigma_num == 0 || p->sigma_den == 0) return false;
    return true;
}

template <class T> int dalloc(T **p, size_t n) {
    if (cudaMalloc((void **)p, sizeof(T) * (n ? n : 1)) != cudaSuccess) { *p = nullptr; return BFV_ERR_OOM; }
    return BFV_OK;
}

void free_ctx(bfv_ctx *c) {
    if (!c) return;
    for (auto &v : c->prof.pending)
        for (auto &pr : v) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (auto e : c->prof.pool) cudaEventDestroy(e);
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second.first);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    cudaFree(c->dmods);
    cudaFree(c->dtw);
    cudaFree(c->dslot);
    cudaFree(c->dmaskpow);
    cudaFree(c->dmaskev);
    cudaFree(c->dcdt);
    cudaFree(c->ddec);
    cudaFree(c->derr);
    delete c;
}

cudaStream_t S(uintptr_t s) { return (cudaStream_t)s; }

}  // namespace

// The buffers a packed product's launches may touch: keys, models, each request's inputs and
// outputs at the sizes the call implies, the workspace (bounds-checked build only).
static void bounds_packed(BoundsCall &bc, const bfv_ctx *ctx, const bfv_keys *keys, int nreq,
                          const bfv_model *const *models, const uint64_t *const *X, const size_t *nXs,
                          uint64_t *const *Y, const void *ws, size_t ws_bytes) {
    const size_t ctb = sizeof(u64) * 2 * ctx->L * ctx->N;
    bc.keys(keys);
    for (int r = 0; r < nreq; ++r) {
        bool seen = false;
        for (int q = 0; q < r && !seen; ++q) seen = models[q] == models[r];
        if (!seen) bc.model(models[r]);
        bc.io(X[r], nXs[r] * models[r]->K * ctb);
        bc.io(Y[r], (nXs[r] * models[r]->nY + ctx->N - 1) / ctx->N * ctb);
    }
    bc.io(ws, ws_bytes);
}

// ====================================================================== C ABI

extern "C" {

int bfv_abi_version(void) { return 1; }

int bfv_params_primes(const bfv_params *p, uint64_t *primes_out) {
    if (!params_ok(p) || !primes_out) return BFV_ERR_INVALID_ARG;
    std::vector<u64> ps;
    if (!ntt_primes_h((int)p->prime_bits, p->N, (int)p->L + 1, ps)) return BFV_ERR_BAD_PARAMS;
    std::copy(ps.begin(), ps.end(), primes_out);
    return BFV_OK;
}

int bfv_gaussian_table(uint32_t sigma_num, uint32_t sigma_den, uint64_t *out, int *len) {
    if (!out || !len) return BFV_ERR_INVALID_ARG;
    int n = gaussian_table_h(sigma_num, sigma_den, (u64 *)out);
    if (n < 0) return BFV_ERR_BAD_PARAMS;
    *len = n;
    return BFV_OK;
}

int bfv_setup(const bfv_params *p, bfv_ctx **out) {
    if (!out) return BFV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params_ok(p)) return BFV_ERR_BAD_PARAMS;
    bfv_ctx *c = new (std::nothrow) bfv_ctx();
    if (!c) return BFV_ERR_OOM;
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return BFV_ERR_CUDA; }
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) { delete c; return BFV_ERR_CUDA; }
    c->N = (int)p->N;
    c->logN = ilog2_h(p->N);
    c->L = (int)p->L;
    c->nqp = c->L + 1;
    c->bits = (int)p->prime_bits;
    c->t = p->t;
    c->sigma_num = p->sigma_num;
    c->sigma_den = p->sigma_den;
    if (!ntt_primes_h(c->bits, p->N, c->nqp, c->primes)) { delete c; return BFV_ERR_BAD_PARAMS; }
    const u64 N = (u64)c->N;
    const int nmod = c->nqp + 1;
    const u64 P = c->primes[c->L];

    // Q, floor(Q/t), floor(Q/2) as multi-word integers
    MW Q{1};
    for (int l = 0; l < c->L; ++l) mw_mul_small(Q, c->primes[l]);
    c->qbits = mw_bits(Q);
    MW Qdt = Q;
    mw_divmod_small(Qdt, c->t);

    // twiddles and per-modulus constants
    std::vector<u64> tw((size_t)nmod * 6 * N);
    c->hmods.assign(nmod, ModTab{});
    c->delta_host.assign(c->L, 0);
    int rc = dalloc(&c->dtw, tw.size());
    if (rc) { free_ctx(c); return rc; }
    for (int j = 0; j < nmod; ++j) {
        const u64 q = (j < c->nqp) ? c->primes[j] : c->t;
        u64 psi;
        if (j < c->nqp) {
            psi = root_2n_h(q, N);
        } else {
            psi = powmod_h(smallest_primitive_root_h(q), (q - 1) / (2 * N), q);
            c->omega = psi;
        }
        const u64 psii = inv_h(psi, q);
        // [j][fw pairs (2N words)][dt pairs (2N words)][tw pairs (2N words)], each pair {w, w'}:
        // fw[k] = psi^brev(k); dt[h + j] = omega^-(j N / 2h) = psi^-(j N / h) for h = 2^s, j < h;
        // tw[k] = N^-1 psi^-k
        u64 *fwv = &tw[(size_t)j * 6 * N], *dtv = fwv + 2 * N, *twv = fwv + 4 * N;
        std::vector<u64> pw(N), ipw(N);
        pw[0] = ipw[0] = 1;
        for (u64 i = 1; i < N; ++i) { pw[i] = mulmod_h(pw[i - 1], psi, q); ipw[i] = mulmod_h(ipw[i - 1], psii, q); }
        const u64 ninv = inv_h(N % q, q);
        dtv[0] = 1; dtv[1] = shoup_h(1, q);   // unused
        for (u64 h = 1; h < N; h <<= 1)
            for (u64 i = 0; i < h; ++i) {
                const u64 w = ipw[i * (N / h)];
                dtv[2 * (h + i)] = w; dtv[2 * (h + i) + 1] = shoup_h(w, q);
            }
        for (u64 k = 0; k < N; ++k) {
            const u64 b = brev_h(k, c->logN);
            fwv[2 * k] = pw[b]; fwv[2 * k + 1] = shoup_h(pw[b], q);
            const u64 t = mulmod_h(ninv, ipw[k], q);
            twv[2 * k] = t; twv[2 * k + 1] = shoup_h(t, q);
        }
        ModTab &T = c->hmods[j];
        T.q = q;
        T.q2 = 2 * q;
        T.ninv = ninv;
        T.ninvp = shoup_h(T.ninv, q);
        T.bits = ilog2_h(q + 1);
        T.mu = (u64)(((u128)1 << (2 * T.bits)) / q);
        if (j < c->L) {
            T.pinv = inv_h(P % q, q);
            T.pinvp = shoup_h(T.pinv, q);
            T.pmod = P % q;
            T.pmodp = shoup_h(T.pmod, q);
            T.phalf = (P / 2) % q;
            T.delta = mw_mod_small(Qdt, q);
            T.deltap = shoup_h(T.delta, q);
            c->delta_host[j] = T.delta;
        } else if (j == c->L) {
            T.phalf = P / 2;
        }
        T.r64 = (u64)(((u128)1 << 64) % q);
        T.r64p = shoup_h(T.r64, q);
        T.onep = shoup_h(1, q);
        const u64 *base = c->dtw + (size_t)j * 6 * N;
        T.fw = (const ulonglong2 *)base;
        T.dt = (const ulonglong2 *)(base + 2 * N);
        T.tw = (const ulonglong2 *)(base + 4 * N);
    }
    if (cudaMemcpy(c->dtw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) { free_ctx(c); return BFV_ERR_CUDA; }
    if ((rc = dalloc(&c->dmods, nmod))) { free_ctx(c); return rc; }
    if (cudaMemcpy(c->dmods, c->hmods.data(), sizeof(ModTab) * nmod, cudaMemcpyHostToDevice) != cudaSuccess) { free_ctx(c); return BFV_ERR_CUDA; }

    // slot map: slot l at exponent e_l (3^c or 2N - 3^c), evaluation position brev((e_l - 1)/2)
    std::vector<u32> slot(N);
    {
        u64 g = 1;
        for (u64 cc = 0; cc < N / 2; ++cc) {
            slot[cc] = (u32)brev_h((g - 1) / 2, c->logN);
            slot[cc + N / 2] = (u32)brev_h((2 * N - g - 1) / 2, c->logN);
            g = g * 3 % (2 * N);
        }
    }
    if ((rc = dalloc(&c->dslot, N))) { free_ctx(c); return rc; }
    if (cudaMemcpy(c->dslot, slot.data(), N * 4, cudaMemcpyHostToDevice) != cudaSuccess) { free_ctx(c); return BFV_ERR_CUDA; }
    // N^-1 omega^i mod t, i < 2N (one-hot mask coefficients)
    std::vector<u32> mp(2 * N);
    {
        const u64 ninvt = inv_h(N % c->t, c->t);
        u64 w = ninvt;
        for (u64 i = 0; i < 2 * N; ++i) { mp[i] = (u32)w; w = mulmod_h(w, c->omega, c->t); }
    }
    if ((rc = dalloc(&c->dmaskpow, 2 * N))) { free_ctx(c); return rc; }
    if (cudaMemcpy(c->dmaskpow, mp.data(), 2 * N * 4, cudaMemcpyHostToDevice) != cudaSuccess) { free_ctx(c); return BFV_ERR_CUDA; }

    // Gaussian thresholds
    u64 cdt[32];
    c->cdt_len = gaussian_table_h(c->sigma_num, c->sigma_den, cdt);
    if (c->cdt_len < 0) { free_ctx(c); return BFV_ERR_BAD_PARAMS; }
    if ((rc = dalloc(&c->dcdt, 32))) { free_ctx(c); return rc; }
    if (cudaMemcpy(c->dcdt, cdt, 32 * 8, cudaMemcpyHostToDevice) != cudaSuccess) { free_ctx(c); return BFV_ERR_CUDA; }

    // decryption constants
    DecConst dc;
    std::memset(&dc, 0, sizeof dc);
    dc.L = c->L;
    dc.t = c->t;
    dc.tbits = ilog2_h(c->t + 1);
    for (int i = 0; i < c->L; ++i)
        for (int j = i + 1; j < c->L; ++j) {
            dc.inv[i][j] = inv_h(c->primes[i] % c->primes[j], c->primes[j]);
            dc.invp[i][j] = shoup_h(dc.inv[i][j], c->primes[j]);
        }
    MW tq = Q;
    mw_mul_small(tq, c->t);
    dc.W = (int)tq.size() + 1;
    if (dc.W > BFV_MAXW) { free_ctx(c); return BFV_ERR_BAD_PARAMS; }
    MW qh = Q;
    mw_divmod_small(qh, 2);
    for (size_t i = 0; i < qh.size(); ++i) dc.qhalf[i] = qh[i];
    for (int b = 0; b < dc.tbits; ++b) {
        MW s = Q;
        mw_mul_small(s, 1ull << b);
        for (size_t i = 0; i < s.size() && (int)i < BFV_MAXW; ++i) dc.qshift[b][i] = s[i];
    }
    if ((rc = dalloc(&c->ddec, 1))) { free_ctx(c); return rc; }
    if ((rc = dalloc(&c->derr, 1))) { free_ctx(c); return rc; }
    if (cudaMemset(c->derr, 0, sizeof(int)) != cudaSuccess ||
        cudaMemcpy(c->ddec, &dc, sizeof dc, cudaMemcpyHostToDevice) != cudaSuccess) {
        free_ctx(c);
        return BFV_ERR_CUDA;
    }

    // rotate-and-sum Galois elements: 2N-1, then 3^(N/4), ..., 3^1 mod 2N
    c->galois.push_back(2 * N - 1);
    for (u64 s = N / 4; s >= 1; s >>= 1) c->galois.push_back(powmod_h(3, s, 2 * N));

    // evaluation form of the slot-0 one-hot mask: the packed product gathers every slot's mask from it
    if ((rc = dalloc(&c->dmaskev, (size_t)c->L * N))) { free_ctx(c); return rc; }
    {
        BoundsCall bc(c);
        if ((rc = bc.upload(0)) || (rc = launch_mask_base(c, 0))) { free_ctx(c); return rc; }
    }

    // the device address of bfv_decrypt_noalloc's fixed scratch array, with this device current
    if ((rc = noalloc_scratch_address(&c->noalloc_scratch, &c->noalloc_bytes))) { free_ctx(c); return rc; }

    if (cudaDeviceSynchronize() != cudaSuccess) { free_ctx(c); return BFV_ERR_CUDA; }
    *out = c;
    return BFV_OK;
}

int bfv_ctx_free(bfv_ctx *ctx) {
    if (!ctx) return BFV_ERR_INVALID_ARG;
    free_ctx(ctx);
    return BFV_OK;
}

int bfv_ctx_query(const bfv_ctx *ctx, uint64_t *primes, uint64_t *omega, uint64_t *delta_mod_q) {
    if (!ctx) return BFV_ERR_INVALID_ARG;
    if (primes) std::copy(ctx->primes.begin(), ctx->primes.end(), primes);
    if (omega) *omega = ctx->omega;
    if (delta_mod_q) std::copy(ctx->delta_host.begin(), ctx->delta_host.end(), delta_mod_q);
    return BFV_OK;
}

int bfv_keygen(bfv_ctx *ctx, uint64_t seed, uintptr_t stream, bfv_keys **out) {
    if (!ctx || !out) return BFV_ERR_INVALID_ARG;
    *out = nullptr;
    bfv_keys *k = new (std::nothrow) bfv_keys();
    if (!k) return BFV_ERR_OOM;
    k->ctx = ctx;
    k->ng = (int)ctx->galois.size();
    const size_t N = ctx->N, L = ctx->L, nqp = ctx->nqp;
    int rc = BFV_OK;
    if ((rc = dalloc(&k->sk, N)) || (rc = dalloc(&k->sk_eval, nqp * N)) || (rc = dalloc(&k->pk_eval, 2 * L * N)) ||
        (rc = dalloc(&k->gk_eval, (size_t)k->ng * L * 2 * nqp * N))) {
        bfv_keys_free(k);
        return rc;
    }
    rc = launch_keygen(ctx, k, seed, S(stream));
    if (rc == BFV_OK && cudaStreamSynchronize(S(stream)) != cudaSuccess) rc = BFV_ERR_CUDA;
    if (rc) { bfv_keys_free(k); return rc; }
    *out = k;
    return BFV_OK;
}

int bfv_keys_free(bfv_keys *k) {
    if (!k) return BFV_ERR_INVALID_ARG;
    cudaFree(k->sk);
    cudaFree(k->sk_eval);
    cudaFree(k->pk_eval);
    cudaFree(k->gk_eval);
    delete k;
    return BFV_OK;
}

int bfv_keys_export(const bfv_ctx *ctx, const bfv_keys *keys, int8_t *sk, uint64_t *pk, uint64_t *gk, uintptr_t stream) {
    if (!ctx || !keys || keys->ctx != ctx) return BFV_ERR_INVALID_ARG;
    BoundsCall bc(ctx);
    bc.keys(keys);
    bc.io(sk, (size_t)ctx->N);
    bc.io(pk, sizeof(u64) * 2 * (size_t)ctx->L * ctx->N);
    bc.io(gk, sizeof(u64) * (size_t)keys->ng * ctx->L * 2 * ctx->nqp * ctx->N);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    int rc = launch_keys_export(ctx, keys, sk, (u64 *)pk, (u64 *)gk, S(stream));
    if (rc) return rc;
    return cudaStreamSynchronize(S(stream)) == cudaSuccess ? BFV_OK : BFV_ERR_CUDA;
}

int bfv_encode(bfv_ctx *ctx, const int64_t *slots, size_t count, uint64_t *pt, uintptr_t stream) {
    if (!ctx || (count && (!slots || !pt))) return BFV_ERR_INVALID_ARG;
    if (!count) return BFV_OK;
    BoundsCall bc(ctx);
    bc.io(slots, sizeof(int64_t) * count * ctx->N);
    bc.io(pt, sizeof(u64) * count * ctx->N);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    return launch_encode(ctx, slots, count, (u64 *)pt, S(stream));
}

int bfv_decode(bfv_ctx *ctx, const uint64_t *pt, size_t count, int64_t *slots, uintptr_t stream) {
    if (!ctx || (count && (!slots || !pt))) return BFV_ERR_INVALID_ARG;
    if (!count) return BFV_OK;
    BoundsCall bc(ctx);
    bc.io(pt, sizeof(u64) * count * ctx->N);
    bc.io(slots, sizeof(int64_t) * count * ctx->N);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    return launch_decode(ctx, (const u64 *)pt, count, slots, S(stream));
}

int bfv_encode_features(bfv_ctx *ctx, const uint8_t *X, size_t nX, size_t f, uint64_t *pt, uintptr_t stream) {
    if (!ctx || (nX && f && (!X || !pt))) return BFV_ERR_INVALID_ARG;
    if (!nX || !f) return BFV_OK;
    BoundsCall bc(ctx);
    bc.io(X, nX * f);
    bc.io(pt, sizeof(u64) * nX * ((f + ctx->N - 1) / ctx->N) * ctx->N);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    return launch_encode_features(ctx, X, nX, f, (u64 *)pt, S(stream));
}

int bfv_encode_feature_columns(bfv_ctx *ctx, const uint8_t *X, size_t nX, size_t f, uint64_t *pt, uintptr_t stream) {
    if (!ctx || nX > (size_t)ctx->N || (nX && f && (!X || !pt))) return BFV_ERR_INVALID_ARG;
    if (!f) return BFV_OK;
    if (!nX) return cudaMemsetAsync(pt, 0, f * ctx->N * 8, S(stream)) == cudaSuccess ? BFV_OK : BFV_ERR_CUDA;
    BoundsCall bc(ctx);
    bc.io(X, nX * f);
    bc.io(pt, sizeof(u64) * f * ctx->N);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    return launch_encode_columns(ctx, X, nX, f, (u64 *)pt, S(stream));
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int bfv_encrypt_workspace(const bfv_ctx *ctx, size_t count, size_t *bytes) {
    if (!ctx || !bytes) return BFV_ERR_INVALID_ARG;
    *bytes = align256(count * 3 * (size_t)ctx->N);
    return BFV_OK;
}

int bfv_encrypt(bfv_ctx *ctx, const bfv_keys *keys, const uint64_t *pt, size_t count, uint64_t seed, uint32_t obj0,
                uint64_t *ct, void *ws, size_t ws_bytes, uintptr_t stream) {
    if (!ctx || !keys || keys->ctx != ctx) return BFV_ERR_INVALID_ARG;
    if (!count) return BFV_OK;
    if (!pt || !ct || !ws) return BFV_ERR_INVALID_ARG;
    size_t need;
    bfv_encrypt_workspace(ctx, count, &need);
    if (ws_bytes < need) return BFV_ERR_OVER_BUDGET;
    BoundsCall bc(ctx);
    bc.keys(keys);
    bc.io(pt, sizeof(u64) * count * ctx->N);
    bc.io(ct, sizeof(u64) * count * 2 * ctx->L * ctx->N);
    bc.io(ws, ws_bytes);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    return launch_encrypt(ctx, keys, (const u64 *)pt, count, seed, obj0, (u64 *)ct, ws, S(stream));
}

int bfv_decrypt_workspace(const bfv_ctx *ctx, size_t count, size_t *bytes) {
    if (!ctx || !bytes) return BFV_ERR_INVALID_ARG;
    *bytes = align256(count * (size_t)ctx->L * ctx->N * 8);
    return BFV_OK;
}

int bfv_decrypt(bfv_ctx *ctx, const bfv_keys *keys, const uint64_t *ct, size_t count, uint64_t *pt, void *ws,
                size_t ws_bytes, uintptr_t stream) {
    if (!ctx || !keys || keys->ctx != ctx) return BFV_ERR_INVALID_ARG;
    if (!count) return BFV_OK;
    if (!ct || !pt || !ws) return BFV_ERR_INVALID_ARG;
    size_t need;
    bfv_decrypt_workspace(ctx, count, &need);
    if (ws_bytes < need) return BFV_ERR_OVER_BUDGET;
    BoundsCall bc(ctx);
    bc.keys(keys);
    bc.io(ct, sizeof(u64) * count * 2 * ctx->L * ctx->N);
    bc.io(pt, sizeof(u64) * count * ctx->N);
    bc.io(ws, ws_bytes);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    return launch_decrypt(ctx, keys, (const u64 *)ct, count, (u64 *)pt, ws, S(stream));
}

int bfv_noise_budget_workspace(const bfv_ctx *ctx, size_t count, size_t *bytes) {
    if (!ctx || !bytes) return BFV_ERR_INVALID_ARG;
    *bytes = align256(count * (size_t)ctx->L * ctx->N * 8) + align256(count * sizeof(int));
    return BFV_OK;
}

int bfv_noise_budget(bfv_ctx *ctx, const bfv_keys *keys, const uint64_t *ct, size_t count, int *budgets, void *ws,
                     size_t ws_bytes, uintptr_t stream) {
    if (!ctx || !keys || keys->ctx != ctx) return BFV_ERR_INVALID_ARG;
    if (!count) return BFV_OK;
    if (!ct || !budgets || !ws) return BFV_ERR_INVALID_ARG;
    size_t need;
    bfv_noise_budget_workspace(ctx, count, &need);
    if (ws_bytes < need) return BFV_ERR_OVER_BUDGET;
    u64 *x = (u64 *)ws;
    int *bits = (int *)((char *)ws + align256(count * (size_t)ctx->L * ctx->N * 8));
    cudaStream_t st = S(stream);
    BoundsCall bc(ctx);
    bc.keys(keys);
    bc.io(ct, sizeof(u64) * count * 2 * ctx->L * ctx->N);
    bc.io(ws, ws_bytes);
    BFV_BOUNDS_UPLOAD(bc, st);
    int rc = launch_noise_bits(ctx, keys, (const u64 *)ct, count, x, bits, st);
    if (rc) return rc;
    std::vector<int> hb(count);
    if (cudaMemcpyAsync(hb.data(), bits, count * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return BFV_ERR_CUDA;
    for (size_t c = 0; c < count; ++c) budgets[c] = std::max(0, ctx->qbits - hb[c] - 1);
    return BFV_OK;
}

int bfv_model_prepare(bfv_ctx *ctx, const int64_t *W, const int64_t *b, size_t f, size_t nY, uintptr_t stream,
                      bfv_model **out) {
    if (!ctx || !W || !b || !out || f == 0 || nY == 0) return BFV_ERR_INVALID_ARG;
    *out = nullptr;
    const size_t N = ctx->N, L = ctx->L, K = (f + N - 1) / N;
    bfv_model *m = new (std::nothrow) bfv_model();
    if (!m) return BFV_ERR_OOM;
    m->ctx = ctx;
    m->f = f;
    m->nY = nY;
    m->K = K;
    int rc;
    int64_t *dslots = nullptr;
    u64 *dpt = nullptr;
    const size_t ngroups = (nY + 15) / 16;
    const size_t f4 = (f + 3) / 4;
    const size_t f16s = (f + 15) / 16;
    if ((rc = dalloc(&m->w_eval, nY * K * L * N)) || (rc = dalloc(&m->w16, ngroups * f * 16)) ||
        (rc = dalloc(&m->w4, ngroups * f4 * 16)) || (rc = dalloc(&m->wtc, ngroups * f16s * 256)) ||
        (rc = dalloc(&m->bias_delta, nY * L)) || (rc = dalloc(&dslots, nY * K * N)) || (rc = dalloc(&dpt, nY * K * N))) {
        cudaFree(dslots);
        cudaFree(dpt);
        bfv_model_free(m);
        return rc;
    }
    for (size_t x = 0; x < f * nY; ++x) {
        const int64_t a = W[x] < 0 ? -W[x] : W[x];
        if (a > m->wmax) m->wmax = a;
    }
    // 16-wide int32 weight rows for the standard product (valid when |w| < 2^31)
    std::vector<int> w16(ngroups * f * 16, 0);
    if (m->wmax < (1ll << 31))
        for (size_t r = 0; r < f; ++r)
            for (size_t j = 0; j < nY; ++j) w16[((j / 16) * f + r) * 16 + j % 16] = (int)W[r * nY + j];
    // four consecutive features' int8 weights per int32 (byte u = feature 4i + u), per class
    std::vector<int> w4(ngroups * f4 * 16, 0);
    if (m->wmax <= 127)
        for (size_t r = 0; r < f; ++r)
            for (size_t j = 0; j < nY; ++j) {
                const uint32_t byte = (uint32_t)(uint8_t)(int8_t)W[r * nY + j];
                w4[((j / 16) * f4 + r / 4) * 16 + j % 16] |= (int)(byte << (8 * (r % 4)));
            }
    // f16 weights for the tensor-core product: per class group and 16 features one B tile of
    // 16 classes x 16 features in the canonical K-major layout [class/8][feature/8][class%8][feature%8]
    std::vector<uint16_t> wtc(ngroups * f16s * 256, 0);
    if (m->wmax <= 127)
        for (size_t r = 0; r < f; ++r)
            for (size_t j = 0; j < nY; ++j) {
                const size_t st = r / 16, k = r % 16, n = j % 16;
                wtc[((j / 16) * f16s + st) * 256 + (n / 8) * 128 + (k / 8) * 64 + (n % 8) * 8 + k % 8] =
                    f16_of_small(W[r * nY + j]);
            }
    // transposed, packed weights: slot s of plaintext (j, k) = W[k N + s][j]
    std::vector<int64_t> slots(nY * K * N, 0);
    for (size_t j = 0; j < nY; ++j)
        for (size_t r = 0; r < f; ++r) slots[(j * K + r / N) * N + r % N] = W[r * nY + j];
    std::vector<u64> bd(nY * L);
    for (size_t j = 0; j < nY; ++j) {
        int64_t bt = b[j] % (int64_t)ctx->t;
        if (bt < 0) bt += (int64_t)ctx->t;
        for (size_t l = 0; l < L; ++l) bd[j * L + l] = mulmod_h(ctx->delta_host[l], (u64)bt % ctx->primes[l], ctx->primes[l]);
    }
    cudaStream_t st = S(stream);
    rc = BFV_OK;
    if (cudaMemcpyAsync(dslots, slots.data(), slots.size() * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(m->w16, w16.data(), w16.size() * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(m->w4, w4.data(), w4.size() * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(m->wtc, wtc.data(), wtc.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(m->bias_delta, bd.data(), bd.size() * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = BFV_ERR_CUDA;
    BoundsCall bc(ctx);
    bc.model(m);
    bc.add(dslots, sizeof(int64_t) * nY * K * N);
    bc.add(dpt, sizeof(u64) * nY * K * N);
    if (!rc) rc = bc.upload(st);
    if (!rc) rc = launch_encode(ctx, dslots, nY * K, dpt, st);
    if (!rc) rc = launch_model_weights(ctx, m, dpt, st);
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = BFV_ERR_CUDA;
    cudaFree(dslots);
    cudaFree(dpt);
    if (rc) { bfv_model_free(m); return rc; }
    *out = m;
    return BFV_OK;
}

int bfv_model_free(bfv_model *m) {
    if (!m) return BFV_ERR_INVALID_ARG;
    cudaFree(m->w_eval);
    cudaFree(m->w16);
    cudaFree(m->w4);
    cudaFree(m->wtc);
    cudaFree(m->bias_delta);
    delete m;
    return BFV_OK;
}

int bfv_lr_scores_packed_workspace(const bfv_ctx *ctx, const bfv_model *model, size_t nX, size_t pair_chunk,
                                   size_t *bytes) {
    if (!ctx || !model || model->ctx != ctx || !bytes || nX == 0) return BFV_ERR_INVALID_ARG;
    *bytes = packed_plan(ctx, model, nX, pair_chunk).total;
    return BFV_OK;
}

int bfv_lr_scores_packed(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint64_t *X_ct, size_t nX,
                         uint64_t *Y_ct, void *ws, size_t ws_bytes, size_t pair_chunk, uintptr_t stream) {
    if (!ctx || !keys || !model || keys->ctx != ctx || model->ctx != ctx) return BFV_ERR_INVALID_ARG;
    if (nX == 0) return BFV_OK;
    if (!X_ct || !Y_ct || !ws) return BFV_ERR_INVALID_ARG;
    PackedPlan plan = packed_plan(ctx, model, nX, pair_chunk);
    if (ws_bytes < plan.total) return BFV_ERR_OVER_BUDGET;
    BoundsCall bc(ctx);
    bounds_packed(bc, ctx, keys, 1, &model, &X_ct, &nX, &Y_ct, ws, ws_bytes);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    return launch_packed(ctx, keys, (const u64 *)X_ct, (u64 *)Y_ct, ws, plan, S(stream));
}

int bfv_lr_scores_packed_multi_workspace(const bfv_ctx *ctx, const bfv_model *model, int nreq, const size_t *nXs,
                                         size_t pair_chunk, size_t *bytes) {
    if (!ctx || !model || model->ctx != ctx || !bytes || !nXs || nreq < 1 || nreq > kMaxReq) return BFV_ERR_INVALID_ARG;
    for (int r = 0; r < nreq; ++r)
        if (!nXs[r]) return BFV_ERR_INVALID_ARG;
    *bytes = packed_plan_multi(ctx, model, nreq, nXs, pair_chunk).total;
    return BFV_OK;
}

int bfv_lr_scores_packed_multi(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, int nreq,
                               const uint64_t *const *X_cts, const size_t *nXs, uint64_t *const *Y_cts, void *ws,
                               size_t ws_bytes, size_t pair_chunk, uintptr_t stream) {
    if (!ctx || !keys || !model || keys->ctx != ctx || model->ctx != ctx) return BFV_ERR_INVALID_ARG;
    if (nreq < 1 || nreq > kMaxReq || !X_cts || !nXs || !Y_cts || !ws) return BFV_ERR_INVALID_ARG;
    for (int r = 0; r < nreq; ++r)
        if (!nXs[r] || !X_cts[r] || !Y_cts[r]) return BFV_ERR_INVALID_ARG;
    PackedPlan plan = packed_plan_multi(ctx, model, nreq, nXs, pair_chunk);
    if (ws_bytes < plan.total) return BFV_ERR_OVER_BUDGET;
    {
        const bfv_model *ms[kMaxReq];
        for (int r = 0; r < nreq; ++r) ms[r] = model;
        BoundsCall bc(ctx);
        bounds_packed(bc, ctx, keys, nreq, ms, X_cts, nXs, Y_cts, ws, ws_bytes);
        BFV_BOUNDS_UPLOAD(bc, S(stream));
    }
    return launch_packed_multi(ctx, keys, nreq, (const u64 *const *)X_cts, (u64 *const *)Y_cts, ws, plan, S(stream));
}

static int models_ok(const bfv_ctx *ctx, int nreq, const bfv_model *const *models, const size_t *nXs) {
    if (!ctx || !models || !nXs || nreq < 1 || nreq > kMaxReq) return BFV_ERR_INVALID_ARG;
    for (int r = 0; r < nreq; ++r)
        if (!models[r] || models[r]->ctx != ctx || !nXs[r]) return BFV_ERR_INVALID_ARG;
    return BFV_OK;
}

int bfv_lr_scores_packed_models_workspace(const bfv_ctx *ctx, int nreq, const bfv_model *const *models,
                                          const size_t *nXs, size_t pair_chunk, size_t *bytes) {
    if (!bytes) return BFV_ERR_INVALID_ARG;
    int rc = models_ok(ctx, nreq, models, nXs);
    if (rc) return rc;
    *bytes = packed_plan_models(ctx, nreq, models, nXs, pair_chunk).total;
    return BFV_OK;
}

int bfv_lr_scores_packed_models(bfv_ctx *ctx, const bfv_keys *keys, int nreq, const bfv_model *const *models,
                                const uint64_t *const *X_cts, const size_t *nXs, uint64_t *const *Y_cts, void *ws,
                                size_t ws_bytes, size_t pair_chunk, uintptr_t stream) {
    int rc = models_ok(ctx, nreq, models, nXs);
    if (rc) return rc;
    if (!keys || keys->ctx != ctx || !X_cts || !Y_cts || !ws) return BFV_ERR_INVALID_ARG;
    for (int r = 0; r < nreq; ++r)
        if (!X_cts[r] || !Y_cts[r]) return BFV_ERR_INVALID_ARG;
    PackedPlan plan = packed_plan_models(ctx, nreq, models, nXs, pair_chunk);
    if (ws_bytes < plan.total) return BFV_ERR_OVER_BUDGET;
    BoundsCall bc(ctx);
    bounds_packed(bc, ctx, keys, nreq, models, X_cts, nXs, Y_cts, ws, ws_bytes);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    return launch_packed_multi(ctx, keys, nreq, (const u64 *const *)X_cts, (u64 *const *)Y_cts, ws, plan, S(stream));
}

int bfv_crt_combine(const int64_t *r0, uint64_t t0, const int64_t *r1, uint64_t t1, size_t n, int64_t *out,
                    uintptr_t stream) {
    if (t0 < 2 || t1 < 2 || (n && (!r0 || !r1 || !out))) return BFV_ERR_INVALID_ARG;
    if ((u128)t0 * t1 >= ((u128)1 << 62)) return BFV_ERR_INVALID_ARG;
    u64 g = t0, h = t1;
    while (h) { const u64 r = g % h; g = h; h = r; }
    if (g != 1) return BFV_ERR_INVALID_ARG;
    const u64 inv = inv_h(t0 % t1, t1);
    BoundsCall bc;
    bc.io(r0, sizeof(int64_t) * n);
    bc.io(r1, sizeof(int64_t) * n);
    bc.io(out, sizeof(int64_t) * n);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    return launch_crt_combine(r0, t0, r1, t1, inv, n, out, S(stream));
}

int bfv_lr_scores_packed_graph(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint64_t *X_ct,
                               size_t nX, uint64_t *Y_ct, void *ws, size_t ws_bytes, size_t pair_chunk,
                               uintptr_t stream) {
    if (!ctx || !keys || !model || keys->ctx != ctx || model->ctx != ctx) return BFV_ERR_INVALID_ARG;
    if (nX == 0) return BFV_OK;
    if (!X_ct || !Y_ct || !ws) return BFV_ERR_INVALID_ARG;
    PackedPlan plan = packed_plan(ctx, model, nX, pair_chunk);
    if (ws_bytes < plan.total) return BFV_ERR_OVER_BUDGET;
    cudaStream_t st = S(stream);
    {
        // on the caller's stream, before the graph is captured or launched (never inside it)
        BoundsCall bc(ctx);
        bounds_packed(bc, ctx, keys, 1, &model, &X_ct, &nX, &Y_ct, ws, ws_bytes);
        BFV_BOUNDS_UPLOAD(bc, st);
    }
    if (ctx->prof.on)   // per-launch event timing needs direct launches
        return launch_packed(ctx, keys, (const u64 *)X_ct, (u64 *)Y_ct, ws, plan, st);
    const size_t splits = plan.sched.prep_split | plan.sched.modup_split << 4 | plan.sched.moddown_p_split << 8 |
                          plan.sched.moddown_split << 12;
    bfv_ctx::GraphKey key(keys, model, X_ct, nX, Y_ct, ws, plan.chunk, splits, st);
    std::lock_guard<std::mutex> g(ctx->graph_mu);
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        if (ctx->graphs.size() >= 64) {   // bounded cache: drop everything and start over
            for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second.first);
            ctx->graphs.clear();
        }
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        // capture on a context-owned stream (the caller's may be the uncapturable legacy stream)
        if (!ctx->capture_stream &&
            cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
            return BFV_ERR_CUDA;
        cudaStream_t cs = ctx->capture_stream;
        const uint64_t before = ctx->launches.load();
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BFV_ERR_CUDA;
        int rc = launch_packed(ctx, keys, (const u64 *)X_ct, (u64 *)Y_ct, ws, plan, cs);
        const uint64_t held = ctx->launches.load() - before;
        ctx->launches.fetch_sub(held);     // counted when the graph runs
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (rc || e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return rc ? rc : BFV_ERR_CUDA; }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return BFV_ERR_CUDA;
        it = ctx->graphs.emplace(key, std::make_pair(exec, held)).first;
    }
    if (cudaGraphLaunch(it->second.first, st) != cudaSuccess) return BFV_ERR_CUDA;
    count_launch(ctx, it->second.second);
    return BFV_OK;
}

int bfv_packed_schedule_get(const bfv_ctx *ctx, size_t npairs, bfv_packed_schedule *out) {
    if (!ctx || !out) return BFV_ERR_INVALID_ARG;
    *out = schedule_for(ctx, npairs, 0);
    return BFV_OK;
}

int bfv_packed_schedule_set(bfv_ctx *ctx, size_t npairs, const bfv_packed_schedule *sched) {
    if (!ctx || !sched || !schedule_ok(*sched)) return BFV_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    ctx->tuned[npairs] = *sched;
    return BFV_OK;
}

int bfv_lr_scores_packed_sched(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint64_t *X_ct,
                               size_t nX, uint64_t *Y_ct, void *ws, size_t ws_bytes, const bfv_packed_schedule *sched,
                               uintptr_t stream) {
    if (!ctx || !keys || !model || keys->ctx != ctx || model->ctx != ctx || !sched) return BFV_ERR_INVALID_ARG;
    if (!schedule_ok(*sched)) return BFV_ERR_INVALID_ARG;
    if (nX == 0) return BFV_OK;
    if (!X_ct || !Y_ct || !ws) return BFV_ERR_INVALID_ARG;
    PackedPlan plan = packed_plan(ctx, model, nX, 0, sched);
    if (ws_bytes < plan.total) return BFV_ERR_OVER_BUDGET;
    BoundsCall bc(ctx);
    bounds_packed(bc, ctx, keys, 1, &model, &X_ct, &nX, &Y_ct, ws, ws_bytes);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    return launch_packed(ctx, keys, (const u64 *)X_ct, (u64 *)Y_ct, ws, plan, S(stream));
}

namespace {
// Times one product with the given schedule (a warm-up run, then a timed run); *ms = its time.
int time_schedule(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint64_t *X_ct, size_t nX,
                  uint64_t *Y_ct, void *ws, const bfv_packed_schedule &sc, cudaStream_t st, cudaEvent_t a,
                  cudaEvent_t b, float *ms) {
    PackedPlan plan = packed_plan(ctx, model, nX, 0, &sc);
    int rc;
    if ((rc = launch_packed(ctx, keys, (const u64 *)X_ct, (u64 *)Y_ct, ws, plan, st))) return rc;   // warm-up
    cudaEventRecord(a, st);
    if ((rc = launch_packed(ctx, keys, (const u64 *)X_ct, (u64 *)Y_ct, ws, plan, st))) return rc;
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) return BFV_ERR_CUDA;
    return cudaEventElapsedTime(ms, a, b) == cudaSuccess ? BFV_OK : BFV_ERR_CUDA;
}

// The pair-chunk search of both autotuners: chunk sizes 128 .. 16384 that fit in ws_bytes, with
// the splits of `base`; returns the fastest in *best (BFV_ERR_OVER_BUDGET if none fits).
int tune_chunk(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint64_t *X_ct, size_t nX,
               uint64_t *Y_ct, void *ws, size_t ws_bytes, cudaStream_t st, cudaEvent_t a, cudaEvent_t b,
               bfv_packed_schedule *best, float *best_t) {
    const size_t npairs = nX * model->nY;
    const size_t cands[] = {128, 256, 512, 1024, 2048, 4096, 8192, 16384};
    bfv_packed_schedule base = *best;
    size_t last = 0;
    bool found = false;
    for (size_t ch : cands) {
        const size_t eff = std::min(ch, npairs);
        if (eff == last) continue;               // larger candidates all mean "every pair at once"
        last = eff;
        bfv_packed_schedule sc = base;
        sc.pair_chunk = eff;
        if (packed_plan(ctx, model, nX, 0, &sc).total > ws_bytes) break;
        float t = 0;
        int rc = time_schedule(ctx, keys, model, X_ct, nX, Y_ct, ws, sc, st, a, b, &t);
        if (rc) return rc;
        if (!found || t < *best_t) { *best = sc; *best_t = t; found = true; }
    }
    return found ? BFV_OK : BFV_ERR_OVER_BUDGET;
}
}  // namespace

int bfv_autotune_packed_schedule(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint64_t *X_ct,
                                 size_t nX, uint64_t *Y_ct, void *ws, size_t ws_bytes, uintptr_t stream,
                                 bfv_packed_schedule *best, double *best_ms) {
    if (!ctx || !keys || !model || keys->ctx != ctx || model->ctx != ctx || !best) return BFV_ERR_INVALID_ARG;
    if (nX == 0 || !X_ct || !Y_ct || !ws) return BFV_ERR_INVALID_ARG;
    cudaStream_t st = S(stream);
    {
        BoundsCall bc(ctx);
        bounds_packed(bc, ctx, keys, 1, &model, &X_ct, &nX, &Y_ct, ws, ws_bytes);
        BFV_BOUNDS_UPLOAD(bc, st);
    }
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess) return BFV_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return BFV_ERR_CUDA; }
    bfv_packed_schedule sc = default_schedule();
    float t = 0;
    int rc = tune_chunk(ctx, keys, model, X_ct, nX, Y_ct, ws, ws_bytes, st, a, b, &sc, &t);
    // coordinate descent over the splits, at the chosen chunk
    uint32_t bfv_packed_schedule::*fields[] = {&bfv_packed_schedule::prep_split, &bfv_packed_schedule::modup_split,
                                               &bfv_packed_schedule::moddown_p_split,
                                               &bfv_packed_schedule::moddown_split};
    const uint32_t values[4][5] = {{1, 2, 3, 0, 0}, {2, 4, 0, 0, 0}, {1, 2, 3, 4, 0}, {1, 2, 3, 0, 0}};   // 0 ends a list
    for (int f = 0; f < 4 && !rc; ++f) {
        for (int v = 0; v < 5 && values[f][v] && !rc; ++v) {
            bfv_packed_schedule cand = sc;
            cand.*fields[f] = values[f][v];
            if (cand.*fields[f] == sc.*fields[f]) continue;
            float tc = 0;
            rc = time_schedule(ctx, keys, model, X_ct, nX, Y_ct, ws, cand, st, a, b, &tc);
            if (!rc && tc < t) { sc = cand; t = tc; }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> g(ctx->tune_mu);
        ctx->tuned[nX * model->nY] = sc;
    }
    // leave Y_ct holding the product of the recorded schedule
    PackedPlan plan = packed_plan(ctx, model, nX, 0, &sc);
    if ((rc = launch_packed(ctx, keys, (const u64 *)X_ct, (u64 *)Y_ct, ws, plan, st))) return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess) return BFV_ERR_CUDA;
    *best = sc;
    if (best_ms) *best_ms = t;
    return BFV_OK;
}

int bfv_autotune_packed(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint64_t *X_ct, size_t nX,
                        uint64_t *Y_ct, void *ws, size_t ws_bytes, uintptr_t stream, size_t *best_chunk,
                        double *best_ms) {
    if (!ctx || !keys || !model || keys->ctx != ctx || model->ctx != ctx || !best_chunk) return BFV_ERR_INVALID_ARG;
    if (nX == 0 || !X_ct || !Y_ct || !ws) return BFV_ERR_INVALID_ARG;
    cudaStream_t st = S(stream);
    {
        BoundsCall bc(ctx);
        bounds_packed(bc, ctx, keys, 1, &model, &X_ct, &nX, &Y_ct, ws, ws_bytes);
        BFV_BOUNDS_UPLOAD(bc, st);
    }
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess) return BFV_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return BFV_ERR_CUDA; }
    const size_t npairs = nX * model->nY;
    bfv_packed_schedule sc = schedule_for(ctx, npairs, 0);   // its splits; the chunk is searched
    float t = 0;
    int rc = tune_chunk(ctx, keys, model, X_ct, nX, Y_ct, ws, ws_bytes, st, a, b, &sc, &t);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> g(ctx->tune_mu);
        ctx->tuned[npairs] = sc;
    }
    *best_chunk = sc.pair_chunk;
    if (best_ms) *best_ms = t;
    return BFV_OK;
}

int bfv_lr_scores_standard_workspace(const bfv_ctx *ctx, const bfv_model *model, size_t *bytes) {
    if (!ctx || !model || model->ctx != ctx || !bytes) return BFV_ERR_INVALID_ARG;
    *bytes = align256(standard_plan(ctx, model).bytes);
    return BFV_OK;
}

int bfv_lr_scores_standard(bfv_ctx *ctx, const bfv_model *model, const uint64_t *X_ct, size_t nX, uint64_t *Y_ct,
                           void *ws, size_t ws_bytes, uintptr_t stream) {
    if (!ctx || !model || model->ctx != ctx || nX > (size_t)ctx->N) return BFV_ERR_INVALID_ARG;
    if (!X_ct || !Y_ct || !ws) return BFV_ERR_INVALID_ARG;
    StandardPlan pl = standard_plan(ctx, model);
    if (ws_bytes < pl.bytes) return BFV_ERR_OVER_BUDGET;
    // signed 64-bit accumulators of w * (split halves) stay exact while |w| f 2^max(s, bits-s) < 2^63
    const int wide = std::max(pl.split_bits, ctx->bits - pl.split_bits);
    if (model->wmax >= (1ll << 31) || (long double)model->wmax * model->f * (long double)(1ull << wide) >= 9.2e18L)
        return BFV_ERR_BAD_PARAMS;
    BoundsCall bc(ctx);
    bc.model(model);
    bc.io(X_ct, sizeof(u64) * model->f * 2 * ctx->L * ctx->N);
    bc.io(Y_ct, sizeof(u64) * model->nY * 2 * ctx->L * ctx->N);
    bc.io(ws, ws_bytes);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    return launch_standard(ctx, model, (const u64 *)X_ct, (u64 *)Y_ct, ws, pl, S(stream));
}

int bfv_set_option(bfv_ctx *ctx, int option, int value) {
    if (!ctx) return BFV_ERR_INVALID_ARG;
    switch (option) {
        case BFV_OPT_ENCRYPT_SPLIT:
            if (value < 1 || value > 3) return BFV_ERR_INVALID_ARG;
            ctx->enc_split = value;
            return BFV_OK;
        case BFV_OPT_STANDARD_KERNEL:
            if (value != 0 && value != 1) return BFV_ERR_INVALID_ARG;
            ctx->std_kernel = value;
            return BFV_OK;
        default: return BFV_ERR_INVALID_ARG;
    }
}

int bfv_get_option(const bfv_ctx *ctx, int option, int *value) {
    if (!ctx || !value) return BFV_ERR_INVALID_ARG;
    switch (option) {
        case BFV_OPT_ENCRYPT_SPLIT: *value = ctx->enc_split; return BFV_OK;
        case BFV_OPT_STANDARD_KERNEL: *value = ctx->std_kernel; return BFV_OK;
        default: return BFV_ERR_INVALID_ARG;
    }
}

int bfv_debug_inject(bfv_ctx *ctx, int what, int value) {
    if (!ctx || value < 0) return BFV_ERR_INVALID_ARG;
    if (what == BFV_INJECT_STREAM_STALL) {
        if (value % 16) return BFV_ERR_INVALID_ARG;
        ctx->inject_extra_tx = value;
        return BFV_OK;
    }
    if (what == BFV_INJECT_BOUNDS_SHRINK) {
#ifdef BFV_BOUNDS
        if (value % 8) return BFV_ERR_INVALID_ARG;
        ctx->inject_shrink = value;
        return BFV_OK;
#else
        return BFV_ERR_INVALID_ARG;   // only a bounds-checked build has the tables
#endif
    }
    return BFV_ERR_INVALID_ARG;
}

int bfv_bounds_checked(void) {
#ifdef BFV_BOUNDS
    return 1;
#else
    return 0;
#endif
}

int bfv_check_error(bfv_ctx *ctx, int *flags) {
    if (!ctx || !flags) return BFV_ERR_INVALID_ARG;
    int v = 0;
    if (cudaMemcpy(&v, ctx->derr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return BFV_ERR_CUDA;
    if (v && cudaMemset(ctx->derr, 0, sizeof(int)) != cudaSuccess) return BFV_ERR_CUDA;
    *flags = v;
    return v ? BFV_ERR_TIMEOUT : BFV_OK;
}

int bfv_lr_packed_pair_from_workspace(bfv_ctx *ctx, const bfv_model *model, size_t nX, size_t pair_chunk,
                                      const void *ws, size_t g, uint64_t *ct_out, uintptr_t stream) {
    if (!ctx || !model || model->ctx != ctx || !ws || !ct_out) return BFV_ERR_INVALID_ARG;
    PackedPlan plan = packed_plan(ctx, model, nX, pair_chunk);
    if (g >= plan.npairs) return BFV_ERR_INVALID_ARG;
    const size_t last_chunk_start = ((plan.npairs - 1) / plan.chunk) * plan.chunk;
    if (g < last_chunk_start) return BFV_ERR_INVALID_ARG;
    BoundsCall bc(ctx);
    bc.io(ws, plan.total);
    bc.io(ct_out, sizeof(u64) * 2 * ctx->L * ctx->N);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    int rc = launch_pair_export(ctx, plan, ws, g - last_chunk_start, (u64 *)ct_out, S(stream));
    if (rc) return rc;
    return cudaStreamSynchronize(S(stream)) == cudaSuccess ? BFV_OK : BFV_ERR_CUDA;
}

// ------------------------------------------------------------------ whole-protocol calls

namespace {
struct PredictPlan {
    PackedPlan packed;
    size_t off_x, off_pt, off_ct, off_encws, off_packed, off_y, off_decws, off_ptout, off_slots, total;
};
PredictPlan predict_plan(const bfv_ctx *c, const bfv_model *m, size_t nX, size_t chunk) {
    PredictPlan p{};
    p.packed = packed_plan(c, m, nX, chunk);
    const size_t N = c->N, L = c->L, K = m->K, nout = p.packed.nout, ctb = 2 * L * N * 8;
    size_t off = 0;
    p.off_x = off; off += align256(nX * m->f);
    p.off_pt = off; off += align256(nX * K * N * 8);
    p.off_ct = off; off += align256(nX * K * ctb);
    p.off_encws = off; off += align256(nX * K * 3 * N);
    p.off_packed = off; off += align256(p.packed.total);
    p.off_y = off; off += align256(nout * ctb);
    p.off_decws = off; off += align256(nout * L * N * 8);
    p.off_ptout = off; off += align256(nout * N * 8);
    p.off_slots = off; off += align256(nout * N * 8);
    p.total = off;
    return p;
}
int run_predict(bfv_ctx *c, const bfv_keys *k, const bfv_model *m, const uint8_t *X, size_t nX, u64 seed,
                const PredictPlan &pl, char *ws, cudaStream_t st) {
    u64 *pt = (u64 *)(ws + pl.off_pt), *ct = (u64 *)(ws + pl.off_ct), *Y = (u64 *)(ws + pl.off_y);
    u64 *ptout = (u64 *)(ws + pl.off_ptout);
    int64_t *slots = (int64_t *)(ws + pl.off_slots);
    int rc;
    if ((rc = launch_encode_features(c, X, nX, m->f, pt, st))) return rc;
    if ((rc = launch_encrypt(c, k, pt, nX * m->K, seed, 0, ct, ws + pl.off_encws, st))) return rc;
    if ((rc = launch_packed(c, k, ct, Y, ws + pl.off_packed, pl.packed, st))) return rc;
    if ((rc = launch_decrypt(c, k, Y, pl.packed.nout, ptout, ws + pl.off_decws, st))) return rc;
    return launch_decode(c, ptout, pl.packed.nout, slots, st);
}
}  // namespace

int bfv_lr_predict_packed_workspace(const bfv_ctx *ctx, const bfv_model *model, size_t nX, size_t pair_chunk,
                                    size_t *bytes) {
    if (!ctx || !model || model->ctx != ctx || !bytes || nX == 0) return BFV_ERR_INVALID_ARG;
    *bytes = predict_plan(ctx, model, nX, pair_chunk).total;
    return BFV_OK;
}

int bfv_lr_predict_packed(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint8_t *X, size_t nX,
                          uint64_t seed, int64_t *scores, void *ws, size_t ws_bytes, size_t pair_chunk,
                          uintptr_t stream) {
    if (!ctx || !keys || !model || keys->ctx != ctx || model->ctx != ctx) return BFV_ERR_INVALID_ARG;
    if (nX == 0) return BFV_OK;
    if (!X || !scores || !ws) return BFV_ERR_INVALID_ARG;
    PredictPlan pl = predict_plan(ctx, model, nX, pair_chunk);
    if (ws_bytes < pl.total) return BFV_ERR_OVER_BUDGET;
    BoundsCall bc(ctx);
    bc.keys(keys);
    bc.model(model);
    bc.io(X, nX * model->f);
    bc.io(ws, ws_bytes);
    BFV_BOUNDS_UPLOAD(bc, S(stream));
    int rc = run_predict(ctx, keys, model, X, nX, seed, pl, (char *)ws, S(stream));
    if (rc) return rc;
    return cudaMemcpyAsync(scores, (char *)ws + pl.off_slots, nX * model->nY * 8, cudaMemcpyDeviceToDevice,
                           S(stream)) == cudaSuccess ? BFV_OK : BFV_ERR_CUDA;
}

int bfv_lr_predict_packed_host(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint8_t *X_host,
                               size_t nX, uint64_t seed, int64_t *scores_host, void *ws, size_t ws_bytes,
                               size_t pair_chunk, uintptr_t stream) {
    if (!ctx || !keys || !model || keys->ctx != ctx || model->ctx != ctx) return BFV_ERR_INVALID_ARG;
    if (nX == 0) return BFV_OK;
    if (!X_host || !scores_host || !ws) return BFV_ERR_INVALID_ARG;
    PredictPlan pl = predict_plan(ctx, model, nX, pair_chunk);
    if (ws_bytes < pl.total) return BFV_ERR_OVER_BUDGET;
    char *w = (char *)ws;
    cudaStream_t st = S(stream);
    BoundsCall bc(ctx);
    bc.keys(keys);
    bc.model(model);
    bc.io(ws, ws_bytes);
    BFV_BOUNDS_UPLOAD(bc, st);
    if (cudaMemcpyAsync(w + pl.off_x, X_host, nX * model->f, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return BFV_ERR_CUDA;
    int rc = run_predict(ctx, keys, model, (const uint8_t *)(w + pl.off_x), nX, seed, pl, w, st);
    if (rc) return rc;
    if (cudaMemcpyAsync(scores_host, w + pl.off_slots, nX * model->nY * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return BFV_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? BFV_OK : BFV_ERR_CUDA;
}

int bfv_profile(bfv_ctx *ctx, int enable) {
    if (!ctx) return BFV_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(ctx->prof.mu);
    ctx->prof.on = enable != 0;
    return BFV_OK;
}

int bfv_profile_read(bfv_ctx *ctx, int kind, uint64_t *launches, double *total_ms) {
    if (!ctx || kind < 0 || kind >= BFV_K_COUNT || !launches || !total_ms) return BFV_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(ctx->prof.mu);
    double ms = 0;
    int rc = BFV_OK;
    for (auto &pr : ctx->prof.pending[kind]) {
        float x = 0;
        if (cudaEventSynchronize(pr.second) != cudaSuccess || cudaEventElapsedTime(&x, pr.first, pr.second) != cudaSuccess)
            rc = BFV_ERR_CUDA;
        ms += x;
        ctx->prof.pool.push_back(pr.first);
        ctx->prof.pool.push_back(pr.second);
    }
    *launches = ctx->prof.pending[kind].size();
    *total_ms = ms;
    ctx->prof.pending[kind].clear();
    return rc;
}

int bfv_launch_count(const bfv_ctx *ctx, uint64_t *count) {
    if (!ctx || !count) return BFV_ERR_INVALID_ARG;
    *count = ctx->launches.load();
    return BFV_OK;
}

}  // extern "C"
