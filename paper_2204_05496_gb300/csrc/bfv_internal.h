// bfv_internal.h -- host-side structures shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "bfv_device.cuh"
#include "../../include/bfv_lr.h"

// Constants for exact decryption (mixed-radix CRT plus multi-word division), device copy.
struct DecConst {
    int L, W;                        // primes, 64-bit words of t*Q + Q/2
    int tbits;                       // bit length of t
    int pad_;
    u64 t;
    u64 inv[BFV_MAXP][BFV_MAXP];     // q_i^-1 mod q_j (i < j)
    u64 invp[BFV_MAXP][BFV_MAXP];    // Shoup companions
    u64 qhalf[BFV_MAXW];             // floor(Q/2)
    u64 qshift[32][BFV_MAXW];        // Q << b for b < tbits
};

// Opt-in per-kernel CUDA-event timing (bfv_profile / bfv_profile_read).
struct Profiler {
    bool on = false;
    std::mutex mu;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[BFV_K_COUNT];
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        cudaEvent_t e = nullptr;
        if (!pool.empty()) { e = pool.back(); pool.pop_back(); }
        else cudaEventCreate(&e);
        return e;
    }
};

struct bfv_ctx {
    int device = 0;
    int N = 0, logN = 0, L = 0, nqp = 0, bits = 0;
    int qbits = 0;                   // bit length of Q
    u64 t = 0, omega = 0;
    uint32_t sigma_num = 16, sigma_den = 5;
    std::vector<u64> primes;         // L+1 (index L = P)
    std::vector<ModTab> hmods;       // host copy, nqp + 1 entries (index nqp = t)
    ModTab *dmods = nullptr;         // device copy
    u64 *dtw = nullptr;              // twiddle tables [nqp+1][6][N]
    u32 *dslot = nullptr;            // [N] evaluation position of slot l (mod-t transform)
    u32 *dmaskpow = nullptr;         // [2N] N^-1 omega^i mod t
    shoup_t *dmaskev = nullptr;      // [L][N] evaluation form of the slot-0 one-hot mask (Shoup form)
    u64 *dcdt = nullptr;             // Gaussian thresholds
    int cdt_len = 0;
    DecConst *ddec = nullptr;        // decryption constants
    std::vector<u64> galois;         // rotate-and-sum Galois elements, in order
    std::vector<u64> delta_host;     // floor(Q/t) mod q_l
    int sms = 0;                     // streaming multiprocessors of the device
    int *derr = nullptr;             // device error word (bounded waits that ran out set bit 0)
    int inject_extra_tx = 0;         // failure injection: bytes a streaming stage waits for in vain
    u64 *noalloc_scratch = nullptr;  // device address of bfv_decrypt_noalloc's fixed array
    size_t noalloc_bytes = 0;        // its size
    int enc_split = 3;               // how the encryption kernel splits a limb at N = 16384 (BFV_OPT_ENCRYPT_SPLIT)
    int std_kernel = 0;              // standard product with int8 weights: 0 tensor cores, 1 dp4a (BFV_OPT_STANDARD_KERNEL)
    int inject_shrink = 0;           // bounds-checked build, tests: caller buffers registered this many bytes short
    std::map<size_t, bfv_packed_schedule> tuned;   // pairs -> schedule (0: any other pair count)
    mutable std::mutex tune_mu;                    // guards tuned (read by every packed plan)
    // CUDA graphs of whole packed products, keyed by every argument of the call
    typedef std::tuple<const void *, const void *, const void *, size_t, void *, void *, size_t, size_t, cudaStream_t>
        GraphKey;   // keys, model, inputs, individuals, outputs, workspace, pair chunk, splits, stream
    std::map<GraphKey, std::pair<cudaGraphExec_t, uint64_t>> graphs;   // exec, kernel launches it holds
    std::mutex graph_mu;
    cudaStream_t capture_stream = nullptr;   // graphs are captured here, then launched on the caller's stream
    std::atomic<uint64_t> launches{0};
    mutable Profiler prof;
};

struct bfv_keys {
    const bfv_ctx *ctx = nullptr;
    int8_t *sk = nullptr;            // [N] ternary
    shoup_t *sk_eval = nullptr;      // [nqp][N] {value, companion} (evaluation layout)
    shoup_t *pk_eval = nullptr;      // [2][L][N]
    shoup_t *gk_eval = nullptr;      // [ng][L digits][2 comps][nqp][N]
    int ng = 0;
};

struct bfv_model {
    const bfv_ctx *ctx = nullptr;
    size_t f = 0, nY = 0, K = 0;
    shoup_t *w_eval = nullptr;       // [nY][K][L][N] {value, companion} (packed product)
    int *w16 = nullptr;              // [ceil(nY/16)][f][16] int32 weights, zero-padded (standard product)
    int *w4 = nullptr;               // [ceil(nY/16)][ceil(f/4)][16] four int8 weights per int32 (|w| <= 127)
    uint16_t *wtc = nullptr;         // [ceil(nY/16)][ceil(f/16)][256] f16 weights, one canonical MMA B tile
                                     // (K-major: [class/8][feature/8][class%8][feature%8]) per 16 features
    u64 *bias_delta = nullptr;       // [nY][L]: Delta [b_j]_t mod q_l
    int64_t wmax = 0;                // max |w| (bounds the standard product's accumulators)
};

// Launch-count bookkeeping.
inline void count_launch(const bfv_ctx *c, uint64_t n = 1) {
    const_cast<bfv_ctx *>(c)->launches.fetch_add(n, std::memory_order_relaxed);
}

// Names of the kernel kinds (BFV_K_*), as NVTX range names.
inline const char *kernel_kind_name(int kind) {
    static const char *names[BFV_K_COUNT] = {"bfv.ntt", "bfv.ks_prep", "bfv.ks_modup", "bfv.ks_moddown_p",
                                             "bfv.ks_moddown", "bfv.mac", "bfv.bias_mask", "bfv.compress",
                                             "bfv.encrypt", "bfv.decrypt", "bfv.encode", "bfv.standard"};
    return kind >= 0 && kind < BFV_K_COUNT ? names[kind] : "bfv";
}

// Around the launches in its scope: an NVTX range named after the kernel kind (host-side
// annotation for profilers; a few nanoseconds when no tool is attached) and, when profiling is
// on, a CUDA event pair on the launching stream.
struct ProfScope {
    const bfv_ctx *c;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfScope(const bfv_ctx *c_, int kind_, cudaStream_t st_) : c(c_), kind(kind_), st(st_) {
        nvtxRangePushA(kernel_kind_name(kind));
        if (c->prof.on) {
            std::lock_guard<std::mutex> g(c->prof.mu);
            a = c->prof.get();
            cudaEventRecord(a, st);
        }
    }
    ~ProfScope() {
        if (a) {
            std::lock_guard<std::mutex> g(c->prof.mu);
            cudaEvent_t b = c->prof.get();
            cudaEventRecord(b, st);
            c->prof.pending[kind].push_back({a, b});
        }
        nvtxRangePop();
    }
};

// ------------------------------------------------------------------ bounds-checked build (host side)
//
// Each C entry point that launches kernels lists the buffers its launches may touch (the
// context's tables, the keys, the models, the caller's buffers at the sizes the call implies,
// internal temporaries) and uploads the list, in stream order, to every translation unit's
// device table before its launches. In the release build this is an empty struct.
#ifdef BFV_BOUNDS
cudaError_t bounds_upload_scheme(const BoundsTable &t, cudaStream_t st);
cudaError_t bounds_upload_packed(const BoundsTable &t, cudaStream_t st);
cudaError_t bounds_upload_standard(const BoundsTable &t, cudaStream_t st);
struct BoundsCall {
    BoundsTable t{};
    bool overflow = false;
    size_t shrink = 0;
    BoundsCall() {}                  // a call without a context (no error word to set)
    explicit BoundsCall(const bfv_ctx *c) : shrink((size_t)c->inject_shrink) {
        t.err = c->derr;
        add(c->dmods, sizeof(ModTab) * (c->nqp + 1));
        add(c->dtw, sizeof(u64) * (size_t)(c->nqp + 1) * 6 * c->N);
        add(c->dslot, sizeof(u32) * c->N);
        add(c->dmaskpow, sizeof(u32) * 2 * c->N);
        add(c->dmaskev, sizeof(shoup_t) * (size_t)c->L * c->N);
        add(c->dcdt, sizeof(u64) * 32);
        add(c->ddec, sizeof(DecConst));
        add(c->derr, sizeof(int));
        add(c->noalloc_scratch, c->noalloc_bytes);
    }
    void add(const void *p, size_t bytes) {
        if (!p || !bytes) return;
        if (t.n >= BFV_MAX_RANGES) { overflow = true; return; }
        t.lo[t.n] = (unsigned long long)p;
        t.hi[t.n] = (unsigned long long)p + bytes;
        ++t.n;
    }
    // a caller's buffer (registered `shrink` bytes short under failure injection)
    void io(const void *p, size_t bytes) { add(p, bytes > shrink ? bytes - shrink : 0); }
    void keys(const bfv_keys *k) {
        if (!k) return;
        const bfv_ctx *c = k->ctx;
        add(k->sk, (size_t)c->N);
        add(k->sk_eval, sizeof(shoup_t) * (size_t)c->nqp * c->N);
        add(k->pk_eval, sizeof(shoup_t) * 2 * (size_t)c->L * c->N);
        add(k->gk_eval, sizeof(shoup_t) * (size_t)k->ng * c->L * 2 * c->nqp * c->N);
    }
    void model(const bfv_model *m) {
        if (!m) return;
        const bfv_ctx *c = m->ctx;
        const size_t ng = (m->nY + 15) / 16;
        add(m->w_eval, sizeof(shoup_t) * m->nY * m->K * c->L * c->N);
        add(m->w16, sizeof(int) * ng * m->f * 16);
        add(m->w4, sizeof(int) * ng * ((m->f + 3) / 4) * 16);
        add(m->wtc, sizeof(uint16_t) * ng * ((m->f + 15) / 16) * 256);
        add(m->bias_delta, sizeof(u64) * m->nY * c->L);
    }
    int upload(cudaStream_t st) const {
        if (overflow) return BFV_ERR_INVALID_ARG;
        if (bounds_upload_scheme(t, st) != cudaSuccess || bounds_upload_packed(t, st) != cudaSuccess ||
            bounds_upload_standard(t, st) != cudaSuccess)
            return BFV_ERR_CUDA;
        return BFV_OK;
    }
};
#else
struct BoundsCall {
    BoundsCall() {}
    explicit BoundsCall(const bfv_ctx *) {}
    void add(const void *, size_t) {}
    void io(const void *, size_t) {}
    void keys(const bfv_keys *) {}
    void model(const bfv_model *) {}
    int upload(cudaStream_t) const { return BFV_OK; }
};
#endif

#define BFV_BOUNDS_UPLOAD(bc, st)                  \
    do {                                           \
        const int brc_ = (bc).upload(st);          \
        if (brc_) return brc_;                     \
    } while (0)

#define BFV_CUDA_TRY(expr)                              \
    do {                                                \
        cudaError_t e_ = (expr);                        \
        if (e_ != cudaSuccess) return BFV_ERR_CUDA;     \
    } while (0)

// Per-limb kernels run Split<LOGN>::S CTAs per limb (a two-CTA cluster at N = 32768): `h` is
// the CTA's part of the limb, `unit` the limb's index in the grid.
#define LIMB_KERNEL_M(LOGN, MODE) __global__ void __launch_bounds__(Split<LOGN, MODE>::NT, Split<LOGN, MODE>::MINB)
#define LIMB_KERNEL(LOGN) LIMB_KERNEL_M(LOGN, 0)
#define LIMB_INDEX_M(LOGN, MODE)                                            \
    constexpr int N = 1 << LOGN, M = Split<LOGN, MODE>::M;                  \
    const int h = Split<LOGN, MODE>::S == 1 ? 0 : (int)cluster_rank();      \
    const u32 unit = blockIdx.x / Split<LOGN, MODE>::S;                     \
    (void)N; (void)M; (void)h; (void)unit
#define LIMB_INDEX(LOGN) LIMB_INDEX_M(LOGN, 0)

// Launches a per-limb kernel over `units` limbs: Split<LOGN>::S CTAs of Split<LOGN>::NT
// threads per limb (one two-CTA cluster per limb when S = 2), limb_smem<LOGN>() bytes of
// dynamic shared memory unless `smem` says otherwise.
template <int LOGN, int MODE = 0> constexpr size_t limb_smem() { return sizeof(u64) * PadSize<Split<LOGN, MODE>::M>::value; }
template <int LOGN, int MODE = 0, class... KArgs, class... Args>
cudaError_t launch_limbs(void (*kern)(KArgs...), size_t units, cudaStream_t st, size_t smem, Args... args) {
    using SP = Split<LOGN, MODE>;
    if (!units) return cudaSuccess;
    if (!smem) smem = limb_smem<LOGN, MODE>();
    cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(units * SP::S), 1, 1);
    cfg.blockDim = dim3(SP::NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = SP::S;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = SP::S > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ------------------------------------------------------------------ launchers (k_*.cu)
// Each returns BFV_OK or BFV_ERR_CUDA (launch error); all are asynchronous on `st`.

int launch_ntt_limbs(const bfv_ctx *c, const u64 *in, u64 *out, size_t nct, bool forward, cudaStream_t st);
int launch_mask_base(const bfv_ctx *c, cudaStream_t st);
int launch_encode(const bfv_ctx *c, const int64_t *slots, size_t count, u64 *pt, cudaStream_t st);
int launch_decode(const bfv_ctx *c, const u64 *pt, size_t count, int64_t *slots, cudaStream_t st);
int launch_encode_features(const bfv_ctx *c, const uint8_t *X, size_t nX, size_t f, u64 *pt, cudaStream_t st);
int launch_encode_columns(const bfv_ctx *c, const uint8_t *X, size_t nX, size_t f, u64 *pt, cudaStream_t st);
int launch_keygen(const bfv_ctx *c, bfv_keys *k, u64 seed, cudaStream_t st);
int launch_keys_export(const bfv_ctx *c, const bfv_keys *k, int8_t *sk, u64 *pk, u64 *gk, cudaStream_t st);
int launch_encrypt(const bfv_ctx *c, const bfv_keys *k, const u64 *pt, size_t count, u64 seed, uint32_t obj0,
                   u64 *ct, void *ws, cudaStream_t st);
int launch_decrypt(const bfv_ctx *c, const bfv_keys *k, const u64 *ct, size_t count, u64 *pt, void *ws,
                   cudaStream_t st);
int launch_noise_bits(const bfv_ctx *c, const bfv_keys *k, const u64 *ct, size_t count, u64 *x, int *bits,
                      cudaStream_t st);
int launch_model_weights(const bfv_ctx *c, bfv_model *m, const u64 *w_pt, cudaStream_t st);
// Device address of bfv_decrypt_noalloc's fixed scratch array on the current device (k_scheme.cu).
int noalloc_scratch_address(u64 **out, size_t *bytes);
int launch_crt_combine(const int64_t *r0, u64 t0, const int64_t *r1, u64 t1, u64 inv, size_t n, int64_t *out,
                       cudaStream_t st);

// Requests fused into one packed product, passed to kernels by value. Every request has its
// own model (several requests may share one).
constexpr int kMaxReq = 64;
struct ReqTable {
    int n;
    int pad_;
    u64 pair_start[kMaxReq + 1];     // first global pair of each request; [n] = number of pairs
    long long xoff[kMaxReq];         // transformed input of request r, individual i, plaintext k sits at
                                     // xoff[r] + i K[r] + k in the chunk's input buffer (set per chunk)
    u32 K[kMaxReq];                  // plaintexts per individual, ceil(f / N), of each request's model
    u32 nY[kMaxReq];                 // classes of each request's model
    const shoup_t *w[kMaxReq];       // encoded weights [nY][K][L][N] of each request's model
    const u64 *bias[kMaxReq];        // Delta [b_j]_t mod q_l, [nY][L]
};

struct PackedPlan {
    size_t nX, nY, K;                // single-model products: individuals, classes, plaintexts per individual
    size_t npairs, nout, chunk;      // chunk = sched.pair_chunk, at most npairs
    bfv_packed_schedule sched;       // how the key-switching kernels split their limbs
    size_t xcts_chunk;               // most input ciphertexts any pair chunk needs in evaluation form
    size_t off_xntt, off_yacc, off_state, off_digits, off_u, off_r, total;
    int nreq;
    ReqTable rt;
    size_t nXs[kMaxReq], ycts[kMaxReq], nouts[kMaxReq];   // per request: individuals, first output, outputs
};

// Individuals [ia, ib) of request r that have pairs in the chunk [g0, g0 + ng) (ia == ib: none).
inline void chunk_window(const PackedPlan &p, int r, size_t g0, size_t ng, size_t &ia, size_t &ib) {
    const size_t pa = p.rt.pair_start[r], pb = p.rt.pair_start[r + 1], nY = p.rt.nY[r];
    const size_t a = pa > g0 ? pa : g0, b = pb < g0 + ng ? pb : g0 + ng;
    if (a >= b) { ia = ib = 0; return; }
    ia = (a - pa) / nY;
    ib = (b - 1 - pa) / nY + 1;
}

// The schedule of a product: `sched` if given, else the one recorded for its pair count (or the
// default), with the pair chunk replaced by `chunk` when non-zero.
bfv_packed_schedule default_schedule();
bool schedule_ok(const bfv_packed_schedule &s);
bfv_packed_schedule schedule_for(const bfv_ctx *c, size_t npairs, size_t chunk);
PackedPlan packed_plan(const bfv_ctx *c, const bfv_model *m, size_t nX, size_t chunk,
                       const bfv_packed_schedule *sched = nullptr);
PackedPlan packed_plan_multi(const bfv_ctx *c, const bfv_model *m, int nreq, const size_t *nXs, size_t chunk,
                             const bfv_packed_schedule *sched = nullptr);
PackedPlan packed_plan_models(const bfv_ctx *c, int nreq, const bfv_model *const *models, const size_t *nXs,
                              size_t chunk, const bfv_packed_schedule *sched = nullptr);
int launch_packed_multi(const bfv_ctx *c, const bfv_keys *k, int nreq, const u64 *const *X_ct, u64 *const *Y_ct,
                        void *ws, const PackedPlan &plan, cudaStream_t st);
int launch_packed(const bfv_ctx *c, const bfv_keys *k, const u64 *X_ct, u64 *Y_ct, void *ws, const PackedPlan &plan,
                  cudaStream_t st);
int launch_pair_export(const bfv_ctx *c, const PackedPlan &plan, const void *ws, size_t slot_in_chunk, u64 *ct_out,
                       cudaStream_t st);
struct StandardPlan {
    size_t ntiles, splits, fper, ngroups, bytes;
    int split_bits;
    bool int8;                       // byte-plane kernels (|w| <= 127): tensor cores or dp4a
    bool tc;                         // byte planes on the tensor cores
};
StandardPlan standard_plan(const bfv_ctx *c, const bfv_model *m);
size_t standard_smem_bytes();
int launch_standard(const bfv_ctx *c, const bfv_model *m, const u64 *X_ct, u64 *Y_ct, void *ws, const StandardPlan &pl,
                    cudaStream_t st);

