/*
 * bfv_lr.h -- C ABI of the GB300 library for BFV-encrypted logistic-regression scoring.
 *
 * Paper: "Scalable privacy-preserving cancer type prediction with homomorphic encryption"
 * (Sarkar et al.). The calls follow the private inference protocol of Section 4.2.2
 * (Fig. 2): the client encodes and encrypts its feature matrix X (|X| x f), the server
 * multiplies the ciphertexts by the encoded transposed weights and adds the encoded
 * biases, the client decrypts and decodes W x + b. The server product is either the
 * packed algorithm of Section 4.2.3 / Algorithm 1 (multiply, add_many, rotate and
 * accumulate, mask, compress) or the "standard" per-element product of Section 5.2.3.
 *
 * Conventions for every call:
 *  - Return value: BFV_OK (0) or a negative BFV_ERR_* code. On error nothing that the
 *    caller owns is freed, and output buffers hold unspecified values.
 *  - Device buffers are plain device pointers (for example from torch tensors); the
 *    library never takes ownership of caller memory. `stream` is a cudaStream_t passed as
 *    uintptr_t (0 = legacy default stream). Calls that take a stream enqueue work and
 *    return without synchronising unless stated otherwise.
 *  - Handles (bfv_ctx, bfv_keys, bfv_model) are opaque, owned by the library, freed by the
 *    matching *_free call, and bound to the CUDA device that was current at creation.
 *  - A ciphertext crossing the boundary is uint64[2][L][N] in coefficient form, limb-major:
 *    component c (0 or 1), prime index l, coefficient k; every residue is in [0, q_l).
 *    A plaintext is uint64[N], coefficients in [0, t).
 *  - Arithmetic is exact modular integer arithmetic; results are bit-for-bit deterministic.
 */
#ifndef BFV_LR_H
#define BFV_LR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BFV_OK 0
#define BFV_ERR_INVALID_ARG (-1) /* null pointer, size out of range, handle mismatch */
#define BFV_ERR_BAD_PARAMS (-2)  /* unsupported or inconsistent BFV parameters */
#define BFV_ERR_OOM (-3)         /* a device allocation failed */
#define BFV_ERR_OVER_BUDGET (-4) /* caller's workspace or memory budget too small */
#define BFV_ERR_TIMEOUT (-5)     /* a bounded wait ran out */
#define BFV_ERR_CUDA (-6)        /* a CUDA runtime call failed */

/* BFV parameter shape. Primes: the L+1 largest primes below 2^prime_bits that are 1 mod 2N,
 * in descending order; the first L form the ciphertext modulus Q, the last is the
 * key-switching prime P. Supported: N in {4096, 8192, 16384, 32768}, 1 <= L <= 15,
 * 30 <= prime_bits <= 59, t prime with t = 1 mod 2N and t < 2^31. The Gaussian error has
 * width sigma = sigma_num / sigma_den and is truncated at floor(6 sigma). At N = 32768 each
 * limb transform runs on a cluster of two CTAs (a limb is larger than one CTA's shared
 * memory). */
typedef struct bfv_params {
    uint32_t N;
    uint32_t L;
    uint32_t prime_bits;
    uint32_t reserved;
    uint64_t t;
    uint32_t sigma_num;
    uint32_t sigma_den;
} bfv_params;

typedef struct bfv_ctx bfv_ctx;
typedef struct bfv_keys bfv_keys;
typedef struct bfv_model bfv_model;

/* ------------------------------------------------------------------ host-only helpers */

/* Library ABI version (currently 1). */
int bfv_abi_version(void);

/* The L+1 primes of a parameter shape (host computation, no GPU needed).
 * primes_out: caller buffer of L+1 uint64. */
int bfv_params_primes(const bfv_params *p, uint64_t *primes_out);

/* Gaussian sampler thresholds T_k = floor(2^64 Pr[|e| <= k]), k = 0 .. len-1, for width
 * sigma_num/sigma_den (host computation). out: caller buffer of at least 32 uint64;
 * *len receives the count (floor(6 sigma)). */
int bfv_gaussian_table(uint32_t sigma_num, uint32_t sigma_den, uint64_t *out, int *len);

/* ------------------------------------------------------------------ context and keys */

/* Builds the parameter set (primes, NTT tables, CRT and rounding constants) on the current
 * CUDA device. The paper uses SEAL's BFV (Section 5.2); these are its textbook parts. */
int bfv_setup(const bfv_params *p, bfv_ctx **out);
int bfv_ctx_free(bfv_ctx *ctx);

/* Copies out: primes (L+1 uint64, may be NULL), the slot-map root omega mod t (may be NULL),
 * and floor(Q/t) mod q_l for l < L (L uint64, may be NULL). */
int bfv_ctx_query(const bfv_ctx *ctx, uint64_t *primes, uint64_t *omega, uint64_t *delta_mod_q);

/* Generates the secret key s (ternary), the public key pk = ([-(a s + e)]_Q, a) and the
 * Galois keys for the rotate-and-sum of Algorithm 1 (the row swap 2N-1, then 3^(N/4), ...,
 * 3^1 mod 2N), one key-switching digit per ciphertext prime over Q*P. Randomness: ChaCha20
 * (RFC 8439) blocks keyed by `seed`. Keys stay resident on the device. Synchronises `stream`. */
int bfv_keygen(bfv_ctx *ctx, uint64_t seed, uintptr_t stream, bfv_keys **out);
int bfv_keys_free(bfv_keys *keys);

/* Debug / parity export of key material in coefficient form (device buffers):
 * sk: int8[N] (may be NULL); pk: uint64[2][L][N] (may be NULL);
 * gk: uint64[n_galois][L][2][L+1][N] (may be NULL), n_galois = log2 N. Synchronises. */
int bfv_keys_export(const bfv_ctx *ctx, const bfv_keys *keys, int8_t *sk, uint64_t *pk, uint64_t *gk,
                    uintptr_t stream);

/* ------------------------------------------------------------------ client side */

/* Batch encoding (Section 4.2.2: n values per plaintext): slots int64[count][N] (any integers,
 * taken mod t) -> plaintext polynomials uint64[count][N] with m(omega^e_l) = slot_l, where
 * slot l = r*(N/2) + c sits at exponent e_l = 3^c (r = 0) or 2N - 3^c (r = 1) mod 2N and
 * omega = g^((t-1)/2N), g the smallest primitive root mod t. Device buffers. */
int bfv_encode(bfv_ctx *ctx, const int64_t *slots, size_t count, uint64_t *pt, uintptr_t stream);

/* Inverse of bfv_encode: plaintexts uint64[count][N] -> slot values int64[count][N] in [0, t). */
int bfv_decode(bfv_ctx *ctx, const uint64_t *pt, size_t count, int64_t *slots, uintptr_t stream);

/* Packs and encodes the client's binary/integer feature matrix X (uint8[nX][f], device) for the
 * packed product: plaintext (i, k) holds features k*N .. k*N+N-1 of individual i in slots
 * 0 .. N-1, zero past f (Section 4.2.2: X is |X| x ceil(f/n) plaintexts).
 * pt: uint64[nX][ceil(f/N)][N]. */
int bfv_encode_features(bfv_ctx *ctx, const uint8_t *X, size_t nX, size_t f, uint64_t *pt, uintptr_t stream);

/* Packs and encodes X (uint8[nX][f], device, nX <= N) for the standard product: plaintext f
 * holds feature f of individual i in slot i (zero for i >= nX). pt: uint64[f][N]. */
int bfv_encode_feature_columns(bfv_ctx *ctx, const uint8_t *X, size_t nX, size_t f, uint64_t *pt,
                               uintptr_t stream);

/* Public-key encryption c = ([pk0 u + e1 + Delta m]_Q, [pk1 u + e2]_Q), Delta = floor(Q/t),
 * of count plaintexts pt (uint64[count][N]) into ct (uint64[count][2][L][N]). Ciphertext c
 * draws (u, e1, e2) from ChaCha20 blocks keyed by `seed` with nonce (6, obj0 + c, 0): block k
 * gives u_k (word 0), e1_k (words 1-3), e2_k (words 4-6). ws: device workspace of at least
 * bfv_encrypt_workspace(count) bytes. */
int bfv_encrypt_workspace(const bfv_ctx *ctx, size_t count, size_t *bytes);
int bfv_encrypt(bfv_ctx *ctx, const bfv_keys *keys, const uint64_t *pt, size_t count, uint64_t seed,
                uint32_t obj0, uint64_t *ct, void *ws, size_t ws_bytes, uintptr_t stream);

/* Decryption m = round(t [c0 + c1 s]_Q / Q) mod t, computed exactly (mixed-radix CRT and
 * multi-word integer division, no floating point): ct uint64[count][2][L][N] ->
 * pt uint64[count][N]. ws: at least bfv_decrypt_workspace(count) bytes. */
int bfv_decrypt_workspace(const bfv_ctx *ctx, size_t count, size_t *bytes);
int bfv_decrypt(bfv_ctx *ctx, const bfv_keys *keys, const uint64_t *ct, size_t count, uint64_t *pt,
                void *ws, size_t ws_bytes, uintptr_t stream);

/* Invariant noise budget, a diagnostic (Section 4.2.2 sizes the plaintext modulus by the noise
 * budget a ciphertext must keep). Per ciphertext, z = [t [c0 + c1 s]_Q]_Q centred in
 * (-Q/2, Q/2] coefficient by coefficient. Since t x = t e - (Q mod t) m mod Q, z / Q is the
 * invariant noise v of (t/Q)(c0 + c1 s) = m + v mod t. The budget is
 * max(0, bitlen(Q) - bitlen(max_k |z_k|) - 1) bits. A positive budget gives |v| < 1/2, so
 * rounding recovers the message. ct: device uint64[count][2][L][N]; budgets: HOST int[count];
 * ws: device workspace of at least bfv_noise_budget_workspace(count) bytes. Synchronises
 * `stream`. */
int bfv_noise_budget_workspace(const bfv_ctx *ctx, size_t count, size_t *bytes);
int bfv_noise_budget(bfv_ctx *ctx, const bfv_keys *keys, const uint64_t *ct, size_t count, int *budgets,
                     void *ws, size_t ws_bytes, uintptr_t stream);

/* Decryption that allocates nothing (no paper counterpart; a library convenience). Some
 * callers cannot call cudaMalloc: it may synchronise the whole device and can fail under a
 * fixed memory reservation, so latency-critical serving threads and processes whose device
 * memory belongs to another allocator need an entry point that never allocates. This one computes exactly
 * what bfv_decrypt computes but keeps its scratch (the per-limb residues) in a fixed 4 MiB
 * device array inside the library, which every GPU that loads the library holds until the
 * process exits. Limits and rules:
 *  - count may be at most bfv_decrypt_noalloc_max_count() ciphertexts, that is
 *    floor(4 MiB / (L N 8)) (4 at N = 16384, L = 7); larger counts return
 *    BFV_ERR_OVER_BUDGET and nothing is launched — split the batch.
 *  - The array's device address is resolved when the context is created (bfv_setup, with
 *    the context's device current; a runtime query, no allocation), so the call itself queries
 *    nothing; a context created after a device reset resolves it again. The current device
 *    must be the context's device.
 *  - Every call shares the one array and it keeps the last call's contents. Nothing in it
 *    needs to start at zero (each call writes every word it reads), but calls whose work
 *    overlaps on the GPU race on it: issue them on one stream or otherwise serialise them.
 * ct: uint64[count][2][L][N], pt: uint64[count][N], device buffers; asynchronous on `stream`. */
int bfv_decrypt_noalloc_max_count(const bfv_ctx *ctx, size_t *count);
int bfv_decrypt_noalloc(bfv_ctx *ctx, const bfv_keys *keys, const uint64_t *ct, size_t count, uint64_t *pt,
                        uintptr_t stream);

/* ------------------------------------------------------------------ server side */

/* Encodes the model (Section 4.2.2): the transposed weights W^T as |Y| x ceil(f/N)
 * plaintexts (weight (k*N + s, j) in slot s of plaintext (j, k)), kept on the device in the
 * evaluation form of every ciphertext prime, and the biases b_j (added as Delta [b_j]_t).
 * W: int64[f][nY] row-major, b: int64[nY], both HOST pointers. Synchronises `stream`. */
int bfv_model_prepare(bfv_ctx *ctx, const int64_t *W, const int64_t *b, size_t f, size_t nY,
                      uintptr_t stream, bfv_model **out);
int bfv_model_free(bfv_model *model);

/* Packed product, Algorithm 1 with bias: for each pair g = i*|Y| + j,
 *   c = sum_k X[i][k] * W[j][k];  c += rot_g(c) for the log2 N Galois elements in order;
 *   c0 += Delta [b_j]_t;  c *= mask_g (one-hot at slot g mod N);  Y[g / N] += c.
 * X_ct: uint64[nX][ceil(f/N)][2][L][N] (device); Y_ct: uint64[ceil(nX*nY/N)][2][L][N].
 * Decrypting Y gives (x_i . W[:, j] + b_j) mod t in slot g mod N of output g / N.
 * ws: at least bfv_lr_scores_packed_workspace(nX) bytes. Up to `pair_chunk` pairs are
 * in flight at once (0 = the library's choice); the workspace size depends on it. */
int bfv_lr_scores_packed_workspace(const bfv_ctx *ctx, const bfv_model *model, size_t nX, size_t pair_chunk,
                                   size_t *bytes);
int bfv_lr_scores_packed(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint64_t *X_ct,
                         size_t nX, uint64_t *Y_ct, void *ws, size_t ws_bytes, size_t pair_chunk,
                         uintptr_t stream);

/* Several independent requests in one fused product (continuous batching): request r has
 * nXs[r] individuals with input ciphertexts X_cts[r] (uint64[nXs[r]][ceil(f/N)][2][L][N],
 * device) and receives its own outputs Y_cts[r] (uint64[ceil(nXs[r] |Y| / N)][2][L][N]),
 * laid out exactly as bfv_lr_scores_packed would for that request alone — the pairs of all
 * requests share every kernel launch, and each request's output is bit-identical to its
 * single-request result. 1 <= nreq <= 64; X_cts, nXs and Y_cts are HOST arrays of length
 * nreq. ws: at least bfv_lr_scores_packed_multi_workspace() bytes. */
int bfv_lr_scores_packed_multi_workspace(const bfv_ctx *ctx, const bfv_model *model, int nreq, const size_t *nXs,
                                         size_t pair_chunk, size_t *bytes);
int bfv_lr_scores_packed_multi(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, int nreq,
                               const uint64_t *const *X_cts, const size_t *nXs, uint64_t *const *Y_cts, void *ws,
                               size_t ws_bytes, size_t pair_chunk, uintptr_t stream);

/* Requests scored by DIFFERENT models of one context in one fused product (an uneven batch:
 * models with different feature counts f_r, classes |Y|_r and batch sizes): request r has
 * nXs[r] individuals with inputs X_cts[r] (uint64[nXs[r]][ceil(f_r/N)][2][L][N], device),
 * is scored by models[r] and receives Y_cts[r] (uint64[ceil(nXs[r] |Y|_r / N)][2][L][N]),
 * laid out and bit-identical as bfv_lr_scores_packed(models[r]) would give it alone. Every
 * pair of every request shares the kernel launches of Algorithm 1 (MAC, log2 N key
 * switches per pair, bias + mask, compression per request). 1 <= nreq <= 64; models, X_cts,
 * nXs and Y_cts are HOST arrays of length nreq; every model belongs to ctx. Inputs are moved
 * to evaluation form one pair chunk at a time, so the workspace holds only the inputs of
 * one chunk. ws: at least bfv_lr_scores_packed_models_workspace() bytes. */
int bfv_lr_scores_packed_models_workspace(const bfv_ctx *ctx, int nreq, const bfv_model *const *models,
                                          const size_t *nXs, size_t pair_chunk, size_t *bytes);
int bfv_lr_scores_packed_models(bfv_ctx *ctx, const bfv_keys *keys, int nreq, const bfv_model *const *models,
                                const uint64_t *const *X_cts, const size_t *nXs, uint64_t *const *Y_cts, void *ws,
                                size_t ws_bytes, size_t pair_chunk, uintptr_t stream);

/* CRT plaintext pair (Section 4.2.2): scores needing more precision than one plaintext modulus
 * are computed in two contexts with coprime moduli t0, t1 (the paper: 1073872897 and 114689)
 * and recombined: out[i] = the x with x = r0[i] mod t0, x = r1[i] mod t1, centred in
 * (-t0 t1 / 2, t0 t1 / 2]. r0, r1, out: DEVICE int64 arrays of n entries (residues in any
 * representative, e.g. bfv_decode's slots); asynchronous on `stream`. BFV_ERR_INVALID_ARG if
 * t0, t1 are not coprime or t0 t1 >= 2^62. No counterpart in the paper beyond the CRT itself. */
int bfv_crt_combine(const int64_t *r0, uint64_t t0, const int64_t *r1, uint64_t t1, size_t n, int64_t *out,
                    uintptr_t stream);

/* The same product replayed from a CUDA graph: the first call with a given set of arguments
 * (handles, pointers, sizes, chunk, stream) captures every launch of bfv_lr_scores_packed
 * into a graph and later calls launch the instantiated graph, so the host issues one call
 * per product. Same results and workspace as bfv_lr_scores_packed. While per-kernel
 * profiling is on (bfv_profile) it launches directly instead. Not thread-safe against
 * concurrent calls on the same stream; the first call must not run inside another capture. */
int bfv_lr_scores_packed_graph(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint64_t *X_ct,
                               size_t nX, uint64_t *Y_ct, void *ws, size_t ws_bytes, size_t pair_chunk,
                               uintptr_t stream);

/* Schedule of the packed product: how many pairs are in flight at once and how each of the
 * four key-switching kernels of a rotation step splits a limb over CTAs. Every schedule gives
 * bit-identical results; they differ only in speed (small pair chunks, one individual, favour
 * finer splits that fill the SMs). A split of 2 CTAs per limb takes effect at N = 16384 only:
 * at N = 32768 every limb kernel already runs on a two-CTA cluster, at N <= 8192 on one CTA.
 *   pair_chunk       pairs in flight at once, >= 1 (workspace grows with it)
 *   prep_split       1 | 2 | 3: CTAs per digit in the inverse transform of the key-switch input:
 *                    1 CTA of 512 threads, 2 CTAs of 256 threads (three per SM), 3 = two CTAs of
 *                    256 threads with twice the registers (two per SM)
 *   modup_split      2 | 4: CTAs per target limb in ModUp (each folds log2 of it stages into its loads)
 *   moddown_p_split  0 | 1 | 2 | 3 | 4: CTAs per P limb in ModDown's inverse transform: 1 CTA of 512
 *                    threads, 2 CTAs of 256 threads (three per SM), 3 = two CTAs of 512 threads,
 *                    4 = two CTAs of 256 threads with twice the registers (0: 2 when the chunk has
 *                    fewer than the SM count of pairs, else 1)
 *   moddown_split    1 | 2 | 3: CTAs per limb in ModDown's forward transform and P^-1 product:
 *                    1 CTA of 512 threads, 2 CTAs of 256 threads (three per SM), 3 = two CTAs of
 *                    256 threads with twice the registers (two per SM)
 * No counterpart in the paper (a GPU launch configuration). */
typedef struct bfv_packed_schedule {
    uint64_t pair_chunk;
    uint32_t prep_split;
    uint32_t modup_split;
    uint32_t moddown_p_split;
    uint32_t moddown_split;
} bfv_packed_schedule;

/* The schedule a product of `npairs` pairs uses when called with pair_chunk = 0: the one recorded
 * for that pair count (bfv_packed_schedule_set or an autotuner), else the one recorded for
 * npairs = 0, else the library default {2048, 1, 2, 0, 2}. */
int bfv_packed_schedule_get(const bfv_ctx *ctx, size_t npairs, bfv_packed_schedule *out);
/* Records `sched` for products of `npairs` pairs (0: every pair count without its own entry);
 * later calls and workspace queries with pair_chunk = 0 use it. BFV_ERR_INVALID_ARG if a field is
 * outside the values listed above. */
int bfv_packed_schedule_set(bfv_ctx *ctx, size_t npairs, const bfv_packed_schedule *sched);
/* bfv_lr_scores_packed with an explicit schedule (workspace: bfv_lr_scores_packed_workspace with
 * pair_chunk = sched->pair_chunk). */
int bfv_lr_scores_packed_sched(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint64_t *X_ct,
                               size_t nX, uint64_t *Y_ct, void *ws, size_t ws_bytes,
                               const bfv_packed_schedule *sched, uintptr_t stream);

/* Autotuner for the whole schedule: first the pair chunk as bfv_autotune_packed does (with the
 * default splits), then each split in turn (coordinate descent over prep_split, modup_split,
 * moddown_p_split, moddown_split), every candidate timed with CUDA events after a warm-up run on
 * the caller's inputs. The fastest schedule is recorded for this number of pairs (as
 * bfv_packed_schedule_set would) and returned in *best with its time in *best_ms. Y_ct receives
 * the product. Synchronises `stream`. No counterpart in the paper. */
int bfv_autotune_packed_schedule(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint64_t *X_ct,
                                 size_t nX, uint64_t *Y_ct, void *ws, size_t ws_bytes, uintptr_t stream,
                                 bfv_packed_schedule *best, double *best_ms);

/* Autotuner for the packed product's pair chunk (how many pairs are in flight at once):
 * runs the product on the caller's inputs for chunk sizes 128 .. 16384 that fit in ws_bytes,
 * times each with CUDA events after a warm-up run, and records the fastest for this number
 * of pairs in the context; later calls and workspace queries with pair_chunk = 0 use it
 * (size workspaces after tuning). Y_ct receives the product. Synchronises `stream`. */
int bfv_autotune_packed(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint64_t *X_ct, size_t nX,
                        uint64_t *Y_ct, void *ws, size_t ws_bytes, uintptr_t stream, size_t *best_chunk,
                        double *best_ms);

/* Standard product (Section 5.2.3): ciphertext f of X_ct holds feature f of individual i in
 * slot i (nX <= N); output j = sum_f w[f][j] X_ct[f] + Delta [b_j]_t, weights as integer
 * scalars (|w| < 2^31 and |w| f 2^ceil(bits/2) < 2^63, else BFV_ERR_BAD_PARAMS).
 * X_ct: uint64[f][2][L][N]; Y_ct: uint64[nY][2][L][N]. ws: device workspace of at least
 * bfv_lr_scores_standard_workspace() bytes (per-split partial sums). A bounded wait inside
 * the streaming kernel that runs out sets the context's error word (see bfv_check_error). */
int bfv_lr_scores_standard_workspace(const bfv_ctx *ctx, const bfv_model *model, size_t *bytes);
int bfv_lr_scores_standard(bfv_ctx *ctx, const bfv_model *model, const uint64_t *X_ct, size_t nX,
                           uint64_t *Y_ct, void *ws, size_t ws_bytes, uintptr_t stream);

/* Synchronises the device, returns the context's device error word in *flags (bit 0: a
 * bounded wait in a kernel ran out; bit 1, bounds-checked build only: an access outside the
 * call's buffers was skipped) and clears it. Returns BFV_ERR_TIMEOUT if it was set. */
int bfv_check_error(bfv_ctx *ctx, int *flags);

/* Launch options of a context (no counterpart in the paper; speed only, every value gives the
 * same bits). BFV_OPT_ENCRYPT_SPLIT: how the encryption kernel splits a limb at N = 16384: 1 (one
 * 512-thread CTA), 2 (a cluster of two 256-thread CTAs, two CTAs per SM at 128 registers) or 3
 * (the same cluster, three CTAs per SM at 80 registers; the default); other rings ignore it. BFV_OPT_STANDARD_KERNEL: the standard product with int8-range
 * weights (|w| <= 127) runs its byte-plane contraction on the tensor cores (0, the default:
 * tcgen05.mma kind::f16, exact f32 sums moved to int64 every 256 features) or on dp4a (1); wider
 * weights always take the 32 x 32 -> 64-bit kernel. bfv_get_option writes the current value to
 * *value. */
#define BFV_OPT_ENCRYPT_SPLIT 1
#define BFV_OPT_STANDARD_KERNEL 2
int bfv_set_option(bfv_ctx *ctx, int option, int value);
int bfv_get_option(const bfv_ctx *ctx, int option, int *value);

/* Failure injection for tests (host-side switch, no fault): with what =
 * BFV_INJECT_STREAM_STALL and value = n > 0 (a multiple of 16), the first pipeline stage of
 * every standard-product CTA waits for n bytes that are never sent, so its bounded wait runs
 * out after a short poll limit, the CTA drains its copies, sets the error word and returns
 * (the output is then invalid; the tensor-core kernel's first stage instead waits for an
 * arrival that never comes). value = 0 turns it off. */
#define BFV_INJECT_STREAM_STALL 1
/* With what = BFV_INJECT_BOUNDS_SHRINK and value = n (a multiple of 8), a bounds-checked build
 * (bfv_bounds_checked() = 1) registers every caller buffer of later calls n bytes shorter than
 * the call implies, so the last accesses into each are reported as out of bounds (skipped, bit 1
 * of the error word) although they stay inside the real buffer. The release build returns
 * BFV_ERR_INVALID_ARG for it. */
#define BFV_INJECT_BOUNDS_SHRINK 2
int bfv_debug_inject(bfv_ctx *ctx, int what, int value);

/* 1 if this library was built with bounds checks (-DBFV_BOUNDS), else 0. In that build every
 * global-memory access of every kernel is checked against the buffers its call may touch (the
 * context's tables, keys, models, and the caller's buffers at the sizes the call implies); an
 * access outside them is skipped (a load reads 0) and sets bit 1 (value 2) of the context's error
 * word (bfv_check_error), so an indexing mistake is reported instead of faulting. Calls of a
 * bounds-checked build must not overlap on the GPU (the table is one per process). No
 * counterpart in the paper (a debugging aid). */
int bfv_bounds_checked(void);

/* ------------------------------------------------------------------ whole-protocol calls */

/* One pass of the private inference protocol (Section 4.2.2, Fig. 2) over a batch, all on
 * the device: bfv_encode_features -> bfv_encrypt (seed, object ids 0 .. nX*ceil(f/N)-1) ->
 * bfv_lr_scores_packed -> bfv_decrypt -> bfv_decode, leaving score(i, j) = (x_i . W[:, j] +
 * b_j) mod t at scores[i*nY + j]. X: uint8[nX][f] (device), scores: int64[nX][nY] (device).
 * ws: at least bfv_lr_predict_packed_workspace(nX, pair_chunk) bytes. */
int bfv_lr_predict_packed_workspace(const bfv_ctx *ctx, const bfv_model *model, size_t nX, size_t pair_chunk,
                                    size_t *bytes);
int bfv_lr_predict_packed(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint8_t *X, size_t nX,
                          uint64_t seed, int64_t *scores, void *ws, size_t ws_bytes, size_t pair_chunk,
                          uintptr_t stream);

/* The same with HOST buffers: copies X_host (uint8[nX][f]; pinned memory gives full copy speed)
 * to the device inside the call, runs bfv_lr_predict_packed, copies the scores back to
 * scores_host (int64[nX][nY]) and synchronises `stream`. Same workspace size. */
int bfv_lr_predict_packed_host(bfv_ctx *ctx, const bfv_keys *keys, const bfv_model *model, const uint8_t *X_host,
                               size_t nX, uint64_t seed, int64_t *scores_host, void *ws, size_t ws_bytes,
                               size_t pair_chunk, uintptr_t stream);

/* ------------------------------------------------------------------ diagnostics */

/* Copies pair g's ciphertext out of a packed-product workspace, in coefficient form
 * (uint64[2][L][N]): after a bfv_lr_scores_packed call whose last chunk contained g this is
 * the masked pair ciphertext before compression. For parity tests at full size. */
int bfv_lr_packed_pair_from_workspace(bfv_ctx *ctx, const bfv_model *model, size_t nX, size_t pair_chunk,
                                      const void *ws, size_t g, uint64_t *ct_out, uintptr_t stream);

/* Number of kernel launches the library issued since bfv_setup (for launch accounting). */
int bfv_launch_count(const bfv_ctx *ctx, uint64_t *count);

/* Per-kernel timing with CUDA events recorded around every launch of the library's kernels on
 * the launching stream (enable = 1 starts recording, 0 stops). bfv_profile_read synchronises
 * the recorded events and returns, for kernel kind `kind` (BFV_K_*), the number of launches
 * and their summed device time in milliseconds since the last read of that kind, then clears
 * it. Recording adds two event records per launch. */
#define BFV_K_NTT 0
#define BFV_K_KS_PREP 1
#define BFV_K_KS_MODUP 2
#define BFV_K_KS_MODDOWN_P 3
#define BFV_K_KS_MODDOWN 4
#define BFV_K_MAC 5
#define BFV_K_BIAS_MASK 6
#define BFV_K_COMPRESS 7
#define BFV_K_ENCRYPT 8
#define BFV_K_DECRYPT 9
#define BFV_K_ENCODE 10
#define BFV_K_STANDARD 11
#define BFV_K_COUNT 12
int bfv_profile(bfv_ctx *ctx, int enable);
int bfv_profile_read(bfv_ctx *ctx, int kind, uint64_t *launches, double *total_ms);

#ifdef __cplusplus
}
#endif
#endif /* BFV_LR_H */
