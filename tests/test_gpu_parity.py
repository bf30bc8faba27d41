"""GPU parity: every stage of the CUDA path against the CPU oracle, bit for bit.

Ciphertexts are compared in coefficient form (the boundary representation); decrypted
scores are also compared with the closed form (x.W + b) mod t. At the full workload sizes
the oracle computes sampled pairs, ciphertexts and coefficients one by one."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2204_05496_gb300 as bfv


def dev(a):
    """numpy (u)int64 array -> CUDA int64 tensor holding the same 64-bit words."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def host(t):
    return bfv.as_u64(t)


def oracle_columns(P, okeys, X, seed, f0=0, f1=None):
    """The oracle's own encryptions of feature columns f0..f1-1 of X (slot i = individual i),
    ciphertext f under object f: the inputs of the standard product."""
    f1 = X.shape[1] if f1 is None else f1
    want = np.zeros((f1 - f0, P.N), dtype=np.int64)
    want[:, :X.shape[0]] = X[:, f0:f1].T
    return oracle.encrypt(P, okeys, oracle.encode(P, want), seed=seed, obj0=f0)


# ----------------------------------------------------------------------------- tiny (N = 4096)

@pytest.fixture(scope="module")
def tiny():
    w = synth.WORKLOADS["tiny-1"]
    ctx = bfv.Context.from_shape(w.params)
    keys = ctx.keygen(w.seed_keys)
    P = oracle.Params.from_shape(w.params)
    okeys = oracle.keygen(P, w.seed_keys)
    return ctx, keys, P, okeys


def test_parameters_match_oracle(tiny):
    ctx, _, P, _ = tiny
    assert ctx.primes == P.qs
    assert ctx.omega == P.omega
    assert ctx.delta_mod_q == [P.delta % q for q in P.q]
    assert bfv.gaussian_table(16, 5) == P.cdt


def test_keygen_parity(tiny):
    ctx, keys, P, okeys = tiny
    sk, pk, gk = ctx.keys_export(keys)
    assert np.array_equal(sk.cpu().numpy(), okeys.sk)
    assert np.array_equal(host(pk), okeys.pk)
    assert np.array_equal(host(gk), okeys.gk_coeff)


def test_encode_decode_parity(tiny):
    ctx, _, P, _ = tiny
    v = synth.slots(21, 5, P.N, P.t)
    v[0, :7] = [-1, -P.t, 3 * P.t + 2, 0, P.t - 1, -(P.t // 2), 2 ** 40]   # any integers, taken mod t
    pt = ctx.encode(dev(v))
    assert np.array_equal(host(pt), oracle.encode(P, v))
    got = ctx.decode(pt).cpu().numpy()
    assert np.array_equal(got, np.mod(v, P.t))


def test_encode_features_parity(tiny):
    ctx, _, P, _ = tiny
    X = synth.features(5, 3, 9000, 0.3)                     # f = 9000: K = 3, ragged last chunk
    pt = ctx.encode_features(dev(X).to(torch.uint8))
    assert pt.shape == (3, 3, P.N)
    assert np.array_equal(host(pt), oracle.encode(P, oracle.pack_inputs(P, X).reshape(-1, P.N)).reshape(3, 3, P.N))
    cols = ctx.encode_feature_columns(dev(X).to(torch.uint8))
    want = np.zeros((9000, P.N), dtype=np.int64)
    want[:, :3] = X.T
    assert np.array_equal(host(cols)[:50], oracle.encode(P, want[:50]))
    assert np.array_equal(host(cols)[-7:], oracle.encode(P, want[-7:]))


def test_encrypt_parity(tiny):
    ctx, keys, P, okeys = tiny
    v = synth.slots(22, 6, P.N, P.t)
    m = oracle.encode(P, v)
    ct = ctx.encrypt(keys, dev(m), seed=777, obj0=40)
    assert np.array_equal(host(ct), oracle.encrypt(P, okeys, m, seed=777, obj0=40))
    assert ctx.encrypt(keys, dev(m[:0]), seed=1).numel() == 0                 # empty batch


def test_decrypt_parity(tiny):
    ctx, keys, P, okeys = tiny
    v = synth.slots(23, 3, P.N, P.t)
    ct = oracle.encrypt(P, okeys, oracle.encode(P, v), seed=5)
    # plus a ciphertext of arbitrary residues: exact rounding must agree everywhere
    rng = np.random.default_rng(3)
    junk = np.stack([np.stack([rng.integers(0, q, P.N, dtype=np.uint64) for q in P.q]) for _ in range(2)])[None]
    allct = np.concatenate([ct, junk])
    pt = ctx.decrypt(keys, dev(allct))
    assert np.array_equal(host(pt), oracle.decrypt(P, okeys.sk, allct))
    assert np.array_equal(host(pt)[:3], oracle.encode(P, v))


@pytest.mark.parametrize("name", ["tiny-1", "tiny-16"])
def test_packed_parity_tiny(name, tiny):
    ctx, keys, P, okeys = tiny
    w = synth.WORKLOADS[name]
    X, W, b = synth.workload_inputs(w)
    X_ct, _, Y = oracle.packed_pipeline(P, okeys, X, W, b, w.seed_enc)
    model = ctx.model_prepare(W, b)
    Yg = ctx.lr_scores_packed(keys, model, dev(X_ct))
    assert np.array_equal(host(Yg), Y)
    # ragged chunking of the pairs gives the same bits
    Yc = ctx.lr_scores_packed(keys, model, dev(X_ct), pair_chunk=5)
    assert np.array_equal(host(Yc), Y)
    slots = ctx.decode(ctx.decrypt(keys, Yg)).cpu().numpy()
    got = bfv.unpack_packed_scores(P.N, slots, X.shape[0], W.shape[1])
    assert np.array_equal(got, oracle.expected_scores(X, W, b, P.t))


def test_packed_graph_replay_and_autotune_tiny(tiny):
    ctx, keys, P, okeys = tiny
    w = synth.WORKLOADS["tiny-16"]
    X, W, b = synth.workload_inputs(w)
    X_ct, _, Y = oracle.packed_pipeline(P, okeys, X, W, b, w.seed_enc)
    model = ctx.model_prepare(W, b)
    Xd = dev(X_ct)
    ws = torch.empty(ctx.packed_workspace(model, 16, 0), dtype=torch.uint8, device="cuda")
    out = ctx.lr_scores_packed_graph(keys, model, Xd, ws=ws)          # captures
    n0 = ctx.launch_count()
    out.zero_()
    ctx.lr_scores_packed_graph(keys, model, Xd, out=out, ws=ws)      # a new key (out differs) ...
    ctx.lr_scores_packed_graph(keys, model, Xd, out=out, ws=ws)      # ... and its replay
    torch.cuda.synchronize()
    assert np.array_equal(host(out), Y)
    assert ctx.launch_count() > n0
    big = torch.empty(ctx.packed_workspace(model, 16, 128), dtype=torch.uint8, device="cuda")
    chunk, ms = ctx.autotune_packed(keys, model, Xd, big)
    assert chunk == 128 and ms > 0                                   # 128 pairs: one chunk holds all
    Yt = ctx.lr_scores_packed(keys, model, Xd, ws=big)               # chunk 0 -> the tuned chunk
    assert np.array_equal(host(Yt), Y)


def test_packed_pair_states_tiny(tiny):
    ctx, keys, P, okeys = tiny
    w = synth.WORKLOADS["tiny-16"]
    X, W, b = synth.workload_inputs(w)
    X_ct, W_pt, Y, pairs = oracle.packed_pipeline(P, okeys, X, W, b, w.seed_enc, return_pairs=True)
    model = ctx.model_prepare(W, b)
    nX = X.shape[0]
    ws = torch.empty(ctx.packed_workspace(model, nX, 0), dtype=torch.uint8, device="cuda")
    ctx.lr_scores_packed(keys, model, dev(X_ct), ws=ws)
    for g in (0, 77, nX * W.shape[1] - 1):
        got = ctx.packed_pair_from_workspace(model, nX, 0, ws, g)
        assert np.array_equal(host(got), pairs[g])


def test_end_to_end_on_gpu_tiny(tiny):
    ctx, keys, P, okeys = tiny
    w = synth.WORKLOADS["tiny-16"]
    X, W, b = synth.workload_inputs(w)
    pt = ctx.encode_features(dev(X).to(torch.uint8))
    X_ct = ctx.encrypt(keys, pt.reshape(-1, P.N), seed=w.seed_enc).reshape(X.shape[0], -1, 2, P.L, P.N)
    oX_ct, _, oY = oracle.packed_pipeline(P, okeys, X, W, b, w.seed_enc)
    assert np.array_equal(host(X_ct), oX_ct)
    model = ctx.model_prepare(W, b)
    Y = ctx.lr_scores_packed(keys, model, X_ct)
    assert np.array_equal(host(Y), oY)
    scores = bfv.unpack_packed_scores(P.N, ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy(), X.shape[0], W.shape[1])
    assert np.array_equal(scores, oracle.expected_scores(X, W, b, P.t))


def test_packed_several_outputs_tiny(tiny):
    # 520 individuals x 8 classes = 4160 pairs > N = 4096: two output ciphertexts, the second
    # holding 64 pairs; closed form for every pair, bit-exact pairs sampled in the last chunk
    ctx, keys, P, okeys = tiny
    rng = np.random.default_rng(17)
    X = (rng.random((520, 700)) < 0.05).astype(np.uint8)
    W = rng.integers(-127, 128, (700, 8))
    b = rng.integers(-127, 128, 8)
    pt = ctx.encode_features(dev(X).to(torch.uint8))
    X_ct = ctx.encrypt(keys, pt.reshape(-1, P.N), seed=9).reshape(520, 1, 2, P.L, P.N)
    model = ctx.model_prepare(W, b)
    chunk = 1500
    ws = torch.empty(ctx.packed_workspace(model, 520, chunk), dtype=torch.uint8, device="cuda")
    Y = ctx.lr_scores_packed(keys, model, X_ct, ws=ws, pair_chunk=chunk)
    assert Y.shape[0] == 2
    slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
    assert np.array_equal(bfv.unpack_packed_scores(P.N, slots, 520, 8), oracle.expected_scores(X, W, b, P.t))
    assert not slots.reshape(-1)[4160:].any()
    W_pt = oracle.encode(P, oracle.pack_weights(P, W).reshape(-1, P.N)).reshape(8, 1, P.N)
    for g in (3000, 4100, 4159):
        i, j = divmod(g, 8)
        xo = oracle.encrypt(P, okeys, oracle.encode(P, oracle.pack_inputs(P, X[i:i + 1])[0]), seed=9, obj0=i)
        assert np.array_equal(host(X_ct[i]), xo)
        c = oracle.pair_rotsum(P, okeys, xo, W_pt[j])
        want = oracle.pair_bias_mask(P, c, int(b[j]), g % P.N)
        assert np.array_equal(host(ctx.packed_pair_from_workspace(model, 520, chunk, ws, g)), want)


def test_standard_parity_tiny(tiny):
    ctx, keys, P, okeys = tiny
    w = synth.WORKLOADS["tiny-16"]
    X, W, b = synth.workload_inputs(w)
    cols = ctx.encode_feature_columns(dev(X).to(torch.uint8))
    X_ct = ctx.encrypt(keys, cols, seed=w.seed_enc)
    model = ctx.model_prepare(W, b)
    Y = ctx.lr_scores_standard(model, X_ct, X.shape[0])
    oX_ct = oracle_columns(P, okeys, X, w.seed_enc)
    assert np.array_equal(host(X_ct), oX_ct)
    oY = oracle.lr_standard(P, oX_ct, W, b)
    assert np.array_equal(host(Y), oY)
    slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
    assert np.array_equal(slots[:, :X.shape[0]].T, oracle.expected_scores(X, W, b, P.t))
    # the encryption of a few feature columns matches the oracle
    want = np.zeros((3, P.N), dtype=np.int64)
    want[:, :X.shape[0]] = X[:, [0, 500, 999]].T
    oc = oracle.encrypt(P, okeys, oracle.encode(P, want[0:1]), seed=w.seed_enc, obj0=0)
    assert np.array_equal(host(X_ct[0:1]), oc)
    oc = oracle.encrypt(P, okeys, oracle.encode(P, want[2:3]), seed=w.seed_enc, obj0=999)
    assert np.array_equal(host(X_ct[999:1000]), oc)


def test_standard_wide_weights_parity(tiny):
    # weights outside the int8 range take the 32 x 32 -> 64 multiply-add kernel
    ctx, keys, P, okeys = tiny
    rng = np.random.default_rng(6)
    X = (rng.random((9, 300)) < 0.3).astype(np.uint8)
    W = rng.integers(-3000, 3001, (300, 19))                   # 19 classes: two class groups
    b = rng.integers(-3000, 3001, 19)
    model = ctx.model_prepare(W, b)
    X_ct = ctx.encrypt(keys, ctx.encode_feature_columns(dev(X).to(torch.uint8)), seed=4)
    Y = ctx.lr_scores_standard(model, X_ct, 9)
    assert ctx.check_error() == 0
    oX_ct = oracle_columns(P, okeys, X, 4)
    assert np.array_equal(host(X_ct), oX_ct)
    assert np.array_equal(host(Y), oracle.lr_standard(P, oX_ct, W, b))
    slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
    assert np.array_equal(slots[:, :9].T, oracle.expected_scores(X, W, b, P.t))


def test_calls_on_a_side_stream_tiny(tiny):
    """Encrypt, packed product and decrypt on a non-default stream with every output and
    workspace allocated by the binding: each call's allocations follow that stream, and the
    results equal the oracle's."""
    ctx, keys, P, okeys = tiny
    w = synth.WORKLOADS["tiny-16"]
    X, W, b = synth.workload_inputs(w)
    oX_ct, _, oY = oracle.packed_pipeline(P, okeys, X, W, b, w.seed_enc)
    model = ctx.model_prepare(W, b)
    pt = ctx.encode_features(dev(X).to(torch.uint8))
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    X_ct = ctx.encrypt(keys, pt.reshape(-1, P.N), seed=w.seed_enc, stream=s).reshape(X.shape[0], -1, 2, P.L, P.N)
    Y = ctx.lr_scores_packed(keys, model, X_ct, stream=s)
    m = ctx.decrypt(keys, Y, stream=s)
    junk = torch.empty(64 << 20, dtype=torch.uint8, device="cuda").fill_(0xA5)   # default-stream traffic
    s.synchronize()
    torch.cuda.synchronize()
    del junk
    assert np.array_equal(host(X_ct), oX_ct) and np.array_equal(host(Y), oY)
    assert np.array_equal(host(m), oracle.decrypt(P, okeys.sk, oY))


def test_noise_budget_parity_tiny(tiny):
    """bfv_noise_budget against the oracle: fresh encryptions, the outputs of a packed product
    (the oracle's own pipeline) and arbitrary residues, whose noise fills the modulus."""
    ctx, keys, P, okeys = tiny
    w = synth.WORKLOADS["tiny-16"]
    X, W, b = synth.workload_inputs(w)
    oX_ct, _, oY = oracle.packed_pipeline(P, okeys, X, W, b, w.seed_enc)
    rng = np.random.default_rng(12)
    junk = np.stack([np.stack([rng.integers(0, q, P.N, dtype=np.uint64) for q in P.q]) for _ in range(2)])[None]
    cts = np.concatenate([oX_ct.reshape(-1, 2, P.L, P.N)[:5], oY, junk])
    got = ctx.noise_budget(keys, dev(cts))
    assert got == oracle.noise_budget(P, okeys.sk, cts)
    assert got[-1] == 0 and min(got[:-1]) > 0 and got[5] < got[0]


def test_stream_stall_reports_timeout_and_context_recovers(tiny):
    # failure injection on the host side: the first pipeline stage waits for 16 bytes that are
    # never sent; the bounded wait runs out, the kernel sets the error word and returns
    ctx, keys, P, okeys = tiny
    rng = np.random.default_rng(5)
    X = (rng.random((4, 200)) < 0.3).astype(np.uint8)
    W = rng.integers(-127, 128, (200, 3))
    b = rng.integers(-127, 128, 3)
    model = ctx.model_prepare(W, b)
    X_ct = ctx.encrypt(keys, ctx.encode_feature_columns(dev(X).to(torch.uint8)), seed=3)
    assert ctx.check_error() == 0
    bfv._call("bfv_debug_inject", ctx.handle, 1, 16)
    try:
        ctx.lr_scores_standard(model, X_ct, 4)
        assert ctx.check_error() & 1
    finally:
        bfv._call("bfv_debug_inject", ctx.handle, 1, 0)
    Y = ctx.lr_scores_standard(model, X_ct, 4)
    assert ctx.check_error() == 0
    slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
    assert np.array_equal(slots[:, :4].T, oracle.expected_scores(X, W, b, P.t))
    oX_ct = oracle_columns(P, okeys, X, 3)
    assert np.array_equal(host(X_ct), oX_ct)
    assert np.array_equal(host(Y), oracle.lr_standard(P, oX_ct, W, b))


def test_invalid_arguments_are_rejected(tiny):
    ctx, keys, P, _ = tiny
    with pytest.raises(bfv.BfvError):
        bfv.Context(5000, 3, 36, 65537)                      # N not supported
    model = ctx.model_prepare(np.ones((10, 2), dtype=np.int64), np.zeros(2, dtype=np.int64))
    X_ct = torch.zeros((1, 1, 2, P.L, P.N), dtype=torch.int64, device="cuda")
    tiny_ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(bfv.BfvError) as e:
        bfv._call("bfv_lr_scores_packed", ctx.handle, keys.handle, model.handle, bfv._ptr(X_ct), 1,
                  bfv._ptr(X_ct), bfv._ptr(tiny_ws), 16, 0, 0)
    assert e.value.code == bfv.BFV_ERR_OVER_BUDGET
    cols = torch.zeros((10, 2, P.L, P.N), dtype=torch.int64, device="cuda")
    with pytest.raises(bfv.BfvError):
        ctx.lr_scores_standard(model, cols, P.N + 1)         # more individuals than slots


def test_binding_checks_buffers_before_the_call(tiny):
    """The C calls read and write exactly the bytes their sizes imply; the binding refuses a
    caller tensor of the wrong shape, element size or memory before any pointer is passed on."""
    ctx, keys, P, _ = tiny
    model = ctx.model_prepare(np.ones((10, 2), dtype=np.int64), np.zeros(2, dtype=np.int64))
    X = torch.zeros((3, 10), dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        ctx.predict_packed(keys, model, X[:, :9], seed=1)                       # one feature short
    with pytest.raises(ValueError):
        ctx.predict_packed(keys, model, X.to(torch.int64), seed=1)              # 8-byte features
    with pytest.raises(ValueError):
        ctx.predict_packed(keys, model, X, seed=1, out=torch.empty((3, 1), dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        ctx.predict_packed_host(keys, model, np.zeros((3, 9), dtype=np.uint8), seed=1)
    with pytest.raises(ValueError):
        ctx.predict_packed_host(keys, model, X, seed=1)                         # device memory
    X_ct = torch.zeros((1, 1, 2, P.L, P.N), dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        ctx.lr_scores_packed(keys, model, X_ct[:, :, :, :2])                    # two limbs of three
    with pytest.raises(ValueError):
        ctx.lr_scores_packed(keys, model, X_ct, out=torch.empty((2, 2, P.L, P.N), dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):                                             # host workspace
        ctx.lr_scores_packed(keys, model, X_ct, ws=torch.empty(ctx.packed_workspace(model, 1), dtype=torch.uint8))
    with pytest.raises(ValueError):
        ctx.packed_pair_from_workspace(model, 1, 0, torch.empty(16, dtype=torch.uint8, device="cuda"), 0)
    with pytest.raises(ValueError):
        ctx.encrypt(keys, torch.zeros(P.N + 1, dtype=torch.int64, device="cuda"), seed=1)
    with pytest.raises(ValueError):
        ctx.decrypt(keys, X_ct[0, 0, :, :2])
    torch.cuda.synchronize()
    assert ctx.predict_packed(keys, model, X[:0], seed=1).shape == (0, 2)
    assert ctx.lr_scores_packed(keys, model, X_ct[:0]).shape[0] == 0


def test_predict_packed_whole_protocol_tiny(tiny):
    """The whole-protocol calls (encode, encrypt, Algorithm 1, decrypt, decode in one C call), on
    device and on host buffers, over 700 individuals x 5,000 features x 8 classes: 5,600 pairs
    in two output ciphertexts and two plaintexts per individual. Every score against the closed
    form, for two encryption seeds and a chunked plan."""
    ctx, keys, P, _ = tiny
    rng = np.random.default_rng(97)
    nX, f, nY = 700, 5000, 8
    X = (rng.random((nX, f)) < 0.05).astype(np.uint8)
    W = rng.integers(-127, 128, (f, nY))
    b = rng.integers(-127, 128, nY)
    model = ctx.model_prepare(W, b)
    want = oracle.expected_scores(X, W, b, P.t)
    assert np.array_equal(ctx.predict_packed(keys, model, dev(X), seed=98).cpu().numpy(), want)
    assert np.array_equal(ctx.predict_packed_host(keys, model, X, seed=99, pair_chunk=1024), want)
    pinned = torch.from_numpy(X).pin_memory()
    out = torch.empty((nX, nY), dtype=torch.int64).pin_memory()
    ctx.predict_packed_host(keys, model, pinned, seed=100, out=out)
    assert np.array_equal(out.numpy(), want)


# ----------------------------------------------------------------------------- paper scale (N = 16384, L = 7)

@pytest.fixture(scope="module")
def paper():
    w = synth.WORKLOADS["single-40k"]
    ctx = bfv.Context.from_shape(w.params)
    keys = ctx.keygen(w.seed_keys)
    P = oracle.Params.from_shape(w.params)
    okeys = oracle.keygen(P, w.seed_keys)
    return ctx, keys, P, okeys


def test_paper_keys_match(paper):
    ctx, keys, P, okeys = paper
    sk, pk, gk = ctx.keys_export(keys)
    assert ctx.primes == P.qs
    assert np.array_equal(sk.cpu().numpy(), okeys.sk)
    assert np.array_equal(host(pk), okeys.pk)
    assert np.array_equal(host(gk), okeys.gk_coeff)


def test_noise_budget_paper_scale(paper):
    # fresh encryptions at N = 16384, L = 7: the GPU's ciphertexts equal the oracle's, and so
    # do their budgets
    ctx, keys, P, okeys = paper
    m = oracle.encode(P, synth.slots(41, 2, P.N, P.t))
    ct = ctx.encrypt(keys, dev(m), seed=42)
    oct_ = oracle.encrypt(P, okeys, m, seed=42)
    assert np.array_equal(host(ct), oct_)
    got = ctx.noise_budget(keys, ct)
    assert got == oracle.noise_budget(P, okeys.sk, oct_) and min(got) > 300


def test_single_individual_packed_bit_exact(paper):
    ctx, keys, P, okeys = paper
    w = synth.WORKLOADS["single-40k"]
    X, W, b = synth.workload_inputs(w)
    pt = ctx.encode_features(dev(X).to(torch.uint8))
    X_ct = ctx.encrypt(keys, pt.reshape(-1, P.N), seed=w.seed_enc).reshape(1, 3, 2, P.L, P.N)
    oX_ct, _, oY = oracle.packed_pipeline(P, okeys, X, W, b, w.seed_enc)
    assert np.array_equal(host(X_ct), oX_ct)
    model = ctx.model_prepare(W, b)
    Y = ctx.lr_scores_packed(keys, model, X_ct)
    assert np.array_equal(host(Y), oY)
    scores = bfv.unpack_packed_scores(P.N, ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy(), 1, 16)
    assert np.array_equal(scores, oracle.expected_scores(X, W, b, P.t))


def test_batch512_packed_full_size(paper):
    """The benchmark's workload and launch configuration: 512 individuals x 40,000 features x 16
    classes. Every score against the closed form; sampled pairs bit-exact against the oracle."""
    ctx, keys, P, okeys = paper
    w = synth.WORKLOADS["batch512-40k"]
    X, W, b = synth.workload_inputs(w)
    pt = ctx.encode_features(dev(X).to(torch.uint8))
    X_ct = ctx.encrypt(keys, pt.reshape(-1, P.N), seed=w.seed_enc).reshape(512, 3, 2, P.L, P.N)
    model = ctx.model_prepare(W, b)
    ws = torch.empty(ctx.packed_workspace(model, 512, 0), dtype=torch.uint8, device="cuda")
    Y = ctx.lr_scores_packed(keys, model, X_ct, ws=ws)
    assert Y.shape[0] == 1
    scores = bfv.unpack_packed_scores(P.N, ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy(), 512, 16)
    assert np.array_equal(scores, oracle.expected_scores(X, W, b, P.t))
    W_pt = oracle.encode(P, oracle.pack_weights(P, W).reshape(-1, P.N)).reshape(16, 3, P.N)
    for g in (6144, 7001, 8191):                      # pairs of the last chunk of 2048
        i, j = divmod(g, 16)
        xo = oracle.encrypt(P, okeys, oracle.encode(P, oracle.pack_inputs(P, X[i:i + 1])[0]), seed=w.seed_enc,
                            obj0=3 * i)
        assert np.array_equal(host(X_ct[i]), xo)
        c = oracle.pair_rotsum(P, okeys, xo, W_pt[j])
        want = oracle.pair_bias_mask(P, c, int(b[j]), g % P.N)
        assert np.array_equal(host(ctx.packed_pair_from_workspace(model, 512, 0, ws, g)), want)


def test_single_individual_standard_full_size(paper):
    """Standard product at 40,000 features (40,000 ciphertexts, 73 GB): closed form for the
    decrypted scores, sampled output coefficients and sampled input ciphertexts bit-exact."""
    ctx, keys, P, okeys = paper
    w = synth.WORKLOADS["single-40k"]
    X, W, b = synth.workload_inputs(w)
    cols = ctx.encode_feature_columns(dev(X).to(torch.uint8))
    X_ct = torch.empty((40000, 2, P.L, P.N), dtype=torch.int64, device="cuda")
    ws = torch.empty(ctx.encrypt_workspace(4000), dtype=torch.uint8, device="cuda")
    for f0 in range(0, 40000, 4000):
        ctx.encrypt(keys, cols[f0:f0 + 4000], seed=w.seed_enc, obj0=f0, out=X_ct[f0:f0 + 4000], ws=ws)
    model = ctx.model_prepare(W, b)
    Y = ctx.lr_scores_standard(model, X_ct, 1)
    slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
    assert np.array_equal(slots[:, 0], oracle.expected_scores(X, W, b, P.t)[0])
    for f in (0, 23456, 39999):
        want = np.zeros((1, P.N), dtype=np.int64)
        want[0, 0] = X[0, f]
        assert np.array_equal(host(X_ct[f:f + 1]), oracle.encrypt(P, okeys, oracle.encode(P, want), seed=w.seed_enc, obj0=f))
    # bit-exact products on a block of 64 features whose inputs the oracle encrypts itself
    # (the same kernel and launch shape; the full-size result is pinned by the closed form)
    f0, f1 = 23456, 23520
    oX = oracle_columns(P, okeys, X, w.seed_enc, f0, f1)
    assert np.array_equal(host(X_ct[f0:f1]), oX)
    sub = ctx.model_prepare(W[f0:f1], b)
    Ys = ctx.lr_scores_standard(sub, X_ct[f0:f1], 1)
    assert np.array_equal(host(Ys), oracle.lr_standard(P, oX, W[f0:f1], b))


# ----------------------------------------------------------------------------- edge cases

def test_max_prime_bits_packed_parity():
    """59-bit primes, the largest allowed: the unreduced forward transforms reach 32q < 2^64 and
    the unreduced key sums 2Lq; ciphertexts must still match the oracle bit for bit."""
    shape = synth.BfvShape(N=4096, L=3, prime_bits=59, t=65537)
    ctx = bfv.Context.from_shape(shape)
    keys = ctx.keygen(91)
    P = oracle.Params.from_shape(shape)
    okeys = oracle.keygen(P, 91)
    assert ctx.primes == P.qs and all(q.bit_length() == 59 for q in P.qs)
    rng = np.random.default_rng(92)
    X = (rng.random((3, 5000)) < 0.3).astype(np.uint8)      # K = 2
    W = rng.integers(-127, 128, (5000, 5))
    b = rng.integers(-127, 128, 5)
    oX_ct, _, oY = oracle.packed_pipeline(P, okeys, X, W, b, 93)
    pt = ctx.encode_features(dev(X).to(torch.uint8))
    X_ct = ctx.encrypt(keys, pt.reshape(-1, P.N), seed=93).reshape(3, 2, 2, P.L, P.N)
    assert np.array_equal(host(X_ct), oX_ct)
    Y = ctx.lr_scores_packed(keys, ctx.model_prepare(W, b), X_ct)
    assert np.array_equal(host(Y), oY)
    slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
    assert np.array_equal(bfv.unpack_packed_scores(P.N, slots, 3, 5), oracle.expected_scores(X, W, b, P.t))


def test_degenerate_shapes_packed_tiny(tiny):
    """One feature and one class (f = 1, |Y| = 1), and pair counts exactly filling the N slots of
    one output (nX |Y| = N) and one past it (a second output holding a single pair)."""
    ctx, keys, P, okeys = tiny
    rng = np.random.default_rng(94)
    X = np.ones((2, 1), dtype=np.uint8)
    W = np.array([[-127]])
    b = np.array([127])
    oX_ct, _, oY = oracle.packed_pipeline(P, okeys, X, W, b, 95)
    Y = ctx.lr_scores_packed(keys, ctx.model_prepare(W, b), dev(oX_ct))
    assert Y.shape[0] == 1 and np.array_equal(host(Y), oY)
    for nX in (P.N // 4, P.N // 4 + 1):                          # |Y| = 4: 4096 and 4100 pairs
        X = (rng.random((nX, 30)) < 0.5).astype(np.uint8)
        W = rng.integers(-127, 128, (30, 4))
        b = rng.integers(-127, 128, 4)
        X_ct = ctx.encrypt(keys, ctx.encode_features(dev(X).to(torch.uint8)).reshape(-1, P.N),
                           seed=96).reshape(nX, 1, 2, P.L, P.N)
        Y = ctx.lr_scores_packed(keys, ctx.model_prepare(W, b), X_ct, pair_chunk=1024)
        assert Y.shape[0] == -(-nX * 4 // P.N)
        slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
        assert np.array_equal(bfv.unpack_packed_scores(P.N, slots, nX, 4), oracle.expected_scores(X, W, b, P.t))


def test_standard_all_slots_tiny(tiny):
    """The standard product with every slot used (nX = N individuals) and a single feature."""
    ctx, keys, P, okeys = tiny
    rng = np.random.default_rng(97)
    X = (rng.random((P.N, 3)) < 0.5).astype(np.uint8)
    W = rng.integers(-127, 128, (3, 2))
    b = rng.integers(-127, 128, 2)
    X_ct = ctx.encrypt(keys, ctx.encode_feature_columns(dev(X).to(torch.uint8)), seed=98)
    oX_ct = oracle_columns(P, okeys, X, 98)
    assert np.array_equal(host(X_ct), oX_ct)
    Y = ctx.lr_scores_standard(ctx.model_prepare(W, b), X_ct, P.N)
    assert np.array_equal(host(Y), oracle.lr_standard(P, oX_ct, W, b))
    slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
    assert np.array_equal(slots.T, oracle.expected_scores(X, W, b, P.t))
    Y1 = ctx.lr_scores_standard(ctx.model_prepare(W[:1], b), X_ct[:1], P.N)
    assert np.array_equal(host(Y1), oracle.lr_standard(P, oX_ct[:1], W[:1], b))
