"""GPU parity at N = 32768 (15 ciphertext primes of 55 bits plus P, log QP = 880,
t = 786433), the ring of the mixed-parameter batch. A limb of this ring (256 KB) is larger
than one CTA's shared memory, so every limb transform runs on a two-CTA cluster (the forward
transform's first stage folded into the loads, the inverse transform's last stage through
distributed shared memory) and ModUp keeps its key sums in tensor memory. Everything is
compared with the oracle bit for bit, and decrypted scores with the closed form."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2204_05496_gb300 as bfv

SEED_KEYS = 402


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def host(t):
    return bfv.as_u64(t)


@pytest.fixture(scope="module")
def wide():
    ctx = bfv.Context.from_shape(synth.WIDE32K)
    keys = ctx.keygen(SEED_KEYS)
    P = oracle.Params.from_shape(synth.WIDE32K)
    okeys = oracle.keygen(P, SEED_KEYS)
    return ctx, keys, P, okeys


def test_wide_parameters_and_keys_match(wide):
    ctx, keys, P, okeys = wide
    assert ctx.N == 32768 and ctx.L == 15
    assert ctx.primes == P.qs and ctx.omega == P.omega
    sk, pk, gk = ctx.keys_export(keys)
    assert np.array_equal(sk.cpu().numpy(), okeys.sk)
    assert np.array_equal(host(pk), okeys.pk)
    g = host(gk)
    assert g.shape == okeys.gk_coeff.shape
    for s in (0, 7, 14):                                  # row swap, a middle and the last rotation
        assert np.array_equal(g[s], okeys.gk_coeff[s])


def test_wide_encode_encrypt_decrypt_match(wide):
    ctx, keys, P, okeys = wide
    v = synth.slots(31, 3, P.N, P.t)
    pt = ctx.encode(dev(v))
    assert np.array_equal(host(pt), oracle.encode(P, v))
    assert np.array_equal(ctx.decode(pt).cpu().numpy(), np.mod(v, P.t))
    m = oracle.encode(P, v)
    ct = ctx.encrypt(keys, dev(m), seed=91, obj0=5)
    oct_ = oracle.encrypt(P, okeys, m, seed=91, obj0=5)
    assert np.array_equal(host(ct), oct_)
    rng = np.random.default_rng(8)
    junk = np.stack([np.stack([rng.integers(0, q, P.N, dtype=np.uint64) for q in P.q]) for _ in range(2)])[None]
    allct = np.concatenate([oct_, junk])
    dec = ctx.decrypt(keys, dev(allct))
    assert np.array_equal(host(dec), oracle.decrypt(P, okeys.sk, allct))
    assert np.array_equal(host(dec)[:3], oracle.encode(P, v))


def test_wide_noise_budget(wide):
    # L = 15: the noise integer spans 14 64-bit words
    ctx, keys, P, okeys = wide
    m = oracle.encode(P, synth.slots(43, 1, P.N, P.t))
    ct = ctx.encrypt(keys, dev(m), seed=44, obj0=9)
    oct_ = oracle.encrypt(P, okeys, m, seed=44, obj0=9)
    assert np.array_equal(host(ct), oct_)
    assert ctx.noise_budget(keys, ct) == oracle.noise_budget(P, okeys.sk, oct_)


def test_wide_single_individual_packed_bit_exact(wide):
    # 40,000 features at N = 32768: K = 2 plaintexts per individual; 16 classes
    ctx, keys, P, okeys = wide
    rng = np.random.default_rng(404)
    X = (rng.random((1, 40000)) < 0.02).astype(np.uint8)
    W = rng.integers(-127, 128, (40000, 16))
    b = rng.integers(-127, 128, 16)
    pt = ctx.encode_features(dev(X).to(torch.uint8))
    X_ct = ctx.encrypt(keys, pt.reshape(-1, P.N), seed=405).reshape(1, 2, 2, P.L, P.N)
    oX_ct, _, oY = oracle.packed_pipeline(P, okeys, X, W, b, 405)
    assert np.array_equal(host(X_ct), oX_ct)
    model = ctx.model_prepare(W, b)
    Y = ctx.lr_scores_packed(keys, model, X_ct)
    assert np.array_equal(host(Y), oY)
    scores = bfv.unpack_packed_scores(P.N, ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy(), 1, 16)
    assert np.array_equal(scores, oracle.expected_scores(X, W, b, P.t))


def test_wide_whole_protocol(wide):
    # bfv_lr_predict_packed at N = 32768: three individuals x 40,000 features x 16 classes
    ctx, keys, P, _ = wide
    rng = np.random.default_rng(410)
    X = (rng.random((3, 40000)) < 0.02).astype(np.uint8)
    W = rng.integers(-127, 128, (40000, 16))
    b = rng.integers(-127, 128, 16)
    model = ctx.model_prepare(W, b)
    got = ctx.predict_packed(keys, model, dev(X), seed=411).cpu().numpy()
    assert np.array_equal(got, oracle.expected_scores(X, W, b, P.t))


def test_wide_binary_model_batch(wide):
    # a binary one-vs-rest model over 300 individuals (600 pairs, ragged chunks of 256):
    # every score against the closed form, one pair of the last chunk bit-exact
    ctx, keys, P, okeys = wide
    rng = np.random.default_rng(406)
    X = (rng.random((300, 5000)) < 0.02).astype(np.uint8)
    W = rng.integers(-127, 128, (5000, 2))
    b = rng.integers(-127, 128, 2)
    pt = ctx.encode_features(dev(X).to(torch.uint8))
    X_ct = ctx.encrypt(keys, pt.reshape(-1, P.N), seed=407).reshape(300, 1, 2, P.L, P.N)
    model = ctx.model_prepare(W, b)
    chunk = 256
    ws = torch.empty(ctx.packed_workspace(model, 300, chunk), dtype=torch.uint8, device="cuda")
    Y = ctx.lr_scores_packed(keys, model, X_ct, ws=ws, pair_chunk=chunk)
    assert Y.shape[0] == 1
    slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
    assert np.array_equal(bfv.unpack_packed_scores(P.N, slots, 300, 2), oracle.expected_scores(X, W, b, P.t))
    assert not slots.reshape(-1)[600:].any()
    W_pt = oracle.encode(P, oracle.pack_weights(P, W).reshape(-1, P.N)).reshape(2, 1, P.N)
    g = 599
    i, j = divmod(g, 2)
    xo = oracle.encrypt(P, okeys, oracle.encode(P, oracle.pack_inputs(P, X[i:i + 1])[0]), seed=407, obj0=i)
    assert np.array_equal(host(X_ct[i]), xo)
    c = oracle.pair_rotsum(P, okeys, xo, W_pt[j])
    want = oracle.pair_bias_mask(P, c, int(b[j]), g % P.N)
    assert np.array_equal(host(ctx.packed_pair_from_workspace(model, 300, chunk, ws, g)), want)


def test_wide_standard_product_bit_exact(wide):
    ctx, keys, P, okeys = wide
    rng = np.random.default_rng(408)
    X = (rng.random((40, 64)) < 0.3).astype(np.uint8)
    W = rng.integers(-127, 128, (64, 8))
    b = rng.integers(-127, 128, 8)
    model = ctx.model_prepare(W, b)
    X_ct = ctx.encrypt(keys, ctx.encode_feature_columns(dev(X).to(torch.uint8)), seed=409)
    Y = ctx.lr_scores_standard(model, X_ct, 40)
    want = np.zeros((64, P.N), dtype=np.int64)
    want[:, :40] = X.T
    oX_ct = oracle.encrypt(P, okeys, oracle.encode(P, want), seed=409)
    assert np.array_equal(host(X_ct), oX_ct)
    assert np.array_equal(host(Y), oracle.lr_standard(P, oX_ct, W, b))
    slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
    assert np.array_equal(slots[:, :40].T, oracle.expected_scores(X, W, b, P.t))
