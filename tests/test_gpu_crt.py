"""The paper's own precision scheme on its own parameter set (Section 4.2.2, Section 5.2.3):
N = 8192, the CRT pair t0 = 1073872897 / t1 = 114689, fixed-point inputs (2^6) and weights
(2^14), biases scaled by 2^20, 11 classes. Each ring's ciphertexts must match the oracle bit for
bit; the recombined scores must equal the exact integer products X_int W_int + b_int, on the
packed and on the standard product."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2204_05496_gb300 as bfv
    from paper_2204_05496_gb300 import crt_pair

SHAPES = (synth.PAPER8K_T0, synth.PAPER8K_T1)


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def host(t):
    return bfv.as_u64(t)


@pytest.fixture(scope="module")
def pair():
    p = crt_pair.CrtPair(8192, 4, 43)
    keys = p.keygen(601)
    Ps = [oracle.Params.from_shape(s) for s in SHAPES]
    okeys = [oracle.keygen(P, 601 + r) for r, P in enumerate(Ps)]
    return p, keys, Ps, okeys


def quantized(seed, nX, f, nY):
    X, W, b = synth.paper_realvalued(seed, nX, f, nY)
    return crt_pair.to_fixed(X, crt_pair.S_X), crt_pair.to_fixed(W, crt_pair.S_W), \
        crt_pair.to_fixed(b, crt_pair.S_X + crt_pair.S_W), (X, W, b)


def test_crt_pair_packed_bit_exact_and_exact_scores(pair):
    p, keys, Ps, okeys = pair
    Xi, Wi, bi, _ = quantized(602, 3, 9000, 11)                # K = 2 at N = 8192
    # a saturated individual and class (all inputs and weights at the fixed-point maximum):
    # its score, about 2^41, exceeds either modulus alone
    Xi = np.vstack([Xi, np.full((1, 9000), 2 ** 14 - 1, dtype=np.int64)])
    Wi[:, 0] = 2 ** 14 - 1
    models = p.model_prepare(Wi, bi)
    X_cts = p.encrypt_rows(keys, dev(Xi), seed=603)
    Y = p.scores_packed(keys, models, X_cts)
    exact = Xi @ Wi + bi[None, :]
    res = []
    for r, (P, ok) in enumerate(zip(Ps, okeys)):
        oX, _, oY = oracle.packed_pipeline(P, ok, Xi, Wi, bi, 603 + r)
        assert np.array_equal(host(X_cts[r]), oX)
        assert np.array_equal(host(Y[r]), oY)
        res.append(oracle.unpack_packed_scores(P, oracle.decode(P, oracle.decrypt(P, ok.sk, oY)), 4, 11))
    assert np.array_equal(oracle.crt_combine(res[0], Ps[0].t, res[1], Ps[1].t), exact)
    z = p.decrypt_scores(keys, Y, 4, 11).cpu().numpy()
    assert np.array_equal(z, exact)
    assert np.abs(exact).max() >= Ps[0].t                       # neither modulus alone would do


def test_crt_pair_standard_exact_scores(pair):
    p, keys, Ps, okeys = pair
    Xi, Wi, bi, _ = quantized(604, 37, 300, 11)
    exact = Xi @ Wi + bi[None, :]
    cols = np.zeros((300, 8192), dtype=np.int64)
    cols[:, :37] = Xi.T
    out = []
    for r, c in enumerate(p.ctx):
        m = c.model_prepare(Wi, bi)
        X_ct = c.encrypt(keys[r], c.encode(dev(cols)), seed=605 + r)
        oX = oracle.encrypt(Ps[r], okeys[r], oracle.encode(Ps[r], cols), seed=605 + r)
        assert np.array_equal(host(X_ct), oX)
        Y = c.lr_scores_standard(m, X_ct, 37)
        assert np.array_equal(host(Y), oracle.lr_standard(Ps[r], oX, Wi, bi))
        out.append(c.decode(c.decrypt(keys[r], Y))[:, :37].T.contiguous())
    z = bfv.crt_combine(out[0], Ps[0].t, out[1], Ps[1].t).cpu().numpy()
    assert np.array_equal(z, exact)


def test_crt_combine_kernel_matches_oracle():
    t0, t1 = crt_pair.T0, crt_pair.T1
    rng = np.random.default_rng(606)
    r0 = rng.integers(-3 * t0, 3 * t0, size=5000)            # any representative
    r1 = rng.integers(-3 * t1, 3 * t1, size=5000)
    got = bfv.crt_combine(dev(r0), t0, dev(r1), t1).cpu().numpy()
    assert np.array_equal(got, oracle.crt_combine(r0 % t0, t0, r1 % t1, t1))
    with pytest.raises(bfv.BfvError):
        bfv.crt_combine(dev(r0), 6, dev(r1), 4)               # not coprime


def test_client_pipeline_realvalued_stage_by_stage(pair):
    """The whole protocol on real-valued inputs shaped like the paper's encodings (Section 4.1.2)
    through the client calls of crt_pair: quantize (2^6) -> encrypt under t0 and t1 -> packed
    product -> decrypt -> CRT -> descale (2^-20) -> argmax (Section 4.2.4). Each ring's input
    ciphertexts, product ciphertexts and decrypted plaintexts equal the oracle's bit for bit; the
    recombined integers equal X_int W_int + b_int; the descaled scores lie within the quantization
    bound of the real model's; the argmax equals the real model's wherever its top two classes
    differ by more than twice that bound."""
    p, keys, Ps, okeys = pair
    X, W, b = synth.paper_realvalued(607, 24, 9000, 11)
    Xi, Wi = crt_pair.to_fixed(X, crt_pair.S_X), crt_pair.to_fixed(W, crt_pair.S_W)
    bi = crt_pair.to_fixed(b, crt_pair.S_X + crt_pair.S_W)
    models = p.quantize_model(W, b)
    seed = 608
    real, cls, z = p.predict(keys, models, X, seed)
    exact = Xi @ Wi + bi[None, :]
    # stage by stage: the same encryptions (same seeds) and products, against the oracle
    X_cts = p.encrypt_rows(keys, dev(Xi), seed=seed)
    Y = p.scores_packed(keys, models, X_cts)
    res = []
    for r, (P, ok) in enumerate(zip(Ps, okeys)):
        oX, _, oY = oracle.packed_pipeline(P, ok, Xi, Wi, bi, seed + r)
        assert np.array_equal(host(X_cts[r]), oX)
        assert np.array_equal(host(Y[r]), oY)
        opt = oracle.decrypt(P, ok.sk, oY)
        assert np.array_equal(host(p.ctx[r].decrypt(keys[r], Y[r])), opt)
        res.append(oracle.unpack_packed_scores(P, oracle.decode(P, opt), 24, 11))
    assert np.array_equal(oracle.crt_combine(res[0], Ps[0].t, res[1], Ps[1].t), exact)
    assert np.array_equal(z, exact)
    assert np.array_equal(real, exact / 2.0 ** (crt_pair.S_X + crt_pair.S_W))
    assert np.array_equal(cls, np.argmax(exact, axis=1))
    ref = X @ W + b[None, :]
    bound = crt_pair.quantization_bound(X, W)
    assert np.all(np.abs(real - ref) <= bound)
    top2 = np.sort(ref, axis=1)[:, -2:]
    sure = (top2[:, 1] - top2[:, 0]) > 2 * bound.max(axis=1)
    assert sure.sum() >= 6
    assert np.array_equal(cls[sure], np.argmax(ref, axis=1)[sure])
