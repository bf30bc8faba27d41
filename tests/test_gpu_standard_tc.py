"""The standard product (Section 5.2.3) on the tensor cores: the byte-plane contraction as
tcgen05.mma kind::f16 with f32 sums moved to int64 every 256 features. Its outputs must equal
the oracle's bit for bit and the dp4a kernel's, across ragged 16-feature stages, several
accumulation chunks, two class groups and every byte-plane count (4 to 8)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2204_05496_gb300 as bfv


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def host(t):
    return bfv.as_u64(t)


def columns(P, okeys, X, seed):
    """The oracle's own encryptions of the feature columns of X (slot i = individual i)."""
    want = np.zeros((X.shape[1], P.N), dtype=np.int64)
    want[:, :X.shape[0]] = X.T
    return oracle.encrypt(P, okeys, oracle.encode(P, want), seed=seed, obj0=0)


def both_kernels(ctx, model, X_ct, nX):
    out = {}
    for kind in (0, 1):                               # tensor cores, dp4a
        ctx.set_option(bfv.BFV_OPT_STANDARD_KERNEL, kind)
        out[kind] = ctx.lr_scores_standard(model, X_ct, nX)
        assert ctx.check_error() == 0
    ctx.set_option(bfv.BFV_OPT_STANDARD_KERNEL, 0)
    return out


@pytest.mark.parametrize("bits,nf,nY", [(36, 1000, 8), (36, 777, 19), (59, 600, 5), (30, 300, 3), (47, 530, 16)])
def test_tensor_core_standard_product_matches_oracle(bits, nf, nY):
    """bits -> byte planes: 30 -> 4, 36 -> 5, 47 -> 6, 59 -> 8. nf not a multiple of 16 (ragged
    last stage) and above 256 (several accumulation chunks); 19 classes take two class groups."""
    shape = synth.BfvShape(N=4096, L=3, prime_bits=bits, t=65537)
    ctx = bfv.Context.from_shape(shape)
    assert ctx.get_option(bfv.BFV_OPT_STANDARD_KERNEL) == 0
    keys = ctx.keygen(61)
    P = oracle.Params.from_shape(shape)
    okeys = oracle.keygen(P, 61)
    rng = np.random.default_rng(62 + bits)
    nX = 13
    X = (rng.random((nX, nf)) < 0.3).astype(np.uint8)
    W = rng.integers(-127, 128, (nf, nY))
    W[0, :] = 127                                      # the extreme weights
    W[1, :] = -127
    b = rng.integers(-127, 128, nY)
    oX = columns(P, okeys, X, 63)
    X_ct = dev(oX)
    model = ctx.model_prepare(W, b)
    out = both_kernels(ctx, model, X_ct, nX)
    want = oracle.lr_standard(P, oX, W, b)
    assert np.array_equal(host(out[0]), want)
    assert torch.equal(out[0], out[1])
    slots = ctx.decode(ctx.decrypt(keys, out[0])).cpu().numpy()
    assert np.array_equal(slots[:, :nX].T, oracle.expected_scores(X, W, b, P.t))


def test_tensor_core_standard_product_extreme_residues():
    """Residues q - 1 in every word with weights of +-127 everywhere: the largest byte values and
    the largest f32 chunk sums (256 x 255 x 127 < 2^23); exact against the oracle."""
    shape = synth.BfvShape(N=4096, L=3, prime_bits=59, t=65537)
    ctx = bfv.Context.from_shape(shape)
    P = oracle.Params.from_shape(shape)
    nf, nY = 520, 16
    X_ct = np.zeros((nf, 2, P.L, P.N), dtype=np.uint64)
    for l, q in enumerate(P.qs[:P.L]):
        X_ct[:, :, l, :] = q - 1
    W = np.where(np.arange(nf * nY).reshape(nf, nY) % 3 == 0, -127, 127)
    b = np.zeros(nY, dtype=np.int64)
    model = ctx.model_prepare(W, b)
    out = both_kernels(ctx, model, dev(X_ct), 1)
    assert np.array_equal(host(out[0]), oracle.lr_standard(P, X_ct, W, b))
    assert torch.equal(out[0], out[1])
