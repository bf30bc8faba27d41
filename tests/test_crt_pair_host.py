"""Host-side arithmetic of the CRT-pair precision scheme (Section 4.2.2), on CPU: the client's
fixed-point rounding, the descaling of recombined scores, and the precision the scaled scores
need against the pair of plaintext moduli. No GPU compute."""
import math

import numpy as np
import pytest

import synth

pytest.importorskip("torch")


@pytest.fixture(scope="module")
def crt_pair():
    from paper_2204_05496_gb300 import crt_pair
    return crt_pair


def test_fixed_point_scores_stay_within_the_rounding_bound(crt_pair):
    """x rounded to 2^-s_x, w to 2^-s_w and b to 2^-(s_x+s_w): the descaled integer score differs
    from x.w + b by at most sum_f (|x_f| 2^-(s_w+1) + |w_f| 2^-(s_x+1) + 2^-(s_x+s_w+2)) +
    2^-(s_x+s_w+1). The integers stay inside the bits the paper budgets and inside the centred
    range of t0 t1."""
    sx, sw = crt_pair.S_X, crt_pair.S_W
    X, W, b = synth.paper_realvalued(71, 24, 4096, 11)
    Xi, Wi, bi = crt_pair.to_fixed(X, sx), crt_pair.to_fixed(W, sw), crt_pair.to_fixed(b, sx + sw)
    assert np.all(np.abs(Xi - X * 2.0 ** sx) <= 0.5) and np.all(np.abs(Wi - W * 2.0 ** sw) <= 0.5)
    z = Xi @ Wi + bi[None, :]                                   # exact in int64 at these sizes
    err = np.abs(crt_pair.scores_to_real(z, sx, sw) - (X @ W + b[None, :]))
    bound = (np.abs(X) @ np.ones_like(W) * 2.0 ** -(sw + 1) + np.ones_like(X) @ np.abs(W) * 2.0 ** -(sx + 1)
             + X.shape[1] * 2.0 ** -(sx + sw + 2) + 2.0 ** -(sx + sw + 1))
    assert np.all(err <= bound * (1 + 1e-12))
    bits = crt_pair.bits_needed(X.shape[1], sx, sw)
    assert np.abs(z).max() < 2 ** (bits - 1)
    assert 2 * np.abs(z).max() < crt_pair.T0 * crt_pair.T1


def test_precision_budget_at_the_paper_size(crt_pair):
    """At f = 40,960 the worst case |z| < 2^8 2^s_x * 2^s_w * f needs 44 bits (Section 4.2.2), more
    than either plaintext modulus holds and less than their product."""
    f = 40960
    worst = (2 ** 8 * 2 ** crt_pair.S_X) * (2 ** crt_pair.S_W) * f
    assert math.ceil(math.log2(worst)) == crt_pair.bits_needed(f) == 44
    assert crt_pair.T0 < 2 ** 43 and crt_pair.T1 < 2 ** 43 < crt_pair.T0 * crt_pair.T1 // 2
    assert math.gcd(crt_pair.T0, crt_pair.T1) == 1


def test_descale_argmax_and_quantization_bound(crt_pair):
    """The client's last step on exact integer scores of quantized real data: the descaled scores
    lie within quantization_bound of the real-valued model's scores, and wherever the real model's
    top two classes differ by more than twice the bound, the argmax agrees with the real model."""
    X, W, b = synth.paper_realvalued(17, 40, 3000, 11)
    Xi, Wi = crt_pair.to_fixed(X, crt_pair.S_X), crt_pair.to_fixed(W, crt_pair.S_W)
    bi = crt_pair.to_fixed(b, crt_pair.S_X + crt_pair.S_W)
    z = Xi @ Wi + bi[None, :]                                  # what the CRT pair recombines to
    real, cls = crt_pair.descale_argmax(z)
    assert cls.dtype == np.int64 and cls.shape == (40,)
    assert np.array_equal(real, z / 2.0 ** 20)
    ref = X @ W + b[None, :]
    bound = crt_pair.quantization_bound(X, W)
    assert np.all(np.abs(real - ref) <= bound)
    top2 = np.sort(ref, axis=1)[:, -2:]
    sure = (top2[:, 1] - top2[:, 0]) > 2 * bound.max(axis=1)
    assert sure.sum() >= 10
    assert np.array_equal(cls[sure], np.argmax(ref, axis=1)[sure])
