"""The paper's precision scheme (Section 4.2.2): fixed-point inputs and weights and a pair of
plaintext moduli recombined by the Chinese remainder theorem.

Real inputs 0 <= x < 2^8 are scaled by 2^s_x (s_x = 6) and weights |w| < 1 by 2^s_w (s_w = 14),
both rounded to integers; biases are scaled by 2^(s_x + s_w). The scores then need
8 + s_x + s_w + ceil(log2 f) bits (44 at f = 40,960), more than one plaintext modulus holds, so
every step runs twice, under t0 = 1073872897 and t1 = 114689 (two contexts with their own keys),
and the client recombines the two decrypted score vectors with bfv_crt_combine.

This module only sequences calls of the C ABI (through the binding) and rounds the client's
real-valued data; it holds no homomorphic arithmetic.
"""
from __future__ import annotations

import math

import numpy as np

from . import Context, crt_combine, pack_rows, unpack_packed_scores

S_X, S_W = 6, 14
T0, T1 = 1073872897, 114689


def to_fixed(a, s: int) -> np.ndarray:
    """Round a * 2^s to the nearest integer (int64)."""
    return np.rint(np.asarray(a, dtype=np.float64) * (2.0 ** s)).astype(np.int64)


def scores_to_real(z, s_x: int = S_X, s_w: int = S_W) -> np.ndarray:
    """Descale recombined integer scores by 2^(s_x + s_w)."""
    return np.asarray(z, dtype=np.float64) / (2.0 ** (s_x + s_w))


def descale_argmax(z, s_x: int = S_X, s_w: int = S_W):
    """The client's last step (Section 4.2.4): recombined integer scores z [nX][nY] (any array or
    CPU/CUDA tensor) -> (real scores z / 2^(s_x + s_w) as float64 [nX][nY], predicted class of
    each individual = the argmax of its linear scores, int64 [nX]). The softmax of the LR model is
    monotone, so the argmax of the scores is the argmax of the class probabilities."""
    if hasattr(z, "cpu"):
        z = z.cpu().numpy()
    z = np.asarray(z, dtype=np.int64)
    return scores_to_real(z, s_x, s_w), np.argmax(z, axis=1).astype(np.int64)


def quantization_bound(X, W, s_x: int = S_X, s_w: int = S_W) -> np.ndarray:
    """Upper bound on |x.w + b - descaled fixed-point score| per individual and class for real X
    [nX][f] and W [f][nY]: with x~ = round(x 2^s_x) / 2^s_x (error <= 2^-(s_x+1)), w~ likewise
    (<= 2^-(s_w+1)) and the bias rounded at 2^-(s_x+s_w), |x w - x~ w~| <= |x - x~| |w| + |x~| |w - w~|,
    summed over the features, plus 2^-(s_x+s_w+1) for the bias. Returns float64 [nX][nY]."""
    X = np.asarray(X, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    xq = to_fixed(X, s_x).astype(np.float64) / 2.0 ** s_x
    return (2.0 ** -(s_x + 1)) * np.abs(W).sum(axis=0)[None, :] + \
        (2.0 ** -(s_w + 1)) * np.abs(xq).sum(axis=1)[:, None] + 2.0 ** -(s_x + s_w + 1)


def bits_needed(f: int, s_x: int = S_X, s_w: int = S_W) -> int:
    """Precision of the scaled scores for f features (Section 4.2.2)."""
    return 8 + s_x + s_w + math.ceil(math.log2(f))


class CrtPair:
    """Two BFV contexts of the same ring and ciphertext modulus with plaintext moduli t0, t1."""

    def __init__(self, N: int, L: int, prime_bits: int, t0: int = T0, t1: int = T1):
        self.t = (t0, t1)
        self.ctx = (Context(N, L, prime_bits, t0), Context(N, L, prime_bits, t1))
        self.N = N

    def keygen(self, seed: int):
        return tuple(c.keygen(seed + r) for r, c in enumerate(self.ctx))

    def model_prepare(self, W_int, b_int):
        return tuple(c.model_prepare(W_int, b_int) for c in self.ctx)

    def encrypt_rows(self, keys, X_int, seed: int):
        """Integer feature rows [nX][f] (device tensor) -> per ring uint64[nX][K][2][L][N]."""
        slots = pack_rows(X_int, self.N)
        nX = X_int.shape[0]
        out = []
        for r, c in enumerate(self.ctx):
            ct = c.encrypt(keys[r], c.encode(slots), seed=seed + r)
            out.append(ct.reshape(nX, -1, 2, c.L, c.N))
        return tuple(out)

    def scores_packed(self, keys, models, X_cts, **kw):
        return tuple(c.lr_scores_packed(keys[r], models[r], X_cts[r], **kw) for r, c in enumerate(self.ctx))

    def decrypt_scores(self, keys, Y, nX: int, nY: int):
        """Decrypt, decode and recombine the two rings' packed outputs -> int64 scores [nX][nY]
        (device tensor), centred in (-t0 t1 / 2, t0 t1 / 2]."""
        slots = [c.decode(c.decrypt(keys[r], Y[r])).reshape(-1)[: nX * nY] for r, c in enumerate(self.ctx)]
        return crt_combine(slots[0], self.t[0], slots[1], self.t[1]).reshape(nX, nY)

    def quantize_model(self, W, b, s_x: int = S_X, s_w: int = S_W):
        """The model owner's step: real weights |w| < 1 and biases -> fixed point (weights by
        2^s_w, biases by 2^(s_x + s_w)) -> both rings' encoded models."""
        return self.model_prepare(to_fixed(W, s_w), to_fixed(b, s_x + s_w))

    def predict(self, keys, models, X, seed: int, s_x: int = S_X, s_w: int = S_W, **kw):
        """The whole protocol for real-valued inputs 0 <= x < 2^8 (Section 4.2.2, Fig. 2): the client
        quantizes (2^s_x) and encrypts under both plaintext moduli, the server runs the packed
        product in each ring, the client decrypts, recombines by CRT, descales by 2^(s_x + s_w) and
        takes the argmax. X: float array [nX][f]. Returns (real scores [nX][nY], predicted class [nX],
        the integer scores [nX][nY])."""
        import torch
        Xi = to_fixed(X, s_x)
        X_cts = self.encrypt_rows(keys, torch.from_numpy(Xi).to(f"cuda:{self.ctx[0].device}"), seed)
        Y = self.scores_packed(keys, models, X_cts, **kw)
        z = self.decrypt_scores(keys, Y, Xi.shape[0], models[0].nY).cpu().numpy()
        real, cls = descale_argmax(z, s_x, s_w)
        return real, cls, z
