"""CPU oracle for BFV-encrypted logistic-regression scoring.

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package. The product
library never calls it, and the two share no code.

What it computes (paper: "Scalable privacy-preserving cancer type prediction with
homomorphic encryption"):
  * the private inference protocol of Section 4.2.2 (encode, encrypt, server-side
    product with encoded weights plus encoded bias, decrypt, decode);
  * the packed matrix product of Section 4.2.3 / Algorithm 1 / Appendix:
    multiply, add_many, rotate-and-accumulate, mask, compress;
  * the "standard" per-element matrix product it is compared with (Section 5.2.3).

BFV itself (keys, encryption, rotation by Galois automorphism plus key switching)
is the textbook scheme the paper uses through SEAL (Section 2.2, Section 5.2); the
paper fixes none of its internal conventions, so this module takes these readings:
  * primes: the largest primes below 2^b with q = 1 (mod 2N), descending; the
    first L form Q, the next one is the key-switching prime P;
  * slot map: omega = g^((t-1)/2N) mod t with g the smallest primitive root mod t;
    slot l sits at omega^e_l, e_l = 3^c (row 0) or 2N - 3^c (row 1), c = l mod N/2;
  * rotate-and-sum: the row swap (Galois element 2N-1), then left row rotations by
    N/4, ..., 1 (elements 3^s mod 2N), each step c += rot(c) - log2 N rotations;
  * Delta = floor(Q/t); plaintexts enter ciphertext-plaintext products through their
    centred representative in (-t/2, t/2]; the bias b_j is added as Delta*[b_j]_t to
    the rotated sum, before masking; the mask for pair g = i*|Y| + j is one-hot at
    slot g mod N, and pair g lands in output ciphertext floor(g / N);
  * key switching: one digit per ciphertext prime, one special prime P, ModDown with
    rounding; encryption randomness: ChaCha20 (RFC 8439) blocks, key = the 64-bit
    seed, nonce = (purpose, object, limb), block counter = coefficient index.

The CRT plaintext pair of Section 4.2.2 is recombined by the textbook CRT formula
(crt_combine). The invariant noise budget (noise_budget, a diagnostic; Section 4.2.2 sizes t by
the budget a ciphertext must keep) is the textbook BFV definition, in whole bits.

Pins (tests/test_oracle_pins.py) tie every function to something other than itself: RFC 8439
vectors, schoolbook convolution, direct evaluation, sympy's primality and CRT, closed forms,
invariants (decryption invariance of key switching, ModDown(P x) = x, the rotate-and-sum slot
total) and the exact result x.W + b of every product. What the paper does not fix -- the exact
ciphertext bits, which follow from the readings above (the generator, the slot map, the
key-switching conventions) -- is "parity unpinned" by the paper: those bits are pinned only by
the readings, which the CUDA library implements independently.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from decimal import Decimal, getcontext

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbfv_oracle.so")
MAXP = 40

# Sampling purposes (first ChaCha20 nonce word).
P_SK, P_PK_A, P_PK_E, P_GK_A, P_GK_E, P_ENC = 1, 2, 3, 4, 5, 6


# --------------------------------------------------------------------------- build

def build(force: bool = False) -> str:
    """Compile the oracle's C part with gcc (OpenMP if available). Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


class _Params(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32), ("L", ctypes.c_int32),
        ("q", ctypes.c_uint64 * MAXP), ("psi", ctypes.c_uint64 * MAXP),
        ("t", ctypes.c_uint64), ("omega", ctypes.c_uint64),
        ("delta", ctypes.c_uint64 * MAXP), ("p_mod", ctypes.c_uint64 * MAXP),
        ("p_inv", ctypes.c_uint64 * MAXP), ("p_half", ctypes.c_uint64),
        ("cdt", ctypes.c_uint64 * 32), ("cdt_len", ctypes.c_int32),
        ("nthreads", ctypes.c_int32),
    ]


_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i8p = ctypes.POINTER(ctypes.c_int8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_pp = ctypes.POINTER(_Params)


def _declare(L):
    sig = {
        "oc_ntt_forward": [_u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64],
        "oc_ntt_inverse": [_u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64],
        "oc_polymul": [_u64p, _u64p, _u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64],
        "oc_polymul_schoolbook": [_u64p, _u64p, _u64p, ctypes.c_int, ctypes.c_uint64],
        "oc_chacha_quarter": [_u32p],
        "oc_chacha20_block": [_u32p, ctypes.c_uint32, _u32p, _u32p],
        "oc_sample_ternary": [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, _i8p],
        "oc_sample_gauss": [_pp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, _i8p],
        "oc_sample_enc": [_pp, ctypes.c_uint64, ctypes.c_uint32, _i8p, _i8p, _i8p],
        "oc_sample_uniform": [_pp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _u64p],
        "oc_automorph": [_u64p, _u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64],
        "oc_galois_elements": [ctypes.c_int, _u64p],
        "oc_encode": [_pp, _i64p, _u64p],
        "oc_decode": [_pp, _u64p, _i64p],
        "oc_keygen_sk": [_pp, ctypes.c_uint64, _i8p],
        "oc_keygen_pk": [_pp, ctypes.c_uint64, _i8p, _u64p],
        "oc_keygen_galois": [_pp, ctypes.c_uint64, _i8p, _u64p, ctypes.c_int, _u64p],
        "oc_galois_to_eval": [_pp, _u64p, ctypes.c_int],
        "oc_encrypt": [_pp, _u64p, _u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, _u64p],
        "oc_decrypt_inner": [_pp, _i8p, _u64p, ctypes.c_int, _u64p],
        "oc_keyswitch": [_pp, _u64p, _u64p, _u64p, _u64p],
        "oc_moddown": [_pp, _u64p, _u64p],
        "oc_mul_plain": [_pp, _u64p, _u64p, _u64p],
        "oc_rotate": [_pp, _u64p, ctypes.c_uint64, _u64p, _u64p],
        "oc_pair_rotsum": [_pp, _u64p, _u64p, ctypes.c_int, _u64p, _u64p, ctypes.c_int, _u64p],
        "oc_pair_bias_mask": [_pp, _u64p, ctypes.c_uint64, ctypes.c_int],
        "oc_lr_packed": [_pp, _u64p, _u64p, ctypes.c_int, _u64p, ctypes.c_int, _u64p, _u64p,
                         ctypes.c_int, ctypes.c_int, _u64p, _u64p],
        "oc_lr_standard": [_pp, _u64p, ctypes.c_int, _i64p, _u64p, ctypes.c_int, _u64p],
        "oc_standard_coeff": [_i64p, _u64p, ctypes.c_int, ctypes.c_uint64],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = None
    L.oc_galois_elements.restype = ctypes.c_int
    L.oc_standard_coeff.restype = ctypes.c_uint64
    L.oc_has_openmp.restype = ctypes.c_int


def _p(a, ty=_u64p):
    return a.ctypes.data_as(ty)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


# --------------------------------------------------------------------------- number theory (Python ints)

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (bases: the first 13 primes)."""
    if n < 2:
        return False
    for b in _MR_BASES:
        if n % b == 0:
            return n == b
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(bits: int, N: int, count: int) -> list[int]:
    """The `count` largest primes below 2^bits that are 1 mod 2N, in descending order."""
    m = 2 * N
    q = (1 << bits) - m + 1
    out = []
    while len(out) < count:
        if q < (1 << (bits - 1)):
            raise ValueError("not enough primes of this size")
        if is_prime(q):
            out.append(q)
        q -= m
    return out


def _factor_small(n: int) -> list[int]:
    fs, d = [], 2
    while d * d <= n:
        if n % d == 0:
            fs.append(d)
            while n % d == 0:
                n //= d
        d += 1
    if n > 1:
        fs.append(n)
    return fs


def smallest_primitive_root(p: int) -> int:
    fs = _factor_small(p - 1)
    g = 2
    while any(pow(g, (p - 1) // f, p) == 1 for f in fs):
        g += 1
    return g


def root_2n(q: int, N: int) -> int:
    """A primitive 2N-th root of unity mod q: x^((q-1)/2N) for the first x = 2, 3, ... whose
    power has order 2N (its N-th power is -1)."""
    x = 2
    while True:
        r = pow(x, (q - 1) // (2 * N), q)
        if pow(r, N, q) == q - 1:
            return r
        x += 1


def gaussian_cdt(num: int, den: int, tail: int | None = None) -> list[int]:
    """Thresholds T_k = floor(2^64 * Pr[|x| <= k]), k = 0..tail-1, for the discrete Gaussian
    Pr[x] ~ exp(-x^2 / (2 sigma^2)), sigma = num/den, truncated to |x| <= tail
    (tail = floor(6 sigma) by default). Computed with 90-digit decimal arithmetic."""
    getcontext().prec = 90
    sigma = Decimal(num) / Decimal(den)
    if tail is None:
        tail = int(6 * num // den)
    rho = [(-(Decimal(k * k)) / (2 * sigma * sigma)).exp() for k in range(tail + 1)]
    Z = rho[0] + 2 * sum(rho[1:])
    out, cum = [], Decimal(0)
    for k in range(tail):
        cum += rho[0] if k == 0 else 2 * rho[k]
        out.append(int(cum / Z * Decimal(2 ** 64)))
    return out


def slot_exponents(N: int) -> list[int]:
    """e_l for every slot l (see the module docstring)."""
    e = [0] * N
    g = 1
    for c in range(N // 2):
        e[c] = g
        e[c + N // 2] = 2 * N - g
        g = g * 3 % (2 * N)
    return e


def galois_elements(N: int) -> list[int]:
    """Rotate-and-sum Galois elements in order: 2N-1, then 3^(N/4), ..., 3^1 mod 2N."""
    out = [2 * N - 1]
    s = N // 4
    while s >= 1:
        out.append(pow(3, s, 2 * N))
        s //= 2
    return out


# --------------------------------------------------------------------------- parameters

class Params:
    """BFV parameters for the oracle: ring degree N, L ciphertext primes of `prime_bits` bits
    plus one special prime, plaintext modulus t, Gaussian width sigma = num/den."""

    def __init__(self, N: int, L: int, prime_bits: int, t: int, sigma_num: int = 16,
                 sigma_den: int = 5, nthreads: int | None = None, primes: list[int] | None = None):
        if (t - 1) % (2 * N):
            raise ValueError("t must be 1 mod 2N for batching")
        self.N, self.L, self.t = N, L, t
        self.logN = int(round(math.log2(N)))
        self.qs = list(primes) if primes is not None else ntt_primes(prime_bits, N, L + 1)
        self.q = self.qs[:L]
        self.P = self.qs[L]
        self.Q = math.prod(self.q)
        self.delta = self.Q // t
        self.omega = pow(smallest_primitive_root(t), (t - 1) // (2 * N), t)
        self.psis = [root_2n(q, N) for q in self.qs]
        self.cdt = gaussian_cdt(sigma_num, sigma_den)
        self.galois = galois_elements(N)
        self.nthreads = nthreads or os.cpu_count() or 1
        c = _Params()
        c.N, c.L, c.t, c.omega = N, L, t, self.omega
        for i, q in enumerate(self.qs):
            c.q[i] = q
            c.psi[i] = self.psis[i]
            c.delta[i] = self.delta % q
            c.p_mod[i] = self.P % q
            c.p_inv[i] = pow(self.P, -1, q) if i < L else 0
        c.p_half = self.P // 2
        for k, v in enumerate(self.cdt):
            c.cdt[k] = v
        c.cdt_len = len(self.cdt)
        c.nthreads = self.nthreads
        self._c = c
        self._cp = ctypes.pointer(c)
        self._gel = np.array(self.galois, dtype=np.uint64)

    @classmethod
    def from_shape(cls, shape, **kw):
        return cls(shape.N, shape.L, shape.prime_bits, shape.t, shape.sigma_num, shape.sigma_den, **kw)

    def set_threads(self, n: int):
        self.nthreads = n
        self._c.nthreads = n

    @property
    def ct_shape(self):
        return (2, self.L, self.N)


# --------------------------------------------------------------------------- NTT / ring helpers

def ntt_forward(a, q: int, psi: int):
    a = _u64(a).copy()
    lib().oc_ntt_forward(_p(a), a.size, q, psi)
    return a


def ntt_inverse(a, q: int, psi: int):
    a = _u64(a).copy()
    lib().oc_ntt_inverse(_p(a), a.size, q, psi)
    return a


def polymul(a, b, q: int, psi: int):
    a, b = _u64(a), _u64(b)
    out = np.empty_like(a)
    lib().oc_polymul(_p(a), _p(b), _p(out), a.size, q, psi)
    return out


def polymul_schoolbook(a, b, q: int):
    a, b = _u64(a), _u64(b)
    out = np.empty_like(a)
    lib().oc_polymul_schoolbook(_p(a), _p(b), _p(out), a.size, q)
    return out


def automorph(a, q: int, g: int):
    a = _u64(a)
    out = np.empty_like(a)
    lib().oc_automorph(_p(a), _p(out), a.size, q, g)
    return out


def chacha_quarter(a, b, c, d):
    w = np.array([a, b, c, d], dtype=np.uint32)
    lib().oc_chacha_quarter(_p(w, _u32p))
    return [int(x) for x in w]


def chacha20_block(key_words, counter: int, nonce_words):
    k = np.array(key_words, dtype=np.uint32)
    n = np.array(nonce_words, dtype=np.uint32)
    out = np.empty(16, dtype=np.uint32)
    lib().oc_chacha20_block(_p(k, _u32p), counter, _p(n, _u32p), _p(out, _u32p))
    return out


def sample_ternary(seed: int, purpose: int, obj: int, N: int):
    out = np.empty(N, dtype=np.int8)
    lib().oc_sample_ternary(seed, purpose, obj, N, _p(out, _i8p))
    return out


def sample_gauss(P: Params, seed: int, purpose: int, obj: int):
    out = np.empty(P.N, dtype=np.int8)
    lib().oc_sample_gauss(P._cp, seed, purpose, obj, P.N, _p(out, _i8p))
    return out


def sample_enc(P: Params, seed: int, obj: int):
    """(u, e1, e2) drawn for ciphertext `obj`."""
    u, e1, e2 = (np.empty(P.N, dtype=np.int8) for _ in range(3))
    lib().oc_sample_enc(P._cp, seed, obj, _p(u, _i8p), _p(e1, _i8p), _p(e2, _i8p))
    return u, e1, e2


def sample_uniform(P: Params, seed: int, purpose: int, obj: int, limb: int):
    out = np.empty(P.N, dtype=np.uint64)
    lib().oc_sample_uniform(P._cp, seed, purpose, obj, limb, _p(out))
    return out


# --------------------------------------------------------------------------- scheme

def encode(P: Params, slots):
    """Slot values (any integers, taken mod t) -> plaintext polynomial coefficients in [0, t)."""
    v = np.ascontiguousarray(slots, dtype=np.int64)
    out = np.empty(v.shape, dtype=np.uint64)
    for idx in np.ndindex(v.shape[:-1]):
        vi = np.ascontiguousarray(v[idx])
        oi = np.empty(P.N, dtype=np.uint64)
        lib().oc_encode(P._cp, _p(vi, _i64p), _p(oi))
        out[idx] = oi
    return out


def decode(P: Params, pt):
    """Plaintext polynomial(s) -> slot values in [0, t)."""
    m = _u64(pt)
    out = np.empty(m.shape, dtype=np.int64)
    for idx in np.ndindex(m.shape[:-1]):
        mi = np.ascontiguousarray(m[idx])
        oi = np.empty(P.N, dtype=np.int64)
        lib().oc_decode(P._cp, _p(mi), _p(oi, _i64p))
        out[idx] = oi
    return out


class Keys:
    def __init__(self, sk, pk, gk_coeff, gk_eval):
        self.sk, self.pk, self.gk_coeff, self.gk_eval = sk, pk, gk_coeff, gk_eval


def keygen(P: Params, seed: int, galois=None) -> Keys:
    """Secret key, public key and the rotate-and-sum Galois keys (coefficient and evaluation form)."""
    L = lib()
    sk = np.empty(P.N, dtype=np.int8)
    L.oc_keygen_sk(P._cp, seed, _p(sk, _i8p))
    pk = np.empty((2, P.L, P.N), dtype=np.uint64)
    L.oc_keygen_pk(P._cp, seed, _p(sk, _i8p), _p(pk))
    gel = np.array(P.galois if galois is None else galois, dtype=np.uint64)
    gk = np.empty((len(gel), P.L, 2, P.L + 1, P.N), dtype=np.uint64)
    L.oc_keygen_galois(P._cp, seed, _p(sk, _i8p), _p(gel), len(gel), _p(gk))
    gke = gk.copy()
    L.oc_galois_to_eval(P._cp, _p(gke), len(gel))
    return Keys(sk, pk, gk, gke)


def encrypt(P: Params, keys: Keys, pt, seed: int, obj0: int = 0):
    """Encrypt plaintexts [count][N] -> ciphertexts [count][2][L][N]; ciphertext c uses object id obj0 + c."""
    m = _u64(pt).reshape(-1, P.N)
    out = np.empty((m.shape[0], 2, P.L, P.N), dtype=np.uint64)
    lib().oc_encrypt(P._cp, _p(keys.pk), _p(m), m.shape[0], seed, obj0, _p(out))
    return out


def decrypt_residues(P: Params, sk, ct):
    """[c0 + c1 s]_{q_l} for each limb: [count][L][N]."""
    c = _u64(ct).reshape(-1, 2, P.L, P.N)
    x = np.empty((c.shape[0], P.L, P.N), dtype=np.uint64)
    lib().oc_decrypt_inner(P._cp, _p(np.ascontiguousarray(sk, dtype=np.int8), _i8p), _p(c), c.shape[0], _p(x))
    return x


def _crt(P: Params, x):
    """Residues [L][N] -> list of N integers in [0, Q)."""
    Q = P.Q
    coefs = [(Q // q) * pow(Q // q, -1, q) for q in P.q]
    cols = [[int(v) for v in x[l]] for l in range(P.L)]
    return [sum(coefs[l] * cols[l][k] for l in range(P.L)) % Q for k in range(P.N)]


def decrypt(P: Params, sk, ct):
    """Plaintext coefficients m = round(t * [c0 + c1 s]_Q / Q) mod t, exactly, per ciphertext."""
    xs = decrypt_residues(P, sk, ct)
    out = np.empty((xs.shape[0], P.N), dtype=np.uint64)
    Q, t = P.Q, P.t
    for c in range(xs.shape[0]):
        X = _crt(P, xs[c])
        out[c] = [((t * v + Q // 2) // Q) % t for v in X]
    return out


def noise_budget_bits(P: Params, sk, ct) -> float:
    """Invariant noise budget log2(Q / (2 max |[t x]_Q|)) of the worst ciphertext; <= 0 means
    decryption may be wrong."""
    xs = decrypt_residues(P, sk, ct)
    Q, t = P.Q, P.t
    worst = 1
    for c in range(xs.shape[0]):
        for v in _crt(P, xs[c]):
            r = (t * v) % Q
            r = min(r, Q - r)
            worst = max(worst, r)
    return math.log2(Q) - math.log2(2 * worst)


def noise_budget(P: Params, sk, ct) -> list[int]:
    """Invariant noise budget of each ciphertext in whole bits. With x = [c0 + c1 s]_Q, the
    integer z = [t x]_Q taken in (-Q/2, Q/2] equals t e - (Q mod t) m for x = Delta m + e, and
    z / Q is the invariant noise v in (t/Q) x = m + v (mod t); decryption rounds correctly while
    |v| < 1/2. Budget = max(0, bitlen(Q) - bitlen(max_k |z_k|) - 1); a positive budget means
    max |z| < 2^(bitlen(Q) - 2) <= Q/2."""
    xs = decrypt_residues(P, sk, ct)
    Q, t = P.Q, P.t
    out = []
    for c in range(xs.shape[0]):
        worst = 0
        for v in _crt(P, xs[c]):
            z = (t * v) % Q
            if z > Q // 2:
                z -= Q
            worst = max(worst, abs(z))
        out.append(max(0, Q.bit_length() - worst.bit_length() - 1))
    return out


def keyswitch(P: Params, gk_eval_g, d):
    """KS of d (coefficient form [L][N]) with one Galois element's evaluation-form key."""
    d = _u64(d)
    o0 = np.empty((P.L, P.N), dtype=np.uint64)
    o1 = np.empty((P.L, P.N), dtype=np.uint64)
    lib().oc_keyswitch(P._cp, _p(np.ascontiguousarray(gk_eval_g)), _p(d), _p(o0), _p(o1))
    return o0, o1


def moddown(P: Params, U):
    """round(U / P) over Q for U over QP, both coefficient form ([L+1][N] -> [L][N])."""
    U = _u64(U)
    out = np.empty((P.L, P.N), dtype=np.uint64)
    lib().oc_moddown(P._cp, _p(U), _p(out))
    return out


def mul_plain(P: Params, ct, pt):
    """Ciphertext [2][L][N] times plaintext [N] (mod t), through the centred lift."""
    ct, pt = _u64(ct), _u64(pt)
    out = np.empty_like(ct)
    lib().oc_mul_plain(P._cp, _p(ct), _p(pt), _p(out))
    return out


def rotate(P: Params, gk_eval_g, g: int, ct):
    ct = _u64(ct)
    out = np.empty_like(ct)
    lib().oc_rotate(P._cp, _p(np.ascontiguousarray(gk_eval_g)), g, _p(ct), _p(out))
    return out


def pair_rotsum(P: Params, keys: Keys, xct, wpt, galois=None):
    """One pair of Algorithm 1 through the rotate-and-accumulate loop.
    xct: [K][2][L][N], wpt: [K][N] plaintexts. Returns [2][L][N]."""
    xct, wpt = _u64(xct), _u64(wpt)
    K = xct.shape[0]
    gel = np.array(P.galois if galois is None else galois, dtype=np.uint64)
    out = np.empty((2, P.L, P.N), dtype=np.uint64)
    lib().oc_pair_rotsum(P._cp, _p(keys.gk_eval), _p(gel), len(gel), _p(xct), _p(wpt), K, _p(out))
    return out


def pair_bias_mask(P: Params, ct, bias_t: int, slot: int):
    ct = _u64(ct).copy()
    lib().oc_pair_bias_mask(P._cp, _p(ct), int(bias_t) % P.t, slot)
    return ct


def lr_packed(P: Params, keys: Keys, X_ct, W_pt, bias, return_pairs: bool = False):
    """Algorithm 1 with bias. X_ct [nX][K][2][L][N], W_pt [nY][K][N], bias [nY] (integers).
    Returns Y [ceil(nX nY / N)][2][L][N] (and the masked pair ciphertexts if asked)."""
    X_ct, W_pt = _u64(X_ct), _u64(W_pt)
    nX, K = X_ct.shape[0], X_ct.shape[1]
    nY = W_pt.shape[0]
    bt = np.array([int(b) % P.t for b in bias], dtype=np.uint64)
    nout = -(-nX * nY // P.N)
    Y = np.empty((nout, 2, P.L, P.N), dtype=np.uint64)
    pairs = np.empty((nX * nY, 2, P.L, P.N), dtype=np.uint64) if return_pairs else None
    lib().oc_lr_packed(P._cp, _p(keys.gk_eval), _p(P._gel), len(P._gel), _p(X_ct), nX, _p(W_pt), _p(bt),
                       nY, K, _p(Y), _p(pairs) if return_pairs else None)
    return (Y, pairs) if return_pairs else Y


def lr_standard(P: Params, X_ct, W, bias):
    """Standard product. X_ct [nF][2][L][N] (slot i = individual i), W [nF][nY], bias [nY]."""
    X_ct = _u64(X_ct)
    W = np.ascontiguousarray(W, dtype=np.int64)
    nF, nY = W.shape
    bt = np.array([int(b) % P.t for b in bias], dtype=np.uint64)
    Y = np.empty((nY, 2, P.L, P.N), dtype=np.uint64)
    lib().oc_lr_standard(P._cp, _p(X_ct), nF, _p(W, _i64p), _p(bt), nY, _p(Y))
    return Y


def standard_coeff(w_col, x_vals, q: int) -> int:
    """sum_f w[f] * x[f] mod q for one output coefficient of the standard product."""
    w = np.ascontiguousarray(w_col, dtype=np.int64)
    x = _u64(x_vals)
    return int(lib().oc_standard_coeff(_p(w, _i64p), _p(x), w.size, q))


# --------------------------------------------------------------------------- packing (Section 4.2.2)

def pack_inputs(P: Params, X):
    """Binary/integer features X [nX][f] -> slot vectors [nX][K][N], K = ceil(f/N); feature
    k*N + s goes to chunk k, slot s; zero padding past f."""
    X = np.asarray(X, dtype=np.int64)
    nX, f = X.shape
    K = -(-f // P.N)
    S = np.zeros((nX, K * P.N), dtype=np.int64)
    S[:, :f] = X
    return S.reshape(nX, K, P.N)


def pack_weights(P: Params, W):
    """W [f][nY] -> transposed slot vectors [nY][K][N] (Section 4.2.2: the weights are transposed)."""
    W = np.asarray(W, dtype=np.int64)
    f, nY = W.shape
    K = -(-f // P.N)
    S = np.zeros((nY, K * P.N), dtype=np.int64)
    S[:, :f] = W.T
    return S.reshape(nY, K, P.N)


def expected_scores(X, W, b, t: int):
    """The closed form: (X W + b) mod t with exact integers."""
    X = np.asarray(X, dtype=np.int64)
    W = np.asarray(W, dtype=np.int64)
    return (X @ W + np.asarray(b, dtype=np.int64)[None, :]) % t


def packed_pipeline(P: Params, keys: Keys, X, W, b, enc_seed: int, return_pairs: bool = False):
    """Client encode+encrypt, server Algorithm 1, returns (X_ct, W_pt, Y[, pairs])."""
    Xs = pack_inputs(P, X)
    nX, K, _ = Xs.shape
    X_pt = encode(P, Xs.reshape(nX * K, P.N))
    X_ct = encrypt(P, keys, X_pt, enc_seed).reshape(nX, K, 2, P.L, P.N)
    W_pt = encode(P, pack_weights(P, W).reshape(-1, P.N)).reshape(W.shape[1], K, P.N)
    res = lr_packed(P, keys, X_ct, W_pt, b, return_pairs=return_pairs)
    if return_pairs:
        return X_ct, W_pt, res[0], res[1]
    return X_ct, W_pt, res


def unpack_packed_scores(P: Params, slots, nX: int, nY: int):
    """Decoded output slots [nout][N] -> scores [nX][nY]: pair g = i*nY + j is slot g mod N of
    output g // N."""
    flat = np.asarray(slots).reshape(-1)
    g = np.arange(nX * nY)
    return flat[(g // P.N) * P.N + g % P.N].reshape(nX, nY)


def crt_combine(r0, t0: int, r1, t1: int):
    """CRT plaintext pair (Section 4.2.2): element-wise, the integer x in (-t0 t1 / 2, t0 t1 / 2]
    with x = r0 mod t0 and x = r1 mod t1, by the textbook formula
    x = r0 t1 (t1^-1 mod t0) + r1 t0 (t0^-1 mod t1) mod t0 t1, in Python integers."""
    T = t0 * t1
    e0, e1 = t1 * pow(t1, -1, t0), t0 * pow(t0, -1, t1)
    a0 = np.asarray(r0).reshape(-1)
    a1 = np.asarray(r1).reshape(-1)
    out = []
    for u, v in zip(a0.tolist(), a1.tolist()):
        x = (int(u) * e0 + int(v) * e1) % T
        out.append(x - T if x > T // 2 else x)
    return np.array(out, dtype=np.int64).reshape(np.shape(r0))


def has_openmp() -> bool:
    return bool(lib().oc_has_openmp())
