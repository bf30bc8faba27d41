"""Pins for the CPU oracle: each check ties an oracle function to something other than
itself - a published test vector, the textbook definition evaluated with Python integers,
an invariant of the scheme, or the closed form x.W + b mod t that the paper's protocol
must reproduce (Section 4.2.2: the client obtains W x + b after decrypting)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import sympy

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def small():
    # N = 16 ring, three 30-bit ciphertext primes + special prime, t = 97 = 1 mod 32
    return oracle.Params(16, 3, 30, 97)


@pytest.fixture(scope="module")
def small_keys(small):
    return oracle.keygen(small, 7)


@pytest.fixture(scope="module")
def tiny():
    return oracle.Params.from_shape(synth.TINY)


@pytest.fixture(scope="module")
def tiny_keys(tiny):
    return oracle.keygen(tiny, synth.WORKLOADS["tiny-1"].seed_keys)


def py_negacyclic(a, b, q):
    """Schoolbook product in Z_q[X]/(X^N + 1): the definition."""
    N = len(a)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            if i + j < N:
                out[i + j] += int(a[i]) * int(b[j])
            else:
                out[i + j - N] -= int(a[i]) * int(b[j])
    return [x % q for x in out]


def lift(vals, q):
    return np.array([int(v) % q for v in vals], dtype=np.uint64)


# ----------------------------------------------------------------------------- ChaCha20

def _golden_words(key):
    for line in open(os.path.join(GOLDEN, "chacha20_rfc8439.txt")):
        if line.startswith(key + " "):
            return [int(w, 16) for w in line.split()[1:]]
    raise KeyError(key)


def test_chacha20_rfc8439_vectors():
    assert oracle.chacha_quarter(*_golden_words("quarter_in")) == _golden_words("quarter_out")
    out = oracle.chacha20_block(_golden_words("block_key"), _golden_words("block_counter")[0],
                                _golden_words("block_nonce"))
    assert [int(x) for x in out] == _golden_words("block_out")


def test_sampler_streams_are_deterministic_and_separated(small):
    a = oracle.sample_ternary(5, oracle.P_SK, 0, 4096)
    assert np.array_equal(a, oracle.sample_ternary(5, oracle.P_SK, 0, 4096))
    assert not np.array_equal(a, oracle.sample_ternary(6, oracle.P_SK, 0, 4096))
    assert not np.array_equal(a, oracle.sample_ternary(5, oracle.P_SK, 1, 4096))
    assert not np.array_equal(a, oracle.sample_ternary(5, oracle.P_ENC, 0, 4096))


def test_ternary_and_uniform_come_from_the_block_words(tiny):
    # ternary = floor(3 w / 2^32) - 1 of word 0; uniform = (128-bit words 0..3) mod q
    key = [9, 0, 0, 0, 0, 0, 0, 0]
    s = oracle.sample_ternary(9, oracle.P_SK, 0, 64)
    u = oracle.sample_uniform(tiny, 9, oracle.P_PK_A, 0, 1)
    for k in range(64):
        blk = oracle.chacha20_block(key, k, [oracle.P_SK, 0, 0])
        assert s[k] == (int(blk[0]) * 3 >> 32) - 1
        blk = oracle.chacha20_block(key, k, [oracle.P_PK_A, 0, 1])
        r = sum(int(blk[i]) << (32 * i) for i in range(4))
        assert int(u[k]) == r % tiny.qs[1]


def test_ternary_and_gaussian_statistics(tiny):
    s = np.concatenate([oracle.sample_ternary(11, oracle.P_SK, o, 4096) for o in range(8)]).astype(np.int64)
    counts = np.array([(s == v).sum() for v in (-1, 0, 1)])
    assert set(np.unique(s)) <= {-1, 0, 1}
    assert np.all(np.abs(counts / s.size - 1 / 3) < 0.02)
    e = np.concatenate([oracle.sample_gauss(tiny, 11, oracle.P_GK_E, o) for o in range(16)]).astype(np.int64)
    assert abs(e.mean()) < 0.1
    assert abs(e.var() / 3.2 ** 2 - 1) < 0.04
    assert np.abs(e).max() <= 19
    # symmetric: positive and negative values equally often
    assert abs((e > 0).mean() - (e < 0).mean()) < 0.02


def test_gaussian_table_against_float_evaluation():
    T = oracle.gaussian_cdt(16, 5)
    assert len(T) == 19                       # |x| <= floor(6 sigma) = 19
    assert all(a < b for a, b in zip(T, T[1:])) and T[-1] < 2 ** 64
    rho = [math.exp(-k * k / (2 * 3.2 ** 2)) for k in range(20)]
    Z = rho[0] + 2 * sum(rho[1:])
    cum = 0.0
    for k in range(19):
        cum += rho[0] if k == 0 else 2 * rho[k]
        assert abs(T[k] / 2 ** 64 - cum / Z) < 1e-14
    # variance of the tabulated distribution is sigma^2 up to the (negligible) truncation
    probs = [T[0] / 2 ** 64] + [(T[k] - T[k - 1]) / 2 ** 64 for k in range(1, 19)] + [1 - T[-1] / 2 ** 64]
    var = sum(p * k * k for k, p in enumerate(probs))
    assert abs(var - 10.24) < 1e-6


# ----------------------------------------------------------------------------- parameters

@pytest.mark.parametrize("bits,N,count", [(30, 16, 4), (36, 4096, 4), (43, 8192, 5), (54, 16384, 8), (55, 32768, 16)])
def test_prime_rule(bits, N, count):
    ps = oracle.ntt_primes(bits, N, count)
    assert len(ps) == count and ps == sorted(ps, reverse=True)
    for p in ps:
        assert sympy.isprime(p) and p % (2 * N) == 1 and p.bit_length() == bits
    # no prime = 1 mod 2N between the smallest chosen one and 2^bits is skipped
    c = (1 << bits) - 2 * N + 1
    while c > ps[-1]:
        assert sympy.isprime(c) == (c in ps)
        c -= 2 * N


def test_parameter_sizes():
    P16 = oracle.Params.from_shape(synth.PAPER16K)
    assert 425 <= math.log2(P16.Q * P16.P) <= 435          # "log Q about 430"
    assert P16.t == 786433 and (P16.t - 1) % (2 * 16384) == 0
    Pt = oracle.Params.from_shape(synth.TINY)
    assert (Pt.t - 1) % (2 * 4096) == 0
    for P in (P16, Pt):
        for q, psi in zip(P.qs, P.psis):
            assert pow(psi, P.N, q) == q - 1        # primitive 2N-th root
        g = sympy.primitive_root(P.t)           # smallest primitive root
        assert P.omega == pow(g, (P.t - 1) // (2 * P.N), P.t)
        assert pow(P.omega, P.N, P.t) == P.t - 1
        assert P.delta == P.Q // P.t


# ----------------------------------------------------------------------------- NTT

@pytest.mark.parametrize("N,bits", [(8, 30), (16, 30), (64, 36), (64, 54)])
def test_ntt_product_is_schoolbook_convolution(N, bits):
    q = oracle.ntt_primes(bits, N, 1)[0]
    psi = oracle.root_2n(q, N)
    rng = np.random.default_rng(N + bits)
    for _ in range(3):
        a = rng.integers(0, q, N, dtype=np.uint64)
        b = rng.integers(0, q, N, dtype=np.uint64)
        assert [int(x) for x in oracle.polymul(a, b, q, psi)] == py_negacyclic(a, b, q)


def test_ntt_product_large_against_c_schoolbook():
    N = 512
    q = oracle.ntt_primes(54, 16384, 1)[0]
    psi = oracle.root_2n(q, N)
    rng = np.random.default_rng(3)
    a = rng.integers(0, q, N, dtype=np.uint64)
    b = rng.integers(0, q, N, dtype=np.uint64)
    assert np.array_equal(oracle.polymul(a, b, q, psi), oracle.polymul_schoolbook(a, b, q))
    # and the C schoolbook agrees with the Python definition on spot coefficients
    full = oracle.polymul_schoolbook(a, b, q)
    for k in (0, 1, 255, 511):
        s = sum(int(a[i]) * int(b[k - i]) for i in range(k + 1)) - sum(int(a[i]) * int(b[N + k - i]) for i in range(k + 1, N))
        assert int(full[k]) == s % q


@pytest.mark.parametrize("N", [16, 4096])
def test_ntt_is_evaluation_at_odd_powers(N):
    q = oracle.ntt_primes(54, N, 1)[0]
    psi = oracle.root_2n(q, N)
    rng = np.random.default_rng(N)
    a = rng.integers(0, q, N, dtype=np.uint64)
    A = oracle.ntt_forward(a, q, psi)
    ms = range(N) if N <= 16 else [0, 1, 77, N // 2, N - 1]
    al = [int(x) for x in a]
    for m in ms:
        z = pow(psi, 2 * m + 1, q)
        v = 0
        for c in reversed(al):          # Horner
            v = (v * z + c) % q
        assert int(A[m]) == v
    assert np.array_equal(oracle.ntt_inverse(A, q, psi), a)


# ----------------------------------------------------------------------------- encoding

@pytest.mark.parametrize("shape", ["small", "tiny"])
def test_encode_is_slot_evaluation(shape, small, tiny):
    P = small if shape == "small" else tiny
    N, t = P.N, P.t
    v = synth.slots(1, 1, N, t)[0]
    m = oracle.encode(P, v)
    e = oracle.slot_exponents(N)
    assert sorted(e) == list(range(1, 2 * N, 2))        # every odd exponent exactly once
    ls = range(N) if N <= 16 else [0, 1, 2, N // 2 - 1, N // 2, N // 2 + 5, N - 1]
    ml = [int(x) for x in m]
    for l in ls:
        z = pow(P.omega, e[l], t)
        val = 0
        for c in reversed(ml):
            val = (val * z + c) % t
        assert val == v[l]
    assert np.array_equal(oracle.decode(P, m), v)
    # negative slot values are taken mod t
    assert np.array_equal(oracle.decode(P, oracle.encode(P, v - t)), v)


def test_automorphism_is_a_ring_homomorphism(small):
    q = small.qs[0]
    rng = np.random.default_rng(5)
    a = rng.integers(0, q, 16, dtype=np.uint64)
    b = rng.integers(0, q, 16, dtype=np.uint64)
    for g in (3, 5, 9, 31, 27):
        lhs = oracle.automorph(np.array(py_negacyclic(a, b, q), dtype=np.uint64), q, g)
        rhs = py_negacyclic(oracle.automorph(a, q, g), oracle.automorph(b, q, g), q)
        assert [int(x) for x in lhs] == rhs
        for h in (3, 7, 31):
            assert np.array_equal(oracle.automorph(oracle.automorph(a, q, h), q, g),
                                  oracle.automorph(a, q, g * h % 32))
    # X -> X^3 on the monomial X^6: X^18 = -X^2
    x6 = np.zeros(16, dtype=np.uint64)
    x6[6] = 1
    out = oracle.automorph(x6, q, 3)
    assert int(out[2]) == q - 1 and int(out.sum()) == q - 1


@pytest.mark.parametrize("shape", ["small", "tiny"])
def test_galois_elements_rotate_rows_and_swap(shape, small, tiny):
    P = small if shape == "small" else tiny
    N, t = P.N, P.t
    v = synth.slots(2, 1, N, t)[0]
    m = oracle.encode(P, v)
    rows = v.reshape(2, N // 2)
    for s in (1, 2, N // 4):
        rot = oracle.decode(P, oracle.automorph(m, t, pow(3, s, 2 * N)))
        assert np.array_equal(rot.reshape(2, N // 2), np.roll(rows, -s, axis=1))
    sw = oracle.decode(P, oracle.automorph(m, t, 2 * N - 1))
    assert np.array_equal(sw.reshape(2, N // 2), rows[::-1])
    # the rotate-and-sum sequence: log2 N steps p += sigma_g(p) leave the total in every slot
    assert oracle.galois_elements(N) == [2 * N - 1] + [pow(3, N >> k, 2 * N) for k in range(2, P.logN + 1)]
    assert len(oracle.galois_elements(N)) == P.logN
    p = m.copy()
    for g in oracle.galois_elements(N):
        p = (p + oracle.automorph(p, t, g)) % t
    assert np.all(oracle.decode(P, p) == int(v.sum()) % t)


@pytest.mark.parametrize("shape", ["small", "tiny"])
def test_slot_masks_are_automorphisms_of_the_slot0_mask(shape, small, tiny):
    """The mask step's one-hot plaintext at slot s is X -> X^f applied to the one at slot 0,
    f = e_s^-1 mod 2N (e_s the slot's exponent): the identity the library's bias/mask kernel uses
    to gather every slot's mask from one transformed mask per limb."""
    P = small if shape == "small" else tiny
    N, t = P.N, P.t
    e = oracle.slot_exponents(N)
    one_hot = np.zeros(N, dtype=np.int64)
    one_hot[0] = 1
    mask0 = oracle.encode(P, one_hot)
    for s in sorted({0, 1, 2, N // 4, N // 2 - 1, N // 2, N // 2 + 3, N - 1}):
        one_hot[:] = 0
        one_hot[s] = 1
        f = pow(e[s], -1, 2 * N)
        assert f == (pow(3, (N // 2 - s % (N // 2)) % (N // 2), 2 * N) * (1 if s < N // 2 else -1)) % (2 * N)
        assert np.array_equal(oracle.encode(P, one_hot), oracle.automorph(mask0, t, f)), s


# ----------------------------------------------------------------------------- keys and encryption

def test_public_key_relation(small, small_keys):
    # pk0 + pk1 s = -e, pk1 = a (uniform), limb by limb, checked with schoolbook products
    e = oracle.sample_gauss(small, 7, oracle.P_PK_E, 0)
    for l, q in enumerate(small.q):
        a = oracle.sample_uniform(small, 7, oracle.P_PK_A, 0, l)
        assert np.array_equal(small_keys.pk[1, l], a)
        lhs = [(int(x) + y) % q for x, y in zip(small_keys.pk[0, l], py_negacyclic(a, lift(small_keys.sk, q), q))]
        assert lhs == [(-int(x)) % q for x in e]
    assert np.array_equal(small_keys.sk, oracle.sample_ternary(7, oracle.P_SK, 0, 16))


def test_galois_key_relation(small, small_keys):
    # k0[i][j] + k1[i][j] s = e_i + [i == j] [P]_{q_j} sigma_g(s)  (mod q_j, over all of QP)
    for gi, g in enumerate(small.galois):
        for i in range(small.L):
            e = oracle.sample_gauss(small, 7, oracle.P_GK_E, gi * 256 + i)
            for j, q in enumerate(small.qs):
                k0 = small_keys.gk_coeff[gi, i, 0, j]
                k1 = small_keys.gk_coeff[gi, i, 1, j]
                lhs = [(int(x) + y) % q for x, y in zip(k0, py_negacyclic(k1, lift(small_keys.sk, q), q))]
                rhs = [int(x) % q for x in e]
                if i == j:
                    sg = oracle.automorph(lift(small_keys.sk, q), q, g)
                    rhs = [(r + (small.P % q) * int(x)) % q for r, x in zip(rhs, sg)]
                assert lhs == rhs


def test_encryption_relation(small, small_keys):
    # c0 + c1 s = Delta m + e1 - u e + e2 s  (mod q_l)
    m = np.random.default_rng(1).integers(0, small.t, 16, dtype=np.uint64)
    ct = oracle.encrypt(small, small_keys, m[None, :], seed=99, obj0=5)[0]
    u, e1, e2 = oracle.sample_enc(small, 99, 5)
    e = oracle.sample_gauss(small, 7, oracle.P_PK_E, 0)
    for l, q in enumerate(small.q):
        s = lift(small_keys.sk, q)
        lhs = [(int(x) + y) % q for x, y in zip(ct[0, l], py_negacyclic(ct[1, l], s, q))]
        ue = py_negacyclic(lift(u, q), lift(e, q), q)
        e2s = py_negacyclic(lift(e2, q), s, q)
        rhs = [(small.delta * int(m[k]) + int(e1[k]) - ue[k] + e2s[k]) % q for k in range(16)]
        assert lhs == rhs


def test_encrypt_decrypt_roundtrip(tiny, tiny_keys):
    v = synth.slots(3, 4, tiny.N, tiny.t)
    ct = oracle.encrypt(tiny, tiny_keys, oracle.encode(tiny, v), seed=5)
    assert np.array_equal(oracle.decode(tiny, oracle.decrypt(tiny, tiny_keys.sk, ct)), v)
    assert oracle.noise_budget_bits(tiny, tiny_keys.sk, ct) > 70


def test_noise_budget_closed_form(small):
    """A ciphertext (Delta m + e, 0) has x = Delta m + e exactly, so t x = t e - (Q mod t) m
    modulo Q: the noise integer z follows from the chosen e and m without any CRT. The budget
    is the bit-length formula on max |z|, and every case still decrypts to m."""
    sk = np.zeros(16, dtype=np.int8)                    # c1 = 0: the secret plays no part
    rng = np.random.default_rng(19)
    Q, t = small.Q, small.t
    delta, r = Q // t, Q % t
    for e_mag in (0, 1, 1000, 2 ** 40, Q // (4 * t)):
        m = [int(v) for v in rng.integers(0, t, 16)]
        e = [int(rng.integers(-2 ** 62, 2 ** 62)) * e_mag // 2 ** 62 for _ in range(16)]
        e[3] = e_mag                                    # the extreme value occurs
        ct = np.zeros((1, 2, small.L, 16), dtype=np.uint64)
        for k in range(16):
            for l, q in enumerate(small.q):
                ct[0, 0, l, k] = (delta * m[k] + e[k]) % q
        z = [t * e[k] - r * m[k] for k in range(16)]
        assert max(abs(v) for v in z) < Q // 2          # no wrap: z is the centred residue
        want = max(0, Q.bit_length() - max(abs(v) for v in z).bit_length() - 1)
        assert oracle.noise_budget(small, sk, ct) == [want]
        assert [int(v) for v in oracle.decrypt(small, sk, ct)[0]] == m
    assert oracle.noise_budget(small, sk, np.zeros((1, 2, small.L, 16), dtype=np.uint64)) == [Q.bit_length() - 1]


def test_noise_budget_falls_with_each_operation(tiny, tiny_keys):
    """Fresh encryption, then a ciphertext-plaintext product, then the whole packed product:
    the budget falls at each step, stays positive while decryption is right, and agrees with
    the real-valued budget to within one bit."""
    w = synth.WORKLOADS["tiny-16"]
    X, W, b = synth.workload_inputs(w)
    X_ct, _, Y = oracle.packed_pipeline(tiny, tiny_keys, X, W, b, w.seed_enc)
    x0 = X_ct[0, 0]
    wpt = oracle.encode(tiny, oracle.pack_weights(tiny, W)[0, 0])
    prod = oracle.mul_plain(tiny, x0, wpt)
    b0, b1, b2 = (oracle.noise_budget(tiny, tiny_keys.sk, c[None])[0] for c in (x0, prod, Y[0]))
    assert b0 > b1 > b2 > 0
    for c, bud in ((x0, b0), (prod, b1), (Y[0], b2)):
        assert abs(bud - oracle.noise_budget_bits(tiny, tiny_keys.sk, c[None])) < 1


def test_decrypt_rounds_to_nearest(small):
    # a ciphertext (x, 0) decrypts to round(t x / Q) mod t for any x in [0, Q)
    sk = np.zeros(16, dtype=np.int8)
    rng = np.random.default_rng(8)
    Q, t = small.Q, small.t
    xs = [int(rng.integers(0, 2 ** 62)) * int(rng.integers(0, 2 ** 62)) % Q for _ in range(13)]
    xs += [Q // t // 2, Q // t // 2 + 1, Q - 1]           # near the half-way points
    ct = np.zeros((1, 2, small.L, 16), dtype=np.uint64)
    for k, x in enumerate(xs):
        for l, q in enumerate(small.q):
            ct[0, 0, l, k] = x % q
    m = oracle.decrypt(small, sk, ct)[0]
    for k, x in enumerate(xs):
        r = Fraction(t * x, Q)
        assert abs(r - int(m[k])) <= Fraction(1, 2) or abs(r - int(m[k]) - t) <= Fraction(1, 2)


def test_moddown_divides_by_p_with_rounding(small):
    Q, P = small.Q, small.P
    rng = np.random.default_rng(4)
    Us = [int(rng.integers(0, 2 ** 63)) ** 2 % (Q * P) for _ in range(12)]
    x0 = 123456789 % Q
    Us += [P * x0 + P // 2 - 1, P * x0 - P // 2 + 1, P * x0, (Q * P - 1)]
    U = np.zeros((small.L + 1, 16), dtype=np.uint64)
    for k, u in enumerate(Us):
        for j, q in enumerate(small.qs):
            U[j, k] = u % q
    out = oracle.moddown(small, U)
    for k, u in enumerate(Us):
        want = math.floor(Fraction(u, P) + Fraction(1, 2)) % Q
        assert [int(out[l, k]) for l in range(small.L)] == [want % q for q in small.q]


def test_keyswitch_preserves_the_secret_relation(tiny, tiny_keys):
    # (u0, u1) = KS_g(d): u0 + u1 s = d sigma_g(s) + err (mod Q). Over QP the key product gives
    # P d sigma_g(s) + sum_i d_i e_i, so after rounding by P, |err| <= sum_i |d_i e_i| / P + |eps0 +
    # eps1 s| <= L N max(q) B / P + (1 + N) / 2, with B = floor(6 sigma) the error cutoff and
    # |eps| <= 1/2 the two roundings
    rng = np.random.default_rng(12)
    d = np.stack([rng.integers(0, q, tiny.N, dtype=np.uint64) for q in tiny.q])
    for gi in (0, 3):
        g = tiny.galois[gi]
        u0, u1 = oracle.keyswitch(tiny, tiny_keys.gk_eval[gi], d)
        res = np.empty_like(u0)
        for l, q in enumerate(tiny.q):
            s = lift(tiny_keys.sk, q)
            sg = oracle.automorph(s, q, g)
            lhs = (u0[l].astype(object) + oracle.polymul(u1[l], s, q, tiny.psis[l]).astype(object)) % q
            rhs = oracle.polymul(d[l], sg, q, tiny.psis[l]).astype(object)
            res[l] = ((lhs - rhs) % q).astype(np.uint64)
        errs = oracle._crt(tiny, res)
        worst = max(min(v, tiny.Q - v) for v in errs)
        B = int(6 * Fraction(16, 5))
        bound = tiny.L * tiny.N * max(tiny.q) * B // tiny.P + (1 + tiny.N) // 2 + 1
        assert 0 < worst <= bound < 2 ** 18


def test_rotation_decrypts_to_rotated_slots(tiny, tiny_keys):
    v = synth.slots(4, 1, tiny.N, tiny.t)[0]
    ct = oracle.encrypt(tiny, tiny_keys, oracle.encode(tiny, v)[None, :], seed=6)[0]
    rows = v.reshape(2, tiny.N // 2)
    for gi in (0, 1, tiny.logN - 1):
        g = tiny.galois[gi]
        out = oracle.rotate(tiny, tiny_keys.gk_eval[gi], g, ct)
        got = oracle.decode(tiny, oracle.decrypt(tiny, tiny_keys.sk, out[None])[0]).reshape(2, -1)
        if g == 2 * tiny.N - 1:
            want = rows[::-1]
        else:
            s = next(s for s in range(tiny.N // 2) if pow(3, s, 2 * tiny.N) == g)
            want = np.roll(rows, -s, axis=1)
        assert np.array_equal(got, want)


def test_mul_plain_uses_centred_lift(small):
    rng = np.random.default_rng(2)
    m = rng.integers(0, small.t, 16, dtype=np.uint64)
    one = np.zeros((2, small.L, 16), dtype=np.uint64)
    one[0, :, 0] = 1
    out = oracle.mul_plain(small, one, m)
    for l, q in enumerate(small.q):
        want = [(int(x) if int(x) <= (small.t - 1) // 2 else int(x) - small.t) % q for x in m]
        assert [int(x) for x in out[0, l]] == want
        assert not out[1, l].any()


# ----------------------------------------------------------------------------- Algorithm 1

def test_pair_rotsum_fills_every_slot_with_the_dot_product(tiny, tiny_keys):
    w = synth.WORKLOADS["tiny-1"]
    X, W, b = synth.workload_inputs(w)
    xs = oracle.pack_inputs(tiny, X)[0]          # [K][N]
    ws = oracle.pack_weights(tiny, W)[2]         # class 2
    xct = oracle.encrypt(tiny, tiny_keys, oracle.encode(tiny, xs), seed=w.seed_enc)
    c = oracle.pair_rotsum(tiny, tiny_keys, xct, oracle.encode(tiny, ws))
    slots = oracle.decode(tiny, oracle.decrypt(tiny, tiny_keys.sk, c[None])[0])
    assert np.all(slots == int(X[0].astype(np.int64) @ W[:, 2]) % tiny.t)
    # bias then mask: only slot l survives, holding dot + b
    l = 77
    cm = oracle.pair_bias_mask(tiny, c, int(b[2]), l)
    slots = oracle.decode(tiny, oracle.decrypt(tiny, tiny_keys.sk, cm[None])[0])
    want = np.zeros(tiny.N, dtype=np.int64)
    want[l] = (int(X[0].astype(np.int64) @ W[:, 2]) + int(b[2])) % tiny.t
    assert np.array_equal(slots, want)
    one_hot = np.zeros(tiny.N, dtype=np.int64)
    one_hot[l] = 1
    assert np.array_equal(oracle.decode(tiny, oracle.encode(tiny, one_hot)), one_hot)


@pytest.mark.parametrize("name", ["tiny-1", "tiny-16"])
def test_packed_scores_equal_closed_form(name, tiny, tiny_keys):
    w = synth.WORKLOADS[name]
    X, W, b = synth.workload_inputs(w)
    _, _, Y = oracle.packed_pipeline(tiny, tiny_keys, X, W, b, w.seed_enc)
    assert Y.shape[0] == -(-X.shape[0] * W.shape[1] // tiny.N)       # ceil(|X||Y| / n) outputs
    slots = oracle.decode(tiny, oracle.decrypt(tiny, tiny_keys.sk, Y))
    got = oracle.unpack_packed_scores(tiny, slots, X.shape[0], W.shape[1])
    assert np.array_equal(got, oracle.expected_scores(X, W, b, tiny.t))
    # every slot beyond the last pair is zero
    assert not slots.reshape(-1)[X.shape[0] * W.shape[1]:].any()
    assert oracle.noise_budget_bits(tiny, tiny_keys.sk, Y) > 10


def test_packed_compression_over_several_outputs(small, small_keys):
    # 5 individuals x 7 classes = 35 pairs > N = 16: three output ciphertexts, ragged tail;
    # f = 40 > N: K = 3 chunks, the last one zero-padded
    rng = np.random.default_rng(9)
    X = (rng.random((5, 40)) < 0.3).astype(np.uint8)
    W = rng.integers(-5, 6, (40, 7))
    b = rng.integers(-5, 6, 7)
    _, _, Y, pairs = oracle.packed_pipeline(small, small_keys, X, W, b, 31, return_pairs=True)
    assert Y.shape[0] == 3
    slots = oracle.decode(small, oracle.decrypt(small, small_keys.sk, Y))
    assert np.array_equal(oracle.unpack_packed_scores(small, slots, 5, 7), oracle.expected_scores(X, W, b, small.t))
    assert not slots.reshape(-1)[35:].any()
    # each masked pair decrypts to a one-hot vector at slot g mod N
    ps = oracle.decode(small, oracle.decrypt(small, small_keys.sk, pairs))
    exp = oracle.expected_scores(X, W, b, small.t).reshape(-1)
    for g in range(35):
        want = np.zeros(16, dtype=np.int64)
        want[g % 16] = exp[g]
        assert np.array_equal(ps[g], want)


def test_standard_scores_equal_closed_form(small, small_keys):
    rng = np.random.default_rng(10)
    nX, f, nY = 10, 40, 3
    X = (rng.random((nX, f)) < 0.3).astype(np.int64)
    W = rng.integers(-127, 128, (f, nY))
    b = rng.integers(-127, 128, nY)
    cols = np.zeros((f, small.N), dtype=np.int64)
    cols[:, :nX] = X.T                              # ciphertext f holds feature f of every individual
    X_ct = oracle.encrypt(small, small_keys, oracle.encode(small, cols), seed=12)
    Y = oracle.lr_standard(small, X_ct, W, b)
    slots = oracle.decode(small, oracle.decrypt(small, small_keys.sk, Y))
    assert np.array_equal(slots[:, :nX].T, oracle.expected_scores(X, W, b, small.t))
    # coefficient view: output = sum_f w_f X_f (+ Delta b at coefficient 0 of c0)
    for (c, l, k) in [(0, 0, 3), (1, 2, 15), (1, 0, 0)]:
        v = oracle.standard_coeff(W[:, 1], X_ct[:, c, l, k], small.q[l])
        assert int(Y[1, c, l, k]) == v


def test_reading_with_two_ciphertext_primes_fails(tiny):
    # "three 36-bit primes" read as 2 ciphertext primes + the special prime leaves no noise
    # budget for the tiny workload; the oracle uses 3 ciphertext primes + a fourth for P.
    w = synth.WORKLOADS["tiny-1"]
    X, W, b = synth.workload_inputs(w)
    PA = oracle.Params(4096, 2, 36, 65537)
    kA = oracle.keygen(PA, w.seed_keys)
    _, _, Y = oracle.packed_pipeline(PA, kA, X, W, b, w.seed_enc)
    got = oracle.unpack_packed_scores(PA, oracle.decode(PA, oracle.decrypt(PA, kA.sk, Y)), 1, 8)
    assert not np.array_equal(got, oracle.expected_scores(X, W, b, PA.t))
    assert oracle.noise_budget_bits(PA, kA.sk, Y) < 1


# ----------------------------------------------------------------------------- CRT plaintext pair

def test_crt_combine_recovers_integers():
    """Section 4.2.2's pair t0 = 1073872897, t1 = 114689: residues of any integer in
    (-t0 t1 / 2, t0 t1 / 2] recombine to it; checked against sympy's CRT as well."""
    from sympy.ntheory.modular import crt
    t0, t1 = 1073872897, 114689
    T = t0 * t1
    rng = np.random.default_rng(5)
    xs = [int(v) for v in rng.integers(-(T // 2) + 1, T // 2, size=200)] + [T // 2, -(T // 2) + 1, 0, 1, -1]
    r0 = np.array([x % t0 for x in xs], dtype=np.int64)
    r1 = np.array([x % t1 for x in xs], dtype=np.int64)
    got = oracle.crt_combine(r0, t0, r1, t1)
    assert got.tolist() == xs
    for x, a, b in zip(xs[:20], r0, r1):
        v, m = crt([t0, t1], [int(a), int(b)])
        assert m == T and (v - x) % T == 0


def test_fixed_point_precision_matches_paper():
    """Section 4.2.2: inputs below 2^8 scaled by 2^6, weights below 1 by 2^14; at f = 40,960 the
    scaled scores need 44 bits, which the CRT pair (about 46 bits) holds and one modulus does not."""
    import math
    from paper_2204_05496_gb300 import crt_pair
    assert crt_pair.bits_needed(40960) == 44
    assert math.log2(crt_pair.T0 * crt_pair.T1) > 44 + 1 > math.log2(crt_pair.T0)
    assert crt_pair.to_fixed([0.5, 255.99, 3.0], crt_pair.S_X).tolist() == [32, 16383, 192]
    assert crt_pair.to_fixed([-0.99994, 0.25], crt_pair.S_W).tolist() == [-16383, 4096]
