"""Seeded synthetic inputs for encrypted logistic-regression scoring.

This module only draws random numbers and names workload shapes. It holds none of
the BFV arithmetic, so both the CPU oracle and the CUDA path may use it.

The paper's data (iDASH 2020 Task I / TCGA somatic mutations, Section 2.1) and its
trained weights are not available. The inputs below stand in for them with the same
shape (Section 4.1.2, encoding 1): binary "SNV present" features per gene, drawn
Bernoulli(p), and integer weights and biases in the int8 range (the paper's model
has real weights scaled by 2^14; Section 4.2.2 - here the scale is 1 and the weights
are integers directly).
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass(frozen=True)
class BfvShape:
    """BFV parameter shape: ring degree N, number of ciphertext primes L, prime
    size in bits, plaintext modulus t, Gaussian width sigma = num/den."""
    N: int
    L: int
    prime_bits: int
    t: int
    sigma_num: int = 16
    sigma_den: int = 5


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    params: BfvShape
    n_features: int
    n_classes: int
    n_individuals: int
    p_feature: float
    seed_data: int
    seed_keys: int
    seed_enc: int


# Ring degree 4096, three 36-bit ciphertext primes (+ one 36-bit special prime),
# t = 65537 = 1 mod 8192.
TINY = BfvShape(N=4096, L=3, prime_bits=36, t=65537)
# Ring degree 16384, seven 54-bit ciphertext primes + one 54-bit special prime
# (log QP ~ 432), t = 786433 = 3*2^18 + 1 = 1 mod 32768.
PAPER16K = BfvShape(N=16384, L=7, prime_bits=54, t=786433)
# Ring degree 32768, fifteen 55-bit primes + special prime (log QP ~ 880).
WIDE32K = BfvShape(N=32768, L=15, prime_bits=55, t=786433)
# the paper's own parameter set (Section 5.2.3): N = 8192 with the CRT pair of plaintext moduli;
# 4 + 1 primes of 43 bits (log QP = 215, within the 218 bits SEAL allows at 128-bit security)
PAPER8K_T0 = BfvShape(N=8192, L=4, prime_bits=43, t=1073872897)
PAPER8K_T1 = BfvShape(N=8192, L=4, prime_bits=43, t=114689)

WORKLOADS = {
    "tiny-1": Workload("tiny-1", TINY, 1000, 8, 1, 0.05, 101, 102, 103),
    "tiny-16": Workload("tiny-16", TINY, 1000, 8, 16, 0.05, 101, 102, 103),
    "single-40k": Workload("single-40k", PAPER16K, 40000, 16, 1, 0.02, 201, 202, 203),
    "batch512-40k": Workload("batch512-40k", PAPER16K, 40000, 16, 512, 0.02, 301, 302, 303),
}


def features(seed: int, n_individuals: int, n_features: int, p: float) -> np.ndarray:
    """Binary feature matrix X (|X| x f, uint8), each entry Bernoulli(p)."""
    rng = np.random.default_rng([seed, 1])
    return (rng.random((n_individuals, n_features)) < p).astype(np.uint8)


def weights(seed: int, n_features: int, n_classes: int, lo: int = -127, hi: int = 127) -> np.ndarray:
    """Weight matrix W (f x |Y|, int64), uniform integers in [lo, hi]."""
    rng = np.random.default_rng([seed, 2])
    return rng.integers(lo, hi + 1, size=(n_features, n_classes), dtype=np.int64)


def bias(seed: int, n_classes: int, lo: int = -127, hi: int = 127) -> np.ndarray:
    """Bias vector b (|Y|, int64), uniform integers in [lo, hi]."""
    rng = np.random.default_rng([seed, 3])
    return rng.integers(lo, hi + 1, size=(n_classes,), dtype=np.int64)


def slots(seed: int, count: int, N: int, t: int) -> np.ndarray:
    """Uniform plaintext slot vectors in [0, t) (count x N, int64) for unit tests."""
    rng = np.random.default_rng([seed, 4])
    return rng.integers(0, t, size=(count, N), dtype=np.int64)


def workload_inputs(w: Workload):
    """(X, W, b) for a named workload."""
    X = features(w.seed_data, w.n_individuals, w.n_features, w.p_feature)
    W = weights(w.seed_data, w.n_features, w.n_classes)
    b = bias(w.seed_data, w.n_classes)
    return X, W, b


def uneven_models(seed: int = 401, count: int = 64):
    """Uneven batch: per model (f, |Y|, |X|, param set name) drawn as
    f in {1k, 5k, 20k, 40k}, |Y| in {2, 8, 16}, |X| uniform in [1, 512], and the
    ring degree 16384 or 32768 parameter set."""
    rng = np.random.default_rng([seed, 5])
    out = []
    for m in range(count):
        f = int(rng.choice([1000, 5000, 20000, 40000]))
        y = int(rng.choice([2, 8, 16]))
        x = int(rng.integers(1, 513))
        ps = "PAPER16K" if rng.random() < 0.5 else "WIDE32K"
        out.append((f, y, x, ps))
    return out


def uneven_batch(seed: int = 401, count: int = 64, x_divisor: int = 1):
    """Inputs of the uneven batch: for model m of uneven_models(seed, count) a dict with the
    parameter-set name, f, |Y|, |X| (the drawn batch size divided by x_divisor, rounded up),
    binary features X ~ Bernoulli(0.02) and int8-range weights W and bias b, generated from
    seed 1000 seed + m; enc_seed = 1000 seed + 500 + m seeds the model's encryptions."""
    out = []
    for m, (f, y, x, ps) in enumerate(uneven_models(seed, count)):
        nX = -(-x // x_divisor)
        sm = 1000 * seed + m
        out.append(dict(params=ps, f=f, nY=y, nX=nX, X=features(sm, nX, f, 0.02), W=weights(sm, f, y),
                        b=bias(sm, y), enc_seed=1000 * seed + 500 + m))
    return out


def paper_realvalued(seed: int, n_individuals: int, n_features: int, n_classes: int):
    """Real-valued inputs shaped like the paper's encodings (Section 4.1.2) and a real LR model:
    the first 57% of the columns are CNV features (integers 0..4, mostly 2), the rest SNV-impact
    features (a gene carries 1..3 SNVs with probability 0.02, each contributing m s with m in
    {1.0, 0.75, 0.5, 0.25} and s uniform in [0, 1)); all inputs lie in [0, 2^8). Weights are
    uniform in (-1, 1) with 70% set to zero (a Lasso-trained model), biases uniform in (-1, 1).
    Returns float64 (X [|X|][f], W [f][|Y|], b [|Y|])."""
    rng = np.random.default_rng([seed, 7])
    f_cnv = int(round(0.57 * n_features))
    X = np.zeros((n_individuals, n_features))
    X[:, :f_cnv] = rng.choice([0, 1, 2, 3, 4], size=(n_individuals, f_cnv), p=[0.05, 0.15, 0.6, 0.15, 0.05])
    f_snv = n_features - f_cnv
    present = rng.random((n_individuals, f_snv)) < 0.02
    count = rng.integers(1, 4, size=(n_individuals, f_snv))
    for k in range(3):
        m = rng.choice([1.0, 0.75, 0.5, 0.25], size=(n_individuals, f_snv))
        s = rng.random((n_individuals, f_snv))
        X[:, f_cnv:] += np.where(present & (count > k), m * s, 0.0)
    W = rng.uniform(-1, 1, size=(n_features, n_classes)) * (rng.random((n_features, n_classes)) < 0.3)
    b = rng.uniform(-1, 1, size=n_classes)
    return X, W, b


def poisson_arrivals(seed: int, rate_per_s: float, n_requests: int,
                     single_frac: float = 0.7, lo: int = 16, hi: int = 512):
    """Serving workload: (arrival time in s, number of individuals) per request.
    Exponential inter-arrival times; 70% single-individual requests, the rest
    uniform in [lo, hi] individuals."""
    rng = np.random.default_rng([seed, 6, int(rate_per_s)])
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    times = np.cumsum(gaps)
    sizes = np.where(rng.random(n_requests) < single_frac, 1,
                     rng.integers(lo, hi + 1, size=n_requests))
    return [(float(a), int(s)) for a, s in zip(times, sizes)]
