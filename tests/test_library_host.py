"""CPU-side checks of the CUDA library: it builds, loads, exports every function declared in
include/bfv_lr.h, and its host-side parameter logic agrees with the oracle's independent
computation. No GPU compute is called here."""
import ctypes
import os
import re

import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bfv():
    import paper_2204_05496_gb300 as m
    m.build()
    return m


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bfv_lr.h")).read()
    return sorted(set(re.findall(r"^int\s+(bfv_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_function(bfv):
    names = declared_functions()
    assert len(names) >= 20
    lib = ctypes.CDLL(bfv.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(bfv.SIGNATURES)
    assert bfv.lib().bfv_abi_version() == 1


@pytest.mark.parametrize("shape", [synth.TINY, synth.PAPER16K, synth.WIDE32K])
def test_host_prime_rule_matches_oracle(bfv, shape):
    assert bfv.primes(shape.N, shape.L, shape.prime_bits, shape.t) == oracle.ntt_primes(shape.prime_bits, shape.N, shape.L + 1)


@pytest.mark.parametrize("num,den", [(16, 5), (8, 5), (3, 1)])
def test_host_gaussian_table_matches_oracle(bfv, num, den):
    # the library computes exp() in 120-bit binary fixed point, the oracle with 90-digit decimals
    assert bfv.gaussian_table(num, den) == oracle.gaussian_cdt(num, den)


def test_bad_parameters_rejected_on_host(bfv):
    p = bfv.Params(4096, 3, 36, 0, 65539, 16, 5)       # t = 65539 is not 1 mod 8192
    out = (ctypes.c_uint64 * 8)()
    assert bfv.lib().bfv_params_primes(ctypes.byref(p), ctypes.cast(out, ctypes.c_void_p)) == bfv.BFV_ERR_INVALID_ARG
    p = bfv.Params(3000, 3, 36, 0, 65537, 16, 5)
    assert bfv.lib().bfv_params_primes(ctypes.byref(p), ctypes.cast(out, ctypes.c_void_p)) == bfv.BFV_ERR_INVALID_ARG
    # primes must stay below 2^59: unreduced forward transforms and key sums reach 32q
    p = bfv.Params(4096, 3, 60, 0, 65537, 16, 5)
    assert bfv.lib().bfv_params_primes(ctypes.byref(p), ctypes.cast(out, ctypes.c_void_p)) == bfv.BFV_ERR_INVALID_ARG
    p = bfv.Params(4096, 3, 59, 0, 65537, 16, 5)
    assert bfv.lib().bfv_params_primes(ctypes.byref(p), ctypes.cast(out, ctypes.c_void_p)) == bfv.BFV_OK
    assert list(out)[:4] == oracle.ntt_primes(59, 4096, 4)


def test_null_handles_rejected_before_any_device_work(bfv):
    """Every entry point checks its handles and pointers first: with null handles each returns
    BFV_ERR_INVALID_ARG and touches no device (this runs without a GPU)."""
    L = bfv.lib()
    n = ctypes.c_size_t()
    budgets = (ctypes.c_int * 2)()
    assert L.bfv_noise_budget_workspace(None, 2, ctypes.byref(n)) == bfv.BFV_ERR_INVALID_ARG
    assert L.bfv_noise_budget(None, None, None, 2, ctypes.cast(budgets, ctypes.c_void_p), None, 0,
                              0) == bfv.BFV_ERR_INVALID_ARG
    assert L.bfv_decrypt_workspace(None, 2, ctypes.byref(n)) == bfv.BFV_ERR_INVALID_ARG
    assert L.bfv_lr_scores_packed_workspace(None, None, 1, 0, ctypes.byref(n)) == bfv.BFV_ERR_INVALID_ARG
    assert L.bfv_lr_predict_packed_workspace(None, None, 1, 0, ctypes.byref(n)) == bfv.BFV_ERR_INVALID_ARG
    assert L.bfv_lr_predict_packed(None, None, None, None, 1, 0, None, None, 0, 0, 0) == bfv.BFV_ERR_INVALID_ARG
    assert L.bfv_lr_scores_packed(None, None, None, None, 1, None, None, 0, 0, 0) == bfv.BFV_ERR_INVALID_ARG
    assert L.bfv_crt_combine(None, 5, None, 9, 4, None, 0) == bfv.BFV_ERR_INVALID_ARG     # null arrays
    assert L.bfv_crt_combine(None, 6, None, 9, 0, None, 0) == bfv.BFV_ERR_INVALID_ARG     # gcd(6, 9) = 3
    assert L.bfv_crt_combine(None, 1 << 31, None, (1 << 31) + 1, 0, None, 0) == bfv.BFV_ERR_INVALID_ARG  # >= 2^62
    assert L.bfv_crt_combine(None, 5, None, 9, 0, None, 0) == bfv.BFV_OK                  # nothing to do


def test_setup_without_gpu_fails_loudly(bfv):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = bfv.Params(4096, 3, 36, 0, 65537, 16, 5)
    h = ctypes.c_void_p()
    rc = bfv.lib().bfv_setup(ctypes.byref(p), ctypes.byref(h))
    assert rc != bfv.BFV_OK and not h.value
    with pytest.raises(RuntimeError):
        bfv.Context(4096, 3, 36, 65537)


def test_binding_refuses_buffers_the_library_would_overrun(bfv):
    """The binding's buffer checks, on host memory: a host buffer must have the element size and
    shape the C call reads, an output must already be contiguous, and a device argument must be
    in device memory."""
    import numpy as np
    import torch
    x = np.zeros((3, 10), dtype=np.uint8)
    assert bfv._host_buf(x, "X", 1, (3, 10)) is x
    assert bfv._host_buf(x.T.copy().T, "X", 1, (3, 10)).flags.c_contiguous      # copied contiguous
    for bad, size, shape in ((x[:, :9], 1, (3, 10)), (x.astype(np.int64), 1, (3, 10)), (x, 8, (3, 10))):
        with pytest.raises(ValueError):
            bfv._host_buf(bad, "X", size, shape)
    with pytest.raises(ValueError):
        bfv._host_buf(np.zeros((10, 3), dtype=np.int64).T, "out", 8, (3, 10), out=True)
    assert bfv._host_buf(torch.zeros((3, 10), dtype=torch.int64), "out", 8, (3, 10), out=True).shape == (3, 10)
    for f in (lambda t: bfv._dev_in(t, "X", 8), lambda t: bfv._dev_out(t, "out", 8, 30)):
        with pytest.raises(ValueError):
            f(torch.zeros((3, 10), dtype=torch.int64))                          # host memory


def test_binding_calls_run_on_their_stream(bfv, monkeypatch):
    """Every binding call that takes a stream runs with it as the current stream (so its own
    allocations follow that stream), whether the stream is passed by keyword or by position;
    without one it runs on the current stream unchanged."""
    import contextlib
    import inspect
    import torch
    for name, fn in vars(bfv.Context).items():
        if inspect.isfunction(fn) and "stream" in inspect.signature(fn).parameters:
            assert hasattr(fn, "__wrapped__"), name
    entered = []

    @contextlib.contextmanager
    def fake_stream(s):
        entered.append(s)
        yield s
    monkeypatch.setattr(torch.cuda, "stream", fake_stream)
    seen = []

    @bfv._on_call_stream
    def call(a, b=None, stream=None):
        seen.append((a, b, stream))
        return a

    assert call(1) == 1 and entered == []
    assert call(2, stream="s1") == 2 and entered == ["s1"]
    assert call(3, 4, "s2") == 3 and entered == ["s1", "s2"]
    assert seen == [(1, None, None), (2, None, "s1"), (3, 4, "s2")]


def test_product_code_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2204_05496_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b", src), f
    for f in ("bfv_lr.h",):
        assert "oracle" not in open(os.path.join(ROOT, "include", f)).read()


@pytest.mark.parametrize("logn,split", [(lg, sp) for lg in (12, 13, 14, 15) for sp in (2, 4)])
def test_modup_tensor_memory_layout_is_a_partition(logn, split):
    """ModUp's key sums in tensor memory: thread t of warp w owns points t + e NT (e < PTS) and
    keeps each in lane 32 (w % 4) + t % 32, columns 4 PTS (w / 4) + 4 e .. + 3. For every ring
    the cells of all threads must tile the allocation (128 lanes x H/32 columns, a power of two
    in 32..512) exactly once, every point must be owned once, and a warp's accesses (16 columns
    at a time) must stay inside its 32-lane quarter and the allocation."""
    logh = logn - (1 if split == 2 else 2)
    H = 1 << logh
    # threads per ModUp CTA: halves as before, quarters 256 from 8,192 points up, else 128
    nt = {11: 128, 12: 256, 13: 256, 14: 512}[logh] if split == 2 else (256 if logh >= 13 else 128)
    pts, cols = H // nt, H // 32
    assert pts % 4 == 0 and 32 <= cols <= 512 and cols & (cols - 1) == 0
    cells, points = set(), set()
    for t in range(nt):
        w, lane = t // 32, 32 * ((t // 32) % 4) + t % 32
        base = 4 * pts * (w // 4)
        for e in range(pts):
            points.add(t + e * nt)
            for k in range(4):
                cells.add((lane, base + 4 * e + k))
        for e0 in range(0, pts, 4):
            first = base + 4 * e0
            assert first % 16 == 0 and first + 15 < cols
    assert points == set(range(H))
    assert cells == {(ln, c) for ln in range(128) for c in range(cols)}


def test_release_library_is_not_the_bounds_checked_build(bfv):
    """The release library reports no bounds checks; the bounds-checked build is a separate
    variant (libbfv_lr_bounds.so, selected with BFV_LIB_VARIANT=bounds)."""
    assert bfv.lib().bfv_bounds_checked() == 0
    assert bfv.VARIANTS["bounds"][1] == ["-DBFV_BOUNDS"]
