"""GB300 (sm_103a) library for BFV-encrypted logistic-regression scoring.

Thin Python binding over the C ABI in include/bfv_lr.h: every call marshals torch
tensors (device memory, streams) into plain pointers and calls the CUDA library of the
same name; every step of the encrypted path runs in the library's kernels. There is no
fallback: if the compiled library is missing, importing the binding's calls raises.

Paper: "Scalable privacy-preserving cancer type prediction with homomorphic encryption",
Section 4.2.2 (protocol), Section 4.2.3 / Algorithm 1 (packed product), Section 5.2.3
(standard product).
"""
from __future__ import annotations

import ctypes
import functools
import inspect
import json
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
# Build variants: the release library, and a bounds-checked one (-DBFV_BOUNDS: every global
# access of every kernel checked against the call's buffers, violations reported through the
# context's error word). BFV_LIB_VARIANT=bounds makes this process load the bounds-checked one.
VARIANTS = {"release": ("libbfv_lr.so", []), "bounds": ("libbfv_lr_bounds.so", ["-DBFV_BOUNDS"])}
VARIANT = os.environ.get("BFV_LIB_VARIANT", "release")
if VARIANT not in VARIANTS:
    raise RuntimeError(f"BFV_LIB_VARIANT={VARIANT!r}: one of {sorted(VARIANTS)} expected")
LIB_PATH = os.path.join(_BUILD, VARIANTS[VARIANT][0])
_ROOT = os.path.dirname(_HERE)
_INCLUDE = os.path.join(_ROOT, "include")
SOURCES = ["capi.cu", "k_scheme.cu", "k_packed.cu", "k_standard.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

BFV_OK, BFV_ERR_INVALID_ARG, BFV_ERR_BAD_PARAMS, BFV_ERR_OOM = 0, -1, -2, -3
BFV_OPT_ENCRYPT_SPLIT, BFV_OPT_STANDARD_KERNEL = 1, 2
BFV_INJECT_STREAM_STALL, BFV_INJECT_BOUNDS_SHRINK = 1, 2
BFV_ERR_OVER_BUDGET, BFV_ERR_TIMEOUT, BFV_ERR_CUDA = -4, -5, -6
_ERRS = {-1: "INVALID_ARG", -2: "BAD_PARAMS", -3: "OOM", -4: "OVER_BUDGET", -5: "TIMEOUT", -6: "CUDA"}


class BfvError(RuntimeError):
    def __init__(self, fn, rc):
        super().__init__(f"{fn} failed: BFV_ERR_{_ERRS.get(rc, rc)} ({rc})")
        self.code = rc


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False, variant: str | None = None) -> str:
    """Compile the CUDA library in-tree for sm_103a (translation units in parallel); `variant`
    (default: the one this process loads) "bounds" builds the bounds-checked library beside the
    release one."""
    variant = variant or VARIANT
    lib_name, extra = VARIANTS[variant]
    lib_path = os.path.join(_BUILD, lib_name)
    objdir = _BUILD if variant == "release" else os.path.join(_BUILD, variant)
    os.makedirs(objdir, exist_ok=True)
    deps = [os.path.join(_CSRC, f) for f in os.listdir(_CSRC)] + [os.path.join(_INCLUDE, "bfv_lr.h")]
    newest = max(os.path.getmtime(d) for d in deps)
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= newest:
        return lib_path
    nvcc = _nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
                    "-I", _INCLUDE, "-I", _CSRC] + extra

    def compile_one(src):
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [nvcc, "-c", os.path.join(_CSRC, src), "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout, r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib_path + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, "-shared", "-cudart", "shared", "-o", tmp] + ARCH + objs, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


class Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("L", ctypes.c_uint32), ("prime_bits", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("t", ctypes.c_uint64), ("sigma_num", ctypes.c_uint32),
                ("sigma_den", ctypes.c_uint32)]


class Schedule(ctypes.Structure):
    """bfv_packed_schedule: pair chunk and the CTAs per limb of each key-switching kernel."""
    _fields_ = [("pair_chunk", ctypes.c_uint64), ("prep_split", ctypes.c_uint32), ("modup_split", ctypes.c_uint32),
                ("moddown_p_split", ctypes.c_uint32), ("moddown_split", ctypes.c_uint32)]
    FIELDS = ("pair_chunk", "prep_split", "modup_split", "moddown_p_split", "moddown_split")

    def as_dict(self):
        return {k: int(getattr(self, k)) for k in self.FIELDS}

    @classmethod
    def from_dict(cls, d):
        return cls(*(int(d[k]) for k in cls.FIELDS))


_lib = None
_lock = threading.Lock()
_vp, _u64, _sz, _up = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_size_t

# (name, argtypes) of every exported function; the CPU tests check the library exports these.
SIGNATURES = {
    "bfv_abi_version": [],
    "bfv_params_primes": [ctypes.POINTER(Params), _vp],
    "bfv_gaussian_table": [ctypes.c_uint32, ctypes.c_uint32, _vp, ctypes.POINTER(ctypes.c_int)],
    "bfv_setup": [ctypes.POINTER(Params), ctypes.POINTER(_vp)],
    "bfv_ctx_free": [_vp],
    "bfv_ctx_query": [_vp, _vp, _vp, _vp],
    "bfv_keygen": [_vp, _u64, _up, ctypes.POINTER(_vp)],
    "bfv_keys_free": [_vp],
    "bfv_keys_export": [_vp, _vp, _vp, _vp, _vp, _up],
    "bfv_encode": [_vp, _vp, _sz, _vp, _up],
    "bfv_decode": [_vp, _vp, _sz, _vp, _up],
    "bfv_encode_features": [_vp, _vp, _sz, _sz, _vp, _up],
    "bfv_encode_feature_columns": [_vp, _vp, _sz, _sz, _vp, _up],
    "bfv_encrypt_workspace": [_vp, _sz, ctypes.POINTER(_sz)],
    "bfv_encrypt": [_vp, _vp, _vp, _sz, _u64, ctypes.c_uint32, _vp, _vp, _sz, _up],
    "bfv_decrypt_workspace": [_vp, _sz, ctypes.POINTER(_sz)],
    "bfv_decrypt": [_vp, _vp, _vp, _sz, _vp, _vp, _sz, _up],
    "bfv_noise_budget_workspace": [_vp, _sz, ctypes.POINTER(_sz)],
    "bfv_noise_budget": [_vp, _vp, _vp, _sz, _vp, _vp, _sz, _up],
    "bfv_model_prepare": [_vp, _vp, _vp, _sz, _sz, _up, ctypes.POINTER(_vp)],
    "bfv_model_free": [_vp],
    "bfv_lr_scores_packed_workspace": [_vp, _vp, _sz, _sz, ctypes.POINTER(_sz)],
    "bfv_lr_scores_packed": [_vp, _vp, _vp, _vp, _sz, _vp, _vp, _sz, _sz, _up],
    "bfv_lr_scores_standard_workspace": [_vp, _vp, ctypes.POINTER(_sz)],
    "bfv_lr_scores_standard": [_vp, _vp, _vp, _sz, _vp, _vp, _sz, _up],
    "bfv_check_error": [_vp, ctypes.POINTER(ctypes.c_int)],
    "bfv_debug_inject": [_vp, ctypes.c_int, ctypes.c_int],
    "bfv_decrypt_noalloc_max_count": [_vp, ctypes.POINTER(_sz)],
    "bfv_lr_scores_packed_multi_workspace": [_vp, _vp, ctypes.c_int, _vp, _sz, ctypes.POINTER(_sz)],
    "bfv_lr_scores_packed_multi": [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _sz, _sz, _up],
    "bfv_crt_combine": [_vp, ctypes.c_uint64, _vp, ctypes.c_uint64, _sz, _vp, _up],
    "bfv_lr_scores_packed_models_workspace": [_vp, ctypes.c_int, _vp, _vp, _sz, ctypes.POINTER(_sz)],
    "bfv_lr_scores_packed_models": [_vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _sz, _sz, _up],
    "bfv_lr_scores_packed_graph": [_vp, _vp, _vp, _vp, _sz, _vp, _vp, _sz, _sz, _up],
    "bfv_autotune_packed": [_vp, _vp, _vp, _vp, _sz, _vp, _vp, _sz, _up, ctypes.POINTER(_sz),
                            ctypes.POINTER(ctypes.c_double)],
    "bfv_decrypt_noalloc": [_vp, _vp, _vp, _sz, _vp, _up],
    "bfv_set_option": [_vp, ctypes.c_int, ctypes.c_int],
    "bfv_bounds_checked": [],
    "bfv_get_option": [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "bfv_packed_schedule_get": [_vp, _sz, ctypes.POINTER(Schedule)],
    "bfv_packed_schedule_set": [_vp, _sz, ctypes.POINTER(Schedule)],
    "bfv_lr_scores_packed_sched": [_vp, _vp, _vp, _vp, _sz, _vp, _vp, _sz, ctypes.POINTER(Schedule), _up],
    "bfv_autotune_packed_schedule": [_vp, _vp, _vp, _vp, _sz, _vp, _vp, _sz, _up, ctypes.POINTER(Schedule),
                                     ctypes.POINTER(ctypes.c_double)],
    "bfv_lr_packed_pair_from_workspace": [_vp, _vp, _sz, _sz, _vp, _sz, _vp, _up],
    "bfv_launch_count": [_vp, ctypes.POINTER(_u64)],
    "bfv_lr_predict_packed_workspace": [_vp, _vp, _sz, _sz, ctypes.POINTER(_sz)],
    "bfv_lr_predict_packed": [_vp, _vp, _vp, _vp, _sz, _u64, _vp, _vp, _sz, _sz, _up],
    "bfv_lr_predict_packed_host": [_vp, _vp, _vp, _vp, _sz, _u64, _vp, _vp, _sz, _sz, _up],
    "bfv_profile": [_vp, ctypes.c_int],
    "bfv_profile_read": [_vp, ctypes.c_int, ctypes.POINTER(_u64), ctypes.POINTER(ctypes.c_double)],
}

# Kernel kinds of bfv_profile_read (BFV_K_* in include/bfv_lr.h).
KERNEL_KINDS = ["ntt", "ks_prep", "ks_modup", "ks_moddown_p", "ks_moddown", "mac", "bias_mask", "compress",
                "encrypt", "decrypt", "encode", "standard"]


def lib():
    """The loaded CUDA library; raises if it has not been built (no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            _lib = L
    return _lib


def _call(name, *args):
    rc = getattr(lib(), name)(*args)
    if rc != BFV_OK:
        raise BfvError(name, rc)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


# The C calls trust the sizes they are given and read or write exactly the bytes those imply, so
# the binding checks every caller tensor against them before a pointer is passed on.
def _dev_in(t, name, itemsize, numel=None, block=None):
    """A device tensor the library reads: element size and count checked, returned contiguous."""
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name}: a CUDA tensor is expected")
    if t.element_size() != itemsize:
        raise ValueError(f"{name}: {itemsize}-byte elements expected, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name}: {numel} elements expected, got {t.numel()}")
    if block is not None and t.numel() % block:
        raise ValueError(f"{name}: a whole number of {block}-element blocks expected, got {t.numel()}")
    return t.contiguous()


def _dev_out(t, name, itemsize, numel):
    """A caller-supplied output: written in place, so contiguous and exactly the written size."""
    if not getattr(t, "is_cuda", False) or not t.is_contiguous():
        raise ValueError(f"{name}: a contiguous CUDA tensor is expected")
    if t.element_size() != itemsize or t.numel() != numel:
        raise ValueError(f"{name}: {numel} elements of {itemsize} bytes expected, got {t.numel()} of "
                         f"{t.element_size()}")
    return t


def _host_buf(a, name, itemsize, shape, out=False):
    """A host array (numpy or CPU torch tensor) passed by address: dtype size and shape checked;
    inputs are made contiguous, outputs must already be."""
    if hasattr(a, "is_cuda"):
        if a.is_cuda:
            raise ValueError(f"{name}: a host buffer is expected")
        size, shp, contig = a.element_size(), tuple(a.shape), a.is_contiguous()
    else:
        a = np.asarray(a) if not out else a
        size, shp, contig = a.itemsize, a.shape, a.flags.c_contiguous
    if size != itemsize or shp != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(shape)} of {itemsize}-byte elements expected, got {shp} of {size}")
    if not contig:
        if out:
            raise ValueError(f"{name}: a contiguous buffer is expected")
        a = a.contiguous() if hasattr(a, "is_cuda") else np.ascontiguousarray(a)
    return a


def _addr(a):
    return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data


def _workspace(ws, need, device):
    """The caller's workspace if it is a large enough device buffer, else a fresh one; returns
    (tensor, size in bytes)."""
    import torch
    if ws is None or ws.numel() * ws.element_size() < need:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=device)
    elif not ws.is_cuda or not ws.is_contiguous():
        raise ValueError("ws: a contiguous CUDA tensor is expected")
    return ws, ws.numel() * ws.element_size()


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


# Autotuned packed-product schedules shipped with the package (written by
# `bench.py --autotune-save` on a GB300), keyed "N=...,L=...,pairs=...".
SCHEDULE_FILE = os.path.join(_HERE, "schedules.json")


def load_schedule_file(path: str) -> dict:
    """{key: schedule fields} of a schedule file written by Context.save_schedules ({} if absent)."""
    try:
        with open(path) as f:
            data = json.load(f)
    except FileNotFoundError:
        return {}
    if not isinstance(data, dict):
        raise ValueError(f"{path}: a JSON object of schedules expected")
    for k, d in data.items():
        if set(d) != set(Schedule.FIELDS):
            raise ValueError(f"{path}: schedule {k} must have exactly the fields {Schedule.FIELDS}")
    return data


def primes(N: int, L: int, prime_bits: int, t: int) -> list[int]:
    """The L+1 primes of a parameter shape (host computation)."""
    p = Params(N, L, prime_bits, 0, t, 16, 5)
    out = (ctypes.c_uint64 * (L + 1))()
    _call("bfv_params_primes", ctypes.byref(p), ctypes.cast(out, _vp))
    return list(out)


def gaussian_table(num: int = 16, den: int = 5) -> list[int]:
    out = (ctypes.c_uint64 * 32)()
    n = ctypes.c_int()
    _call("bfv_gaussian_table", num, den, ctypes.cast(out, _vp), ctypes.byref(n))
    return list(out)[: n.value]


class Keys:
    def __init__(self, ctx, handle):
        self.ctx, self.handle = ctx, handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bfv_keys_free(self.handle)
            self.handle = None


class Model:
    def __init__(self, ctx, handle, f, nY):
        self.ctx, self.handle, self.f, self.nY = ctx, handle, f, nY
        self.K = -(-f // ctx.N)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bfv_model_free(self.handle)
            self.handle = None


class Context:
    """A BFV parameter set on the current CUDA device (bfv_setup)."""

    def __init__(self, N: int, L: int, prime_bits: int, t: int, sigma_num: int = 16, sigma_den: int = 5):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the library has no CPU path")
        self.N, self.L, self.t = N, L, t
        self.params = Params(N, L, prime_bits, 0, t, sigma_num, sigma_den)
        h = _vp()
        _call("bfv_setup", ctypes.byref(self.params), ctypes.byref(h))
        self.handle = h
        pr = (ctypes.c_uint64 * (L + 1))()
        om = ctypes.c_uint64()
        de = (ctypes.c_uint64 * L)()
        _call("bfv_ctx_query", h, ctypes.cast(pr, _vp), ctypes.byref(om), ctypes.cast(de, _vp))
        self.primes, self.omega, self.delta_mod_q = list(pr), om.value, list(de)
        self.device = torch.cuda.current_device()
        # schedules the autotuner chose on this GPU model for this ring (SCHEDULE_FILE), used by
        # every packed product called with pair_chunk = 0
        if os.path.exists(SCHEDULE_FILE):
            self.load_schedules(SCHEDULE_FILE)

    @classmethod
    def from_shape(cls, shape):
        return cls(shape.N, shape.L, shape.prime_bits, shape.t, shape.sigma_num, shape.sigma_den)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bfv_ctx_free(self.handle)
            self.handle = None

    # -- helpers
    def _empty_u64(self, *shape):
        import torch
        return torch.empty(shape, dtype=torch.int64, device=f"cuda:{self.device}")

    def launch_count(self) -> int:
        n = _u64()
        _call("bfv_launch_count", self.handle, ctypes.byref(n))
        return n.value

    # -- keys
    def keygen(self, seed: int, stream=None) -> Keys:
        h = _vp()
        _call("bfv_keygen", self.handle, seed, _stream(stream), ctypes.byref(h))
        return Keys(self, h)

    def keys_export(self, keys: Keys, stream=None):
        """(sk int8[N], pk [2][L][N], gk [log2 N][L][2][L+1][N]) in coefficient form, device tensors."""
        import torch
        ng = int(round(np.log2(self.N)))
        sk = torch.empty(self.N, dtype=torch.int8, device=f"cuda:{self.device}")
        pk = self._empty_u64(2, self.L, self.N)
        gk = self._empty_u64(ng, self.L, 2, self.L + 1, self.N)
        _call("bfv_keys_export", self.handle, keys.handle, _ptr(sk), _ptr(pk), _ptr(gk), _stream(stream))
        return sk, pk, gk

    # -- client
    def encode(self, slots, stream=None):
        slots = _dev_in(slots, "slots", 8, block=self.N)
        count = slots.numel() // self.N
        pt = self._empty_u64(*slots.shape)
        _call("bfv_encode", self.handle, _ptr(slots), count, _ptr(pt), _stream(stream))
        return pt

    def decode(self, pt, stream=None):
        import torch
        pt = _dev_in(pt, "pt", 8, block=self.N)
        count = pt.numel() // self.N
        out = torch.empty(pt.shape, dtype=torch.int64, device=pt.device)
        _call("bfv_decode", self.handle, _ptr(pt), count, _ptr(out), _stream(stream))
        return out

    def encode_features(self, X, stream=None):
        nX, f = X.shape
        X = _dev_in(X, "X", 1)
        K = -(-f // self.N)
        pt = self._empty_u64(nX, K, self.N)
        _call("bfv_encode_features", self.handle, _ptr(X), nX, f, _ptr(pt), _stream(stream))
        return pt

    def encode_feature_columns(self, X, stream=None):
        nX, f = X.shape
        X = _dev_in(X, "X", 1)
        pt = self._empty_u64(f, self.N)
        _call("bfv_encode_feature_columns", self.handle, _ptr(X), nX, f, _ptr(pt), _stream(stream))
        return pt

    def encrypt_workspace(self, count: int) -> int:
        n = _sz()
        _call("bfv_encrypt_workspace", self.handle, count, ctypes.byref(n))
        return n.value

    def encrypt(self, keys: Keys, pt, seed: int, obj0: int = 0, out=None, ws=None, stream=None):
        pt = _dev_in(pt, "pt", 8, block=self.N)
        count = pt.numel() // self.N
        ct = (_dev_out(out, "out", 8, count * 2 * self.L * self.N) if out is not None
              else self._empty_u64(*pt.shape[:-1], 2, self.L, self.N))
        ws, nb = _workspace(ws, self.encrypt_workspace(count), pt.device)
        _call("bfv_encrypt", self.handle, keys.handle, _ptr(pt), count, seed, obj0, _ptr(ct), _ptr(ws), nb,
              _stream(stream))
        return ct

    def decrypt_workspace(self, count: int) -> int:
        n = _sz()
        _call("bfv_decrypt_workspace", self.handle, count, ctypes.byref(n))
        return n.value

    def decrypt(self, keys: Keys, ct, out=None, ws=None, stream=None):
        ct = _dev_in(ct, "ct", 8, block=2 * self.L * self.N)
        count = ct.numel() // (2 * self.L * self.N)
        pt = (_dev_out(out, "out", 8, count * self.N) if out is not None
              else self._empty_u64(*ct.shape[:-3], self.N))
        ws, nb = _workspace(ws, self.decrypt_workspace(count), ct.device)
        _call("bfv_decrypt", self.handle, keys.handle, _ptr(ct), count, _ptr(pt), _ptr(ws), nb, _stream(stream))
        return pt

    def noise_budget(self, keys: Keys, ct, ws=None, stream=None) -> list[int]:
        """Invariant noise budget in bits of each ciphertext of ct [..][2][L][N] (bfv_noise_budget;
        synchronises)."""
        ct = _dev_in(ct, "ct", 8, block=2 * self.L * self.N)
        count = ct.numel() // (2 * self.L * self.N)
        if count == 0:
            return []
        n = _sz()
        _call("bfv_noise_budget_workspace", self.handle, count, ctypes.byref(n))
        ws, nb = _workspace(ws, n.value, ct.device)
        out = (ctypes.c_int * count)()
        _call("bfv_noise_budget", self.handle, keys.handle, _ptr(ct), count, ctypes.cast(out, _vp), _ptr(ws), nb,
              _stream(stream))
        return list(out)

    # -- server
    def model_prepare(self, W, b, stream=None) -> Model:
        W = np.ascontiguousarray(W, dtype=np.int64)
        b = np.ascontiguousarray(b, dtype=np.int64)
        f, nY = W.shape
        h = _vp()
        _call("bfv_model_prepare", self.handle, W.ctypes.data_as(_vp), b.ctypes.data_as(_vp), f, nY,
              _stream(stream), ctypes.byref(h))
        return Model(self, h, f, nY)

    def packed_workspace(self, model: Model, nX: int, pair_chunk: int = 0) -> int:
        n = _sz()
        _call("bfv_lr_scores_packed_workspace", self.handle, model.handle, nX, pair_chunk, ctypes.byref(n))
        return n.value

    def _packed_args(self, model: Model, X_ct, out, name="X_ct"):
        """Input ciphertexts uint64[nX][K][2][L][N] and the output buffer uint64[nout][2][L][N]."""
        nX = X_ct.shape[0]
        ctw = 2 * self.L * self.N
        X_ct = _dev_in(X_ct, name, 8, numel=nX * model.K * ctw)
        nout = -(-nX * model.nY // self.N)
        Y = _dev_out(out, "out", 8, nout * ctw) if out is not None else self._empty_u64(nout, 2, self.L, self.N)
        return nX, X_ct, Y

    def lr_scores_packed(self, keys: Keys, model: Model, X_ct, out=None, ws=None, pair_chunk: int = 0, stream=None):
        nX, X_ct, Y = self._packed_args(model, X_ct, out)
        if nX == 0:
            return Y
        ws, nb = _workspace(ws, self.packed_workspace(model, nX, pair_chunk), X_ct.device)
        _call("bfv_lr_scores_packed", self.handle, keys.handle, model.handle, _ptr(X_ct), nX, _ptr(Y), _ptr(ws), nb,
              pair_chunk, _stream(stream))
        return Y

    def standard_workspace(self, model: Model) -> int:
        n = _sz()
        _call("bfv_lr_scores_standard_workspace", self.handle, model.handle, ctypes.byref(n))
        return n.value

    def multi_workspace(self, model: Model, nXs, pair_chunk: int = 0) -> int:
        arr = (ctypes.c_size_t * len(nXs))(*nXs)
        n = _sz()
        _call("bfv_lr_scores_packed_multi_workspace", self.handle, model.handle, len(nXs), ctypes.cast(arr, _vp),
              pair_chunk, ctypes.byref(n))
        return n.value

    def lr_scores_packed_multi(self, keys: Keys, model: Model, X_cts, outs=None, ws=None, pair_chunk: int = 0,
                               stream=None):
        """Several requests (a list of input-ciphertext tensors) in one fused packed product; returns
        one output tensor per request, each identical to its single-request result."""
        xs, outs = self._models_args([model] * len(X_cts), X_cts, outs)
        nXs = [x.shape[0] for x in xs]
        ws, nb = _workspace(ws, self.multi_workspace(model, nXs, pair_chunk), f"cuda:{self.device}")
        xp = (ctypes.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
        yp = (ctypes.c_void_p * len(outs))(*[y.data_ptr() for y in outs])
        na = (ctypes.c_size_t * len(nXs))(*nXs)
        _call("bfv_lr_scores_packed_multi", self.handle, keys.handle, model.handle, len(xs), ctypes.cast(xp, _vp),
              ctypes.cast(na, _vp), ctypes.cast(yp, _vp), _ptr(ws), nb, pair_chunk, _stream(stream))
        return outs

    def _models_args(self, models, X_cts, outs):
        """Per request: its input ciphertexts and its output buffer, checked like lr_scores_packed's."""
        if len(models) != len(X_cts) or (outs is not None and len(outs) != len(X_cts)):
            raise ValueError("one model and one output per request expected")
        if not X_cts:
            raise ValueError("at least one request expected")
        xs, ys = [], []
        for r, (m, x) in enumerate(zip(models, X_cts)):
            _, x, y = self._packed_args(m, x, outs[r] if outs is not None else None, name=f"X_cts[{r}]")
            xs.append(x)
            ys.append(y)
        return xs, ys

    def models_workspace(self, models, nXs, pair_chunk: int = 0) -> int:
        mp = (ctypes.c_void_p * len(models))(*[m.handle for m in models])
        na = (ctypes.c_size_t * len(nXs))(*nXs)
        n = _sz()
        _call("bfv_lr_scores_packed_models_workspace", self.handle, len(models), ctypes.cast(mp, _vp),
              ctypes.cast(na, _vp), pair_chunk, ctypes.byref(n))
        return n.value

    def lr_scores_packed_models(self, keys: Keys, models, X_cts, outs=None, ws=None, pair_chunk: int = 0,
                                stream=None):
        """Requests of different models (request r: inputs X_cts[r], model models[r]) in one fused
        packed product; returns one output tensor per request, each identical to its
        single-request result."""
        xs, outs = self._models_args(models, X_cts, outs)
        nXs = [x.shape[0] for x in xs]
        ws, nb = _workspace(ws, self.models_workspace(models, nXs, pair_chunk), f"cuda:{self.device}")
        mp = (ctypes.c_void_p * len(models))(*[m.handle for m in models])
        xp = (ctypes.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
        yp = (ctypes.c_void_p * len(outs))(*[y.data_ptr() for y in outs])
        na = (ctypes.c_size_t * len(nXs))(*nXs)
        _call("bfv_lr_scores_packed_models", self.handle, keys.handle, len(xs), ctypes.cast(mp, _vp),
              ctypes.cast(xp, _vp), ctypes.cast(na, _vp), ctypes.cast(yp, _vp), _ptr(ws), nb, pair_chunk,
              _stream(stream))
        return outs

    def lr_scores_packed_graph(self, keys: Keys, model: Model, X_ct, out=None, ws=None, pair_chunk: int = 0,
                               stream=None):
        """lr_scores_packed replayed from a cached CUDA graph (one host call per product)."""
        nX, X_ct, Y = self._packed_args(model, X_ct, out)
        if nX == 0:
            return Y
        ws, nb = _workspace(ws, self.packed_workspace(model, nX, pair_chunk), X_ct.device)
        _call("bfv_lr_scores_packed_graph", self.handle, keys.handle, model.handle, _ptr(X_ct), nX, _ptr(Y),
              _ptr(ws), nb, pair_chunk, _stream(stream))
        return Y

    def autotune_packed(self, keys: Keys, model: Model, X_ct, ws, out=None, stream=None):
        """Times pair-chunk sizes that fit in `ws` and makes the fastest the default for this
        number of pairs. Returns (chunk, ms)."""
        nX, X_ct, Y = self._packed_args(model, X_ct, out)
        ws = _dev_in(ws, "ws", ws.element_size())
        ch, ms = _sz(), ctypes.c_double()
        _call("bfv_autotune_packed", self.handle, keys.handle, model.handle, _ptr(X_ct), nX, _ptr(Y), _ptr(ws),
              ws.numel() * ws.element_size(), _stream(stream), ctypes.byref(ch), ctypes.byref(ms))
        return ch.value, ms.value

    # -- launch options (bfv_set_option)
    def set_option(self, option: int, value: int):
        _call("bfv_set_option", self.handle, option, value)

    def get_option(self, option: int) -> int:
        v = ctypes.c_int()
        _call("bfv_get_option", self.handle, option, ctypes.byref(v))
        return v.value

    # -- schedules of the packed product (bfv_packed_schedule)
    def packed_schedule(self, npairs: int) -> Schedule:
        """The schedule a product of npairs pairs uses with pair_chunk = 0."""
        s = Schedule()
        _call("bfv_packed_schedule_get", self.handle, npairs, ctypes.byref(s))
        return s

    def set_packed_schedule(self, npairs: int, sched: Schedule):
        """Records sched for products of npairs pairs (0: every pair count without its own entry)."""
        _call("bfv_packed_schedule_set", self.handle, npairs, ctypes.byref(sched))

    def lr_scores_packed_sched(self, keys: Keys, model: Model, X_ct, sched: Schedule, out=None, ws=None,
                               stream=None):
        """lr_scores_packed with an explicit schedule."""
        nX, X_ct, Y = self._packed_args(model, X_ct, out)
        if nX == 0:
            return Y
        ws, nb = _workspace(ws, self.packed_workspace(model, nX, sched.pair_chunk), X_ct.device)
        _call("bfv_lr_scores_packed_sched", self.handle, keys.handle, model.handle, _ptr(X_ct), nX, _ptr(Y),
              _ptr(ws), nb, ctypes.byref(sched), _stream(stream))
        return Y

    def autotune_packed_schedule(self, keys: Keys, model: Model, X_ct, ws, out=None, stream=None):
        """Tunes the pair chunk, then each kernel split (coordinate descent), records the fastest
        schedule for this number of pairs and returns (Schedule, ms)."""
        nX, X_ct, Y = self._packed_args(model, X_ct, out)
        ws = _dev_in(ws, "ws", ws.element_size())
        best, ms = Schedule(), ctypes.c_double()
        _call("bfv_autotune_packed_schedule", self.handle, keys.handle, model.handle, _ptr(X_ct), nX, _ptr(Y),
              _ptr(ws), ws.numel() * ws.element_size(), _stream(stream), ctypes.byref(best), ctypes.byref(ms))
        return best, ms.value

    def schedule_key(self, npairs: int) -> str:
        """Key of a tuned schedule in a schedule file: ring degree, ciphertext primes, pairs."""
        return f"N={self.N},L={self.L},pairs={npairs}"

    def save_schedules(self, path: str, npairs_list):
        """Writes the schedules of the given pair counts to a JSON file (merged with what it holds)."""
        data = load_schedule_file(path)
        for n in npairs_list:
            data[self.schedule_key(n)] = self.packed_schedule(n).as_dict()
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)

    def load_schedules(self, path: str) -> int:
        """Records every schedule of a JSON file that belongs to this ring (N, L); returns how many."""
        n = 0
        for key, d in load_schedule_file(path).items():
            parts = dict(kv.split("=") for kv in key.split(","))
            if int(parts["N"]) == self.N and int(parts["L"]) == self.L:
                self.set_packed_schedule(int(parts["pairs"]), Schedule.from_dict(d))
                n += 1
        return n

    def lr_scores_standard(self, model: Model, X_ct, nX: int, out=None, ws=None, stream=None):
        ctw = 2 * self.L * self.N
        X_ct = _dev_in(X_ct, "X_ct", 8, numel=model.f * ctw)
        Y = _dev_out(out, "out", 8, model.nY * ctw) if out is not None else self._empty_u64(model.nY, 2, self.L, self.N)
        ws, nb = _workspace(ws, self.standard_workspace(model), X_ct.device)
        _call("bfv_lr_scores_standard", self.handle, model.handle, _ptr(X_ct), nX, _ptr(Y), _ptr(ws), nb,
              _stream(stream))
        return Y

    def check_error(self) -> int:
        """Device error word (bit 0: a bounded wait ran out); clears it. Raises BfvError on timeout."""
        f = ctypes.c_int()
        rc = lib().bfv_check_error(self.handle, ctypes.byref(f))
        if rc not in (BFV_OK, BFV_ERR_TIMEOUT):
            raise BfvError("bfv_check_error", rc)
        return f.value

    def predict_workspace(self, model: Model, nX: int, pair_chunk: int = 0) -> int:
        n = _sz()
        _call("bfv_lr_predict_packed_workspace", self.handle, model.handle, nX, pair_chunk, ctypes.byref(n))
        return n.value

    def predict_packed(self, keys: Keys, model: Model, X, seed: int, out=None, ws=None, pair_chunk: int = 0,
                       stream=None):
        """Whole protocol on device buffers: X uint8[nX][f] -> scores int64[nX][nY] (mod t)."""
        import torch
        nX = X.shape[0]
        X = _dev_in(X, "X", 1, numel=nX * model.f)
        scores = (_dev_out(out, "out", 8, nX * model.nY) if out is not None
                  else torch.empty((nX, model.nY), dtype=torch.int64, device=X.device))
        if nX == 0:
            return scores
        ws, nb = _workspace(ws, self.predict_workspace(model, nX, pair_chunk), X.device)
        _call("bfv_lr_predict_packed", self.handle, keys.handle, model.handle, _ptr(X), nX, seed, _ptr(scores),
              _ptr(ws), nb, pair_chunk, _stream(stream))
        return scores

    def predict_packed_host(self, keys: Keys, model: Model, X_host, seed: int, out=None, ws=None,
                            pair_chunk: int = 0, stream=None):
        """Whole protocol with HOST buffers (the copies happen inside the C call): X_host uint8
        [nX][f] (numpy or pinned torch) -> scores int64[nX][nY] on the host."""
        nX = X_host.shape[0]
        X_host = _host_buf(X_host, "X_host", 1, (nX, model.f))
        if out is None:
            out = np.empty((nX, model.nY), dtype=np.int64)
        out = _host_buf(out, "out", 8, (nX, model.nY), out=True)
        if nX == 0:
            return out
        ws, nb = _workspace(ws, self.predict_workspace(model, nX, pair_chunk), f"cuda:{self.device}")
        _call("bfv_lr_predict_packed_host", self.handle, keys.handle, model.handle, ctypes.c_void_p(_addr(X_host)), nX,
              seed, ctypes.c_void_p(_addr(out)), _ptr(ws), nb, pair_chunk, _stream(stream))
        return out

    def profile(self, enable: bool):
        _call("bfv_profile", self.handle, 1 if enable else 0)

    def profile_read(self) -> dict:
        """{kernel kind: (launches, total ms)} since the last read."""
        out = {}
        for k, name in enumerate(KERNEL_KINDS):
            n, ms = _u64(), ctypes.c_double()
            _call("bfv_profile_read", self.handle, k, ctypes.byref(n), ctypes.byref(ms))
            out[name] = (n.value, ms.value)
        return out

    def packed_pair_from_workspace(self, model: Model, nX: int, pair_chunk: int, ws, g: int, stream=None):
        if not 0 <= g < nX * model.nY:
            raise ValueError(f"pair {g} outside 0..{nX * model.nY - 1}")
        ws = _dev_in(ws, "ws", ws.element_size())
        if ws.numel() * ws.element_size() < self.packed_workspace(model, nX, pair_chunk):
            raise ValueError("ws is smaller than this product's workspace")
        out = self._empty_u64(2, self.L, self.N)
        _call("bfv_lr_packed_pair_from_workspace", self.handle, model.handle, nX, pair_chunk, _ptr(ws), g, _ptr(out),
              _stream(stream))
        return out


def _on_call_stream(fn):
    """Runs a binding call with its `stream` argument as the current CUDA stream. What the call
    allocates (outputs, workspaces, contiguous copies of inputs) then comes from, and returns to,
    the pool of the stream its kernels run on, so the caching allocator cannot hand that memory
    to other work while those kernels may still use it."""
    sig = inspect.signature(fn)

    @functools.wraps(fn)
    def call(*args, **kwargs):
        stream = sig.bind(*args, **kwargs).arguments.get("stream")
        if stream is None:
            return fn(*args, **kwargs)
        import torch
        with torch.cuda.stream(stream):
            return fn(*args, **kwargs)
    return call


for _name, _fn in list(vars(Context).items()):
    if inspect.isfunction(_fn) and "stream" in inspect.signature(_fn).parameters:
        setattr(Context, _name, _on_call_stream(_fn))


def as_u64(t) -> np.ndarray:
    """Device/host int64 tensor holding raw 64-bit words -> numpy uint64 array."""
    return t.detach().cpu().numpy().view(np.uint64)


@_on_call_stream
def crt_combine(r0, t0: int, r1, t1: int, out=None, stream=None):
    """CRT plaintext pair (bfv_crt_combine): device int64 residue tensors r0 (mod t0) and r1
    (mod t1) of equal shape -> the integers x = r0 mod t0, x = r1 mod t1, centred in
    (-t0 t1 / 2, t0 t1 / 2]."""
    import torch
    if r0.shape != r1.shape or r0.dtype != torch.int64 or r1.dtype != torch.int64:
        raise ValueError("r0 and r1 must be int64 tensors of the same shape")
    r0, r1 = _dev_in(r0, "r0", 8), _dev_in(r1, "r1", 8)
    out = torch.empty_like(r0) if out is None else _dev_out(out, "out", 8, r0.numel())
    _call("bfv_crt_combine", _ptr(r0), t0, _ptr(r1), t1, r0.numel(), _ptr(out), _stream(stream))
    return out


def pack_rows(X, N: int):
    """Integer feature rows X [nX][f] (device tensor) -> slot vectors [nX * ceil(f/N)][N]: row i's
    features k N .. k N + N - 1 in plaintext i ceil(f/N) + k, zero-padded (the packing of
    Section 4.2.2; encode() then maps them to plaintexts)."""
    import torch
    nX, f = X.shape
    K = -(-f // N)
    out = torch.zeros((nX, K * N), dtype=torch.int64, device=X.device)
    out[:, :f] = X
    return out.reshape(nX * K, N)


def unpack_packed_scores(N: int, slots, nX: int, nY: int):
    """Decoded packed output slots [nout][N] -> scores [nX][nY] (pair g = i nY + j at slot g mod N
    of output g // N)."""
    flat = np.asarray(slots).reshape(-1)
    return flat[: nX * nY].reshape(nX, nY)
