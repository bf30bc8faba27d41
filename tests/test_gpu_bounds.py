"""The bounds-checked build (-DBFV_BOUNDS): every global-memory access of every kernel is checked
against the buffers its call may touch (the context's tables, keys, models, the caller's buffers
at the sizes the call implies); an access outside them is skipped and reported in bit 1 of the
context's error word instead of faulting. The tiny packed and standard pipelines must run under it
without a report and with the oracle's bits. With the caller's buffers registered 8 bytes short
(host-side injection: every access still lies inside the real buffers) the kernels must report
the accesses to the last 8 bytes, and the context must keep working afterwards."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np
import torch
import oracle
import synth
import paper_2204_05496_gb300 as bfv

assert bfv.VARIANT == "bounds" and bfv.lib().bfv_bounds_checked() == 1
w = synth.WORKLOADS["tiny-16"]
X, W, b = synth.workload_inputs(w)
ctx = bfv.Context.from_shape(w.params)
keys = ctx.keygen(w.seed_keys)
P = oracle.Params.from_shape(w.params)
okeys = oracle.keygen(P, w.seed_keys)
assert ctx.check_error() == 0, "key generation"

# packed product, whole protocol
oX, _, oY = oracle.packed_pipeline(P, okeys, X, W, b, w.seed_enc)
pt = ctx.encode_features(torch.from_numpy(X).cuda())
X_ct = ctx.encrypt(keys, pt.reshape(-1, P.N), seed=w.seed_enc).reshape(16, 1, 2, P.L, P.N)
assert np.array_equal(bfv.as_u64(X_ct), oX)
model = ctx.model_prepare(W, b)
Y = ctx.lr_scores_packed(keys, model, X_ct)
assert np.array_equal(bfv.as_u64(Y), oY)
slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
assert np.array_equal(bfv.unpack_packed_scores(P.N, slots, 16, 8), oracle.expected_scores(X, W, b, P.t))
assert ctx.check_error() == 0, "packed pipeline"

# standard product, tensor-core and dp4a kernels
cols = np.zeros((X.shape[1], P.N), dtype=np.int64)
cols[:, :16] = X.T
oXs = oracle.encrypt(P, okeys, oracle.encode(P, cols), seed=5, obj0=0)
X_std = ctx.encrypt(keys, ctx.encode(torch.from_numpy(cols).cuda()), seed=5)
assert np.array_equal(bfv.as_u64(X_std), oXs)
want = oracle.lr_standard(P, oXs, W, b)
for kind in (0, 1):
    ctx.set_option(bfv.BFV_OPT_STANDARD_KERNEL, kind)
    assert np.array_equal(bfv.as_u64(ctx.lr_scores_standard(model, X_std, 16)), want), kind
ctx.set_option(bfv.BFV_OPT_STANDARD_KERNEL, 0)
assert ctx.check_error() == 0, "standard product"

# the caller's buffers registered 8 bytes short: the accesses to their last word are reported
bfv._call("bfv_debug_inject", ctx.handle, bfv.BFV_INJECT_BOUNDS_SHRINK, 8)
try:
    ctx.decode(ctx.decrypt(keys, Y))
    flags = ctx.check_error()
    assert flags & 2, flags
finally:
    bfv._call("bfv_debug_inject", ctx.handle, bfv.BFV_INJECT_BOUNDS_SHRINK, 0)
slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
assert np.array_equal(bfv.unpack_packed_scores(P.N, slots, 16, 8), oracle.expected_scores(X, W, b, P.t))
assert ctx.check_error() == 0, "after the injection"
print("BOUNDS OK")
'''


def test_bounds_checked_build_runs_the_tiny_pipelines_clean():
    import paper_2204_05496_gb300 as bfv
    bfv.build(variant="bounds")
    env = dict(os.environ, BFV_LIB_VARIANT="bounds")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "BOUNDS OK" in r.stdout


def test_release_build_rejects_the_bounds_injection():
    import torch
    import synth
    import paper_2204_05496_gb300 as bfv
    assert bfv.lib().bfv_bounds_checked() == 0
    ctx = bfv.Context.from_shape(synth.TINY)
    assert bfv.lib().bfv_debug_inject(ctx.handle, bfv.BFV_INJECT_BOUNDS_SHRINK, 8) == bfv.BFV_ERR_INVALID_ARG
    torch.cuda.synchronize()
