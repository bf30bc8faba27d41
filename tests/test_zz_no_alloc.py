"""The allocation-free decryption entry point (bfv_decrypt_noalloc) against bfv_decrypt.

bfv_decrypt_noalloc exists for callers that must not call cudaMalloc (it can synchronise the
device and fail under a fixed memory reservation): it keeps its scratch in a fixed device
array inside the library. Its output must equal bfv_decrypt's exactly (decryption is exact
integer arithmetic, so the tolerance is zero), on consecutive calls that share the array.
This file is collected last so that a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(bfv, ctx, keys, ct):
    count = ct.numel() // (2 * ctx.L * ctx.N)
    pt = torch.empty((count, ctx.N), dtype=torch.int64, device=ct.device)
    bfv._call("bfv_decrypt_noalloc", ctx.handle, keys.handle, bfv._ptr(ct.contiguous()), count, bfv._ptr(pt),
              bfv._stream())
    return pt


@pytest.mark.parametrize("shape", [synth.TINY, synth.PAPER16K])
def test_decrypt_noalloc_matches_decrypt_on_two_calls(shape):
    import paper_2204_05496_gb300 as bfv
    ctx = bfv.Context.from_shape(shape)
    keys = ctx.keygen(7)
    n = ctypes.c_size_t()
    bfv._call("bfv_decrypt_noalloc_max_count", ctx.handle, ctypes.byref(n))
    cap = n.value
    assert cap == (4 << 20) // (ctx.L * ctx.N * 8) and cap >= 1
    rng = np.random.default_rng(11)
    results = []
    for call, count in enumerate((cap, max(1, cap - 1))):
        v = rng.integers(0, ctx.t, size=(count, ctx.N), dtype=np.int64)
        ct = ctx.encrypt(keys, ctx.encode(torch.from_numpy(v).cuda()), seed=100 + call)
        want = ctx.decrypt(keys, ct)
        got = _noalloc(bfv, ctx, keys, ct)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
        assert np.array_equal(ctx.decode(got).cpu().numpy(), v)
        results.append(got)
    # one ciphertext more than the array holds is rejected before anything is launched
    v = np.zeros((cap + 1, ctx.N), dtype=np.int64)
    ct = ctx.encrypt(keys, ctx.encode(torch.from_numpy(v).cuda()), seed=1)
    with pytest.raises(bfv.BfvError) as e:
        _noalloc(bfv, ctx, keys, ct)
    assert e.value.code == bfv.BFV_ERR_OVER_BUDGET
