"""The uneven batch: 64 independent models (f in {1k, 5k, 20k, 40k}, |Y| in {2, 8, 16}, batch
sizes drawn from 1..512 -- divided by 32 here to bound the run time), each on the N = 16384
or the N = 32768 parameter set. The models of each ring run as ONE fused packed product
(bfv_lr_scores_packed_models), and the two products are captured into one CUDA graph that is
replayed as one launch. Each request's outputs must be bit-identical (tolerance zero) to its
single-request product, every decrypted score must equal the closed form (x.W + b) mod t, and
the smallest request of each ring must match the oracle's whole pipeline bit for bit."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2204_05496_gb300 as bfv

SEED_KEYS = 402
RINGS = ("PAPER16K", "WIDE32K")


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


@pytest.fixture(scope="module")
def batch():
    items = synth.uneven_batch(x_divisor=32)
    ctxs = {r: bfv.Context.from_shape(getattr(synth, r)) for r in RINGS}
    keys = {r: ctxs[r].keygen(SEED_KEYS) for r in RINGS}
    for it in items:
        ctx = ctxs[it["params"]]
        it["model"] = ctx.model_prepare(it["W"], it["b"])
        pt = ctx.encode_features(dev(it["X"]).to(torch.uint8))
        it["X_ct"] = ctx.encrypt(keys[it["params"]], pt.reshape(-1, ctx.N), seed=it["enc_seed"]).reshape(
            it["nX"], -1, 2, ctx.L, ctx.N)
    return items, ctxs, keys


def test_uneven_batch_in_one_graph(batch):
    items, ctxs, keys = batch
    groups = {r: [it for it in items if it["params"] == r] for r in RINGS}
    assert all(1 <= len(g) <= 64 for g in groups.values())
    alone = [ctxs[it["params"]].lr_scores_packed(keys[it["params"]], it["model"], it["X_ct"]) for it in items]
    # both rings' fused products in one CUDA graph
    plan = {}
    for r, grp in groups.items():
        ctx = ctxs[r]
        models = [it["model"] for it in grp]
        nXs = [it["nX"] for it in grp]
        ws = torch.empty(ctx.models_workspace(models, nXs), dtype=torch.uint8, device="cuda")
        outs = [ctx._empty_u64(-(-it["nX"] * it["nY"] // ctx.N), 2, ctx.L, ctx.N) for it in grp]
        plan[r] = (models, [it["X_ct"] for it in grp], outs, ws)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        st = torch.cuda.current_stream()
        for r in RINGS:
            models, xs, outs, ws = plan[r]
            ctxs[r].lr_scores_packed_models(keys[r], models, xs, outs=outs, ws=ws, stream=st)
    for rep in range(2):                                   # replays reuse the workspace
        for r in RINGS:
            for o in plan[r][2]:
                o.zero_()
        g.replay()
        torch.cuda.synchronize()
        k = {r: 0 for r in RINGS}
        for it, a in zip(items, alone):
            r = it["params"]
            assert torch.equal(plan[r][2][k[r]], a)
            k[r] += 1
    for it, a in zip(items, alone):
        ctx = ctxs[it["params"]]
        slots = ctx.decode(ctx.decrypt(keys[it["params"]], a)).cpu().numpy()
        got = bfv.unpack_packed_scores(ctx.N, slots, it["nX"], it["nY"])
        assert np.array_equal(got, oracle.expected_scores(it["X"], it["W"], it["b"], ctx.t))


@pytest.mark.parametrize("ring", RINGS)
def test_uneven_batch_smallest_request_matches_oracle(batch, ring):
    items, ctxs, keys = batch
    it = min((x for x in items if x["params"] == ring), key=lambda x: x["nX"] * x["nY"])
    P = oracle.Params.from_shape(getattr(synth, ring))
    okeys = oracle.keygen(P, SEED_KEYS)
    oX_ct, _, oY = oracle.packed_pipeline(P, okeys, it["X"], it["W"], it["b"], it["enc_seed"])
    assert np.array_equal(bfv.as_u64(it["X_ct"]), oX_ct)
    ctx = ctxs[ring]
    Y = ctx.lr_scores_packed_models(keys[ring], [it["model"]], [it["X_ct"]])[0]
    assert np.array_equal(bfv.as_u64(Y), oY)
