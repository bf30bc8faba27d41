"""Continuous batching: several requests fused into one packed product, and the serving loop.
Each request's output ciphertexts must be bit-identical (tolerance zero) whether it runs
alone or in a mix with others, and decrypt to its closed-form scores."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import paper_2204_05496_gb300 as bfv
    w = synth.WORKLOADS["tiny-1"]
    ctx = bfv.Context.from_shape(w.params)
    keys = ctx.keygen(w.seed_keys)
    rng = np.random.default_rng(41)
    X = (rng.random((40, 1000)) < 0.05).astype(np.uint8)
    W = rng.integers(-127, 128, (1000, 8))
    b = rng.integers(-127, 128, 8)
    model = ctx.model_prepare(W, b)
    pt = ctx.encode_features(torch.from_numpy(X).cuda())
    X_ct = ctx.encrypt(keys, pt.reshape(-1, ctx.N), seed=5).reshape(40, 1, 2, ctx.L, ctx.N)
    return bfv, ctx, keys, model, X, W, b, X_ct


def _alone(ctx, keys, model, X_ct):
    return ctx.lr_scores_packed(keys, model, X_ct)


@pytest.mark.parametrize("chunk", [0, 20])
def test_fused_requests_match_single_requests(env, chunk):
    bfv, ctx, keys, model, X, W, b, X_ct = env
    sizes = [1, 3, 1, 7, 2]
    starts = np.cumsum([0] + sizes)
    reqs = [X_ct[starts[k]:starts[k + 1]] for k in range(len(sizes))]
    outs = ctx.lr_scores_packed_multi(keys, model, reqs, pair_chunk=chunk)
    for k, (r, o) in enumerate(zip(reqs, outs)):
        assert torch.equal(o, _alone(ctx, keys, model, r))
        slots = ctx.decode(ctx.decrypt(keys, o)).cpu().numpy()
        got = bfv.unpack_packed_scores(ctx.N, slots, sizes[k], 8)
        assert np.array_equal(got, oracle.expected_scores(X[starts[k]:starts[k + 1]], W, b, ctx.t))


def test_server_fuses_and_overlaps_and_keeps_results(env):
    from paper_2204_05496_gb300 import serve
    bfv, ctx, keys, model, X, W, b, X_ct = env
    sizes = [1, 1, 4, 1, 2, 1, 8, 1, 1, 3, 1, 1]
    starts = np.cumsum([0] + sizes)
    # a burst at t = 0 and more requests arriving while it is on the GPU
    arrivals = [(0.0 if k < 6 else 0.002 * (k - 5), n) for k, n in enumerate(sizes)]
    srv = serve.Server(ctx, keys, model, hbm_budget_bytes=8 << 30, n_streams=2)
    done = srv.run(arrivals, lambda k, n: X_ct[starts[k]:starts[k] + n])
    assert len(done) == len(sizes) and all(r.t_done is not None and r.t_done >= r.t_arrival for r in done)
    assert srv.nbatches < len(sizes)                  # requests were fused
    for r in done:
        assert torch.equal(r.out, _alone(ctx, keys, model, r.X_ct))
    rep = serve.latency_report(done, 8)
    assert rep["predictions"] == sum(sizes) and rep["p99_ms"] >= rep["p50_ms"] > 0


def test_server_hbm_budget_limits_admission(env):
    from paper_2204_05496_gb300 import serve
    bfv, ctx, keys, model, X, W, b, X_ct = env
    one = ctx.multi_workspace(model, [2])
    srv = serve.Server(ctx, keys, model, hbm_budget_bytes=one, n_streams=2)   # room for one 2-individual launch
    done = srv.run([(0.0, 2)] * 4, lambda k, n: X_ct[2 * k:2 * k + n])
    assert srv.nbatches == 4                          # nothing fused, nothing concurrent
    for r in done:
        assert torch.equal(r.out, _alone(ctx, keys, model, r.X_ct))


def test_server_overlaps_a_second_batch_with_the_first(env):
    from paper_2204_05496_gb300 import serve
    bfv, ctx, keys, model, X, W, b, X_ct = env
    srv = serve.Server(ctx, keys, model, hbm_budget_bytes=8 << 30, n_streams=2)
    srv.start()
    first = [srv.submit(k, X_ct[4 * k:4 * k + 4]) for k in range(3)]
    srv.step()                                        # batch 0 (3 requests) goes to stream 0
    late = [srv.submit(3 + k, X_ct[12 + k:13 + k]) for k in range(2)]
    srv.step()                                        # arrived while batch 0 runs -> stream 1
    assert srv.nbatches == 2 and srv.max_concurrent == 2
    while not srv.idle():
        srv.step()
    torch.cuda.synchronize()
    srv.step()
    for r in first + late:
        assert r.t_done is not None
        assert torch.equal(r.out, _alone(ctx, keys, model, r.X_ct))
    # the two launches' device intervals (events recorded on each stream before and after its
    # product) intersect: the second batch began on the device before the first had finished
    iv = sorted(srv.intervals, key=lambda d: d["batch"])
    assert len(iv) == 2 and iv[0]["stream"] != iv[1]["stream"]
    assert iv[1]["start_s"] < iv[0]["end_s"] and iv[0]["start_s"] < iv[1]["end_s"]


def test_server_waits_for_inputs_encrypted_on_another_stream(env):
    """make_inputs encrypts on the default stream and returns without synchronising: each
    launch must wait for that work (an event recorded at submission), so every result is still
    the single-request product of the finished ciphertexts."""
    from paper_2204_05496_gb300 import serve
    bfv, ctx, keys, model, X, W, b, X_ct = env
    sizes = [3, 1, 5, 1, 2, 6]
    starts = np.cumsum([0] + sizes)
    Xd = torch.from_numpy(X).cuda()

    def make_inputs(k, n):
        pt = ctx.encode_features(Xd[starts[k]:starts[k] + n])
        return ctx.encrypt(keys, pt.reshape(-1, ctx.N), seed=5, obj0=int(starts[k])).reshape(n, 1, 2, ctx.L, ctx.N)

    srv = serve.Server(ctx, keys, model, hbm_budget_bytes=8 << 30, n_streams=2)
    done = srv.run([(0.0, n) for n in sizes], make_inputs)
    for r in done:
        n = sizes[r.rid]
        assert torch.equal(r.X_ct, X_ct[starts[r.rid]:starts[r.rid] + n])   # the same encryptions
        assert torch.equal(r.out, _alone(ctx, keys, model, X_ct[starts[r.rid]:starts[r.rid] + n]))


def test_server_priority_classes_keep_results(env):
    from paper_2204_05496_gb300 import serve
    bfv, ctx, keys, model, X, W, b, X_ct = env
    sizes = [12, 1, 1, 9, 1, 2, 1]
    starts = np.cumsum([0] + sizes)
    srv = serve.Server(ctx, keys, model, hbm_budget_bytes=8 << 30, n_streams=2, small_pairs=2 * 8)
    done = srv.run([(0.0, n) for n in sizes], lambda k, n: X_ct[starts[k]:starts[k] + n])
    small = [r.batch for r in done if r.nX * 8 <= 16]
    large = [r.batch for r in done if r.nX * 8 > 16]
    assert not set(small) & set(large)                # the two classes never share a launch
    for r in done:
        assert torch.equal(r.out, _alone(ctx, keys, model, r.X_ct))


def test_server_binary_bank_mixes_models(env):
    """The paper's bank of one-vs-rest binary models (one per cancer type, each with its own
    features): every patient is scored by all 11 models; requests of different models fuse into
    shared launches and each output equals its model's single-request product."""
    from paper_2204_05496_gb300 import serve
    bfv, ctx, keys, model, X, W, b, X_ct = env
    rng = np.random.default_rng(43)
    fs = [int(v) for v in rng.integers(200, 3000, size=11)]
    bank_W = [rng.integers(-127, 128, (f, 2)) for f in fs]
    bank_b = [rng.integers(-127, 128, 2) for _ in fs]
    bank = [ctx.model_prepare(Wm, bm) for Wm, bm in zip(bank_W, bank_b)]
    patients = [(rng.random((1 + (p % 3), 3000)) < 0.05).astype(np.uint8) for p in range(4)]
    inputs = {}
    arrivals = []
    for p, Xp in enumerate(patients):
        for m, f in enumerate(fs):
            k = len(arrivals)
            Xm = Xp[:, :f]
            pt = ctx.encode_features(torch.from_numpy(Xm).cuda())
            inputs[k] = (ctx.encrypt(keys, pt.reshape(-1, ctx.N), seed=900 + k).reshape(Xm.shape[0], -1, 2, ctx.L, ctx.N),
                         Xm, m)
            arrivals.append((0.0005 * p, Xm.shape[0], m))
    srv = serve.Server(ctx, keys, bank, hbm_budget_bytes=8 << 30, n_streams=2)
    done = srv.run(arrivals, lambda k, n: inputs[k][0])
    assert len(done) == len(arrivals) and srv.nbatches < len(arrivals)
    assert any(len({r.model for r in done if r.batch == bt}) > 1 for bt in {r.batch for r in done})
    for r in done:
        X_k, Xm, m = inputs[r.rid]
        assert r.model == m
        assert torch.equal(r.out, ctx.lr_scores_packed(keys, bank[m], X_k))
        slots = ctx.decode(ctx.decrypt(keys, r.out)).cpu().numpy()
        got = bfv.unpack_packed_scores(ctx.N, slots, Xm.shape[0], 2)
        assert np.array_equal(got, oracle.expected_scores(Xm, bank_W[m], bank_b[m], ctx.t))
