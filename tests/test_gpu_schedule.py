"""Schedules of the packed product (bfv_packed_schedule): the pair chunk and how each of the four
key-switching kernels splits a limb over CTAs. Every schedule must give the oracle's bits; the
autotuner's choice is recorded for its pair count, written to a schedule file and read back."""
import itertools

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2204_05496_gb300 as bfv


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def host(t):
    return bfv.as_u64(t)


def schedules(chunk):
    for p, m, mp, md in itertools.product((1, 2, 3), (2, 4), (1, 2, 3, 4), (1, 2, 3)):
        yield bfv.Schedule(chunk, p, m, mp, md)


def run(ctx, keys, P, okeys, name):
    """(model, device inputs, oracle output) of a workload; the oracle encrypts its own inputs."""
    w = synth.WORKLOADS[name]
    X, W, b = synth.workload_inputs(w)
    X_ct, _, Y = oracle.packed_pipeline(P, okeys, X, W, b, w.seed_enc)
    return X, W, b, ctx.model_prepare(W, b), dev(X_ct), Y


@pytest.fixture(scope="module")
def tiny():
    w = synth.WORKLOADS["tiny-16"]
    ctx = bfv.Context.from_shape(w.params)
    P = oracle.Params.from_shape(w.params)
    return ctx, ctx.keygen(w.seed_keys), P, oracle.keygen(P, w.seed_keys)


@pytest.fixture(scope="module")
def paper():
    w = synth.WORKLOADS["single-40k"]
    ctx = bfv.Context.from_shape(w.params)
    P = oracle.Params.from_shape(w.params)
    return ctx, ctx.keygen(w.seed_keys), P, oracle.keygen(P, w.seed_keys)


def test_every_schedule_matches_oracle_tiny(tiny):
    """128 pairs at N = 4096: all 72 split combinations, one chunk holding every pair and a
    ragged chunk of 5 pairs."""
    ctx, keys, P, okeys = tiny
    X, W, b, model, Xd, Y = run(ctx, keys, P, okeys, "tiny-16")
    for chunk in (128, 5):
        for sc in schedules(chunk):
            got = ctx.lr_scores_packed_sched(keys, model, Xd, sc)
            assert np.array_equal(host(got), Y), sc.as_dict()


def test_every_schedule_matches_oracle_single_individual(paper):
    """One individual x 40,000 features x 16 classes at N = 16384 (the latency workload), where
    every split takes effect: all 72 combinations bit-exact, and a ragged chunk of 3 pairs."""
    ctx, keys, P, okeys = paper
    X, W, b, model, Xd, Y = run(ctx, keys, P, okeys, "single-40k")
    for sc in schedules(16):
        got = ctx.lr_scores_packed_sched(keys, model, Xd, sc)
        assert np.array_equal(host(got), Y), sc.as_dict()
    got = ctx.lr_scores_packed_sched(keys, model, Xd, bfv.Schedule(3, 2, 4, 2, 1))
    assert np.array_equal(host(got), Y)
    scores = bfv.unpack_packed_scores(P.N, ctx.decode(ctx.decrypt(keys, got)).cpu().numpy(), 1, 16)
    assert np.array_equal(scores, oracle.expected_scores(X, W, b, P.t))


def test_autotuned_schedule_is_recorded_persisted_and_bit_exact(paper, tmp_path):
    ctx, keys, P, okeys = paper
    X, W, b, model, Xd, Y = run(ctx, keys, P, okeys, "single-40k")
    ws = torch.empty(ctx.packed_workspace(model, 1, 16), dtype=torch.uint8, device="cuda")
    best, ms = ctx.autotune_packed_schedule(keys, model, Xd, ws)
    assert ms > 0 and best.pair_chunk == 16
    assert ctx.packed_schedule(16).as_dict() == best.as_dict()
    assert ctx.packed_schedule(17).pair_chunk == 2048                 # other pair counts: the default
    got = ctx.lr_scores_packed(keys, model, Xd, ws=ws)               # pair_chunk 0 -> the tuned schedule
    assert np.array_equal(host(got), Y)
    path = str(tmp_path / "schedules.json")
    ctx.save_schedules(path, [16])
    w = synth.WORKLOADS["single-40k"]
    ctx2 = bfv.Context.from_shape(w.params)
    assert ctx2.load_schedules(path) == 1
    assert ctx2.packed_schedule(16).as_dict() == best.as_dict()
    keys2 = ctx2.keygen(w.seed_keys)
    got2 = ctx2.lr_scores_packed(keys2, ctx2.model_prepare(W, b), Xd)
    assert np.array_equal(host(got2), Y)


def test_schedule_fields_are_checked(tiny):
    ctx, keys, P, okeys = tiny
    for bad in (bfv.Schedule(0, 1, 2, 0, 2), bfv.Schedule(8, 4, 2, 0, 2), bfv.Schedule(8, 0, 2, 0, 2),
                bfv.Schedule(8, 1, 3, 0, 2), bfv.Schedule(8, 1, 2, 5, 2), bfv.Schedule(8, 1, 2, 0, 0),
                bfv.Schedule(8, 1, 2, 0, 4)):
        with pytest.raises(bfv.BfvError):
            ctx.set_packed_schedule(5, bad)


def test_wide_ring_modup_quarters_bit_identical():
    """N = 32768 (two-CTA clusters per limb): ModUp on quarters of a limb gives the bits of ModUp
    on halves (the default, pinned to the oracle by the wide-ring tests) and the closed form."""
    ctx = bfv.Context.from_shape(synth.WIDE32K)
    keys = ctx.keygen(402)
    rng = np.random.default_rng(406)
    X = (rng.random((1, 40000)) < 0.02).astype(np.uint8)
    W = rng.integers(-127, 128, (40000, 16))
    b = rng.integers(-127, 128, 16)
    pt = ctx.encode_features(dev(X).to(torch.uint8))
    X_ct = ctx.encrypt(keys, pt.reshape(-1, ctx.N), seed=407).reshape(1, 2, 2, ctx.L, ctx.N)
    model = ctx.model_prepare(W, b)
    halves = ctx.lr_scores_packed_sched(keys, model, X_ct, bfv.Schedule(16, 1, 2, 0, 2))
    quarters = ctx.lr_scores_packed_sched(keys, model, X_ct, bfv.Schedule(16, 1, 4, 0, 2))
    assert np.array_equal(host(halves), host(quarters))
    scores = bfv.unpack_packed_scores(ctx.N, ctx.decode(ctx.decrypt(keys, quarters)).cpu().numpy(), 1, 16)
    assert np.array_equal(scores, oracle.expected_scores(X, W, b, ctx.t))


def test_encryption_split_options_match_oracle(paper):
    """Encryption at N = 16384 with one 512-thread CTA per limb and with a cluster of two
    256-thread CTAs per limb, two or three (the default) of them per SM: every split gives the
    oracle's ciphertexts."""
    ctx, keys, P, okeys = paper
    assert ctx.get_option(bfv.BFV_OPT_ENCRYPT_SPLIT) == 3
    v = synth.slots(77, 5, P.N, P.t)
    pt = ctx.encode(dev(v))
    want = oracle.encrypt(P, okeys, oracle.encode(P, v), seed=78, obj0=9)
    for split in (1, 2, 3):
        ctx.set_option(bfv.BFV_OPT_ENCRYPT_SPLIT, split)
        assert np.array_equal(host(ctx.encrypt(keys, pt, seed=78, obj0=9)), want), split
    with pytest.raises(bfv.BfvError):
        ctx.set_option(bfv.BFV_OPT_ENCRYPT_SPLIT, 4)
    assert ctx.get_option(bfv.BFV_OPT_ENCRYPT_SPLIT) == 3
