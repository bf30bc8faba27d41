"""Host-side scheduling logic of the serving loop, exercised on CPU with a fake context and
fake CUDA objects: admission by class and HBM budget, fusion, and termination."""
import types

import pytest

from paper_2204_05496_gb300 import serve


class FakeEvent:
    def __init__(self, *a, **k):
        self.t = None

    def record(self, stream=None):
        self.t = serve.time.perf_counter()

    def query(self):
        return True

    def elapsed_time(self, other):
        return 1.0

    def synchronize(self):
        pass


class FakeStream:
    def __init__(self, priority=0):
        self.priority = priority
        self.waited = []

    def wait_event(self, ev):
        self.waited.append(ev)

    @staticmethod
    def priority_range():
        return (0, -5)


class _Ctx:
    device = 0
    N = 16

    def __init__(self):
        self.launches = []
        self.models_seen = []

    def models_workspace(self, models, nXs, chunk=0):
        return 100 * sum(nXs)

    def lr_scores_packed_models(self, keys, models, xs, ws=None, pair_chunk=0, stream=None):
        self.launches.append([x.shape[0] for x in xs])
        self.models_seen.append(list(models))
        return [object() for _ in xs]


class _X:
    device = "cuda:0"

    def __init__(self, n):
        self.shape = (n,)
        self.recorded_on = []

    def record_stream(self, s):
        self.recorded_on.append(s)


@pytest.fixture
def fake_torch():
    class _Cuda:
        Stream = FakeStream
        Event = FakeEvent

        producer = FakeStream()

        @staticmethod
        def synchronize():
            pass

        @staticmethod
        def current_stream(device=None):
            return _Cuda.producer

        @staticmethod
        def stream(s):
            class _C:
                def __enter__(self):
                    return s

                def __exit__(self, *a):
                    return False
            return _C()

    return types.SimpleNamespace(cuda=_Cuda, empty=lambda *a, **k: None, uint8=None)


def make(fake_torch, **kw):
    ctx = _Ctx()
    srv = serve.Server(ctx, None, types.SimpleNamespace(nY=2), torch_module=fake_torch, **kw)
    return srv, ctx


def test_both_classes_launch_when_only_large_requests_wait(fake_torch):
    srv, ctx = make(fake_torch, hbm_budget_bytes=10 ** 6, n_streams=2, small_pairs=4)
    srv.start()
    srv.submit(0, _X(9))          # 18 pairs: large class only
    srv.step()
    assert ctx.launches == [[9]]


def test_fusion_respects_budget_and_classes(fake_torch):
    srv, ctx = make(fake_torch, hbm_budget_bytes=500, n_streams=2, small_pairs=4)
    srv.start()
    for k, n in enumerate([1, 2, 1, 3, 1]):   # small: 1, 2, 1, 1 (<= 2 individuals), large: 3
        srv.submit(k, _X(n))
    srv.step()
    # small stream fuses small requests until the 500-byte budget (100 bytes per individual)
    # is reached; the large stream gets nothing because the budget is used up
    assert ctx.launches[0] == [1, 2, 1, 1]
    srv.step()                    # first launch retired (fake events complete) -> room again
    assert [3] in ctx.launches


def test_request_larger_than_budget_raises(fake_torch):
    srv, ctx = make(fake_torch, hbm_budget_bytes=150, n_streams=2)
    with pytest.raises(MemoryError):
        srv.run([(0.0, 2)], lambda k, n: _X(n), max_seconds=5)


def test_requests_of_different_models_fuse_and_count_their_own_pairs(fake_torch):
    # a bank of binary (2-class) models and a 16-class model: pairs = individuals x classes
    # of each request's own model
    ctx = _Ctx()
    bank = [types.SimpleNamespace(nY=2, name=f"binary{k}") for k in range(3)] + [types.SimpleNamespace(nY=16)]
    srv = serve.Server(ctx, None, bank, hbm_budget_bytes=10 ** 6, n_streams=1, max_pairs=39,
                       torch_module=fake_torch)
    srv.start()
    for k, (n, m) in enumerate([(1, 0), (1, 1), (1, 2), (2, 3), (1, 0)]):
        srv.submit(k, _X(n), model=m)
    srv.step()
    # 2 + 2 + 2 + 32 = 38 pairs fit the 39-pair cap; the fifth request (2 more pairs) waits
    assert ctx.launches == [[1, 1, 1, 2]]
    assert [getattr(m, "name", "y16") for m in ctx.models_seen[0]] == ["binary0", "binary1", "binary2", "y16"]
    with pytest.raises(ValueError):
        srv.submit(9, _X(1), model=7)


def test_priority_class_keeps_small_requests_off_the_large_stream(fake_torch):
    # small_pairs = 4 with 2-class models: requests of <= 2 individuals are "small" and go to
    # the high-priority stream 0, larger ones to the normal stream 1, never mixed
    srv, ctx = make(fake_torch, hbm_budget_bytes=10 ** 6, n_streams=2, small_pairs=4)
    assert srv.classes == ["small", "large"] and srv.streams[0].priority < srv.streams[1].priority
    srv.start()
    for k, n in enumerate([5, 1, 9, 2]):
        srv.submit(k, _X(n))
    srv.step()
    assert sorted(ctx.launches) == [[1, 2], [5, 9]]
    small = [b for b in srv.busy if b is not None and all(r.nX <= 2 for r in b[1])]
    assert len(small) == 1 and srv.busy.index(small[0]) == 0


def test_run_replays_a_trace_and_reports_latency(fake_torch):
    srv, ctx = make(fake_torch, hbm_budget_bytes=10 ** 6, n_streams=2)
    trace = [(0.0, 1), (0.0, 3), (0.001, 1), (0.002, 2, 0)]
    done = srv.run(trace, lambda k, n: _X(n), poll_s=0.0001, max_seconds=5)
    assert [r.rid for r in done] == [0, 1, 2, 3] and all(r.t_done is not None for r in done)
    assert sum(len(x) for x in ctx.launches) == 4 and srv.idle()
    rep = serve.latency_report(done, 2)
    assert rep["requests"] == 4 and rep["predictions"] == 7
    assert {"p50_ms", "p99_ms", "predictions_per_s", "single_p50_ms", "single_p99_ms"} <= set(rep)


def test_run_gives_up_after_max_seconds(fake_torch):
    class _Never(FakeEvent):
        def query(self):
            return False

    torch_never = types.SimpleNamespace(cuda=types.SimpleNamespace(**{**vars(fake_torch.cuda), "Event": _Never}),
                                        empty=fake_torch.empty, uint8=None)
    srv, _ = make(torch_never, hbm_budget_bytes=10 ** 6, n_streams=1)
    with pytest.raises(TimeoutError):
        srv.run([(0.0, 1)], lambda k, n: _X(n), poll_s=0.0001, max_seconds=0.05)


def test_launch_waits_for_the_inputs_producer_and_holds_their_memory(fake_torch):
    # a request records an event on the submitting thread's current stream (where its inputs may
    # still be written); its launch stream waits for that event before the product, and the
    # inputs are marked as used by the launch stream
    srv, ctx = make(fake_torch, hbm_budget_bytes=10 ** 6, n_streams=2)
    srv.start()
    xs = [_X(1), _X(2)]
    reqs = [srv.submit(k, x) for k, x in enumerate(xs)]
    srv.step()
    launched = [srv.streams[s] for s, b in enumerate(srv.busy) if b is not None]
    assert len(launched) == 1
    st = launched[0]
    assert [id(e) for e in st.waited] == [id(r.ready) for r in reqs]
    assert all(x.recorded_on == [st] for x in xs)
    srv.step()
    assert srv.intervals and srv.intervals[0]["requests"] == [0, 1]
    assert {"start_s", "end_s", "stream", "batch"} <= set(srv.intervals[0])


def test_inputs_written_on_their_own_stream_bring_their_event(fake_torch):
    # make_inputs may return (X_ct, event) when it writes the inputs on a stream of its own: the
    # launch then waits for that event instead of one recorded on the current stream
    srv, ctx = make(fake_torch, hbm_budget_bytes=10 ** 6, n_streams=1)
    evs = {}

    def make_inputs(k, n):
        evs[k] = FakeEvent()
        return _X(n), evs[k]

    done = srv.run([(0.0, 1), (0.0, 2)], make_inputs, poll_s=0.0001, max_seconds=5)
    assert [r.ready for r in done] == [evs[0], evs[1]]
    assert [id(e) for e in srv.streams[0].waited] == [id(evs[0]), id(evs[1])]
