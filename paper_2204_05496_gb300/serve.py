"""Continuous-batching request loop for encrypted LR scoring (packed product, Algorithm 1).

A request carries the encrypted inputs of one or more individuals (already on the device,
uint64[nX][ceil(f/N)][2][L][N]), names the model that scores it (the server may hold several,
e.g. a bank of one-vs-rest binary models with their own feature counts) and receives its own
output ciphertexts. The server keeps the Galois keys and the encoded models resident, and:

  * admits waiting requests while the workspace of the launch they would join fits the HBM
    budget next to the launches already in flight (larger requests wait for memory);
  * fuses every admitted request (up to 64 requests / `max_pairs` pairs, any mix of models)
    into ONE packed product (bfv_lr_scores_packed_models), each request keeping its own outputs;
  * runs up to `n_streams` such launches at once on separate CUDA streams, so a batch formed
    from requests that arrived while another batch was on the GPU overlaps with it;
  * with `small_pairs` > 0, keeps two classes: requests of at most `small_pairs` pairs are
    fused and launched on a high-priority stream of their own, so a single-individual request
    is not held behind a large batch (the GPU block scheduler prefers its CTAs);
  * orders every launch after the work that produced its inputs: a request records an event on
    the submitting thread's current stream, and the launch's stream waits for it (the inputs
    may still be being encrypted or copied there);
  * detects completion from CUDA events and reports per-request latency (arrival to the end
    of its product) with p50/p99 and predictions/s, and each launch's device interval (events
    recorded on its stream before and after the product), which shows whether launches on
    different streams overlapped on the device.

Every request's output is bit-identical to running it alone (the fused product computes each
pair exactly as the single-request call does).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    X_ct: object                 # device tensor [nX][K][2][L][N]
    t_arrival: float             # seconds on the server clock
    model: int = 0               # index of the scoring model in the server's list
    out: object = None           # device tensor of output ciphertexts, set at launch
    t_done: float | None = None  # seconds on the server clock, set at completion
    batch: int = -1
    ready: object = None         # CUDA event: the inputs are written (recorded at submission)
    result: object = None        # what the server's post step returned for this request

    @property
    def nX(self) -> int:
        return int(self.X_ct.shape[0])


class Server:
    def __init__(self, ctx, keys, model, hbm_budget_bytes: int, n_streams: int = 2, max_pairs: int = 8192,
                 pair_chunk: int = 0, small_pairs: int = 0, torch_module=None, post=None):
        if torch_module is None:
            import torch as torch_module
        torch = self.torch = torch_module
        self.ctx, self.keys = ctx, keys
        self.models = list(model) if isinstance(model, (list, tuple)) else [model]
        self.budget = int(hbm_budget_bytes)
        self.max_pairs, self.pair_chunk = max_pairs, pair_chunk
        # post(request, output) runs on the launch's stream right after its product (for instance
        # the client's decryption in a simulation); its return value is kept in request.result and
        # the request completes when it has finished on the device
        self.post = post
        self.small_pairs = small_pairs
        # stream classes: None = any request; "small" / "large" when the classes are split
        if small_pairs > 0:
            lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
            self.streams = [torch.cuda.Stream(priority=min(lo, hi))] + [torch.cuda.Stream() for _ in range(n_streams - 1)]
            self.classes = ["small"] + ["large"] * (n_streams - 1)
        else:
            self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
            self.classes = [None] * n_streams
        self.busy = [None] * n_streams          # (end event, requests, ws bytes, ws, start event, batch) per stream
        self.intervals: list[dict] = []         # device interval of every finished launch
        self.waiting: list[Request] = []
        self.done: list[Request] = []
        self.in_flight_bytes = 0
        self.nbatches = 0
        self.max_concurrent = 0                 # most launches in flight at once
        self.t0_event = torch.cuda.Event(enable_timing=True)
        self.t0_host = None

    # -- clock: host seconds since start; completions come from CUDA events against t0_event
    def start(self):
        self.torch.cuda.synchronize()
        self.t0_event.record()
        self.torch.cuda.synchronize()
        self.t0_host = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0_host

    def submit(self, rid: int, X_ct, t_arrival: float | None = None, model: int = 0, ready=None) -> Request:
        """Queues a request. `ready`: a CUDA event recorded after the work that writes X_ct; by
        default one is recorded now on the current stream of X_ct's device."""
        if not 0 <= model < len(self.models):
            raise ValueError(f"request {rid} names model {model}; the server holds {len(self.models)}")
        r = Request(rid, X_ct, self.now() if t_arrival is None else t_arrival, model)
        if ready is None:
            ready = self.torch.cuda.Event()
            ready.record(self.torch.cuda.current_stream(X_ct.device))
        r.ready = ready
        self.waiting.append(r)
        return r

    def _pairs(self, r: Request) -> int:
        return r.nX * self.models[r.model].nY

    def _ws_bytes(self, reqs) -> int:
        return self.ctx.models_workspace([self.models[r.model] for r in reqs], [r.nX for r in reqs], self.pair_chunk)

    def _retire(self):
        for s, b in enumerate(self.busy):
            if b is not None and b[0].query():
                ev, reqs, nbytes, _, ev0, bt = b
                t = self.t0_event.elapsed_time(ev) / 1e3
                for r in reqs:
                    r.t_done = t
                    self.done.append(r)
                self.intervals.append({"batch": bt, "stream": s, "start_s": self.t0_event.elapsed_time(ev0) / 1e3,
                                       "end_s": t, "requests": [r.rid for r in reqs]})
                self.in_flight_bytes -= nbytes
                self.busy[s] = None

    def _class(self, r: Request) -> str:
        return "small" if self._pairs(r) <= self.small_pairs else "large"

    def _launch(self):
        torch = self.torch
        for s, b in enumerate(self.busy):
            if b is not None or not self.waiting:
                continue
            # admission: take waiting requests of this stream's class in arrival order while
            # pairs, request count and the HBM budget allow
            take, pairs = [], 0
            for r in self.waiting:
                if self.classes[s] is not None and self._class(r) != self.classes[s]:
                    continue
                p = self._pairs(r)
                if take and (pairs + p > self.max_pairs or len(take) == 64):
                    break
                if self.in_flight_bytes + self._ws_bytes(take + [r]) > self.budget:
                    break
                take.append(r)
                pairs += p
            if not take:
                continue
            nbytes = self._ws_bytes(take)
            stream = self.streams[s]
            with torch.cuda.stream(stream):
                for r in take:                  # the inputs' producers come first
                    if r.ready is not None:
                        stream.wait_event(r.ready)
                ev0 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                ws = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{self.ctx.device}")
                outs = self.ctx.lr_scores_packed_models(self.keys, [self.models[r.model] for r in take],
                                                        [r.X_ct for r in take], ws=ws, pair_chunk=self.pair_chunk,
                                                        stream=stream)
                if self.post is not None:
                    for r, o in zip(take, outs):
                        r.result = self.post(r, o)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(stream)
            for r, o in zip(take, outs):
                r.out, r.batch = o, self.nbatches
                # the inputs were allocated on another stream: keep their memory from being reused
                # before this stream has read them, even if the caller drops its reference
                r.X_ct.record_stream(stream)
            self.nbatches += 1
            taken = set(id(r) for r in take)
            self.waiting = [r for r in self.waiting if id(r) not in taken]
            self.in_flight_bytes += nbytes
            self.busy[s] = (ev, take, nbytes, ws, ev0, self.nbatches - 1)
            self.max_concurrent = max(self.max_concurrent, sum(x is not None for x in self.busy))

    def step(self):
        """One scheduling round: retire finished launches, start new ones on free streams."""
        self._retire()
        self._launch()

    def idle(self) -> bool:
        return not self.waiting and all(b is None for b in self.busy)

    def _check_admissible(self):
        """With nothing in flight, every waiting request must fit the budget on its own."""
        if all(b is None for b in self.busy):
            for r in self.waiting:
                if self._ws_bytes([r]) > self.budget:
                    raise MemoryError(f"request {r.rid} needs {self._ws_bytes([r])} bytes, "
                                      f"more than the HBM budget of {self.budget}")

    def run(self, arrivals, make_inputs, poll_s: float = 0.0005, max_seconds: float = 600.0):
        """Replays an arrival trace: arrivals = [(t_seconds, nX)] or [(t_seconds, nX, model)],
        make_inputs(i, nX) -> X_ct, or (X_ct, event) when the inputs are written on a stream of
        their own (the event recorded after that work). Returns the completed requests. Raises
        TimeoutError after max_seconds of wall time."""
        self.start()
        k = 0
        while k < len(arrivals) or not self.idle():
            now = self.now()
            if now > max_seconds:
                raise TimeoutError(f"trace not served within {max_seconds} s")
            while k < len(arrivals) and arrivals[k][0] <= now:
                a = arrivals[k]
                X, ready = _inputs_and_event(make_inputs(k, a[1]))
                self.submit(k, X, a[0], a[2] if len(a) > 2 else 0, ready=ready)
                k += 1
            self.step()
            self._check_admissible()
            if k < len(arrivals) and self.idle():
                time.sleep(max(0.0, min(poll_s * 20, arrivals[k][0] - self.now())))
            else:
                time.sleep(poll_s)
        self.torch.cuda.synchronize()
        self._retire()
        return sorted(self.done, key=lambda r: r.rid)


def _inputs_and_event(inp):
    """make_inputs' result as (X_ct, ready event or None)."""
    return inp if isinstance(inp, tuple) else (inp, None)


def latency_report(reqs, nY: int) -> dict:
    """p50/p99 latency (arrival to completion) and throughput of a finished trace, overall and
    for single-individual requests."""
    lat = np.array([r.t_done - r.t_arrival for r in reqs])
    span = max(r.t_done for r in reqs) - min(r.t_arrival for r in reqs)
    preds = sum(r.nX for r in reqs)
    single = np.array([r.t_done - r.t_arrival for r in reqs if r.nX == 1])
    out = {"requests": len(reqs), "predictions": preds, "p50_ms": float(np.percentile(lat, 50) * 1e3),
           "p99_ms": float(np.percentile(lat, 99) * 1e3), "predictions_per_s": preds / span if span > 0 else 0.0,
           "span_s": span}
    if len(single):
        out["single_p50_ms"] = float(np.percentile(single, 50) * 1e3)
        out["single_p99_ms"] = float(np.percentile(single, 99) * 1e3)
    return out


def run_unbatched(ctx, keys, model, arrivals, make_inputs, pair_chunk: int = 0, post=None):
    """The same trace served one request at a time (FIFO, one stream, no fusion). `model` may be
    a list indexed by the arrivals' third field, as for Server.run; `post` as for Server."""
    import torch
    models = list(model) if isinstance(model, (list, tuple)) else [model]
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t0.record()
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    done = []
    for k, a in enumerate(arrivals):
        ta, nX = a[0], a[1]
        m = a[2] if len(a) > 2 else 0
        while time.perf_counter() - h0 < ta:
            time.sleep(0.0005)
        X, ready = _inputs_and_event(make_inputs(k, nX))
        if ready is not None:
            torch.cuda.current_stream().wait_event(ready)
        r = Request(k, X, ta, m)
        out = ctx.lr_scores_packed(keys, models[m], X, pair_chunk=pair_chunk)
        if post is not None:
            r.result = post(r, out)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record()
        ev.synchronize()
        r.t_done = t0.elapsed_time(ev) / 1e3
        done.append(r)
    return done
