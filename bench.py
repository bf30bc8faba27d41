#!/usr/bin/env python
"""Benchmark: encrypted logistic-regression predictions per second on GB300.

Workload (the headline configuration): BFV ring degree N = 16384, seven 54-bit ciphertext
primes plus one 54-bit key-switching prime, t = 786433; 512 individuals x 40,000 binary
features (Bernoulli 0.02) x 16 classes, int8-range integer weights and biases; synthetic,
seeded inputs. One step = one pass of the whole private inference protocol over the batch
(Section 4.2.2): pack+encode the features, encrypt them (1,536 ciphertexts), the packed
product of Algorithm 1 (8,192 pairs, 14 key-switched rotations each), decrypt, decode.

value     : predictions/s with the features resident in device memory (CUDA events per step,
            L2 flushed between steps; max over ranks under torchrun).
e2e       : the same through the C ABI with HOST buffers (bfv_lr_predict_packed_host:
            pinned features copied in, scores copied out, inside the timed call).
roofline  : the dominant kernel's algorithmic 64-bit modular multiplications per launch over
            its live CUDA-event launch time, against the integer-pipe peak (SMs x 64 32-bit
            multiply-adds per clock x the sampled SM clock / 15 per 64-bit Shoup product).
Also reported: 1-individual latency (p50/p99), the server product alone, the standard
per-element product at the same parameters, per-kernel time shares, and the CPU oracle on a
bounded sample (cpu_baseline). `--impl reference` times the CPU oracle itself.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "encrypted predictions/s @40k features, batch 512; 1-individual p50 latency"
UNIT = "predictions/s"
WORKLOAD = "batch512-40k"
LATENCY_WORKLOAD = "single-40k"

# Integer-pipe peak for 64-bit modular multiplication (the packed path's roofline). An SM issues
# at most 64 32-bit multiply-adds (IMAD) per clock (sm_100-class SMs: 4 sub-partitions x 16 IMAD
# lanes; 59.9 per SM per clock measured in registers on this GPU). A Shoup product x w mod q of
# 64-bit words is 15 32-bit half-products: 7 for the high 64 bits of x * w' (3 full 32x32
# products of the high word pairs plus the carries of the partial sums), 4 for the low 64 bits of
# x * w and 4 for the low 64 bits of floor(x w' / 2^64) * q. So the peak in 64-bit modular
# multiplications per second is SMs x 64 x SM clock / 15, with the SM count of the device and the
# median SM clock sampled during the timed region.
IMAD_PER_CLK_SM, IMAD_PER_MODMUL = 64, 15
SM_MAX_MHZ_NOMINAL = 2070.0


def alu_peak_gmodmul(sms, sm_mhz):
    return sms * IMAD_PER_CLK_SM * sm_mhz * 1e6 / IMAD_PER_MODMUL / 1e9


HBM_FALLBACK_GBS = 6800.0


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    p.add_argument("--pair-chunk", type=int, default=0)
    p.add_argument("--latency-reps", type=int, default=20)
    p.add_argument("--no-standard", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-threads", type=int, default=0,
                   help="threads of the CPU oracle in the cpu_baseline / reference leg (0 = all host cores)")
    p.add_argument("--sweep", action="store_true", help="also time the server product at several pair chunks")
    p.add_argument("--only-packed", action="store_true",
                   help="profiling case: time only the packed product on --individuals of the batch")
    p.add_argument("--individuals", type=int, default=512)
    p.add_argument("--sched-sweep", action="store_true",
                   help="with --only-packed: time every split combination of the key-switching kernels")
    p.add_argument("--autotune", action="store_true",
                   help="with --only-packed: run the schedule autotuner and report its choice")
    p.add_argument("--autotune-save", type=str, default="",
                   help="tune the schedules of the benchmark's packed products (1 and 512 individuals) and "
                        "write them to this schedule file")
    p.add_argument("--ring", choices=["16k", "32k"], default="16k", help="parameter set of --only-packed")
    p.add_argument("--uneven", action="store_true",
                   help="the uneven batch: 64 models on the N = 16384 and N = 32768 sets in one CUDA graph")
    p.add_argument("--uneven-divisor", type=int, default=1, help="divide the drawn batch sizes by this")
    p.add_argument("--paper8k", action="store_true",
                   help="the paper's own workload and parameters: 543 x 40,960 x 11, N = 8192, CRT pair")
    p.add_argument("--only-standard", action="store_true",
                   help="profiling case: time only the standard product on the first --features features")
    p.add_argument("--features", type=int, default=40000)
    p.add_argument("--serve", action="store_true",
                   help="serving case: Poisson request traces through the continuous-batching loop")
    p.add_argument("--rates", type=str, default="1,2,5,20,100,500")
    p.add_argument("--serve-cap", type=int, default=1024, help="predictions offered per rate")
    p.add_argument("--serve-bank", action="store_true",
                   help="serving with the bank of 11 binary one-vs-rest models: every arrival queries all 11")
    return p.parse_args(argv)


# ----------------------------------------------------------------------------- host helpers

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def modmuls_per_pair(kind, N, L, K):
    """Algorithmic 64-bit modular multiplications per pair (one rotation step for the key
    switching kinds). B = butterflies of one length-N NTT."""
    B = (N // 2) * int(round(np.log2(N)))
    return {
        "ks_modup": L * L * B + 2 * L * (L + 1) * N + L * N,   # L^2 digit NTTs + key inner product + P sigma(c0)
        "ks_prep": L * B,                                       # inverse NTT of the L digits
        "ks_moddown_p": 2 * B,                              # inverse NTT of the two P limbs
        "ks_moddown": 2 * L * B + 2 * L * N,                # NTT of the corrections + P^-1 product
        "mac": 2 * L * K * N,
        "bias_mask": 2 * L * N,                             # the two mask products (masks gathered)
    }[kind]


# The source that defines ModUp: its region of k_packed.cu (shape, key products, kernel) and the
# device header (transforms, arithmetic, tensor memory).
MODUP_REGION = ("paper_2204_05496_gb300/csrc/k_packed.cu", "// ModUp works on parts", "// Limb unit (g, c): R[g][c]")


def modup_source_hash():
    path, start, end = MODUP_REGION
    txt = open(os.path.join(ROOT, path)).read()
    h = hashlib.sha256()
    h.update(txt[txt.index(start):txt.index(end)].encode())
    with open(os.path.join(ROOT, "paper_2204_05496_gb300/csrc/bfv_device.cuh"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def recorded_counters(kernel):
    """(DRAM bytes per launch, FMA-heavy pipe % of peak) from the committed ncu summary, if it was
    taken on the kernel's current source (None otherwise)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.md")
    try:
        txt = open(path).read()
    except OSError:
        return None, None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    f = re.search(r"fmaheavy_pct:\s*([0-9.]+)", txt)
    h = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    if not h or h.group(1) != modup_source_hash():
        return None, None
    return (float(m.group(1)) if m else None), (float(f.group(1)) if f else None)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd.insert(1, f"--id={self.uuid}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gather_step_ms(step_ms, world, device):
    """Every rank's mean step time, gathered to all ranks (torch.distributed; NCCL on the GPU
    ranks, gloo in the CPU tests). One rank: no collective."""
    if world <= 1:
        return [step_ms]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(step_ms)], dtype=torch.float64, device=device)
    allt = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(allt, t)
    return [float(x.item()) for x in allt]


def aggregate(per_rank_ms, units_per_rank):
    """Whole-job throughput from per-rank step times: every rank processes its own batch;
    the job takes as long as the slowest rank (max over ranks)."""
    slow = max(per_rank_ms)
    return units_per_rank * len(per_rank_ms) / (slow / 1e3), slow


# ----------------------------------------------------------------------------- CPU oracle (baseline / reference)

def oracle_sample(n_individuals, steps=1, warmup=0, threads=0):
    """The CPU oracle, as it stands, on `n_individuals` of the headline batch: encode, encrypt,
    Algorithm 1, decrypt, decode, on `threads` host threads (0 = all). Returns (predictions/s,
    threads used, seconds per step)."""
    import oracle
    w = synth.WORKLOADS[WORKLOAD]
    X, W, b = synth.workload_inputs(w)
    P = oracle.Params.from_shape(w.params, nthreads=threads or None)
    keys = oracle.keygen(P, w.seed_keys)
    W_pt = oracle.encode(P, oracle.pack_weights(P, W).reshape(-1, P.N)).reshape(W.shape[1], -1, P.N)
    times = []
    for s in range(warmup + steps):
        i0 = (s * n_individuals) % X.shape[0]
        Xs = X[i0:i0 + n_individuals]
        t0 = time.perf_counter()
        pt = oracle.encode(P, oracle.pack_inputs(P, Xs).reshape(-1, P.N))
        ct = oracle.encrypt(P, keys, pt, w.seed_enc, obj0=3 * i0).reshape(len(Xs), -1, 2, P.L, P.N)
        Y = oracle.lr_packed(P, keys, ct, W_pt, b)
        slots = oracle.decode(P, oracle.decrypt(P, keys.sk, Y))
        dt = time.perf_counter() - t0
        got = oracle.unpack_packed_scores(P, slots, len(Xs), W.shape[1])
        assert np.array_equal(got, oracle.expected_scores(Xs, W, b, P.t))
        if s >= warmup:
            times.append(dt)
    sec = sum(times) / len(times)
    return n_individuals / sec, P.nthreads, sec


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    sample = 1
    v, cores, sec = oracle_sample(sample, steps=args.steps, warmup=args.warmup, threads=args.cpu_threads)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": config_block(args, chunk=None),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} individual (16 pairs) of the 512-individual batch per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_block(args, chunk, schedule=None):
    w = synth.WORKLOADS[WORKLOAD]
    out = {
        "workload": (f"{WORKLOAD}: BFV N={w.params.N}, L={w.params.L} x {w.params.prime_bits}-bit primes + 1 "
                     f"special prime, t={w.params.t}; {w.n_individuals} individuals x {w.n_features} "
                     f"Bernoulli({w.p_feature}) binary features x {w.n_classes} classes, int8-range weights"),
        "global_batch": w.n_individuals * max(1, args.gpus),
        "individuals_per_gpu": w.n_individuals,
        "features": w.n_features,
        "classes": w.n_classes,
        "pair_chunk": chunk,
        "l2": "flushed (256 MB write) between timed steps; per-step working set ~15 GB >> 129 MB L2",
        "parallelism": f"independent replicas x{max(1, args.gpus)}",
    }
    if schedule is not None:
        out["packed_schedule"] = schedule
    return out


# ----------------------------------------------------------------------------- GPU arm

def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import paper_2204_05496_gb300 as bfv
    bfv.build()

    w = synth.WORKLOADS[WORKLOAD]
    X, W, b = synth.workload_inputs(w)
    nX, nY = X.shape[0], W.shape[1]
    ctx = bfv.Context.from_shape(w.params)
    keys = ctx.keygen(w.seed_keys)
    model = ctx.model_prepare(W, b)
    chunk = args.pair_chunk
    Xd = torch.from_numpy(X).to(dev)
    ws = torch.empty(ctx.predict_workspace(model, nX, chunk), dtype=torch.uint8, device=dev)
    scores = torch.empty((nX, nY), dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    want = (X.astype(np.int64) @ W + b[None, :]) % w.params.t

    def step(i):
        ctx.predict_packed(keys, model, Xd, seed=w.seed_enc + i, out=scores, ws=ws, pair_chunk=chunk)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if not np.array_equal(scores.cpu().numpy(), want):
        raise SystemExit("benchmarked path produced wrong scores")

    uuid = None
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        uuid = f"GPU-{u}" if u and not str(u).startswith("GPU-") else str(u)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    sampler.start()
    ctx.profile(True)
    ctx.profile_read()
    evs = []
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step(args.warmup + i)
        z.record()
        evs.append((a, z))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ctx.profile(False)
    kern = ctx.profile_read()
    clocks = sampler.stop()
    gpu_launches = ctx.launch_count() - launches0
    step_ms = sum(a.elapsed_time(z) for a, z in evs) / args.steps
    per_rank = gather_step_ms(step_ms, world, dev)
    if world > 1:
        dist.barrier()
    value, slow_ms = aggregate(per_rank, nX)
    if not np.array_equal(scores.cpu().numpy(), want):
        raise SystemExit("benchmarked path produced wrong scores")

    extras = {}
    if rank == 0:
        extras = gpu_extras(args, ctx, keys, model, X, W, b, ws, chunk, dev, kern, step_ms, clocks)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return 0

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": slow_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded; stands in for iDASH/TCGA)",
        "config": config_block(args, chunk, ctx.packed_schedule(nX * nY).as_dict() if not chunk else None),
        "clocks": clocks,
        "gpu_launches": gpu_launches,
        "wall_s_timed_region": wall,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    return 0


def gpu_extras(args, ctx, keys, model, X, W, b, ws, chunk, dev, kern, step_ms, clocks):
    import torch
    w = synth.WORKLOADS[WORKLOAD]
    N, L, K = w.params.N, w.params.L, model.K
    nX, nY = X.shape[0], model.nY
    out = {}

    # per-kernel shares over the timed steps and the dominant kernel's roofline
    total = sum(ms for _, ms in kern.values()) or 1.0
    pairs = nX * nY
    plan_chunk = min(pairs, chunk if chunk else ctx.packed_schedule(pairs).pair_chunk)
    rot = int(round(np.log2(N)))
    shares = {}
    work = {}
    for name, (n, ms) in kern.items():
        if n == 0:
            continue
        d = {"launches": n, "ms_total": round(ms, 3), "share": round(ms / total, 4)}
        if name in ("ks_modup", "ks_prep", "ks_moddown_p", "ks_moddown", "mac", "bias_mask"):
            work[name] = modmuls_per_pair(name, N, L, K) * pairs * (rot if name.startswith("ks_") else 1) * args.steps
            d["gmodmul_per_s"] = round(work[name] / (ms / 1e3) / 1e9, 1)
        shares[name] = d
    out["kernels"] = shares
    top = max(shares, key=lambda k: shares[k]["ms_total"])
    n, ms = kern[top]
    if top in work:
        per_launch = work[top] / n
        achieved = per_launch / (ms / n / 1e3) / 1e9
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = clocks.get("sm_mhz") or SM_MAX_MHZ_NOMINAL
        peak = alu_peak_gmodmul(sms, mhz)
        traffic, fma = recorded_counters(top) if top == "ks_modup" else (None, None)
        out["roofline"] = {"kernel": top, "bound": "alu", "achieved": round(achieved, 1),
                           "peak": round(peak, 1), "unit": "Gmodmul/s",
                           "frac": round(achieved / peak, 4), "traffic": traffic,
                           "ncu_fmaheavy_pipe_pct": fma,
                           "work_per_launch": f"{per_launch:.4g} 64-bit modular multiplications "
                                              f"({plan_chunk} pairs x one key switch)",
                           "peak_basis": f"{sms} SMs x 64 IMAD/clk x {mhz:.0f} MHz (median sampled SM clock) / "
                                         f"15 32-bit half-products per Shoup product"}

    # server product alone (inputs already encrypted)
    pt = ctx.encode_features(torch.from_numpy(X).to(dev))
    X_ct = ctx.encrypt(keys, pt.reshape(-1, N), seed=w.seed_enc).reshape(nX, K, 2, L, N)
    pws = torch.empty(ctx.packed_workspace(model, nX, chunk), dtype=torch.uint8, device=dev)
    Y = ctx.lr_scores_packed(keys, model, X_ct, ws=pws, pair_chunk=chunk)
    torch.cuda.synchronize()
    reps = 2
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        ctx.lr_scores_packed(keys, model, X_ct, out=Y, ws=pws, pair_chunk=chunk)
    z.record()
    torch.cuda.synchronize()
    sms = a.elapsed_time(z) / reps
    out["server_only"] = {"ms": round(sms, 2), "predictions_per_s": round(nX / (sms / 1e3), 1)}
    # the same product replayed from a CUDA graph (one host call per product)
    ctx.lr_scores_packed_graph(keys, model, X_ct, out=Y, ws=pws, pair_chunk=chunk)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        ctx.lr_scores_packed_graph(keys, model, X_ct, out=Y, ws=pws, pair_chunk=chunk)
    z.record()
    torch.cuda.synchronize()
    out["server_only"]["graph_ms"] = round(a.elapsed_time(z) / reps, 2)
    if args.sweep:
        del pws
        sweep = {}
        for ch in (512, 1024, 2048, 4096, 8192):
            sw = torch.empty(ctx.packed_workspace(model, nX, ch), dtype=torch.uint8, device=dev)
            ctx.lr_scores_packed(keys, model, X_ct, out=Y, ws=sw, pair_chunk=ch)
            a.record()
            ctx.lr_scores_packed(keys, model, X_ct, out=Y, ws=sw, pair_chunk=ch)
            z.record()
            torch.cuda.synchronize()
            sweep[ch] = round(a.elapsed_time(z), 1)
            del sw
        out["server_only"]["chunk_sweep_ms"] = sweep
    else:
        del pws
    del Y, X_ct, pt

    # end to end through the C ABI with host buffers
    Xh = torch.from_numpy(X).pin_memory()
    sh = torch.empty((nX, nY), dtype=torch.int64).pin_memory()
    e2e_t = []
    for i in range(max(2, args.steps)):
        t0 = time.perf_counter()
        ctx.predict_packed_host(keys, model, Xh, seed=w.seed_enc + i, out=sh, ws=ws, pair_chunk=chunk)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e_t[1:]) if len(e2e_t) > 1 else e2e_t[0]
    out["e2e"] = {"value": round(nX / e2e_s, 2), "unit": UNIT, "h2d_bytes_per_step": int(X.nbytes),
                  "d2h_bytes_per_step": int(nX * nY * 8), "ms_per_step": round(e2e_s * 1e3, 2)}

    # one individual: latency of the whole protocol (the metric's second half)
    lw = synth.WORKLOADS[LATENCY_WORKLOAD]
    X1, W1, b1 = synth.workload_inputs(lw)
    k1 = ctx.keygen(lw.seed_keys)
    m1 = ctx.model_prepare(W1, b1)
    X1d = torch.from_numpy(X1).to(dev)
    ws1 = torch.empty(ctx.predict_workspace(m1, 1, 0), dtype=torch.uint8, device=dev)
    s1 = torch.empty((1, W1.shape[1]), dtype=torch.int64, device=dev)
    lat = []
    for i in range(3 + args.latency_reps):
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.predict_packed(k1, m1, X1d, seed=lw.seed_enc + i, out=s1, ws=ws1)
        z.record()
        torch.cuda.synchronize()
        if i >= 3:
            lat.append(a.elapsed_time(z))
    # the server product alone for one individual, launched directly and from a graph
    pt1 = ctx.encode_features(X1d)
    X1_ct = ctx.encrypt(k1, pt1.reshape(-1, lw.params.N), seed=lw.seed_enc).reshape(1, m1.K, 2, lw.params.L, lw.params.N)
    pw1 = torch.empty(ctx.packed_workspace(m1, 1, 0), dtype=torch.uint8, device=dev)
    Y1 = ctx.lr_scores_packed(k1, m1, X1_ct, ws=pw1)
    srv = {}
    for name, fn in (("direct", ctx.lr_scores_packed), ("graph", ctx.lr_scores_packed_graph)):
        fn(k1, m1, X1_ct, out=Y1, ws=pw1)
        ts = []
        for _ in range(10):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn(k1, m1, X1_ct, out=Y1, ws=pw1)
            z.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(z))
        srv[name] = round(sorted(ts)[len(ts) // 2], 3)
    del pw1, Y1, X1_ct, pt1
    want1 = (X1.astype(np.int64) @ W1 + b1[None, :]) % lw.params.t
    assert np.array_equal(s1.cpu().numpy(), want1)
    X1h = torch.from_numpy(X1).pin_memory()
    s1h = torch.empty((1, W1.shape[1]), dtype=torch.int64).pin_memory()
    lat_e2e = []
    for i in range(3 + args.latency_reps):
        t0 = time.perf_counter()
        ctx.predict_packed_host(k1, m1, X1h, seed=lw.seed_enc + i, out=s1h, ws=ws1)
        if i >= 3:
            lat_e2e.append((time.perf_counter() - t0) * 1e3)
    lat.sort()
    lat_e2e.sort()
    out["latency_1_individual"] = {
        "p50_ms": round(lat[len(lat) // 2], 3), "p99_ms": round(lat[min(len(lat) - 1, int(0.99 * len(lat)))], 3),
        "e2e_p50_ms": round(lat_e2e[len(lat_e2e) // 2], 3), "reps": len(lat),
        "server_product_p50_ms": srv,
        "workload": f"{LATENCY_WORKLOAD}: 1 individual x {lw.n_features} features x {lw.n_classes} classes, same BFV parameters"}
    del ws1

    if not args.no_standard:
        out["standard"] = standard_leg(args, ctx, keys, model, X, W, b, dev, step_ms, lat[len(lat) // 2])
    if not args.no_cpu_baseline and int(os.environ.get("WORLD_SIZE", "1")) == 1:
        n = 4 if not args.cpu_threads or args.cpu_threads > 4 else 1    # ~10-40 s of CPU work
        v, cores, sec = oracle_sample(n, threads=args.cpu_threads)
        out["cpu_baseline"] = {"value": round(v, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{n} individual(s) ({n * W.shape[1]} pairs) of the 512-individual batch, "
                                         f"whole protocol ({sec:.1f} s)"}
    return out


def standard_leg(args, ctx, keys, model, X, W, b, dev, packed_step_ms, packed_lat_ms):
    """The standard per-element product at the same parameters (Section 5.2.3): encode the
    40,000 feature columns, encrypt them (73 GB), scalar-weighted sums, decrypt |Y| outputs."""
    import torch
    w = synth.WORKLOADS[WORKLOAD]
    N, L = w.params.N, w.params.L
    nX, f = X.shape
    nY = model.nY
    Xd = torch.from_numpy(X).to(dev)
    X_ct = torch.empty((f, 2, L, N), dtype=torch.int64, device=dev)
    blk = 4000
    ews = torch.empty(ctx.encrypt_workspace(blk), dtype=torch.uint8, device=dev)
    Y = torch.empty((nY, 2, L, N), dtype=torch.int64, device=dev)
    sws = torch.empty(ctx.standard_workspace(model), dtype=torch.uint8, device=dev)

    def run(seed):
        cols = ctx.encode_feature_columns(Xd)
        for f0 in range(0, f, blk):
            ctx.encrypt(keys, cols[f0:f0 + blk], seed=seed, obj0=f0, out=X_ct[f0:f0 + blk], ws=ews)
        del cols
        ctx.lr_scores_standard(model, X_ct, nX, out=Y, ws=sws)
        return ctx.decode(ctx.decrypt(keys, Y))

    slots = run(1)
    torch.cuda.synchronize()
    want = (X.astype(np.int64) @ W + b[None, :]) % w.params.t
    if not np.array_equal(slots.cpu().numpy()[:, :nX].T, want):
        raise SystemExit("standard product produced wrong scores")
    ctx.profile(True)
    ctx.profile_read()
    times = []
    for i in range(max(2, min(3, args.steps))):
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run(2 + i)
        z.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(z))
    ctx.profile(False)
    kern = ctx.profile_read()
    ms = statistics.mean(times)
    n, kms = kern["standard"]
    bytes_per_launch = f * 2 * L * N * 8 + nY * 2 * L * N * 8
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", HBM_FALLBACK_GBS)
    gbs = bytes_per_launch / (kms / n / 1e3) / 1e9
    res = {
        "ms_per_batch": round(ms, 2), "predictions_per_s_batch512": round(nX / (ms / 1e3), 2),
        "latency_1_individual_ms": round(ms, 2),
        "note": "cost is independent of the batch size up to N = 16384 individuals",
        "product_kernel_ms": round(kms / n, 2),
        "product_roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                             "frac": round(gbs / hbm, 4),
                             "traffic_algorithmic_bytes": bytes_per_launch,
                             "peak_basis": "measured" if "hbm_gbs" in peaks else "fallback"},
        "packed_speedup_batch512": round(ms / packed_step_ms, 2),
        "packed_speedup_1_individual": round(ms / packed_lat_ms, 1),
        "encrypt_ms": round(kern["encrypt"][1] / max(1, len(times)), 2),
    }
    if ctx.check_error():
        raise SystemExit("a bounded wait in the standard product ran out")
    del X_ct, ews, sws
    torch.cuda.empty_cache()
    return res


def run_only_packed(args):
    """Small profiling case: the packed product alone on the first --individuals of the batch
    (same kernels, fewer pairs; --ring 32k runs it on the N = 32768 parameter set),
    --warmup untimed then --steps timed calls, then one call with per-kernel timing."""
    import torch
    import paper_2204_05496_gb300 as bfv
    bfv.build()
    torch.cuda.set_device(0)
    w = synth.WORKLOADS[WORKLOAD]
    X, W, b = synth.workload_inputs(w)
    X = X[:args.individuals]
    shape = synth.WIDE32K if args.ring == "32k" else w.params
    N, L = shape.N, shape.L
    ctx = bfv.Context.from_shape(shape)
    keys = ctx.keygen(w.seed_keys)
    model = ctx.model_prepare(W, b)
    pt = ctx.encode_features(torch.from_numpy(X).cuda())
    X_ct = ctx.encrypt(keys, pt.reshape(-1, N), seed=w.seed_enc).reshape(len(X), model.K, 2, L, N)
    ws = torch.empty(ctx.packed_workspace(model, len(X), args.pair_chunk), dtype=torch.uint8, device="cuda")
    Y = ctx.lr_scores_packed(keys, model, X_ct, ws=ws, pair_chunk=args.pair_chunk)
    for _ in range(args.warmup - 1):
        ctx.lr_scores_packed(keys, model, X_ct, out=Y, ws=ws, pair_chunk=args.pair_chunk)
    torch.cuda.synchronize()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        ctx.lr_scores_packed(keys, model, X_ct, out=Y, ws=ws, pair_chunk=args.pair_chunk)
    z.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(z) / args.steps
    # per-kernel device time of one call (an event pair around every launch) against the call's
    # own time: the rest is the gap between dependent launches
    ctx.profile(True)
    ctx.profile_read()
    a.record()
    ctx.lr_scores_packed(keys, model, X_ct, out=Y, ws=ws, pair_chunk=args.pair_chunk)
    z.record()
    torch.cuda.synchronize()
    ctx.profile(False)
    prof_call_ms = a.elapsed_time(z)
    kern = {k: round(v[1], 3) for k, v in ctx.profile_read().items() if v[0]}
    slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
    got = bfv.unpack_packed_scores(N, slots, len(X), W.shape[1])
    ok = bool(np.array_equal(got, (X.astype(np.int64) @ W + b[None, :]) % shape.t))
    pairs = len(X) * W.shape[1]
    # the same product from a CUDA graph
    ctx.lr_scores_packed_graph(keys, model, X_ct, out=Y, ws=ws, pair_chunk=args.pair_chunk)
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.steps):
        ctx.lr_scores_packed_graph(keys, model, X_ct, out=Y, ws=ws, pair_chunk=args.pair_chunk)
    z.record()
    torch.cuda.synchronize()
    graph_ms = a.elapsed_time(z) / args.steps
    res = {"case": "only-packed", "ring": N, "individuals": len(X), "pairs": pairs,
           "schedule": ctx.packed_schedule(pairs).as_dict() if not args.pair_chunk else {"pair_chunk": args.pair_chunk},
           "ms_per_call": round(ms, 3), "graph_ms_per_call": round(graph_ms, 3),
           "us_per_pair": round(ms * 1e3 / pairs, 2), "kernel_ms": kern,
           "launch_gap_frac": round(1 - sum(kern.values()) / prof_call_ms, 4), "correct": ok}
    if args.sched_sweep:
        # every split combination at the plan's chunk (bit-identical results; times only)
        chunk = args.pair_chunk or ctx.packed_schedule(pairs).pair_chunk
        sweep = {}
        for p_, m_, mp_, md_ in [(p_, m_, mp_, md_) for p_ in (1, 2, 3) for m_ in (2, 4) for mp_ in (1, 2, 3, 4)
                                 for md_ in (1, 2, 3)]:
            sc = bfv.Schedule(chunk, p_, m_, mp_, md_)
            Ys = ctx.lr_scores_packed_sched(keys, model, X_ct, sc, ws=ws)
            ok = ok and bool(torch.equal(Ys, Y))
            a.record()
            for _ in range(args.steps):
                ctx.lr_scores_packed_sched(keys, model, X_ct, sc, out=Ys, ws=ws)
            z.record()
            torch.cuda.synchronize()
            sweep[f"p{p_}m{m_}dp{mp_}d{md_}"] = round(a.elapsed_time(z) / args.steps, 3)
        res["sched_sweep_ms"] = sweep
        best = min(sweep, key=sweep.get)
        res["sched_best"] = best
        res["correct"] = ok
    if args.autotune:
        big = torch.empty(ctx.packed_workspace(model, len(X), 16384), dtype=torch.uint8, device="cuda") \
            if not args.pair_chunk else ws
        best, bms = ctx.autotune_packed_schedule(keys, model, X_ct, big)
        res["autotuned"] = {"schedule": best.as_dict(), "ms": round(bms, 3)}
        del big
    print(json.dumps(res), flush=True)
    return 0 if res["correct"] else 1


def run_uneven(args):
    """The uneven batch: 64 models (f in {1k, 5k, 20k, 40k}, |Y| in {2, 8, 16}, |X| in 1..512 divided
    by --uneven-divisor) on the N = 16384 and N = 32768 parameter sets. The models of each ring
    form one fused packed product; both products are captured into one CUDA graph. A sub-sampled
    pass (batch sizes / 64) through the same path loads every kernel first; then the graph of the
    requested batch is replayed once, timed with CUDA events, and every score is checked."""
    import torch
    import paper_2204_05496_gb300 as bfv
    bfv.build()
    torch.cuda.set_device(0)
    rings = ("PAPER16K", "WIDE32K")
    ctxs = {r: bfv.Context.from_shape(getattr(synth, r)) for r in rings}
    keys = {r: ctxs[r].keygen(402) for r in rings}

    def prepare(div):
        items = synth.uneven_batch(x_divisor=div)
        for it in items:
            ctx = ctxs[it["params"]]
            it["model"] = ctx.model_prepare(it["W"], it["b"])
            pt = ctx.encode_features(torch.from_numpy(it["X"]).cuda())
            it["X_ct"] = ctx.encrypt(keys[it["params"]], pt.reshape(-1, ctx.N), seed=it["enc_seed"]).reshape(
                it["nX"], -1, 2, ctx.L, ctx.N)
            del pt
        plan = {}
        for r in rings:
            grp = [it for it in items if it["params"] == r]
            ctx = ctxs[r]
            models = [it["model"] for it in grp]
            ws = torch.empty(ctx.models_workspace(models, [it["nX"] for it in grp]), dtype=torch.uint8, device="cuda")
            outs = [ctx._empty_u64(-(-it["nX"] * it["nY"] // ctx.N), 2, ctx.L, ctx.N) for it in grp]
            plan[r] = (grp, models, [it["X_ct"] for it in grp], outs, ws)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            st = torch.cuda.current_stream()
            for r in rings:
                grp, models, xs, outs, ws = plan[r]
                ctxs[r].lr_scores_packed_models(keys[r], models, xs, outs=outs, ws=ws, stream=st)
        return items, plan, g

    def check(plan):
        for r in rings:
            grp, models, xs, outs, ws = plan[r]
            ctx = ctxs[r]
            for it, o in zip(grp, outs):
                slots = ctx.decode(ctx.decrypt(keys[r], o)).cpu().numpy()
                got = bfv.unpack_packed_scores(ctx.N, slots, it["nX"], it["nY"])
                want = (it["X"].astype(np.int64) @ it["W"] + it["b"][None, :]) % ctx.t
                if not np.array_equal(got, want):
                    return False
        return True

    items, plan, g = prepare(64)
    g.replay()
    torch.cuda.synchronize()
    ok_small = check(plan)
    del items, plan, g
    torch.cuda.empty_cache()
    items, plan, g = prepare(args.uneven_divisor)
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    g.replay()
    z.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(z)
    ok = ok_small and check(plan)
    per = {}
    for r in rings:
        grp = plan[r][0]
        per[r] = {"models": len(grp), "individuals": sum(it["nX"] for it in grp),
                  "pairs": sum(it["nX"] * it["nY"] for it in grp),
                  "input_ciphertexts": sum(it["X_ct"].shape[0] * it["X_ct"].shape[1] for it in grp)}
    preds = sum(it["nX"] for it in items)
    pairs = sum(v["pairs"] for v in per.values())
    print(json.dumps({"case": "uneven", "batch_divisor": args.uneven_divisor, "graph_launches": 1,
                      "ms": round(ms, 1), "predictions": preds, "pairs": pairs,
                      "predictions_per_s": round(preds / (ms / 1e3), 2), "pairs_per_s": round(pairs / (ms / 1e3), 1),
                      "rings": per, "correct": ok}), flush=True)
    return 0 if ok else 1


def run_paper8k(args):
    """The paper's own configuration (Section 5.2.3): 543 patients x 40,960 features x 11 classes,
    N = 8192, plaintext moduli t0 = 1073872897 and t1 = 114689 (CRT pair), fixed-point inputs
    (2^6) and weights (2^14). Real-valued synthetic inputs (synth.paper_realvalued). Timed with
    CUDA events per phase, like the paper's figure: encryption (encode + encrypt, both rings),
    computation (packed product, both rings), decryption (decrypt + decode + CRT). Every score
    is checked against the exact integer product. The standard product runs on the same data."""
    import torch
    import paper_2204_05496_gb300 as bfv
    from paper_2204_05496_gb300 import crt_pair
    bfv.build()
    torch.cuda.set_device(0)
    nX, f, nY = 543, 40960, 11
    X, W, b = synth.paper_realvalued(701, nX, f, nY)
    Xi, Wi, bi = crt_pair.to_fixed(X, crt_pair.S_X), crt_pair.to_fixed(W, crt_pair.S_W), \
        crt_pair.to_fixed(b, crt_pair.S_X + crt_pair.S_W)
    exact = Xi @ Wi + bi[None, :]
    pair = crt_pair.CrtPair(8192, 4, 43)
    keys = pair.keygen(702)
    models = pair.model_prepare(Wi, bi)
    Xd = torch.from_numpy(Xi).cuda()

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        return e

    def once(seed):
        e0 = ev()
        X_cts = pair.encrypt_rows(keys, Xd, seed=seed)
        e1 = ev()
        Y = pair.scores_packed(keys, models, X_cts)
        e2 = ev()
        z = pair.decrypt_scores(keys, Y, nX, nY)
        e3 = ev()
        torch.cuda.synchronize()
        return z, (e0.elapsed_time(e1), e1.elapsed_time(e2), e2.elapsed_time(e3))

    z, _ = once(703)                                        # warm-up
    ok = bool(np.array_equal(z.cpu().numpy(), exact))
    runs = [once(704 + 2 * i)[1] for i in range(max(1, args.steps))]
    enc, comp, dec = (statistics.median(r[k] for r in runs) for k in range(3))
    total = enc + comp + dec
    # standard product on the same data: feature columns, slot i = patient i
    cols = torch.zeros((f, 8192), dtype=torch.int64, device="cuda")
    cols[:, :nX] = Xd.T
    std = []
    for rep in range(2):
        e0 = ev()
        outs = []
        for r, c in enumerate(pair.ctx):
            X_ct = c.encrypt(keys[r], c.encode(cols), seed=800 + rep)
            Ys = c.lr_scores_standard(models[r], X_ct, nX)
            outs.append(c.decode(c.decrypt(keys[r], Ys))[:, :nX].T.contiguous())
            del X_ct
        zs = bfv.crt_combine(outs[0], pair.t[0], outs[1], pair.t[1])
        e1 = ev()
        torch.cuda.synchronize()
        std.append(e0.elapsed_time(e1))
        ok = ok and bool(np.array_equal(zs.cpu().numpy(), exact))
    argmax_ok = bool(np.array_equal(np.argmax(exact, axis=1), np.argmax(z.cpu().numpy(), axis=1)))
    print(json.dumps({
        "case": "paper8k", "workload": "543 patients x 40,960 real-valued features x 11 classes; BFV N=8192, "
        "4+1 x 43-bit primes, CRT pair t0=1073872897 / t1=114689, s_x=6, s_w=14",
        "encryption_ms": round(enc, 2), "computation_ms": round(comp, 2), "decryption_ms": round(dec, 2),
        "total_ms": round(total, 2), "predictions_per_s": round(nX / (total / 1e3), 1),
        "paper_total_s": 46.77, "paper_computation_s": 35.52, "paper_encryption_s": 10.40,
        "speedup_vs_paper_total": round(46.77e3 / total, 1),
        "standard_total_ms": round(min(std), 2), "packed_speedup_vs_standard": round(min(std) / total, 2),
        "paper_standard_total_s": "about 600 (10 min)",
        "max_score_bits": round(float(np.log2(np.abs(exact).max())), 1), "correct": ok, "argmax_correct": argmax_ok}),
        flush=True)
    return 0 if ok else 1


def run_only_standard(args):
    """Small profiling case: the standard product alone on the first --features features of the
    batch (same parameters and kernels), --warmup untimed then --steps timed calls, for the
    tensor-core and the dp4a kernel; also the encryption of the feature columns with one and with
    two CTAs per limb."""
    import torch
    import paper_2204_05496_gb300 as bfv
    bfv.build()
    torch.cuda.set_device(0)
    w = synth.WORKLOADS[WORKLOAD]
    X, W, b = synth.workload_inputs(w)
    X, W = X[:, :args.features], W[:args.features]
    N, L = w.params.N, w.params.L
    ctx = bfv.Context.from_shape(w.params)
    keys = ctx.keygen(w.seed_keys)
    model = ctx.model_prepare(W, b)
    cols = ctx.encode_feature_columns(torch.from_numpy(X).cuda())
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    enc = {}
    X_ct = None
    for split in (1, 2, 3):
        ctx.set_option(bfv.BFV_OPT_ENCRYPT_SPLIT, split)
        X_ct = ctx.encrypt(keys, cols, seed=w.seed_enc, out=X_ct)
        torch.cuda.synchronize()
        a.record()
        ctx.encrypt(keys, cols, seed=w.seed_enc, out=X_ct)
        z.record()
        torch.cuda.synchronize()
        enc[f"split{split}"] = round(a.elapsed_time(z), 3)
    ctx.set_option(bfv.BFV_OPT_ENCRYPT_SPLIT, 3)
    del cols
    sws = torch.empty(ctx.standard_workspace(model), dtype=torch.uint8, device="cuda")
    want = (X.astype(np.int64) @ W + b[None, :]) % w.params.t
    res = {"case": "only-standard", "features": args.features, "encrypt_ms": enc}
    ok = True
    Yref = None
    for name, kind in (("tensor", 0), ("dp4a", 1)):
        ctx.set_option(bfv.BFV_OPT_STANDARD_KERNEL, kind)
        Y = ctx.lr_scores_standard(model, X_ct, len(X), ws=sws)
        for _ in range(args.warmup - 1):
            ctx.lr_scores_standard(model, X_ct, len(X), out=Y, ws=sws)
        torch.cuda.synchronize()
        a.record()
        for _ in range(args.steps):
            ctx.lr_scores_standard(model, X_ct, len(X), out=Y, ws=sws)
        z.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(z) / args.steps
        slots = ctx.decode(ctx.decrypt(keys, Y)).cpu().numpy()
        good = bool(np.array_equal(slots[:, :len(X)].T, want)) and ctx.check_error() == 0
        if Yref is None:
            Yref = Y.clone()
        else:
            good = good and bool(torch.equal(Y, Yref))
        ok = ok and good
        gb = args.features * 2 * L * N * 8 / 1e9
        res[name] = {"ms_per_call": round(ms, 3), "gb_per_s": round(gb / (ms / 1e3), 1), "correct": good}
    ctx.set_option(bfv.BFV_OPT_STANDARD_KERNEL, 0)
    res["correct"] = ok
    print(json.dumps(res), flush=True)
    return 0 if ok else 1


def run_serve(args):
    """Serving workload: Poisson arrivals, 70% single-individual and 30% 16..512-individual
    requests on the 40,000-feature x 16-class model; keys and model resident; the
    continuous-batching loop (HBM budget 64 GB, two streams) against the same requests served
    one at a time. Each rate's trace stops once --serve-cap predictions have been offered."""
    import torch
    import paper_2204_05496_gb300 as bfv
    from paper_2204_05496_gb300 import serve
    bfv.build()
    torch.cuda.set_device(0)
    w = synth.WORKLOADS[WORKLOAD]
    X, W, b = synth.workload_inputs(w)
    N, L = w.params.N, w.params.L
    ctx = bfv.Context.from_shape(w.params)
    keys = ctx.keygen(w.seed_keys)
    model = ctx.model_prepare(W, b)
    pt = ctx.encode_features(torch.from_numpy(X).cuda())
    pool = ctx.encrypt(keys, pt.reshape(-1, N), seed=w.seed_enc).reshape(len(X), model.K, 2, L, N)
    del pt

    def inputs(k, n):
        i0 = (k * 131) % (len(X) - n + 1)
        return pool[i0:i0 + n]

    # the client's side when it is in the measured latency: encrypt the request's rows at arrival
    # and decrypt + decode its outputs right after the product, on the launch's stream. A real
    # client encrypts on its own machine; simulated on the server's GPU, its encryption runs on a
    # high-priority stream of its own so that it does not queue behind the CTAs of the server's
    # large products, and the launch waits for the event recorded after it
    Xdev = torch.from_numpy(X).cuda()
    lo_pri, hi_pri = torch.cuda.Stream.priority_range()
    client_stream = torch.cuda.Stream(priority=min(lo_pri, hi_pri))

    def client_inputs(k, n):
        i0 = (k * 131) % (len(X) - n + 1)
        with torch.cuda.stream(client_stream):
            ptk = ctx.encode_features(Xdev[i0:i0 + n])
            ct = ctx.encrypt(keys, ptk.reshape(-1, N), seed=w.seed_enc + k, obj0=0).reshape(n, model.K, 2, L, N)
            ev = torch.cuda.Event()
            ev.record(client_stream)
        return ct, ev

    def client_decrypt(r, out):
        return ctx.decode(ctx.decrypt(keys, out))

    # warm-up: one fused launch and one single request
    ctx.lr_scores_packed_multi(keys, model, [pool[:1], pool[1:17]])
    ctx.lr_scores_packed(keys, model, pool[:1])
    torch.cuda.synchronize()
    # one large cached block, so that the trace's allocations (workspaces, the simulated clients'
    # ciphertexts) are carved from PyTorch's cache instead of cudaMalloc / cudaFree calls that
    # would synchronise the device in the middle of a trace
    warm = torch.empty(96 << 30, dtype=torch.uint8, device="cuda")
    del warm
    results = {}
    for rate in [float(r) for r in args.rates.split(",")]:
        trace, offered = [], 0
        for t, n in synth.poisson_arrivals(501, rate, 100000):
            if offered >= args.serve_cap:
                break
            trace.append((t, n))
            offered += n
        srv = serve.Server(ctx, keys, model, hbm_budget_bytes=64 << 30, n_streams=2)
        batched = serve.latency_report(srv.run(trace, inputs), model.nY)
        batched.update(launches=srv.nbatches, max_concurrent=srv.max_concurrent)
        srv = serve.Server(ctx, keys, model, hbm_budget_bytes=64 << 30, n_streams=2, small_pairs=16 * model.nY)
        split = serve.latency_report(srv.run(trace, inputs), model.nY)
        split.update(launches=srv.nbatches, max_concurrent=srv.max_concurrent)
        single = serve.latency_report(serve.run_unbatched(ctx, keys, model, trace, inputs), model.nY)
        # the same with the client's encryption and decryption inside each request's latency
        srv = serve.Server(ctx, keys, model, hbm_budget_bytes=64 << 30, n_streams=2, small_pairs=16 * model.nY,
                           post=client_decrypt)
        done = srv.run(trace, client_inputs)
        split_e2e = serve.latency_report(done, model.nY)
        split_e2e.update(launches=srv.nbatches, max_concurrent=srv.max_concurrent)
        for r in done[:3]:                            # spot-check the decrypted scores
            i0 = (r.rid * 131) % (len(X) - r.nX + 1)
            got = bfv.unpack_packed_scores(N, r.result.cpu().numpy(), r.nX, model.nY)
            if not np.array_equal(got, (X[i0:i0 + r.nX].astype(np.int64) @ W + b[None, :]) % w.params.t):
                raise SystemExit("served scores are wrong")
        single_e2e = serve.latency_report(serve.run_unbatched(ctx, keys, model, trace, client_inputs,
                                                              post=client_decrypt), model.nY)
        results[str(rate)] = {"offered_req_per_s": rate, "batched": batched, "batched_priority": split,
                              "one_by_one": single, "batched_priority_client_e2e": split_e2e,
                              "one_by_one_client_e2e": single_e2e}
        print(json.dumps({"rate": rate, "batched": batched, "batched_priority": split, "one_by_one": single,
                          "batched_priority_client_e2e": split_e2e, "one_by_one_client_e2e": single_e2e}),
              flush=True)
    print(json.dumps({"case": "serve", "workload": "batch512-40k model, Poisson arrivals (70% x1, 30% x16..512)",
                      "results": results}), flush=True)
    return 0


def run_serve_bank(args):
    """Serving the paper's bank of one-vs-rest binary models (Section 4.2.1): 11 models with 2
    classes each and their own feature counts (seeded draws from {5k, 10k, 20k, 40k}) at
    N = 16384. Every Poisson arrival (70% one individual, 30% 16..512) queries all 11 models;
    the server fuses requests across models (priority class for requests of <= 16 individuals)
    against the same requests served one at a time. Latency of an arrival = until its last
    model's scores are done."""
    import torch
    import paper_2204_05496_gb300 as bfv
    from paper_2204_05496_gb300 import serve
    bfv.build()
    torch.cuda.set_device(0)
    w = synth.WORKLOADS[WORKLOAD]
    X, _, _ = synth.workload_inputs(w)
    N, L = w.params.N, w.params.L
    ctx = bfv.Context.from_shape(w.params)
    keys = ctx.keygen(w.seed_keys)
    rng = np.random.default_rng([503, 1])
    fs = [int(v) for v in rng.choice([5000, 10000, 20000, 40000], size=11)]
    bank = [ctx.model_prepare(synth.weights(503 + m, f, 2), synth.bias(503 + m, 2)) for m, f in enumerate(fs)]
    pt = ctx.encode_features(torch.from_numpy(X).cuda())
    pool = ctx.encrypt(keys, pt.reshape(-1, N), seed=w.seed_enc).reshape(len(X), -1, 2, L, N)
    del pt
    trace_of = {}

    def inputs(k, n):
        i0, m = trace_of[k]
        return pool[i0:i0 + n, :bank[m].K]      # model m reads the first ceil(f_m / N) plaintexts

    ctx.lr_scores_packed_models(keys, bank[:2], [pool[:1, :bank[0].K], pool[1:17, :bank[1].K]])
    torch.cuda.synchronize()
    results = {}
    for rate in [float(r) for r in args.rates.split(",")]:
        trace, offered = [], 0
        for a, (t, n) in enumerate(synth.poisson_arrivals(502, rate, 100000)):
            if offered >= args.serve_cap:
                break
            i0 = (a * 131) % (len(X) - n + 1)
            for m in range(11):
                trace_of[len(trace)] = (i0, m)
                trace.append((t, n, m))
            offered += n
        out = {}
        for mode, kw in (("batched_priority", dict(small_pairs=16 * 2)), ("batched", {})):
            srv = serve.Server(ctx, keys, bank, hbm_budget_bytes=64 << 30, n_streams=2, **kw)
            done = srv.run(trace, inputs)
            out[mode] = bank_report(done, srv.nbatches)
            torch.cuda.empty_cache()
        out["one_by_one"] = bank_report(serve.run_unbatched(ctx, keys, bank, trace, inputs), None)
        results[str(rate)] = out
        print(json.dumps({"rate": rate, **out}), flush=True)
    print(json.dumps({"case": "serve-bank", "models": 11, "features": fs,
                      "workload": "11 binary models, every arrival queries all (70% x1, 30% x16..512)",
                      "results": results}), flush=True)
    return 0


def bank_report(done, launches):
    """Per-arrival latency (until the last of its 11 model requests is done) and throughput."""
    by_arrival = {}
    for r in done:
        key = (r.t_arrival, r.rid // 11)
        lat = r.t_done - r.t_arrival
        prev = by_arrival.get(key)
        by_arrival[key] = (max(prev[0], lat) if prev else lat, r.nX)
    lat = np.array([v[0] for v in by_arrival.values()])
    single = np.array([v[0] for v in by_arrival.values() if v[1] == 1])
    span = max(r.t_done for r in done) - min(r.t_arrival for r in done)
    preds = sum(v[1] for v in by_arrival.values())
    out = {"arrivals": len(by_arrival), "predictions_x11_models": preds,
           "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "single_p50_ms": float(np.percentile(single, 50) * 1e3) if len(single) else None,
           "single_p99_ms": float(np.percentile(single, 99) * 1e3) if len(single) else None,
           "patients_per_s": preds / span if span > 0 else 0.0}
    if launches is not None:
        out["launches"] = launches
    return out


def run_autotune_save(args):
    """The autotuner on the benchmark's two packed products (one individual, 16 pairs; 512
    individuals, 8,192 pairs) at N = 16384, L = 7; writes the chosen schedules to a schedule file
    (the package reads paper_2204_05496_gb300/schedules.json at context creation)."""
    import torch
    import paper_2204_05496_gb300 as bfv
    bfv.build()
    torch.cuda.set_device(0)
    w = synth.WORKLOADS[WORKLOAD]
    X, W, b = synth.workload_inputs(w)
    N, L = w.params.N, w.params.L
    ctx = bfv.Context.from_shape(w.params)
    keys = ctx.keygen(w.seed_keys)
    model = ctx.model_prepare(W, b)
    out = {}
    for n in (1, 512):
        pt = ctx.encode_features(torch.from_numpy(X[:n]).cuda())
        X_ct = ctx.encrypt(keys, pt.reshape(-1, N), seed=w.seed_enc).reshape(n, model.K, 2, L, N)
        ws = torch.empty(ctx.packed_workspace(model, n, 16384 if n > 1 else 16), dtype=torch.uint8, device="cuda")
        best, ms = ctx.autotune_packed_schedule(keys, model, X_ct, ws)
        out[n] = {"schedule": best.as_dict(), "ms": round(ms, 3)}
        del ws, X_ct, pt
        torch.cuda.empty_cache()
    ctx.save_schedules(args.autotune_save, [n * model.nY for n in (1, 512)])
    print(json.dumps({"case": "autotune-save", "file": args.autotune_save, "tuned": out}), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.serve_bank:
        return run_serve_bank(args)
    if args.serve:
        return run_serve(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.only_packed:
        return run_only_packed(args)
    if args.uneven:
        return run_uneven(args)
    if args.paper8k:
        return run_paper8k(args)
    if args.only_standard:
        return run_only_standard(args)
    if args.autotune_save:
        return run_autotune_save(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
