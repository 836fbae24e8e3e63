"""Benchmark of the chunked DAS chain on the paper-scale stream.

Workload (one "step"): 6,000 channels x 60 s at 1.5 kHz, float32, pushed as 60
chunks of 1,500 samples through the whole chain -- order-8 Butterworth bandpass
0.5-100 Hz (8 SOS), 9-channel spatial mean, STA/LTA 150/3000 samples -- with
the ratio written to device memory.  The input (2.16 GB) and output stay
resident in HBM; a step re-pushes the same recording as a continuation of the
stream (the state keeps carrying), so every step does identical work on inputs
larger than L2.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores instead (the reference arm; there is no published GPU code).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "channel-samples/s of chunked filter chain (device-timed), % of HBM roofline"
UNIT = "channel-samples/s"
# GB300 HBM3e nominal bandwidth, quoted beside the measured copy peak
NOMINAL_HBM_GBS = 7900.0
# channel-tile groups pushed on the chain's own streams (filark_chain_set_lanes);
# each step's outputs are joined into the timing stream at the step's end
LANES = 2
# a push is cut into launches of at most this many samples
# (filark_chain_set_launch_samples); with pushes enqueued back to back, one
# launch per push and lane is fastest here (1,024-sample launches in three
# lanes: 94.9 against 85.6 us per push)
LAUNCH_SAMPLES = 2048


def workload():
    from paper_2605_20132_gb300 import synth
    w = dict(synth.PAPER_SCALE)
    return w


def algorithmic_bytes_per_push(C: int, T: int, S: int, ns: int, nl: int) -> int:
    """Bytes one push must move at minimum: input, ratio output, the cf values
    written to the history ring, the exiting cf values read back from it
    (min(T, nl) + min(T, ns) per channel), and the carried state (IIR state in
    FP64 and the detector sums, read and written)."""
    per_ch = 4 * T + 4 * T + 4 * min(T, nl) + 4 * (min(T, nl) + min(T, ns))
    state = 2 * (8 * 2 * S + 8 * 4)
    return C * (per_ch + state)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons.  Start it before
    the warm-up (nvidia-smi takes a moment to print its first line) and mark
    the timed region with begin()/end(): the summary keeps the samples that
    arrived inside it (host receive time)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[tuple[float, str]] = []
        self._t = None
        self.t_begin = None
        self.t_end = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.PERIOD_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def begin(self):
        self.t_begin = time.perf_counter()

    def end(self):
        self.t_end = time.perf_counter()

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self._t:
                self._t.join(timeout=2)
        return False

    def summary(self) -> dict:
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        lo = self.t_begin if self.t_begin is not None else -float("inf")
        # a line can lag its sample by up to one period
        hi = (self.t_end + self.PERIOD_MS / 1e3) if self.t_end is not None else float("inf")
        for t, ln in self.lines:
            if not (lo <= t <= hi):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm), "period_ms": self.PERIOD_MS}


def measured_peak_hbm() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------ oracle timing --

def oracle_run(x: np.ndarray, sos, K: int, ns: int, nl: int, T: int, n_push: int, threads: int,
               c_lo: int = 0, c_hi: int | None = None) -> float:
    """Run the FP64 oracle (unmodified) over channels [c_lo, c_hi) of x for
    n_push pushes of T samples, split into contiguous channel groups, one
    oracle chain per host thread (each with its own halo).  Returns seconds."""
    import concurrent.futures as cf
    import ctypes as ct

    import oracle
    N, C = x.shape
    c_hi = C if c_hi is None else c_hi
    h = (K - 1) // 2
    span = c_hi - c_lo
    groups = [(c_lo + span * i // threads, c_lo + span * (i + 1) // threads) for i in range(threads)]
    lib, pre = oracle._load(False)
    push = getattr(lib, pre + "chain_push")

    def work(g):
        a, b = g
        lo, hi = max(0, a - h), min(C, b + h)
        ch = oracle.Chain(hi - lo, sos, K, ns, nl)
        out = np.empty((T, hi - lo), dtype=np.float64)
        base = x.ctypes.data
        for p in range(n_push):
            ptr = ct.cast(base + 4 * ((p * T) * C + lo), ct.POINTER(ct.c_float))
            rc = push(ch._h, ptr, C, T, None, None, out.ctypes.data_as(ct.POINTER(ct.c_double)), hi - lo)
            assert rc == 0
        return None

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(work, groups))
    return time.perf_counter() - t0


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    import oracle
    w = workload()
    from paper_2605_20132_gb300 import synth
    x = synth.paper_scale_stream(w["n_channels"], w["n_samples"], w["seed"])
    sos = oracle.butter_bandpass(w["order"], *w["band"], w["fs"])
    C, T = w["n_channels"], w["chunk"]
    cores = host_cores()
    n_push = 6          # one step: every channel, 6 pushes of 1,500 samples
    for _ in range(args.warmup):
        oracle_run(x, sos, w["spatial_width"], w["sta"], w["lta"], T, n_push, cores)
    secs = [oracle_run(x, sos, w["spatial_width"], w["sta"], w["lta"], T, n_push, cores)
            for _ in range(args.steps)]
    total = sum(secs)
    units = C * T * n_push * args.steps
    value = units / total
    sample = f"{C} channels x {n_push} pushes of {T} samples per step, FP64 oracle, {cores} threads"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["name"], "channels": C, "fs": w["fs"],
                                        "chunk": T, "sections": w["order"], "spatial_width": w["spatial_width"],
                                        "sta": w["sta"], "lta": w["lta"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU timing --

def max_over_ranks(value: float, dist, device=None) -> float:
    """The slowest rank's time (every rank gets it); the value itself when
    running alone."""
    if not dist:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling:
    every rank runs its own replica of the workload)."""
    return units_per_rank * world / seconds

def run_gpu(args, rank: int, world: int, dist) -> None:
    import ctypes as ct

    import torch

    from paper_2605_20132_gb300 import abi, synth
    from paper_2605_20132_gb300.chain import Chain, butter_bandpass

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload()
    C, N, T = w["n_channels"], w["n_samples"], w["chunk"]
    K, ns, nl = w["spatial_width"], w["sta"], w["lta"]
    n_push = N // T
    x_host = synth.paper_scale_stream(C, N, w["seed"])
    sos = butter_bandpass(w["order"], *w["band"], w["fs"])
    S = sos.shape[0]
    lib = abi.load()
    chain = Chain(C, sos, w["fs"], K, ns, nl, outputs=abi.FILARK_OUT_RATIO, max_chunk=T, device=local)
    chain.set_lanes(LANES)
    chain.set_launch_samples(LAUNCH_SAMPLES)
    info = chain.info()
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    xd = torch.from_numpy(x_host).to(dev)
    rd = torch.empty((N, C), dtype=torch.float32, device=dev)
    push = lib.filark_chain_push_chunk
    join = lib.filark_chain_join
    h = chain._h
    row = 4 * C
    xp, rp = xd.data_ptr(), rd.data_ptr()
    ptrs = [(xp + i * T * row, rp + i * T * row) for i in range(n_push)]

    def step():
        for xi, ri in ptrs:
            st = push(h, xi, C, T, ri, None, None, C, sh)
            if st:
                abi.check(st, "push")
        # every push of the step is complete on `stream` after this
        st = join(h, sh)
        if st:
            abi.check(st, "join")

    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    with sampler:
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        sampler.begin()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        ev1.synchronize()
        sampler.end()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    abi.check(abi.filark_chain_sync_status(h, sh), "sync")
    launches_per_push = -(-T // LAUNCH_SAMPLES)
    lanes = min(LANES, -(-C // info["tile_channels"]))
    launches = args.steps * n_push * launches_per_push * lanes
    value = whole_job_rate(C * N * args.steps, world, ms / 1e3)

    # ---- end to end through the host-buffer entry point (pinned host memory),
    # in the same lanes as the timed region
    e2e_steps = max(1, min(args.steps, 3))
    xh = torch.from_numpy(x_host).pin_memory()
    rh = torch.empty((N, C), dtype=torch.float32).pin_memory()
    push_h = lib.filark_chain_push_host_async
    xhp, rhp = xh.data_ptr(), rh.data_ptr()

    def step_host():
        # pipelined: the copies of one push overlap the computation of the
        # neighbouring pushes; the step ends when every ratio row is in host memory
        for i in range(n_push):
            st = push_h(h, xhp + i * T * row, C, T, rhp + i * T * row, None, None, C, sh)
            if st:
                abi.check(st, "push_host_async")
        abi.check(lib.filark_chain_host_sync(h, sh), "host_sync")

    step_host()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step_host()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e_value = whole_job_rate(C * N * e2e_steps, world, e2e_s)

    # ---- the same pushes in one lane: each push complete on `stream` when
    # its launch ends (the stream-ordered mode, the API's default)
    chain.set_lanes(1)
    so_steps = max(3, min(args.steps, 20))
    with torch.cuda.stream(stream):
        for _ in range(3):
            step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(so_steps):
        step()
    ev3.record(stream)
    ev3.synchronize()
    ms_so = max_over_ranks(ev2.elapsed_time(ev3), dist, dev)
    so_value = whole_job_rate(C * N * so_steps, world, ms_so / 1e3)

    chain.close()
    link = host_link_rates(xh, rh, C * T)

    if rank != 0:
        return
    # ---- roofline of the (only) kernel
    bytes_push = algorithmic_bytes_per_push(C, T, S, ns, nl)
    # the lanes' launches overlap: achieved = algorithmic bytes of every push
    # of the timed region / the timed region (= bytes per push / time per push)
    ms_push = ms / (args.steps * n_push)
    achieved = bytes_push / (ms_push / 1e3) / 1e9
    ms_push_so = ms_so / (so_steps * n_push)
    peak, peak_kind = measured_peak_hbm()
    traffic = None
    tp = os.path.join(ROOT, "profiles", "chain_fwd_paper_scale_traffic.json")
    if os.path.exists(tp):
        try:
            with open(tp) as f:
                tj = json.load(f)
            if (tj.get("kernel_source_sha") == kernel_sha() and tj.get("lanes") == lanes
                    and tj.get("launch_samples") == LAUNCH_SAMPLES):
                traffic = tj.get("dram_bytes_per_push")
        except (OSError, ValueError):
            traffic = None

    # ---- CPU baseline: the oracle on the host cores, bounded sample
    cores = host_cores()
    cpu_push = 6
    cpu_s = oracle_run(x_host, sos, K, ns, nl, T, cpu_push, cores)
    cpu_value = C * T * cpu_push / cpu_s

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {
            "workload": w["name"], "channels": C, "samples_per_step": N, "fs": w["fs"], "chunk": T,
            "pushes_per_step": n_push, "sections": S, "spatial_width": K, "sta": ns, "lta": nl,
            "precision": {1: "modal32", 2: "dense64", 3: "all32"}.get(info["precision"], "?"),
            "l2": "inputs larger than L2 (2.16 GB per step)", "parallelism": "replicas" if world > 1 else "1 GPU",
            "lanes": lanes, "launch_samples": LAUNCH_SAMPLES,
            "completion": "each step's 60 pushes complete on the timing stream at the step's end (filark_chain_join)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "traffic_source": ("ncu DRAM read + write of one push, profiles/chain_fwd_paper_scale_traffic.json "
                                        "(taken on this kernel source; not measured in this run)")
                     if traffic is not None else "no capture on this kernel source",
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "unit_of_work": f"one push of {T} x {C} ({lanes * launches_per_push} launches: "
                                     f"{launches_per_push} per lane, the lanes overlapping)",
                     "bytes_per_push": bytes_push, "ms_per_push": ms_push},
        "stream_ordered": {"value": so_value, "unit": UNIT, "lanes": 1, "steps": so_steps,
                           "ms_per_push": ms_push_so,
                           "frac": bytes_push / (ms_push_so / 1e3) / 1e9 / peak,
                           "note": "every push complete on its stream when its launch ends"},
        "cpu_baseline": {"value": cpu_value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{C} channels x {cpu_push} pushes of {T} samples, FP64 oracle, {cores} threads"},
        "e2e": {"value": e2e_value, "unit": UNIT, "lanes": lanes, "h2d_bytes_per_step": 4 * C * N,
                "d2h_bytes_per_step": 4 * C * N,
                # the host link's own rates on this machine, measured right after:
                # the pipelined e2e moves 4 B in and 4 B out per channel-sample
                "host_link_gbs": link,
                "link_bound": link["both"] * 1e9 / 8.0,
                "frac_of_link_bound": e2e_value / (link["both"] * 1e9 / 8.0)},
        "gpu_launches": launches,
        "clocks": sampler.summary(),
    }
    print(json.dumps(line), flush=True)


def kernel_sha() -> str:
    import hashlib
    hsh = hashlib.sha256()
    for f in ("chain_body.cuh", "chain_kernel.cu", "filark_internal.h"):
        with open(os.path.join(ROOT, "paper_2605_20132_gb300", "csrc", f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()[:16]


def host_link_rates(xh, rh, n: int) -> dict:
    """Copy-engine rates between page-locked host memory and the device for
    pushes of n floats: H2D alone, D2H alone, both directions at once
    (GB/s, 8 copies each)."""
    import torch
    d1 = torch.empty(n, device="cuda")
    d2 = torch.empty(n, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    src, dst = xh.view(-1), rh.view(-1)
    k = max(1, min(8, src.numel() // n))

    def run(h2d, d2h):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(k):
            if h2d:
                with torch.cuda.stream(s1):
                    d1.copy_(src[i * n:(i + 1) * n], non_blocking=True)
            if d2h:
                with torch.cuda.stream(s2):
                    dst[i * n:(i + 1) * n].copy_(d2, non_blocking=True)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    run(True, True)
    b = 4.0 * n * k
    return {"h2d": b / run(True, False) / 1e9, "d2h": b / run(False, True) / 1e9,
            "both": 2 * b / run(True, True) / 1e9}


# ------------------------------------------------- other workloads (lines) --

def _event_ms(fn, reps: int, stream=None) -> float:
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def run_batch_workload(args) -> None:
    """32 independent streams (500..10,000 channels, 200..3,000 samples per
    push, drawn per stream and push) through one persistent launch per push,
    after the autotuner picked the launch geometry; against the same pushes
    made stream by stream through single-stream chains."""
    import torch

    from paper_2605_20132_gb300 import abi, synth
    from paper_2605_20132_gb300.chain import Batch, Chain, butter_bandpass
    cfg = synth.BATCH
    specs = synth.batch_streams(cfg["seed"], cfg["n_streams"], cfg["channels"], cfg["chunk"])
    Cs = [s["n_channels"] for s in specs]
    P = 6
    T = synth.batch_chunk_lengths(cfg["seed"], cfg["n_streams"], P, cfg["chunk"])
    sos = butter_bandpass(cfg["order"], *cfg["band"], cfg["fs"])
    K, ns, nl = cfg["spatial_width"], cfg["sta"], cfg["lta"]
    tot = T.sum(axis=0)
    g = torch.Generator(device="cuda").manual_seed(cfg["seed"])
    xs = [torch.randn((int(tot[i]), C), device="cuda", generator=g) for i, C in enumerate(Cs)]
    rs = [torch.empty_like(x) for x in xs]
    offs = np.vstack([np.zeros((1, len(Cs)), dtype=np.int64), np.cumsum(T, axis=0)])
    views = [[(xs[i][offs[p, i]:offs[p + 1, i]], rs[i][offs[p, i]:offs[p + 1, i]]) for i in range(len(Cs))]
             for p in range(P)]
    b = Batch(Cs, sos, cfg["fs"], K, ns, nl, outputs=abi.FILARK_OUT_RATIO, max_chunk=cfg["chunk"][1])
    info = b.tune([v[0] for v in views[0]], ratios=[v[1] for v in views[0]], timed_pushes=3)

    def step_batch():
        for p in range(P):
            b.push([v[0] for v in views[p]], ratios=[v[1] for v in views[p]])

    for _ in range(max(args.warmup, 3)):
        step_batch()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    with sampler:
        ms = _event_ms(step_batch, args.steps)
    b.sync()
    b.close()
    chains = [Chain(C, sos, cfg["fs"], K, ns, nl, outputs=abi.FILARK_OUT_RATIO, max_chunk=cfg["chunk"][1])
              for C in Cs]

    def step_single():
        for p in range(P):
            for i in range(len(Cs)):
                chains[i].push(views[p][i][0], ratio=views[p][i][1])

    for _ in range(3):
        step_single()
    ms_single = _event_ms(step_single, args.steps)
    for c in chains:
        c.close()
    units = float((T * np.array(Cs)[None, :]).sum())
    byts = float(sum(algorithmic_bytes_per_push(Cs[i], int(T[p, i]), sos.shape[0], ns, nl)
                     for p in range(P) for i in range(len(Cs))))
    peak, peak_kind = measured_peak_hbm()
    achieved = byts / (ms / 1e3) / 1e9
    line = {
        "workload": cfg["name"], "metric": "channel-samples/s of batched pushes (device-timed)",
        "value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": args.steps, "pushes_per_step": P,
        "single_stream": {"value": units / (ms_single / 1e3), "unit": UNIT, "ms_per_step": ms_single,
                          "launches_per_step": int(sum(-(-int(t) // 2048) for t in T.ravel() if t))},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind},
        "tuner": {"cluster": info["cluster"], "n_clusters": info["n_clusters"],
                  "blocks_per_cta": info["blocks_per_cta"], "use_graph": info["use_graph"],
                  "stream_path_ms": info["stream_ms"], "candidates": info["tuned"]},
        "gpu_launches": args.steps * P, "dtype": "f32", "data": "synthetic N(0,1) noise generated on the device",
        "config": {"streams": len(Cs), "channels": int(sum(Cs)), "chunk_range": list(cfg["chunk"]),
                   "sections": int(sos.shape[0]), "spatial_width": K, "sta": ns, "lta": nl},
        "clocks": sampler.summary(),
    }
    print(json.dumps(line), flush=True)


# warp instructions executed by one forward + backward of the adjoint workload
# (2,048 ch x 30,000 samples, order-4 bandpass, checkpoints every 3,000),
# summed over its kernels from one ncu capture
ADJOINT_WARP_INSTRUCTIONS = 2.653e9


def run_adjoint_workload(args) -> None:
    """Forward with checkpoints + reverse-time adjoint through the order-4
    bandpass on 2,048 channels x 30,000 samples (checkpoints every 3,000),
    against the chain's plain forward bandpass on the same record."""
    import torch

    from paper_2605_20132_gb300 import abi, synth
    from paper_2605_20132_gb300.chain import Chain, butter_bandpass
    cfg = synth.ADJOINT
    C, N, ck = cfg["n_channels"], cfg["n_samples"], cfg["checkpoint"]
    sos = butter_bandpass(cfg["order"], *cfg["band"], cfg["fs"])
    S = sos.shape[0]
    x = torch.from_numpy(synth.adjoint_stream(C, N, cfg["seed"])).cuda()
    gy = torch.randn_like(x)
    nb, wb = abi.filark_iir_ckpt_bytes(S, C, N, ck), abi.filark_iir_work_bytes(S, C, N, ck)
    ckb = torch.empty(nb, dtype=torch.uint8, device="cuda")
    wk = torch.empty(wb, dtype=torch.uint8, device="cuda")
    y, gx = torch.empty_like(x), torch.empty_like(x)
    gs = torch.empty((S, 6), dtype=torch.float64, device="cuda")
    sh = torch.cuda.current_stream().cuda_stream

    def fwd():
        abi.check(abi.filark_iir_forward_ckpt(sos, S, C, x.data_ptr(), C, N, y.data_ptr(), C, ck, ckb.data_ptr(),
                                              nb, sh), "forward")

    def bwd():
        abi.check(abi.filark_iir_backward(sos, S, C, x.data_ptr(), C, N, gy.data_ptr(), C, ck, ckb.data_ptr(), nb,
                                          wk.data_ptr(), wb, gx.data_ptr(), C, gs.data_ptr(), sh), "backward")

    def both():
        fwd()
        bwd()

    chain = Chain(C, sos, cfg["fs"], 1, 0, 0, outputs=abi.FILARK_OUT_BANDPASS, max_chunk=ck)

    def plain():
        for t in range(0, N, ck):
            chain.push(x[t:t + ck], bandpass=y[t:t + ck])

    for f in (fwd, bwd, plain):
        for _ in range(3):
            f()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    with sampler:
        ms_both = _event_ms(both, args.steps)
    ms_fwd = _event_ms(fwd, args.steps)
    ms_bwd = _event_ms(bwd, args.steps)
    ms_plain = _event_ms(plain, args.steps)
    chain.close()
    units = C * N
    clocks = sampler.summary()
    # FP32-issue roofline: the warp instructions of one forward + backward
    # (ncu smsp__inst_executed.sum summed over its kernels on this workload)
    # over the timed forward + backward, against one instruction per cycle on
    # all 4 schedulers of the 152 SMs at the sampled SM clock
    mhz = clocks.get("sm_mhz") or 2070.0
    peak_ginst = 4 * 152 * mhz / 1e3
    got_ginst = ADJOINT_WARP_INSTRUCTIONS / (ms_both / 1e3) / 1e9
    line = {
        "workload": cfg["name"], "metric": "channel-samples/s of forward + adjoint (device-timed)",
        "value": units / (ms_both / 1e3), "unit": UNIT, "ms_per_step": ms_both, "steps": args.steps,
        "forward_ckpt_ms": ms_fwd, "backward_ms": ms_bwd,
        "plain_forward": {"value": units / (ms_plain / 1e3), "unit": UNIT, "ms": ms_plain,
                          "what": "chain bandpass only, FP32 block scan, pushes of 3,000"},
        "memory": {"checkpoint_bytes": nb, "work_bytes": wb, "all_intermediates_fp64_bytes": 8 * S * C * N},
        "dtype": "f32x2 (double-float)", "data": "synthetic noise + Ricker events (seeded)",
        "config": {"channels": C, "samples": N, "sections": S, "checkpoint": ck},
        "roofline": {"bound": "alu", "achieved": got_ginst, "peak": peak_ginst,
                     "unit": "G warp instructions/s (FP32 issue)", "frac": got_ginst / peak_ginst,
                     "instructions": ADJOINT_WARP_INSTRUCTIONS,
                     "instructions_source": "ncu smsp__inst_executed.sum of one forward + backward, "
                                            "profiles/iir_adjoint_2048x30000.md"},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_precision_workload(args) -> None:
    """The precision-stress shape: order-8 Butterworth 0.01-1 Hz at 1.5 kHz
    (poles within 1e-4 of z = 1) on 10,000 channels, pushes of 1,500 samples,
    bandpass output (N(0,1) noise plus a 0.05 Hz sine generated on the device,
    16 pushes = 960 MB per step, larger than L2).  The planner's choice (the
    dense double-float carry for this filter) against the modal FP32 carry and the
    all-FP32 carry forced on the same filter; their accuracy over the whole
    600 s record is in profiles/precision_stress_10000ch_600s.md."""
    import torch

    from paper_2605_20132_gb300 import abi, synth
    from paper_2605_20132_gb300.chain import Chain, butter_bandpass
    cfg = synth.PRECISION
    C, T, P = cfg["n_channels"], cfg["chunk"], 16
    sos = butter_bandpass(cfg["order"], *cfg["band"], cfg["fs"])
    g = torch.Generator(device="cuda").manual_seed(cfg["seed"])
    x = torch.randn((T * P, C), device="cuda", generator=g)
    t = torch.arange(T * P, device="cuda", dtype=torch.float64).unsqueeze(1) / cfg["fs"]
    ph = torch.rand((1, C), device="cuda", generator=g, dtype=torch.float64) * 2 * np.pi
    x += (cfg["sine_amp"] * torch.sin(2 * np.pi * cfg["sine_hz"] * t + ph)).float()
    del t
    y = torch.empty_like(x)
    peak, peak_kind = measured_peak_hbm()
    rows = []
    for name, prec in [("planner", abi.FILARK_PREC_AUTO), ("modal32", abi.FILARK_PREC_MODAL32),
                       ("all32", abi.FILARK_PREC_ALL32)]:
        try:
            ch = Chain(C, sos, cfg["fs"], 1, 0, 0, outputs=abi.FILARK_OUT_BANDPASS, precision=prec, max_chunk=T)
        except abi.FilarkError as e:
            rows.append({"mode": name, "unavailable": str(e)})
            continue
        mode = {1: "modal32", 2: "dense64", 3: "all32"}.get(ch.info()["precision"], "?")

        def step():
            for i in range(P):
                ch.push(x[i * T:(i + 1) * T], bandpass=y[i * T:(i + 1) * T])

        for _ in range(max(args.warmup, 3)):
            step()
        ms = _event_ms(step, args.steps)
        ch.close()
        # input read + bandpass written + the carried state read and written
        byts = 8.0 * C * T * P + 2 * 2 * 8.0 * 2 * sos.shape[0] * C * P
        rows.append({"mode": name, "carry": mode, "channel_samples_per_s": C * T * P / (ms / 1e3),
                     "us_per_push": 1e3 * ms / P, "frac_of_hbm": byts / (ms / 1e3) / 1e9 / peak})
    print(json.dumps({
        "workload": "precision-stress-10000ch-1500Hz", "metric": "channel-samples/s of the bandpass (device-timed)",
        "rows": rows, "peak_gbs": peak, "peak_kind": peak_kind, "steps": args.steps, "pushes_per_step": P,
        "dtype": "f32 scan, carries as named", "data": "synthetic N(0,1) + 0.05 Hz sine on the device",
        "config": {"channels": C, "chunk": T, "fs": cfg["fs"], "sections": int(sos.shape[0]),
                   "band": list(cfg["band"])}}), flush=True)


def run_trigger_workload(args) -> None:
    """Triggers (hysteresis 6 / 2) on the paper-scale chain's ratio, 60 pushes
    of 1,500 samples x 6,000 channels, and the event merge of all of them."""
    import torch

    from paper_2605_20132_gb300 import abi, synth
    from paper_2605_20132_gb300.chain import Chain, Trigger, butter_bandpass, merge_events
    w = workload()
    C, N, T = w["n_channels"], w["n_samples"], w["chunk"]
    x = torch.from_numpy(synth.paper_scale_stream(C, N, w["seed"])).cuda()
    r = torch.empty_like(x)
    ch = Chain(C, butter_bandpass(w["order"], *w["band"], w["fs"]), w["fs"], w["spatial_width"], w["sta"],
               w["lta"], outputs=abi.FILARK_OUT_RATIO, max_chunk=T)
    for t in range(0, N, T):
        ch.push(x[t:t + T], ratio=r[t:t + T])
    ch.sync()
    ch.close()
    tr = Trigger(C, 6.0, 2.0, max_chunk=T, capacity=1 << 22)

    def step():
        tr.reset()
        for t in range(0, N, T):
            tr.push(r[t:t + T])
        tr.join()

    # stream-ordered pushes, then the overlap mode (a push's summaries beside
    # the previous push's scan and emission; the step's triggers joined at its end)
    for _ in range(max(args.warmup, 3)):
        step()
    ms_so = _event_ms(step, args.steps)
    tr.set_overlap(True)
    for _ in range(max(args.warmup, 3)):
        step()
    ms = _event_ms(step, args.steps)
    tr.flush()
    n = int(tr.count.item())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, m = merge_events(tr.records, n, C)
    e1.record()
    e1.synchronize()
    ms_merge = e0.elapsed_time(e1)
    tr.close()
    # the chain and the triggers per push, in the benchmark's lanes: a chain
    # push, its lanes joined, then a trigger push -- against the chain push with
    # the trigger summaries fused into its detector (filark_chain_push_triggers)
    sos = butter_bandpass(w["order"], *w["band"], w["fs"])
    cf = Chain(C, sos, w["fs"], w["spatial_width"], w["sta"], w["lta"], outputs=abi.FILARK_OUT_RATIO, max_chunk=T)
    cf.set_lanes(LANES)
    tf = Trigger(C, 6.0, 2.0, max_chunk=T, capacity=1 << 22)

    def step_sep():
        cf.reset()
        tf.reset()
        for t in range(0, N, T):
            cf.push(x[t:t + T], ratio=r[t:t + T])
            cf.join()
            tf.push(r[t:t + T])

    def step_fused():
        cf.reset()
        tf.reset()
        for t in range(0, N, T):
            cf.push_triggers(x[t:t + T], r[t:t + T], tf)
        cf.join()
        tf.join()

    pipe = {}
    for name, fn, ov in (("separate", step_sep, False), ("fused", step_fused, False),
                         ("fused_overlap", step_fused, True)):
        tf.set_overlap(ov)
        for _ in range(3):
            fn()
        pipe[name] = _event_ms(fn, max(1, min(args.steps, 5)))
    cf.close()
    tf.close()
    del x
    peak, peak_kind = measured_peak_hbm()
    byts = 4.0 * C * N   # the ratio is read once; the triggers are a few MB
    achieved = byts / (ms / 1e3) / 1e9
    line = {
        "workload": "trigger-" + w["name"], "metric": "channel-samples/s of trigger extraction (device-timed)",
        "value": C * N / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": args.steps,
        "triggers": n, "events": m, "event_merge_ms": ms_merge, "overlap": True,
        "chain_and_triggers": {k: {"ms_per_step": v, "us_per_push": v / (N // T) * 1e3,
                                   "channel_samples_per_s": C * N / (v / 1e3)} for k, v in pipe.items()},
        "stream_ordered": {"value": C * N / (ms_so / 1e3), "unit": UNIT, "ms_per_step": ms_so,
                           "frac": byts / (ms_so / 1e3) / 1e9 / peak},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "bytes_per_step": byts},
        "gpu_launches": 3 * (N // T) * args.steps, "dtype": "u8/i64 (comparisons, indices)",
        "data": "the paper-scale chain's ratio on synthetic input", "config": {"on": 6.0, "off": 2.0},
    }
    print(json.dumps(line), flush=True)


def run_ops_workload(args) -> None:
    """The other streaming operators on the paper-scale shape (6,000 channels,
    pushes of 1,500 samples at 1.5 kHz; 6 pushes per step, 216 MB of input,
    larger than L2): realtime FIR (101 taps), running mean and AGC (3,000-sample
    window), EMA equalisation, overlap-add FFT bandpass (4,001 taps), and the
    display path (2,048 rows of 3 channels, 10 samples per column, display
    filter = the paper-scale bandpass).  One line per operator."""
    import torch

    from paper_2605_20132_gb300 import abi, synth
    from paper_2605_20132_gb300.chain import FFTFilter, TemporalOp, View, butter_bandpass
    w = workload()
    C, T, P = w["n_channels"], w["chunk"], 6
    g = torch.Generator(device="cuda").manual_seed(9)
    x = torch.randn((T * P, C), device="cuda", generator=g)
    y = torch.empty_like(x)
    peak, peak_kind = measured_peak_hbm()
    sos = butter_bandpass(w["order"], *w["band"], w["fs"])
    # algorithmic bytes per channel-sample: input read + output written, plus
    # the state each operator must read and write per push (FIR history and
    # FFT overlap tail: M - 1 samples per channel each way; running mean/AGC:
    # the double-float prefix written and the exiting prefix read back)
    state = lambda M: 8.0 * (M - 1) / T
    ops = [
        ("fir-101", lambda: TemporalOp(abi.FILARK_TOP_FIR, C, 101,
                                       synth.windowed_sinc_bandpass(101, 5.0, 100.0, w["fs"]), max_chunk=T),
         8 + state(101), 3),
        ("running-mean-3000", lambda: TemporalOp(abi.FILARK_TOP_MEAN, C, 3000, max_chunk=T), 24, 2),
        ("running-agc-3000", lambda: TemporalOp(abi.FILARK_TOP_AGC, C, 3000, max_chunk=T), 24, 2),
        ("ema-equalisation", lambda: TemporalOp(abi.FILARK_TOP_EMA, C, alpha=1e-3, max_chunk=T), 8, 1),
        ("fft-bandpass-4001", lambda: FFTFilter(C, synth.windowed_sinc_bandpass(4001, 0.5, 100.0, w["fs"]),
                                                max_chunk=T), 8 + state(4001), 1),
    ]
    for name, make, bps, launches in ops:
        op = make()

        def step():
            for i in range(P):
                op.push(x[i * T:(i + 1) * T], y[i * T:(i + 1) * T])

        for _ in range(3):
            step()
        ms = _event_ms(step, args.steps)
        op.close()
        achieved = bps * C * T * P / (ms / 1e3) / 1e9
        print(json.dumps({
            "workload": name + "-6000ch-1500", "metric": "channel-samples/s (device-timed)",
            "value": C * T * P / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "bytes_per_channel_sample": bps, "note": "input read + output written + carried state"},
            "gpu_launches": launches * P * args.steps, "dtype": "f32", "data": "synthetic N(0,1) on the device"}),
            flush=True)
    v = View(C, 3, 10, 2048, abi.FILARK_VIEW_PEAK, sos, max_chunk=T)

    def vstep():
        for i in range(P):
            v.push(x[i * T:(i + 1) * T])
        v.image()

    for _ in range(3):
        vstep()
    ms = _event_ms(vstep, args.steps)
    v.close()
    achieved = 4 * C * T * P / (ms / 1e3) / 1e9
    print(json.dumps({
        "workload": "display-path-2000rows-6000ch-1500", "metric": "channel-samples/s (device-timed)",
        "value": C * T * P / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "bytes_per_channel_sample": 4, "note": "input read once"},
        "dtype": "f32", "data": "synthetic N(0,1) on the device",
        "config": {"rows": 2000, "channels_per_row": 3, "samples_per_column": 10, "width": 2048, "mode": "peak",
                   "display_filter": "order-8 0.5-100 Hz bandpass"}}), flush=True)


def run_waves_workload(args) -> None:
    """Grid-fill staircase of the chain kernel: the paper-scale chain (order-8
    bandpass, K = 9, STA/LTA 150/3000) on n x 56 channels (n channel tiles of
    56 outputs, one cluster of time ranges each) for pushes of 1,500 and 2,048
    samples; device time per push over 30 consecutive pushes.  One line per
    push length, with the tile counts at which a new wave of clusters starts
    visible as steps; then the paper-scale chain in 1 to 4 lanes."""
    import torch

    from paper_2605_20132_gb300 import abi
    from paper_2605_20132_gb300.chain import Chain, butter_bandpass
    w = workload()
    sos = butter_bandpass(w["order"], *w["band"], w["fs"])
    tiles = (24, 36, 44, 48, 56, 72, 84, 90, 94, 96, 100, 108, 112, 120, 132, 144)
    n_push = 30
    wout = 56
    for T in (w["chunk"], 2048):
        g = torch.Generator(device="cuda").manual_seed(0)
        x = torch.randn((n_push * T, wout * max(tiles)), device="cuda", generator=g)
        r = torch.empty_like(x)
        rows = []
        for nt in tiles:
            C = wout * nt
            xs, rs = x[:, :C], r[:, :C]
            ch = Chain(C, sos, w["fs"], w["spatial_width"], w["sta"], w["lta"],
                       outputs=abi.FILARK_OUT_RATIO, max_chunk=T)

            def step():
                for t in range(0, n_push * T, T):
                    ch.push(xs[t:t + T], ratio=rs[t:t + T])

            for _ in range(3):
                step()
            ms = _event_ms(step, max(1, min(args.steps, 5)))
            ch.close()
            us = ms / n_push * 1e3
            rows.append({"tiles": nt, "channels": C, "us_per_push": round(us, 2),
                         "channel_samples_per_s": C * T / (us / 1e6)})
        nblk = (T + 31) // 32
        print(json.dumps({"workload": f"chain-grid-fill-T{T}", "metric": "device time per push",
                          "push_samples": T, "ctas_per_cluster": (nblk + 7) // 8, "outputs_per_tile": wout,
                          "rows": rows, "dtype": "f32", "data": "synthetic N(0,1) on the device"}), flush=True)
        del x, r
    # the paper-scale chain in 1-4 lanes and launches of at most 2048, 1024 and
    # 512 samples: 60 pushes, joined at the end
    C, T = w["n_channels"], w["chunk"]
    n_push = 60
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((n_push * T, C), device="cuda", generator=g)
    r = torch.empty_like(x)
    ch = Chain(C, sos, w["fs"], w["spatial_width"], w["sta"], w["lta"], outputs=abi.FILARK_OUT_RATIO, max_chunk=T)
    rows = []
    for launch in (2048, 1024, 512):
        ch.set_launch_samples(launch)
        for lanes in range(1, abi.FILARK_MAX_LANES + 1):
            ch.set_lanes(lanes)

            def lstep():
                for t in range(0, n_push * T, T):
                    ch.push(x[t:t + T], ratio=r[t:t + T])
                ch.join()

            for _ in range(3):
                lstep()
            ms = _event_ms(lstep, max(1, min(args.steps, 5)))
            us = ms / n_push * 1e3
            rows.append({"launch_samples": launch, "lanes": lanes, "us_per_push": round(us, 2),
                         "channel_samples_per_s": C * T / (us / 1e6)})
    # the chain's own autotuner on the same push (enqueued back to back)
    tuned = ch.tune(x[:T], ratio=r[:T], timed_pushes=20)
    ch.close()
    print(json.dumps({"workload": f"chain-lanes-{C}ch-T{T}", "metric": "device time per push", "rows": rows,
                      "tuner": tuned, "dtype": "f32", "data": "synthetic N(0,1) on the device"}), flush=True)


def ncu_case() -> None:
    """Small profiling case for ncu captures: the paper-scale chain on 6,000
    channels in the benchmark's lanes and launch length, 4 pushes
    of 1,500 samples of Gaussian noise (144 MB of input, larger than L2), ratio
    output only."""
    import torch

    from paper_2605_20132_gb300 import abi
    from paper_2605_20132_gb300.chain import Chain, butter_bandpass
    w = workload()
    C, T, n_push = w["n_channels"], w["chunk"], 4
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((T * n_push, C), device="cuda", generator=g)
    r = torch.empty_like(x)
    ch = Chain(C, butter_bandpass(w["order"], *w["band"], w["fs"]), w["fs"], w["spatial_width"], w["sta"],
               w["lta"], outputs=abi.FILARK_OUT_RATIO, max_chunk=T)
    ch.set_lanes(LANES)
    ch.set_launch_samples(LAUNCH_SAMPLES)
    for i in range(n_push):
        ch.push(x[i * T:(i + 1) * T], ratio=r[i * T:(i + 1) * T])
    ch.sync()
    ch.close()
    print("ncu case done")


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="filark", choices=["filark", "reference"])
    ap.add_argument("--ncu-case", action="store_true", help="run the small profiling case only")
    ap.add_argument("--workload", default="chain",
                    choices=["chain", "batch", "adjoint", "trigger", "ops", "waves", "precision"],
                    help="chain: the paper-scale chain (the benchmark line); the others print their own line")
    args = ap.parse_args()
    if args.ncu_case:
        ncu_case()
        return
    if args.workload != "chain":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        {"batch": run_batch_workload, "adjoint": run_adjoint_workload,
         "trigger": run_trigger_workload, "ops": run_ops_workload,
         "waves": run_waves_workload, "precision": run_precision_workload}[args.workload](args)
        return
    args.warmup = max(args.warmup, 3) if args.impl == "filark" else args.warmup
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        if args.impl == "reference":
            dist_mod.init_process_group("gloo")
        else:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            dist_mod.init_process_group("nccl")
        dist = dist_mod
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_gpu(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
