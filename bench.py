"""Benchmark of the MPNL detection path on GB300 (one JSON line on stdout).

A step is one pass of the whole path over one slot of synthetic input:
sorted QR + z = Q^H y, position-vector selection, the N_pe walks with argmin
and max-log LLRs, and the linear MMSE baseline.  Default workload: 16x16
64-QAM, 3276 subcarriers x 14 OFDM symbols (one 0.5 ms slot of the real-time
load), N_pe = 256, i.i.d. Rayleigh, SNR 21 dB.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mpnl|reference]

Multi-GPU (torchrun): every rank detects its own slots (subcarriers are
independent; no collective on the data path), `value` is the total over all
ranks divided by the slowest rank's time ("scaling": "weak").

`--impl reference` times the FP64 CPU oracle (the only reference the paper
allows; it has no code) on the host cores on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2409_14355_gb300 import inputs  # noqa: E402

METRIC = "MIMO detections/s (hard decisions + max-log LLRs, with the MMSE baseline in the same step)"
UNIT = "detections/s"
BITS = {4: 2, 16: 4, 64: 6}
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["mpnl", "reference"], default="mpnl")
    ap.add_argument("--workload", default="16x16-64qam-3276sc")
    ap.add_argument("--n-pe", type=int, default=256)
    ap.add_argument("--snr-index", type=int, default=2)
    ap.add_argument("--ring", type=int, default=16, help="distinct slots cycled through (> L2)")
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--inflight", type=int, default=3,
                    help="slots in flight on their own streams (MMSE on a side stream each); "
                         "three keep the end-to-end path's copies off the critical path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--precision", choices=["fp32", "fp16"], default="fp32",
                    help="walk residuals in FP32 (mpnl_detect) or FP16 (mpnl_detect_mixed)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the N_pe / precision sweep reported beside the main line")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-size persistent batch measured beside the main line")
    ap.add_argument("--mixed-units", type=int, default=64)
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving-loop latency measurement beside the main line")
    ap.add_argument("--serving-rus", type=int, default=200)
    ap.add_argument("--serving-seconds", type=float, default=1.0)
    ap.add_argument("--n-sc", type=int, default=None,
                    help="override the subcarrier count (smaller profiling cases)")
    return ap.parse_args()


def workload_config(args, w):
    return {
        "workload": args.workload, "nr": w["nr"], "nt": w["nt"], "qam": w["qam"],
        "n_sc": w["n_sc"], "n_sym": 14, "n_pe": args.n_pe, "channel": w["channel"],
        "snr_db": w["snrs"][args.snr_index],
    }


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power = [], [], []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# CPU oracle timing (baseline only)
# --------------------------------------------------------------------------
def time_oracle(sl, qam, n_pe, seconds: float, max_sc: int | None = None, n_threads: int = 0,
                keep: list | None = None):
    """Run the oracle on growing prefixes of the slot's subcarriers until one
    run takes >= `seconds` (or the cap is reached).  Returns (dets/s, threads,
    subcarriers, elapsed); the last run's outputs go to `keep` if given.
    n_threads 0 = all host cores."""
    import oracle

    n = 4
    cap = sl.n_sc if max_sc is None else min(max_sc, sl.n_sc)
    while True:
        n = min(n, cap)
        t0 = time.perf_counter()
        out = oracle.detect_slot(sl.H[:n], sl.Y[:n], sl.sigma2, qam, n_pe, with_mmse=True,
                                 n_threads=n_threads)
        dt = time.perf_counter() - t0
        if dt >= seconds or n >= cap:
            if keep is not None:
                keep.append(out)
            return n * sl.n_sym / dt, out["threads"], n, dt
        grow = max(2.0, min(8.0, 1.2 * seconds / max(dt, 1e-3)))
        n = int(n * grow) + 1


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a per-rank scalar over the process group (identity when no
    group is initialised).  Works with nccl (device tensor) and gloo (CPU)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds: float, device=None) -> tuple[float, float]:
    """Weak-scaling aggregate: every rank processed `units_per_rank`; the job
    took as long as its slowest rank.  Returns (units/s over all ranks, max s)."""
    import torch.distributed as dist

    world = dist.get_world_size() if (dist.is_available() and dist.is_initialized()) else 1
    slowest = max_over_ranks(seconds, device)
    return world * units_per_rank / slowest, slowest


def source_hash(paths) -> str:
    h = hashlib.sha256()
    for p in paths:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def one_slot_graph_latency(ring, buf, precision, n, stream):
    """Latency of one slot alone through the whole path (the MMSE baseline
    beside it on a side stream), each ring slot's path captured once as a CUDA
    graph on its fixed inputs and `buf`, replayed one slot at a time and
    synchronised after each; sorted, in ms."""
    import torch

    from paper_2409_14355_gb300 import mpnl

    graphs = [mpnl.SlotGraph(buf, H, Y, s2, mmse=True, precision=precision) for H, Y, s2 in ring]
    for g in graphs[:3]:
        g.replay()
    torch.cuda.synchronize()
    out = []
    for i in range(n):
        a = torch.cuda.Event(enable_timing=True)
        c = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        with torch.cuda.stream(stream):
            graphs[i % len(graphs)].replay()
        c.record(stream)
        c.synchronize()
        out.append(a.elapsed_time(c))
    del graphs
    return sorted(out)


def walk_hbm(n_sc, n_sym, nt, B, n_pe, launch_ms):
    """The walk kernel against HBM, for completeness (it is ALU-bound):
    algorithmic bytes of one launch -- reads R (packed), 1/R_ll, perm, the
    table and z; writes hard decisions, LLRs and the PED pairs -- over its
    live launch time, against the measured copy bandwidth."""
    reads = n_sc * (nt * (nt + 1) // 2 * 8 + nt * 4 + nt + n_pe * nt) + n_sc * n_sym * nt * 8
    writes = n_sc * n_sym * (nt + nt * B * 4 + 8)
    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        pass
    gbs = (reads + writes) / (launch_ms / 1e3) / 1e9
    return {"bytes_per_launch": reads + writes, "read_bytes": reads, "write_bytes": writes,
            "achieved_gbs": gbs, "peak_gbs": peak, "peak_note": "measured copy bandwidth",
            "frac": gbs / peak if peak else None}


def load_traffic(kernel_src: list[str]):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "detect_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != source_hash(kernel_src):
        return None
    return rec.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------
# reference arm: the FP64 oracle on host cores
# --------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = inputs.WORKLOADS[args.workload]
    sl = inputs.workload_slot(args.workload, args.snr_index)
    import oracle

    oracle.build()
    qam, nt = w["qam"], w["nt"]
    # a bounded sample per step: sized from a calibration run so K + W steps
    # take a few minutes at most
    _, _, n_cal, dt_cal = time_oracle(sl, qam, args.n_pe, 1.0)
    per_sc = dt_cal / n_cal
    budget = 150.0 / max(1, args.steps + args.warmup)
    n_step = int(max(2, min(sl.n_sc, budget / per_sc)))
    for i in range(args.warmup):
        j = (i * n_step) % (sl.n_sc - n_step + 1)
        oracle.detect_slot(sl.H[j:j + n_step], sl.Y[j:j + n_step], sl.sigma2, qam, args.n_pe,
                           with_mmse=True)
    t0 = time.perf_counter()
    threads = 0
    for i in range(args.steps):
        j = ((args.warmup + i) * n_step) % (sl.n_sc - n_step + 1)
        o = oracle.detect_slot(sl.H[j:j + n_step], sl.Y[j:j + n_step], sl.sigma2, qam,
                               args.n_pe, with_mmse=True)
        threads = o["threads"]
    dt = time.perf_counter() - t0
    dets = args.steps * n_step * sl.n_sym
    value = dets / dt
    sample = (f"{n_step} of {sl.n_sc} subcarriers x 14 symbols per step "
              f"(full pipeline incl. MMSE), FP64")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gb_per_s": value * nt * BITS[qam] / 1e9,
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def run_mpnl(args):
    import torch
    import torch.distributed as dist

    from paper_2409_14355_gb300 import build as cuda_build
    from paper_2409_14355_gb300 import mpnl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        cuda_build.build()
    if world > 1:
        dist.barrier()
    mpnl.load_library()

    w = dict(inputs.WORKLOADS[args.workload])
    if args.n_sc is not None:
        w["n_sc"] = args.n_sc
    nr, nt, qam, n_sc = w["nr"], w["nt"], w["qam"], w["n_sc"]
    n_sym, n_pe, B = 14, args.n_pe, BITS[qam]
    ring = []
    for i in range(args.ring):
        sl = inputs.workload_slot(args.workload, args.snr_index, n_sc=n_sc,
                                  extra_seed=1 + i + 1000 * rank)
        ring.append((torch.from_numpy(sl.H).to(dev), torch.from_numpy(sl.Y).to(dev), sl.sigma2))
    sigma2 = ring[0][2]
    ring_bytes = sum(h.numel() * 8 + y.numel() * 8 for h, y, _ in ring)
    buf = mpnl.SlotBuffers(n_sc, n_sym, nr, nt, qam, n_pe, dev, mmse=True)
    stream = torch.cuda.current_stream(dev)

    def run_step(b, npe, precision, i, ev=None):
        H, Y, s2 = ring[i % len(ring)]
        mpnl.preprocess(H, Y, out=(b.R, b.inv_diag, b.perm, b.Z))
        mpnl.select_paths(b.R, s2, qam, npe, nt, out=b.paths)
        if ev is not None:
            ev[0].record(stream)
        mpnl.detect(b.R, b.inv_diag, b.perm, b.paths, b.Z, s2, qam,
                    out=(b.hard, b.llr, b.ped2), precision=precision)
        if ev is not None:
            ev[1].record(stream)
        mpnl.linear_mmse(H, Y, s2, qam, out=(b.mmse_hard, b.mmse_llr))

    def step(i, ev=None):
        run_step(buf, n_pe, args.precision, i, ev)

    for i in range(args.warmup):
        step(i)
    mpnl.check_status(local)
    torch.cuda.synchronize()

    K = args.steps
    # ---- the walk kernel alone (sequential steps, nothing overlapping it):
    # its per-launch time for the roofline
    det_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(max(10, K // 10))]
    for i, ev in enumerate(det_ev):
        step(i, ev)
    torch.cuda.synchronize()
    det_ms = [a.elapsed_time(b) for a, b in det_ev]
    det_avg = sum(det_ms) / len(det_ms)

    # ---- the timed steps: `inflight` slots in flight, each on its own stream
    # with its own buffers, the MMSE baseline of a slot on a side stream (it
    # needs only H and Y); consecutive slots overlap on the device
    nf = max(1, args.inflight)
    lanes = []
    for j in range(nf):
        b = buf if j == 0 else mpnl.SlotBuffers(n_sc, n_sym, nr, nt, qam, n_pe, dev, mmse=True)
        lanes.append((b, torch.cuda.Stream(dev), torch.cuda.Stream(dev)))

    def lane_step(i, ev):
        b, st, sm = lanes[i % nf]
        H, Y, s2 = ring[i % len(ring)]
        ev[0].record(st)
        sm.wait_event(ev[0])
        with torch.cuda.stream(sm):
            mpnl.linear_mmse(H, Y, s2, qam, out=(b.mmse_hard, b.mmse_llr))
        with torch.cuda.stream(st):
            mpnl.preprocess(H, Y, out=(b.R, b.inv_diag, b.perm, b.Z))
            mpnl.select_paths(b.R, s2, qam, n_pe, nt, out=b.paths)
            mpnl.detect(b.R, b.inv_diag, b.perm, b.paths, b.Z, s2, qam,
                        out=(b.hard, b.llr, b.ped2), precision=args.precision)
        st.wait_stream(sm)
        ev[1].record(st)

    for i in range(args.warmup):
        lane_step(i, (torch.cuda.Event(), torch.cuda.Event()))
    mpnl.check_status(local)
    torch.cuda.synchronize()
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)  # let the sampler attach
    t_start.record(stream)
    for _, st, sm in lanes:
        st.wait_event(t_start)
    for i in range(K):
        lane_step(args.warmup + i, step_ev[i])
    for _, st, _ in lanes:
        stream.wait_stream(st)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    mpnl.check_status(local)
    lat = sorted(a.elapsed_time(b) for a, b in step_ev)

    # ---- one slot in flight: the latency of a single slot through the whole
    # path (QR + z, selection, walks; the MMSE baseline beside them on a side
    # stream), nothing else on the device -- the figure to hold against the
    # 0.5 ms slot
    lat1 = []
    b0, st0, sm0 = lanes[0]
    for i in range(max(20, min(K, 100))):
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        lane_step(i, ev)  # lane 0 when nf == 1; else the lanes in turn, each alone
        ev[1].synchronize()
        lat1.append(ev[0].elapsed_time(ev[1]))
    lat1.sort()
    # the same with each slot's path replayed as one CUDA graph (mpnl.SlotGraph,
    # captured once per ring slot on its fixed buffers): no launch gaps
    latg = one_slot_graph_latency(ring, b0, args.precision, max(20, min(K, 100)), stream)

    # ---- end to end through the public host API (pinned host buffers)
    e2e_value = None
    h2d = d2h = 0
    hs = []
    for i in range(min(args.ring, 4)):
        H, Y, _ = ring[i]
        hs.append((H.cpu().pin_memory(), Y.cpu().pin_memory()))
    if args.e2e_steps > 0:
        # the streaming host API: every slot's H and Y copied in from pinned
        # host memory and its results (decisions, LLRs, PED pairs, MMSE
        # outputs) copied back into pinned host memory, `inflight` slots in
        # flight; each result is waited for in order
        pipe = mpnl.SlotPipeline(n_sc, n_sym, nr, nt, qam, n_pe, dev, depth=nf, mmse=True,
                                 precision=args.precision)

        def run_e2e(n):
            tickets = []
            for i in range(n):
                Hh, Yh = hs[i % len(hs)]
                tickets.append(pipe.submit(Hh, Yh, sigma2))
                if len(tickets) >= nf:
                    pipe.result(tickets.pop(0))
            for t in tickets:
                pipe.result(t)

        run_e2e(max(3, nf))
        pipe.check_status()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run_e2e(args.e2e_steps)
        e2e_dt = time.perf_counter() - t0
        h2d, d2h = pipe.h2d_bytes, pipe.d2h_bytes
        e2e_value, _ = whole_job_rate(args.e2e_steps * n_sc * n_sym, e2e_dt, dev)

    dets_per_step = n_sc * n_sym
    value, elapsed = whole_job_rate(K * dets_per_step, elapsed, dev)

    # ---- the other N_pe points of this workload and the other precision
    # (fewer steps; reported beside the main line, not instead of it)
    sweep = None
    if not args.no_sweep:
        sweep = []
        points = [(p, args.precision) for p in (32, 64, 128, 256) if p != n_pe and p <= qam ** nt]
        points.append((n_pe, "fp16" if args.precision == "fp32" else "fp32"))
        ks = max(10, K // 4)
        for npe, prec in points:
            b2 = mpnl.SlotBuffers(n_sc, n_sym, nr, nt, qam, npe, dev, mmse=True)
            for i in range(args.warmup):
                run_step(b2, npe, prec, i)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(ks)]
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for i in range(ks):
                run_step(b2, npe, prec, args.warmup + i, ev[i])
            a1.record(stream)
            torch.cuda.synchronize()
            mpnl.check_status(local)
            t = a0.elapsed_time(a1) / 1e3
            dms = sum(x.elapsed_time(y) for x, y in ev) / ks
            v, _ = whole_job_rate(ks * dets_per_step, t, dev)
            fl = npe * (4 * nt * nt + 4 * nt) * dets_per_step
            # one slot alone through the whole path (QR + z, selection, walks;
            # the MMSE baseline beside them on a side stream, as in the main
            # line's one-slot figure and in mpnl_detect_slot), synchronised
            # after each: the latency against the 0.5 ms slot at this N_pe
            one = one_slot_graph_latency(ring, b2, prec, 20, stream)
            sweep.append({"n_pe": npe, "precision": prec, "steps": ks, "value": v,
                          "ms_per_step": 1e3 * t / ks, "detect_ms": dms,
                          "detect_tflops": fl / (dms / 1e3) / 1e12,
                          "one_slot_ms": {"p50": one[len(one) // 2], "p99": one[-1],
                                          "note": "20 slots, one at a time, the MMSE baseline on a side stream, each slot's path one CUDA graph (mpnl.SlotGraph)"}})
            del b2

    # ---- the table-driven rank model beside the geometric one: the table's
    # build, the selection time and the BER of the slot with each table
    rank_lut = None
    rvd = None
    if not args.no_sweep:
        rank_lut = run_rank_lut(args, dev, n_pe)
        rvd = run_rvd(dev)

    # ---- mixed-size batch (64 radio units of random sizes) in persistent
    # launches under a CUDA graph, knobs from the autotuner, beside the same
    # units launched one by one
    mixed = None
    if not args.no_mixed:
        mixed = run_mixed(args, dev, rank)

    # ---- serving loop: Poisson slot requests from many radio units,
    # continuous batching, p50/p99 and deadline misses at 50-100% load
    serving_res = None
    if not args.no_serving:
        serving_res = run_serving(args, dev)

    # ---- measured FP32 FMA throughput (probe kernel), beside the derived peak
    props = torch.cuda.get_device_properties(dev)
    probe_tflops = ffma_probe_tflops(dev, stream, props.multi_processor_count * 8)

    # ---- roofline of the dominant kernel (walk kernel, FP32 ALU bound)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    flop_per_det = n_pe * (4 * nt * nt + 4 * nt)
    achieved_tflops = flop_per_det * dets_per_step / (det_avg / 1e3) / 1e12
    det_src = [os.path.join(ROOT, "paper_2409_14355_gb300", "csrc", f)
               for f in ("detect_impl.cuh", "detect_f32.cu", "mpnl_common.cuh")]
    traffic = load_traffic(det_src)

    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            sl0 = inputs.workload_slot(args.workload, args.snr_index, extra_seed=1)
            kept = []
            v, thr, n_used, dt = time_oracle(sl0, qam, n_pe, args.cpu_seconds, keep=kept)
            accuracy = accuracy_vs_oracle(sl0, kept[0], n_used, qam, n_pe, dev)
            accuracy["per_snr"] = accuracy_per_snr(args.workload, n_pe, dev)
            # the 8x8 16-QAM Kronecker-correlated workload's SNR sweep (the
            # MPNL walks at N_pe 64 against the linear MMSE baseline), whole slots
            if args.workload != "8x8-16qam-936sc":
                accuracy["per_snr_8x8_16qam_kronecker"] = accuracy_per_snr(
                    "8x8-16qam-936sc", 64, dev, n_sc=936)
            v1, _, n1, dt1 = time_oracle(sl0, qam, n_pe, args.cpu_seconds / 3, n_threads=1)
            cpu = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                   "sample": f"{n_used} of {n_sc} subcarriers x 14 symbols of one slot "
                             f"(whole path incl. MMSE), FP64, {dt:.1f} s",
                   "one_core": {"value": v1, "cores": 1,
                                "sample": f"{n1} subcarriers x 14 symbols, {dt1:.1f} s"},
                   "accuracy": accuracy}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f16+f32", "data": "synthetic",
            "config": dict(workload_config(args, w), parallelism=f"replicas{world}",
                           precision=args.precision, slots_in_flight=nf,
                           l2=f"ring of {len(ring)} distinct slots, {ring_bytes / 1e6:.0f} MB of "
                              f"H+Y > 129 MB L2"),
            "gb_per_s": value * nt * B / 1e9,
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "max": lat[-1], "deadline": 0.5,
                           "note": f"per step with {nf} slots in flight (throughput mode)"},
            "latency_one_in_flight_ms": {
                "p50": latg[len(latg) // 2], "p99": latg[min(len(latg) - 1, int(0.99 * len(latg)))],
                "max": latg[-1], "deadline": 0.5, "slots": len(latg),
                "per_call": {"p50": lat1[len(lat1) // 2],
                             "p99": lat1[min(len(lat1) - 1, int(0.99 * len(lat1)))]},
                "note": "one slot at a time through the whole path (MMSE baseline on a side "
                        "stream), synchronised after each, replayed as one CUDA graph per slot "
                        "(mpnl.SlotGraph); per_call: the same with one launch per kernel"},
            "roofline": {"bound": "alu", "kernel": "detect_walk_kernel",
                         "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved_tflops / peak_tflops, "traffic": traffic,
                         "flop_per_launch": flop_per_det * dets_per_step,
                         "launch_ms": det_avg,
                         "launch_timing": "walk kernel alone: sequential steps, CUDA events "
                                          "around its launches",
                         "peak_note": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x "
                                      f"{sm_max:.0f} MHz (max SM clock)",
                         "peak_measured_ffma": probe_tflops,
                         "frac_of_measured_ffma": achieved_tflops / probe_tflops,
                         "hbm": walk_hbm(n_sc, n_sym, nt, B, n_pe, det_avg)},
            "sweep": sweep,
            "rank_lut": rank_lut,
            "rvd": rvd,
            "mixed_batch": mixed,
            "serving": serving_res,
            "cpu_baseline": cpu,
            "e2e": None if e2e_value is None else
                   {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "path": f"mpnl_detect_slot (C ABI) on pinned host buffers, {nf} slots in "
                            f"flight on their own streams and workspaces"},
            "gpu_launches": 4 * K,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def ffma_probe_tflops(dev, stream, n_blk: int, iters: int = 8192, reps: int = 6) -> float:
    """FP32 FMA rate of the probe kernel of libmpnl_bench.so (8 independent
    fmaf chains per thread), best of `reps` launches timed with CUDA events."""
    import ctypes

    import torch

    from paper_2409_14355_gb300 import build as cuda_build

    lib = ctypes.CDLL(cuda_build.BENCH_LIB)
    lib.mpnl_bench_ffma_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    lib.mpnl_bench_ffma_probe.restype = ctypes.c_int
    out = torch.empty(n_blk * 256, dtype=torch.float32, device=dev)
    fl = ctypes.c_double(0.0)
    best = None
    for _ in range(reps):
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        st = lib.mpnl_bench_ffma_probe(n_blk, iters, ctypes.c_void_p(out.data_ptr()),
                                       ctypes.byref(fl), ctypes.c_void_p(stream.cuda_stream))
        a1.record(stream)
        torch.cuda.synchronize()
        if st != 0:
            raise RuntimeError(f"FMA probe failed ({st})")
        t = a0.elapsed_time(a1) / 1e3
        best = t if best is None else min(best, t)
    return fl.value / best / 1e12


def run_rank_lut(args, dev, n_pe):
    """Table-driven rank model on the bench workload: build a table (0.5 dB
    bins from -10 to 40 dB, 2^20 Monte-Carlo trials each) on the GPU, time
    mpnl_select_paths_lut against mpnl_select_paths on one slot, and compare
    the BER of the whole GPU path with either table."""
    import torch

    from paper_2409_14355_gb300 import mpnl

    sl = inputs.workload_slot(args.workload, args.snr_index, n_sc=args.n_sc)
    qam, nt, nr = sl.qam, sl.nt, sl.nr
    n_sc, n_sym = sl.H.shape[0], sl.Y.shape[1]
    B = {4: 2, 16: 4, 64: 6}[qam]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    trials = 1 << 20
    e0.record()
    lut = mpnl.RankLut.build(qam, -10.0, 40.0, 0.5, n_trials=trials, device=dev)
    e1.record()
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1)
    H = torch.from_numpy(sl.H).to(dev)
    Y = torch.from_numpy(sl.Y).to(dev)
    R, invd, perm, Z = mpnl.preprocess(H, Y)
    pg = mpnl.select_paths(R, sl.sigma2, qam, n_pe, nt)
    pt = mpnl.select_paths_lut(R, sl.sigma2, lut, n_pe, nt)

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_g = timed(lambda: mpnl.select_paths(R, sl.sigma2, qam, n_pe, nt, out=pg))
    ms_t = timed(lambda: mpnl.select_paths_lut(R, sl.sigma2, lut, n_pe, nt, out=pt))
    labels = sl.labels

    def ber(paths):
        hard, _, _ = mpnl.detect(R, invd, perm, paths, Z, sl.sigma2, qam, want_llr=False)
        h = hard.cpu().numpy()
        e = sum(int(np.sum(((h >> (B - 1 - b)) & 1) != ((labels >> (B - 1 - b)) & 1)))
                for b in range(B))
        return e / (labels.size * B)

    differ = (pg != pt).flatten(1).any(dim=1).float().mean().item()
    mpnl.check_status(dev.index)
    return {"bins": lut.n_bins, "db_range": [-10.0, 40.0, 0.5], "trials_per_bin": trials,
            "build_ms": build_ms, "select_ms_geometric": ms_g, "select_ms_table": ms_t,
            "tables_differ_frac": differ, "ber_geometric": ber(pg), "ber_table": ber(pt)}


def run_rvd(dev, name: str = "8x8-16qam-936sc", snr_index: int = 3, n_pe: int = 64):
    """The real-valued decomposition beside the complex path on the 8x8
    16-QAM workload (16 real levels; the 16x16 workload would need 32):
    walk-kernel and whole-path time per slot, and the BER of each."""
    import torch

    from paper_2409_14355_gb300 import mpnl

    sl = inputs.workload_slot(name, snr_index)
    qam, nt = sl.qam, sl.nt
    B = {4: 2, 16: 4, 64: 6}[qam]
    H = torch.from_numpy(sl.H).to(dev)
    Y = torch.from_numpy(sl.Y).to(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    rv = mpnl.run_slot_rvd(H, Y, sl.sigma2, qam, n_pe)
    ms_rvd = timed(lambda: mpnl.run_slot_rvd(H, Y, sl.sigma2, qam, n_pe))
    ms_rvd_walk = timed(lambda: mpnl.detect_rvd(rv["R"], rv["inv_diag"], rv["perm"], rv["paths"],
                                                rv["Z"], sl.sigma2, qam,
                                                out=(rv["hard"], rv["llr"], rv["ped2"])))
    buf = mpnl.SlotBuffers(sl.H.shape[0], sl.Y.shape[1], sl.nr, nt, qam, n_pe, dev, mmse=False)
    ms_cx = timed(lambda: mpnl.run_slot(buf, H, Y, sl.sigma2, mmse=False))
    ms_cx_walk = timed(lambda: mpnl.detect(buf.R, buf.inv_diag, buf.perm, buf.paths, buf.Z,
                                           sl.sigma2, qam, out=(buf.hard, buf.llr, buf.ped2)))
    mpnl.check_status(dev.index)

    def ber(hard):
        h = hard.cpu().numpy()
        e = sum(int(np.sum(((h >> (B - 1 - b)) & 1) != ((sl.labels >> (B - 1 - b)) & 1)))
                for b in range(B))
        return e / (sl.labels.size * B)

    dets = sl.H.shape[0] * sl.Y.shape[1]
    return {"workload": f"{name} snr {inputs.WORKLOADS[name]['snrs'][snr_index]} dB, N_pe {n_pe}",
            "rvd_ms_per_slot": ms_rvd, "rvd_walk_ms": ms_rvd_walk,
            "complex_ms_per_slot": ms_cx, "complex_walk_ms": ms_cx_walk,
            "rvd_detections_per_s": dets / (ms_rvd / 1e3),
            "complex_detections_per_s": dets / (ms_cx / 1e3),
            "ber_rvd": ber(rv["hard"]), "ber_complex": ber(buf.hard)}


def accuracy_vs_oracle(sl, ref, n_used, qam, n_pe, dev):
    """Decision-mismatch rate and BER of the GPU path (FP32 and FP16
    residuals) against the FP64 oracle on the subcarriers the oracle ran."""
    import torch

    from paper_2409_14355_gb300 import mpnl

    B = BITS[qam]
    labels = sl.labels[:n_used]

    def ber(hard):
        e = 0
        for b in range(B):
            e += np.sum(((hard >> (B - 1 - b)) & 1) != ((labels >> (B - 1 - b)) & 1))
        return float(e / (labels.size * B))

    out = {"subcarriers": int(n_used), "ber_oracle": ber(ref["hard"]),
           "ber_oracle_mmse": ber(ref["mmse_hard"])}
    H = torch.from_numpy(sl.H).to(dev)
    Y = torch.from_numpy(sl.Y).to(dev)
    for prec in ("fp32", "fp16"):
        g = mpnl.detect_slot(H, Y, sl.sigma2, qam, n_pe, mmse=True, precision=prec)
        hard = g["hard"].cpu().numpy()[:n_used]
        out[prec] = {"decision_mismatch": float(np.mean(np.any(hard != ref["hard"], axis=-1))),
                     "ber": ber(hard), "ber_delta": ber(hard) - out["ber_oracle"]}
        if prec == "fp32":
            out["ber_mmse_gpu"] = ber(g["mmse_hard"].cpu().numpy()[:n_used])
    return out


def accuracy_per_snr(name, n_pe, dev, n_sc: int = 96):
    """BER of the oracle, the FP32 path and the mixed-precision walks, and the
    two forms' decision mismatch against the oracle, at every SNR point of
    the workload (the first n_sc subcarriers of each point's slot)."""
    import oracle
    from paper_2409_14355_gb300 import mpnl

    import torch

    w = inputs.WORKLOADS[name]
    B = BITS[w["qam"]]
    rows = []
    for k, snr in enumerate(w["snrs"]):
        sl = inputs.workload_slot(name, k, n_sc=min(n_sc, w["n_sc"]))
        ref = oracle.detect_slot(sl.H, sl.Y, sl.sigma2, sl.qam, n_pe)

        def ber(h):
            e = sum(np.sum(((h >> (B - 1 - b)) & 1) != ((sl.labels >> (B - 1 - b)) & 1))
                    for b in range(B))
            return float(e / (sl.labels.size * B))

        row = {"snr_db": snr, "ber_oracle": ber(ref["hard"])}
        H = torch.from_numpy(sl.H).to(dev)
        Y = torch.from_numpy(sl.Y).to(dev)
        for prec in ("fp32", "fp16"):
            g = mpnl.detect_slot(H, Y, sl.sigma2, sl.qam, n_pe, precision=prec)
            h = g["hard"].cpu().numpy()
            row[prec] = {"ber": ber(h), "ber_delta": ber(h) - row["ber_oracle"],
                         "decision_mismatch": float(np.mean(np.any(h != ref["hard"], axis=-1)))}
        # beside them: the paper's own N_p = 32 and the linear MMSE baseline
        g32 = mpnl.detect_slot(H, Y, sl.sigma2, sl.qam, min(32, n_pe), mmse=True)
        row["ber_n_pe_32"] = ber(g32["hard"].cpu().numpy())
        row["ber_mmse"] = ber(g32["mmse_hard"].cpu().numpy())
        # the walks over the MMSE-extended sorted QR ([H; sigma I]), against
        # the oracle's same pre-processing
        ref_q = oracle.detect_slot(sl.H, sl.Y, sl.sigma2, sl.qam, n_pe, mmse_qr=True)
        gq = mpnl.detect_slot(H, Y, sl.sigma2, sl.qam, n_pe, mmse_qr=True)
        hq = gq["hard"].cpu().numpy()
        row["mmse_qr"] = {"ber": ber(hq), "ber_oracle": ber(ref_q["hard"]),
                          "decision_mismatch": float(np.mean(np.any(hq != ref_q["hard"], axis=-1)))}
        rows.append(row)
    return {"subcarriers_per_point": min(n_sc, w["n_sc"]), "points": rows}


def run_mixed(args, dev, rank):
    import torch

    from paper_2409_14355_gb300 import autotune, mpnl

    units = inputs.mixed_units(args.mixed_units, seed=inputs.seed_for(inputs.MIXED_CONFIG) + rank)
    tuning, report = autotune.tune(units, dev.index)
    mpnl.set_tuning(tuning, dev.index)
    try:
        bufs = []
        for u in units:
            sl = inputs.unit_slot(u)
            b = mpnl.SlotBuffers(u.n_sc, 14, u.nr, u.nt, u.qam, u.n_pe, dev, mmse=True)
            b.H.copy_(torch.from_numpy(sl.H))
            b.Y.copy_(torch.from_numpy(sl.Y))
            bufs.append((b, sl.sigma2, False, True))
        dets = sum(u.n_sc for u in units) * 14
        batch = mpnl.Batch(bufs, dev)
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        steps = max(10, args.steps // 10)

        def timed(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b_ = torch.cuda.Event(enable_timing=True)
            a.record(side)
            for _ in range(steps):
                fn()
            b_.record(side)
            torch.cuda.synchronize()
            return a.elapsed_time(b_) / steps

        with torch.cuda.stream(side):
            ms_graph = timed(lambda: batch.run(graph=True, stream=side))
            ms_seq = timed(lambda: [mpnl.run_slot(b, b.H, b.Y, s2, mmse=mm, mmse_qr=mq)
                                    for b, s2, mq, mm in bufs])
        mpnl.check_status(dev.index)
        batch.close()
    finally:
        mpnl.set_tuning(None, dev.index)
    return {"workload": f"{len(units)} radio units, rx in {{4,8,16}}, users rx/2..rx, QAM "
                        f"{{4,16,64}}, sc {{312,936,3276}}, N_pe 16..256 (uniform, seeded)",
            "detections_per_step": dets, "value": dets / (ms_graph / 1e3), "unit": UNIT,
            "ms_per_step": ms_graph, "steps": steps, "launch": "persistent per stage, CUDA graph",
            "per_unit_launches_ms": ms_seq,
            "tuning": autotune.to_dict(tuning),
            "tuning_batch_ms": report["batch_ms"], "tuning_choice": report["batch_choice"]}


def run_serving(args, dev, sm_split: int = 0, capacity: float | None = None):
    """The serving loop on the RU mix: its capacity (or the one given, so
    that two configurations see the same offered loads), then latency at 50,
    75 and 100% of it.  sm_split > 0: the small units' rounds on a group of
    that many SMs of their own."""
    import torch

    from paper_2409_14355_gb300 import serving

    units = serving.serving_units(args.serving_rus)
    server = serving.Server(dev, mem_budget=4 << 30, max_units_per_round=64, sm_split=sm_split)
    payloads = {}
    for k, u in enumerate(units):
        sl = inputs.unit_slot(u)
        server.register(serving.RU(k, u.nr, u.nt, u.qam, u.n_sc, u.n_pe, sl.sigma2),
                        torch.from_numpy(sl.H))
        payloads[k] = {"slot": [torch.from_numpy(sl.Y).pin_memory()],
                       "channel": [torch.from_numpy(sl.H).pin_memory()]}
    dets = {k: u.n_sc * 14 for k, u in enumerate(units)}
    mean_dets = float(np.mean(list(dets.values())))
    # capacity: every RU's slot offered at once, twice over (rounds stay full);
    # a first pass warms the loop up (each round slot creates its batch and
    # the pinned pools are touched), the second is measured
    sat = [(0.0, k, "slot") for _ in range(2) for k in range(len(units))]
    serving.run_trace(server, sat, payloads)
    reqs = serving.run_trace(server, sat, payloads)
    span = max(q.done for q in reqs) - min(q.arrival for q in reqs)
    own_capacity = sum(dets[q.ru] for q in reqs) / span
    if capacity is None:
        capacity = own_capacity
    loads = {}
    for rho in (0.5, 0.75, 1.0):
        rate = rho * capacity / mean_dets
        trace = serving.poisson_trace(units, rate, args.serving_seconds, seed=int(100 * rho))
        server.round_sizes.clear()
        server.host_launch_s = 0.0
        reqs = serving.run_trace(server, trace, payloads)
        st = serving.latency_stats(reqs, dets_of=lambda q: dets[q.ru],
                                   big_of=lambda q: server.rus[q.ru].cost >= server.big_cost)
        st.update(offered_detections_per_s=rho * capacity, mean_round=float(
            np.mean(server.round_sizes)) if server.round_sizes else 0.0,
            rounds=len(server.round_sizes),
            host_ms_per_round=1e3 * server.host_launch_s / max(1, len(server.round_sizes)))
        loads[str(rho)] = st
    sms = list(server.split_sms) if server.split_sms is not None else None
    server.close()
    realtime = [serving_realtime(dev, n_pe) for n_pe in (32, 64)] if sm_split == 0 else None
    n_big = sum(1 for u in units if (u.nr, u.nt, u.qam, u.n_sc) == (16, 16, 64, 3276))
    return {"workload": f"{len(units)} radio units ({n_big} of them 16x16 64-QAM 3276 sc), "
                        f"sizes as the mixed batch, Poisson slot requests, channel update every "
                        f"8th slot of a unit; large units: walk work >= a 16x16 936-sc N_pe 64 "
                        f"slot", "deadline_ms": 0.5,
            "capacity_detections_per_s": capacity, "own_capacity_detections_per_s": own_capacity,
            "sm_split": sms, "seconds_per_load": args.serving_seconds,
            "resident_state_MB": server.state_bytes / 1e6, "loads": loads,
            "realtime": realtime}


def serving_realtime(dev, n_pe: int, slots: int = 2000, warm: int = 200) -> dict:
    """The real-time load of one 16x16 64-QAM 3276-subcarrier radio unit
    through the serving loop: a slot request every 0.5 ms (the slot period),
    a channel update with every 8th, the LLRs computed into the slot's
    device buffers and left there for a decoder on the device (the hard
    decisions are copied back).  p50/p99 latency and the deadline-miss rate
    over `slots` slots after `warm` warm-up slots."""
    import torch

    from paper_2409_14355_gb300 import serving

    u = inputs.UnitSpec(16, 16, 64, 3276, n_pe, 21.0, "iid", 12345)
    sl = inputs.unit_slot(u)
    server = serving.Server(dev, mem_budget=4 << 30, llr_to_host=False)
    server.register(serving.RU(0, u.nr, u.nt, u.qam, u.n_sc, u.n_pe, sl.sigma2),
                    torch.from_numpy(sl.H))
    alts = [inputs.unit_slot(inputs.UnitSpec(**{**u.__dict__, "seed": u.seed + j}))
            for j in range(1, 4)]
    payloads = {0: {"slot": [torch.from_numpy(a.Y).pin_memory() for a in [sl] + alts],
                    "channel": [torch.from_numpy(a.H).pin_memory() for a in alts]}}

    def trace(n):
        out = []
        for i in range(n):
            if i % 8 == 7:
                out.append((i * serving.DEADLINE_S, 0, "channel"))
            out.append((i * serving.DEADLINE_S, 0, "slot"))
        return out

    serving.run_trace(server, trace(warm), payloads)
    st = serving.latency_stats(serving.run_trace(server, trace(slots), payloads))
    server.close()
    return {"workload": "one 16x16 64-QAM 3276-sc radio unit, a slot every 0.5 ms, channel "
                        "update every 8th slot, LLRs left on the device", "n_pe": n_pe,
            "slots": st["slots_done"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "miss_rate": st["miss_rate"]}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_mpnl(args)


if __name__ == "__main__":
    sys.exit(main())
