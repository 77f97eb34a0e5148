"""Autotuner for the launch-shape knobs (mpnl_tuning).

The knobs change how work is spread over threads, never the results:
symbols per lane of the walk kernel (1 or 2: how many walks one lane runs per
staged column of R), warps per subcarrier of the selection (1, 2 or 4: the
slice each thread merges), and, for the persistent batch launches, CTAs per
SM of the walk launch and the selection's warps per subcarrier.  For every
problem class that occurs in a workload (nt class x QAM x N_pe class, see
mpnl.problem_class) the tuner times each candidate of the per-call knobs on
a representative problem of that class with CUDA events and keeps the
fastest; then it times the whole batch in its persistent launches for every
combination of the batch knobs (and of the symbols-per-lane table: tuned per
class, all 1, all 2) and keeps the fastest.
Results can be cached in a JSON file keyed by the GPU and the library build.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import inputs, mpnl

SYM_CHOICES = (1, 2)
SELECT_WARP_CHOICES = (1, 2, 4)
CTA_CHOICES = (2, 3)


def _time_ms(fn, reps: int = 5, warmup: int = 2) -> float:
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _representative(units):
    """The largest unit (by subcarriers x N_pe) of each problem class."""
    best = {}
    for u in units:
        c = mpnl.problem_class(u.nt, u.qam, u.n_pe)
        if c not in best or u.n_sc * u.n_pe > best[c].n_sc * best[c].n_pe:
            best[c] = u
    return best


def tune(units, device=None, max_sc: int = 512, reps: int = 5) -> tuple[mpnl.Tuning, dict]:
    """Pick the knobs for a workload given as inputs.UnitSpec's.  Returns the
    Tuning (not installed) and a report of every timing taken."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    report = {"classes": {}, "batch_ms": {}}
    t = mpnl.Tuning()
    try:
        for c, u in sorted(_representative(units).items()):
            n_sc = min(u.n_sc, max_sc)
            sl = inputs.unit_slot(inputs.UnitSpec(u.nr, u.nt, u.qam, n_sc, u.n_pe, u.snr_db,
                                                  u.channel, u.seed))
            buf = mpnl.SlotBuffers(n_sc, 14, u.nr, u.nt, u.qam, u.n_pe, dev, mmse=False)
            buf.H.copy_(torch.from_numpy(sl.H))
            buf.Y.copy_(torch.from_numpy(sl.Y))
            mpnl.preprocess(buf.H, buf.Y, out=(buf.R, buf.inv_diag, buf.perm, buf.Z))
            rec = {"unit": [u.nr, u.nt, u.qam, n_sc, u.n_pe], "select_ms": {}, "detect_ms": {}}
            for w in SELECT_WARP_CHOICES:
                probe = mpnl.Tuning()
                probe.select_warps[c[0]][c[1]][c[2]] = w
                mpnl.set_tuning(probe, dev.index)
                rec["select_ms"][w] = _time_ms(lambda: mpnl.select_paths(
                    buf.R, sl.sigma2, u.qam, u.n_pe, u.nt, out=buf.paths), reps)
            for s in SYM_CHOICES:
                probe = mpnl.Tuning()
                probe.detect_sym[c[0]][c[1]][c[2]] = s
                mpnl.set_tuning(probe, dev.index)
                rec["detect_ms"][s] = _time_ms(lambda: mpnl.detect(
                    buf.R, buf.inv_diag, buf.perm, buf.paths, buf.Z, sl.sigma2, u.qam,
                    out=(buf.hard, buf.llr, buf.ped2)), reps)
            t.select_warps[c[0]][c[1]][c[2]] = min(rec["select_ms"], key=rec["select_ms"].get)
            t.detect_sym[c[0]][c[1]][c[2]] = min(rec["detect_ms"], key=rec["detect_ms"].get)
            report["classes"][str(c)] = rec
        # the whole batch in its persistent launches, per combination of the
        # batch knobs
        bufs = []
        for u in units:
            sl = inputs.unit_slot(u)
            b = mpnl.SlotBuffers(u.n_sc, 14, u.nr, u.nt, u.qam, u.n_pe, dev, mmse=False)
            b.H.copy_(torch.from_numpy(sl.H))
            b.Y.copy_(torch.from_numpy(sl.Y))
            bufs.append((b, sl.sigma2, False, False))
        best = None
        for sym_mode in ("tuned", 1, 2):
            for warps in SELECT_WARP_CHOICES:
                for k in CTA_CHOICES:
                    probe = mpnl.Tuning()
                    ctypes_copy(probe, t)
                    if sym_mode != "tuned":
                        for a in range(3):
                            for b_ in range(3):
                                for c_ in range(2):
                                    probe.detect_sym[a][b_][c_] = sym_mode
                    probe.persistent_ctas_per_sm = k
                    probe.persistent_select_warps = warps
                    mpnl.set_tuning(probe, dev.index)
                    batch = mpnl.Batch(bufs, dev)
                    ms = _time_ms(lambda: batch.run(mpnl.STAGES_ALL & ~mpnl.STAGE_MMSE), reps)
                    batch.close()
                    key = f"sym={sym_mode},select_warps={warps},ctas={k}"
                    report["batch_ms"][key] = ms
                    if best is None or ms < best[0]:
                        best = (ms, sym_mode, warps, k)
        _, sym_mode, warps, k = best
        batch_sym = mpnl.Tuning()
        ctypes_copy(batch_sym, t)
        if sym_mode != "tuned":
            for a in range(3):
                for b_ in range(3):
                    for c_ in range(2):
                        batch_sym.detect_sym[a][b_][c_] = sym_mode
        report["batch_choice"] = {"sym": sym_mode, "select_warps": warps, "ctas": k}
        # the per-call table stays the per-class choice; the batch knobs join it
        # (a batch built with this tuning uses the per-class symbols per lane)
        if sym_mode != "tuned":
            ctypes_copy(t, batch_sym)
        t.persistent_ctas_per_sm = k
        t.persistent_select_warps = warps
    finally:
        mpnl.set_tuning(None, dev.index)
    return t, report


def ctypes_copy(dst: mpnl.Tuning, src: mpnl.Tuning) -> None:
    for a in range(3):
        for b in range(3):
            for c in range(2):
                dst.detect_sym[a][b][c] = src.detect_sym[a][b][c]
                dst.select_warps[a][b][c] = src.select_warps[a][b][c]
    dst.persistent_ctas_per_sm = src.persistent_ctas_per_sm
    dst.persistent_select_warps = src.persistent_select_warps


def to_dict(t: mpnl.Tuning) -> dict:
    return {"detect_sym": [[list(t.detect_sym[a][b]) for b in range(3)] for a in range(3)],
            "select_warps": [[list(t.select_warps[a][b]) for b in range(3)] for a in range(3)],
            "persistent_ctas_per_sm": int(t.persistent_ctas_per_sm),
            "persistent_select_warps": int(t.persistent_select_warps)}


def from_dict(d: dict) -> mpnl.Tuning:
    t = mpnl.Tuning()
    for a in range(3):
        for b in range(3):
            for c in range(2):
                t.detect_sym[a][b][c] = d["detect_sym"][a][b][c]
                t.select_warps[a][b][c] = d["select_warps"][a][b][c]
    t.persistent_ctas_per_sm = d["persistent_ctas_per_sm"]
    t.persistent_select_warps = d.get("persistent_select_warps", 0)
    return t


def cache_key(device=None) -> str:
    """GPU name + a hash of the built library: a tuning is reused only on the
    same hardware and code."""
    dev = torch.cuda.current_device() if device is None else device
    h = hashlib.sha256()
    with open(mpnl.LIB_PATH, "rb") as f:
        h.update(f.read())
    return f"{torch.cuda.get_device_name(dev)}|{h.hexdigest()[:16]}"


def load_or_tune(units, cache_path: str | None = None, device=None) -> tuple[mpnl.Tuning, dict]:
    """Tuning for the workload from the cache file if it holds one for this
    GPU and build, else tuned now (and written to the cache when a path is
    given)."""
    key = cache_key(device)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return from_dict(cache[key]["tuning"]), {"cached": True, **cache[key]["report"]}
    t, report = tune(units, device)
    if cache_path:
        cache[key] = {"tuning": to_dict(t), "report": report}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return t, {"cached": False, **report}
