"""Serving loop for slot-detection requests from many radio units (RUs).

An O-RAN distributed unit serves many RUs (§I, §IV: one DU, many RUs, the
compute allocated where the load is).  Each RU has its own antenna, user,
QAM and subcarrier counts.  This module keeps every RU's channel state on
the device -- the antenna rows of Q, R, 1/R_ll, the sorted order and the
N_pe position vectors, all computed from the channel alone when the RU
reports a new channel (§II: the candidate positions are found before the
data arrives) -- and serves two kinds of requests:

  channel  new H for an RU: sorted QR keeping Q (FP16 units: re-factorised
           in FP64 where the channel is ill-conditioned), then the path
           selection;
  slot     the received symbols Y of one slot: z = Q^H y, the N_pe walks,
           hard decisions and max-log LLRs.

Continuous batching: requests wait in arrival order; whenever one of the
`max_inflight` round slots is free, the waiting requests that fit the
device-memory budget (their input, scratch and output buffers) form a round,
which runs as one mixed-size batch in the persistent launches (QR, selection,
Q^H y, walks) on its own stream.  Requests arriving while rounds run join the
next round, and up to `max_inflight` rounds overlap on the device.  A round
copies its inputs from pinned host memory, runs, copies hard decisions and
LLRs back, and records an event; a request's latency is the time from its
arrival to the completion of its round, against the 0.5 ms slot deadline
(§III-B).  An RU's channel update never shares the device with a round that
still reads the RU's previous state: it waits for those rounds to finish,
and the RU's later slots wait behind it (they may join its round: the
stages run in order, QR and selection before Q^H y and the walks; a slot
never joins another round while the update is in flight).

Nothing here does arithmetic of the detector: all of it runs in the CUDA
kernels behind the C ABI (mpnl.py).
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import inputs, mpnl

DEADLINE_S = 0.5e-3
# FP16 units' channels whose FP32 factor has max R_ll / min R_ll above this
# are re-factorised in FP64 (the threshold the mixed-precision path is
# stated for; the batch stage uses the same)
REFINE_COND = 1e3


@dataclass
class RU:
    """One radio unit and its device-resident channel state."""
    ru_id: int
    nr: int
    nt: int
    qam: int
    n_sc: int
    n_pe: int
    sigma2: float
    mmse_qr: bool = False
    n_sym: int = 14
    precision: str = "fp32"   # "fp16": tensor-core Q^H y and FP16-residual walks
    state: dict = field(default_factory=dict)   # Q, R, inv_diag, perm, paths (device)
    busy_rounds: set = field(default_factory=set)
    update_round: int = -1    # round of the RU's channel update in flight (-1: none)
    gone: bool = False        # deregistered; state released when its rounds retire
    item: object = None       # the resident state as an mpnl_batch_item (rounds refer to it)
    pool: list = field(default_factory=list)    # free per-slot buffer sets
    H_dev: torch.Tensor | None = None           # device staging of a channel update

    @property
    def dims(self):
        return (self.n_sc, self.n_sym, self.nr, self.nt, self.qam, self.n_pe)

    @property
    def cost(self) -> float:
        """Relative work of one slot (the walks dominate)."""
        return float(self.n_sc * self.n_sym * self.n_pe * self.nt * (self.nt + 4))

    def state_bytes(self) -> int:
        n_sc, nr, nt = self.n_sc, self.nr, self.nt
        return n_sc * (nr * nt * 8 + nt * (nt + 1) // 2 * 8 + nt * 4 + nt + self.n_pe * nt)


class SlotBuffers:
    """Device and pinned host buffers of one in-flight slot request of an RU
    (allocated at registration, reused)."""

    def __init__(self, ru: "RU", device, llr: bool, llr_to_host: bool = True):
        n_sc, n_sym, nr, nt = ru.n_sc, ru.n_sym, ru.nr, ru.nt
        kw = dict(device=device)
        self.Y = torch.empty((n_sc, n_sym, nr), dtype=torch.complex64, **kw)
        self.Z = torch.empty((n_sc, n_sym, nt), dtype=torch.complex64, **kw)
        self.hard = torch.empty((n_sc, n_sym, nt), dtype=torch.uint8, **kw)
        self.llr = (torch.empty((n_sc, n_sym, nt, mpnl.BITS[ru.qam]), dtype=torch.float32, **kw)
                    if llr else None)
        pin = device.type == "cuda"
        self.hard_host = torch.empty(self.hard.shape, dtype=torch.uint8, pin_memory=pin)
        # None when the LLRs stay on the device (for a decoder there)
        self.llr_host = (torch.empty(self.llr.shape, dtype=torch.float32, pin_memory=pin)
                         if llr and llr_to_host else None)


@dataclass
class Request:
    rid: int
    ru: int
    kind: str                 # "slot" or "channel"
    arrival: float            # seconds since the start of the run
    payload: torch.Tensor     # pinned host: Y [n_sc][n_sym][nr] or H [n_sc][nr][nt]
    admitted: float = -1.0
    done: float = -1.0
    round_id: int = -1
    hard: torch.Tensor | None = None   # host results (slot requests)
    llr: torch.Tensor | None = None
    bufs: SlotBuffers | None = None


def request_bytes(ru: RU, kind: str, llr: bool) -> int:
    """Device bytes a request holds while it is in flight."""
    n = ru.n_sc
    if kind == "channel":
        return n * ru.nr * ru.nt * 8
    b = n * ru.n_sym * (ru.nr * 8 + ru.nt * 8 + ru.nt + 8)
    if llr:
        b += n * ru.n_sym * ru.nt * mpnl.BITS[ru.qam] * 4
    return b


class _Round:
    def __init__(self, server, slot_index: int):
        self.server = server
        self.index = slot_index
        self._streams = {}
        self.big = False
        self.batch = None
        self.requests: list[Request] = []
        self.buffers: list = []
        self.bytes = 0
        self.event = None
        self.round_id = -1

    def stream_for(self, big: bool):
        """The round's stream for its size class, created on first use (the
        loop's logic needs no GPU): small units' rounds run on a
        high-priority stream, so their CTAs are scheduled ahead of a large
        unit's walks still in flight; with an SM split, each class's rounds
        run on its own group of SMs."""
        if big not in self._streams:
            lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") \
                else (0, -1)
            prio = lo if big else hi
            if self.server.split is not None:
                self._streams[big] = self.server.split.stream(1 if big else 0, prio, self.index)
            else:
                self._streams[big] = torch.cuda.Stream(self.server.device, priority=prio)
        return self._streams[big]

    @property
    def free(self) -> bool:
        return self.event is None


class Server:
    """Continuous-batching serving loop over device-resident RU state."""

    def __init__(self, device=None, mem_budget: int = 2 << 30, max_units_per_round: int = 64,
                 max_inflight: int = 4, llr: bool = True, starve_s: float = 5e-3,
                 slots_per_ru: int = 2, keep_results: bool = False,
                 big_cost: float = 936 * 14 * 64 * 16 * 20, max_large_rounds: int | None = None,
                 share_sms: bool = False, large_per_unit: bool = True,
                 small_short_ctas: bool = True, native_rounds: bool = True,
                 sm_split: int = 0, llr_to_host: bool = True):
        self.device = (torch.device("cuda", torch.cuda.current_device()) if device is None
                       else torch.device(device))
        self.mem_budget = int(mem_budget)
        self.max_units = int(max_units_per_round)
        self.llr = llr
        # llr_to_host False: the LLRs are computed into the slot's device
        # buffer and left there (a decoder on the device reads them); only
        # the hard decisions are copied back
        self.llr_to_host = llr_to_host
        self.starve_s = starve_s
        self.slots_per_ru = slots_per_ru
        self.big_cost = big_cost  # units at least this costly form rounds of their own
        # at most this many large units' rounds in flight, so that a small
        # unit's slot always finds a round to go into
        self.max_large_rounds = (max(1, max_inflight // 2) if max_large_rounds is None
                                 else max_large_rounds)
        # large units' rounds leave a CTA slot per SM to the small units'
        # high-priority rounds (MPNL_RUN_SHARE_SMS); off by default: measured
        # on the serving mix it slowed the large units more than it sped up
        # the small ones
        self.share_sms = share_sms
        # large units' rounds as per-call launches (short CTAs the small units'
        # high-priority rounds can slip between) rather than persistent ones
        self.large_per_unit = large_per_unit
        # small units' rounds with one CTA per work item (MPNL_RUN_SHORT_CTAS):
        # a persistent round would do all its items on the few CTAs that find
        # an SM free beside the large units' walks
        self.small_short_ctas = small_short_ctas
        # rounds after a batch's first as one native call (mpnl_serve_round)
        self.native_rounds = native_rounds
        # sm_split > 0: the small units' rounds get a group of at least that
        # many SMs of their own (mpnl_sm_split_*), the large units' the rest;
        # made on first use of a round stream (one split per size per process)
        self.sm_split = int(sm_split)
        self._split = None
        self.split_sms = None   # (small units' SMs, large units' SMs) once made
        self.keep_results = keep_results  # copy each result out (else a view valid
        # until the RU's pool buffer is reused)
        self.rus: dict[int, RU] = {}
        self.state_bytes = 0
        self.in_use = 0
        self.waiting: collections.deque[Request] = collections.deque()
        self.rounds = [_Round(self, k) for k in range(max_inflight)]
        self.completed: list[Request] = []
        self.dropped: list[Request] = []
        self.n_rounds = 0
        self.t0 = time.perf_counter()
        self.peak_in_use = 0
        self.round_sizes: list[int] = []
        self.host_launch_s = 0.0  # host time spent forming and enqueueing rounds

    # ---- RU registration (setup, synchronous)
    def register(self, ru: RU, H: torch.Tensor) -> None:
        """Allocate the RU's resident state and compute it from channel H."""
        dev = self.device
        n_sc, nr, nt = ru.n_sc, ru.nr, ru.nt
        st = dict(Q=torch.empty((n_sc, nr, nt), dtype=torch.complex64, device=dev),
                  R=torch.empty((n_sc, nt * (nt + 1) // 2), dtype=torch.complex64, device=dev),
                  inv_diag=torch.empty((n_sc, nt), dtype=torch.float32, device=dev),
                  perm=torch.empty((n_sc, nt), dtype=torch.uint8, device=dev),
                  paths=torch.empty((n_sc, ru.n_pe, nt), dtype=torch.uint8, device=dev))
        ru.state = st
        ru.pool = [SlotBuffers(ru, dev, self.llr, self.llr_to_host)
                   for _ in range(self.slots_per_ru)]
        ru.H_dev = torch.empty((n_sc, nr, nt), dtype=torch.complex64, device=dev)
        # the unit's resident state as a batch item: what a round's request refers to
        ru.item = mpnl.batch_item(ru.dims, ru.sigma2, self._unit_flags(ru), 0, Q=st["Q"], R=st["R"],
                                  inv_diag=st["inv_diag"], perm=st["perm"], paths=st["paths"])
        Hd = H.to(dev)
        mpnl.factor(Hd, ru.sigma2 if ru.mmse_qr else None,
                    out=(st["Q"], st["R"], st["inv_diag"], st["perm"]))
        if ru.precision == "fp16":
            mpnl.refine_qr(Hd, None, st["R"], st["inv_diag"], st["perm"], Q=st["Q"],
                           sigma2=ru.sigma2 if ru.mmse_qr else None, cond_threshold=REFINE_COND)
        mpnl.select_paths(st["R"], ru.sigma2, ru.qam, ru.n_pe, nt, out=st["paths"])
        torch.cuda.synchronize(dev)
        self.rus[ru.ru_id] = ru
        self.state_bytes += ru.state_bytes()

    @staticmethod
    def _unit_flags(ru: RU) -> int:
        return (mpnl.ITEM_MMSE_QR if ru.mmse_qr else 0) \
            | (mpnl.ITEM_FP16 | mpnl.ITEM_REFINE_QR if ru.precision == "fp16" else 0)

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request) -> bool:
        """Queue a request; a request of an unknown or deregistered RU is
        dropped (done = -2, kept in `dropped`) and False returned."""
        ru = self.rus.get(req.ru)
        if ru is None or ru.gone:
            req.done = -2.0
            self.dropped.append(req)
            return False
        self.waiting.append(req)
        return True

    def deregister(self, ru_id: int) -> list[Request]:
        """An RU that disappears (its fronthaul link drops, it powers
        down): its waiting requests are dropped (done = -2) and returned,
        later submissions for it are refused, and its device state and
        buffers are released as soon as no round in flight still uses them
        (at once if none does).  Its requests already in a round complete
        normally."""
        ru = self.rus.get(ru_id)
        if ru is None:
            return []
        ru.gone = True
        out = [q for q in self.waiting if q.ru == ru_id]
        self.waiting = collections.deque(q for q in self.waiting if q.ru != ru_id)
        for q in out:
            q.done = -2.0
        self.dropped.extend(out)
        self._release_if_idle(ru)
        return out

    def _release_if_idle(self, ru: RU) -> None:
        if ru.gone and not ru.busy_rounds and ru.ru_id in self.rus:
            self.state_bytes -= ru.state_bytes() if ru.state else 0
            ru.state, ru.pool, ru.H_dev = {}, [], None
            del self.rus[ru.ru_id]

    # ---- the loop
    def poll(self) -> int:
        """Retire finished rounds; returns how many finished."""
        n = 0
        for r in self.rounds:
            if r.event is not None and r.event.query():
                t = self.now()
                for q in r.requests:
                    q.done = t
                    self.completed.append(q)
                    ru = self.rus[q.ru]
                    ru.busy_rounds.discard(r.round_id)
                    if ru.update_round == r.round_id:
                        ru.update_round = -1
                    if q.bufs is not None:
                        llr = q.bufs.llr_host if q.bufs.llr_host is not None else q.bufs.llr
                        if self.keep_results:
                            q.hard = q.bufs.hard_host.clone()
                            q.llr = llr.clone() if llr is not None else None
                            if llr is not None and llr.is_cuda:
                                # the device copy runs on the current stream; it
                                # must be done before the buffer goes back to the
                                # pool, where a round on another stream reuses it
                                torch.cuda.current_stream(llr.device).synchronize()
                        else:
                            q.hard, q.llr = q.bufs.hard_host, llr
                        ru.pool.append(q.bufs)
                        q.bufs = None
                self.in_use -= r.bytes
                for q in r.requests:
                    ru = self.rus.get(q.ru)
                    if ru is not None:
                        self._release_if_idle(ru)
                r.requests, r.buffers, r.bytes, r.event = [], [], 0, None
                n += 1
        return n

    def _form(self):
        """Pick waiting requests for one round: smallest radio units first
        (their slots can still meet the deadline), requests that waited
        longer than `starve_s` before all others, within the memory budget
        and the per-RU ordering rules."""
        chosen, nbytes = [], 0
        budget = self.mem_budget - self.in_use
        blocked_rus = set()
        keep = collections.deque()
        now = self.now()
        order = sorted(self.waiting, key=lambda q: (now - q.arrival <= self.starve_s,
                                                    self.rus[q.ru].cost, q.arrival))
        self.waiting = collections.deque(order)
        size_class = None
        large_ok = sum(1 for r in self.rounds if not r.free and r.big) < self.max_large_rounds
        while self.waiting and len(chosen) < self.max_units:
            q = self.waiting.popleft()
            ru = self.rus[q.ru]
            need = request_bytes(ru, q.kind, self.llr)
            ok = q.ru not in blocked_rus and nbytes + need <= budget
            # small and large units in separate rounds: a small unit's slot does
            # not wait for a large unit's walks in the same round
            big = ru.cost >= self.big_cost
            if ok and size_class is not None and big != size_class:
                ok = False
            if ok and big and not large_ok:
                ok = False
            if ok and q.kind == "slot":
                # the RU's channel update, if one is in flight in another
                # round (on another stream), is still rewriting the state this
                # slot reads: the slot waits until that round has finished
                # (an update formed into this same round runs its stages first)
                ok = ru.update_round < 0
            if ok and q.kind == "slot":
                # a free buffer set of the RU (its earlier slots in this round hold theirs)
                ok = len(ru.pool) > sum(1 for c in chosen if c.ru == q.ru and c.kind == "slot")
            if ok and q.kind == "channel":
                # the update rewrites the RU's state: no round in flight may
                # still read it, and no earlier slot of the RU may share this
                # round (its stages would see the new state)
                ok = not ru.busy_rounds and not any(c.ru == q.ru for c in chosen)
            if ok:
                chosen.append(q)
                nbytes += need
                size_class = big
            else:
                keep.append(q)
                blocked_rus.add(q.ru)  # the RU's later requests stay behind (per-RU order)
        keep.extend(self.waiting)
        self.waiting = collections.deque(sorted(keep, key=lambda q: q.arrival))
        return chosen, nbytes

    def _launch(self, r: _Round) -> bool:
        t_host = time.perf_counter()
        try:
            return self._launch_round(r)
        finally:
            self.host_launch_s += time.perf_counter() - t_host

    def _launch_round(self, r: _Round) -> bool:
        reqs, nbytes = self._form()
        if not reqs:
            return False
        dev = self.device
        t_adm = self.now()
        if r.batch is None:
            r.items = (mpnl.BatchItemC * self.max_units)()
        items = r.items
        big = any(self.rus[q.ru].cost >= self.big_cost for q in reqs)
        r.big = big
        st = r.stream_for(big)
        if big and self.large_per_unit:
            self._launch_per_unit(r, reqs, st, t_adm)
            self._finish_launch(r, reqs, nbytes)
            return True
        if r.batch is not None and self.native_rounds:
            self._launch_native(r, reqs, st, t_adm, big)
            self._finish_launch(r, reqs, nbytes)
            return True
        n = 0
        with torch.cuda.stream(st):
            # channel updates first in the item list (the batch runs stages in
            # order, so a slot of the same RU in this round sees the new state)
            for q in sorted(reqs, key=lambda q: q.kind != "channel"):
                ru = self.rus[q.ru]
                s_ = ru.state
                q.admitted = t_adm
                it = items[n]
                n += 1
                it.dims = mpnl.Dims(*ru.dims)
                it.sigma2 = ru.sigma2
                it.flags = self._unit_flags(ru)
                it.Q, it.R = s_["Q"].data_ptr(), s_["R"].data_ptr()
                it.inv_diag, it.perm = s_["inv_diag"].data_ptr(), s_["perm"].data_ptr()
                it.paths = s_["paths"].data_ptr()
                if q.kind == "channel":
                    ru.H_dev.copy_(q.payload, non_blocking=True)
                    it.stages = mpnl.STAGE_PREPROCESS | mpnl.STAGE_SELECT
                    it.H = ru.H_dev.data_ptr()
                    it.Y = it.Z = it.hard = it.llr = it.ped2 = None
                else:
                    b = ru.pool.pop()
                    q.bufs = b
                    b.Y.copy_(q.payload, non_blocking=True)
                    it.stages = mpnl.STAGE_QHY | mpnl.STAGE_DETECT
                    it.H = it.ped2 = None
                    it.Y, it.Z, it.hard = b.Y.data_ptr(), b.Z.data_ptr(), b.hard.data_ptr()
                    it.llr = b.llr.data_ptr() if b.llr is not None else None
                it.mmse_hard = it.mmse_llr = None
            if r.batch is None:
                # created once with room for a full round (padded with copies
                # of this round's first item, replaced right away)
                for k in range(n, self.max_units):
                    items[k] = items[0]
                r.batch = mpnl.Batch(items=list(items), device=dev)
            r.batch.reset((mpnl.BatchItemC * n).from_buffer(items), trusted_pointers=True)
            r.batch.run(mpnl.STAGE_PREPROCESS | mpnl.STAGE_SELECT | mpnl.STAGE_QHY |
                        mpnl.STAGE_DETECT, stream=st, share_sms=big and self.share_sms,
                        short_ctas=not big and self.small_short_ctas)
            for q in reqs:
                if q.bufs is not None:
                    q.bufs.hard_host.copy_(q.bufs.hard, non_blocking=True)
                    if q.bufs.llr_host is not None:
                        q.bufs.llr_host.copy_(q.bufs.llr, non_blocking=True)
            r.event = torch.cuda.Event()
            r.event.record(st)
        self._finish_launch(r, reqs, nbytes)
        return True

    def _launch_native(self, r: _Round, reqs, st, t_adm: float, big: bool) -> None:
        """A round as one mpnl_serve_round call: the inputs' copies, the
        batch's descriptors, the stages and the results' copies are all
        enqueued by the library; this side only names each request's buffers."""
        if getattr(r, "reqs_c", None) is None:
            r.reqs_c = (mpnl.RoundReqC * self.max_units)()
        rc = r.reqs_c
        for k, q in enumerate(reqs):
            ru = self.rus[q.ru]
            q.admitted = t_adm
            c = rc[k]
            c.unit = ctypes.pointer(ru.item)
            c.payload = q.payload.data_ptr()
            if q.kind == "channel":
                c.kind = mpnl.ROUND_CHANNEL
                c.staging = ru.H_dev.data_ptr()
                c.Z = c.hard = c.llr = c.hard_host = c.llr_host = None
            else:
                b = ru.pool.pop()
                q.bufs = b
                c.kind = mpnl.ROUND_SLOT
                c.staging, c.Z, c.hard = b.Y.data_ptr(), b.Z.data_ptr(), b.hard.data_ptr()
                c.hard_host = b.hard_host.data_ptr()
                c.llr = b.llr.data_ptr() if b.llr is not None else None
                c.llr_host = b.llr_host.data_ptr() if b.llr_host is not None else None
        flags = (mpnl.RUN_SHARE_SMS if big and self.share_sms else 0) \
            | (mpnl.RUN_SHORT_CTAS if not big and self.small_short_ctas else 0)
        r.batch.serve_round(rc, len(reqs), flags, stream=st)
        r.event = torch.cuda.Event()
        r.event.record(st)

    def _launch_per_unit(self, r: _Round, reqs, st, t_adm: float) -> None:
        """A large units' round as plain per-call launches (one CTA per
        subcarrier in the walks) instead of the persistent batch kernels:
        their CTAs are short, so the small units' rounds on the high-priority
        streams take SMs as the large units' CTAs retire instead of waiting
        for a persistent launch to drain."""
        with torch.cuda.stream(st):
            for q in sorted(reqs, key=lambda q: q.kind != "channel"):
                ru = self.rus[q.ru]
                s_ = ru.state
                q.admitted = t_adm
                s2 = ru.sigma2 if ru.mmse_qr else None
                if q.kind == "channel":
                    ru.H_dev.copy_(q.payload, non_blocking=True)
                    mpnl.factor(ru.H_dev, s2, out=(s_["Q"], s_["R"], s_["inv_diag"], s_["perm"]))
                    if ru.precision == "fp16":
                        mpnl.refine_qr(ru.H_dev, None, s_["R"], s_["inv_diag"], s_["perm"],
                                       Q=s_["Q"], sigma2=s2, cond_threshold=REFINE_COND)
                    mpnl.select_paths(s_["R"], ru.sigma2, ru.qam, ru.n_pe, ru.nt, out=s_["paths"])
                else:
                    b = ru.pool.pop()
                    q.bufs = b
                    b.Y.copy_(q.payload, non_blocking=True)
                    mpnl.qhy(s_["Q"], b.Y, out=b.Z, precision=ru.precision)
                    mpnl.detect(s_["R"], s_["inv_diag"], s_["perm"], s_["paths"], b.Z, ru.sigma2,
                                ru.qam, want_llr=b.llr is not None, want_ped2=False,
                                out=(b.hard, b.llr, None), precision=ru.precision)
                    b.hard_host.copy_(b.hard, non_blocking=True)
                    if b.llr_host is not None:
                        b.llr_host.copy_(b.llr, non_blocking=True)
            r.event = torch.cuda.Event()
            r.event.record(st)

    def _finish_launch(self, r: _Round, reqs, nbytes: int) -> None:
        self.n_rounds += 1
        r.round_id = self.n_rounds
        for q in reqs:
            q.round_id = r.round_id
            self.rus[q.ru].busy_rounds.add(r.round_id)
            if q.kind == "channel":
                self.rus[q.ru].update_round = r.round_id
        r.requests, r.bytes = reqs, nbytes
        self.in_use += nbytes
        self.peak_in_use = max(self.peak_in_use, self.in_use)
        self.round_sizes.append(len(reqs))

    def step(self) -> None:
        self.poll()
        for r in self.rounds:
            if not self.waiting:
                break
            if r.free:
                self._launch(r)

    def drain(self, timeout_s: float = 60.0) -> None:
        t_end = time.perf_counter() + timeout_s
        while (self.waiting or any(not r.free for r in self.rounds)) and time.perf_counter() < t_end:
            self.step()

    @property
    def split(self):
        """The SM split of the two size classes (None without one)."""
        if self.sm_split and self._split is None:
            self._split = mpnl.SmSplit.get(self.sm_split, self.device)
            self.split_sms = self._split.sms
        return self._split

    def close(self) -> None:
        torch.cuda.synchronize(self.device)
        for r in self.rounds:
            if r.batch is not None:
                r.batch.close()
                r.batch = None
            r._streams.clear()
        self._split = None   # kept by the process (mpnl.SmSplit.get)


# ---------------------------------------------------------------------------
# workload: RUs, payloads and Poisson arrivals
# ---------------------------------------------------------------------------
def serving_units(n_rus: int = 200, big_fraction: float = 0.2, seed: int | None = None,
                  sc_scale: float = 1.0) -> list[inputs.UnitSpec]:
    """RU sizes as in the mixed batch; a fraction of them 16x16 64-QAM with
    3276 subcarriers (N_pe drawn as in the mixed batch)."""
    units = inputs.mixed_units(n_rus, seed=seed, sc_scale=sc_scale, config=5)
    rng = np.random.Generator(np.random.PCG64(inputs.seed_for(5, 1) if seed is None else seed + 1))
    big = rng.choice(n_rus, size=int(round(big_fraction * n_rus)), replace=False)
    for k in big:
        u = units[k]
        units[k] = inputs.UnitSpec(16, 16, 64, max(1, int(round(3276 * sc_scale))),
                                   u.n_pe, 20.0 + 6.0 * rng.random(), u.channel, u.seed)
    return units


def poisson_trace(units, rate_per_s: float, duration_s: float, coherence_slots: int = 8,
                  seed: int = 0):
    """Arrival times and RUs of slot requests (Poisson, RU chosen uniformly);
    every `coherence_slots`-th slot of an RU is preceded by a channel update
    arriving with it."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = rng.poisson(rate_per_s * duration_s)
    times = np.sort(rng.uniform(0.0, duration_s, size=n))
    rus = rng.integers(0, len(units), size=n)
    count = np.zeros(len(units), dtype=np.int64)
    out = []
    for t, k in zip(times, rus):
        if count[k] % coherence_slots == coherence_slots - 1:
            out.append((float(t), int(k), "channel"))
        out.append((float(t), int(k), "slot"))
        count[k] += 1
    return out


def run_trace(server: Server, trace, payloads, t_limit_s: float = 120.0):
    """Replay `trace` in real time: requests are submitted at their arrival
    times (relative to the start) and the loop runs until all complete.
    payloads[ru][kind] -> list of pinned host tensors, used cyclically."""
    use = collections.defaultdict(int)
    reqs = []
    server.t0 = time.perf_counter()
    i = 0
    t_end = time.perf_counter() + t_limit_s
    while (i < len(trace) or server.waiting or any(not r.free for r in server.rounds)) \
            and time.perf_counter() < t_end:
        now = server.now()
        while i < len(trace) and trace[i][0] <= now:
            t, k, kind = trace[i]
            pl = payloads[k][kind]
            q = Request(len(reqs), k, kind, t, pl[use[(k, kind)] % len(pl)])
            use[(k, kind)] += 1
            reqs.append(q)
            server.submit(q)
            i += 1
        server.step()
    return reqs


def latency_stats(reqs, deadline_s: float = DEADLINE_S, dets_of=None, big_of=None) -> dict:
    """p50/p99 latency and deadline-miss rate of the completed slot requests;
    with big_of (request -> bool) also per size class."""
    def stats(slots):
        lat = np.array([q.done - q.arrival for q in slots]) if slots else np.zeros(0)
        return {"slots_done": len(slots),
                "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
                "miss_rate": float(np.mean(lat > deadline_s)) if len(lat) else None}

    slots = [q for q in reqs if q.kind == "slot" and q.done >= 0]
    out = {"requests": len(reqs), **stats(slots)}
    if dets_of is not None and slots:
        span = max(q.done for q in slots) - min(q.arrival for q in slots)
        out["detections_per_s"] = sum(dets_of(q) for q in slots) / max(span, 1e-9)
    if big_of is not None:
        out["large_units"] = stats([q for q in slots if big_of(q)])
        out["small_units"] = stats([q for q in slots if not big_of(q)])
    return out
