"""Python binding of libmpnl.so (include/mpnl.h): argument marshalling only.

Every step of the detection path runs in the CUDA kernels behind the C ABI;
this module allocates output tensors with PyTorch, passes raw device
pointers and the current CUDA stream, and turns error codes into
exceptions.  There is no CPU fallback: if the library is missing or no GPU is
present, every call raises.

Layouts (complex = torch.complex64, interleaved re/im float32):
  H [n_sc][nr][nt], Y [n_sc][n_sym][nr]          inputs
  R [n_sc][nt(nt+1)/2] packed upper triangle     preprocess output
  inv_diag f32 [n_sc][nt], perm u8 [n_sc][nt], Z [n_sc][n_sym][nt]
  paths u8 [n_sc][n_pe][nt] (ranks 1..qam)
  hard u8 [n_sc][n_sym][nt], llr f32 [n_sc][n_sym][nt][log2 qam],
  ped2 f32 [n_sc][n_sym][2]
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmpnl.so")
BITS = {4: 2, 16: 4, 64: 6}
LLR_MAX = 20.0
MAX_NT, MAX_NR, MAX_NSYM, MAX_NPE = 16, 32, 32, 1024

OK = 0
ERR_INVALID_ARG = -1
ERR_UNSUPPORTED = -2
ERR_CUDA = -3
ERR_TIMEOUT = -4

EXPORTED = ("mpnl_create", "mpnl_destroy", "mpnl_last_error", "mpnl_workspace_bytes",
            "mpnl_preprocess", "mpnl_preprocess_mmse", "mpnl_select_paths", "mpnl_detect",
            "mpnl_detect_mixed",
            "mpnl_linear_mmse", "mpnl_check_status", "mpnl_set_tuning",
            "mpnl_get_tuning", "mpnl_batch_create", "mpnl_batch_run", "mpnl_batch_destroy",
            "mpnl_batch_reset", "mpnl_factor", "mpnl_qhy", "mpnl_refine_qr",
            "mpnl_select_paths_lut", "mpnl_rank_counts", "mpnl_rank_costs",
            "mpnl_rvd_embed", "mpnl_select_paths_pam", "mpnl_detect_rvd", "mpnl_qhy_mixed",
            "mpnl_detect_units_noalloc", "mpnl_detect_slot", "mpnl_slot_workspace_bytes",
            "mpnl_serve_round", "mpnl_sm_split_create", "mpnl_sm_split_stream",
            "mpnl_sm_split_destroy")
ITEM_MMSE_QR, ITEM_LINEAR_MMSE, ITEM_FP16, ITEM_REFINE_QR = 1, 2, 4, 8
STAGE_PREPROCESS, STAGE_SELECT, STAGE_DETECT, STAGE_MMSE, STAGE_QHY = 1, 2, 4, 8, 32
STAGES_ALL = 47
RUN_GRAPH = 16
RUN_SHARE_SMS = 64
RUN_SHORT_CTAS = 128
RESET_TRUSTED_POINTERS = 1
NOALLOC_MAX_UNITS = 64
SLOT_MMSE, SLOT_FP16, SLOT_MMSE_QR = 1, 2, 4
PRECISIONS = ("fp32", "fp16")


class RankLutC(ctypes.Structure):
    """mpnl_rank_lut."""
    _fields_ = [("qam", ctypes.c_int), ("n_bins", ctypes.c_int),
                ("edges", ctypes.c_void_p), ("cost", ctypes.c_void_p)]


class MpnlError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mpnl error {code}: {msg}")
        self.code = code


class Dims(ctypes.Structure):
    _fields_ = [("n_sc", ctypes.c_int), ("n_sym", ctypes.c_int), ("nr", ctypes.c_int),
                ("nt", ctypes.c_int), ("qam", ctypes.c_int), ("n_pe", ctypes.c_int)]


_lib = None
_lib_lock = threading.Lock()
_ctxs: dict[int, ctypes.c_void_p] = {}


class Tuning(ctypes.Structure):
    """Launch-shape knobs (mpnl_tuning): [nt class][qam class][N_pe class],
    0 = built-in choice.  Results never depend on them."""
    _fields_ = [("detect_sym", ((ctypes.c_uint8 * 2) * 3) * 3),
                ("select_warps", ((ctypes.c_uint8 * 2) * 3) * 3),
                ("persistent_ctas_per_sm", ctypes.c_uint8),
                ("persistent_select_warps", ctypes.c_uint8)]


ROUND_SLOT, ROUND_CHANNEL = 0, 1


class BatchItemC(ctypes.Structure):
    """mpnl_batch_item."""
    _fields_ = [("dims", Dims), ("sigma2", ctypes.c_float), ("flags", ctypes.c_int),
                ("stages", ctypes.c_int), ("Q", ctypes.c_void_p)] + [
        (n, ctypes.c_void_p) for n in ("H", "Y", "R", "inv_diag", "perm", "Z", "paths", "hard",
                                       "llr", "ped2", "mmse_hard", "mmse_llr")]


class RoundReqC(ctypes.Structure):
    """mpnl_round_req: one request of a serving round (mpnl_serve_round)."""
    _fields_ = [("unit", ctypes.POINTER(BatchItemC)), ("kind", ctypes.c_int)] + [
        (n, ctypes.c_void_p) for n in ("payload", "staging", "Z", "hard", "llr", "hard_host",
                                       "llr_host")]


def problem_class(nt: int, qam: int, n_pe: int) -> tuple[int, int, int]:
    """Index of a problem in the Tuning tables."""
    return (0 if nt <= 4 else (1 if nt <= 8 else 2), {4: 0, 16: 1, 64: 2}[qam],
            1 if n_pe >= 256 else 0)


def load_library(path: str = LIB_PATH):
    """Load libmpnl.so and declare its signatures (no GPU needed)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise MpnlError(ERR_CUDA, f"{path} not built: run paper_2409_14355_gb300.build.build()")
        lib = ctypes.CDLL(path)
        P, I, F, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
        D = ctypes.POINTER(Dims)
        lib.mpnl_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), I]
        lib.mpnl_create.restype = I
        lib.mpnl_destroy.argtypes = [P]
        lib.mpnl_destroy.restype = None
        lib.mpnl_last_error.argtypes = [P]
        lib.mpnl_last_error.restype = ctypes.c_char_p
        lib.mpnl_workspace_bytes.argtypes = [D]
        lib.mpnl_workspace_bytes.restype = S
        lib.mpnl_preprocess.argtypes = [P, D, P, P, P, P, P, P, P, P]
        lib.mpnl_preprocess.restype = I
        lib.mpnl_preprocess_mmse.argtypes = [P, D, P, P, F, P, P, P, P, P, P]
        lib.mpnl_preprocess_mmse.restype = I
        lib.mpnl_select_paths.argtypes = [P, D, P, F, P, P, P]
        lib.mpnl_select_paths.restype = I
        lib.mpnl_select_paths_lut.argtypes = [P, D, P, F, ctypes.POINTER(RankLutC), P, P, P]
        lib.mpnl_select_paths_lut.restype = I
        LL, ULL = ctypes.c_longlong, ctypes.c_ulonglong
        lib.mpnl_rank_counts.argtypes = [P, I, I, P, LL, ULL, P, P]
        lib.mpnl_rank_counts.restype = I
        lib.mpnl_rank_costs.argtypes = [P, I, I, P, LL, P, P]
        lib.mpnl_rank_costs.restype = I
        lib.mpnl_rvd_embed.argtypes = [P, D, P, P, P, P, P]
        lib.mpnl_rvd_embed.restype = I
        lib.mpnl_select_paths_pam.argtypes = [P, D, P, F, P, P, P]
        lib.mpnl_select_paths_pam.restype = I
        lib.mpnl_detect_rvd.argtypes = [P, D, P, P, P, P, P, F, P, P, P, P, P]
        lib.mpnl_detect_rvd.restype = I
        lib.mpnl_detect.argtypes = [P, D, P, P, P, P, P, F, P, P, P, P, P]
        lib.mpnl_detect.restype = I
        lib.mpnl_detect_mixed.argtypes = [P, D, P, P, P, P, P, F, P, P, P, P, P]
        lib.mpnl_detect_mixed.restype = I
        lib.mpnl_linear_mmse.argtypes = [P, D, P, P, F, P, P, P, P]
        lib.mpnl_linear_mmse.restype = I
        lib.mpnl_check_status.argtypes = [P, P]
        lib.mpnl_check_status.restype = I
        lib.mpnl_batch_create.argtypes = [P, ctypes.POINTER(BatchItemC), I,
                                          ctypes.POINTER(ctypes.c_void_p)]
        lib.mpnl_batch_create.restype = I
        lib.mpnl_batch_reset.argtypes = [P, P, ctypes.POINTER(BatchItemC), I, I]
        lib.mpnl_batch_reset.restype = I
        lib.mpnl_factor.argtypes = [P, D, P, F, P, P, P, P, P, P]
        lib.mpnl_factor.restype = I
        lib.mpnl_refine_qr.argtypes = [P, D, P, P, F, F, P, P, P, P, P, P, P, P]
        lib.mpnl_refine_qr.restype = I
        lib.mpnl_qhy.argtypes = [P, D, P, P, P, P, P]
        lib.mpnl_qhy.restype = I
        lib.mpnl_qhy_mixed.argtypes = [P, D, P, P, P, P, P]
        lib.mpnl_qhy_mixed.restype = I
        lib.mpnl_batch_run.argtypes = [P, P, I, P]
        lib.mpnl_batch_run.restype = I
        lib.mpnl_batch_destroy.argtypes = [P]
        lib.mpnl_batch_destroy.restype = None
        lib.mpnl_detect_units_noalloc.argtypes = [ctypes.POINTER(BatchItemC), I, P]
        lib.mpnl_detect_units_noalloc.restype = I
        lib.mpnl_serve_round.argtypes = [P, P, ctypes.POINTER(RoundReqC), I, I, P]
        lib.mpnl_serve_round.restype = I
        lib.mpnl_slot_workspace_bytes.argtypes = [D, I]
        lib.mpnl_slot_workspace_bytes.restype = S
        lib.mpnl_detect_slot.argtypes = [P, D, F, P, P, P, P, P, P, P, I, P, S, P]
        lib.mpnl_detect_slot.restype = I
        lib.mpnl_sm_split_create.argtypes = [P, I, ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.POINTER(I)]
        lib.mpnl_sm_split_create.restype = I
        lib.mpnl_sm_split_stream.argtypes = [P, P, I, I, ctypes.POINTER(ctypes.c_void_p)]
        lib.mpnl_sm_split_stream.restype = I
        lib.mpnl_sm_split_destroy.argtypes = [P, P]
        lib.mpnl_sm_split_destroy.restype = I
        lib.mpnl_set_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
        lib.mpnl_set_tuning.restype = I
        lib.mpnl_get_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
        lib.mpnl_get_tuning.restype = I
        _lib = lib
        return lib


def context(device: int | None = None) -> ctypes.c_void_p:
    """The per-device mpnl_ctx (created on first use, kept for the process)."""
    lib = load_library()
    if not torch.cuda.is_available():
        raise MpnlError(ERR_CUDA, "no CUDA device: the MPNL path has no CPU fallback")
    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _ctxs:
        h = ctypes.c_void_p()
        st = lib.mpnl_create(ctypes.byref(h), dev)
        if st != OK:
            raise MpnlError(st, f"mpnl_create(device={dev}) failed")
        _ctxs[dev] = h
    return _ctxs[dev]


class SmSplit:
    """mpnl_sm_split_*: the device's SMs in two disjoint groups (CUDA green
    contexts), group 0 of at least `sms_first` SMs and group 1 the rest;
    `stream(part)` gives a torch stream whose kernels run on that group's SMs
    only.  One split per (device, sms_first) is made per process
    (`SmSplit.get`) and kept, with its streams, for the life of the process,
    as torch keeps its own streams: torch records events on the streams it
    uses (caching allocators, copies from pinned memory) and may touch them
    long after, so neither the streams nor their green contexts may go away
    under it.  `sync()` waits for the work on the split's streams."""

    _cache: dict = {}

    def __init__(self, sms_first: int, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self._ctx = context(self.device.index)
        self._h = ctypes.c_void_p()
        sms = (ctypes.c_int * 2)()
        _raise(load_library().mpnl_sm_split_create(self._ctx, int(sms_first),
                                                   ctypes.byref(self._h), sms), self._ctx)
        self.sms = (int(sms[0]), int(sms[1]))
        self._streams: dict = {}

    @classmethod
    def get(cls, sms_first: int, device=None) -> "SmSplit":
        dev = torch.cuda.current_device() if device is None else torch.device(device).index or 0
        key = (dev, int(sms_first))
        if key not in cls._cache:
            cls._cache[key] = cls(sms_first, dev)
        return cls._cache[key]

    def stream(self, part: int, priority: int = 0, index: int = 0) -> torch.cuda.ExternalStream:
        """The index-th stream of group `part` at `priority` (made on first
        request, then the same one)."""
        key = (int(part), int(priority), int(index))
        if key not in self._streams:
            p = ctypes.c_void_p()
            _raise(load_library().mpnl_sm_split_stream(self._ctx, self._h, key[0], key[1],
                                                       ctypes.byref(p)), self._ctx)
            self._streams[key] = torch.cuda.ExternalStream(p.value, device=self.device)
        return self._streams[key]

    def sync(self) -> None:
        for st in self._streams.values():
            st.synchronize()


def _raise(st: int, ctx) -> None:
    if st != OK:
        msg = load_library().mpnl_last_error(ctx).decode(errors="replace")
        raise MpnlError(st, msg)


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t) -> ctypes.c_void_p | None:
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev_of(t: torch.Tensor) -> torch.device:
    if t.device.type != "cuda":
        raise MpnlError(ERR_INVALID_ARG, "tensor must live on a CUDA device")
    return t.device


def _need(t: torch.Tensor, dtype, shape, name):
    if t.dtype != dtype:
        raise MpnlError(ERR_INVALID_ARG, f"{name}: dtype {t.dtype}, expected {dtype}")
    if tuple(t.shape) != tuple(shape):
        raise MpnlError(ERR_INVALID_ARG, f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise MpnlError(ERR_INVALID_ARG, f"{name}: must be contiguous")


def workspace_bytes(n_sc, n_sym, nr, nt, qam, n_pe) -> int:
    d = Dims(n_sc, n_sym, nr, nt, qam, n_pe)
    return int(load_library().mpnl_workspace_bytes(ctypes.byref(d)))


def preprocess(H: torch.Tensor, Y: torch.Tensor, out=None, sigma2: float | None = None):
    """Sorted QR + z = Q^H y.  Returns (R, inv_diag, perm, Z).  With sigma2,
    the MMSE-extended factorisation of [H; sqrt(sigma2) I] (allows nt > nr)."""
    dev = _dev_of(H)
    n_sc, nr, nt = H.shape
    n_sym = Y.shape[1]
    _need(H, torch.complex64, (n_sc, nr, nt), "H")
    _need(Y, torch.complex64, (n_sc, n_sym, nr), "Y")
    if out is None:
        R = torch.empty((n_sc, nt * (nt + 1) // 2), dtype=torch.complex64, device=dev)
        inv_diag = torch.empty((n_sc, nt), dtype=torch.float32, device=dev)
        perm = torch.empty((n_sc, nt), dtype=torch.uint8, device=dev)
        Z = torch.empty((n_sc, n_sym, nt), dtype=torch.complex64, device=dev)
    else:
        R, inv_diag, perm, Z = out
    ctx = context(dev.index)
    d = Dims(n_sc, n_sym, nr, nt, 4, 1)
    lib = load_library()
    if sigma2 is None:
        st = lib.mpnl_preprocess(ctx, ctypes.byref(d), _ptr(H), _ptr(Y), _ptr(R), _ptr(inv_diag),
                                 _ptr(perm), _ptr(Z), None, _stream(dev))
    else:
        st = lib.mpnl_preprocess_mmse(ctx, ctypes.byref(d), _ptr(H), _ptr(Y), float(sigma2),
                                      _ptr(R), _ptr(inv_diag), _ptr(perm), _ptr(Z), None,
                                      _stream(dev))
    _raise(st, ctx)
    return R, inv_diag, perm, Z


def factor(H: torch.Tensor, sigma2: float | None = None, out=None):
    """Sorted QR keeping Q: returns (Q [n_sc][nr][nt], R, inv_diag, perm).
    With sigma2 the MMSE-extended factor of [H; sqrt(sigma2) I]."""
    dev = _dev_of(H)
    n_sc, nr, nt = H.shape
    _need(H, torch.complex64, (n_sc, nr, nt), "H")
    if out is None:
        out = (torch.empty((n_sc, nr, nt), dtype=torch.complex64, device=dev),
               torch.empty((n_sc, nt * (nt + 1) // 2), dtype=torch.complex64, device=dev),
               torch.empty((n_sc, nt), dtype=torch.float32, device=dev),
               torch.empty((n_sc, nt), dtype=torch.uint8, device=dev))
    Q, R, inv_diag, perm = out
    ctx = context(dev.index)
    d = Dims(n_sc, 1, nr, nt, 4, 1)
    st = load_library().mpnl_factor(ctx, ctypes.byref(d), _ptr(H), float(sigma2 or 0.0), _ptr(Q),
                                    _ptr(R), _ptr(inv_diag), _ptr(perm), None, _stream(dev))
    _raise(st, ctx)
    return Q, R, inv_diag, perm


def refine_qr(H, Y, R, inv_diag, perm, Z=None, Q=None, sigma2: float | None = None,
              cond_threshold: float = 1e3, count: torch.Tensor | None = None) -> None:
    """FP64 re-factorisation, in place, of the subcarriers whose FP32 R has
    max R_ll / min R_ll above cond_threshold.  `count` (device int32 [1])
    receives the number redone."""
    dev = _dev_of(H)
    n_sc, nr, nt = H.shape
    n_sym = Y.shape[1] if Y is not None else 1
    ctx = context(dev.index)
    d = Dims(n_sc, n_sym, nr, nt, 4, 1)
    _raise(load_library().mpnl_refine_qr(ctx, ctypes.byref(d), _ptr(H), _ptr(Y),
                                         float(sigma2 or 0.0), float(cond_threshold), _ptr(R),
                                         _ptr(inv_diag), _ptr(perm), _ptr(Z), _ptr(Q),
                                         _ptr(count), None, _stream(dev)), ctx)


def qhy(Q: torch.Tensor, Y: torch.Tensor, out=None, precision: str = "fp32"):
    """z = Q^H y for every symbol (Q from factor).  precision "fp16":
    mpnl_qhy_mixed (tensor cores, FP16 operands, FP32 accumulation)."""
    if precision not in PRECISIONS:
        raise MpnlError(ERR_INVALID_ARG, f"precision {precision!r} not in {PRECISIONS}")
    dev = _dev_of(Q)
    n_sc, nr, nt = Q.shape
    n_sym = Y.shape[1]
    _need(Q, torch.complex64, (n_sc, nr, nt), "Q")
    _need(Y, torch.complex64, (n_sc, n_sym, nr), "Y")
    Z = out if out is not None else torch.empty((n_sc, n_sym, nt), dtype=torch.complex64, device=dev)
    ctx = context(dev.index)
    d = Dims(n_sc, n_sym, nr, nt, 4, 1)
    fn = load_library().mpnl_qhy_mixed if precision == "fp16" else load_library().mpnl_qhy
    _raise(fn(ctx, ctypes.byref(d), _ptr(Q), _ptr(Y), _ptr(Z), None, _stream(dev)), ctx)
    return Z


def select_paths(R: torch.Tensor, sigma2: float, qam: int, n_pe: int, nt: int, out=None):
    """Position-vector table u8 [n_sc][n_pe][nt] from the R diagonal."""
    dev = _dev_of(R)
    n_sc = R.shape[0]
    _need(R, torch.complex64, (n_sc, nt * (nt + 1) // 2), "R")
    paths = out if out is not None else torch.empty((n_sc, n_pe, nt), dtype=torch.uint8, device=dev)
    ctx = context(dev.index)
    d = Dims(n_sc, 1, nt, nt, qam, n_pe)
    st = load_library().mpnl_select_paths(ctx, ctypes.byref(d), _ptr(R), float(sigma2),
                                          _ptr(paths), None, _stream(dev))
    _raise(st, ctx)
    return paths


def rank_counts(qam: int, gamma: torch.Tensor, n_trials: int, seed: int, out=None):
    """Monte-Carlo rank histogram u64 (as int64) [n_bins][qam] for the linear
    SNRs `gamma` (f64 device tensor) (mpnl_rank_counts)."""
    dev = _dev_of(gamma)
    _need(gamma, torch.float64, (gamma.shape[0],), "gamma")
    n_bins = gamma.shape[0]
    counts = out if out is not None else torch.empty((n_bins, qam), dtype=torch.int64, device=dev)
    ctx = context(dev.index)
    _raise(load_library().mpnl_rank_counts(ctx, qam, n_bins, _ptr(gamma), int(n_trials),
                                           ctypes.c_ulonglong(seed), _ptr(counts), _stream(dev)),
           ctx)
    return counts


def rank_costs(counts: torch.Tensor, n_trials: int, out=None):
    """Rank costs f32 [n_bins][qam] from a histogram (mpnl_rank_costs)."""
    dev = _dev_of(counts)
    n_bins, qam = counts.shape
    _need(counts, torch.int64, (n_bins, qam), "counts")
    cost = out if out is not None else torch.empty((n_bins, qam), dtype=torch.float32, device=dev)
    ctx = context(dev.index)
    _raise(load_library().mpnl_rank_costs(ctx, qam, n_bins, _ptr(counts), int(n_trials),
                                          _ptr(cost), _stream(dev)), ctx)
    return cost


class RankLut:
    """A rank-cost table on the device: `edges` f32 [n_bins - 1] (ascending
    linear SNRs) and `cost` f32 [n_bins][qam]."""

    def __init__(self, qam: int, edges: torch.Tensor, cost: torch.Tensor):
        self.qam = qam
        self.edges = edges
        self.cost = cost
        self.n_bins = cost.shape[0]
        if edges.shape[0] != self.n_bins - 1 or cost.shape[1] != qam:
            raise ValueError("edges must hold n_bins - 1 values and cost [n_bins][qam]")

    @classmethod
    def build(cls, qam: int, db_min: float = -10.0, db_max: float = 40.0, db_step: float = 0.5,
              n_trials: int = 1 << 20, seed: int = 0x2409_14355, device=None) -> "RankLut":
        """Bins centred every db_step dB from db_min to db_max, the edges
        half-way between centres (in dB); costs from n_trials Monte-Carlo
        trials per bin, on the GPU."""
        dev = torch.device("cuda", torch.cuda.current_device() if device is None
                           else torch.device(device).index or 0)
        n_bins = int(round((db_max - db_min) / db_step)) + 1
        centres = [db_min + b * db_step for b in range(n_bins)]
        gamma = torch.tensor([10.0 ** (c / 10.0) for c in centres], dtype=torch.float64,
                             device=dev)
        edges = torch.tensor([10.0 ** ((c + 0.5 * db_step) / 10.0) for c in centres[:-1]],
                             dtype=torch.float32, device=dev)
        with torch.cuda.device(dev):
            counts = rank_counts(qam, gamma, n_trials, seed)
            cost = rank_costs(counts, n_trials)
        lut = cls(qam, edges, cost)
        lut.counts, lut.gamma = counts, gamma
        return lut

    def c_struct(self) -> RankLutC:
        return RankLutC(self.qam, self.n_bins,
                        self.edges.data_ptr() if self.edges.numel() else None,
                        self.cost.data_ptr())


def select_paths_lut(R: torch.Tensor, sigma2: float, lut: RankLut, n_pe: int, nt: int, out=None):
    """Position-vector table u8 [n_sc][n_pe][nt] under the table-driven rank
    model (mpnl_select_paths_lut)."""
    dev = _dev_of(R)
    n_sc = R.shape[0]
    _need(R, torch.complex64, (n_sc, nt * (nt + 1) // 2), "R")
    paths = out if out is not None else torch.empty((n_sc, n_pe, nt), dtype=torch.uint8, device=dev)
    ctx = context(dev.index)
    d = Dims(n_sc, 1, nt, nt, lut.qam, n_pe)
    c = lut.c_struct()
    _raise(load_library().mpnl_select_paths_lut(ctx, ctypes.byref(d), _ptr(R), float(sigma2),
                                                ctypes.byref(c), _ptr(paths), None, _stream(dev)),
           ctx)
    return paths


def rvd_embed(H: torch.Tensor, Y: torch.Tensor, out=None):
    """Real-valued decomposition of a slot (mpnl_rvd_embed): returns
    (Hr [n_sc][2nr][2nt], Yr [n_sc][n_sym][2nr]), complex with zero imaginary
    parts, ready for preprocess()."""
    dev = _dev_of(H)
    n_sc, nr, nt = H.shape
    n_sym = Y.shape[1]
    _need(H, torch.complex64, (n_sc, nr, nt), "H")
    _need(Y, torch.complex64, (n_sc, n_sym, nr), "Y")
    if out is None:
        Hr = torch.empty((n_sc, 2 * nr, 2 * nt), dtype=torch.complex64, device=dev)
        Yr = torch.empty((n_sc, n_sym, 2 * nr), dtype=torch.complex64, device=dev)
    else:
        Hr, Yr = out
    ctx = context(dev.index)
    d = Dims(n_sc, n_sym, nr, nt, 4, 1)
    _raise(load_library().mpnl_rvd_embed(ctx, ctypes.byref(d), _ptr(H), _ptr(Y), _ptr(Hr),
                                         _ptr(Yr), _stream(dev)), ctx)
    return Hr, Yr


def select_paths_pam(R: torch.Tensor, sigma2: float, qam: int, n_pe: int, nt: int, out=None):
    """Position vectors over the 2 nt real levels (ranks 1..sqrt qam),
    u8 [n_sc][n_pe][2nt] (mpnl_select_paths_pam); nt = users."""
    dev = _dev_of(R)
    n_sc = R.shape[0]
    ntr = 2 * nt
    _need(R, torch.complex64, (n_sc, ntr * (ntr + 1) // 2), "R")
    paths = out if out is not None else torch.empty((n_sc, n_pe, ntr), dtype=torch.uint8,
                                                    device=dev)
    ctx = context(dev.index)
    d = Dims(n_sc, 1, nt, nt, qam, n_pe)
    _raise(load_library().mpnl_select_paths_pam(ctx, ctypes.byref(d), _ptr(R), float(sigma2),
                                                _ptr(paths), None, _stream(dev)), ctx)
    return paths


def detect_rvd(R, inv_diag, perm, paths, Z, sigma2: float, qam: int, want_llr: bool = True,
               want_ped2: bool = True, out=None):
    """Walks over the real levels (mpnl_detect_rvd); R, inv_diag, perm, paths,
    Z over 2 nt levels.  Returns (hard [n_sc][n_sym][nt], llr or None, ped2
    or None) in the complex users' layout."""
    dev = _dev_of(R)
    n_sc, n_sym, ntr = Z.shape
    nt = ntr // 2
    n_pe = paths.shape[1]
    B = BITS[qam]
    _need(paths, torch.uint8, (n_sc, n_pe, ntr), "paths")
    if out is None:
        hard = torch.empty((n_sc, n_sym, nt), dtype=torch.uint8, device=dev)
        llr = torch.empty((n_sc, n_sym, nt, B), dtype=torch.float32, device=dev) if want_llr else None
        ped2 = torch.empty((n_sc, n_sym, 2), dtype=torch.float32, device=dev) if want_ped2 else None
    else:
        hard, llr, ped2 = out
    ctx = context(dev.index)
    d = Dims(n_sc, n_sym, nt, nt, qam, n_pe)
    _raise(load_library().mpnl_detect_rvd(ctx, ctypes.byref(d), _ptr(R), _ptr(inv_diag),
                                          _ptr(perm), _ptr(paths), _ptr(Z), float(sigma2),
                                          _ptr(hard), _ptr(llr), _ptr(ped2), None, _stream(dev)),
           ctx)
    return hard, llr, ped2


def run_slot_rvd(H: torch.Tensor, Y: torch.Tensor, sigma2: float, qam: int, n_pe: int) -> dict:
    """The real-valued path over a slot on device tensors: embedding, sorted
    QR of the real matrix + z, PAM-level selection, walks."""
    Hr, Yr = rvd_embed(H, Y)
    R, inv_diag, perm, Z = preprocess(Hr, Yr)
    nt = H.shape[2]
    paths = select_paths_pam(R, sigma2, qam, n_pe, nt)
    hard, llr, ped2 = detect_rvd(R, inv_diag, perm, paths, Z, sigma2, qam)
    return dict(hard=hard, llr=llr, ped2=ped2, R=R, inv_diag=inv_diag, perm=perm, Z=Z,
                paths=paths, Hr=Hr, Yr=Yr)


def detect(R, inv_diag, perm, paths, Z, sigma2: float, qam: int, want_llr: bool = True,
           want_ped2: bool = True, out=None, precision: str = "fp32"):
    """Walks + argmin + max-log LLRs.  Returns (hard, llr or None, ped2 or None).
    precision "fp16" selects mpnl_detect_mixed (FP16 residuals, FP32 ranking,
    PED and re-check of the best and runner-up paths)."""
    if precision not in PRECISIONS:
        raise MpnlError(ERR_INVALID_ARG, f"precision {precision!r} not in {PRECISIONS}")
    dev = _dev_of(R)
    n_sc, n_sym, nt = Z.shape
    n_pe = paths.shape[1]
    B = BITS[qam]
    _need(R, torch.complex64, (n_sc, nt * (nt + 1) // 2), "R")
    _need(inv_diag, torch.float32, (n_sc, nt), "inv_diag")
    _need(perm, torch.uint8, (n_sc, nt), "perm")
    _need(paths, torch.uint8, (n_sc, n_pe, nt), "paths")
    _need(Z, torch.complex64, (n_sc, n_sym, nt), "Z")
    if out is None:
        hard = torch.empty((n_sc, n_sym, nt), dtype=torch.uint8, device=dev)
        llr = torch.empty((n_sc, n_sym, nt, B), dtype=torch.float32, device=dev) if want_llr else None
        ped2 = torch.empty((n_sc, n_sym, 2), dtype=torch.float32, device=dev) if want_ped2 else None
    else:
        hard, llr, ped2 = out
    ctx = context(dev.index)
    d = Dims(n_sc, n_sym, nt, nt, qam, n_pe)
    lib = load_library()
    fn = lib.mpnl_detect if precision == "fp32" else lib.mpnl_detect_mixed
    st = fn(ctx, ctypes.byref(d), _ptr(R), _ptr(inv_diag), _ptr(perm), _ptr(paths), _ptr(Z),
            float(sigma2), _ptr(hard), _ptr(llr), _ptr(ped2), None, _stream(dev))
    _raise(st, ctx)
    return hard, llr, ped2


def linear_mmse(H, Y, sigma2: float, qam: int, want_llr: bool = True, out=None):
    """Linear MMSE baseline.  Returns (hard, llr or None)."""
    dev = _dev_of(H)
    n_sc, nr, nt = H.shape
    n_sym = Y.shape[1]
    B = BITS[qam]
    _need(H, torch.complex64, (n_sc, nr, nt), "H")
    _need(Y, torch.complex64, (n_sc, n_sym, nr), "Y")
    if out is None:
        hard = torch.empty((n_sc, n_sym, nt), dtype=torch.uint8, device=dev)
        llr = torch.empty((n_sc, n_sym, nt, B), dtype=torch.float32, device=dev) if want_llr else None
    else:
        hard, llr = out
    ctx = context(dev.index)
    d = Dims(n_sc, n_sym, nr, nt, qam, 1)
    st = load_library().mpnl_linear_mmse(ctx, ctypes.byref(d), _ptr(H), _ptr(Y), float(sigma2),
                                         _ptr(hard), _ptr(llr), None, _stream(dev))
    _raise(st, ctx)
    return hard, llr


def check_status(device: int | None = None) -> None:
    """Synchronise the current stream and raise on device-side argument errors."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    ctx = context(dev.index)
    _raise(load_library().mpnl_check_status(ctx, _stream(dev)), ctx)


def set_tuning(tuning: Tuning | None, device: int | None = None) -> None:
    """Install launch-shape knobs on the device's context (None: built-in)."""
    dev = torch.cuda.current_device() if device is None else device
    ctx = context(dev)
    _raise(load_library().mpnl_set_tuning(ctx, None if tuning is None else ctypes.byref(tuning)),
           ctx)


def get_tuning(device: int | None = None) -> Tuning:
    dev = torch.cuda.current_device() if device is None else device
    ctx = context(dev)
    t = Tuning()
    _raise(load_library().mpnl_get_tuning(ctx, ctypes.byref(t)), ctx)
    return t


class SlotBuffers:
    """Device buffers for one slot of a given size, reused across calls."""

    def __init__(self, n_sc, n_sym, nr, nt, qam, n_pe, device, mmse: bool = True):
        B = BITS[qam]
        kw = dict(device=device)
        self.dims = (n_sc, n_sym, nr, nt, qam, n_pe)
        self.H = torch.empty((n_sc, nr, nt), dtype=torch.complex64, **kw)
        self.Y = torch.empty((n_sc, n_sym, nr), dtype=torch.complex64, **kw)
        self.R = torch.empty((n_sc, nt * (nt + 1) // 2), dtype=torch.complex64, **kw)
        self.inv_diag = torch.empty((n_sc, nt), dtype=torch.float32, **kw)
        self.perm = torch.empty((n_sc, nt), dtype=torch.uint8, **kw)
        self.Z = torch.empty((n_sc, n_sym, nt), dtype=torch.complex64, **kw)
        self.paths = torch.empty((n_sc, n_pe, nt), dtype=torch.uint8, **kw)
        self.hard = torch.empty((n_sc, n_sym, nt), dtype=torch.uint8, **kw)
        self.llr = torch.empty((n_sc, n_sym, nt, B), dtype=torch.float32, **kw)
        self.ped2 = torch.empty((n_sc, n_sym, 2), dtype=torch.float32, **kw)
        self.mmse_hard = torch.empty((n_sc, n_sym, nt), dtype=torch.uint8, **kw) if mmse else None
        self.mmse_llr = torch.empty((n_sc, n_sym, nt, B), dtype=torch.float32, **kw) if mmse else None


def run_slot(buf: SlotBuffers, H, Y, sigma2: float, mmse: bool = True,
             precision: str = "fp32", mmse_qr: bool = False,
             refine_threshold: float | None = None) -> None:
    """The whole path on device tensors H, Y (enqueued on the current stream):
    preprocess -> select_paths -> detect (hard, LLR, PED pair) [-> MMSE].
    mmse_qr selects the MMSE-extended pre-processing (needed when nt > nr)."""
    n_sc, n_sym, nr, nt, qam, n_pe = buf.dims
    preprocess(H, Y, out=(buf.R, buf.inv_diag, buf.perm, buf.Z),
               sigma2=sigma2 if mmse_qr else None)
    if refine_threshold is not None:
        refine_qr(H, Y, buf.R, buf.inv_diag, buf.perm, Z=buf.Z,
                  sigma2=sigma2 if mmse_qr else None, cond_threshold=refine_threshold)
    select_paths(buf.R, sigma2, qam, n_pe, nt, out=buf.paths)
    detect(buf.R, buf.inv_diag, buf.perm, buf.paths, buf.Z, sigma2, qam,
           out=(buf.hard, buf.llr, buf.ped2), precision=precision)
    if mmse:
        linear_mmse(H, Y, sigma2, qam, out=(buf.mmse_hard, buf.mmse_llr))


class SlotGraph:
    """The whole path of one slot on fixed device tensors, captured once as a
    CUDA graph and replayed: the sorted QR + z, the selection and the walks
    on the capturing stream, and the MMSE baseline (it needs only H and Y)
    beside them on a side stream, forked and joined inside the graph.  A
    replay reads whatever H and Y hold when it runs -- write the next slot
    into them, then replay -- and costs one launch instead of five, which
    takes the launch gaps (about 35 us a slot) off a slot's latency.  sigma2
    and the sizes are fixed at capture."""

    def __init__(self, buf: SlotBuffers, H: torch.Tensor, Y: torch.Tensor, sigma2: float,
                 mmse: bool = True, precision: str = "fp32", mmse_qr: bool = False):
        if precision not in PRECISIONS:
            raise MpnlError(ERR_INVALID_ARG, f"precision {precision!r} not in {PRECISIONS}")
        if mmse and buf.mmse_hard is None:
            raise ValueError("SlotGraph(mmse=True) needs SlotBuffers(mmse=True)")
        dev = _dev_of(H)
        self.buf, self.H, self.Y = buf, H, Y
        n_sc, n_sym, nr, nt, qam, n_pe = buf.dims
        side = torch.cuda.Stream(dev) if mmse else None

        def path():
            cur = torch.cuda.current_stream(dev)
            if side is not None:
                side.wait_stream(cur)
                with torch.cuda.stream(side):
                    linear_mmse(H, Y, sigma2, qam, out=(buf.mmse_hard, buf.mmse_llr))
            preprocess(H, Y, out=(buf.R, buf.inv_diag, buf.perm, buf.Z),
                       sigma2=sigma2 if mmse_qr else None)
            select_paths(buf.R, sigma2, qam, n_pe, nt, out=buf.paths)
            detect(buf.R, buf.inv_diag, buf.perm, buf.paths, buf.Z, sigma2, qam,
                   out=(buf.hard, buf.llr, buf.ped2), precision=precision)
            if side is not None:
                cur.wait_stream(side)

        cap = torch.cuda.Stream(dev)
        cap.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(cap):   # once eagerly: kernel attributes, contexts
            path()
        cap.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=cap):
            path()
        self._side = side

    def replay(self) -> None:
        """Enqueue the slot's path on the current stream."""
        self.graph.replay()


def slot_flags(mmse: bool, precision: str, mmse_qr: bool) -> int:
    if precision not in PRECISIONS:
        raise MpnlError(ERR_INVALID_ARG, f"precision {precision!r} not in {PRECISIONS}")
    return (SLOT_MMSE if mmse else 0) | (SLOT_FP16 if precision == "fp16" else 0) \
        | (SLOT_MMSE_QR if mmse_qr else 0)


def slot_workspace_bytes(n_sc, n_sym, nr, nt, qam, n_pe, flags: int = 0) -> int:
    d = Dims(n_sc, n_sym, nr, nt, qam, n_pe)
    return int(load_library().mpnl_slot_workspace_bytes(ctypes.byref(d), flags))


class SlotOutputs:
    """Result buffers of one slot (host, pinned when `pin`), as mpnl_detect_slot writes them."""

    def __init__(self, n_sc, n_sym, nt, qam, mmse: bool, pin: bool = True):
        B = BITS[qam]
        kw = dict(pin_memory=pin)
        self.hard = torch.empty((n_sc, n_sym, nt), dtype=torch.uint8, **kw)
        self.llr = torch.empty((n_sc, n_sym, nt, B), dtype=torch.float32, **kw)
        self.ped2 = torch.empty((n_sc, n_sym, 2), dtype=torch.float32, **kw)
        self.mmse_hard = torch.empty((n_sc, n_sym, nt), dtype=torch.uint8, **kw) if mmse else None
        self.mmse_llr = (torch.empty((n_sc, n_sym, nt, B), dtype=torch.float32, **kw)
                         if mmse else None)

    def as_dict(self) -> dict:
        out = dict(hard=self.hard, llr=self.llr, ped2=self.ped2)
        if self.mmse_hard is not None:
            out["mmse_hard"] = self.mmse_hard
            out["mmse_llr"] = self.mmse_llr
        return out


def detect_slot_into(H, Y, sigma2: float, qam: int, n_pe: int, out: SlotOutputs,
                     workspace: torch.Tensor, flags: int = 0, stream=None) -> None:
    """mpnl_detect_slot: the whole path of one slot on the caller's buffers
    (host or device tensors), enqueued on `stream` (default: the current
    stream of the workspace's device); `workspace` is a device uint8 tensor of
    at least slot_workspace_bytes(...) bytes, one call in flight per workspace."""
    n_sc, nr, nt = H.shape
    n_sym = Y.shape[1]
    _need(H, torch.complex64, (n_sc, nr, nt), "H")
    _need(Y, torch.complex64, (n_sc, n_sym, nr), "Y")
    dev = _dev_of(workspace)
    ctx = context(dev.index)
    d = Dims(n_sc, n_sym, nr, nt, qam, n_pe)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    _raise(load_library().mpnl_detect_slot(
        ctx, ctypes.byref(d), float(sigma2), _ptr(H), _ptr(Y), _ptr(out.hard), _ptr(out.llr),
        _ptr(out.ped2), _ptr(out.mmse_hard), _ptr(out.mmse_llr), int(flags), _ptr(workspace),
        workspace.numel(), ctypes.c_void_p(st.cuda_stream)), ctx)


def detect_slot(H, Y, sigma2: float, qam: int, n_pe: int, mmse: bool = False,
                buffers: SlotBuffers | None = None, device=None, precision: str = "fp32",
                mmse_qr: bool = False):
    """End-to-end call a user makes: accepts host (ideally pinned) or device
    tensors.  Host inputs go through mpnl_detect_slot (copies in, the path,
    copies out, one C-ABI call) and the results come back as host tensors;
    device inputs run the per-call steps into `buffers`.  Returns a dict."""
    host = H.device.type == "cpu"
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device()) if host else H.device
    n_sc, nr, nt = H.shape
    n_sym = Y.shape[1]
    if host:
        device = torch.device(device)
        flags = slot_flags(mmse, precision, mmse_qr)
        ws = torch.empty(slot_workspace_bytes(n_sc, n_sym, nr, nt, qam, n_pe, flags),
                         dtype=torch.uint8, device=device)
        out = SlotOutputs(n_sc, n_sym, nt, qam, mmse, pin=True)
        st = torch.cuda.current_stream(device)
        detect_slot_into(H, Y, sigma2, qam, n_pe, out, ws, flags, stream=st)
        st.synchronize()
        return out.as_dict()
    buf = buffers or SlotBuffers(n_sc, n_sym, nr, nt, qam, n_pe, device, mmse)
    run_slot(buf, H, Y, sigma2, mmse, precision, mmse_qr)
    out = dict(hard=buf.hard, llr=buf.llr, ped2=buf.ped2)
    if mmse:
        out["mmse_hard"] = buf.mmse_hard
        out["mmse_llr"] = buf.mmse_llr
    return out


class SlotPipeline:
    """End-to-end detection of a stream of slots held in host memory, with
    `depth` slots in flight.  Each slot is one mpnl_detect_slot call on the
    slot's own stream and workspace: the copies of H and Y in, the path (and
    the MMSE baseline), the copies of the results out -- so one slot's copies
    overlap another slot's kernels.  Inputs should be pinned host tensors
    (pageable ones are copied synchronously).  Results land in pinned host
    buffers owned by the pipeline: ``result(ticket)`` waits for that slot and
    returns views that stay valid until the same buffers are reused, `depth`
    submissions later."""

    def __init__(self, n_sc, n_sym, nr, nt, qam, n_pe, device=None, depth: int = 2,
                 mmse: bool = True, precision: str = "fp32", mmse_qr: bool = False):
        if depth < 1:
            raise ValueError("depth must be >= 1")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.dims = (n_sc, n_sym, nr, nt, qam, n_pe)
        self.flags = slot_flags(mmse, precision, mmse_qr)
        self.mmse = mmse
        nbytes = slot_workspace_bytes(n_sc, n_sym, nr, nt, qam, n_pe, self.flags)
        self._lanes = []
        for _ in range(depth):
            self._lanes.append(dict(
                ws=torch.empty(nbytes, dtype=torch.uint8, device=self.device),
                out=SlotOutputs(n_sc, n_sym, nt, qam, mmse, pin=True), ticket=-1,
                stream=torch.cuda.Stream(self.device), done=torch.cuda.Event()))
        self._next = 0

    @property
    def h2d_bytes(self) -> int:
        n_sc, n_sym, nr, nt, _, _ = self.dims
        return n_sc * nr * nt * 8 + n_sc * n_sym * nr * 8

    @property
    def d2h_bytes(self) -> int:
        return sum(v.numel() * v.element_size() for v in self._lanes[0]["out"].as_dict().values())

    def submit(self, H, Y, sigma2: float) -> int:
        """Enqueue one slot (host H [n_sc][nr][nt], Y [n_sc][n_sym][nr],
        complex64); returns its ticket.  Waits first for the slot that last
        used the same buffers."""
        lane = self._lanes[self._next % len(self._lanes)]
        ticket = self._next
        self._next += 1
        if lane["ticket"] >= 0:
            lane["done"].synchronize()
        lane["ticket"] = ticket
        qam, n_pe = self.dims[4], self.dims[5]
        detect_slot_into(H, Y, sigma2, qam, n_pe, lane["out"], lane["ws"], self.flags,
                         stream=lane["stream"])
        lane["done"].record(lane["stream"])
        return ticket

    def result(self, ticket: int) -> dict:
        """Wait for a submitted slot and return its host results."""
        lane = self._lanes[ticket % len(self._lanes)]
        if lane["ticket"] != ticket:
            raise ValueError(f"ticket {ticket} is no longer held (buffers reused)")
        lane["done"].synchronize()
        return lane["out"].as_dict()

    def check_status(self) -> None:
        """Raise on device-side errors recorded by the slots' launches."""
        for lane in self._lanes:
            lane["done"].synchronize()
        check_status(self.device.index)


def batch_item(dims, sigma2: float, flags: int = 0, stages: int = 0, **arrays) -> BatchItemC:
    """One mpnl_batch_item from device tensors given by field name (H, Y, Q,
    R, inv_diag, perm, Z, paths, hard, llr, ped2, mmse_hard, mmse_llr)."""
    it = BatchItemC()
    it.dims = Dims(*dims)
    it.sigma2 = float(sigma2)
    it.flags = flags
    it.stages = stages
    for name, t in arrays.items():
        if t is not None:
            setattr(it, name, t.data_ptr())
    return it


class Batch:
    """A mixed-size batch of radio units' slots run by the persistent
    launches (mpnl_batch_*).  Units are SlotBuffers given as (buffers,
    sigma2, mmse_qr, mmse[, precision[, refine]]) tuples ("fp32" and no FP64
    re-factorisation when left out), whose H and Y the caller fills; ``run``
    writes their R/perm/Z/paths state and results.  Alternatively pass
    ready-made BatchItemC items (``items=``) that reference tensors the
    caller keeps alive."""

    def __init__(self, units=(), device=None, items=None):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.units = list(units)
        if items is None:
            items = [self._unit_item(u) for u in self.units]
        arr = (BatchItemC * len(items))(*items)
        self._ctx = context(self.device.index)
        h = ctypes.c_void_p()
        _raise(load_library().mpnl_batch_create(self._ctx, arr, len(items), ctypes.byref(h)),
               self._ctx)
        self._h = h
        self.capacity = len(items)

    @staticmethod
    def _unit_item(unit) -> BatchItemC:
        buf, sigma2, mmse_qr, mmse = unit[:4]
        precision = unit[4] if len(unit) > 4 else "fp32"
        refine = bool(unit[5]) if len(unit) > 5 else False
        if precision not in ("fp32", "fp16"):
            raise ValueError(f"precision must be fp32 or fp16, not {precision!r}")
        flags = (ITEM_MMSE_QR if mmse_qr else 0) | (ITEM_LINEAR_MMSE if mmse else 0) \
            | (ITEM_FP16 if precision == "fp16" else 0) | (ITEM_REFINE_QR if refine else 0)
        names = ("H", "Y", "R", "inv_diag", "perm", "Z", "paths", "hard", "llr", "ped2")
        arrays = {n: getattr(buf, n) for n in names}
        if mmse:
            arrays.update(mmse_hard=buf.mmse_hard, mmse_llr=buf.mmse_llr)
        return batch_item(buf.dims, sigma2, flags, 0, **arrays)

    def reset(self, items, trusted_pointers: bool = False) -> None:
        """Replace the units (at most the creation count), reusing the
        allocations; `items` is a sequence of BatchItemC or a ctypes array."""
        arr = items if isinstance(items, ctypes.Array) else (BatchItemC * len(items))(*items)
        _raise(load_library().mpnl_batch_reset(self._ctx, self._h, arr, len(items),
                                               RESET_TRUSTED_POINTERS if trusted_pointers else 0),
               self._ctx)

    def run(self, stages: int = STAGES_ALL, graph: bool = False, stream=None,
            share_sms: bool = False, short_ctas: bool = False) -> None:
        """Enqueue the stages on `stream` (default: the current stream; a
        graph needs a non-default stream).  share_sms leaves room on every SM
        for other streams' work (MPNL_RUN_SHARE_SMS); short_ctas launches one
        CTA (or warp) per work item instead of persistent ones
        (MPNL_RUN_SHORT_CTAS)."""
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        flags = stages | (RUN_GRAPH if graph else 0) | (RUN_SHARE_SMS if share_sms else 0) \
            | (RUN_SHORT_CTAS if short_ctas else 0)
        _raise(load_library().mpnl_batch_run(self._ctx, self._h, flags,
                                             ctypes.c_void_p(st.cuda_stream)), self._ctx)

    def serve_round(self, reqs, n: int, run_flags: int = 0, stream=None) -> None:
        """One serving round in one C call (mpnl_serve_round): `reqs` is a
        RoundReqC array whose first n entries are this round's requests."""
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        _raise(load_library().mpnl_serve_round(self._ctx, self._h, reqs, int(n), int(run_flags),
                                               ctypes.c_void_p(st.cuda_stream)), self._ctx)

    def close(self) -> None:
        if getattr(self, "_h", None):
            torch.cuda.synchronize(self.device)
            load_library().mpnl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def detect_units_noalloc(items, stream=None) -> None:
    """Walks of up to NOALLOC_MAX_UNITS units in one persistent launch with
    no device allocation (mpnl_detect_units_noalloc).  `items` are BatchItemC
    descriptors (see batch_item) of device tensors the caller keeps alive:
    R, inv_diag, perm, Z, paths in, hard, llr, ped2 out.  The walks run on
    `stream` (default: the current stream) of the current device; calls whose
    work overlaps on the device share one scratch array and race."""
    arr = items if isinstance(items, ctypes.Array) else (BatchItemC * len(items))(*items)
    dev = torch.device("cuda", torch.cuda.current_device())
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    code = load_library().mpnl_detect_units_noalloc(arr, len(arr), ctypes.c_void_p(st.cuda_stream))
    if code != OK:
        raise MpnlError(code, "mpnl_detect_units_noalloc failed (no context: the code is the report)")
