"""ctypes binding of libgotoh_gb300.so (argument marshalling only).

Every step of the alignment runs in the library's CUDA kernels; this module
only turns torch tensors / numpy arrays into pointers and sizes.  There is no
CPU fallback: if the shared library is missing or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LOCAL, GLOBAL, SEMIGLOBAL = 0, 1, 2
_MODES = {"local": LOCAL, "global": GLOBAL, "semiglobal": SEMIGLOBAL, "semi": SEMIGLOBAL}

GA_OK = 0
GA_ERR_ARG = 1
GA_ERR_ALPHABET = 2
GA_ERR_OOM = 3
GA_ERR_CUDA = 4
GA_ERR_RESIDUE = 5
GA_ERR_TIMEOUT = 6
GA_ERR_RANGE = 7

# Symbols declared in include/gotoh_align.h (checked by the CPU tests).
EXPORTED = ("ga_align_batch", "ga_align_batch_modes", "ga_align_batch_host", "ga_align_batch_host_modes",
            "ga_align_cross", "ga_align_long",
            "ga_align_long_noalloc", "ga_align_banded", "ga_strerror", "ga_version",
            "ga_band_features", "ga_band_min_w", "ga_band_predict",
            "ga_mlp_forward", "ga_mlp_loss_grad", "ga_mlp_train", "ga_mlp_cast",
            "ga_server_create", "ga_server_add_scoring", "ga_server_submit_batch",
            "ga_server_poll", "ga_server_drain", "ga_server_clock_ns", "ga_server_stats_get",
            "ga_server_destroy", "ga_plan_create", "ga_plan_run", "ga_plan_capture",
            "ga_plan_launch", "ga_plan_stats", "ga_plan_autotune", "ga_plan_get_tuning",
            "ga_plan_set_tuning", "ga_plan_destroy", "ga_probe_bounded_wait")
TILE_K = (6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 24, 32)  # columns per lane of tile 0..16
TILE_ALT_MASK = 0x1D47F  # tiles with an alternative lane-group size (8 lanes: 0..6; 32 lanes: 10, 12, 14..16)
SERVE_MAX_LEN = 65536
BAND_NFEAT = 32
MLP_NPARAMS = 6337
NOALLOC_MAX_LEN = 65536


class Scoring(ctypes.Structure):
    _fields_ = [("alphabet_size", ctypes.c_int32), ("matrix", ctypes.POINTER(ctypes.c_int8)),
                ("gap_open", ctypes.c_int32), ("gap_extend", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("pairs_int16", ctypes.c_int64), ("pairs_int32", ctypes.c_int64),
                ("pairs_int32_rerun", ctypes.c_int64), ("band_retries", ctypes.c_int64),
                ("banded_cells", ctypes.c_int64), ("kernel_ms", ctypes.c_float),
                ("dp_ms", ctypes.c_float), ("dp_launches", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("status", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("max_tasks", ctypes.c_int32), ("device", ctypes.c_int32), ("idle_us", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("cells_completed", ctypes.c_int64),
                ("arena_high_water", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("scheduler_ticks", ctypes.c_int64), ("admit_host_ns", ctypes.c_int64),
                ("copy_ns", ctypes.c_int64), ("complete_ns", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(ctypes.Structure):
    """ga_tuning: active tiles of the int16x2 / int32 bins, packed tiles run
    with their alternative lane-group size, and bin concurrency."""
    _fields_ = [("tiles16", ctypes.c_uint32), ("tiles32", ctypes.c_uint32),
                ("concurrent", ctypes.c_int32), ("lanes_alt", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {"tiles16": [TILE_K[k] for k in range(len(TILE_K)) if self.tiles16 >> k & 1],
                "tiles32": [TILE_K[k] for k in range(len(TILE_K)) if self.tiles32 >> k & 1],
                "lanes_alt": [TILE_K[k] for k in range(len(TILE_K)) if self.lanes_alt >> k & 1],
                "concurrent": int(self.concurrent)}


RESULT_DTYPE = np.dtype([("id", np.int64), ("score", np.int32), ("status", np.int32),
                         ("release_ns", np.int64), ("admit_ns", np.int64), ("done_ns", np.int64),
                         ("cells", np.int64)])


class GotohError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} (code {code})" if what else strerror(code))


_lib = None


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = False):
    """Load the CUDA library; raises when it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: run paper_2205_07610_gb300.build.build() "
                               "(the CUDA extension is required; there is no CPU fallback)")
        _build.build()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    sp = ctypes.POINTER(Scoring)
    stp = ctypes.POINTER(Stats)
    lib.ga_align_batch.argtypes = [P, P, P, P, i64, sp, i32, P, P, stp]
    lib.ga_align_batch_host.argtypes = [P, P, P, P, i64, sp, i32, P, P, stp]
    lib.ga_align_batch_host_modes.argtypes = [P, P, P, P, i64, sp, P, i32, P, P, stp]
    lib.ga_align_batch_modes.argtypes = [P, P, P, P, i64, sp, P, i32, P, P, stp]
    lib.ga_align_cross.argtypes = [P, P, i64, P, P, i64, sp, i32, P, P, stp]
    lib.ga_align_long.argtypes = [P, i64, P, i64, sp, i32, P, P, stp]
    lib.ga_align_banded.argtypes = [P, P, P, P, i64, sp, P, i32, P, P, P, stp]
    lib.ga_align_long_noalloc.argtypes = [P, i64, P, i64, sp, i32, P, P]
    f32 = ctypes.c_float
    lib.ga_band_features.argtypes = [P, P, P, P, i64, P, P, stp]
    lib.ga_band_min_w.argtypes = [P, P, P, P, i64, sp, P, P, P, stp]
    lib.ga_band_predict.argtypes = [P, P, P, P, i64, P, f32, P, P, P, stp]
    lib.ga_mlp_forward.argtypes = [P, P, i64, P, P]
    lib.ga_mlp_loss_grad.argtypes = [P, P, P, i32, P, P, P]
    lib.ga_mlp_train.argtypes = [P, P, P, P, P, P, i64, P, i32, i32, i32, f32, f32, f32, f32, P, P]
    lib.ga_mlp_cast.argtypes = [P, P, P]
    vp = ctypes.POINTER(ctypes.c_void_p)
    lib.ga_server_create.argtypes = [ctypes.POINTER(ServerConfig), vp]
    lib.ga_server_add_scoring.argtypes = [P, sp, ctypes.POINTER(i32)]
    lib.ga_server_submit_batch.argtypes = [P, i64, P, P, P, P, P, P, P, ctypes.POINTER(i64)]
    lib.ga_server_poll.argtypes = [P, P, i32, ctypes.POINTER(i32)]
    lib.ga_server_drain.argtypes = [P, i64]
    lib.ga_server_clock_ns.argtypes = [P]
    lib.ga_server_clock_ns.restype = i64
    lib.ga_server_stats_get.argtypes = [P, ctypes.POINTER(ServerStats)]
    lib.ga_server_destroy.argtypes = [P]
    lib.ga_probe_bounded_wait.argtypes = [i32, i32, i64, ctypes.POINTER(i32), ctypes.POINTER(i64)]
    for f in ("ga_server_create", "ga_server_add_scoring", "ga_server_submit_batch",
              "ga_server_poll", "ga_server_drain", "ga_server_stats_get", "ga_server_destroy",
              "ga_probe_bounded_wait"):
        getattr(lib, f).restype = i32
    tp = ctypes.POINTER(Tuning)
    lib.ga_plan_create.argtypes = [sp, i32, i64, i64, i32, vp]
    lib.ga_plan_run.argtypes = [P, P, P, P, P, i64, P, P]
    lib.ga_plan_capture.argtypes = [P, P, P, P, P, i64, P]
    lib.ga_plan_launch.argtypes = [P, P]
    lib.ga_plan_stats.argtypes = [P, P, stp]
    lib.ga_plan_autotune.argtypes = [P, P, P, P, P, i64, P, i32, P, tp, ctypes.POINTER(f32)]
    lib.ga_plan_get_tuning.argtypes = [P, tp]
    lib.ga_plan_set_tuning.argtypes = [P, tp]
    lib.ga_plan_destroy.argtypes = [P]
    for f in ("ga_align_batch", "ga_align_batch_modes", "ga_align_batch_host", "ga_align_batch_host_modes",
              "ga_align_cross",
              "ga_align_long",
              "ga_align_long_noalloc", "ga_align_banded", "ga_band_features", "ga_band_min_w",
              "ga_band_predict", "ga_mlp_forward", "ga_mlp_loss_grad", "ga_mlp_train",
              "ga_mlp_cast", "ga_plan_create", "ga_plan_run", "ga_plan_capture", "ga_plan_launch",
              "ga_plan_stats", "ga_plan_autotune", "ga_plan_get_tuning", "ga_plan_set_tuning",
              "ga_plan_destroy"):
        getattr(lib, f).restype = i32
    lib.ga_strerror.argtypes = [ctypes.c_int]
    lib.ga_strerror.restype = ctypes.c_char_p
    lib.ga_version.argtypes = []
    lib.ga_version.restype = ctypes.c_int
    _lib = lib
    return lib


def probe_bounded_wait(flag_value: int, need: int, limit_ns: int):
    """(status, waited_ns) of the strip kernel's bounded wait run alone on a
    device flag that nothing writes (gotoh_serve.h)."""
    st = ctypes.c_int32(-1)
    waited = ctypes.c_int64(-1)
    rc = load().ga_probe_bounded_wait(int(flag_value), int(need), int(limit_ns), ctypes.byref(st),
                                      ctypes.byref(waited))
    if rc:
        raise GotohError(rc, "ga_probe_bounded_wait")
    return int(st.value), int(waited.value)


def strerror(code: int) -> str:
    return load().ga_strerror(int(code)).decode()


def version() -> int:
    return int(load().ga_version())


def _mode(mode) -> int:
    return _MODES[mode] if isinstance(mode, str) else int(mode)


def make_scoring(matrix, gap_open: int, gap_extend: int):
    """(Scoring struct, keep-alive buffer) for an A x A int8 matrix."""
    m = np.ascontiguousarray(np.asarray(matrix, dtype=np.int8))
    if m.ndim != 2 or m.shape[0] != m.shape[1]:
        raise ValueError("substitution matrix must be square")
    sc = Scoring(int(m.shape[0]), m.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), int(gap_open),
                 int(gap_extend))
    return sc, m


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _check_dev(*ts):
    import torch
    for t in ts:
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
            raise TypeError("expected contiguous CUDA tensors")


def align_batch(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, mode, scores=None,
                stream=None, stats: bool = False):
    """Scores of pairs (q_p, t_p) given as device CSR tensors (uint8 codes, int64 offsets)."""
    import torch
    _check_dev(q_codes, q_off, t_codes, t_off)
    npairs = q_off.numel() - 1
    if scores is None:
        scores = torch.empty(max(npairs, 0), dtype=torch.int32, device=q_codes.device)
    sc, keep = make_scoring(matrix, gap_open, gap_extend)
    st = Stats()
    rc = load().ga_align_batch(_ptr(q_codes), _ptr(q_off), _ptr(t_codes), _ptr(t_off), npairs,
                               ctypes.byref(sc), _mode(mode), _ptr(scores), _stream_ptr(stream),
                               ctypes.byref(st) if stats else None)
    if rc:
        raise GotohError(rc, "ga_align_batch")
    return (scores, st.as_dict()) if stats else scores


def align_batch_modes(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, modes, scores=None,
                      stream=None, stats: bool = False):
    """Scores [len(modes), npairs] of the pairs in several modes; the inputs are packed once."""
    import torch
    _check_dev(q_codes, q_off, t_codes, t_off)
    npairs = q_off.numel() - 1
    md = np.ascontiguousarray([_mode(m) for m in modes], dtype=np.int32)
    if scores is None:
        scores = torch.empty((len(md), max(npairs, 0)), dtype=torch.int32, device=q_codes.device)
    sc, keep = make_scoring(matrix, gap_open, gap_extend)
    st = Stats()
    rc = load().ga_align_batch_modes(_ptr(q_codes), _ptr(q_off), _ptr(t_codes), _ptr(t_off), npairs,
                                     ctypes.byref(sc), md.ctypes.data, len(md), _ptr(scores),
                                     _stream_ptr(stream), ctypes.byref(st) if stats else None)
    if rc:
        raise GotohError(rc, "ga_align_batch_modes")
    return (scores, st.as_dict()) if stats else scores


def align_batch_host(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, mode,
                     scores=None, stream=None, stats: bool = False):
    """ga_align_batch_host: host arrays in (numpy or pinned torch CPU tensors), host scores out."""
    def host_ptr(a, dtype):
        if hasattr(a, "data_ptr"):
            return a, int(a.data_ptr())
        a = np.ascontiguousarray(a, dtype=dtype)
        return a, a.ctypes.data
    q_codes, qc = host_ptr(q_codes, np.uint8)
    q_off, qo = host_ptr(q_off, np.int64)
    t_codes, tc = host_ptr(t_codes, np.uint8)
    t_off, to = host_ptr(t_off, np.int64)
    npairs = (q_off.numel() if hasattr(q_off, "numel") else len(q_off)) - 1
    if scores is None:
        scores = np.empty(max(npairs, 0), dtype=np.int32)
    scores, sp = host_ptr(scores, np.int32)
    sc, keep = make_scoring(matrix, gap_open, gap_extend)
    st = Stats()
    rc = load().ga_align_batch_host(qc, qo, tc, to, npairs, ctypes.byref(sc), _mode(mode), sp,
                                    _stream_ptr(stream), ctypes.byref(st) if stats else None)
    if rc:
        raise GotohError(rc, "ga_align_batch_host")
    return (scores, st.as_dict()) if stats else scores


def align_batch_host_modes(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, modes,
                           scores=None, stream=None, stats: bool = False):
    """ga_align_batch_host_modes: host arrays in, host scores [len(modes), npairs] out; the
    inputs cross the host link once for all modes."""
    def host_ptr(a, dtype):
        if hasattr(a, "data_ptr"):
            return a, int(a.data_ptr())
        a = np.ascontiguousarray(a, dtype=dtype)
        return a, a.ctypes.data
    q_codes, qc = host_ptr(q_codes, np.uint8)
    q_off, qo = host_ptr(q_off, np.int64)
    t_codes, tc = host_ptr(t_codes, np.uint8)
    t_off, to = host_ptr(t_off, np.int64)
    npairs = (q_off.numel() if hasattr(q_off, "numel") else len(q_off)) - 1
    md = np.ascontiguousarray([_mode(m) for m in modes], dtype=np.int32)
    if scores is None:
        scores = np.empty((len(md), max(npairs, 0)), dtype=np.int32)
    scores, sp = host_ptr(scores, np.int32)
    sc, keep = make_scoring(matrix, gap_open, gap_extend)
    st = Stats()
    rc = load().ga_align_batch_host_modes(qc, qo, tc, to, npairs, ctypes.byref(sc), md.ctypes.data, len(md), sp,
                                          _stream_ptr(stream), ctypes.byref(st) if stats else None)
    if rc:
        raise GotohError(rc, "ga_align_batch_host_modes")
    return (scores, st.as_dict()) if stats else scores


def align_cross(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, mode, scores=None,
                stream=None, stats: bool = False):
    """Scores [nq, nt] of every query against every target (device tensors)."""
    import torch
    _check_dev(q_codes, q_off, t_codes, t_off)
    nq, nt = q_off.numel() - 1, t_off.numel() - 1
    if scores is None:
        scores = torch.empty((max(nq, 0), max(nt, 0)), dtype=torch.int32, device=q_codes.device)
    sc, keep = make_scoring(matrix, gap_open, gap_extend)
    st = Stats()
    rc = load().ga_align_cross(_ptr(q_codes), _ptr(q_off), nq, _ptr(t_codes), _ptr(t_off), nt,
                               ctypes.byref(sc), _mode(mode), _ptr(scores), _stream_ptr(stream),
                               ctypes.byref(st) if stats else None)
    if rc:
        raise GotohError(rc, "ga_align_cross")
    return (scores, st.as_dict()) if stats else scores


def align_long(q, t, matrix, gap_open, gap_extend, mode, stream=None, stats: bool = False):
    """Score of one (long) pair on the intra-sequence kernel; device tensors."""
    import torch
    _check_dev(q, t)
    out = torch.empty(1, dtype=torch.int32, device=q.device)
    sc, keep = make_scoring(matrix, gap_open, gap_extend)
    st = Stats()
    rc = load().ga_align_long(_ptr(q), q.numel(), _ptr(t), t.numel(), ctypes.byref(sc), _mode(mode),
                              _ptr(out), _stream_ptr(stream), ctypes.byref(st) if stats else None)
    if rc:
        raise GotohError(rc, "ga_align_long")
    return (out, st.as_dict()) if stats else out


def align_long_noalloc(q, t, matrix, gap_open, gap_extend, mode, out=None, stream=None):
    """ga_align_long_noalloc: one pair, no device allocation by the library.

    For callers that cannot allocate device memory while aligning (memory held
    by a pooling allocator, latency-critical loops).  `out` (a 1-element int32
    CUDA tensor) may be passed in so that nothing at all is allocated here.
    """
    import torch
    _check_dev(q, t)
    if out is None:
        out = torch.empty(1, dtype=torch.int32, device=q.device)
    sc, keep = make_scoring(matrix, gap_open, gap_extend)
    rc = load().ga_align_long_noalloc(_ptr(q), q.numel(), _ptr(t), t.numel(), ctypes.byref(sc),
                                      _mode(mode), _ptr(out), _stream_ptr(stream))
    if rc:
        raise GotohError(rc, "ga_align_long_noalloc")
    return out


def align_banded(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, w0=None,
                 default_w0: int = 16, scores=None, w_used=None, stream=None, stats: bool = False):
    """Exact global scores by certified band doubling; returns (scores, w_used)."""
    import torch
    _check_dev(q_codes, q_off, t_codes, t_off)
    npairs = q_off.numel() - 1
    dev = q_codes.device
    if scores is None:
        scores = torch.empty(max(npairs, 0), dtype=torch.int32, device=dev)
    if w_used is None:
        w_used = torch.empty(max(npairs, 0), dtype=torch.int32, device=dev)
    if w0 is not None:
        _check_dev(w0)
    sc, keep = make_scoring(matrix, gap_open, gap_extend)
    st = Stats()
    rc = load().ga_align_banded(_ptr(q_codes), _ptr(q_off), _ptr(t_codes), _ptr(t_off), npairs,
                                ctypes.byref(sc), _ptr(w0), int(default_w0), _ptr(scores),
                                _ptr(w_used), _stream_ptr(stream),
                                ctypes.byref(st) if stats else None)
    if rc:
        raise GotohError(rc, "ga_align_banded")
    return (scores, w_used, st.as_dict()) if stats else (scores, w_used)


def _check_dtype(t, dtype, n=None, what=""):
    _check_dev(t)
    if t.dtype != dtype or (n is not None and t.numel() != n):
        raise TypeError(f"{what}: expected {dtype} with {n} elements")


def band_features(q_codes, q_off, t_codes, t_off, out=None, stream=None, stats: bool = False):
    """float32[npairs, 32] pair features of the band predictor (DNA pairs)."""
    import torch
    _check_dev(q_codes, q_off, t_codes, t_off)
    npairs = q_off.numel() - 1
    if out is None:
        out = torch.empty((max(npairs, 0), BAND_NFEAT), dtype=torch.float32, device=q_codes.device)
    st = Stats()
    rc = load().ga_band_features(_ptr(q_codes), _ptr(q_off), _ptr(t_codes), _ptr(t_off), npairs,
                                 _ptr(out), _stream_ptr(stream), ctypes.byref(st) if stats else None)
    if rc:
        raise GotohError(rc, "ga_band_features")
    return (out, st.as_dict()) if stats else out


def band_min_w(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, stream=None,
               stats: bool = False):
    """(w_min, scores): minimal certified band half-width per global pair, exact scores."""
    import torch
    _check_dev(q_codes, q_off, t_codes, t_off)
    npairs = q_off.numel() - 1
    dev = q_codes.device
    w = torch.empty(max(npairs, 0), dtype=torch.int32, device=dev)
    scores = torch.empty(max(npairs, 0), dtype=torch.int32, device=dev)
    sc, keep = make_scoring(matrix, gap_open, gap_extend)
    st = Stats()
    rc = load().ga_band_min_w(_ptr(q_codes), _ptr(q_off), _ptr(t_codes), _ptr(t_off), npairs,
                              ctypes.byref(sc), _ptr(w), _ptr(scores), _stream_ptr(stream),
                              ctypes.byref(st) if stats else None)
    if rc:
        raise GotohError(rc, "ga_band_min_w")
    return (w, scores, st.as_dict()) if stats else (w, scores)


def band_predict(q_codes, q_off, t_codes, t_off, params_bf16, margin: float = 0.0, stream=None,
                 stats: bool = False):
    """(w0 int32[npairs], y float32[npairs]) from the fused features + network kernel."""
    import torch
    _check_dev(q_codes, q_off, t_codes, t_off)
    _check_dtype(params_bf16, torch.int16, MLP_NPARAMS, "params_bf16")
    npairs = q_off.numel() - 1
    dev = q_codes.device
    w0 = torch.empty(max(npairs, 0), dtype=torch.int32, device=dev)
    y = torch.empty(max(npairs, 0), dtype=torch.float32, device=dev)
    st = Stats()
    rc = load().ga_band_predict(_ptr(q_codes), _ptr(q_off), _ptr(t_codes), _ptr(t_off), npairs,
                                _ptr(params_bf16), float(margin), _ptr(w0), _ptr(y),
                                _stream_ptr(stream), ctypes.byref(st) if stats else None)
    if rc:
        raise GotohError(rc, "ga_band_predict")
    return (w0, y, st.as_dict()) if stats else (w0, y)


def mlp_forward(params_bf16, x, stream=None):
    """y[n] = net(x[n, 32]) with bf16 weights (int16 tensor of bf16 bit patterns)."""
    import torch
    _check_dtype(params_bf16, torch.int16, MLP_NPARAMS, "params_bf16")
    _check_dtype(x, torch.float32, None, "x")
    n = x.numel() // BAND_NFEAT
    y = torch.empty(n, dtype=torch.float32, device=x.device)
    rc = load().ga_mlp_forward(_ptr(params_bf16), _ptr(x), n, _ptr(y), _stream_ptr(stream))
    if rc:
        raise GotohError(rc, "ga_mlp_forward")
    return y


def mlp_loss_grad(params_bf16, x, target, stream=None):
    """(loss float32[1], grad float32[6337]) of the mean squared error over all samples."""
    import torch
    _check_dtype(params_bf16, torch.int16, MLP_NPARAMS, "params_bf16")
    _check_dtype(x, torch.float32, None, "x")
    n = x.numel() // BAND_NFEAT
    _check_dtype(target, torch.float32, n, "target")
    grad = torch.empty(MLP_NPARAMS, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    rc = load().ga_mlp_loss_grad(_ptr(params_bf16), _ptr(x), _ptr(target), n, _ptr(grad),
                                 _ptr(loss), _stream_ptr(stream))
    if rc:
        raise GotohError(rc, "ga_mlp_loss_grad")
    return loss, grad


def mlp_train(master, params_bf16, adam_m, adam_v, x, target, batch_idx, step0: int = 0,
              lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
              stream=None):
    """Adam steps over batch_idx[steps, batch] (device int32); updates the tensors in place.

    Returns the per-step minibatch losses (float32[steps], device)."""
    import torch
    for t, what in ((master, "master"), (adam_m, "adam_m"), (adam_v, "adam_v")):
        _check_dtype(t, torch.float32, MLP_NPARAMS, what)
    _check_dtype(params_bf16, torch.int16, MLP_NPARAMS, "params_bf16")
    _check_dtype(x, torch.float32, None, "x")
    n = x.numel() // BAND_NFEAT
    _check_dtype(target, torch.float32, n, "target")
    _check_dtype(batch_idx, torch.int32, None, "batch_idx")
    steps, batch = batch_idx.shape
    losses = torch.empty(max(steps, 1), dtype=torch.float32, device=x.device)
    rc = load().ga_mlp_train(_ptr(master), _ptr(params_bf16), _ptr(adam_m), _ptr(adam_v), _ptr(x),
                             _ptr(target), n, _ptr(batch_idx), int(steps), int(batch), int(step0),
                             float(lr), float(beta1), float(beta2), float(eps), _ptr(losses),
                             _stream_ptr(stream))
    if rc:
        raise GotohError(rc, "ga_mlp_train")
    return losses[:steps]


def mlp_cast(master, params_bf16=None, stream=None):
    """bf16 (round to nearest even) copy of float32 parameters, as an int16 tensor."""
    import torch
    _check_dtype(master, torch.float32, MLP_NPARAMS, "master")
    if params_bf16 is None:
        params_bf16 = torch.empty(MLP_NPARAMS, dtype=torch.int16, device=master.device)
    rc = load().ga_mlp_cast(_ptr(master), _ptr(params_bf16), _stream_ptr(stream))
    if rc:
        raise GotohError(rc, "ga_mlp_cast")
    return params_bf16


class Server:
    """Alignment server (include/gotoh_serve.h): continuous batching of requests.

    Requests are host CSR arrays (copied at submission); results come back
    through poll() as a numpy structured array (RESULT_DTYPE)."""

    def __init__(self, arena_bytes: int = 0, max_inflight: int = 0, max_tasks: int = 0,
                 device: int = 0, idle_us: int = 0):
        cfg = ServerConfig(int(arena_bytes), int(max_inflight), int(max_tasks), int(device),
                           int(idle_us))
        h = ctypes.c_void_p()
        rc = load().ga_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc:
            raise GotohError(rc, "ga_server_create")
        self._h = h
        self._keep = []

    def add_scoring(self, matrix, gap_open: int, gap_extend: int) -> int:
        sc, keep = make_scoring(matrix, gap_open, gap_extend)
        sid = ctypes.c_int32(-1)
        rc = load().ga_server_add_scoring(self._h, ctypes.byref(sc), ctypes.byref(sid))
        if rc:
            raise GotohError(rc, "ga_server_add_scoring")
        return int(sid.value)

    def submit(self, q_codes, q_off, t_codes, t_off, modes, scoring_ids, release_ns=None) -> int:
        """Submit requests (host arrays); returns the id of the first one."""
        qc = np.ascontiguousarray(q_codes, dtype=np.uint8)
        qo = np.ascontiguousarray(q_off, dtype=np.int64)
        tc = np.ascontiguousarray(t_codes, dtype=np.uint8)
        to = np.ascontiguousarray(t_off, dtype=np.int64)
        n = len(qo) - 1
        md = np.ascontiguousarray(np.broadcast_to(np.asarray(modes, dtype=np.int32), (n,)))
        si = np.ascontiguousarray(np.broadcast_to(np.asarray(scoring_ids, dtype=np.int32), (n,)))
        rel = None if release_ns is None else np.ascontiguousarray(release_ns, dtype=np.int64)
        first = ctypes.c_int64(-1)
        rc = load().ga_server_submit_batch(self._h, n, qc.ctypes.data, qo.ctypes.data, tc.ctypes.data,
                                           to.ctypes.data, md.ctypes.data, si.ctypes.data,
                                           None if rel is None else rel.ctypes.data,
                                           ctypes.byref(first))
        if rc:
            raise GotohError(rc, "ga_server_submit_batch")
        return int(first.value)

    def poll(self, max_results: int = 1 << 16) -> np.ndarray:
        out = np.zeros(max_results, dtype=RESULT_DTYPE)
        cnt = ctypes.c_int32(0)
        rc = load().ga_server_poll(self._h, out.ctypes.data, int(max_results), ctypes.byref(cnt))
        if rc:
            raise GotohError(rc, "ga_server_poll")
        return out[:cnt.value]

    def drain(self, timeout_ms: int = 600_000) -> None:
        rc = load().ga_server_drain(self._h, int(timeout_ms))
        if rc:
            raise GotohError(rc, "ga_server_drain")

    def clock_ns(self) -> int:
        return int(load().ga_server_clock_ns(self._h))

    def stats(self) -> dict:
        st = ServerStats()
        rc = load().ga_server_stats_get(self._h, ctypes.byref(st))
        if rc:
            raise GotohError(rc, "ga_server_stats_get")
        return st.as_dict()

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().ga_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Batch plan (include/gotoh_plan.h): ga_align_batch with its workspace
    allocated once, capture-safe runs, CUDA-graph replay and an autotuner.

    Inputs are device CSR tensors as for align_batch; q_off[npairs] and
    t_off[npairs] must not exceed max_residues, sequences not max_len."""

    def __init__(self, matrix, gap_open: int, gap_extend: int, mode, max_pairs: int,
                 max_residues: int, max_len: int):
        sc, keep = make_scoring(matrix, gap_open, gap_extend)
        h = ctypes.c_void_p()
        rc = load().ga_plan_create(ctypes.byref(sc), _mode(mode), int(max_pairs), int(max_residues),
                                   int(max_len), ctypes.byref(h))
        if rc:
            raise GotohError(rc, "ga_plan_create")
        self._h = h
        self._captured = None

    def run(self, q_codes, q_off, t_codes, t_off, scores=None, stream=None):
        import torch
        _check_dev(q_codes, q_off, t_codes, t_off)
        npairs = q_off.numel() - 1
        if scores is None:
            scores = torch.empty(max(npairs, 0), dtype=torch.int32, device=q_codes.device)
        rc = load().ga_plan_run(self._h, _ptr(q_codes), _ptr(q_off), _ptr(t_codes), _ptr(t_off), npairs,
                                _ptr(scores), _stream_ptr(stream))
        if rc:
            raise GotohError(rc, "ga_plan_run")
        return scores

    def capture(self, q_codes, q_off, t_codes, t_off, scores):
        """Record one run on these buffers into the plan's CUDA graph."""
        _check_dev(q_codes, q_off, t_codes, t_off, scores)
        npairs = q_off.numel() - 1
        rc = load().ga_plan_capture(self._h, _ptr(q_codes), _ptr(q_off), _ptr(t_codes), _ptr(t_off),
                                    npairs, _ptr(scores))
        if rc:
            raise GotohError(rc, "ga_plan_capture")
        self._captured = (q_codes, q_off, t_codes, t_off, scores)  # keep the buffers alive

    def launch(self, stream=None):
        rc = load().ga_plan_launch(self._h, _stream_ptr(stream))
        if rc:
            raise GotohError(rc, "ga_plan_launch")

    def stats(self, stream=None) -> dict:
        st = Stats()
        rc = load().ga_plan_stats(self._h, _stream_ptr(stream), ctypes.byref(st))
        if rc:
            raise GotohError(rc, "ga_plan_stats")
        return st.as_dict()

    def autotune(self, q_codes, q_off, t_codes, t_off, reps: int = 5, stream=None):
        """(tuning dict, median ms) of the fastest tuning on this sample batch."""
        import torch
        _check_dev(q_codes, q_off, t_codes, t_off)
        npairs = q_off.numel() - 1
        scores = torch.empty(max(npairs, 1), dtype=torch.int32, device=q_codes.device)
        tu = Tuning()
        ms = ctypes.c_float(0.0)
        rc = load().ga_plan_autotune(self._h, _ptr(q_codes), _ptr(q_off), _ptr(t_codes), _ptr(t_off),
                                     npairs, _ptr(scores), int(reps), _stream_ptr(stream),
                                     ctypes.byref(tu), ctypes.byref(ms))
        if rc:
            raise GotohError(rc, "ga_plan_autotune")
        self._captured = None
        return tu.as_dict(), float(ms.value)

    @property
    def tuning(self) -> Tuning:
        tu = Tuning()
        rc = load().ga_plan_get_tuning(self._h, ctypes.byref(tu))
        if rc:
            raise GotohError(rc, "ga_plan_get_tuning")
        return tu

    @tuning.setter
    def tuning(self, tu: Tuning):
        rc = load().ga_plan_set_tuning(self._h, ctypes.byref(tu))
        if rc:
            raise GotohError(rc, "ga_plan_set_tuning")
        self._captured = None

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().ga_plan_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
