"""ctypes binding of libhmat.so (include/hmat.h): argument marshalling only.

Every entry point has the name of the C function it calls. Device buffers are
passed as torch CUDA tensors (or raw device addresses); the stream is a
torch.cuda.Stream, a raw cudaStream_t or None for torch's current stream.
Nothing here computes: if the library is missing, importing works but every
call raises, so no caller can silently fall back to another path.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import List, Optional, Sequence

import numpy as np

HMAT_OK = 0
HMAT_EINVAL = -1
HMAT_ENOMEM = -2
HMAT_ECUDA = -3
HMAT_ETIMEOUT = -4
HMAT_EUNSUPPORTED = -5
HMAT_EDEVICE = -6
HMAT_EBUSY = -7

HMAT_MODE_FP64 = 0
HMAT_MODE_MIXED = 1
HMAT_LOAD_MIXED = 1
HMAT_LOAD_MIXED_ONLY = 8
HMAT_DTYPE_F64 = 0
HMAT_DTYPE_F32 = 1

PHASES = ("near", "up_leaf", "up_transfer", "coupling", "down_transfer", "down_leaf", "split", "far_up", "far_down")

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "lib", "libhmat.so")
_HEADER = os.path.join(os.path.dirname(_PKG), "include", "hmat.h")

_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_i32p = ctypes.POINTER(ctypes.c_int32)
_c_dpp = ctypes.POINTER(ctypes.c_void_p)


class HmatDesc(ctypes.Structure):
    _fields_ = [
        ("n_points", ctypes.c_int64),
        ("levels", ctypes.c_int32),
        ("node_begin", _c_i64p),
        ("node_size", _c_i64p),
        ("rank", _c_i32p),
        ("near_ptr", _c_i64p),
        ("near_idx", _c_i32p),
        ("far_ptr", _c_i64p),
        ("far_idx", _c_i32p),
        ("basis", _c_dpp),
        ("coupling", _c_dpp),
        ("near", _c_dpp),
        ("perm", _c_i64p),
    ]


HMAT_KERNEL_GAUSSIAN = 0
HMAT_KERNEL_IMQ = 1
HMAT_KERNEL_INVDIST = 2
HMAT_ADM_HSS = 0
HMAT_ADM_GEOMETRIC = 1
HMAT_ADM_NONE = 2
HMAT_ADM_TAU = 3
HMAT_ADM_BUDGET = 4
HMAT_BUILD_ID_GPU = 2
HMAT_BUILD_NEAR_OTF = 4
HMAT_TREE_KD = 0
HMAT_TREE_TWO_MEANS = 1

_KERNELS = {"gaussian": HMAT_KERNEL_GAUSSIAN, "imq": HMAT_KERNEL_IMQ, "invdist": HMAT_KERNEL_INVDIST}
_ADMISSIBILITY = {"hss": HMAT_ADM_HSS, "geometric": HMAT_ADM_GEOMETRIC, "none": HMAT_ADM_NONE, "tau": HMAT_ADM_TAU,
                  "budget": HMAT_ADM_BUDGET}
_TREES = {"kd": HMAT_TREE_KD, "two_means": HMAT_TREE_TWO_MEANS}


class HmatBuildParams(ctypes.Structure):
    _fields_ = [
        ("n_points", ctypes.c_int64),
        ("dim", ctypes.c_int32),
        ("points", ctypes.POINTER(ctypes.c_double)),
        ("kernel", ctypes.c_int32),
        ("kernel_param", ctypes.c_double),
        ("admissibility", ctypes.c_int32),
        ("eta", ctypes.c_double),
        ("leaf_size", ctypes.c_int32),
        ("tol", ctypes.c_double),
        ("max_rank", ctypes.c_int32),
        ("exact_columns", ctypes.c_int32),
        ("sample_seed", ctypes.c_uint64),
        ("threads", ctypes.c_int32),
        ("tree", ctypes.c_int32),
    ]


class HmatPlanParams(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("dim", ctypes.c_int32), ("points", ctypes.POINTER(ctypes.c_double)),
                ("admissibility", ctypes.c_int32), ("eta", ctypes.c_double), ("leaf_size", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("tree", ctypes.c_int32)]


class HmatCompressParams(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("kernel_param", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_rank", ctypes.c_int32), ("exact_columns", ctypes.c_int32), ("sample_seed", ctypes.c_uint64)]


class HmatServerParams(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("memory_budget", ctypes.c_int64), ("max_q", ctypes.c_int64),
                ("mode", ctypes.c_int), ("max_pending", ctypes.c_int64)]


class HmatTuneReport(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int64), ("mode", ctypes.c_int32), ("launches_tuned", ctypes.c_int32),
                ("default_ms", ctypes.c_double), ("tuned_ms", ctypes.c_double), ("near_cols", ctypes.c_int32),
                ("chain_grid", ctypes.c_int32)]


class HmatError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {hmat_strerror(status)} (status {status})")
        self.status = status


_lib = None


def library() -> ctypes.CDLL:
    """The loaded libhmat.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libhmat.so is not built ({_LIB_PATH}); run paper_1812_07152_gb300.build.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        lib.hmat_load.argtypes = [ctypes.POINTER(HmatDesc), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
        lib.hmat_eval.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                  ctypes.c_int, ctypes.c_void_p]
        lib.hmat_build.argtypes = [ctypes.POINTER(HmatBuildParams), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
        lib.hmat_structure.argtypes = [ctypes.c_void_p, _c_i64p, _c_i32p, _c_i64p, _c_i32p, _c_i64p, _c_i32p]
        lib.hmat_reserve.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        lib.hmat_eval_host.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_int, ctypes.c_void_p]
        lib.hmat_eval_typed.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        lib.hmat_eval_host_typed.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        lib.hmat_batch_eval_typed.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                              ctypes.POINTER(ctypes.c_void_p), _c_i64p, ctypes.c_int, ctypes.c_void_p]
        lib.hmat_server_submit_typed.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                                 ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _c_i64p]
        lib.hmat_server_matrix_stats.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                 ctypes.c_int]
        lib.hmat_profile.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.hmat_phase_times.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), _c_i64p, ctypes.c_int]
        lib.hmat_measure_fp64_peak.argtypes = [ctypes.POINTER(ctypes.c_double)]
        lib.hmat_batch_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_void_p)]
        lib.hmat_batch_eval.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p), _c_i64p, ctypes.c_void_p]
        lib.hmat_batch_free.argtypes = [ctypes.c_void_p]
        lib.hmat_batch_info.argtypes = [ctypes.c_void_p, _c_i64p, ctypes.c_int]
        lib.hmat_batch_schedule.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.hmat_batch_autotune.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.POINTER(ctypes.c_void_p), _c_i64p, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.hmat_server_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                           ctypes.POINTER(HmatServerParams), ctypes.POINTER(ctypes.c_void_p)]
        lib.hmat_server_submit.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, _c_i64p]
        lib.hmat_server_wait.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
        lib.hmat_server_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        lib.hmat_server_free.argtypes = [ctypes.c_void_p]
        lib.hmat_status_poll.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        lib.hmat_info.argtypes = [ctypes.c_void_p, _c_i64p, ctypes.c_int]
        lib.hmat_free.argtypes = [ctypes.c_void_p]
        lib.hmat_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.POINTER(HmatTuneReport)]
        lib.hmat_selftest_timeout.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        lib.hmat_tune_apply.argtypes = [ctypes.c_void_p, ctypes.POINTER(HmatTuneReport)]
        lib.hmat_selftest_device_check.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
        lib.hmat_selftest_row_id.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_double, ctypes.c_int32, _c_i32p, _c_i32p,
                                             ctypes.POINTER(ctypes.c_double)]
        lib.hmat_selftest_chain_timeout.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                                    ctypes.c_void_p]
        lib.hmat_selftest_conversions.argtypes = [ctypes.c_int64, ctypes.c_uint64, _c_i64p]
        lib.hmat_plan_create.argtypes = [ctypes.POINTER(HmatPlanParams), ctypes.POINTER(ctypes.c_void_p)]
        lib.hmat_plan_build.argtypes = [ctypes.c_void_p, ctypes.POINTER(HmatCompressParams), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_void_p)]
        lib.hmat_plan_free.argtypes = [ctypes.c_void_p]
        lib.hmat_strerror.argtypes = [ctypes.c_int]
        lib.hmat_strerror.restype = ctypes.c_char_p
        for name in ("hmat_load", "hmat_build", "hmat_structure", "hmat_eval", "hmat_reserve", "hmat_status_poll",
                     "hmat_info", "hmat_free", "hmat_eval_host", "hmat_profile", "hmat_phase_times",
                     "hmat_measure_fp64_peak", "hmat_batch_create", "hmat_batch_eval", "hmat_batch_free",
                     "hmat_server_create", "hmat_server_submit", "hmat_server_wait", "hmat_server_stats",
                     "hmat_server_free", "hmat_autotune", "hmat_selftest_timeout", "hmat_selftest_chain_timeout", "hmat_tune_apply", "hmat_selftest_row_id", "hmat_selftest_device_check",
                     "hmat_eval_typed", "hmat_eval_host_typed", "hmat_batch_eval_typed", "hmat_server_submit_typed",
                     "hmat_server_matrix_stats", "hmat_batch_info", "hmat_batch_autotune", "hmat_batch_schedule",
                     "hmat_plan_create", "hmat_plan_build",
                     "hmat_plan_free", "hmat_selftest_conversions"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def exported_symbols() -> List[str]:
    """Entry points declared in include/hmat.h."""
    with open(_HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:hmat_status|const char\*)\s+(hmat_\w+)\s*\(", text, re.M)))


def _check(status: int, what: str) -> None:
    if status != HMAT_OK:
        raise HmatError(status, what)


def _ptr(x) -> Optional[int]:
    """Device address of a torch tensor, or an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def hmat_strerror(status: int) -> str:
    return library().hmat_strerror(int(status)).decode()


def hmat_load(n_points: int, levels: int, node_begin, node_size, rank, near_ptr, near_idx, far_ptr, far_idx,
              basis: Sequence[Optional[np.ndarray]], coupling: Sequence[Optional[np.ndarray]],
              near: Sequence[Optional[np.ndarray]], perm, flags: int = 0) -> int:
    """Validate and upload one HMatrix; returns the handle (an opaque address).
    Block arrays are FP64 row-major; the host arrays may be freed after the call."""
    keep = []

    def arr(x, dtype):
        a = np.ascontiguousarray(np.asarray(x), dtype=dtype)
        keep.append(a)
        return a.ctypes.data_as(_c_i64p if dtype == np.int64 else _c_i32p)

    def blocks(lst):
        ptrs = (ctypes.c_void_p * max(len(lst), 1))()
        for i, b in enumerate(lst):
            if b is None or np.asarray(b).size == 0:
                ptrs[i] = None
            else:
                a = np.ascontiguousarray(b, dtype=np.float64)
                keep.append(a)
                ptrs[i] = a.ctypes.data
        keep.append(ptrs)
        return ctypes.cast(ptrs, _c_dpp)

    d = HmatDesc(int(n_points), int(levels), arr(node_begin, np.int64), arr(node_size, np.int64),
                 arr(rank, np.int32), arr(near_ptr, np.int64), arr(near_idx, np.int32), arr(far_ptr, np.int64),
                 arr(far_idx, np.int32), blocks(basis), blocks(coupling), blocks(near), arr(perm, np.int64))
    h = ctypes.c_void_p()
    _check(library().hmat_load(ctypes.byref(d), int(flags), ctypes.byref(h)), "hmat_load")
    return int(h.value)


def hmat_build(points: np.ndarray, kernel: str, kernel_param: float, admissibility: str, leaf_size: int,
               tol: float, max_rank: int, eta: float = 2.0, exact_columns: int = -1, sample_seed: int = 2,
               threads: int = 0, flags: int = 0, tree: str = "kd") -> int:
    """Compress the kernel matrix of `points` (n x d, caller order) and load it; returns the handle."""
    X = np.ascontiguousarray(points, dtype=np.float64)
    p = HmatBuildParams(X.shape[0], X.shape[1], X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        _KERNELS[kernel], float(kernel_param), _ADMISSIBILITY[admissibility], float(eta),
                        int(leaf_size), float(tol), int(max_rank), int(exact_columns), int(sample_seed), int(threads),
                        _TREES[tree])
    h = ctypes.c_void_p()
    _check(library().hmat_build(ctypes.byref(p), int(flags), ctypes.byref(h)), "hmat_build")
    return int(h.value)


def hmat_plan_create(points: np.ndarray, admissibility: str, leaf_size: int, eta: float = 2.0,
                     threads: int = 0, tree: str = "kd") -> int:
    """Inspector-p1: cluster tree and near/far lists of `points` (n x d, caller order); returns a plan."""
    X = np.ascontiguousarray(points, dtype=np.float64)
    p = HmatPlanParams(X.shape[0], X.shape[1], X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       _ADMISSIBILITY[admissibility], float(eta), int(leaf_size), int(threads), _TREES[tree])
    plan = ctypes.c_void_p()
    _check(library().hmat_plan_create(ctypes.byref(p), ctypes.byref(plan)), "hmat_plan_create")
    return int(plan.value)


def hmat_plan_build(plan: int, kernel: str, kernel_param: float, tol: float, max_rank: int,
                    exact_columns: int = -1, sample_seed: int = 2, flags: int = 0) -> int:
    """Inspector-p2 and load for one kernel and accuracy, reusing the plan; returns the handle."""
    c = HmatCompressParams(_KERNELS[kernel], float(kernel_param), float(tol), int(max_rank), int(exact_columns),
                           int(sample_seed))
    h = ctypes.c_void_p()
    _check(library().hmat_plan_build(plan, ctypes.byref(c), int(flags), ctypes.byref(h)), "hmat_plan_build")
    return int(h.value)


def hmat_plan_free(plan: int) -> None:
    _check(library().hmat_plan_free(plan), "hmat_plan_free")


def hmat_structure(handle: int) -> dict:
    """perm, rank and the near/far CSR lists of a loaded HMatrix, as numpy arrays."""
    info = hmat_info(handle)
    levels = info["levels"]
    n_nodes, n_leaves = 2 ** (levels + 1) - 1, 2 ** levels
    out = dict(perm=np.zeros(info["n_points"], np.int64), rank=np.zeros(n_nodes, np.int32),
               near_ptr=np.zeros(n_leaves + 1, np.int64), near_idx=np.zeros(info["near_entries"], np.int32),
               far_ptr=np.zeros(n_nodes + 1, np.int64), far_idx=np.zeros(info["far_entries"], np.int32))
    args = [out[k].ctypes.data_as(_c_i64p if out[k].dtype == np.int64 else _c_i32p)
            for k in ("perm", "rank", "near_ptr", "near_idx", "far_ptr", "far_idx")]
    _check(library().hmat_structure(handle, *args), "hmat_structure")
    return out


def hmat_eval(handle: int, W, Y, q: int, mode: int = HMAT_MODE_FP64, stream=None) -> None:
    """Enqueue Y = K~ W on `stream` (W, Y: n_points x q FP64 device buffers)."""
    _check(library().hmat_eval(handle, _ptr(W), _ptr(Y), int(q), int(mode), _stream(stream)), "hmat_eval")


def _dtype_of(x) -> int:
    name = str(getattr(x, "dtype", ""))
    if name.endswith("float32"):
        return HMAT_DTYPE_F32
    if name.endswith("float64"):
        return HMAT_DTYPE_F64
    raise ValueError(f"W and Y must be float32 or float64, not {name}")


def hmat_eval_typed(handle: int, W, Y, q: int, mode: int = HMAT_MODE_FP64, dtype: Optional[int] = None,
                    stream=None) -> None:
    """Enqueue Y = K~ W with W and Y of element type dtype (default: W's, torch float32 or float64)."""
    dt = _dtype_of(W) if dtype is None else int(dtype)
    _check(library().hmat_eval_typed(handle, _ptr(W), _ptr(Y), int(q), int(mode), dt, _stream(stream)),
           "hmat_eval_typed")


def hmat_eval_host(handle: int, W: np.ndarray, Y: np.ndarray, mode: int = HMAT_MODE_FP64, stream=None) -> None:
    """Y = K~ W with host arrays (n x q FP64, C-contiguous; pinned memory copies fastest).
    W and Y may be numpy arrays or CPU torch tensors; synchronises the stream."""
    if hasattr(W, "data_ptr"):
        wp, yp, q = int(W.data_ptr()), int(Y.data_ptr()), int(W.shape[1])
    else:
        if not (W.flags.c_contiguous and Y.flags.c_contiguous and W.dtype == np.float64 and Y.dtype == np.float64):
            raise ValueError("W and Y must be C-contiguous float64 arrays")
        wp, yp, q = W.ctypes.data, Y.ctypes.data, int(W.shape[1])
    _check(library().hmat_eval_host(handle, wp, yp, q, int(mode), _stream(stream)), "hmat_eval_host")


def hmat_eval_host_typed(handle: int, W, Y, mode: int = HMAT_MODE_FP64, stream=None) -> None:
    """hmat_eval_host for host W and Y of float32 or float64 (numpy arrays or CPU torch tensors, C-contiguous)."""
    dt = _dtype_of(W)
    if _dtype_of(Y) != dt:
        raise ValueError("W and Y must have the same dtype")
    if hasattr(W, "data_ptr"):
        wp, yp, q = int(W.data_ptr()), int(Y.data_ptr()), int(W.shape[1])
    else:
        if not (W.flags.c_contiguous and Y.flags.c_contiguous):
            raise ValueError("W and Y must be C-contiguous")
        wp, yp, q = W.ctypes.data, Y.ctypes.data, int(W.shape[1])
    _check(library().hmat_eval_host_typed(handle, wp, yp, q, int(mode), dt, _stream(stream)), "hmat_eval_host_typed")


def hmat_profile(handle: int, enable=True) -> None:
    """enable: True/1 (event timing of every launch), 2 (the same with the mixed mode's far chain serialised
    on the caller's stream, so that each launch is timed alone) or False/0."""
    _check(library().hmat_profile(handle, int(enable) if not isinstance(enable, bool) else (1 if enable else 0)),
           "hmat_profile")


def hmat_phase_times(handle: int) -> dict:
    """{phase: (summed ms, launches)} of the evaluations recorded since hmat_profile."""
    n = len(PHASES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    _check(library().hmat_phase_times(handle, ms, cnt, n), "hmat_phase_times")
    return {PHASES[k]: (float(ms[k]), int(cnt[k])) for k in range(n)}


def hmat_measure_fp64_peak() -> float:
    """FP64 FMA throughput of the current device in GFLOP/s."""
    g = ctypes.c_double()
    _check(library().hmat_measure_fp64_peak(ctypes.byref(g)), "hmat_measure_fp64_peak")
    return float(g.value)


def hmat_autotune(handle: int, q: int, mode: int = HMAT_MODE_FP64, stream=None) -> dict:
    """Time the tile-shape candidates for (q, mode) on the device and keep the fastest
    for later evaluations of the handle; returns the call's report."""
    rep = HmatTuneReport()
    _check(library().hmat_autotune(handle, int(q), int(mode), _stream(stream), ctypes.byref(rep)), "hmat_autotune")
    return {"q": int(rep.q), "mode": int(rep.mode), "launches_tuned": int(rep.launches_tuned),
            "default_ms": float(rep.default_ms), "tuned_ms": float(rep.tuned_ms), "near_cols": int(rep.near_cols),
            "chain_grid": int(rep.chain_grid)}


def hmat_tune_apply(handle: int, q: int, near_cols: int = 0, chain_grid: int = 0,
                    mode: int = HMAT_MODE_MIXED) -> None:
    """Install a mixed-mode choice for q columns without timing: near-field CTA width (0: default) and the
    persistent far chain's CTAs (0: every resident CTA)."""
    rep = HmatTuneReport(int(q), int(mode), 0, 0.0, 0.0, int(near_cols), int(chain_grid))
    _check(library().hmat_tune_apply(handle, ctypes.byref(rep)), "hmat_tune_apply")


def hmat_reserve(handle: int, q_max: int) -> None:
    _check(library().hmat_reserve(handle, int(q_max)), "hmat_reserve")


def hmat_status_poll(handle: int, stream=None) -> int:
    """Synchronise the stream and return (and clear) the device status word."""
    return int(library().hmat_status_poll(handle, _stream(stream)))


def hmat_selftest_timeout(handle: int, limit_ns: int, stream=None) -> None:
    """Enqueue one bounded device wait that runs out after limit_ns and latches
    HMAT_ETIMEOUT in the handle's status word (read it with hmat_status_poll)."""
    _check(library().hmat_selftest_timeout(handle, int(limit_ns), _stream(stream)), "hmat_selftest_timeout")


def hmat_selftest_chain_timeout(handle: int, q: int, limit_ns: int, mode: int = HMAT_MODE_MIXED, stream=None) -> None:
    """Enqueue the persistent far-chain launch of `mode` with requirements no item can meet: every wait runs out
    after limit_ns and latches HMAT_ETIMEOUT in the handle's status word."""
    _check(library().hmat_selftest_chain_timeout(handle, int(q), int(mode), int(limit_ns), _stream(stream)),
           "hmat_selftest_chain_timeout")


def hmat_selftest_device_check(handle: int, q: int, mode: int = HMAT_MODE_FP64, stream=None) -> None:
    """Enqueue a far-chain launch whose only ticket names an item past the item array: its index check latches
    HMAT_EDEVICE in the handle's status word before anything is read."""
    _check(library().hmat_selftest_device_check(handle, int(q), int(mode), _stream(stream)),
           "hmat_selftest_device_check")


def hmat_selftest_row_id(M: np.ndarray, tol: float, max_rank: int):
    """The GPU row ID of the inspector on the rows of M (host, float64): (rank, pivot order, T)."""
    A = np.ascontiguousarray(M, dtype=np.float64)
    n, m = A.shape
    piv = np.zeros(n, dtype=np.int32)
    rank = ctypes.c_int32()
    T = np.zeros(n * n, dtype=np.float64)
    _check(library().hmat_selftest_row_id(A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n, m, float(tol),
                                          int(max_rank), piv.ctypes.data_as(_c_i32p), ctypes.byref(rank),
                                          T.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "hmat_selftest_row_id")
    k = int(rank.value)
    return k, piv, T[: k * (n - k)].reshape(k, n - k)


def hmat_selftest_conversions(n: int, seed: int = 0) -> dict:
    """Bitwise check of the mixed mode's integer-unit FP32 <-> FP64 conversions against the
    hardware's on n hashed samples; returns the mismatch counts per conversion."""
    out = (ctypes.c_int64 * 3)()
    _check(library().hmat_selftest_conversions(int(n), int(seed) & (2**64 - 1), out), "hmat_selftest_conversions")
    return {"widen": out[0], "narrow": out[1], "scale": out[2]}


def hmat_info(handle: int) -> dict:
    out = (ctypes.c_int64 * 11)()
    _check(library().hmat_info(handle, out, 11), "hmat_info")
    keys = ("n_points", "levels", "near_entries", "far_entries", "near_values", "basis_values",
            "coupling_values", "sum_rank", "device_bytes", "coupling_engine", "near_on_the_fly")
    return dict(zip(keys, [int(v) for v in out]))


def hmat_free(handle: int) -> None:
    _check(library().hmat_free(handle), "hmat_free")


def hmat_batch_create(handles: Sequence[int], mode: int = HMAT_MODE_FP64) -> int:
    arr = (ctypes.c_void_p * len(handles))(*handles)
    b = ctypes.c_void_p()
    _check(library().hmat_batch_create(arr, len(handles), int(mode), ctypes.byref(b)), "hmat_batch_create")
    return int(b.value)


def hmat_batch_eval(batch: int, Ws, Ys, stream=None) -> None:
    """Y[i] = K~_i W[i] for every member (torch CUDA tensors n_i x q_i), one graph launch."""
    n = len(Ws)
    w = (ctypes.c_void_p * n)(*[_ptr(x) for x in Ws])
    y = (ctypes.c_void_p * n)(*[_ptr(x) for x in Ys])
    q = (ctypes.c_int64 * n)(*[int(x.shape[1]) for x in Ws])
    _check(library().hmat_batch_eval(batch, w, y, q, _stream(stream)), "hmat_batch_eval")


def hmat_batch_eval_typed(batch: int, Ws, Ys, stream=None) -> None:
    """hmat_batch_eval for members' W and Y of one element type (float32 or float64 torch CUDA tensors)."""
    n = len(Ws)
    dt = _dtype_of(Ws[0])
    w = (ctypes.c_void_p * n)(*[_ptr(x) for x in Ws])
    y = (ctypes.c_void_p * n)(*[_ptr(x) for x in Ys])
    q = (ctypes.c_int64 * n)(*[int(x.shape[1]) for x in Ws])
    _check(library().hmat_batch_eval_typed(batch, w, y, q, dt, _stream(stream)), "hmat_batch_eval_typed")


def hmat_batch_info(batch: int) -> dict:
    out = (ctypes.c_int64 * 6)()
    _check(library().hmat_batch_info(batch, out, 6), "hmat_batch_info")
    return {"members": int(out[0]), "kernels": int(out[1]), "device_bytes": int(out[2]), "chain_grid": int(out[3]),
            "branched": int(out[4]), "default_widths": int(out[5])}


def hmat_batch_schedule(batch: int, branched: int = 0, chain_grid: int = 0, default_widths: int = 0) -> None:
    _check(library().hmat_batch_schedule(batch, int(branched), int(chain_grid), int(default_widths)),
           "hmat_batch_schedule")


def hmat_batch_autotune(batch: int, Ws, Ys, stream=None) -> dict:
    """Time whole replays of the batch with several chain grids and keep the fastest (bitwise neutral)."""
    n = len(Ws)
    dt = _dtype_of(Ws[0])
    w = (ctypes.c_void_p * n)(*[_ptr(x) for x in Ws])
    y = (ctypes.c_void_p * n)(*[_ptr(x) for x in Ys])
    q = (ctypes.c_int64 * n)(*[int(x.shape[1]) for x in Ws])
    d, t = ctypes.c_double(), ctypes.c_double()
    _check(library().hmat_batch_autotune(batch, w, y, q, dt, _stream(stream), ctypes.byref(d), ctypes.byref(t)),
           "hmat_batch_autotune")
    return {"default_ms": float(d.value), "tuned_ms": float(t.value), **hmat_batch_info(batch)}


def hmat_batch_free(batch: int) -> None:
    _check(library().hmat_batch_free(batch), "hmat_batch_free")


def hmat_server_create(handles: Sequence[int], slots: int, memory_budget: int, max_q: int,
                       mode: int = HMAT_MODE_FP64, max_pending: int = 0) -> int:
    arr = (ctypes.c_void_p * len(handles))(*handles)
    p = HmatServerParams(int(slots), int(memory_budget), int(max_q), int(mode), int(max_pending))
    sv = ctypes.c_void_p()
    _check(library().hmat_server_create(arr, len(handles), ctypes.byref(p), ctypes.byref(sv)), "hmat_server_create")
    return int(sv.value)


def hmat_server_submit(server: int, matrix: int, W, Y) -> int:
    """Queue Y = K~_matrix W; W and Y are pinned CPU (or CUDA) tensors of n x q whose rows are contiguous
    (column slices of a wider tensor are fine), float64 or float32 (both the same). Returns the request id;
    raises HmatError with status HMAT_EBUSY when the server's queue is full."""
    if W.stride(1) != 1 or Y.stride(1) != 1 or tuple(W.shape) != tuple(Y.shape):
        raise ValueError("W and Y must be n x q with contiguous rows")
    dt = _dtype_of(W)
    if _dtype_of(Y) != dt:
        raise ValueError("W and Y must have the same dtype")
    rid = ctypes.c_int64()
    _check(library().hmat_server_submit_typed(server, int(matrix), _ptr(W), int(W.stride(0)), _ptr(Y),
                                              int(Y.stride(0)), int(W.shape[1]), dt, ctypes.byref(rid)),
           "hmat_server_submit")
    return int(rid.value)


def hmat_server_wait(server: int, request: int, timeout_ms: int = -1) -> int:
    """Status of a request once it has completed (HMAT_ETIMEOUT if not within timeout_ms)."""
    return int(library().hmat_server_wait(server, int(request), int(timeout_ms)))


def hmat_server_stats(server: int) -> dict:
    out = (ctypes.c_double * 7)()
    _check(library().hmat_server_stats(server, out, 7), "hmat_server_stats")
    keys = ("completed", "p50_ms", "p99_ms", "requests_per_evaluation", "evaluations", "peak_bytes", "rejected")
    return dict(zip(keys, [float(v) for v in out]))


def hmat_server_matrix_stats(server: int, matrix: int) -> dict:
    out = (ctypes.c_double * 3)()
    _check(library().hmat_server_matrix_stats(server, int(matrix), out, 3), "hmat_server_matrix_stats")
    return dict(zip(("completed", "p50_ms", "p99_ms"), [float(v) for v in out]))


def hmat_server_free(server: int) -> None:
    _check(library().hmat_server_free(server), "hmat_server_free")


class DeviceHMatrix:
    """Owns one libhmat handle; ``evaluate`` returns Y = K~ W as a torch tensor."""

    def __init__(self, handle: int):
        self.handle = handle
        self.info = hmat_info(handle)

    @classmethod
    def load(cls, **desc) -> "DeviceHMatrix":
        return cls(hmat_load(**desc))

    @classmethod
    def build(cls, points, **params) -> "DeviceHMatrix":
        return cls(hmat_build(points, **params))

    def structure(self) -> dict:
        return hmat_structure(self.handle)

    @property
    def n_points(self) -> int:
        return self.info["n_points"]

    def evaluate(self, W, Y=None, mode: int = HMAT_MODE_FP64, stream=None):
        import torch
        if Y is None:
            Y = torch.empty_like(W)
        hmat_eval(self.handle, W, Y, W.shape[1], mode, stream)
        return Y

    def reserve(self, q_max: int) -> None:
        hmat_reserve(self.handle, q_max)

    def poll(self, stream=None) -> int:
        return hmat_status_poll(self.handle, stream)

    def close(self) -> None:
        if self.handle:
            hmat_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
