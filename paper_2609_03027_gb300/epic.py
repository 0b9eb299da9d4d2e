"""Thin ctypes binding of libepic.so (include/epic.h).

Argument marshalling only: every step of the imaging path runs in the CUDA
library.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library cannot be built or loaded, or the device is not an
sm_103 GPU, these calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import buildlib as _build

PATH_PLAIN_FP32 = 0
PATH_FUSED_FP32 = 1
PATH_DFTGEMM_FP16 = 2
PATH_AUTO = 3
PATHS = {"plain": PATH_PLAIN_FP32, "fused": PATH_FUSED_FP32, "dftgemm": PATH_DFTGEMM_FP16, "auto": PATH_AUTO}
PATH_NAMES = {v: k for k, v in PATHS.items()}

GCF_GAUSSIAN = 0
GCF_TABLE = 1

RESET = 0
ACCUMULATE = 1
TIME_KERNELS = 2
GRAPH = 4

STATUS = {0: "EPIC_OK", 1: "EPIC_ERR_INVALID_ARG", 2: "EPIC_ERR_GRID_OVERFLOW", 3: "EPIC_ERR_OOM",
          4: "EPIC_ERR_BUSY", 5: "EPIC_ERR_TIMEOUT", 6: "EPIC_ERR_CUDA", 7: "EPIC_ERR_UNSUPPORTED",
          8: "EPIC_ERR_NOT_FOUND"}

# Every symbol declared in include/epic.h (checked by the ABI tests).
EXPORTED = ["epic_plan_create", "epic_plan_destroy", "epic_image", "epic_image_host", "epic_sync",
            "epic_kernel_times", "epic_plan_get_info", "epic_status_str", "epic_last_error",
            "epic_device_query", "epic_server_create", "epic_server_submit", "epic_server_poll",
            "epic_server_wait", "epic_server_stats", "epic_server_destroy", "epic_plan_tune",
            "epic_plan_set_param", "epic_plan_get_param", "epic_image_static_scratch"]


class EpicError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class _Gcf(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("K", ctypes.c_int), ("sigma_cells", ctypes.c_double),
                ("f_ref_hz", ctypes.c_double), ("freq_scaled", ctypes.c_int), ("oversample", ctypes.c_int),
                ("table", ctypes.POINTER(ctypes.c_float))]


class _PlanDesc(ctypes.Structure):
    _fields_ = [("n_ant", ctypes.c_int), ("pos_m", ctypes.POINTER(ctypes.c_double)), ("n_pol", ctypes.c_int),
                ("n_chan", ctypes.c_int), ("freq_hz", ctypes.POINTER(ctypes.c_double)),
                ("cell_m", ctypes.POINTER(ctypes.c_double)), ("grid_n", ctypes.c_int), ("gcf", _Gcf),
                ("path", ctypes.c_int), ("max_time", ctypes.c_int), ("input_bits", ctypes.c_int),
                ("sub_int", ctypes.c_int), ("jones", ctypes.POINTER(ctypes.c_float))]


class _TuneReport(ctypes.Structure):
    _fields_ = [("n_timed", ctypes.c_int), ("default_ms", ctypes.c_float), ("best_ms", ctypes.c_float),
                ("n_params", ctypes.c_int), ("names", ctypes.c_char_p * 8), ("values", ctypes.c_int * 8)]


class _PlanInfo(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("n_prod", ctypes.c_int), ("box_max_x", ctypes.c_int),
                ("box_max_y", ctypes.c_int), ("time_chunk", ctypes.c_int), ("device_bytes", ctypes.c_size_t),
                ("scratch_bytes", ctypes.c_size_t), ("n_kernels", ctypes.c_int),
                ("gemm_flops_per_sample", ctypes.c_double), ("input_bits", ctypes.c_int), ("sub_int", ctypes.c_int),
                ("pol_mix", ctypes.c_int), ("tc_kernel", ctypes.c_int), ("row_parts", ctypes.c_int)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libepic.so (building it first if absent or stale when nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libepic.so not found at {path}; run paper_2609_03027_gb300.build.build()")
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp, i, u = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint
        L.epic_plan_create.argtypes = [P(_PlanDesc), P(vp)]
        L.epic_plan_destroy.argtypes = [vp]
        L.epic_image.argtypes = [vp, vp, i, vp, vp, u]
        L.epic_image_host.argtypes = [vp, vp, i, vp, vp, u]
        L.epic_sync.argtypes = [vp]
        L.epic_selftest_bounded_wait.argtypes = [vp, ctypes.c_longlong, vp]
        L.epic_kernel_times.argtypes = [vp, P(ctypes.c_char_p), P(ctypes.c_float), i, P(i)]
        L.epic_plan_get_info.argtypes = [vp, P(_PlanInfo)]
        L.epic_status_str.argtypes = [i]
        L.epic_status_str.restype = ctypes.c_char_p
        L.epic_last_error.argtypes = [vp]
        L.epic_last_error.restype = ctypes.c_char_p
        L.epic_device_query.argtypes = [P(i), P(i), P(i), P(i)]
        L.epic_server_create.argtypes = [ctypes.c_size_t, i, P(vp)]
        L.epic_server_submit.argtypes = [vp, vp, vp, i, vp, u, P(ctypes.c_uint64)]
        L.epic_server_poll.argtypes = [vp, ctypes.c_uint64, P(i), P(ctypes.c_double)]
        L.epic_server_wait.argtypes = [vp, ctypes.c_uint64, i, P(ctypes.c_double)]
        L.epic_server_stats.argtypes = [vp, P(i), P(ctypes.c_double), P(ctypes.c_double), P(i)]
        L.epic_server_destroy.argtypes = [vp]
        L.epic_plan_tune.argtypes = [vp, vp, i, vp, vp, i, P(_TuneReport)]
        L.epic_plan_set_param.argtypes = [vp, ctypes.c_char_p, i]
        L.epic_plan_get_param.argtypes = [vp, ctypes.c_char_p, P(i)]
        L.epic_image_static_scratch.argtypes = [vp, vp, i, vp, vp, u]
        for name in EXPORTED:
            if name not in ("epic_status_str", "epic_last_error"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(L, st: int, plan=None):
    if st != 0:
        msg = L.epic_last_error(plan).decode(errors="replace")
        raise EpicError(st, msg)


def device_query() -> Dict[str, int]:
    L = load()
    a, b, c, d = (ctypes.c_int() for _ in range(4))
    _check(L, L.epic_device_query(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return {"sm_count": a.value, "smem_optin": b.value, "cc_major": c.value, "cc_minor": d.value}


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """An imaging plan: geometry, GCF taps and tables resident on the current GPU.

    ``path`` is one of "plain", "fused", "dftgemm", "auto".
    """

    def __init__(self, pos_m, freq_hz, n_pol: int, grid_n: int, gcf_k: int, sigma_cells: float = 1.0,
                 f_ref_hz: Optional[float] = None, freq_scaled: bool = False, cell_m=None, path: str = "auto",
                 max_time: int = 1024, gcf_table=None, oversample: int = 1, input_bits: int = 4, sub_int: int = 0,
                 jones=None):
        """``jones``: optional complex [C][A][2][2] polarisation-mixing matrices J_{c,e}^{ap} (output
        pol a, input pol p); the element kernel is then W_e^{ap}(r) = J^{ap} W(r) (Eq. 1)."""
        self._lib = load()
        self.pos = np.ascontiguousarray(pos_m, dtype=np.float64).reshape(-1, 2)
        self.freq = np.ascontiguousarray(freq_hz, dtype=np.float64).ravel()
        self.cell = None if cell_m is None else np.ascontiguousarray(cell_m, dtype=np.float64).ravel()
        self.table = None if gcf_table is None else np.ascontiguousarray(gcf_table, dtype=np.float32).ravel()
        self.n_ant, self.n_chan, self.n_pol, self.grid_n = self.pos.shape[0], self.freq.shape[0], int(n_pol), int(grid_n)
        self.n_prod = 1 if self.n_pol == 1 else 4
        self.max_time = int(max_time)
        self.input_bits = int(input_bits)
        self.sub_int = int(sub_int)
        self._sample = (2,) if self.input_bits == 8 else ()      # trailing byte-pair axis of 8+8-bit input
        d = _PlanDesc()
        d.n_ant = self.n_ant
        d.pos_m = self.pos.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.n_pol = self.n_pol
        d.n_chan = self.n_chan
        d.freq_hz = self.freq.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.cell_m = None if self.cell is None else self.cell.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.grid_n = self.grid_n
        d.gcf.kind = GCF_GAUSSIAN if self.table is None else GCF_TABLE
        d.gcf.K = int(gcf_k)
        d.gcf.sigma_cells = float(sigma_cells)
        d.gcf.f_ref_hz = float(f_ref_hz if f_ref_hz is not None else self.freq.max())
        d.gcf.freq_scaled = int(bool(freq_scaled))
        d.gcf.oversample = int(oversample)
        d.gcf.table = None if self.table is None else self.table.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        d.path = PATHS[path] if isinstance(path, str) else int(path)
        d.max_time = self.max_time
        d.input_bits = self.input_bits
        d.sub_int = self.sub_int
        self.jones = None
        if jones is not None:
            j = np.asarray(jones)
            if j.shape != (self.n_chan, self.n_ant, 2, 2):
                raise ValueError(f"jones must have shape {(self.n_chan, self.n_ant, 2, 2)}, got {j.shape}")
            self.jones = np.ascontiguousarray(j, dtype=np.complex64).view(np.float32)
            d.jones = self.jones.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        h = ctypes.c_void_p()
        _check(self._lib, self._lib.epic_plan_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_config(cls, cfg, path: str = "auto", max_time: Optional[int] = None) -> "Plan":
        return cls(cfg.pos_m, cfg.freq_hz, cfg.n_pol, cfg.grid_n, cfg.gcf_k, cfg.sigma_cells, cfg.f_ref_hz,
                   cfg.freq_scaled, None, path, cfg.n_time if max_time is None else max_time,
                   input_bits=getattr(cfg, "input_bits", 4), sub_int=getattr(cfg, "sub_int", 0),
                   jones=getattr(cfg, "jones", None))

    def image_shape(self, T: int):
        """Shape of the images of a T-sample block (image sets x C x n_prod x N x N with sub-integrations)."""
        base = (self.n_chan, self.n_prod, self.grid_n, self.grid_n)
        return ((T // self.sub_int,) + base) if self.sub_int > 0 else base

    # ------------------------------------------------------------------ calls
    def _handle(self):
        if self._h is None or not self._h.value:
            raise EpicError(1, "plan is closed")
        return self._h

    def image(self, volt, out=None, accumulate: bool = False, stream=None, time_kernels: bool = False,
              graph: bool = False):
        """Images of a device voltage block uint8[T][C][A][P] -> float32[C][n_prod][N][N] (device).

        ``graph=True`` replays the call's kernels as one recorded CUDA graph (EPIC_GRAPH)."""
        import torch
        if not (isinstance(volt, torch.Tensor) and volt.is_cuda and volt.dtype == torch.uint8):
            raise TypeError("volt must be a CUDA uint8 tensor [T][C][A][P]")
        want = (self.n_chan, self.n_ant, self.n_pol) + self._sample
        if not volt.is_contiguous() or volt.dim() != 1 + len(want) or tuple(volt.shape[1:]) != want:
            raise ValueError(f"volt must be contiguous [T]{list(want)}")
        shape = self.image_shape(int(volt.shape[0]))
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=volt.device)
        elif tuple(out.shape) != shape or out.dtype != torch.float32 or not out.is_contiguous() or not out.is_cuda:
            raise ValueError(f"out must be a contiguous CUDA float32 tensor {shape}")
        flags = (ACCUMULATE if accumulate else RESET) | (TIME_KERNELS if time_kernels else 0) | (GRAPH if graph else 0)
        T = int(volt.shape[0])
        st = self._lib.epic_image(self._handle(), volt.data_ptr() if T else None, T, _stream_handle(stream),
                                  out.data_ptr(), flags)
        _check(self._lib, st, self._h)
        return out

    def image_host(self, volt: np.ndarray, out: Optional[np.ndarray] = None, accumulate: bool = False,
                   stream=None, time_kernels: bool = False) -> np.ndarray:
        """Host-buffer call: H2D copy, imaging, D2H copy, stream synchronised on return."""
        v = np.asarray(volt)
        want = (self.n_chan, self.n_ant, self.n_pol) + self._sample
        if v.dtype != np.uint8 or v.ndim != 1 + len(want) or v.shape[1:] != want:
            raise ValueError(f"volt must be uint8 [T]{list(want)}")
        if not v.flags.c_contiguous:
            raise ValueError("volt must be C-contiguous")
        shape = self.image_shape(int(v.shape[0]))
        if out is None:
            out = np.zeros(shape, dtype=np.float32)
        if out.shape != shape or out.dtype != np.float32 or not out.flags.c_contiguous:
            raise ValueError(f"out must be C-contiguous float32 {shape}")
        flags = (ACCUMULATE if accumulate else RESET) | (TIME_KERNELS if time_kernels else 0)
        st = self._lib.epic_image_host(self._handle(), v.ctypes.data if v.shape[0] else None, int(v.shape[0]),
                                       _stream_handle(stream), out.ctypes.data, flags)
        _check(self._lib, st, self._h)
        return out

    def image_host_ptr(self, volt_ptr: int, T: int, out_ptr: int, accumulate: bool = False, stream=None,
                       graph: bool = False):
        """Host-buffer call on raw host pointers (e.g. pinned torch tensors)."""
        flags = (ACCUMULATE if accumulate else RESET) | (GRAPH if graph else 0)
        st = self._lib.epic_image_host(self._handle(), volt_ptr, int(T), _stream_handle(stream), out_ptr, flags)
        _check(self._lib, st, self._h)

    def tune(self, volt, out=None, reps: int = 3, stream=None) -> Dict[str, object]:
        """Autotune the plan's tiling on a device block (epic_plan_tune); out is overwritten."""
        import torch
        if not (isinstance(volt, torch.Tensor) and volt.is_cuda and volt.dtype == torch.uint8 and volt.is_contiguous()):
            raise TypeError("volt must be a contiguous CUDA uint8 tensor [T][C][A][P]")
        shape = self.image_shape(int(volt.shape[0]))
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=volt.device)
        rep = _TuneReport()
        st = self._lib.epic_plan_tune(self._handle(), volt.data_ptr(), int(volt.shape[0]), _stream_handle(stream),
                                      out.data_ptr(), int(reps), ctypes.byref(rep))
        _check(self._lib, st, self._h)
        params = {rep.names[i].decode(): int(rep.values[i]) for i in range(rep.n_params)}
        return {"n_timed": rep.n_timed, "default_ms": rep.default_ms, "best_ms": rep.best_ms, "params": params}

    def set_param(self, name: str, value: int):
        """Set one tuning parameter (epic_plan_set_param)."""
        _check(self._lib, self._lib.epic_plan_set_param(self._handle(), name.encode(), int(value)), self._h)

    def get_param(self, name: str) -> int:
        v = ctypes.c_int()
        _check(self._lib, self._lib.epic_plan_get_param(self._handle(), name.encode(), ctypes.byref(v)), self._h)
        return int(v.value)

    def sync(self):
        _check(self._lib, self._lib.epic_sync(self._handle()), self._h)

    def selftest_bounded_wait(self, budget_cycles: int, stream=None):
        """Launch the failure-detection self-test (a wait that runs out); see epic.h."""
        _check(self._lib, self._lib.epic_selftest_bounded_wait(self._handle(), int(budget_cycles),
                                                               _stream_handle(stream)), self._h)

    def kernel_times(self) -> List[Tuple[str, float]]:
        n = ctypes.c_int()
        _check(self._lib, self._lib.epic_kernel_times(self._handle(), None, None, 0, ctypes.byref(n)), self._h)
        k = n.value
        names = (ctypes.c_char_p * max(k, 1))()
        ms = (ctypes.c_float * max(k, 1))()
        _check(self._lib, self._lib.epic_kernel_times(self._handle(), names, ms, k, ctypes.byref(n)), self._h)
        return [(names[i].decode(), float(ms[i])) for i in range(k)]

    def info(self) -> Dict[str, int]:
        inf = _PlanInfo()
        _check(self._lib, self._lib.epic_plan_get_info(self._handle(), ctypes.byref(inf)), self._h)
        d = {f: getattr(inf, f) for f, _ in _PlanInfo._fields_}
        d["path_name"] = PATH_NAMES.get(d["path"], str(d["path"]))
        return d

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.epic_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server over the C ABI (epic_server_*).

    Blocks of different plans run concurrently on ``slots`` streams; blocks are
    admitted by queue length and a device pool of ``device_bytes``.  Host blocks
    passed to submit() are kept referenced until their ticket is waited for.
    """

    def __init__(self, device_bytes: int, slots: int = 4):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib, self._lib.epic_server_create(int(device_bytes), int(slots), ctypes.byref(h)))
        self._h = h
        self._keep: Dict[int, object] = {}

    def submit(self, plan: "Plan", volt: np.ndarray, out, accumulate: bool = False) -> Optional[int]:
        """Queue a host block; returns a ticket, or None when the server is busy."""
        v = np.ascontiguousarray(volt, dtype=np.uint8)
        want = (plan.n_chan, plan.n_ant, plan.n_pol) + plan._sample
        if v.ndim != 1 + len(want) or v.shape[1:] != want:
            raise ValueError(f"block must be uint8 [T]{list(want)} of the plan")
        t = ctypes.c_uint64()
        st = self._lib.epic_server_submit(self._h, plan._handle(), v.ctypes.data if v.shape[0] else None,
                                          int(v.shape[0]), out.data_ptr(), ACCUMULATE if accumulate else RESET,
                                          ctypes.byref(t))
        if st == 4:  # EPIC_ERR_BUSY
            return None
        _check(self._lib, st)
        self._keep[t.value] = (v, out)
        return int(t.value)

    def submit_ptr(self, plan: "Plan", volt_ptr: int, T: int, out, accumulate: bool = False) -> Optional[int]:
        """Queue a block given by a raw host pointer (e.g. a pinned tensor the caller keeps
        alive and unchanged until the ticket completes); None when the server is busy."""
        t = ctypes.c_uint64()
        st = self._lib.epic_server_submit(self._h, plan._handle(), volt_ptr, int(T), out.data_ptr(),
                                          ACCUMULATE if accumulate else RESET, ctypes.byref(t))
        if st == 4:  # EPIC_ERR_BUSY
            return None
        _check(self._lib, st)
        return int(t.value)

    def poll(self, ticket: int) -> Tuple[bool, float]:
        d, lat = ctypes.c_int(), ctypes.c_double()
        _check(self._lib, self._lib.epic_server_poll(self._h, ticket, ctypes.byref(d), ctypes.byref(lat)))
        return bool(d.value), float(lat.value)

    def wait(self, ticket: int, timeout_ms: int = 60000) -> float:
        lat = ctypes.c_double()
        st = self._lib.epic_server_wait(self._h, ticket, int(timeout_ms), ctypes.byref(lat))
        self._keep.pop(ticket, None)
        _check(self._lib, st)
        return float(lat.value)

    def stats(self) -> Dict[str, float]:
        n, p50, p99, fl = ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        _check(self._lib, self._lib.epic_server_stats(self._h, ctypes.byref(n), ctypes.byref(p50), ctypes.byref(p99),
                                                      ctypes.byref(fl)))
        return {"completed": n.value, "p50_ms": p50.value, "p99_ms": p99.value, "in_flight": fl.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.epic_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
