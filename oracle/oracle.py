"""ctypes front end of the FP64 C oracle (test infrastructure; see package docstring)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libepic_oracle.so")
_lock = threading.Lock()
_lib = None

GCF_GAUSSIAN = 0
GCF_TABLE = 1


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Plain C, no CUDA."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            d, i = ctypes.c_double, ctypes.c_int
            L.eo_unpack.argtypes = [ctypes.c_uint8, P(i), P(i)]
            L.eo_unpack.restype = None
            L.eo_fft2.argtypes = [P(d), i]
            L.eo_fft2.restype = i
            common = [i, P(d), d, d, i, i, i, d, d, i, i, P(ctypes.c_float)]
            L.eo_footprint.argtypes = common + [P(i), P(i), P(d)]
            L.eo_footprint.restype = i
            plan = [i, P(d), i, i, P(d), P(d), i, i, i, d, d, i, i, P(ctypes.c_float)]
            L.eo_grid_frame.argtypes = plan + [P(ctypes.c_uint8), i, i, i, P(d)]
            L.eo_grid_frame.restype = i
            L.eo_image.argtypes = plan + [P(ctypes.c_uint8), i, i, P(i), P(d), i]
            L.eo_image.restype = i
            L.eo_image_ext.argtypes = plan + [P(ctypes.c_uint8), i, i, i, P(d), i, P(i), P(d), i]
            L.eo_image_ext.restype = i
            L.eo_unpack8.argtypes = [P(ctypes.c_uint8), P(i), P(i)]
            L.eo_unpack8.restype = None
            L.eo_max_threads.argtypes = []
            L.eo_max_threads.restype = i
            _lib = L
    return _lib


def _p(a, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc} "
                          f"({ {1: 'invalid argument', 2: 'grid overflow', 3: 'out of memory'}.get(rc, '?') })")


def max_threads() -> int:
    return int(lib().eo_max_threads())


def unpack_table() -> np.ndarray:
    """int[256][2]: the oracle's (re, im) for every byte value."""
    L = lib()
    out = np.zeros((256, 2), dtype=np.int64)
    a, b = ctypes.c_int(), ctypes.c_int()
    for v in range(256):
        L.eo_unpack(v, ctypes.byref(a), ctypes.byref(b))
        out[v] = (a.value, b.value)
    return out


def unpack8_pairs(pairs: np.ndarray) -> np.ndarray:
    """int[n][2]: the oracle's (re, im) for 8+8-bit byte pairs uint8[n][2]."""
    L = lib()
    pr = np.ascontiguousarray(pairs, dtype=np.uint8).reshape(-1, 2)
    out = np.zeros((pr.shape[0], 2), dtype=np.int64)
    a, b = ctypes.c_int(), ctypes.c_int()
    for k in range(pr.shape[0]):
        L.eo_unpack8(_p(pr[k], ctypes.c_uint8), ctypes.byref(a), ctypes.byref(b))
        out[k] = (a.value, b.value)
    return out


def fft2(g: np.ndarray) -> np.ndarray:
    """The oracle's 2-D + sign unnormalised transform of complex g[N][N]."""
    g = np.asarray(g, dtype=np.complex128)
    n = g.shape[0]
    buf = np.ascontiguousarray(np.stack([g.real, g.imag], axis=-1))
    _check(lib().eo_fft2(_p(buf, ctypes.c_double), n), "fft2")
    return buf[..., 0] + 1j * buf[..., 1]


class _Geom:
    def __init__(self, pos_m, freq_hz, cell_m, n_pol, grid_n, gcf_kind, gcf_k, sigma_cells, f_ref_hz,
                 freq_scaled, oversample, table):
        self.pos = np.ascontiguousarray(pos_m, dtype=np.float64).reshape(-1, 2)
        self.freq = np.ascontiguousarray(freq_hz, dtype=np.float64).ravel()
        self.cell = None if cell_m is None else np.ascontiguousarray(cell_m, dtype=np.float64).ravel()
        self.n_pol, self.N, self.kind, self.K = int(n_pol), int(grid_n), int(gcf_kind), int(gcf_k)
        self.sigma, self.fref, self.fs = float(sigma_cells), float(f_ref_hz), int(bool(freq_scaled))
        self.os = int(oversample)
        self.table = None if table is None else np.ascontiguousarray(table, dtype=np.float32).ravel()

    def args(self):
        return [self.pos.shape[0], _p(self.pos, ctypes.c_double), self.n_pol, self.freq.shape[0],
                _p(self.freq, ctypes.c_double), _p(self.cell, ctypes.c_double), self.N, self.kind, self.K,
                self.sigma, self.fref, self.fs, self.os, _p(self.table, ctypes.c_float)]


def footprint(pos_m, freq_hz: float, grid_n: int, gcf_k: int, sigma_cells: float, f_ref_hz: float = 1.0,
              freq_scaled: bool = False, cell_m: float = 0.0, gcf_kind: int = GCF_GAUSSIAN,
              oversample: int = 1, table=None):
    """(tap_x[A][K], tap_y[A][K], w[A][K][K] complex) of one channel."""
    pos = np.ascontiguousarray(pos_m, dtype=np.float64).reshape(-1, 2)
    A, K = pos.shape[0], int(gcf_k)
    tx = np.zeros((A, K), dtype=np.int32)
    ty = np.zeros((A, K), dtype=np.int32)
    w = np.zeros((A, K, K, 2), dtype=np.float64)
    tab = None if table is None else np.ascontiguousarray(table, dtype=np.float32).ravel()
    rc = lib().eo_footprint(A, _p(pos, ctypes.c_double), float(freq_hz), float(cell_m), int(grid_n),
                            int(gcf_kind), K, float(sigma_cells), float(f_ref_hz), int(bool(freq_scaled)),
                            int(oversample), _p(tab, ctypes.c_float), _p(tx, ctypes.c_int),
                            _p(ty, ctypes.c_int), _p(w, ctypes.c_double))
    _check(rc, "footprint")
    return tx, ty, w[..., 0] + 1j * w[..., 1]


def grid_frame(volt: np.ndarray, t: int, c: int, p: int, pos_m, freq_hz, n_pol: int, grid_n: int,
               gcf_k: int, sigma_cells: float, f_ref_hz: float = 1.0, freq_scaled: bool = False,
               cell_m=None, gcf_kind: int = GCF_GAUSSIAN, oversample: int = 1, table=None) -> np.ndarray:
    """The oracle's complex grid G[N][N] of one (t, c, p) frame."""
    geo = _Geom(pos_m, freq_hz, cell_m, n_pol, grid_n, gcf_kind, gcf_k, sigma_cells, f_ref_hz, freq_scaled,
                oversample, table)
    v = np.ascontiguousarray(volt, dtype=np.uint8)
    g = np.zeros((grid_n, grid_n, 2), dtype=np.float64)
    _check(lib().eo_grid_frame(*geo.args(), _p(v, ctypes.c_uint8), int(t), int(c), int(p),
                               _p(g, ctypes.c_double)), "grid_frame")
    return g[..., 0] + 1j * g[..., 1]


def image(volt: np.ndarray, pos_m, freq_hz, n_pol: int, grid_n: int, gcf_k: int, sigma_cells: float,
          f_ref_hz: float = 1.0, freq_scaled: bool = False, cell_m=None, chans: Optional[Sequence[int]] = None,
          gcf_kind: int = GCF_GAUSSIAN, oversample: int = 1, table=None, threads: int = 0,
          input_bits: int = 4, sub_int: int = 0, jones=None) -> np.ndarray:
    """Accumulated images of the selected channels: float64[n_sel][nprod][N][N], or with
    sub-integrations (sub_int > 0) float64[T / sub_int][n_sel][nprod][N][N].

    volt holds ALL channels: uint8[T][C][A][P] (4+4-bit) or uint8[T][C][A][P][2] (8+8-bit:
    real byte, imaginary byte); chans selects which are imaged.  jones: optional complex
    [C][A][2][2] polarisation-mixing matrices J^{ap} (element kernel J^{ap} W(r), Eq. 1).
    """
    geo = _Geom(pos_m, freq_hz, cell_m, n_pol, grid_n, gcf_kind, gcf_k, sigma_cells, f_ref_hz, freq_scaled,
                oversample, table)
    v = np.ascontiguousarray(volt, dtype=np.uint8)
    T = v.shape[0]
    C = geo.freq.shape[0]
    per = 2 if input_bits == 8 else 1
    if v.size != T * C * geo.pos.shape[0] * geo.n_pol * per:
        raise OracleError("voltage array does not match T x C x A x P (x 2 for 8+8-bit)")
    sel = None if chans is None else np.ascontiguousarray(chans, dtype=np.int32)
    n_sel = C if sel is None else sel.shape[0]
    nprod = 1 if n_pol == 1 else 4
    n_int = T // sub_int if sub_int > 0 else 1
    out = np.zeros((n_int, n_sel, nprod, grid_n, grid_n), dtype=np.float64)
    jd = None
    if jones is not None:
        j = np.asarray(jones)
        if j.shape != (C, geo.pos.shape[0], 2, 2):
            raise OracleError("jones must be complex [C][A][2][2]")
        jd = np.ascontiguousarray(j, dtype=np.complex128).view(np.float64)
    rc = lib().eo_image_ext(*geo.args(), _p(v, ctypes.c_uint8), T, int(input_bits), int(sub_int),
                            _p(jd, ctypes.c_double), n_sel, _p(sel, ctypes.c_int), _p(out, ctypes.c_double),
                            int(threads))
    _check(rc, "image")
    return out if sub_int > 0 else out[0]


def image_cfg(cfg, volt: np.ndarray, chans: Optional[Sequence[int]] = None, threads: int = 0) -> np.ndarray:
    """image() for an ``epic_synth.EpicConfig`` (its input bits and sub-integration)."""
    return image(volt, cfg.pos_m, cfg.freq_hz, cfg.n_pol, cfg.grid_n, cfg.gcf_k, cfg.sigma_cells,
                 cfg.f_ref_hz, cfg.freq_scaled, None, chans, threads=threads,
                 input_bits=getattr(cfg, "input_bits", 4), sub_int=getattr(cfg, "sub_int", 0),
                 jones=getattr(cfg, "jones", None))
