"""Shared helpers of the GPU parity tests (imported by tests only)."""
import numpy as np

import oracle

# Tolerances: max |gpu - oracle| / peak of the channel's XX (and YY) image, per
# channel and per product (XX, YY, Re XY, Im XY).  FP32 paths: 1e-5; the FP16
# tensor-core DFT-as-GEMM path: 2e-3 of the image peak.
TOL = {"plain": 1e-5, "fused": 1e-5, "dftgemm": 2e-3}
GPU_PATHS = ["plain", "fused", "dftgemm"]


def rel_errors(gpu: np.ndarray, ref: np.ndarray):
    """[n_chan][n_prod] max error over pixels / peak of the co-polar images."""
    n_prod = ref.shape[1]
    peaks = ref[:, :min(2, n_prod)].reshape(ref.shape[0], -1).max(axis=1)
    err = np.abs(gpu.astype(np.float64) - ref).reshape(ref.shape[0], n_prod, -1).max(axis=2)
    return err / peaks[:, None]


def assert_parity(gpu: np.ndarray, ref: np.ndarray, path: str, what: str = ""):
    e = rel_errors(gpu, ref)
    tol = TOL[path]
    assert np.all(np.isfinite(gpu)), f"{what}: non-finite GPU output"
    assert e.max() <= tol, f"{what} [{path}]: max rel error {e.max():.3e} > {tol:.0e}; per chan/prod:\n{e}"
    return e


def oracle_image(cfg, volt, chans=None):
    return oracle.image_cfg(cfg, volt, chans=chans)
