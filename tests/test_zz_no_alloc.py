"""Imaging through the entry point that allocates no device memory
(epic_image_static_scratch): its grid scratch is a fixed array in the library's
device image, for callers that may not call cudaMalloc while imaging (code whose
device memory is owned by another framework's pool, or real-time loops where an
allocation could stall).  Checked against epic_image, two calls in a row, through
the C ABI.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import epic_synth as synth
from gpu_common import TOL, assert_parity

torch = pytest.importorskip("torch")

import paper_2609_03027_gb300 as E  # noqa: E402


def _entry():
    L = E.load()
    f = L.epic_image_static_scratch
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint]
    f.restype = ctypes.c_int
    return L, f


@pytest.mark.gpu
def test_static_scratch_matches_epic_image_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    torch.cuda.set_device(0)
    L, f = _entry()
    cfg = synth.small_config(n_ant=48, n_chan=3, n_pol=2, grid_n=64, gcf_k=3, n_time=11, seed=91, diameter_m=16.0)
    with E.Plan.from_config(cfg, path="plain") as plan:
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):                                   # the array keeps the last call's contents
            v = torch.from_numpy(synth.make_voltages(cfg, t0=13 * call, n_time=cfg.n_time)).cuda()
            ref = plan.image(v)
            out = torch.full_like(ref, 7.0)
            st = f(plan._h, v.data_ptr(), v.shape[0], stream, out.data_ptr(), 0)
            assert st == 0, L.epic_last_error(plan._h).decode()
            torch.cuda.synchronize()
            assert_parity(out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64), "plain",
                          f"static-scratch call {call}")
            # accumulate: a second block added to the first
            st = f(plan._h, v.data_ptr(), v.shape[0], stream, out.data_ptr(), 1)
            assert st == 0
            torch.cuda.synchronize()
            rel = (out - 2 * ref).abs().max().item() / ref[:, :2].abs().max().item()
            assert rel <= TOL["plain"]


@pytest.mark.gpu
def test_static_scratch_rejects_blocks_beyond_its_size():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    L, f = _entry()
    # 160 channels x 2 pols x 128^2 x 8 bytes = 40 MiB per time sample > 32 MiB
    cfg = synth.small_config(n_ant=16, n_chan=160, n_pol=2, grid_n=128, gcf_k=3, n_time=2, seed=92, diameter_m=20.0)
    with E.Plan.from_config(cfg, path="plain") as plan:
        v = torch.zeros((2, 160, 16, 2), dtype=torch.uint8, device="cuda")
        out = torch.zeros((160, 4, 128, 128), device="cuda")
        st = f(plan._h, v.data_ptr(), 2, torch.cuda.current_stream().cuda_stream, out.data_ptr(), 0)
        assert st == 7                                          # EPIC_ERR_UNSUPPORTED
        assert "MiB" in L.epic_last_error(plan._h).decode()


@pytest.mark.gpu
def test_static_scratch_rejects_formats_it_does_not_take():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import dataclasses
    L, f = _entry()
    base = synth.small_config(n_ant=16, n_chan=2, n_pol=2, grid_n=32, gcf_k=3, n_time=4, seed=93, diameter_m=8.0)
    variants = [dataclasses.replace(base, input_bits=8), dataclasses.replace(base, sub_int=2),
                dataclasses.replace(base, jones=synth.make_jones(base, seed=1))]
    for cfg in variants:
        with E.Plan.from_config(cfg, path="plain") as plan:
            v = torch.from_numpy(synth.make_voltages(cfg)).cuda()
            out = torch.zeros(plan.image_shape(cfg.n_time), device="cuda")
            st = f(plan._h, v.data_ptr(), cfg.n_time, torch.cuda.current_stream().cuda_stream, out.data_ptr(), 0)
            assert st == 7, L.epic_last_error(plan._h).decode()        # EPIC_ERR_UNSUPPORTED


@pytest.mark.gpu
def test_static_scratch_smallest_grid_many_samples():
    # N = 8, one channel, one pol: 65,536 samples fit the array at once, more than one launch
    # dimension takes, so the call runs in chunks; two calls in a row against epic_image
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    L, f = _entry()
    cfg = synth.small_config(n_ant=6, n_chan=1, n_pol=1, grid_n=8, gcf_k=3, n_time=70000, seed=94, diameter_m=3.0)
    with E.Plan.from_config(cfg, path="plain") as plan:
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            v = torch.from_numpy(synth.random_bytes((cfg.n_time, 1, 6, 1), seed=40 + call)).cuda()
            ref = plan.image(v)
            out = torch.full_like(ref, 3.0)
            st = f(plan._h, v.data_ptr(), cfg.n_time, stream, out.data_ptr(), 0)
            assert st == 0, L.epic_last_error(plan._h).decode()
            torch.cuda.synchronize()
            assert_parity(out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64), "plain",
                          f"N=8 static-scratch call {call}")
