"""GPU parity: every CUDA path against the FP64 CPU oracle, element by element.

Small cases cover several tiles, ragged time chunks and the method's edge
cases; the four fixed workloads run at full size in the launch configuration
the benchmark times, with the oracle checking sampled channels (lowest and
highest frequency, full integration).
"""
import dataclasses

import numpy as np
import pytest

import epic_synth as synth
from gpu_common import GPU_PATHS, TOL, assert_parity, oracle_image

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_03027_gb300 as E  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)


def run_gpu(cfg, volt, path, **kw):
    with E.Plan.from_config(cfg, path=path, max_time=max(1, volt.shape[0])) as plan:
        v = torch.from_numpy(volt).cuda()
        out = plan.image(v, **kw)
        plan.sync()                                     # also reports a device-side wait timeout
        return out.cpu().numpy()


SMALL = {
    # name: (A, C, P, N, K, T, extra)
    "dual-pol-ragged": (40, 3, 2, 64, 3, 37, {}),
    "single-pol": (25, 2, 1, 32, 3, 19, {}),
    "paper-2x2-gcf": (30, 2, 2, 32, 2, 11, {}),
    "k1-point-gcf": (12, 2, 2, 16, 1, 7, {}),
    "k5-freq-scaled": (50, 4, 2, 64, 5, 9, {"freq_scaled": True}),
    "k7-wide": (64, 2, 2, 128, 7, 5, {}),
    "n8-smallest": (6, 2, 2, 8, 3, 5, {"diameter_m": 3.0}),
    "n256-largest": (300, 2, 2, 256, 3, 3, {"diameter_m": 60.0}),
    "single-time-sample": (33, 3, 2, 32, 4, 1, {}),
}


@pytest.mark.parametrize("path", GPU_PATHS)
@pytest.mark.parametrize("case", list(SMALL))
def test_small_cases_match_oracle(path, case):
    A, C, P, N, K, T, extra = SMALL[case]
    diam = extra.get("diameter_m", 0.28 * N)
    cfg = synth.small_config(n_ant=A, n_chan=C, n_pol=P, grid_n=N, gcf_k=K, n_time=T, seed=100 + A,
                             diameter_m=diam, freq_scaled=extra.get("freq_scaled", False), sigma=0.7)
    v = synth.make_voltages(cfg)
    got = run_gpu(cfg, v, path)
    assert_parity(got, oracle_image(cfg, v), path, case)


@pytest.mark.parametrize("path", GPU_PATHS)
def test_every_byte_code_including_minus_eight(path):
    cfg = synth.small_config(n_ant=64, n_chan=2, n_pol=2, grid_n=32, gcf_k=3, n_time=8, seed=7, diameter_m=9.0)
    v = synth.random_bytes((8, 2, 64, 2), seed=3)
    assert set(np.unique(v)) == set(range(256))
    assert_parity(run_gpu(cfg, v, path), oracle_image(cfg, v), path, "all codes")
    # 8+8-bit: every real and imaginary byte, including -128
    cfg8 = dataclasses.replace(cfg, input_bits=8)
    v8 = synth.random_bytes((8, 2, 64, 2, 2), seed=4)
    assert set(np.unique(v8[..., 0])) == set(range(256)) == set(np.unique(v8[..., 1]))
    assert_parity(run_gpu(cfg8, v8, path), oracle_image(cfg8, v8), path, "all 8-bit codes")


@pytest.mark.parametrize("path", GPU_PATHS)
def test_tabulated_complex_gcf(path):
    K, os_ = 4, 8
    cfg = synth.small_config(n_ant=30, n_chan=2, n_pol=2, grid_n=32, gcf_k=K, n_time=6, seed=17)
    v = synth.make_voltages(cfg)
    side = K * os_ + 1
    s = np.arange(side) / os_ - K / 2.0
    dy, dx = np.meshgrid(s, s, indexing="ij")
    W = np.exp(-(dx ** 2 + 0.7 * dy ** 2) / 2) * np.exp(1j * (0.8 * dx - 0.5 * dy))
    tab = np.stack([W.real, W.imag], -1).astype(np.float32)
    import oracle
    ref = oracle.image(v, cfg.pos_m, cfg.freq_hz, 2, 32, K, 1.0, gcf_kind=oracle.GCF_TABLE, oversample=os_,
                       table=tab)
    with E.Plan(cfg.pos_m, cfg.freq_hz, 2, 32, K, path=path, max_time=6, gcf_table=tab, oversample=os_) as plan:
        got = plan.image(torch.from_numpy(v).cuda()).cpu().numpy()
    assert_parity(got, ref, path, "table gcf")


@pytest.mark.parametrize("path", GPU_PATHS)
def test_tiny_workload_full(path):
    cfg = synth.config(1)
    v = synth.make_voltages(cfg)
    got = run_gpu(cfg, v, path)
    assert_parity(got, oracle_image(cfg, v), path, "64-element 32x32 workload")
    for c in range(cfg.n_chan):                         # the injected source is where Eq. 1 puts it
        iy, ix = np.unravel_index(np.argmax(got[c, 0]), got.shape[2:])
        assert ix in (19, 20) and iy in (14, 15)


_BIG = {}


def _big(idx):
    if idx not in _BIG:
        cfg = synth.config(idx)
        _BIG[idx] = (cfg, synth.make_voltages(cfg))
    return _BIG[idx]


@pytest.mark.parametrize("path", GPU_PATHS)
@pytest.mark.parametrize("idx", [2, 3, 4])
def test_full_workloads_sampled_channels(path, idx):
    cfg, v = _big(idx)
    got = run_gpu(cfg, v, path)
    chans = [0, cfg.n_chan // 2 + 1, cfg.n_chan - 1]
    e = assert_parity(got[chans], oracle_image(cfg, v, chans=chans), path, cfg.name)
    print(f"{path} {cfg.name} T={cfg.n_time}: max error / peak {e.max():.2e} (channels {chans})")
    assert np.all(np.isfinite(got))
    # XX and YY are sums of squares everywhere
    assert got[:, :2].min() >= -TOL[path] * got[:, :2].max()


@pytest.mark.parametrize("path", GPU_PATHS)
def test_accumulate_zero_length_and_split_blocks(path):
    cfg = synth.small_config(n_ant=20, n_chan=3, n_pol=2, grid_n=32, gcf_k=3, n_time=13, seed=23)
    v = synth.make_voltages(cfg)
    ref = oracle_image(cfg, v)
    with E.Plan.from_config(cfg, path=path) as plan:
        d = torch.from_numpy(v).cuda()
        out = torch.full((3, 4, 32, 32), 123.0, device="cuda")
        plan.image(d[:0], out=out)                      # T = 0, reset: zero images
        torch.cuda.synchronize()
        assert float(out.abs().max()) == 0.0
        plan.image(d[:5], out=out)
        plan.image(d[5:5], out=out, accumulate=True)    # T = 0, accumulate: unchanged
        plan.image(d[5:], out=out, accumulate=True)
        assert_parity(out.cpu().numpy(), ref, path, "split block")


@pytest.mark.parametrize("path", GPU_PATHS)
def test_deterministic_and_host_call_identical(path):
    cfg = synth.small_config(n_ant=48, n_chan=2, n_pol=2, grid_n=64, gcf_k=3, n_time=10, seed=31)
    v = synth.make_voltages(cfg)
    with E.Plan.from_config(cfg, path=path) as plan:
        d = torch.from_numpy(v).cuda()
        a = plan.image(d).cpu().numpy()
        b = plan.image(d).cpu().numpy()
        h = plan.image_host(v)
        h2 = plan.image_host(v, out=h.copy(), accumulate=True)
    assert np.array_equal(a, b)                         # no atomics: bitwise reruns
    assert np.array_equal(a, h)
    assert np.allclose(h2, 2 * a, rtol=1e-6, atol=0)


@pytest.mark.parametrize("path", GPU_PATHS)
def test_invalid_calls_fail_before_launch(path):
    cfg = synth.small_config(n_ant=10, n_chan=1, n_pol=2, grid_n=16, gcf_k=3, n_time=4, seed=1, diameter_m=5.0)
    v = synth.make_voltages(cfg)
    with E.Plan.from_config(cfg, path=path, max_time=4) as plan:
        L = E.load()
        out = torch.zeros((1, 4, 16, 16), device="cuda")
        d = torch.from_numpy(v).cuda()
        assert L.epic_image(plan._h, d.data_ptr(), 5, None, out.data_ptr(), 0) == 1       # T > max_time
        assert L.epic_image(plan._h, d.data_ptr(), -1, None, out.data_ptr(), 0) == 1
        assert L.epic_image(plan._h, v.ctypes.data, 4, None, out.data_ptr(), 0) == 1      # host pointer
        assert L.epic_image(plan._h, d.data_ptr(), 4, None, out.data_ptr(), 8) == 1       # unknown flag
        plan.sync()


@pytest.mark.parametrize("path", GPU_PATHS)
def test_one_plan_many_block_lengths(path):
    # the same plan images blocks of many lengths in a row (the tensor path splits
    # the (item, frame) pairs of a launch over the SMs differently for each length)
    cfg = synth.small_config(n_ant=30, n_chan=3, n_pol=2, grid_n=32, gcf_k=3, n_time=40, seed=27)
    v = synth.make_voltages(cfg)
    d = torch.from_numpy(v).cuda()
    with E.Plan.from_config(cfg, path=path) as plan:
        for T in (1, 8, 3, 40, 13, 2, 29):
            got = plan.image(d[:T].contiguous()).cpu().numpy()
            assert_parity(got, oracle_image(cfg, v[:T]), path, f"T={T}")


@pytest.mark.parametrize("path", GPU_PATHS)
def test_512_grid_matches_oracle(path):
    # the largest grid the library takes, a sparse array whose occupied box is 90 cells wide
    cfg = synth.small_config(n_ant=60, n_chan=2, n_pol=2, grid_n=512, gcf_k=3, n_time=3, seed=31,
                             diameter_m=0.32 * 90 * 2.0, sigma=0.7)
    v = synth.make_voltages(cfg)
    got = run_gpu(cfg, v, path)
    assert_parity(got, oracle_image(cfg, v), path, "512 grid")


def test_large_grid_workload_plain_sampled():
    # 20,000 dual-pol elements on a 512 x 512 grid: one frame of voltages (40 KB of bytes,
    # 320 KB unpacked) exceeds shared memory, so the plain path grids from global memory
    cfg = synth.config(6)
    cfg.n_time = 2
    v = synth.make_voltages(cfg)
    got = run_gpu(cfg, v, "plain")
    assert_parity(got, oracle_image(cfg, v), "plain", cfg.name)


@pytest.mark.parametrize("path", GPU_PATHS)
@pytest.mark.parametrize("bits,sub", [(8, 0), (8, 4), (4, 2), (8, 1)])
def test_eight_bit_input_and_sub_integrations(path, bits, sub):
    # 8+8-bit voltages and high-cadence sub-integrations (paper Sec. 4): one image set per
    # `sub` samples, each matching the oracle's; a T = 0 call and a wrong T are handled
    cfg = dataclasses.replace(synth.small_config(n_ant=36, n_chan=3, n_pol=2, grid_n=32, gcf_k=3, n_time=12,
                                                 seed=51 + bits + sub, diameter_m=9.0, sigma=0.7),
                              input_bits=bits, sub_int=sub)
    v = synth.make_voltages(cfg)
    ref = oracle_image(cfg, v)
    with E.Plan.from_config(cfg, path=path) as plan:
        d = torch.from_numpy(v).cuda()
        got = plan.image(d).cpu().numpy()
        assert got.shape == ref.shape
        if sub:
            for k in range(ref.shape[0]):
                assert_parity(got[k], ref[k], path, f"bits={bits} sub={sub} set {k}")
            acc = plan.image(d, out=torch.from_numpy(got).cuda(), accumulate=True).cpu().numpy()
            assert_parity(acc[1] / 2, ref[1], path, "accumulated sub-integration")
            if sub > 1:
                with pytest.raises(E.EpicError):
                    plan.image(d[:sub + 1].contiguous())
        else:
            assert_parity(got, ref, path, f"bits={bits}")
        host = plan.image_host(v)
        assert np.array_equal(host, got)


@pytest.mark.parametrize("path", GPU_PATHS)
@pytest.mark.parametrize("bits,sub", [(4, 0), (8, 3)])
def test_polarisation_mixing_kernels(path, bits, sub):
    # per-element, per-channel 2x2 mixing kernels J W (Eq. 1's W_e^{ap}); then the exchange
    # kernel [[0, 1], [1, 0]] must permute the unmixed products exactly (XX <-> YY, XY -> conj)
    cfg = dataclasses.replace(synth.small_config(n_ant=40, n_chan=3, n_pol=2, grid_n=32, gcf_k=3, n_time=12,
                                                 seed=71 + bits, diameter_m=9.0, sigma=0.7),
                              input_bits=bits, sub_int=sub)
    J = synth.make_jones(cfg, seed=5, gain_rms=0.2, leak_rms=0.2)
    mixed = dataclasses.replace(cfg, jones=J)
    v = synth.make_voltages(cfg)
    ref = oracle_image(mixed, v)
    got = run_gpu(mixed, v, path)
    assert got.shape == ref.shape
    for k in range(ref.shape[0] if sub else 1):
        assert_parity(got[k] if sub else got, ref[k] if sub else ref, path, f"mixed, set {k}")
    swap = np.broadcast_to(np.array([[0, 1], [1, 0]], dtype=np.complex128), J.shape)
    base = run_gpu(cfg, v, path)
    sw = run_gpu(dataclasses.replace(cfg, jones=swap), v, path)
    assert np.array_equal(sw[..., 0, :, :], base[..., 1, :, :])
    assert np.array_equal(sw[..., 1, :, :], base[..., 0, :, :])
    assert np.array_equal(sw[..., 2, :, :], base[..., 2, :, :])
    # Im XY = Im X conj(Y) accumulates with fused multiply-adds whose rounding is not odd under
    # the exchange: equal to FP32 rounding
    assert np.abs(sw[..., 3, :, :] + base[..., 3, :, :]).max() <= 1e-6 * np.abs(base[..., :2, :, :]).max()
    with E.Plan.from_config(mixed, path=path) as plan:
        assert plan.info()["pol_mix"] == 1


TALL = {
    # name: (A, C, P, N, K, T, diameter_m, extra); occupied boxes 54-93 rows tall, so the
    # tensor path cuts them into row parts (channels of one plan into different numbers)
    "dual-pol": (80, 3, 2, 128, 5, 7, 85.0, {}),
    "dual-pol-wide-gcf": (64, 2, 2, 128, 7, 4, 80.0, {"freq_scaled": True}),
    "single-pol": (60, 2, 1, 128, 3, 5, 100.0, {}),
    "n256": (200, 2, 2, 256, 3, 3, 88.0, {}),
    "dual-pol-sub-int": (70, 2, 2, 128, 5, 9, 85.0, {"sub_int": 3}),
    "dual-pol-8bit-mixed": (50, 2, 2, 128, 3, 4, 90.0, {"bits": 8, "jones": True}),
}


@pytest.mark.parametrize("split", [-1, 0, 1])
@pytest.mark.parametrize("case", list(TALL))
def test_tall_boxes_in_row_parts(case, split):
    # occupied grids too tall for the stage-1 results, the stage-2 operand and the stage-2
    # result to sit in tensor memory at once go through the warp-specialised kernel in parts
    # of rows; stage 2 adds the parts up (Eq. 1's sum over the grid rows)
    A, C, P, N, K, T, diam, extra = TALL[case]
    cfg = synth.small_config(n_ant=A, n_chan=C, n_pol=P, grid_n=N, gcf_k=K, n_time=T, seed=300 + A,
                             diameter_m=diam, freq_scaled=extra.get("freq_scaled", False), sigma=0.7)
    cfg = dataclasses.replace(cfg, input_bits=extra.get("bits", 4), sub_int=extra.get("sub_int", 0))
    if extra.get("jones"):
        cfg = dataclasses.replace(cfg, jones=synth.make_jones(cfg, seed=9, gain_rms=0.2, leak_rms=0.2))
    if split == 1 and cfg.sub_int:
        pytest.skip("sub-integrations run whole items")
    v = synth.random_bytes((T, C, A, P) + ((2,) if cfg.input_bits == 8 else ()), seed=A + T)
    ref = oracle_image(cfg, v)
    with E.Plan.from_config(cfg, path="dftgemm", max_time=T) as plan:
        info = plan.info()
        assert info["tc_kernel"] == 3 and info["row_parts"] >= 2, info
        if not cfg.sub_int:
            plan.set_param("split", split)
        d = torch.from_numpy(v).cuda()
        got = plan.image(d).cpu().numpy()
        plan.sync()
        again = plan.image(d).cpu().numpy()
    assert np.array_equal(got, again)
    if cfg.sub_int:
        for k in range(ref.shape[0]):
            assert_parity(got[k], ref[k], "dftgemm", f"{case} set {k}")
    else:
        assert_parity(got, ref, "dftgemm", case)


@pytest.mark.parametrize("grid_kernel", [1, 2, 3])
@pytest.mark.parametrize("case", ["dual-pol", "single-pol", "dual-pol-8bit-mixed", "small"])
def test_every_gridding_kernel_matches_oracle(case, grid_kernel):
    # the tensor path's gridding kernels (row-major cell lists, balanced task lists, row-major
    # pair lists) each write the tiles the transform reads; any of them gives oracle images
    if case == "small":
        cfg = synth.small_config(n_ant=40, n_chan=3, n_pol=2, grid_n=64, gcf_k=5, n_time=9, seed=77, diameter_m=16.0)
        T, A, C, P = 9, 40, 3, 2
    else:
        A, C, P, N, K, T, diam, extra = TALL[case]
        cfg = synth.small_config(n_ant=A, n_chan=C, n_pol=P, grid_n=N, gcf_k=K, n_time=T, seed=500 + A,
                                 diameter_m=diam, sigma=0.7)
        cfg = dataclasses.replace(cfg, input_bits=extra.get("bits", 4))
        if extra.get("jones"):
            cfg = dataclasses.replace(cfg, jones=synth.make_jones(cfg, seed=9, gain_rms=0.2, leak_rms=0.2))
    v = synth.random_bytes((T, C, A, P) + ((2,) if cfg.input_bits == 8 else ()), seed=A + 3 * T)
    ref = oracle_image(cfg, v)
    with E.Plan.from_config(cfg, path="dftgemm", max_time=T) as plan:
        try:
            plan.set_param("grid_kernel", grid_kernel)
        except E.EpicError as ex:
            assert "UNSUPPORTED" in str(ex)
            pytest.skip(f"gridding kernel {grid_kernel} does not take this plan")
        for F in (1, 2, 4, 8):
            try:
                plan.set_param("grid_frames", F)
            except E.EpicError:
                continue
            got = plan.image(torch.from_numpy(v).cuda()).cpu().numpy()
            plan.sync()
            assert_parity(got, ref, "dftgemm", f"{case} grid_kernel={grid_kernel} F={F}")


def test_pair_list_gridding_is_the_default_where_the_balanced_kernel_does_not_fit():
    cfg = synth.config(3).subset([383], n_time=4)   # the tallest SKA-Low channel
    with E.Plan.from_config(cfg, path="dftgemm", max_time=4) as plan:
        assert plan.get_param("grid_kernel") == 3


@pytest.mark.gpu
def test_host_call_of_several_channel_groups_overlaps_copies_and_matches():
    # The SKA-Low station (384 channels: three channel groups on the tensor path) through the
    # host-buffer call, whose per-group copies run beside the other groups' kernels: the same
    # images as the device call, bit for bit, in reset mode, in accumulate mode (one copy, no
    # overlap) and for a pinned buffer given by pointer; and a channel of it against the oracle.
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    cfg = dataclasses.replace(synth.config(3), n_time=24)
    v = synth.make_voltages(cfg)
    with E.Plan.from_config(cfg, path="dftgemm", max_time=cfg.n_time) as plan:
        dev = plan.image(torch.from_numpy(v).cuda()).cpu().numpy()
        torch.cuda.synchronize()
        host = plan.image_host(v)
        assert np.array_equal(host, dev)
        acc = plan.image_host(v, out=host.copy(), accumulate=True)
        assert np.allclose(acc, 2 * dev, rtol=1e-6, atol=0)
        hv = torch.from_numpy(v).pin_memory()
        ho = torch.empty(dev.shape, dtype=torch.float32).pin_memory()
        plan.image_host_ptr(hv.data_ptr(), cfg.n_time, ho.data_ptr(), graph=True)
        assert np.array_equal(ho.numpy(), dev)
        plan.set_param("chunk_mb", 96)                   # several time chunks inside each group
        assert plan.info()["time_chunk"] < cfg.n_time
        dev2 = plan.image(torch.from_numpy(v).cuda()).cpu().numpy()
        torch.cuda.synchronize()
        assert np.array_equal(plan.image_host(v), dev2)
        assert np.allclose(dev2, dev, rtol=1e-5, atol=1e-6 * np.abs(dev).max())
    for c in (0, 200, 383):
        ref = oracle_image(cfg, v, chans=[c])
        assert_parity(host[c:c + 1], ref, "dftgemm", f"host call, channel {c}")


@pytest.mark.parametrize("N", [8, 32, 128, 512])
def test_plain_fft_forms_match_the_oracle(N):
    # both FFT forms of the plain path (register-resident two-pass, shared-memory Stockham)
    cfg = synth.small_config(n_ant=min(40, N * N // 8), n_chan=2, n_pol=2, grid_n=N, gcf_k=3, n_time=5,
                             seed=70 + N, diameter_m=0.28 * N, sigma=0.7)
    v = synth.make_voltages(cfg)
    ref = oracle_image(cfg, v)
    with E.Plan.from_config(cfg, path="plain") as plan:
        d = torch.from_numpy(v).cuda()
        assert plan.get_param("fft") == 0
        a = plan.image(d).cpu().numpy()
        plan.set_param("fft", 1)
        b = plan.image(d).cpu().numpy()
    assert_parity(a, ref, "plain", f"register FFT, N={N}")
    assert_parity(b, ref, "plain", f"Stockham FFT, N={N}")


def test_one_launch_for_every_channel_matches_channel_groups():
    # group = 1: all 384 channels of the SKA-Low station in one launch per kernel (equal-cost
    # shares) against the default channel groups; both against the oracle on sampled channels
    cfg = dataclasses.replace(synth.config(3), n_time=16)
    v = synth.make_voltages(cfg)
    with E.Plan.from_config(cfg, path="dftgemm", max_time=cfg.n_time) as plan:
        d = torch.from_numpy(v).cuda()
        a = plan.image(d).cpu().numpy()
        plan.set_param("group", 1)
        assert plan.get_param("group") == 1
        b = plan.image(d).cpu().numpy()
    assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(a).max())
    for c in (0, 150, 300, 383):
        ref = oracle_image(cfg, v, chans=[c])
        assert_parity(b[c:c + 1], ref, "dftgemm", f"one launch, channel {c}")
