"""CUDA-graph replay (EPIC_GRAPH), the autotuner and its parameters, and the
persistent gridding kernel's partition of (channel, frame) work: every variant
gives the images of the plain call, and matches the FP64 oracle."""
import numpy as np
import pytest

import epic_synth as synth
from gpu_common import GPU_PATHS, assert_parity, oracle_image, rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_03027_gb300 as E  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)


def _cfg(**kw):
    base = dict(n_ant=48, n_chan=5, n_pol=2, grid_n=64, gcf_k=5, n_time=90, seed=41, diameter_m=16.0)
    base.update(kw)
    return synth.small_config(**base)


@pytest.mark.parametrize("path", GPU_PATHS)
def test_graph_replay_equals_plain_call(path):
    cfg = _cfg()
    v = torch.from_numpy(synth.make_voltages(cfg)).cuda()
    with E.Plan.from_config(cfg, path=path) as plan:
        ref = plan.image(v).clone()
        ref_acc = plan.image(v, out=ref.clone(), accumulate=True).clone()
        out = torch.full_like(ref, 7.0)
        for _ in range(3):                       # record once, then replay
            plan.image(v, out=out, graph=True)
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
        out2 = ref.clone()                       # other flags and buffer: recorded again
        plan.image(v, out=out2, accumulate=True, graph=True)
        torch.cuda.synchronize()
        assert torch.equal(out2, ref_acc)
        half = v[: cfg.n_time // 2].contiguous()  # other T
        plan.image(half, out=out, graph=True)
        assert torch.equal(out, plan.image(half))
        plan.image(v, out=out, graph=True, time_kernels=True)
        plan.sync()
        kt = plan.kernel_times()
        assert len(kt) >= 1 and all(ms > 0 for _, ms in kt)
        assert torch.equal(out, ref)


@pytest.mark.parametrize("path", GPU_PATHS)
def test_tuner_keeps_parity_and_reports_params(path):
    cfg = _cfg(seed=42)
    vn = synth.make_voltages(cfg)
    v = torch.from_numpy(vn).cuda()
    with E.Plan.from_config(cfg, path=path) as plan:
        before = plan.image(v).cpu().numpy()
        rep = plan.tune(v, reps=2)
        assert rep["n_timed"] >= 1 and rep["best_ms"] <= rep["default_ms"] + 1e-6
        for name, val in rep["params"].items():
            assert plan.get_param(name) == val
        after = plan.image(v).cpu().numpy()
    # FP32 summation order only; on the tensor path the two gridding kernels sum a cell in
    # different orders, which can flip the rounding of an FP16 grid value
    assert rel_errors(after, before.astype(np.float64)).max() <= (1e-5 if path == "dftgemm" else 1e-6)
    assert_parity(after, oracle_image(cfg, vn), path, "after tuning")


def test_gridding_frames_per_pass_bitwise_identical():
    # more (channel, frame) pairs than gridding blocks: passes of several frames,
    # block ranges that cross channel boundaries, a ragged last pass
    cfg = _cfg(n_chan=7, n_time=301, seed=43)
    vn = synth.make_voltages(cfg)
    v = torch.from_numpy(vn).cuda()
    with E.Plan.from_config(cfg, path="dftgemm") as plan:
        outs = {}
        for F in (1, 2, 4, 8):
            try:
                plan.set_param("grid_frames", F)
            except E.EpicError as ex:            # F frames may not fit in shared memory
                assert ex.status == 7
                continue
            assert plan.get_param("grid_frames") == F
            outs[F] = plan.image(v).cpu().numpy()
        assert len(outs) >= 2
        first = next(iter(outs.values()))
        for F, o in outs.items():
            assert np.array_equal(o, first), F
        # both gridding kernels (row-major walk in element order; length-sorted cell lists in
        # an order chosen for the shared-memory banks) alike up to FP32 summation order, and
        # each bitwise the same for every number of frames per pass
        last = first
        for gk in (1, 2):
            try:
                plan.set_param("grid_kernel", gk)
            except E.EpicError as ex:
                assert ex.status in (7, 8)
                continue
            o = plan.image(v).cpu().numpy()
            assert rel_errors(o, first.astype(np.float64)).max() <= 1e-5, gk
            for F in (1, 2):
                try:
                    plan.set_param("grid_frames", F)
                except E.EpicError as ex:
                    assert ex.status == 7
                    continue
                assert np.array_equal(plan.image(v).cpu().numpy(), o), (gk, F)
            last = o
        # voltage block at an address that is not 16-byte aligned: no bulk copies
        raw = torch.zeros(v.numel() + 16, dtype=torch.uint8, device="cuda")
        va = raw[1:1 + v.numel()].view(v.shape)
        va.copy_(v)
        assert va.data_ptr() % 16 == 1
        assert np.array_equal(plan.image(va).cpu().numpy(), last)
    assert_parity(first, oracle_image(cfg, vn), "dftgemm", "frames per pass")


@pytest.mark.parametrize("path,name,values", [("plain", "chunk_mb", [128, 1024]),
                                              ("dftgemm", "chunk_mb", [24, 192]),
                                              ("fused", "slab", [8, 16, 32])])
def test_set_param_values_match_oracle(path, name, values):
    cfg = _cfg(n_time=64, seed=44)
    vn = synth.make_voltages(cfg)
    v = torch.from_numpy(vn).cuda()
    ref = oracle_image(cfg, vn)
    with E.Plan.from_config(cfg, path=path) as plan:
        with pytest.raises(E.EpicError) as ex:
            plan.set_param("no_such_parameter", 1)
        assert ex.value.status == 8
        for val in values:
            plan.set_param(name, val)
            assert_parity(plan.image(v).cpu().numpy(), ref, path, f"{name}={val}")


@pytest.mark.parametrize("path", GPU_PATHS)
def test_plan_created_later_does_not_break_earlier_plan(path):
    # kernels are shared by all plans: a later plan with smaller boxes must not
    # lower the shared-memory limit the earlier plan's launches need
    big = _cfg(n_ant=120, n_chan=3, grid_n=128, gcf_k=7, n_time=20, seed=45, diameter_m=40.0)
    small = _cfg(n_ant=10, n_chan=2, grid_n=16, gcf_k=3, n_time=20, seed=46, diameter_m=4.0)
    vb, vs = synth.make_voltages(big), synth.make_voltages(small)
    with E.Plan.from_config(big, path=path) as pb, E.Plan.from_config(small, path=path) as ps:
        ob = pb.image(torch.from_numpy(vb).cuda()).cpu().numpy()
        os_ = ps.image(torch.from_numpy(vs).cuda()).cpu().numpy()
        pb.sync()
        ps.sync()
    assert_parity(ob, oracle_image(big, vb), path, "earlier plan")
    assert_parity(os_, oracle_image(small, vs), path, "later plan")


def test_auto_path_tunes_the_path_and_keeps_parity():
    # an AUTO plan starts on the tensor path; the tuner times every path that takes the plan
    # and keeps the fastest, then tunes that path's own parameters
    cfg = _cfg(seed=44)
    vn = synth.make_voltages(cfg)
    v = torch.from_numpy(vn).cuda()
    ref = oracle_image(cfg, vn)
    with E.Plan.from_config(cfg, path="auto") as plan:
        assert plan.info()["path_name"] == "dftgemm"
        rep = plan.tune(v, reps=1)
        assert "path" in rep["params"] and rep["params"]["path"] == plan.info()["path"]
        got = plan.image(v).cpu().numpy()
        plan.sync()
        assert_parity(got, ref, plan.info()["path_name"], "auto after tuning")
        for name, path in (("plain", 0), ("fused", 1), ("dftgemm", 2)):   # each path on demand
            plan.set_param("path", path)
            assert plan.get_param("path") == path and plan.info()["path_name"] == name
            assert_parity(plan.image(v).cpu().numpy(), ref, name, f"auto plan set to {name}")


def test_auto_path_takes_a_grid_the_tensor_path_refuses():
    # 20,000 dual-pol elements on a 512 x 512 grid: the occupied box is too tall for the
    # tensor-core kernels, so an AUTO plan lands on the plain FP32 path and images correctly
    cfg = synth.config(6)
    cfg.n_time = 2
    vn = synth.make_voltages(cfg)
    with E.Plan.from_config(cfg, path="auto", max_time=2) as plan:
        assert plan.info()["path_name"] == "plain"
        got = plan.image(torch.from_numpy(vn).cuda()).cpu().numpy()
        plan.sync()
        rep = plan.tune(torch.from_numpy(vn).cuda(), reps=1)
        assert rep["params"]["path"] in (0, 1)
    assert_parity(got, oracle_image(cfg, vn), "plain", cfg.name)
