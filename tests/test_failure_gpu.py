"""Failure detection without a GPU fault: a bounded device wait is made to run out
(a barrier nothing signals, a budget of a few thousand cycles), the plan reports
EPIC_ERR_TIMEOUT once, and the next calls image correctly."""
import threading

import numpy as np
import pytest

import epic_synth as synth
from gpu_common import assert_parity, oracle_image

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_03027_gb300 as E  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)


def _cfg():
    return synth.small_config(n_ant=30, n_chan=2, n_pol=2, grid_n=32, gcf_k=3, n_time=6, seed=91, diameter_m=9.0)


@pytest.mark.parametrize("path", ["dftgemm", "plain"])
def test_wait_that_runs_out_is_reported_once_and_the_plan_recovers(path):
    cfg = _cfg()
    v = synth.make_voltages(cfg)
    ref = oracle_image(cfg, v)
    with E.Plan.from_config(cfg, path=path) as plan:
        d = torch.from_numpy(v).cuda()
        plan.selftest_bounded_wait(5000)
        with pytest.raises(E.EpicError, match="TIMEOUT"):
            plan.sync()
        plan.sync()                                   # reported once, then cleared
        got = plan.image(d).cpu().numpy()
        plan.sync()
        assert_parity(got, ref, path, "after a timed-out wait")
        # the host-buffer call reports a timed-out wait of an earlier, unreported call ...
        plan.selftest_bounded_wait(5000)
        with pytest.raises(E.EpicError, match="TIMEOUT"):
            plan.image_host(v)
        # ... and then images correctly
        assert_parity(plan.image_host(v), ref, path, "host call after a timed-out wait")


def test_tensor_kernels_run_normally_after_the_selftest():
    # the self-test frees the tensor memory it held: the tensor-core kernels that allocate
    # all of an SM's tensor memory still run, back to back, on the same stream
    cfg = _cfg()
    v = synth.make_voltages(cfg)
    with E.Plan.from_config(cfg, path="dftgemm") as plan:
        d = torch.from_numpy(v).cuda()
        base = plan.image(d).cpu().numpy()
        for _ in range(3):
            plan.selftest_bounded_wait(2000)
            out = plan.image(d)
        with pytest.raises(E.EpicError, match="TIMEOUT"):
            plan.sync()
        assert np.array_equal(out.cpu().numpy(), base)


def test_selftest_rejects_bad_budgets():
    with E.Plan.from_config(_cfg(), path="plain") as plan:
        for b in (0, -5, 5_000_000_000):
            with pytest.raises(E.EpicError, match="INVALID"):
                plan.selftest_bounded_wait(b)


def test_ticket_collected_by_exactly_one_of_two_waiters():
    cfg = _cfg()
    v = synth.make_voltages(cfg)
    with E.Plan.from_config(cfg, path="dftgemm") as plan, E.Server(device_bytes=8 << 20, slots=2) as srv:
        out = torch.empty((cfg.n_chan, 4, 32, 32), device="cuda")
        torch.cuda.synchronize()
        t = srv.submit(plan, v, out)
        L = E.load()
        import ctypes
        results = []

        def waiter():
            lat = ctypes.c_double()
            results.append(L.epic_server_wait(srv._h, t, 60000, ctypes.byref(lat)))

        th = [threading.Thread(target=waiter) for _ in range(2)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        assert sorted(results) == [0, 8]              # EPIC_OK once, EPIC_ERR_NOT_FOUND once
        assert np.abs(out.cpu().numpy()).max() > 0
