"""Streaming server (continuous batching): every block's images are the same when
imaged alone and in the mix, integrations continue across blocks, and latency
statistics are reported."""
import ctypes

import numpy as np
import pytest

import epic_synth as synth
from gpu_common import assert_parity, oracle_image

torch = pytest.importorskip("torch")

import paper_2609_03027_gb300 as E  # noqa: E402


def _stations():
    # four station types of different sizes, each with its own plan and path
    specs = [
        dict(n_ant=24, n_chan=3, n_pol=2, grid_n=32, gcf_k=3, n_time=9, seed=61, diameter_m=9.0),
        dict(n_ant=64, n_chan=2, n_pol=2, grid_n=64, gcf_k=5, n_time=20, seed=62, diameter_m=16.0),
        dict(n_ant=120, n_chan=4, n_pol=2, grid_n=64, gcf_k=3, n_time=12, seed=63, diameter_m=17.0),
        dict(n_ant=40, n_chan=2, n_pol=1, grid_n=32, gcf_k=3, n_time=7, seed=64, diameter_m=9.0),
    ]
    paths = ["dftgemm", "fused", "dftgemm", "plain"]
    return [(synth.small_config(**sp), path) for sp, path in zip(specs, paths)]


@pytest.mark.gpu
def test_each_block_same_alone_and_in_the_mix():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    stations = _stations()
    plans = [E.Plan.from_config(cfg, path=path) for cfg, path in stations]
    blocks = []
    for si, (cfg, _) in enumerate(stations):
        for b in range(3):
            T = cfg.n_time - b
            v = synth.make_voltages(cfg, t0=5 * b, n_time=T)
            blocks.append((si, v))
    # alone
    alone = []
    for si, v in blocks:
        out = plans[si].image(torch.from_numpy(v).cuda())
        torch.cuda.synchronize()
        alone.append(out.cpu().numpy())
    # in the mix: all submitted at once, different stations overlap on the device
    outs = [torch.full((stations[si][0].n_chan, stations[si][0].n_prod, stations[si][0].grid_n,
                        stations[si][0].grid_n), -1.0, device="cuda") for si, _ in blocks]
    torch.cuda.synchronize()                  # the server's streams do not wait for torch's
    with E.Server(device_bytes=64 << 20, slots=4) as srv:
        tickets = []
        for (si, v), o in zip(blocks, outs):
            t = None
            while t is None:
                t = srv.submit(plans[si], v, o)
            tickets.append(t)
        lat = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(blocks)
    assert all(x > 0 for x in lat)
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    for (si, v), o, ref in zip(blocks, outs, alone):
        assert np.array_equal(o.cpu().numpy(), ref), f"station {si}"
    # a seeded sample of the served blocks against the FP64 oracle
    for k in np.random.default_rng(5).choice(len(blocks), size=3, replace=False):
        si, v = blocks[k]
        cfg, path = stations[si]
        assert_parity(outs[k].cpu().numpy(), oracle_image(cfg, v), path, f"served block {k} (station {si})")
    for p in plans:
        p.close()


@pytest.mark.gpu
def test_integration_continues_across_blocks():
    cfg, path = _stations()[1]
    plan = E.Plan.from_config(cfg, path="dftgemm")
    vs = [synth.make_voltages(cfg, t0=7 * b, n_time=cfg.n_time) for b in range(3)]
    ref = torch.empty((cfg.n_chan, 4, cfg.grid_n, cfg.grid_n), device="cuda")
    for b, v in enumerate(vs):
        plan.image(torch.from_numpy(v).cuda(), out=ref, accumulate=b > 0)
    acc = torch.full_like(ref, 5.0)
    torch.cuda.synchronize()                  # the server's streams do not wait for torch's
    with E.Server(device_bytes=32 << 20, slots=2) as srv:
        ts = [srv.submit(plan, v, acc, accumulate=b > 0) for b, v in enumerate(vs)]
        for t in ts:
            srv.wait(t)
    assert torch.equal(acc, ref)
    plan.close()


@pytest.mark.gpu
def test_block_larger_than_pool_is_refused():
    cfg, _ = _stations()[0]
    plan = E.Plan.from_config(cfg, path="plain")
    v = synth.make_voltages(cfg)
    out = torch.empty((cfg.n_chan, 4, cfg.grid_n, cfg.grid_n), device="cuda")
    with E.Server(device_bytes=1024, slots=1) as srv:
        with pytest.raises(E.EpicError, match="OOM"):
            srv.submit(plan, v, out)
    plan.close()


def test_server_argument_checks_on_host():
    L = E.load()
    h = ctypes.c_void_p()
    assert L.epic_server_create(1 << 20, 0, ctypes.byref(h)) == 1      # no slots
    assert L.epic_server_create(1 << 20, 65, ctypes.byref(h)) == 1     # too many slots
    assert L.epic_server_create(16, 2, ctypes.byref(h)) == 1           # pool too small
    assert L.epic_server_create(1 << 20, 2, None) == 1
    t = ctypes.c_uint64()
    assert L.epic_server_submit(None, None, None, 0, None, 0, ctypes.byref(t)) == 1
    d, lat = ctypes.c_int(), ctypes.c_double()
    assert L.epic_server_poll(None, 1, ctypes.byref(d), ctypes.byref(lat)) == 1
    assert L.epic_server_destroy(None) == 0


# (station type of the streaming mix, channels per block): every type, including the
# dual-pol 64-element 32 x 32 station and the 1024-element lattice, at its full block
# length, with the mix's channel plan
MIX_BLOCKS = [(0, 384), (1, 128), (2, 64), (3, 32)]


@pytest.mark.gpu
@pytest.mark.parametrize("path", ["plain", "dftgemm"])
def test_streaming_mix_station_types_match_oracle(path):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    types = synth.mixed_station_types()
    cfgs = [synth.serving_config(types[t], C) for t, C in MIX_BLOCKS]
    plans = [E.Plan.from_config(cfg, path=path, max_time=cfg.n_time) for cfg in cfgs]
    volts = [synth.make_voltages(cfg) for cfg in cfgs]
    outs = [torch.empty((cfg.n_chan, cfg.n_prod, cfg.grid_n, cfg.grid_n), device="cuda") for cfg in cfgs]
    torch.cuda.synchronize()
    pool = 2 * max(v.nbytes for v in volts)
    with E.Server(device_bytes=pool, slots=4) as srv:
        tickets = []
        for plan, v, o in zip(plans, volts, outs):
            t = None
            while t is None:
                t = srv.submit(plan, v, o)
            tickets.append(t)
        for t in tickets:
            srv.wait(t, timeout_ms=600000)
    for cfg, v, o in zip(cfgs, volts, outs):
        chans = [0, cfg.n_chan // 2, cfg.n_chan - 1]
        e = assert_parity(o.cpu().numpy()[chans], oracle_image(cfg, v, chans=chans), path, cfg.name)
        print(f"{path} {cfg.name} T={cfg.n_time}: max error / peak {e.max():.2e}")
    for p in plans:
        p.close()


@pytest.mark.gpu
def test_small_and_large_blocks_under_concurrent_load_never_time_out():
    # Stress for the tensor kernel's barrier hand-offs: thousands of short blocks (32 x 32
    # grids, three or four tile buffers, many sub-frames per item) served four at a time next
    # to long ones.  A copy thread that waited for buffer reuse on a barrier shared by two
    # buffers once let one such block in about 3 000 run into its bounded wait; every block
    # must complete with EPIC_OK and the small plan's images must equal its lone call's.
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    types = synth.mixed_station_types()
    small = synth.serving_config(types[0], 128)              # 64-element station, 32 x 32 grid
    large = synth.serving_config(types[1], 64)               # 256-element station, 128 x 128 grid
    plans = [E.Plan.from_config(cfg, path="dftgemm", max_time=cfg.n_time) for cfg in (small, large)]
    vs = [torch.from_numpy(synth.make_voltages(cfg)) for cfg in (small, large)]
    ref = plans[0].image(vs[0].cuda())
    torch.cuda.synchronize()
    n_small = 8                                              # outputs of the small plan in flight
    outs = [torch.empty_like(ref) for _ in range(n_small)]
    out_large = torch.empty((large.n_chan, large.n_prod, large.grid_n, large.grid_n), device="cuda")
    h = [v.pin_memory() for v in vs]
    torch.cuda.synchronize()
    with E.Server(device_bytes=4 * max(v.numel() for v in vs) + (64 << 20), slots=4) as srv:
        tickets = []
        for i in range(3000):
            k, out = (1, out_large) if i % 10 == 9 else (0, outs[i % n_small])
            t = None
            while t is None:
                t = srv.submit_ptr(plans[k], h[k].data_ptr(), (small, large)[k].n_time, out)
            tickets.append(t)
        for t in tickets:
            srv.wait(t, timeout_ms=600000)                   # raises on any status but EPIC_OK
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o, ref)
    for p in plans:
        p.close()
