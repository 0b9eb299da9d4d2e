"""Multi-rank plumbing of bench.py on CPU: two gloo ranks (127.0.0.1) run the
replica path's barrier and max-over-ranks reduction, and rank 0's aggregate
equals the units of all ranks over the slowest rank's time (weak scaling)."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), EPIC_BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    step_s = 0.010 * (rank + 1)                   # rank 1 is the slower one
    slowest = bench.reduce_max(step_s, w)
    units = 1000
    value = units * w / slowest
    q.put((rank, slowest, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_and_weak_scaling_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value in res:
        assert slowest == pytest.approx(0.020)
        assert value == pytest.approx(2 * 1000 / 0.020)


def test_recorded_traffic_only_for_the_captured_launch_configuration():
    sys.path.insert(0, ROOT)
    import bench
    import epic_synth as synth
    cfg = synth.config(3)
    rec = bench.json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["k_dftgemm_ws3@cfg3"]
    got = bench.recorded_traffic("k_dftgemm_ws3", 3, 250, cfg, dict(rec["params"]))
    src = open(os.path.join(ROOT, "paper_2609_03027_gb300", "csrc", rec["source"]), "rb").read()
    if bench.hashlib.sha256(src).hexdigest()[:16] != rec["sha"]:
        assert got is None                         # kernel changed since the capture
        return
    assert got == pytest.approx(rec["bytes_per_sample"] * 250)
    other = dict(rec["params"], grid_frames=4)                 # another kernel variant: no record
    assert bench.recorded_traffic("k_dftgemm_ws3", 3, 250, cfg, other) is None
    assert bench.recorded_traffic("k_dftgemm_ws3", 3, 250, cfg, dict(rec["params"], chunk_mb=24576)) == \
        pytest.approx(rec["bytes_per_sample"] * 250)              # chunk size: not part of the key
    assert bench.recorded_traffic("k_dftgemm_ws3", 3, 250, cfg, None) is None
    import dataclasses
    assert bench.recorded_traffic("k_dftgemm_ws3", 3, 250, dataclasses.replace(cfg, input_bits=8),
                                  dict(rec["params"])) is None


def test_reference_arm_prints_one_contract_line():
    # the --impl reference arm runs the FP64 oracle on the host cores, no GPU needed
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--config", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["config"]["workload"].startswith("tiny")
