#!/usr/bin/env python3
"""Throughput benchmark of the EPIC imaging path on GB300.

One step = one epic_image call over one whole voltage block of the SKA-Low-
station-like workload (256 dual-pol elements in a 38 m disc, 384 channels from
50 to 350 MHz, 128x128 grid, 7x7 frequency-scaled Gaussian GCF, 512 time
samples; the largest of the single-GPU workloads): every (t, c, p) is unpacked,
gridded, transformed, multiplied and accumulated.  --config picks another.

Metric: pixel-updates/s = N^2 x channels x pols x time samples / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--path dftgemm|fused|plain]
  python bench.py --impl reference ...   (the FP64 CPU oracle, timed on host cores)

Prints one JSON line (rank 0).  Under torchrun every rank images its own block
(independent replicas, weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import epic_synth as synth  # noqa: E402

METRIC = "pixel-updates/s (grid²×chan×pol×t)"
UNIT = "pixel-updates/s"
L2_BYTES = 129 * 1024 * 1024
FLUSH_BYTES = 256 * 1024 * 1024

WORKLOADS = {
    1: "tiny: 64 el, 1 pol, 4 ch, 32x32 grid, 3x3 GCF, T=256",
    2: "lwa-station: 256 dual-pol el in 100x110 m ellipse, 128 ch x 25 kHz @ 56 MHz, 128x128 grid, 5x5 GCF, T=1000",
    3: "skalow-station: 256 dual-pol el in 38 m disc, 384 ch 50-350 MHz, 128x128 grid, 7x7 freq-scaled GCF, T=512",
    4: "dense-4096: 64x64 jittered lattice dual-pol, 64 ch from 150 MHz, 256x256 grid, 3x3 GCF, T=256",
    6: "large-grid: 20000 dual-pol el in 240 m disc, 1 x 781.25 kHz ch @ 159 MHz, 512x512 grid, 2x2 GCF, T=1000",
}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"), "sm_max_mhz": d.get("sm_max_mhz", 2070.0),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
            "source": "fallback"}


# ----------------------------------------------------------------------------- algorithmic work models

def fft_flops_per_block(cfg, T):
    """Method's own work (FFT count 5 M log2 M per M = N^2 point transform, gridding 8 A K^2
    per pol-frame, products 4 N^2 / 12 N^2 per frame), per block of T samples."""
    N, C, P, A, K = cfg.grid_n, cfg.n_chan, cfg.n_pol, cfg.n_ant, cfg.gcf_k
    M = N * N
    per_frame = P * (5.0 * M * np.log2(M) + 8.0 * A * K * K) + (12.0 if P == 2 else 4.0) * M
    return per_frame * C * T


def kernel_model(name, cfg, T, info):
    """(bound, algorithmic units per launch, unit) for a kernel of one step."""
    N, C, P, A = cfg.grid_n, cfg.n_chan, cfg.n_pol, cfg.n_ant
    nprod = 4 if P == 2 else 1
    tc = max(1, info.get("time_chunk") or T)
    nt = min(tc, T)
    grid_bytes = nt * C * P * N * N * 8
    if name == "k_plain_grid":
        return "hbm", nt * C * A * P + grid_bytes, "B"
    if name in ("k_plain_fft_rows", "k_plain_fft_cols"):
        return "hbm", 2 * grid_bytes, "B"
    if name == "k_plain_sqacc":
        return "hbm", grid_bytes + 2 * C * nprod * N * N * 4, "B"
    if name.startswith("k_fused"):
        return "alu", fft_flops_per_block(cfg, T), "flop"
    if name in ("k_dftgemm_mma", "k_dftgemm_mma_fast", "k_dftgemm_ws", "k_dftgemm_ws2", "k_dftgemm_ws3"):
        return "tensor", float(info.get("gemm_flops_per_sample", 0.0)) * T, "flop"
    if name == "k_dftgemm_grid":
        tile = 4 * P * info.get("box_max_x", 0) * info.get("box_max_y", 0)
        return "hbm", T * C * A * P + T * C * tile, "B"
    return "hbm", T * C * A * P + C * nprod * N * N * 4, "B"


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        out.update(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


# ----------------------------------------------------------------------------- distributed plumbing

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("EPIC_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x: float, world: int, device=None) -> float:
    """Max of a float over ranks (timing: the slowest rank decides)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- CPU baseline (oracle)

def cpu_baseline(cfg, volt, seconds_hint: float = 20.0, n_time=None):
    """The FP64 oracle as it stands on a bounded sample: n channels x T samples, all cores."""
    import oracle
    cores = os.cpu_count() or 1
    n_ch = min(cfg.n_chan, cores)
    T = volt.shape[0] if n_time is None else n_time
    chans = list(np.linspace(0, cfg.n_chan - 1, n_ch).astype(int))
    # repeat the sample until about seconds_hint of CPU work has been timed (at most 3x that)
    reps, dt = 0, 0.0
    while dt < seconds_hint and reps < 1000:
        t0 = time.perf_counter()
        oracle.image_cfg(cfg, volt[:T], chans=chans, threads=n_ch)
        dt += time.perf_counter() - t0
        reps += 1
        if dt / reps * (reps + 1) > 3 * seconds_hint:
            break
    units = cfg.grid_n ** 2 * n_ch * cfg.n_pol * T * reps
    t1 = time.perf_counter()                       # and one core on one of those channels
    oracle.image_cfg(cfg, volt[:T], chans=chans[:1], threads=1)
    dt1 = time.perf_counter() - t1
    return {"value": units / dt, "unit": UNIT, "cores": n_ch, "kind": "oracle",
            "value_one_core": cfg.grid_n ** 2 * cfg.n_pol * T / dt1,
            "sample": f"{n_ch} of {cfg.n_chan} channels x {T} samples, {reps} times, OpenMP over channels "
                      f"({dt:.1f} s); one core: 1 channel x {T} samples ({dt1:.2f} s)"}


def run_reference(args, cfg, world, rank):
    """--impl reference: the FP64 CPU oracle on host cores, same metric and workload."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    T = min(cfg.n_time, args.ref_time)
    volt = synth.make_voltages(cfg, 0, T)
    cores = os.cpu_count() or 1
    n_ch = min(cfg.n_chan, cores)
    chans = list(np.linspace(0, cfg.n_chan - 1, n_ch).astype(int))
    for _ in range(args.warmup):
        oracle.image_cfg(cfg, volt, chans=chans, threads=n_ch)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.image_cfg(cfg, volt, chans=chans, threads=n_ch)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    units = cfg.grid_n ** 2 * n_ch * cfg.n_pol * T
    val = units / (ms / 1e3)
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOADS[args.config], "path": "cpu-oracle-fp64",
                       "sample_per_step": f"{n_ch} channels x {T} samples"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": n_ch, "kind": "oracle",
                             "sample": f"{n_ch} of {cfg.n_chan} channels x {T} samples per step"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- traffic record

def recorded_traffic(kernel: str, workload: int, samples: int, cfg, params):
    """DRAM bytes of one launch processing `samples` time samples, from the committed ncu
    summary (profiles/traffic.json: bytes per sample of one capture), if the kernel source,
    the input format and the plan parameters are those of the capture; None otherwise."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path) or cfg.input_bits != 4 or cfg.sub_int or cfg.jones is not None:
        return None
    key = "k_dftgemm_grid" if kernel.startswith("k_dftgemm_grid") else kernel
    rec = json.load(open(path)).get(f"{key}@cfg{workload}")
    if not rec:
        return None
    if any((params or {}).get(k) != v for k, v in rec.get("params", {}).items()):
        return None
    src = os.path.join(ROOT, "paper_2609_03027_gb300", "csrc", rec["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != rec["sha"]:
        return None
    return float(rec["bytes_per_sample"]) * samples


def run_e2e(E, cfg, volt, out, T, units, world, dev, args, tuning=None):
    """Same metric through the host-buffer call: pinned H2D + imaging + D2H every step."""
    import torch
    plan = E.Plan.from_config(cfg, path=args.path, max_time=T)
    for name, val in (tuning or {}).items():       # the values the autotuner chose for the device run
        plan.set_param(name, val)
    graph = not args.no_graph
    h_volt = torch.from_numpy(volt).pin_memory()
    h_out = torch.empty(out.shape, dtype=torch.float32).pin_memory()
    for _ in range(2):
        plan.image_host_ptr(h_volt.data_ptr(), T, h_out.data_ptr(), graph=graph)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        plan.image_host_ptr(h_volt.data_ptr(), T, h_out.data_ptr(), graph=graph)
    e2e_s = reduce_max((time.perf_counter() - t0) / args.e2e_steps, world, dev)
    plan.close()
    return {"value": units * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(volt.nbytes),
            "d2h_bytes_per_step": int(h_out.numel() * 4), "ms_per_step": 1e3 * e2e_s}


# ----------------------------------------------------------------------------- serving (streaming mix)

SERVE_CHANNELS = synth.SERVE_CHANNELS


def serving_plans_spec():
    """Config of every (station type, channel count) of the streaming mix: the
    64/256/1024/4096-element station types, C contiguous 25 kHz channels from each
    type's first frequency."""
    return [synth.serving_config(st, C) for st in synth.mixed_station_types() for C in SERVE_CHANNELS]


def run_serving(E, args, dev):
    """Poisson arrivals (mean 10 ms) of blocks from the station mix for args.serve_seconds,
    imaged by the continuous-batching server; p50/p99 latency and pixel-updates/s."""
    import torch
    rng = np.random.default_rng(5)
    specs = serving_plans_spec()
    plans, outs, blocks = [], [], []
    for cfg in specs:
        plans.append(E.Plan.from_config(cfg, path=args.path, max_time=cfg.n_time))
        outs.append(torch.empty((cfg.n_chan, cfg.n_prod, cfg.grid_n, cfg.grid_n), dtype=torch.float32, device=dev))
        n = cfg.voltage_bytes()
        d = torch.randint(0, 256, (n,), dtype=torch.uint8, device=dev)
        h = torch.empty(n, dtype=torch.uint8).pin_memory()
        h.copy_(d)
        blocks.append(h)
        del d
    torch.cuda.synchronize()
    pool = 2 * max(b.numel() for b in blocks) + (256 << 20)
    n_types = len(synth.mixed_station_types())
    arrivals, t = [], 0.0
    while t < args.serve_seconds:
        t += rng.exponential(0.010)
        arrivals.append((t, int(rng.integers(0, n_types)) * len(SERVE_CHANNELS) + int(rng.integers(0, len(SERVE_CHANNELS)))))
    tickets = []
    with E.Server(device_bytes=pool, slots=4) as srv:
        for k in range(len(specs)):              # warm-up: every plan's first block outside the window
            tk = None
            while tk is None:
                tk = srv.submit_ptr(plans[k], blocks[k].data_ptr(), specs[k].n_time, outs[k])
            srv.wait(tk)
        srv_base = srv.stats()["completed"]
        t0 = time.perf_counter()
        for at, k in arrivals:
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            tk = None
            while tk is None:
                tk = srv.submit_ptr(plans[k], blocks[k].data_ptr(), specs[k].n_time, outs[k])
                if tk is None:
                    time.sleep(2e-4)
            tickets.append((tk, at, time.perf_counter() - t0, k))
        lat_arrival, units = [], 0
        for tk, at, sub, k in tickets:
            lat = srv.wait(tk, timeout_ms=600000)
            lat_arrival.append(1e3 * (sub - at) + lat)
            units += specs[k].pixel_updates()
        wall = time.perf_counter() - t0
        st = srv.stats()
    torch.cuda.synchronize()
    # the FP64 oracle on a seeded 2% sample of the served blocks: a plan's blocks all image the
    # same bytes into the same images, so its images after the run are those of every block
    check = serving_oracle_check(rng, tickets, specs, blocks, outs, args.path)
    for p in plans:
        p.close()
    la = np.array(lat_arrival)
    return {"workload": "streaming mix: 64/256/1024/4096-el dual-pol stations, C in {32,64,128,256,384} x 25 kHz, "
                        "Poisson arrivals mean 10 ms",
            "seconds": args.serve_seconds, "blocks": len(tickets), "value": units / wall, "unit": UNIT,
            "p50_ms": float(np.percentile(la, 50)), "p99_ms": float(np.percentile(la, 99)),
            "server_p50_ms": st["p50_ms"], "server_p99_ms": st["p99_ms"],
            "latency": "from arrival (incl. admission wait) to completion; server_* from submission",
            "completed": st["completed"] - srv_base, "oracle_check": check}


def serving_oracle_check(rng, tickets, specs, blocks, outs, path):
    """Max error / peak of a seeded 2% sample of the served blocks (first and last channel of
    each sampled block's station and channel plan) against the FP64 oracle."""
    import oracle
    oracle.build()
    n = max(1, int(round(0.02 * len(tickets))))
    picked = sorted({tickets[i][3] for i in rng.choice(len(tickets), size=n, replace=False)})
    worst = 0.0
    for k in picked:
        cfg = specs[k]
        v = blocks[k].numpy().reshape(cfg.n_time, cfg.n_chan, cfg.n_ant, cfg.n_pol)
        chans = [0, cfg.n_chan - 1]
        ref = oracle.image_cfg(cfg, v, chans=chans)
        got = outs[k].cpu().numpy()[chans].astype(np.float64)
        peak = ref[:, :2].reshape(len(chans), -1).max(axis=1)
        worst = max(worst, float((np.abs(got - ref).reshape(len(chans), ref.shape[1], -1).max(axis=2)
                                  / peak[:, None]).max()))
    tol = 1e-5 if path in ("plain", "fused") else 2e-3
    return {"blocks_sampled": n, "plans_checked": len(picked), "max_err_over_peak": worst, "tolerance": tol,
            "pass": worst <= tol}


# ----------------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="epic", choices=["epic", "reference"])
    ap.add_argument("--path", default="dftgemm", choices=["plain", "fused", "dftgemm", "auto"])
    ap.add_argument("--config", type=int, default=3, choices=[1, 2, 3, 4, 6])
    ap.add_argument("--compare", default="plain", help="also time this path (comma list; 'none' or '' for none)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--ref-time", type=int, default=250, help="time samples per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--time", type=int, default=0, help="override the block length T (small profiling cases)")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (plan defaults)")
    ap.add_argument("--params", default="", help="tuning parameters to set instead of tuning, e.g. split=1,chunk_mb=768")
    ap.add_argument("--no-graph", action="store_true", help="launch kernel by kernel instead of a CUDA graph")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the streaming-mix serving run (0 = skip)")
    ap.add_argument("--input-bits", type=int, default=4, choices=[4, 8], help="voltage sample format")
    ap.add_argument("--sub-int", type=int, default=0, help="samples per image set (0 = whole block)")
    ap.add_argument("--pol-mix", action="store_true",
                    help="per-element polarisation-mixing kernels (seeded random 2x2 gains and leakage)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world, rank, local = dist_setup()
    cfg = synth.config(args.config)
    if args.time > 0:
        cfg.n_time = args.time
    cfg.input_bits = args.input_bits
    cfg.sub_int = args.sub_int
    if args.pol_mix:
        cfg.jones = synth.make_jones(cfg, seed=cfg.seed)
    if args.impl == "reference":
        run_reference(args, cfg, world, rank)
        return

    import torch
    import paper_2609_03027_gb300 as E
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (sm_103a)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    T = cfg.n_time
    volt = synth.make_voltages(cfg)
    units = cfg.pixel_updates(T)
    d_volt = torch.from_numpy(volt).to(dev)
    sets = (T // cfg.sub_int,) if cfg.sub_int > 0 else ()
    out = torch.empty(sets + (cfg.n_chan, cfg.n_prod, cfg.grid_n, cfg.grid_n), dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    use_graph = not args.no_graph

    def time_path(path, steps, warmup, sample_clocks=False):
        plan = E.Plan.from_config(cfg, path=path, max_time=T)
        if args.params and path == args.path:
            fixed = {k: int(v) for k, v in (kv.split("=") for kv in args.params.split(","))}
            for k, v in fixed.items():
                plan.set_param(k, v)
            tuning = {"params": fixed}
        else:
            tuning = None if args.no_tune else plan.tune(d_volt, out=out, reps=2)
        info = plan.info()
        if tuning is not None:
            info["tuning"] = tuning["params"]
        for _ in range(warmup):
            plan.image(d_volt, out=out, graph=use_graph, time_kernels=True)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.start()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        stops = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ktimes = {}
        launches = 0
        for i in range(steps):
            flush.fill_(i & 0xFF)                       # evict the previous step's data from L2
            starts[i].record(stream)
            plan.image(d_volt, out=out, time_kernels=True, graph=use_graph)
            stops[i].record(stream)
            kt = plan.kernel_times()                   # events on the launching stream
            launches += len(kt)
            for name, ms in kt:
                ktimes.setdefault(name, []).append(ms)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        ms = float(np.mean([a.elapsed_time(b) for a, b in zip(starts, stops)]))
        plan_info = dict(info)
        plan.close()
        return ms, ktimes, launches, clocks, plan_info

    ms_local, ktimes, launches, clocks, info = time_path(args.path, args.steps, args.warmup, sample_clocks=True)
    ms = reduce_max(ms_local, world, dev)
    value = units * world / (ms / 1e3)

    # dominant kernel -> roofline
    pk = peaks()
    dom = max(ktimes, key=lambda k: sum(ktimes[k]))
    per_step_launches = len(ktimes[dom]) / args.steps
    bound, algo_step, algo_unit = kernel_model(dom, cfg, T, info)
    if dom.startswith("k_plain"):                   # model is per launch for the chunked plain kernels
        algo_step = algo_step * per_step_launches
    kstep_ms = float(np.sum(ktimes[dom])) / args.steps
    kavg_ms = kstep_ms / per_step_launches
    if bound == "tensor":
        achieved = algo_step / (kstep_ms / 1e3) / 1e12
        peak, unit = pk["bf16_tflops"], "TFLOP/s"
    elif bound == "alu":
        achieved = algo_step / (kstep_ms / 1e3) / 1e12
        peak, unit = 152 * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12, "TFLOP/s"
    else:
        achieved = algo_step / (kstep_ms / 1e3) / 1e9
        peak, unit = pk["hbm_gbs"], "GB/s"
    roof = {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak,
            "traffic": recorded_traffic(dom, args.config, int(round(T / per_step_launches)), cfg, info.get("tuning")),
            "peak_source": pk["source"] if bound != "alu" else "derived: 152 SM x 128 FP32 lanes x 2 x max SM clock",
            "kernel_ms": kavg_ms, "launches_per_step": per_step_launches,
            "kernel_share": sum(ktimes[dom]) / sum(sum(v) for v in ktimes.values())}

    # the plain comparator (and any other path) on the same inputs
    compare = {}
    for cp in [c for c in args.compare.split(",") if c and c not in (args.path, "none")]:
        cms, ck, _, _, _ = time_path(cp, max(3, args.steps // 4), 3)
        cms = reduce_max(cms, world, dev)
        compare[cp] = {"value": units * world / (cms / 1e3), "ms_per_step": cms}

    # end to end through the public host-buffer call: pinned H2D + imaging + D2H each step
    e2e = None
    if args.e2e_steps > 0:
        e2e = run_e2e(E, cfg, volt, out, T, units, world, dev, args, info.get("tuning"))

    serving = None
    if args.serve_seconds > 0 and world == 1:
        try:
            serving = run_serving(E, args, dev)
        except Exception as ex:  # reported, never fatal to the throughput line
            serving = {"error": f"{type(ex).__name__}: {ex}"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg, volt)

    if rank == 0:
        dtype = {"plain": "f32", "fused": "f32", "dftgemm": "f16", "auto": "f16"}[args.path]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                "config": {"workload": WORKLOADS[args.config] + ("" if cfg.input_bits == 4 else ", 8+8-bit input")
                           + (f", image set every {cfg.sub_int} samples" if cfg.sub_int else "")
                           + (", per-element polarisation mixing" if cfg.jones is not None else ""),
                           "path": info.get("path_name", args.path),
                           "global_batch_pixel_updates": units * world, "l2": "flushed between steps (256 MB write)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "launch": "cuda-graph" if use_graph else "per-kernel",
                           "tuning": info.get("tuning")},
                "roofline": roof, "e2e": e2e, "gpu_launches": launches * world, "clocks": clocks,
                "cpu_baseline": cpu, "compare": compare, "serving": serving}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
