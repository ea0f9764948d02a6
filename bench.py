"""Benchmark: medium events/s of the GPU light tracer on the Cornell-box workload.

Workload (one step): the 4-sphere Cornell box, 4 Gaussian dyes on 128^3 fp32 grids, Lambertian
walls, a ceiling light with 4 lines, 512x512 pinhole film x 81 bins, 16 paths per pixel
(4,194,304 photon paths). `value` is whole-job events/s of the forward (wavefront) form with the
scene resident in HBM; `forms` also reports the plain one-thread-per-path kernel on the same
paths (same estimator, same paths, hence equal RMSE). `e2e` runs the same step through the C ABI
from pinned host buffers: grid upload, flr_set_medium, flr_render and the film read-back.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank traces its own path-id range (weak scaling, no collective on the data
path); timing is the max over ranks. --impl reference times the CPU oracle (fp64, the machine's host
cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenegen as sg  # noqa: E402

METRIC = "medium events/s (fwd, batched, adjoint) vs plain GPU kernel at equal RMSE"
WORKLOAD = "cornell box: 4 dye spheres, 128^3 x4 fp32 grids, 512x512 pinhole x 81 bins, 16 spp"

# Algorithmic work per unit, as the hot-path scope table counts it (32-bit lane operations):
#   tracking step       one uniform (a quarter of a Philox4x32-10 block, about 15 integer
#                       operations), one MUFU logarithm and about 10 FP32 operations      -> 26
#   real event (extra)  three uniforms, sincos and a square root, about 30 FP32           -> 78
#   sensor connection   projection into the film and visibility                           -> 45
#   ratio-tracking step as a tracking step                                                -> 26
# Empty-space leaps and local-majorant cell visits are optimisations of the kernels, not work the
# method asks for, so they are not counted. MUFU (special-function unit) operations per unit:
# a logarithm per tracking or ratio-tracking step, sincos and a square root per event, a
# reciprocal square root and a reciprocal per pinhole connection.
OPS_STEP = 26
OPS_EVENT = 78
OPS_CONNECT = 45
OPS_CONNECT_STEP = 26
MUFU_STEP, MUFU_EVENT, MUFU_CONNECT, MUFU_CONNECT_STEP = 1, 3, 2, 1

# The kernels' random-number contract (one Philox4x32-10 block per (path, step, slot), so that any
# decision can be replayed from its counter alone) draws whole blocks: a block is 112 lane
# operations (10 rounds of 2 mul.lo + 2 mul.hi + 4 xor + 2 key adds, plus 4 x 3 for the uniforms).
# Counted that way a tracking step is a block + 55, a real event a second block + 30, a
# ratio-tracking step a quarter block + 36: reported beside the headline as `rng_contract`.
OPS_PHILOX = 112
RNG_OPS = {"steps": OPS_PHILOX + 55, "events": OPS_PHILOX + 30, "connections": 45,
           "connect_steps": OPS_PHILOX // 4 + 36}


def algorithmic_ops(c):
    return (c["steps"] * OPS_STEP + c["events"] * OPS_EVENT + c["connections"] * OPS_CONNECT
            + c["connect_steps"] * OPS_CONNECT_STEP)


def mufu_ops(c):
    return (c["steps"] * MUFU_STEP + c["events"] * MUFU_EVENT + c["connections"] * MUFU_CONNECT
            + c["connect_steps"] * MUFU_CONNECT_STEP)


def rng_contract_ops(c):
    return sum(c[k] * v for k, v in RNG_OPS.items())


# A render with a film launches the trace kernel and the fold of its fixed-point film sums.
FILM_RENDER_LAUNCHES = 2


def count_launches(steps, plain_renders, batched, adjoint, paper, paper_steps, sheet, cube, hero,
                   adjoint_steps):
    """The library's kernel launches inside the timed regions: the Cornell box's timed and
    kernel-only steps and its plain renders (a film each), the batch (no film: one launch per
    graph replay, one per medium for the plain baseline), the adjoint's passes (no film), the
    paper model's camera and light renders, the light sheet's and the cube's timed renders and
    their plain baselines, and the hero forms' renders."""
    n = FILM_RENDER_LAUNCHES * (2 * steps + plain_renders)
    if batched is not None:
        n += batched["steps"] + batched["plain_launches"]
    if adjoint is not None:
        n += adjoint["launches_per_step"] * adjoint_steps
    if paper is not None:
        n += 2 * paper["launches_per_step"] * paper_steps
    for w in (sheet, cube):
        if w is not None:
            n += w["launches_per_step"] * (w["steps"] + 1)
    if hero is not None:
        n += hero["launches"]
    return n


def rooflines(c, seconds, sms, sm_mhz):
    """ALU roofline of one launch from its counters (headline), its MUFU ceiling and the ALU
    figure under the random-number contract's counts. peak ALU = SMs x 128 lanes x clock; peak
    MUFU = SMs x 16 x clock."""
    f = sm_mhz * 1e6
    alu_peak = sms * 128 * f
    mufu_peak = sms * 16 * f
    a = algorithmic_ops(c) / seconds
    m = mufu_ops(c) / seconds
    r = rng_contract_ops(c) / seconds
    note = f"peak = {sms} SMs x 128 lanes x {sm_mhz:.0f} MHz (maximum SM clock)"
    src = peak_source("sm_max_mhz")
    return ({"bound": "alu", "achieved": a / 1e12, "peak": alu_peak / 1e12, "unit": "Tops/s",
             "frac": a / alu_peak, "note": note, "peak_source": src},
            {"bound": "mufu", "achieved": m / 1e12, "peak": mufu_peak / 1e12, "unit": "Tops/s",
             "frac": m / mufu_peak, "ceiling_ms": 1000.0 * mufu_ops(c) / mufu_peak,
             "note": f"peak = {sms} SMs x 16 x {sm_mhz:.0f} MHz", "peak_source": src},
            {"bound": "alu", "achieved": r / 1e12, "peak": alu_peak / 1e12, "unit": "Tops/s",
             "frac": r / alu_peak, "note": "per-unit counts of the random-number contract",
             "peak_source": src})


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def start_clock_sampler(gpu_index, path):
    cmd = ["nvidia-smi", f"--id={gpu_index}",
           "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        f = open(path, "w")
        return subprocess.Popen(cmd, stdout=f, stderr=subprocess.DEVNULL), f
    except (OSError, FileNotFoundError):
        return None, None


def stop_clock_sampler(proc, f, path):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    f.close()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def peak_source(key):
    """Where a roofline denominator comes from: the per-pod measurement, else the fallback."""
    if key in measured_peaks():
        return f"of measured ({key} in MEASURED_PEAKS.json)"
    return {"hbm_gbs": "of fallback (6.8 TB/s, an earlier GB300 copy measurement)",
            "sm_max_mhz": "of fallback (2070 MHz, the GB300's maximum SM clock)"}.get(key, "of fallback")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def kernel_traffic(name):
    """DRAM bytes per launch from a committed ncu summary, or None once the kernel source has
    changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            info = json.load(f)
        h = hashlib.sha256()
        for src in info["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        sha = h.hexdigest()
    except (OSError, ValueError, KeyError):
        return None
    return info.get("bytes_per_launch") if sha == info.get("sources_sha256") else None


def kernel_profile(name):
    """Utilisation figures of a kernel from a committed ncu summary (issue slots, FP32 pipe, threads
    per warp instruction, L2 hit rate, L2 reduction requests), or None once the kernel source has
    changed since they were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            info = json.load(f)
        h = hashlib.sha256()
        for src in info["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
    except (OSError, ValueError, KeyError):
        return None
    return info.get("metrics") if h.hexdigest() == info.get("sources_sha256") else None


def cpu_oracle_rate(sc, n_paths, n_threads=0, film=True, medium_id=0):
    import oracle
    t = time.perf_counter()
    r = oracle.render(sc, n_paths=n_paths, n_threads=n_threads, film=film, medium_id=medium_id)
    dt = time.perf_counter() - t
    c = r["counters"]
    return {"events": c["events"], "paths": c["paths"], "seconds": dt}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    sc = sg.cfg2_cornell_box()
    n_sample = args.ref_paths
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        cpu_oracle_rate(sc, max(n_sample // 8, 1024))
    ev, sec = 0, 0.0
    for _ in range(args.steps):
        r = cpu_oracle_rate(sc, n_sample)
        ev += r["events"]
        sec += r["seconds"]
    value = ev / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "paths_per_step": n_sample,
                   "note": "CPU oracle on a bounded sample of the same scene"},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n_sample} paths of the Cornell-box workload per step"},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_rates(fn, sample, single_fraction=16):
    """The oracle on the machine's host cores (all of them, then one) on a bounded sample:
    fn(scale, n_threads) -> (events, paths) runs the sample (scale 1) or a 1/single_fraction
    slice of it (scale 1/single_fraction)."""
    out = {}
    for name, scale, threads in (("all_cores", 1.0, 0), ("single_core", 1.0 / single_fraction, 1)):
        t = time.perf_counter()
        ev, paths = fn(scale, threads)
        dt = time.perf_counter() - t
        out[name] = {"events_per_s": ev / dt, "paths_per_s": paths / dt, "seconds": dt,
                     "paths": paths}
    return {"value": out["all_cores"]["events_per_s"], "unit": "events/s",
            "cores": os.cpu_count() or 1, "kind": "oracle", "sample": sample,
            "paths_per_s": out["all_cores"]["paths_per_s"], "seconds": out["all_cores"]["seconds"],
            "single_core": {"value": out["single_core"]["events_per_s"], "unit": "events/s",
                            "paths": out["single_core"]["paths"],
                            "seconds": out["single_core"]["seconds"]}}


def bench_batched(args, local, rank, flush, stream, barrier, reduce_max, reduce_sum):
    """256 independent media (grid edges 16-128, 1-3 dyes, albedo 0.5-0.999, 1e4-1e6 paths each):
    one persistent launch replayed from a CUDA graph, its block size and resident blocks per SM
    chosen by the autotuner, against the plain single-scene kernel run medium by medium on the
    same paths (same estimator and paths: equal RMSE)."""
    import torch
    from paper_1706_03024_gb300.autotune import tune_batch
    from paper_1706_03024_gb300.scene import Batch, Scene

    media = sg.cfg3_batched_media(n_media=args.batch_media, seed=0)
    tune = None
    block, bps = 0, 0
    if args.autotune:
        res = tune_batch(lambda b, k: Batch(media, device=local, seed=rank, medium_id=0,
                                            block_size=b, blocks_per_sm=k))
        block, bps = res.best.block_size, res.best.regroup
        tune = {"chosen": {"block_size": block, "blocks_per_sm": bps},
                "trials": [{"block_size": c.block_size, "blocks_per_sm": c.regroup,
                            "events_per_s": v} for c, v in res.trials]}
    bt = Batch(media, device=local, seed=rank, medium_id=0, block_size=block, blocks_per_sm=bps)
    for _ in range(max(1, args.warmup - 2)):
        bt.launch()
    torch.cuda.synchronize()
    ms = []
    counters = None
    barrier()
    for i in range(args.batch_steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bt.launch()
        b.record(stream)
        counters = bt.read()["counters"]
        ms.append(a.elapsed_time(b))
    barrier()
    step_ms = reduce_max(sum(ms) / len(ms))
    ev = reduce_sum(float(counters["events"]))
    value = ev / (step_ms / 1000.0)
    # plain kernel, one medium after another (each its own launch), same paths
    plain_ms = 0.0
    plain_events = 0
    scenes = []
    for m, sc in enumerate(media):
        S = Scene(sc, device=local)
        S.render(form="plain", seed=rank, medium_id=m, film=False)  # warm-up
        scenes.append(S)
    torch.cuda.synchronize()
    flush.fill_(0.5)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for m, S in enumerate(scenes):
        S.render(form="plain", seed=rank, medium_id=m, film=False)
    b.record(stream)
    for S in scenes:
        plain_events += S.read()["counters"]["events"]
    torch.cuda.synchronize()
    plain_ms = reduce_max(a.elapsed_time(b))
    plain_value = reduce_sum(float(plain_events)) / (plain_ms / 1000.0)
    for S in scenes:
        S.close()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu, mufu, rng = rooflines(counters, sum(ms) / len(ms) / 1000.0, sms,
                               float(measured_peaks().get("sm_max_mhz", 2070.0)))
    cpu = None
    if rank == 0 and not args.no_cpu:
        sub = media[:16]

        def run(scale, threads):
            ev_, paths = 0, 0
            for m, sc in enumerate(sub):
                n = max(int(int(sc["params"]["n_paths"]) * scale), 64)
                r = cpu_oracle_rate(sc, n, n_threads=threads, film=False, medium_id=m)
                ev_ += r["events"]
                paths += n
            return ev_, paths
        cpu = cpu_rates(run, "the first 16 of the 256 media with their full path counts "
                             "(fp64); one core: 1/16 of each medium's paths")
    n_total = int(bt.n_paths.sum())
    bt.close()
    return {"workload": "256 media, edges 16-128, 1-3 dyes, albedo 0.5-0.999, 1e4-1e6 paths each"
                        f" ({n_total} paths)",
            "autotune": tune, "launch": {"block_size": block, "blocks_per_sm": bps},
            "events_per_s": value, "paths_per_s": reduce_sum(float(n_total)) / (step_ms / 1000.0),
            "ms_per_step": step_ms, "steps": len(ms),
            "ms_steps": [round(v, 3) for v in ms],
            "plain_per_medium_events_per_s": plain_value, "plain_ms": plain_ms,
            "plain_launches": len(media), "speedup_vs_plain": value / plain_value,
            "events_per_step": counters["events"], "counters_per_step": counters,
            "roofline": alu, "roofline_mufu": mufu, "roofline_rng_contract": rng,
            "cpu_baseline": cpu}


def bench_adjoint(args, local, rank, flush, stream, barrier, reduce_max, reduce_sum):
    """Gradient of sum((I - T)^2) over the 256x256x81 film w.r.t. 2 x 64^3 concentrations and
    sigma_s (32 paths per pixel): the forward (warp-regrouped and plain) and the path-replay
    adjoint (two warp-regrouped passes, and the one-thread replay) on the same paths, so every form
    carries the same estimator."""
    import torch
    from paper_1706_03024_gb300.scene import Scene

    sc = sg.cfg4_adjoint(field_seed=0, seed=rank)
    if args.adjoint_paths:
        sc["params"]["n_paths"] = int(args.adjoint_paths)
    n = sc["params"]["n_paths"]
    tgt_sc = sg.cfg4_adjoint(field_seed=1, seed=1000 + rank)
    tgt_sc["params"]["n_paths"] = min(8 * n, 1 << 24)
    T = Scene(tgt_sc, device=local).render(form="wavefront_warp").clone()
    S = Scene(sc, device=local)
    gc = torch.zeros(S.conc_t.shape, dtype=torch.float32, device=torch.device("cuda", local))
    gs = torch.zeros(1, dtype=torch.float32, device=gc.device)
    mc = args.macro_cell
    mg = 0.1  # the score estimator needs sigma_bar > sigma_t: forward and replay share the margin
    film = S.render(form="wavefront_warp", macro_cell=mc, majorant_margin=mg)
    adj = (2.0 * (film - T)).contiguous()
    S.adjoint(adj, gc, gs, macro_cell=mc, majorant_margin=mg)
    torch.cuda.synchronize()

    def timed(fn, steps):
        ms = []
        for i in range(steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return reduce_max(sum(ms) / len(ms)), ms

    barrier()
    fwd_ms, _ = timed(lambda: S.render(form="wavefront_warp", macro_cell=mc, majorant_margin=mg),
                      args.adjoint_steps)
    events = S.read()["counters"]["events"]
    plain_ms, _ = timed(lambda: S.render(form="plain", majorant_margin=mg), args.adjoint_steps)
    adj_ms, adj_steps = timed(lambda: S.adjoint(adj, gc, gs, macro_cell=mc, majorant_margin=mg),
                              args.adjoint_steps)
    adj_plain_ms, _ = timed(lambda: S.adjoint(adj, gc, gs, macro_cell=mc, majorant_margin=mg,
                                              form="plain"), args.adjoint_steps)
    ev = reduce_sum(float(events))
    chunks = -(-n // (1 << 21))   # the replay runs its two passes per chunk of 2^21 paths
    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle
        adj_h = adj.double().cpu().numpy()
        n1 = 256 * 256   # one path per pixel

        def run(scale, threads):
            m = max(int(n1 * scale), 256)
            r = oracle.render(sc, n_paths=m, n_threads=threads, majorant_scale=1.0 + mg)
            oracle.adjoint(sc, adj_h, n_paths=m, n_threads=threads, majorant_scale=1.0 + mg)
            return r["counters"]["events"], m
        cpu = cpu_rates(run, "65,536 paths (1 per pixel) of the same scene, forward render and "
                             "path-replay adjoint (fp64; events of the forward over the time of both)")
    return {"workload": f"2 x 64^3 blob dyes, 256x256x81 ortho film, {n} paths, loss sum((I-T)^2)",
            "macro_cell": mc,
            "adjoint_events_per_s": ev / (adj_ms / 1000.0), "adjoint_ms": adj_ms,
            "adjoint_ms_steps": [round(v, 3) for v in adj_steps],
            "adjoint_plain_replay_ms": adj_plain_ms,
            "adjoint_speedup_vs_plain_replay": adj_plain_ms / adj_ms,
            "forward_warp_events_per_s": ev / (fwd_ms / 1000.0), "forward_warp_ms": fwd_ms,
            "plain_events_per_s": ev / (plain_ms / 1000.0), "plain_ms": plain_ms,
            "adjoint_over_forward": adj_ms / fwd_ms, "events_per_step": events,
            "launches_per_step": 3 + 2 * chunks,
            "grad_sigma_s": float(gs.item()), "grad_conc_abs_max": float(gc.abs().max().item()),
            "cpu_baseline": cpu}


def bench_paper(args, local, rank, flush, stream, barrier, reduce_max, reduce_sum):
    """The paper's single-inelastic model (Sec. 4.1-4.3) on a 64^3 x 2 blobby-dye scene with a
    256x256 pinhole film: its own camera-side estimator (flr_render_camera, 16 paths per pixel)
    against the light tracer in paper mode (4,194,304 paths, warp-regrouped), both timed, and each
    film's RMSE against a reference averaged from both estimators at 16x the paths, so that the
    comparison is at equal RMSE: efficiency = 1 / (RMSE^2 x time)."""
    import torch
    from paper_1706_03024_gb300.scene import Scene

    sc = sg.paper_mode_scene(n=64, width=256, seed=7)
    S = Scene(sc, device=local)
    n_cam = 256 * 256 * 16
    n_light = 4_194_304
    off = rank * (1 << 32)

    def cam(seed=None, k=0):
        return S.render_camera(n_paths=n_cam, path_offset=off + k * n_cam, seed=seed)

    def light(seed=None, k=0):
        return S.render(n_paths=n_light, path_offset=off + k * n_light, form="wavefront_warp",
                        paper_mode=True, seed=seed)

    ref = torch.zeros_like(S.film_tensor(), dtype=torch.float64)
    for k in range(8):
        ref += cam(seed=4242, k=k + 1).double() / 16
        ref += light(seed=4243, k=k + 1).double() / 16
    cam()
    light()
    torch.cuda.synchronize()

    def timed(fn, steps):
        ms = []
        for i in range(steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return reduce_max(sum(ms) / len(ms))

    barrier()
    cam_ms = timed(cam, args.paper_steps)
    cam_counters = S.read()["counters"]
    cam_rmse = float(torch.sqrt(torch.mean((cam().double() - ref) ** 2)))
    light_ms = timed(light, args.paper_steps)
    light_counters = S.read()["counters"]
    light_rmse = float(torch.sqrt(torch.mean((light().double() - ref) ** 2)))
    eff_cam = 1.0 / (cam_rmse ** 2 * cam_ms)
    eff_light = 1.0 / (light_rmse ** 2 * light_ms)
    return {"workload": "2 x 64^3 blob dyes in a scattering solvent, collimated beam, 256x256 pinhole "
                        "film, the paper's single-inelastic model",
            "camera": {"paths": n_cam, "ms": cam_ms,
                       "events_per_s": reduce_sum(float(cam_counters["events"])) / (cam_ms / 1000.0),
                       "rmse": cam_rmse},
            "light_paper_mode": {"paths": n_light, "ms": light_ms,
                                 "events_per_s": reduce_sum(float(light_counters["events"])) / (light_ms / 1000.0),
                                 "rmse": light_rmse},
            "camera_over_light_at_equal_rmse": eff_cam / eff_light,
            "reference": "mean of 8 camera (16 spp) and 8 light-tracer (4.2M paths) films, other seeds",
            "launches_per_step": FILM_RENDER_LAUNCHES}


def bench_sheet(args, local, rank, flush, stream, barrier, reduce_max, reduce_sum):
    """The light-sheet workload at full size: 256^3 x 4 blob dyes (268 MB of grids, larger than
    the L2), albedo 0.999, a 0.05 cm sheet at 488 nm entering the -x face, 1024x1024x81 ortho film
    (340 MB) viewing it from +z, 64 paths per pixel (67,108,864 paths). The warp-regrouped form in
    the bench's launch shape, against the plain kernel on the first eighth of the same path ids
    (same estimator: events/s compares at equal RMSE). Rooflines: ALU from the counters, and HBM
    on the grid gathers (16 bytes, one float4 of 4 dyes, per tracking and ratio-tracking step)."""
    import torch
    from paper_1706_03024_gb300.scene import Scene

    from paper_1706_03024_gb300 import shard
    sc = sg.cfg5_light_sheet()
    n = int(args.sheet_paths) if args.sheet_paths else sc["params"]["n_paths"]
    off, _ = shard.path_range(n, rank)
    S = Scene(sc, device=local)
    kw = {"form": "wavefront_warp", "block_size": 128, "regroup": 1, "skip_cell": 0,
          "macro_cell": 0}
    n_plain = max(n // 8, 1)
    S.render(n_paths=n, path_offset=off, **kw)                     # warm-up
    S.render(n_paths=n_plain, path_offset=off, form="plain")
    torch.cuda.synchronize()

    def timed(fn, steps):
        ms, counters = [], None
        for i in range(steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            counters = S.read()["counters"]
            ms.append(a.elapsed_time(b))
        return ms, counters

    barrier()
    ms, c = timed(lambda: S.render(n_paths=n, path_offset=off, **kw), args.sheet_steps)
    ms_p, c_p = timed(lambda: S.render(n_paths=n_plain, path_offset=off, form="plain"), 1)
    step_ms = reduce_max(sum(ms) / len(ms))
    plain_ms = reduce_max(ms_p[0])
    value = reduce_sum(float(c["events"])) / (step_ms / 1000.0)
    plain_value = reduce_sum(float(c_p["events"])) / (plain_ms / 1000.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    t = sum(ms) / len(ms) / 1000.0
    alu, mufu, rng = rooflines(c, t, sms, float(peaks.get("sm_max_mhz", 2070.0)))
    gathers = c["steps"] + c["connect_steps"]
    D = int(sc["dyes"]["abs_shape"].shape[0])
    # the film's L2 reduction requests: ncu's per-path count on the 2M-path capture, scaled
    prof = kernel_profile("trace_wavefront_warp_sheet_ncu.json")
    film_atomics = None
    if prof and prof.get("film_red_requests_per_path"):
        reqs = prof["film_red_requests_per_path"] * n
        film_atomics = {"requests_per_step": reqs, "per_s": reqs / t,
                        "source": "ncu L2 reduction requests per path on the 2M-path capture, "
                                  "scaled to the step's paths"}
    alg_bytes = 4 * D * gathers
    cpu = None
    if rank == 0 and not args.no_cpu:
        n_cpu = args.sheet_cpu_paths

        def run(scale, threads):
            m = max(int(n_cpu * scale), 256)
            r = cpu_oracle_rate(sc, m, n_threads=threads, film=True)
            return r["events"], m
        cpu = cpu_rates(run, f"{n_cpu} paths (1/{n // n_cpu} of the workload's) of the same scene "
                             "with the film (fp64)")
    return {"workload": "light sheet: 256^3 x 4 blob dyes, albedo 0.999, 0.05 cm sheet at 488 nm, "
                        f"1024x1024x81 ortho film, {n} paths",
            "launch": kw, "events_per_s": value, "paths_per_s": reduce_sum(float(n)) / (step_ms / 1000.0),
            "ms_per_step": step_ms, "steps": len(ms), "ms_steps": [round(v, 3) for v in ms],
            "plain_events_per_s": plain_value, "plain_ms": plain_ms, "plain_paths": n_plain,
            "speedup_vs_plain": value / plain_value,
            "per_path": {k: c[k] / n for k in ("events", "steps", "connections", "connect_steps")},
            "roofline_alu": alu, "roofline_mufu": mufu, "roofline_rng_contract": rng,
            "cpu_baseline": cpu,
            "roofline_hbm_gathers": {"bound": "hbm", "achieved": alg_bytes / t / 1e9, "peak": hbm,
                                     "unit": "GB/s", "frac": alg_bytes / t / 1e9 / hbm,
                                     "sector_frac": 8 * alg_bytes / D / t / 1e9 / hbm,
                                     "peak_source": peak_source("hbm_gbs"),
                                     "bytes_per_gather": 4 * D,
                                     "traffic": kernel_traffic(
                                         "trace_wavefront_warp_sheet_traffic.json")},
            "ncu": prof,
            "film_atomics": film_atomics,
            "launches_per_step": FILM_RENDER_LAUNCHES}


def bench_cube(args, local, rank, flush, stream, barrier, reduce_max, reduce_sum):
    """The homogeneous cube (1 cm, sigma_s 20, one dye, QY 0.9, pencil beam at 490 nm, 64x64x81
    ortho film) at 1e8 paths: no grid, so tracking and connections are arithmetic alone (closed-form
    transmittance) and the ALU roofline bounds it. The warp-regrouped form against the plain kernel
    on the first eighth of the same path ids (same estimator: equal RMSE); the oracle on 1e7 paths
    of the same cube (the 1e5-path parity case takes it 0.1 s, too short to time)."""
    import torch
    from paper_1706_03024_gb300 import shard
    from paper_1706_03024_gb300.scene import Scene

    n = int(args.cube_paths)
    sc = sg.cfg1_homogeneous_cube(n_paths=n)
    off, _ = shard.path_range(n, rank)
    S = Scene(sc, device=local)
    kw = {"form": "wavefront_warp", "block_size": 128, "regroup": 1}
    n_plain = max(n // 8, 1)
    S.render(n_paths=n, path_offset=off, **kw)                     # warm-up
    S.render(n_paths=n_plain, path_offset=off, form="plain")
    torch.cuda.synchronize()

    def timed(fn, steps):
        ms, counters = [], None
        for i in range(steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            counters = S.read()["counters"]
            ms.append(a.elapsed_time(b))
        return ms, counters

    barrier()
    ms, c = timed(lambda: S.render(n_paths=n, path_offset=off, **kw), args.cube_steps)
    ms_p, c_p = timed(lambda: S.render(n_paths=n_plain, path_offset=off, form="plain"), 1)
    S.close()
    step_ms = reduce_max(sum(ms) / len(ms))
    plain_ms = reduce_max(ms_p[0])
    value = reduce_sum(float(c["events"])) / (step_ms / 1000.0)
    plain_value = reduce_sum(float(c_p["events"])) / (plain_ms / 1000.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu, mufu, rng = rooflines(c, sum(ms) / len(ms) / 1000.0, sms,
                               float(measured_peaks().get("sm_max_mhz", 2070.0)))
    cpu = None
    if rank == 0 and not args.no_cpu:
        small = sg.cfg1_homogeneous_cube()
        n_cpu = int(args.cube_cpu_paths)

        def run(scale, threads):
            m = max(int(n_cpu * scale), 256)
            r = cpu_oracle_rate(small, m, n_threads=threads, film=True)
            return r["events"], m
        cpu = cpu_rates(run, f"{n_cpu} paths of the same cube with the film (fp64)")
    return {"workload": f"homogeneous cube: sigma_s 20, one dye, pencil beam, 64x64x81 ortho film, {n} paths",
            "launch": kw, "events_per_s": value, "paths_per_s": reduce_sum(float(n)) / (step_ms / 1000.0),
            "ms_per_step": step_ms, "steps": len(ms), "ms_steps": [round(v, 3) for v in ms],
            "plain_events_per_s": plain_value, "plain_ms": plain_ms, "plain_paths": n_plain,
            "speedup_vs_plain": value / plain_value,
            "per_path": {k: c[k] / n for k in ("events", "steps", "connections", "connect_steps")},
            "roofline_alu": alu, "roofline_mufu": mufu, "roofline_rng_contract": rng,
            "cpu_baseline": cpu, "launches_per_step": FILM_RENDER_LAUNCHES}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1706_03024_gb300 import build as B
    from paper_1706_03024_gb300 import native as N
    from paper_1706_03024_gb300.scene import Scene

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    B.build()
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    sc = sg.cfg2_cornell_box()
    if args.paths:
        sc["params"]["n_paths"] = int(args.paths)
    n_paths = sc["params"]["n_paths"]
    S = Scene(sc, device=local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    from paper_1706_03024_gb300 import shard
    offset, _ = shard.path_range(n_paths, rank)   # each rank its own path-id range

    # launch configuration of the optimised form: autotuned on half of the paths (outside
    # the timed region), or taken from the command line
    tuned = {"form": args.form, "block_size": 0, "regroup": args.regroup,
             "skip_cell": args.skip_cell, "macro_cell": args.macro_cell}
    tune_info = None
    if args.autotune:
        from paper_1706_03024_gb300.autotune import tune_render
        res = tune_render(S, max(n_paths // 2, 1 << 16), path_offset=offset, repeats=3)
        tuned = res.best.kwargs()
        tune_info = {"chosen": tuned, "candidates": len({c for c, _ in res.trials}),
                     "best_events_per_s_on_slice": max(v for _, v in res.trials)}

    def one_step(form):
        # the plain kernel is the baseline: one thread per path, one majorant per bin; with the
        # tuned form's empty-space leaps or local majorants it separates their share of the
        # speed-up from the regrouping's
        if form == "plain":
            S.render(form="plain", path_offset=offset)
        elif form == "plain_leaps":
            S.render(form="plain", path_offset=offset, skip_cell=tuned["skip_cell"],
                     macro_cell=tuned["macro_cell"])
        else:
            S.render(path_offset=offset, **tuned)

    def timed(form, steps, sampler_path=None):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        events = 0
        counters = None
        proc = f = None
        if sampler_path:
            # nvidia-smi's own start-up must not overlap the timed steps
            proc, f = start_clock_sampler(local, sampler_path)
            one_step(form)
            torch.cuda.synchronize()
            time.sleep(1.0)
        barrier()
        torch.cuda.synchronize()
        for i in range(steps):
            flush.fill_(float(i))          # evict the scene and film from L2 between steps
            evs[i][0].record(stream)
            one_step(form)
            evs[i][1].record(stream)
            r = S.read() if i == steps - 1 else None
            if r is not None:
                counters = r["counters"]
        torch.cuda.synchronize()
        barrier()
        clocks = stop_clock_sampler(proc, f, sampler_path) if sampler_path else None
        ms = [a.elapsed_time(b) for a, b in evs]
        events = counters["events"]
        return ms, events, counters, clocks

    for _ in range(args.warmup):
        one_step("wavefront")
        one_step("plain")
    torch.cuda.synchronize()

    clock_dir = tempfile.mkdtemp(prefix="fluoro_clocks_")
    ms_w, ev_w, cnt_w, clocks = timed("wavefront", args.steps,
                                      os.path.join(clock_dir, f"clocks_rank{rank}.csv"))
    ms_p, ev_p, cnt_p, _ = timed("plain", max(1, min(args.steps, args.plain_steps)))
    one_step("plain_leaps")
    ms_pl, ev_pl, _, _ = timed("plain_leaps", max(1, min(args.steps, args.plain_steps)))
    step_ms_w_local = sum(ms_w) / len(ms_w)

    # equal-RMSE check: each form's one-step film against a 16x-path reference (independent seed)
    rmse = None
    if not args.no_rmse:
        ref = torch.zeros_like(S.film_tensor())
        n_ref = 16
        for k in range(n_ref):
            S.render(seed=7777, path_offset=k * n_paths, **tuned)
            ref += S.film_tensor() / n_ref
        out = {}
        for form in ("plain", "wavefront"):
            one_step(form)
            f = S.film_tensor()
            out[form] = float(torch.sqrt(torch.mean((f.double() - ref.double()) ** 2)))
        rmse = {"plain": out["plain"], "wavefront": out["wavefront"],
                "reference_paths": n_ref * n_paths,
                "ratio_wavefront_over_plain": out["wavefront"] / out["plain"]}

    # hero-wavelength paths (four wavelengths per path, spectral MIS) against one wavelength per
    # path: the warp-regrouped form against the timed warp form above, and the plain forms with
    # the same empty-space leaps; time per step and film RMSE against the reference above,
    # efficiency = 1 / (RMSE^2 x time)
    hero = None
    if rmse is not None and not args.no_hero and tuned["macro_cell"] == 0:
        sk = tuned["skip_cell"]
        warp_kw = {"form": "wavefront_warp", "block_size": 128, "regroup": 1}
        hero_ms, hero_rmse = {}, {}
        for name, kw in (("warp_hero4", dict(warp_kw, hero=4)), ("plain_single", {"form": "plain"}),
                         ("plain_hero4", {"form": "plain", "hero": 4})):
            S.render(path_offset=offset, skip_cell=sk, **kw)   # warm-up
            ms_h = []
            for i in range(args.hero_steps):
                flush.fill_(float(i))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                S.render(path_offset=offset, skip_cell=sk, **kw)
                b.record(stream)
                torch.cuda.synchronize()
                ms_h.append(a.elapsed_time(b))
            hero_ms[name] = sum(ms_h) / len(ms_h)
            hero_rmse[name] = float(torch.sqrt(torch.mean((S.film_tensor().double() - ref.double()) ** 2)))
            if name == "warp_hero4":
                hero_events = S.read()["counters"]["events"]
        hero_ms["warp_single"], hero_rmse["warp_single"] = step_ms_w_local, rmse["wavefront"]
        eff = {k: 1.0 / (hero_rmse[k] ** 2 * hero_ms[k]) for k in hero_ms}
        hero = {"members": 4, "skip_cell": sk, "ms": hero_ms, "rmse": hero_rmse,
                "warp_hero4_events_per_s": hero_events / (hero_ms["warp_hero4"] / 1000.0),
                "efficiency_warp_hero4_over_warp_single": eff["warp_hero4"] / eff["warp_single"],
                "efficiency_plain_hero4_over_plain_single": eff["plain_hero4"] / eff["plain_single"],
                "equal_rmse_time_ms": {"warp_single": hero_ms["warp_single"],
                                       "warp_hero4": hero_ms["warp_hero4"] * (hero_rmse["warp_hero4"] / hero_rmse["warp_single"]) ** 2},
                "launches": 3 * args.hero_steps * FILM_RENDER_LAUNCHES}

    def reduce_max(x):
        return shard.reduce_scalar(x, "max", device=dev)

    def reduce_sum(x):
        return shard.reduce_scalar(x, "sum", device=dev)

    step_ms_w = reduce_max(sum(ms_w) / len(ms_w))
    step_ms_p = reduce_max(sum(ms_p) / len(ms_p))
    total_ev_w = reduce_sum(float(ev_w))
    total_ev_p = reduce_sum(float(ev_p))
    value = total_ev_w / (step_ms_w / 1000.0)
    plain_value = total_ev_p / (step_ms_p / 1000.0)
    step_ms_pl = reduce_max(sum(ms_pl) / len(ms_pl))
    plain_leaps_value = reduce_sum(float(ev_pl)) / (step_ms_pl / 1000.0)
    paths_per_s = reduce_sum(float(n_paths)) / (step_ms_w / 1000.0)

    # --- batched persistent form: 256 media in one launch (CUDA graph) ----------------------
    batched = None
    if not args.no_batch:
        batched = bench_batched(args, local, rank, flush, stream, barrier, reduce_max, reduce_sum)

    # --- adjoint (path replay) -------------------------------------------------------------
    paper = None
    if not args.no_paper:
        paper = bench_paper(args, local, rank, flush, stream, barrier, reduce_max, reduce_sum)
    sheet = None
    if not args.no_sheet:
        sheet = bench_sheet(args, local, rank, flush, stream, barrier, reduce_max, reduce_sum)
    cube = None
    if not args.no_cube:
        cube = bench_cube(args, local, rank, flush, stream, barrier, reduce_max, reduce_sum)
    adjoint = None
    if not args.no_adjoint:
        adjoint = bench_adjoint(args, local, rank, flush, stream, barrier, reduce_max, reduce_sum)

    # --- end to end through the C ABI with host buffers ------------------------------------
    # Every step copies its grids in from pinned host memory, uploads the medium, renders, and
    # copies its film and tallies out. Measured twice: one step after another on one context
    # (serial), and as a stream of scenes: two contexts on two streams alternate, the host issues
    # step k+1 (its copies and upload on its own stream) before it reads step k's results, so one
    # step's film readback and the next step's upload overlap a render. The pipelined rate is the
    # line's e2e.
    md = sc["medium"]
    conc_h = torch.from_numpy(np.ascontiguousarray(md["conc"])).pin_memory()
    solv_h = torch.from_numpy(np.ascontiguousarray(md["solvent"])).pin_memory()
    h2d = conc_h.numel() * 4 + solv_h.numel()
    d2h = S.film_tensor().numel() * 4 + 2 * 6 * S.B * 8
    ctxs = [S, Scene(sc, device=local)]
    streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    bufs = [(torch.empty_like(conc_h, device=dev), torch.empty_like(solv_h, device=dev),
             torch.empty(S.film_tensor().shape, dtype=torch.float32).pin_memory()) for _ in range(2)]

    def e2e_issue(j):
        X, st = ctxs[j], streams[j]
        cd, sd, fh = bufs[j]
        with torch.cuda.stream(st):
            cd.copy_(conc_h, non_blocking=True)
            sd.copy_(solv_h, non_blocking=True)
        X.set_medium(md, grids={"conc": cd, "solvent": sd}, stream=st)
        f = X.render(path_offset=offset, stream=st, **tuned)
        with torch.cuda.stream(st):
            fh.copy_(f, non_blocking=True)

    def e2e_collect(j):
        return ctxs[j].read(stream=streams[j])["counters"]["events"]

    for j in (0, 1):
        e2e_issue(j)
        e2e_collect(j)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    serial_events = 0
    for _ in range(args.e2e_steps):
        e2e_issue(0)
        serial_events += e2e_collect(0)
    torch.cuda.synchronize()
    serial_s = reduce_max((time.perf_counter() - t0) / args.e2e_steps)
    serial_value = reduce_sum(float(serial_events / args.e2e_steps)) / serial_s
    barrier()
    t0 = time.perf_counter()
    e2e_events = 0
    for k in range(args.e2e_steps):
        e2e_issue(k % 2)
        if k > 0:
            e2e_events += e2e_collect((k - 1) % 2)
    e2e_events += e2e_collect((args.e2e_steps - 1) % 2)
    torch.cuda.synchronize()
    e2e_s = reduce_max((time.perf_counter() - t0) / args.e2e_steps)
    e2e_value = reduce_sum(float(e2e_events / args.e2e_steps)) / e2e_s
    ctxs[1].close()
    S.set_medium(md)

    # the trace kernel: the same renders without the tally and film clears (accumulate), timed with
    # CUDA events on the launching stream; the span also holds the film accumulator's clear and the
    # fold of its sums into the film (about 0.07 ms of the Cornell box's 13 ms)
    kevs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        kevs[i][0].record(stream)
        S.render(path_offset=offset, accumulate=True, **tuned)
        kevs[i][1].record(stream)
    torch.cuda.synchronize()
    kernel_ms = reduce_max(sum(a.elapsed_time(b) for a, b in kevs) / args.steps)

    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu, mufu, rng = rooflines(cnt_w, kernel_ms / 1000.0, sms, sm_max)
    alu["kernel_ms"] = kernel_ms
    alu["traffic"] = kernel_traffic("trace_wavefront_warp_cornell_traffic.json")
    prof = kernel_profile("trace_wavefront_warp_cornell_ncu.json")
    film_atomics = None
    if prof and prof.get("film_red_requests_per_path"):
        reqs = prof["film_red_requests_per_path"] * n_paths
        film_atomics = {"requests_per_step": reqs, "per_s": reqs / (kernel_ms / 1000.0),
                        "source": "ncu L2 reduction requests per path on the reduced capture, "
                                  "scaled to the step's paths"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        r = cpu_oracle_rate(sc, args.cpu_paths)
        r1 = cpu_oracle_rate(sc, max(args.cpu_paths // 16, 1024), n_threads=1)
        cpu = {"value": r["events"] / r["seconds"], "unit": "events/s",
               "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"{args.cpu_paths} paths of the same workload (fp64, all host cores), "
                         f"{r['seconds']:.1f} s",
               "single_core": {"value": r1["events"] / r1["seconds"], "unit": "events/s",
                               "sample": f"{r1['paths']} paths on one core, {r1['seconds']:.1f} s"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms_w,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if not args.paths else WORKLOAD + f" ({n_paths} paths)",
                       "paths_per_gpu": n_paths, "launch": tuned, "autotune": tune_info,
                       "l2": "flushed between timed steps (256 MB write)",
                       "events_per_step": ev_w, "parallelism": f"paths sharded over {world} GPU(s)"},
            "paths_per_s": paths_per_s,
            "forms": {
                "wavefront": {"events_per_s": value, "ms_per_step": step_ms_w,
                              "ms_steps": [round(v, 3) for v in ms_w]},
                "plain": {"events_per_s": plain_value, "ms_per_step": step_ms_p,
                          "steps": len(ms_p), "ms_steps": [round(v, 3) for v in ms_p]},
                "plain_leaps": {"events_per_s": plain_leaps_value, "ms_per_step": step_ms_pl,
                                "steps": len(ms_pl), "ms_steps": [round(v, 3) for v in ms_pl],
                                "launch": {"skip_cell": tuned["skip_cell"],
                                           "macro_cell": tuned["macro_cell"]}},
                "speedup_vs_plain": value / plain_value,
                "speedup_from_leaps": plain_leaps_value / plain_value,
                "speedup_from_regrouping": value / plain_leaps_value,
                "equal_rmse": "same estimator and path ids; film RMSE against a 16x-path reference"
                              " in `rmse` (the local majorants of the wavefront form also lower the"
                              " transmittance estimate's variance)",
                "rmse": rmse,
                "batched": batched,
                "adjoint": adjoint,
                "paper_model": paper,
                "light_sheet": sheet,
                "homogeneous_cube": cube,
                "hero_wavelength": hero,
            },
            "counters_per_step": cnt_w,
            "roofline": alu,
            "roofline_mufu": mufu,
            "roofline_rng_contract": rng,
            "ncu": prof,
            "film_atomics": film_atomics,
            "e2e": {"value": e2e_value, "unit": "events/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
                    "how": "two contexts on two streams, step k+1 issued before step k is read",
                    "serial_value": serial_value},
            "gpu_launches": count_launches(args.steps, len(ms_p) + len(ms_pl), batched, adjoint,
                                           paper, args.paper_steps, sheet, cube, hero,
                                           args.adjoint_steps),
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="wavefront_warp",
                    choices=["wavefront", "wavefront_warp", "wavefront_pool"],
                    help="optimised form when not autotuning")
    ap.add_argument("--regroup", type=int, default=1)
    ap.add_argument("--macro-cell", type=int, default=0,
                    help="local-majorant cell edge in voxels for the optimised forms (0: global)")
    ap.add_argument("--skip-cell", type=int, default=2,
                    help="empty-space leap cell edge in voxels for the optimised form (0: off)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="use --regroup/--skip-cell/--macro-cell instead of tuning")
    ap.add_argument("--plain-steps", type=int, default=5)
    ap.add_argument("--paths", type=int, default=0,
                    help="override the path count (small profiling cases only)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-paths", type=int, default=1 << 21)
    ap.add_argument("--ref-paths", type=int, default=1 << 16)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-rmse", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--batch-media", type=int, default=256,
                    help="media in the batched workload (fewer for small profiling cases only)")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-paper", action="store_true",
                    help="skip the paper's own (camera-side) estimator of its single-inelastic model")
    ap.add_argument("--paper-steps", type=int, default=3)
    ap.add_argument("--adjoint-steps", type=int, default=3)
    ap.add_argument("--no-hero", action="store_true",
                    help="skip the hero-wavelength comparison (needs the film RMSE reference)")
    ap.add_argument("--hero-steps", type=int, default=2)
    ap.add_argument("--no-sheet", action="store_true",
                    help="skip the full-size light-sheet workload (256^3 x 4 grids, 67M paths)")
    ap.add_argument("--sheet-steps", type=int, default=2)
    ap.add_argument("--no-cube", action="store_true",
                    help="skip the homogeneous cube at 1e8 paths")
    ap.add_argument("--cube-paths", type=int, default=100_000_000)
    ap.add_argument("--cube-steps", type=int, default=2)
    ap.add_argument("--cube-cpu-paths", type=int, default=10_000_000)
    ap.add_argument("--sheet-cpu-paths", type=int, default=1 << 20,
                    help="light-sheet paths the CPU oracle baseline traces")
    ap.add_argument("--sheet-paths", type=int, default=0,
                    help="override the light-sheet path count (small profiling cases only)")
    ap.add_argument("--adjoint-paths", type=int, default=0,
                    help="override the adjoint path count (small profiling cases only)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
