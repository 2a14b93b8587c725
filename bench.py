"""Benchmark of the black-hole beam tracer on GB300.

A step renders one 1920x1080 frame of the orbiting-camera workload (camera
at r = 6 r_s, theta = 85 deg, moving at 0.5 c along e_phi; thin disc 3-12 r_s;
1M synthetic stars in a 6 x 2048^2 FP16 cube map; 512x512 and 64x32 FP32
tables) through the C ABI.  Tables and cube map are built once, untimed
(their build times are reported separately).  L2 is flushed (a 256 MiB
write) before every timed frame; each frame's render is timed with CUDA
events on the launching stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: replicas only -- every rank renders its own frames, no collective
on the data path; value = frames of all ranks / max over ranks of the time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "1080p frames/s"
WORKLOAD = "orbit_1080p"
# FP32 work per unit, counted from the render kernel source (FMA = 2 flops):
# beam set-up + TRACERAY + footprint + colour lookup + store per pixel, the
# tent-filter inner loop per visited texel, disc shading per hit.
FLOP_PER_PIXEL = 420
FLOP_PER_TEXEL = 26
FLOP_PER_HIT = 60
FP32_LANES_PER_SM = 128


def max_over_ranks(value: float, device, ws: int) -> float:
    """The largest of every rank's value (the slowest replica sets the time)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(steps: int, ws: int, t_max: float) -> float:
    """Frames/s of the whole job: every one of the ws replicas renders `steps`
    frames; the job takes as long as its slowest replica."""
    return ws * steps / t_max


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                mhz.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(mhz)}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return json.loads(p.read_text())
    return None


def render_traffic():
    """DRAM bytes per render launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    f = ROOT / "profiles" / "render_traffic.json"
    if not f.exists():
        return None
    d = json.loads(f.read_text())
    src = (ROOT / "paper_2010_08735_gb300" / "csrc" / "bh_render.cu").read_bytes()
    if d.get("kernel_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return d.get("dram_bytes_per_launch")


def workload_config(wk, ws=1):
    W, H = wk["camera"]["width"], wk["camera"]["height"]
    return {"workload": WORKLOAD, "width": W, "height": H, "camera": "r=6, theta=85deg, v=0.5c e_phi",
            "stars": wk["n_stars"], "cube_face": wk["cube_n"], "cube_dtype": wk["cube_dtype"],
            "tables": "512x512 D + 64x32 U, FP32", "l2": "flushed (256 MiB write) before each frame",
            "parallelism": f"replicas x{ws}"}


def orbit_camera(wk, step):
    cam = dict(wk["camera"])
    cam["phi"] = cam["phi"] + 0.002 * step  # the camera moves along its orbit between frames
    return cam


def cpu_baseline(wk, seconds=12.0, impl_line=False):
    """The oracle, as it stands, on the host cores: full-resolution rows of the
    same workload until about `seconds` of rendering, scaled to frames/s."""
    import oracle
    from paper_2010_08735_gb300 import synth
    t0 = time.perf_counter()
    D, U = oracle.tables_exact(512, 64, 32, 1e-3)
    Ct, dl = oracle.colour_table(), oracle.disc_colour_table()
    st = synth.stars(wk["n_stars"], wk["star_seed"])
    rec = oracle.build_cubemap(st, wk["cube_n"], 1 if wk["cube_dtype"] == "f16" else 2)
    scene = oracle.SceneTables(D.astype(np.float32), U.astype(np.float32), Ct.astype(np.float32),
                               dl.astype(np.float32), rec, wk["cube_n"],
                               1 if wk["cube_dtype"] == "f16" else 2)
    setup = time.perf_counter() - t0
    cam = wk["camera"]
    H = cam["height"]
    cores = os.cpu_count() or 1
    rows, tr = 0, 0.0
    band = 40
    y = (H // 2 - 200) // 2 * 2
    while tr < seconds and rows < H:
        y0 = y % H
        y0 -= y0 % 2
        y1 = min(y0 + band, H, y0 + (H - rows))
        t = time.perf_counter()
        oracle.render(cam, wk["disc"], scene, exposure_stars=0.01, y0=y0, y1=y1, nthreads=cores)
        tr += time.perf_counter() - t
        rows += y1 - y0
        y += band
    fps = (rows / H) / tr
    # one core: a 16-row band through the frame's centre
    y0 = (H // 2 - 8) // 2 * 2
    t = time.perf_counter()
    oracle.render(cam, wk["disc"], scene, exposure_stars=0.01, y0=y0, y1=y0 + 16, nthreads=1)
    fps1 = (16 / H) / (time.perf_counter() - t)
    return {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "one_core_value": fps1,
            "sample": f"{rows} of {H} rows of the 1920x1080 frame ({rows * cam['width']} px), "
                      f"FP64 C oracle with {cores} threads (one_core_value: 16 central rows on one thread); "
                      f"oracle set-up {setup:.1f} s untimed"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2010_08735_gb300 import synth
    wk = synth.WORKLOADS[WORKLOAD]
    cb = cpu_baseline(wk, seconds=max(5.0, 2.0 * args.steps), impl_line=True)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "frames/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / cb["value"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wk, args.gpus),
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2010_08735_gb300 import bh, synth

    wk = synth.WORKLOADS[WORKLOAD]
    cam0 = wk["camera"]
    W, H = cam0["width"], cam0["height"]
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    ctx = bh.bh_create(local, 0)
    sh = bh.make_shading(1.0, 0.01)
    disc = wk["disc"]
    # --- build (untimed for the frame metric; reported)
    t_ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with torch.cuda.stream(stream):
        t_ev[0].record(stream)
        tables = bh.bh_precompute_tables(ctx, 512, 64, 32, bh.BH_F32, stream)
        t_ev[1].record(stream)
        stars = torch.from_numpy(synth.stars(wk["n_stars"], wk["star_seed"])).to(dev)
        t_ev[2].record(stream)
        cube = bh.bh_build_star_cubemap(ctx, stars, wk["cube_n"],
                                        bh.BH_F16 if wk["cube_dtype"] == "f16" else bh.BH_BF16, stream)
        t_ev[3].record(stream)
    stream.synchronize()
    precompute_ms = t_ev[0].elapsed_time(t_ev[1])
    cubemap_ms = t_ev[2].elapsed_time(t_ev[3])

    out = torch.empty((H, W, 4), device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    # launch shape for this frame size from the autotuner (untimed)
    tuned = bh.bh_autotune_batch(ctx, tables, cube, [cam0], disc, sh, [out])
    # --- work counts for the roofline (one untimed debug render)
    dbg = torch.empty((H, W, bh.NDBG), device=dev)
    bh.bh_render_debug(ctx, tables, cube, cam0, disc, sh, out, dbg, stream)
    stream.synchronize()
    d = dbg.view(-1, bh.NDBG)
    texels = float(d[:, 15].sum().item())
    hits = float(d[:, 3].sum().item())
    del dbg, d
    flops_frame = W * H * FLOP_PER_PIXEL + texels * FLOP_PER_TEXEL + hits * FLOP_PER_HIT

    # --- warm-up
    for s in range(args.warmup):
        bh.bh_render(ctx, tables, cube, orbit_camera(wk, s), disc, sh, out, stream)
    stream.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches0 = bh.bh_kernel_launches(ctx)
    sampler = ClockSampler(local)
    sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.zero_()  # L2 flush between timed frames (256 MiB > 129 MB L2)
            evs[s][0].record(stream)
            bh.bh_render(ctx, tables, cube, orbit_camera(wk, args.warmup + s), disc, sh, out, stream)
            evs[s][1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    clocks = sampler.stop()
    launches = bh.bh_kernel_launches(ctx) - launches0
    frame_ms = [a.elapsed_time(b) for a, b in evs]
    t_dev = max_over_ranks(sum(frame_ms) / 1000.0, dev, ws)
    ms_per_step = 1000.0 * t_dev / args.steps
    fps = replica_throughput(args.steps, ws, t_dev)

    # --- end to end through the C ABI with host buffers (D2H of every frame)
    host = torch.empty((H, W, 4), dtype=torch.float32).pin_memory()
    for s in range(2):
        bh.bh_render_to_host(ctx, tables, cube, orbit_camera(wk, s), disc, sh, host, stream)
    e2e_steps = max(5, min(200, args.steps // 2))
    t = time.perf_counter()
    for s in range(e2e_steps):
        bh.bh_render_to_host(ctx, tables, cube, orbit_camera(wk, s), disc, sh, host, stream)
    e2e_t = time.perf_counter() - t
    e2e_fps = ws * e2e_steps / e2e_t

    # --- served (continuous batching) and batched forms on the same frames
    served = serve_run(bh, ctx, tables, cube, wk, sh, dev, frames=max(32, args.steps))
    batched = batch_run(bh, ctx, tables, cube, sh, dev)
    orbits = orbit_run(bh, ctx, tables, cube, sh, dev)
    animated = animated_run(bh, ctx, tables, cube, wk, sh, out, flush, stream)
    served_orbits = serve_orbits_run(bh, ctx, tables, cube, wk, sh, dev, frames=max(32, min(args.steps, 2000)))
    served_mixed = serve_workload(bh, dev, tables, cube, sh) if args.serve_workload else None
    if served_mixed is not None:
        # the largest per-viewer request rate whose p99 latency stays within two
        # 60 Hz frame periods
        sweep = []
        for hz in (5.0, 10.0, 15.0, 20.0, 30.0):
            r = serve_workload(bh, dev, tables, cube, sh, duration=0.6, rate_hz=hz)
            sweep.append({"rate_hz": hz, "p99_ms": r["p99_ms"], "frames_per_s": r["frames_per_s"],
                          "mpix_per_s": r["mpix_per_s"], "refused": r["refused"]})
        ok = [x["rate_hz"] for x in sweep if x["p99_ms"] is not None and x["p99_ms"] <= 2000.0 / 60.0]
        served_mixed["rate_sweep"] = sweep
        served_mixed["max_rate_hz_p99_within_2_frames"] = max(ok) if ok else None

    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = (clocks or {}).get("sm_max_mhz") or (peaks or {}).get("sm_max_mhz") or 2070.0
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = flops_frame / (ms_per_step / 1000.0) / 1e12
    line = {
        "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(wk, ws),
        "mpix_per_s": fps * W * H / 1e6,
        "autotune_choice": tuned,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": render_traffic(),
                     "peak_note": f"FP32 issue: {props.multi_processor_count} SMs x 128 lanes x 2 x {sm_max:.0f} MHz",
                     "flops_per_frame": flops_frame, "texels_per_pixel": texels / (W * H)},
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": 200,
                "d2h_bytes_per_step": W * H * 16},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s_timed_region": wall,
        "precompute_ms": {"tables_D_U_colour": precompute_ms, "cubemap_1M_stars": cubemap_ms},
        "served": served, "served_orbits": served_orbits, "batched": batched, "orbits": orbits,
        "animated_disc": animated,
        "served_mixed": served_mixed,
    }
    if rank == 0 and args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wk, seconds=12.0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    bh.bh_cubemap_free(cube)
    bh.bh_tables_free(tables)
    bh.bh_destroy(ctx)
    if ws > 1:
        torch.distributed.destroy_process_group()


def serve_run(bh, ctx, tables, cube, wk, sh, dev, frames=64, viewers=16):
    """Serve `frames` 1080p frame requests from `viewers` viewers as fast as they
    complete (each viewer resubmits when its frame is done)."""
    import torch
    cam0 = wk["camera"]
    W, H = cam0["width"], cam0["height"]
    outs = [torch.empty((H, W, 4), device=dev) for _ in range(viewers)]
    pending = {}
    lat = []
    submitted = done = 0
    t0 = time.perf_counter()
    while done < frames:
        for v in range(viewers):
            if v not in pending and submitted < frames:
                cam = orbit_camera(wk, submitted)
                st, tk = bh.bh_serve_submit(ctx, tables, cube, v, cam, wk["disc"], sh, outs[v])
                if st == bh.BH_OK:
                    pending[v] = tk
                    submitted += 1
        for v, tk in list(pending.items()):
            st, ms = bh.bh_serve_poll(ctx, tk, 0)
            if st == bh.BH_OK:
                lat.append(ms)
                done += 1
                del pending[v]
        time.sleep(0)
    el = time.perf_counter() - t0
    lat.sort()
    return {"frames_per_s": frames / el, "unit": "1080p frames/s", "viewers": viewers,
            "frames": frames, "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))]}


# Orientation of a camera on an orbit, rows e_w, e_h, e_d on the boosted
# (r', chi', psi') axes: looking at the hole (-e_d = -e_r'), e_w along the motion.
LOOK_AT_HOLE = (0.0, 0.0, 1.0, 0.0, -1.0, 0.0, 1.0, 0.0, 0.0)
RS_PER_SECOND = 60.0  # served trajectories advance 1 r_s/c of proper time per 60 Hz frame


def viewer_orbit(bh, v):
    """Free-fall orbit (Appendix C) of a served viewer from its seeded
    parameters: a circular orbit at r0 in a plane inclined by theta - 90 deg, or
    a fall towards the hole from r0 at the viewer's speed."""
    import math
    if v["kind"] == "circular":
        delta0, v0 = math.pi / 2, min(math.sqrt(1.0 / (2.0 * (v["r0"] - 1.0))), 0.95)
    else:
        delta0, v0 = math.pi - 0.02, v["speed"]
    return bh.bh_orbit_init(v["r0"], delta0, v0, v["theta"] - math.pi / 2, LOOK_AT_HOLE, math.radians(60.0),
                            v["width"], v["height"])


def serve_workload(bh, dev, tables, cube, sh, duration=1.5, viewers=256, rate_hz=60.0,
                   budget=40 << 30):
    """The served workload: `viewers` viewers with Poisson frame requests at
    rate_hz each (mixed 720p/1080p/4K) on free-fall orbits resident on the
    device (each admitted request advances its viewer's orbit by the proper time
    since the viewer's last admitted request), admission under a device-memory
    budget, one disc-parameter change half way that switches new requests to
    freshly rebuilt tables (frames queued on the old tables finish on them).
    Open loop in wall-clock time; reports completed frames/s, Mpix/s, p50/p99
    latency and the refused requests."""
    import torch
    from paper_2010_08735_gb300 import synth
    tr = synth.viewer_traffic(viewers, seed=4, rate_hz=rate_hz, duration_s=duration)
    ctx = bh.bh_create(dev.index or 0, budget)
    vs = tr["viewers"]
    raw = bh.orbits_to_bytes([viewer_orbit(bh, v) for v in vs])
    osize = len(raw) // len(vs)
    orbit_buf = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(dev)
    last_t = [0.0] * len(vs)
    bufs = [[torch.empty((v["height"], v["width"], 4), device=dev) for _ in range(2)] for v in vs]
    disc_a, disc_b = synth.disc(3.0, 12.0), synth.disc(3.0, 14.0)
    cur_tables, old_tables = tables, None
    pending = {}   # ticket -> (viewer, pixels)
    slot = [0] * len(vs)
    lat, px_done, refused, submitted = [], 0, 0, 0
    switched = False
    t0 = time.perf_counter()
    for te, vid in tr["events"]:
        while time.perf_counter() - t0 < te:
            for tk in list(pending):
                st, ms = bh.bh_serve_poll(ctx, tk, 0)
                if st == bh.BH_OK:
                    lat.append(ms)
                    px_done += pending.pop(tk)[1]
        if not switched and te >= duration / 2:
            old_tables = cur_tables
            cur_tables = bh.bh_precompute_tables(ctx, 512, 64, 32, bh.BH_F32)
            switched = True
        v = vs[vid]
        disc = disc_b if switched else disc_a
        if sum(1 for p in pending.values() if p[0] == vid) >= 2:
            refused += 1  # both of the viewer's frame buffers are still in use
            continue
        out = bufs[vid][slot[vid]]
        dtau = RS_PER_SECOND * (te - last_t[vid])
        st, tk = bh.bh_serve_submit_orbit(ctx, cur_tables, cube, vid, orbit_buf.data_ptr() + vid * osize, dtau,
                                          8 if dtau > 0 else 0, v["width"], v["height"], disc, sh, out)
        submitted += 1
        if st == bh.BH_OK:
            pending[tk] = (vid, v["width"] * v["height"])
            slot[vid] ^= 1
            last_t[vid] = te
        else:
            refused += 1
    while pending:
        for tk in list(pending):
            st, ms = bh.bh_serve_poll(ctx, tk, 1000)
            if st == bh.BH_OK:
                lat.append(ms)
                px_done += pending.pop(tk)[1]
    el = time.perf_counter() - t0
    torch.cuda.synchronize()
    if old_tables is not None and cur_tables is not tables:
        bh.bh_tables_free(cur_tables)
    bh.bh_destroy(ctx)
    lat.sort()
    n = len(lat)
    return {"viewers": viewers, "rate_hz_per_viewer": rate_hz, "duration_s": el,
            "offered_req_per_s": len(tr["events"]) / duration, "submitted": submitted,
            "refused": refused, "completed": n, "frames_per_s": n / el,
            "mpix_per_s": px_done / 1e6 / el, "frames_1080p_equiv_per_s": px_done / (1920 * 1080) / el,
            "p50_ms": lat[n // 2] if n else None, "p99_ms": lat[min(n - 1, int(0.99 * n))] if n else None,
            "table_rebuilds": 1, "budget_bytes": budget,
            "mix": "720p/1080p/4K uniform; circular or infalling free-fall orbits advanced on the device"}


def serve_orbits_run(bh, ctx, tables, cube, wk, sh, dev, frames=2000, viewers=16):
    """Viewers on free-fall orbits resident on the device (Appendix C), served
    at 1080p: every request advances its viewer's orbit by 1 r_s/c of proper
    time (8 RK4 steps; an orbit at r = 10 takes about 280 frames) and renders
    it; each viewer resubmits when its frame is done."""
    import math
    import torch
    W, H = wk["camera"]["width"], wk["camera"]["height"]
    rng = np.random.Generator(np.random.PCG64(6))
    orbits = []
    for _ in range(viewers):
        r0 = float(rng.uniform(5.0, 20.0))
        v0 = math.sqrt(1.0 / (2.0 * (r0 - 1.0))) * float(rng.uniform(0.8, 1.1))  # near circular
        orbits.append(bh.bh_orbit_init(r0, math.pi / 2, min(v0, 0.95), float(rng.uniform(-0.5, 0.5)),
                                       LOOK_AT_HOLE, math.radians(60.0), W, H))
    raw = bh.orbits_to_bytes(orbits)
    size = len(raw) // viewers
    buf = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(dev)
    outs = [torch.empty((H, W, 4), device=dev) for _ in range(viewers)]
    dtau = 1.0  # proper time per frame, r_s/c
    pending, lat = {}, []
    submitted = done = 0
    t0 = time.perf_counter()
    while done < frames:
        for v in range(viewers):
            if v not in pending and submitted < frames:
                st, tk = bh.bh_serve_submit_orbit(ctx, tables, cube, v, buf.data_ptr() + v * size, dtau, 8, W, H,
                                                  wk["disc"], sh, outs[v])
                if st == bh.BH_OK:
                    pending[v] = tk
                    submitted += 1
        for v, tk in list(pending.items()):
            st, ms = bh.bh_serve_poll(ctx, tk, 0)
            if st == bh.BH_OK:
                lat.append(ms)
                done += 1
                del pending[v]
        time.sleep(0)
    el = time.perf_counter() - t0
    lat.sort()
    return {"frames_per_s": frames / el, "unit": "1080p frames/s", "viewers": viewers, "frames": frames,
            "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "note": "orbits advanced and cameras set up on the device inside each served batch"}


def animated_run(bh, ctx, tables, cube, wk, sh, out, flush, stream, frames=400, n_particles=16):
    """The same 1080p frames with the animated disc of Appendix B: 16 linear
    particles, each disc crossing shaded at its retarded time; the frame time
    advances by 1 r_s/c per frame.  CUDA-event timed, L2 flushed."""
    import torch
    from paper_2010_08735_gb300 import synth
    parts = synth.disc_particles(n_particles, 5, wk["disc"]["r_in"], wk["disc"]["r_out"])
    handle = bh.bh_disc_particles_create(ctx, parts)
    dt = 1.0  # frame period in r_s / c
    try:
        for s in range(3):
            disc = dict(wk["disc"], particles_handle=handle, time=s * dt)
            bh.bh_render(ctx, tables, cube, orbit_camera(wk, s), disc, sh, out, stream)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(frames)]
        with torch.cuda.stream(stream):
            for s in range(frames):
                disc = dict(wk["disc"], particles_handle=handle, time=(3 + s) * dt)
                flush.zero_()
                evs[s][0].record(stream)
                bh.bh_render(ctx, tables, cube, orbit_camera(wk, 3 + s), disc, sh, out, stream)
                evs[s][1].record(stream)
        stream.synchronize()
    finally:
        bh.bh_disc_particles_free(handle)
    ms = sum(a.elapsed_time(b) for a, b in evs) / frames
    return {"frames_per_s": 1000.0 / ms, "ms_per_frame": ms, "unit": "1080p frames/s", "particles": n_particles,
            "frames": frames, "frame_dt_rs_over_c": dt}


def orbit_run(bh, ctx, tables, cube, sh, dev, n=64, reps=5):
    """64 cameras on free-fall orbits (Appendix C), resident on the device:
    each step advances every orbit by one 60 Hz frame of proper time and
    renders them all (camera set-up on the device, one persistent launch)."""
    import math
    import torch
    from paper_2010_08735_gb300 import synth
    rng = np.random.Generator(np.random.PCG64(5))
    res = synth.BATCH_RESOLUTIONS
    orbits = []
    for _ in range(n):
        w, h = res[int(rng.integers(len(res)))]
        r0 = float(rng.uniform(4.0, 30.0))
        u0 = 1.0 / r0
        v0 = math.sqrt(u0 / (2 * (1 - u0))) * float(rng.uniform(0.9, 1.1))
        orbits.append(bh.bh_orbit_init(r0, float(rng.uniform(1.2, 1.9)), min(v0, 0.9),
                                       float(rng.uniform(0, math.pi)), None, math.pi / 3, w, h))
    buf = torch.frombuffer(bytearray(bh.orbits_to_bytes(orbits)), dtype=torch.uint8).to(dev)
    outs = [torch.empty((o.height, o.width, 4), device=dev) for o in orbits]
    disc = synth.disc()
    s = torch.cuda.Stream(device=dev)
    bh.bh_orbits_advance(ctx, buf, n, 0.05, 8, s)
    bh.bh_render_orbits(ctx, tables, cube, n, buf, disc, sh, outs, s)
    s.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        bh.bh_orbits_advance(ctx, buf, n, 0.05, 8, s)
        bh.bh_render_orbits(ctx, tables, cube, n, buf, disc, sh, outs, s)
    e1.record(s)
    s.synchronize()
    ms = e0.elapsed_time(e1) / reps
    px = sum(o.width * o.height for o in orbits)
    return {"cameras": n, "ms_per_step": ms, "mpix_per_s": px / 1e6 / (ms / 1000.0),
            "frames_1080p_equiv_per_s": px / (1920 * 1080) / (ms / 1000.0),
            "note": "advance + on-device camera set-up + render, per step"}


def batch_run(bh, ctx, tables, cube, sh, dev, n=64, reps=5):
    """64 cameras of mixed resolution in one persistent launch; Mpix/s and
    1080p-equivalent frames/s, after the autotuner picked a launch shape."""
    import torch
    from paper_2010_08735_gb300 import synth
    cams = synth.batch_cameras(n, seed=1)
    outs = [torch.empty((c["height"], c["width"], 4), device=dev) for c in cams]
    disc = synth.disc()
    chosen = bh.bh_autotune_batch(ctx, tables, cube, cams, disc, sh, outs)
    s = torch.cuda.Stream(device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bh.bh_render_batch(ctx, tables, cube, cams, disc, sh, outs, s)
    s.synchronize()
    e0.record(s)
    for _ in range(reps):
        bh.bh_render_batch(ctx, tables, cube, cams, disc, sh, outs, s)
    e1.record(s)
    s.synchronize()
    ms = e0.elapsed_time(e1) / reps
    px = sum(c["width"] * c["height"] for c in cams)
    return {"cameras": n, "mpix_per_batch": px / 1e6, "ms_per_batch": ms,
            "mpix_per_s": px / 1e6 / (ms / 1000.0), "frames_1080p_equiv_per_s": px / (1920 * 1080) / (ms / 1000.0),
            "autotune_choice": chosen}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-serve-workload", dest="serve_workload", action="store_false")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
