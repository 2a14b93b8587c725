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
# The algorithmic work of a frame of each workload, tallied by the oracle's
# counting build (tests/golden/make_work_counts.py): arithmetic by class,
# texels read and the unique cube-map records a frame touches.
WORK_COUNTS = ROOT / "tests" / "golden" / "work_counts.json"


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


def kernel_traffic(record="render_traffic.json", source="bh_render.cu"):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    f = ROOT / "profiles" / record
    if not f.exists():
        return None
    d = json.loads(f.read_text())
    src = (ROOT / "paper_2010_08735_gb300" / "csrc" / source).read_bytes()
    if d.get("kernel_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return d.get("dram_bytes_per_launch")


def render_traffic():
    return kernel_traffic("render_traffic.json", "bh_render.cu")


def work_counts(name):
    return json.loads(WORK_COUNTS.read_text())[name]


def roofline(name, ms_per_frame, rates, sm_mhz, hbm_gbs, traffic=None):
    """Roofline of the render kernel on one frame of workload `name`: the
    slowest of three legs, each the method's own work (oracle counts) at the
    measured peak of its unit:
      fp32 -- add/sub + mul + div (one flop each, two per FMA lane-cycle) at the
              measured FMA rate;
      sfu  -- sqrt + elementary functions (at least one special-function
              operation each) at the measured special-function rate;
      hbm  -- 16 B per pixel stored + 8 B per unique cube-map record the frame
              touches, at the measured copy bandwidth.
    frac = (roofline time) / (measured time) = the largest leg's
    achieved / peak."""
    c = work_counts(name)
    t = ms_per_frame / 1000.0
    sms, hz = rates["sms"], sm_mhz * 1e6
    flops = c["add"] + c["mul"] + c["div"]
    sfu = c["sqrt"] + c["transcendental"]
    nbytes = 16 * c["pixels"] + 8 * c["unique_cube_records"]
    legs = {
        "fp32": {"work_per_frame": flops, "unit": "TFLOP/s", "achieved": flops / t / 1e12,
                 "peak": sms * rates["fp32_fma_per_sm_clk"] * 2 * hz / 1e12},
        "sfu": {"work_per_frame": sfu, "unit": "Top/s", "achieved": sfu / t / 1e12,
                "peak": sms * rates["mufu_per_sm_clk"] * hz / 1e12},
        "hbm": {"work_per_frame": nbytes, "unit": "GB/s", "achieved": nbytes / t / 1e9, "peak": hbm_gbs},
    }
    for v in legs.values():
        v["frac"] = v["achieved"] / v["peak"]
        v["roofline_us"] = v["work_per_frame"] / (v["peak"] * (1e9 if v["unit"] == "GB/s" else 1e12)) * 1e6
    top = max(legs, key=lambda k: legs[k]["frac"])
    L = legs[top]
    return {"bound": "hbm" if top == "hbm" else "alu", "leg": top, "achieved": L["achieved"],
            "peak": L["peak"], "unit": L["unit"], "frac": L["frac"], "traffic": traffic,
            "peak_note": (f"of measured: {sms} SMs x {rates['fp32_fma_per_sm_clk']:.1f} FMA / "
                          f"{rates['mufu_per_sm_clk']:.1f} SFU results per SM per clock (the library's "
                          f"microbenchmark) x {sm_mhz:.0f} MHz (median SM clock of the timed region); "
                          f"HBM {hbm_gbs:.0f} GB/s (MEASURED_PEAKS.json)"),
            "work_source": "tests/golden/work_counts.json (oracle counting build)",
            "legs": legs, "measured_us": ms_per_frame * 1000.0}


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


def oracle_scene(wk, tables64=False):
    """The oracle's tables and star cube map for workload wk (FP32-stored
    tables as the renderer reads them, or the FP64 tables themselves)."""
    import oracle
    from paper_2010_08735_gb300 import synth
    D, U = oracle.tables_exact(512, 64, 32, 1e-3)
    Ct, dl = oracle.colour_table(), oracle.disc_colour_table()
    dt = 1 if wk["cube_dtype"] == "f16" else 2
    rec = oracle.build_cubemap(synth.stars(wk["n_stars"], wk["star_seed"]), wk["cube_n"], dt)
    f = (lambda a: a) if tables64 else (lambda a: a.astype(np.float32))
    return oracle.SceneTables(f(D), f(U), Ct.astype(np.float32), dl.astype(np.float32), rec, wk["cube_n"], dt), (D, U)


def cpu_baseline(wk, seconds=12.0, scene=None, setup_s=0.0):
    """The oracle, as it stands, on the host cores: full-resolution rows of the
    same workload until about `seconds` of rendering, scaled to frames/s; and
    on one core, 16 rows spread over the frame (two-row bands at eight
    heights, so the shadow and the star field are both sampled)."""
    import oracle
    t0 = time.perf_counter()
    if scene is None:
        scene, _ = oracle_scene(wk)
    setup = time.perf_counter() - t0 + setup_s
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
    t1 = 0.0
    for k in range(8):
        y0 = (k * H // 8 + H // 16) // 2 * 2
        t = time.perf_counter()
        oracle.render(cam, wk["disc"], scene, exposure_stars=0.01, y0=y0, y1=y0 + 2, nthreads=1)
        t1 += time.perf_counter() - t
    fps1 = (16 / H) / t1
    return {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "one_core_value": fps1,
            "sample": f"{rows} of {H} rows of the {cam['width']}x{H} frame ({rows * cam['width']} px), "
                      f"FP64 C oracle with {cores} threads (one_core_value: 16 rows in eight 2-row bands spread "
                      f"over the frame, one thread); oracle set-up {setup:.1f} s untimed"}


def edge_mask(cap, hits):
    """Pixels within 1 px of a change of capture state or disc-hit count (the
    shadow silhouette and the disc edges), where no tolerance applies."""
    e = np.zeros(cap.shape, dtype=bool)
    for a in (cap, hits):
        d = np.zeros(cap.shape, dtype=bool)
        d[:, 1:] |= a[:, 1:] != a[:, :-1]
        d[:, :-1] |= a[:, 1:] != a[:, :-1]
        d[1:] |= a[1:] != a[:-1]
        d[:-1] |= a[1:] != a[:-1]
        e |= d
    m = e.copy()
    m[1:] |= e[:-1]
    m[:-1] |= e[1:]
    m2 = m.copy()
    m2[:, 1:] |= m[:, :-1]
    m2[:, :-1] |= m[:, 1:]
    return m2


def rel_error(img, ref, mask):
    """Per-pixel relative linear-RGB error (denominator max(|ref|, 1e-4 max|ref|))
    outside `mask`: mean, p99 and max."""
    g = img[..., :3].astype(np.float64)
    o = ref[..., :3].astype(np.float64)
    floor = 1e-4 * max(np.abs(o).max(), 1e-30)
    r = (np.abs(g - o) / np.maximum(np.abs(o), floor)).max(-1)[~mask]
    return {"mean_rel": float(r.mean()), "p99_rel": float(np.percentile(r, 99)), "max_rel": float(r.max()),
            "pixels": int(r.size), "masked": int(mask.sum())}


def oracle_leg(wk, gpu_frames, seconds=12.0):
    """Everything that runs the oracle (rank 0, one GPU): the CPU baseline, and
    the error statement of the GPU's outputs against the FP64 oracle:
    1080p frames rendered with FP32- and FP16-stored tables against the oracle
    on the FP64 tables themselves (the tables' storage error), and the table
    method against the table-free photon orbit on 1000 beams of the frame
    (Sec. 4's accuracy statement, delta' in rad and u = r_s/r)."""
    import oracle
    from paper_2010_08735_gb300 import synth
    t0 = time.perf_counter()
    scene32, (D, U) = oracle_scene(wk)
    cb = cpu_baseline(wk, seconds, scene=scene32, setup_s=time.perf_counter() - t0)
    cam, disc = wk["camera"], wk["disc"]
    exact = oracle.SceneTables(D, U, scene32.C, scene32.disc_ln, scene32.cube, scene32.cube_n,
                               scene32.cube_dtype)
    ref, dbg, _ = oracle.render(cam, disc, exact, exposure_stars=0.01, debug=True)
    mask = edge_mask(~np.isfinite(dbg[..., 2]), dbg[..., 3])
    # the parity tests' full exclusion (reading C19): also mip-level and face
    # decisions within 2 % / 2e-3 of their thresholds, degenerate footprints and
    # star pixels whose RGB changes by more than 1 % for the 1e-6 rad an FP32
    # escape direction can be off (oracle channels 6, 16, 17, 18, 8, 20-22)
    lvl, hm = dbg[..., 6], dbg[..., 16]
    has = lvl >= 0
    ratio = np.where(has, 2 * hm / (8 * 2.0 ** np.maximum(lvl, 0)), 0.0)
    prev = np.where(has & (lvl > 0), 2 * hm / (8 * 2.0 ** np.maximum(lvl - 1, 0)), 0.0)
    floor = 1e-4 * max(np.abs(ref[..., :3]).max(), 1e-30)
    sens = (dbg[..., 20:23] / np.maximum(np.abs(ref[..., :3]), floor)).max(-1)
    shift_px = 1e-6 * np.sqrt(np.maximum(dbg[..., 8], 0.0)) / (cam["fov_y"] / cam["height"])
    c19 = (mask | (has & (ratio > 0.98) & (ratio <= 1)) | (has & (lvl > 0) & (prev < 1.02)) |
           (has & (dbg[..., 17] < 2e-3)) | (has & (dbg[..., 18] < 1e-5)) | (sens * shift_px > 1e-2))
    del dbg
    errors = {"workload": WORKLOAD, "reference": "FP64 oracle on the FP64 tables",
              "mask": "pixels within 1 px of the shadow silhouette or a disc edge",
              "mask_c19": "that mask plus the parity tests' threshold-margin, degenerate and "
                          "FP32-ill-conditioned star pixels (reading C19)"}
    for k, img in gpu_frames.items():
        errors[k] = rel_error(img, ref, mask)
        errors[k + "_c19"] = rel_error(img, ref, c19)
    # table method vs the table-free 3D photon orbit (Sec. 4)
    W, H = cam["width"], cam["height"]
    th, ph = cam["theta"], cam["phi"]
    er = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    rng = np.random.default_rng(11)
    de, ue, nb = [], [], 0
    while nb < 1000:
        i, j = int(rng.integers(0, W)), int(rng.integers(0, H))
        b = oracle.beam(cam, i + 0.5 - W / 2, H / 2 - j - 0.5)
        tr = oracle.trace_ray(D, U, cam["r"], b["delta"], b["alpha"], 1 / disc["r_in"], 1 / disc["r_out"],
                              b["alpha_valid"])
        bf = oracle.bruteforce_ray(cam["r"] * er, b["dcart"], disc["r_in"], disc["r_out"])
        nb += 1
        if not bf["captured"] and not math.isinf(tr["delta_p"]):
            dp = math.cos(tr["delta_p"]) * er + math.sin(tr["delta_p"]) * b["ey"]
            de.append(math.acos(min(1.0, float(dp @ bf["dir"]))))
        hits = [h[0] for h in tr["hits"]]
        if len(hits) == len(bf["hits_u"][:2]):
            ue += [abs(a - c) for a, c in zip(hits, bf["hits_u"][:2])]
    de, ue = np.array(de), np.array(ue)
    errors["table_method_vs_bruteforce"] = {
        "beams": nb, "delta_prime_rad": {"p50": float(np.median(de)), "p99": float(np.percentile(de, 99)),
                                         "max": float(de.max()), "n": int(de.size)},
        "hit_u": {"p50": float(np.median(ue)), "p99": float(np.percentile(ue, 99)), "max": float(ue.max()),
                  "n": int(ue.size)},
        "paper_bound": 1e-3}
    return cb, errors


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2010_08735_gb300 import synth
    wk = synth.WORKLOADS[WORKLOAD]
    cb = cpu_baseline(wk, seconds=max(5.0, 2.0 * args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "frames/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / cb["value"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wk, args.gpus),
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_frames(bh, ctx, tables, cube, wk, sh, out, flush, stream, steps, step0=0):
    """Render `steps` frames of workload wk (camera moving along its orbit),
    each after an L2 flush, each timed by CUDA events on its stream; returns
    the per-frame milliseconds."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for s in range(steps):
            flush.zero_()  # L2 flush between timed frames (256 MiB > 129 MB L2)
            evs[s][0].record(stream)
            bh.bh_render(ctx, tables, cube, orbit_camera(wk, step0 + s), wk["disc"], sh, out, stream)
            evs[s][1].record(stream)
    stream.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * len(xs)))]


def plain_wall_run(bh, ctx, tables, cube, wk, sh, out, stream, frames=2000):
    """The plain form, measured like the served one: one bh_render per frame,
    then a stream synchronisation; wall-clock latency per frame (launch to
    completion seen by the host), no L2 flush (as in serving)."""
    lat = []
    for s in range(20):
        bh.bh_render(ctx, tables, cube, orbit_camera(wk, s), wk["disc"], sh, out, stream)
    stream.synchronize()
    t0 = time.perf_counter()
    for s in range(frames):
        t = time.perf_counter()
        bh.bh_render(ctx, tables, cube, orbit_camera(wk, s), wk["disc"], sh, out, stream)
        stream.synchronize()
        lat.append((time.perf_counter() - t) * 1000.0)
    el = time.perf_counter() - t0
    return {"frames_per_s": frames / el, "unit": "1080p frames/s", "frames": frames,
            "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99), "l2": "not flushed (as served)"}


def other_workload(bh, ctx, tables, name, sh, dev, stream, flush, rates, steps=200, warmup=5):
    """Device-timed frames of another workload (its own star cube map), with
    its roofline; returns (line, cube handle) -- the caller frees the cube."""
    import torch
    from paper_2010_08735_gb300 import synth
    wk = synth.WORKLOADS[name]
    W, H = wk["camera"]["width"], wk["camera"]["height"]
    stars = torch.from_numpy(synth.stars(wk["n_stars"], wk["star_seed"])).to(dev)
    cube = bh.bh_build_star_cubemap(ctx, stars, wk["cube_n"],
                                    bh.BH_F16 if wk["cube_dtype"] == "f16" else bh.BH_BF16, stream)
    del stars
    out = torch.empty((H, W, 4), device=dev)
    for s in range(warmup):
        bh.bh_render(ctx, tables, cube, orbit_camera(wk, s), wk["disc"], sh, out, stream)
    ms = timed_frames(bh, ctx, tables, cube, wk, sh, out, flush, stream, steps, warmup)
    ms_frame = sum(ms) / len(ms)
    line = {"workload": name, "width": W, "height": H, "stars": wk["n_stars"], "cube_face": wk["cube_n"],
            "cube_dtype": wk["cube_dtype"], "frames": steps, "ms_per_frame": ms_frame,
            "frames_per_s": 1000.0 / ms_frame, "mpix_per_s": W * H / ms_frame / 1000.0,
            "l2": "flushed before each frame",
            "roofline": roofline(name, ms_frame, rates, rates["sm_mhz_timed"],
                                 (measured_peaks() or {}).get("hbm_gbs", 6800.0))}
    return line, cube, out


def bloom_run(bh, ctx, out, W, H, fov_y, flush, stream, frames=400, levels=6):
    """The lens-glare bloom (Sec. 3.4.3) of the 1080p frame, in place, each
    call after an L2 flush, CUDA-event timed; HBM roofline on its algorithmic
    bytes: the frame read and written once, each pyramid level written and
    read twice (box level, blurred level)."""
    import torch
    w = bh.bh_bloom_weights(fov_y, H, levels)
    buf = out.clone()
    for _ in range(3):
        bh.bh_bloom(ctx, buf, buf, W, H, w, stream)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(frames)]
    with torch.cuda.stream(stream):
        for s in range(frames):
            flush.zero_()
            evs[s][0].record(stream)
            bh.bh_bloom(ctx, buf, buf, W, H, w, stream)
            evs[s][1].record(stream)
    stream.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / frames
    texels, w_, h_ = 0, W, H
    for _ in range(levels):
        w_, h_ = (w_ + 1) // 2, (h_ + 1) // 2
        texels += w_ * h_
    nbytes = 16 * 2 * W * H + 16 * 4 * texels
    hbm = (measured_peaks() or {}).get("hbm_gbs", 6800.0)
    ach = nbytes / (ms / 1000.0) / 1e9
    return {"ms_per_frame": ms, "frames_per_s": 1000.0 / ms, "levels": levels, "launches_per_frame": 1,
            "weights": [float(x) for x in w],
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                         "bytes_per_frame": nbytes,
                         "traffic": kernel_traffic("bloom_traffic.json", "bh_bloom.cu")}}


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
    # SM issue rates of this GPU (the library's microbenchmark; untimed)
    rates = bh.bh_measure_issue_rates(local)
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

    # --- warm-up, then the timed frames
    for s in range(args.warmup):
        bh.bh_render(ctx, tables, cube, orbit_camera(wk, s), disc, sh, out, stream)
    stream.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches0 = bh.bh_kernel_launches(ctx)
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    frame_ms = timed_frames(bh, ctx, tables, cube, wk, sh, out, flush, stream, args.steps, args.warmup)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    clocks = sampler.stop()
    launches = bh.bh_kernel_launches(ctx) - launches0
    t_dev = max_over_ranks(sum(frame_ms) / 1000.0, dev, ws)
    ms_per_step = 1000.0 * t_dev / args.steps
    fps = replica_throughput(args.steps, ws, t_dev)
    rates["sm_mhz_timed"] = (clocks or {}).get("sm_mhz") or rates["sm_mhz"]
    hbm = (measured_peaks() or {}).get("hbm_gbs", 6800.0)
    rl = roofline(WORKLOAD, ms_per_step, rates, rates["sm_mhz_timed"], hbm, render_traffic())

    if not args.extras:
        # the timed frames alone (for profiling runs): no extra measurement legs
        line = {"metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(wk, ws),
                "roofline": rl, "gpu_launches": int(launches), "clocks": clocks, "extras": False}
        if rank == 0:
            print(json.dumps(line), flush=True)
        bh.bh_cubemap_free(cube)
        bh.bh_tables_free(tables)
        bh.bh_destroy(ctx)
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    # --- end to end through the C ABI with host buffers (D2H of every frame):
    # the packed linear-RGB form (12 B/px) and, for reference, the RGBA one
    e2e_steps = max(200, min(1000, args.steps // 4))
    e2e = {}
    for name, fn, ch in (("rgb", bh.bh_render_to_host_rgb, 3), ("rgba", bh.bh_render_to_host, 4)):
        host = torch.empty((H, W, ch), dtype=torch.float32).pin_memory()
        for s in range(3):
            fn(ctx, tables, cube, orbit_camera(wk, s), disc, sh, host, stream)
        t = time.perf_counter()
        for s in range(e2e_steps):
            fn(ctx, tables, cube, orbit_camera(wk, s), disc, sh, host, stream)
        e2e[name] = ws * e2e_steps / (time.perf_counter() - t)
        del host
    # two frames in flight (bh_render_to_host_async): frame s renders while
    # frame s - 1 is copied to the host; every frame is in host memory
    # (bh_host_wait) inside the timed region
    hosts = [torch.empty((H, W, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
    for s in range(3):
        bh.bh_host_wait(ctx, bh.bh_render_to_host_async(ctx, tables, cube, orbit_camera(wk, s), disc, sh,
                                                        hosts[s & 1], True, stream))
    t = time.perf_counter()
    prev = None
    for s in range(e2e_steps):
        tk = bh.bh_render_to_host_async(ctx, tables, cube, orbit_camera(wk, s), disc, sh, hosts[s & 1], True,
                                        stream)
        if prev is not None:
            bh.bh_host_wait(ctx, prev)
        prev = tk
    bh.bh_host_wait(ctx, prev)
    e2e["rgb_async"] = ws * e2e_steps / (time.perf_counter() - t)
    del hosts
    e2e_fps = e2e["rgb_async"]
    # the link's own bandwidth (the library's measurement, the frame's size)
    link = bh.bh_measure_host_link(local, W * H * 12)
    link_gbs = max(link["copy_engine_gbs"], link["kernel_stores_gbs"])

    # --- plain and served forms on equal terms: host wall clock per frame,
    # 2000 frames each, the same cameras, no L2 flush on either side
    plain = plain_wall_run(bh, ctx, tables, cube, wk, sh, out, stream, frames=2000)
    served = serve_run(bh, ctx, tables, cube, wk, sh, dev, frames=2000)
    served["served_over_plain"] = served["frames_per_s"] / plain["frames_per_s"]
    batched = batch_run(bh, ctx, tables, cube, sh, dev)
    orbits = orbit_run(bh, ctx, tables, cube, sh, dev)
    animated = animated_run(bh, ctx, tables, cube, wk, sh, out, flush, stream)
    bloom = bloom_run(bh, ctx, out, W, H, cam0["fov_y"], flush, stream)
    served_orbits = serve_orbits_run(bh, ctx, tables, cube, wk, sh, dev, frames=2000)
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

    # --- the other workloads, device-timed with their rooflines; the 4K
    # frame's BF16 cube-map storage error (against the same frame on an FP16
    # cube map, whose rounding is 8x finer)
    others = {}
    line256, cube256, _ = other_workload(bh, ctx, tables, "static_256", sh, dev, stream, flush, rates)
    bh.bh_cubemap_free(cube256)
    others["static_256"] = line256
    line4k, cube4k, out4k = other_workload(bh, ctx, tables, "infall_4k", sh, dev, stream, flush, rates)
    wk4 = synth.WORKLOADS["infall_4k"]
    cam4 = wk4["camera"]
    stars4 = torch.from_numpy(synth.stars(wk4["n_stars"], wk4["star_seed"])).to(dev)
    cube4k16 = bh.bh_build_star_cubemap(ctx, stars4, wk4["cube_n"], bh.BH_F16, stream)
    del stars4
    dbg4 = torch.empty((cam4["height"], cam4["width"], bh.NDBG), device=dev)
    bh.bh_render_debug(ctx, tables, cube4k, cam4, wk4["disc"], sh, out4k, dbg4, stream)
    stream.synchronize()
    cap4 = torch.isinf(dbg4[..., 2]).cpu().numpy()
    hits4 = dbg4[..., 3].cpu().numpy()
    del dbg4
    img_bf16 = out4k.cpu().numpy()
    bh.bh_render(ctx, tables, cube4k16, cam4, wk4["disc"], sh, out4k, stream)
    stream.synchronize()
    img_f16 = out4k.cpu().numpy()
    bh.bh_cubemap_free(cube4k)
    bh.bh_cubemap_free(cube4k16)
    del out4k
    line4k["bf16_cube_storage_error"] = dict(rel_error(img_bf16, img_f16, edge_mask(cap4, hits4)),
                                             reference="the same 4K frame on an FP16 cube map of the same stars")
    del img_bf16, img_f16
    others["infall_4k"] = line4k

    # --- GPU frames for the error statement: FP32- and FP16-stored tables
    bh.bh_render(ctx, tables, cube, cam0, disc, sh, out, stream)
    stream.synchronize()
    frames = {"tables_f32": out.cpu().numpy()}
    t16 = bh.bh_precompute_tables(ctx, 512, 64, 32, bh.BH_F16, stream)
    bh.bh_render(ctx, t16, cube, cam0, disc, sh, out, stream)
    stream.synchronize()
    frames["tables_f16"] = out.cpu().numpy()
    bh.bh_tables_free(t16)

    line = {
        "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(wk, ws),
        "mpix_per_s": fps * W * H / 1e6,
        "autotune_choice": tuned,
        "roofline": rl,
        "issue_rates": rates,
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": 200,
                "d2h_bytes_per_step": W * H * 12, "frames": e2e_steps,
                "api": "bh_render_to_host_async + bh_host_wait (packed linear RGB into pinned host memory, "
                       "two frames in flight: one renders while the other is copied)",
                "one_at_a_time_frames_per_s": e2e["rgb"], "rgba_one_at_a_time_frames_per_s": e2e["rgba"],
                "host_link": {"copy_engine_gbs": link["copy_engine_gbs"],
                              "kernel_stores_gbs": link["kernel_stores_gbs"],
                              "achieved_gbs": e2e_fps * W * H * 12 / 1e9,
                              "frac": e2e_fps * W * H * 12 / 1e9 / link_gbs,
                              "note": "bh_measure_host_link on this box: the frame's bytes device -> pinned host"}},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s_timed_region": wall,
        "precompute_ms": {"tables_D_U_colour": precompute_ms, "cubemap_1M_stars": cubemap_ms},
        "plain_wall": plain, "served": served, "served_orbits": served_orbits, "batched": batched,
        "orbits": orbits, "animated_disc": animated, "served_mixed": served_mixed, "bloom": bloom,
        "other_workloads": others,
    }
    if rank == 0 and args.cpu_baseline:
        line["cpu_baseline"], line["errors"] = oracle_leg(wk, frames, seconds=12.0)
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
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="after the timed frames, skip the other measurement legs (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
