"""Benchmark of the motion-focus path on GB300: 1080p frames/s and % of HBM roofline.

Workload: one stream of 900 frames at 1920x1080 (fx = fy = 1500, principal
point (960, 540)), window 16, 15-sample fit, ACCEL mode, FP32 depth and
maps; synthetic walker with turns, depth ray-cast from a seeded box scene
(ring of 8 rendered images over 900 distinct HBM planes).  One step is one
pass of the whole path over the batch through the C ABI: reset, push of the
900 poses and depth planes (anchoring + motion points), and mf_get_maps of
all 900 frames (motion-focus map, guided depth, per-frame records).

The timed region holds K steps between CUDA events on the library's stream,
bracketed by a barrier and synchronisation; the inputs (7.5 GB) and outputs
(15 GB) are far larger than L2, so no flush is needed.  ``e2e`` repeats the
measurement with host buffers (pinned), host<->device copies inside.

``--impl reference`` times the FP64 CPU oracle (the test oracle, not a
product path) on the host cores on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p frames/s & % HBM roofline; p99 frame latency, served vs plain, same GPU"
WIDTH, HEIGHT, FRAMES, WINDOW, SMOOTH = 1920, 1080, 900, 16, 15
BYTES_PER_PX = 12  # depth read + focus map write + guided depth write (FP32)
FRAME_BYTES = WIDTH * HEIGHT * BYTES_PER_PX
# committed ncu summary and the sources it was taken from, per map kernel
PROFILES = {
    ("map_stream_kernel", "default"): ("map_kernel_1080p_f32.txt", ("mf_map_kernel.cuh", "mf_map_n16.cu",
                                                                    "mf_map_unit.cuh")),
    ("map_stream_kernel", "heading"): ("map_kernel_1080p_f32_heading.txt",
                                       ("mf_map_kernel.cuh", "mf_map_n16.cu", "mf_map_unit.cuh")),
    ("map_tc_kernel", "default"): ("map_tc_kernel_1080p_f32.txt", ("mf_map_tc.cu", "mf_map_unit.cuh")),
}
# workloads of the 1080p line: the default (config 2: ACCEL, constant-speed
# walker with turns), HEADING on the same frames, ACCEL on a walker that also
# speeds up and slows down (1.5 m/s^2), whose points land in view
WORKLOADS = {"default": ("accel", 0.0), "heading": ("heading", 0.0), "accel_in_view": ("accel", 1.5)}


PIECE_FRAMES = max(1, min(64, (128 << 20) // (12 * WIDTH * HEIGHT)))  # library transfer piece


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def workload_config(frames=FRAMES, workload="default"):
    mode, acc = WORKLOADS[workload]
    walker = "walker with turns" + (f" and forward speed changes up to {acc:g} m/s^2" if acc else "")
    return {"workload": f"1 stream, {frames} frames 1920x1080, window 16, K=15 fit, {mode.upper()}, "
                        f"FP32 depth+maps, {walker}, ray-cast box scene",
            "frames_per_step": frames, "width": WIDTH, "height": HEIGHT, "window": WINDOW,
            "smooth_len": SMOOTH, "l2": "inputs+outputs 22.4 GB per step >> 129 MB L2 (no flush)"}


# ------------------------------------------------------------------ peaks --
def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def map_kernel_name(stats):
    """Kernel of the stream's last map launch, by its CUDA function name."""
    import paper_2601_07154_gb300 as mf
    return {mf._mf.MF_FLAG_MAP_TENSOR_CORES: "map_tc_kernel",
            mf._mf.MF_FLAG_MAP_CUDA_CORES: "map_stream_kernel"}.get(int(stats.last_map_kernel),
                                                                   "unknown")


def map_source_hash(key):
    h = hashlib.sha256()
    for f in PROFILES[key][1]:
        path = os.path.join(ROOT, "paper_2601_07154_gb300", "csrc", f)
        if os.path.exists(path):
            h.update(open(path, "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(frames, kernel, workload="default"):
    """DRAM bytes per launch from the committed ncu summary of `kernel` on
    `workload`, if the summary was taken from the current sources."""
    key = (kernel, workload)
    if key not in PROFILES:
        return None
    try:
        text = open(os.path.join(ROOT, "profiles", PROFILES[key][0])).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256_16") != map_source_hash(key):
        return None
    try:
        per_frame = float(vals["dram_bytes_per_frame"])
    except (KeyError, ValueError):
        return None
    return per_frame * frames


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def smi_index(torch, dev, local):
    """nvidia-smi index of the torch device: by UUID, else PCI bus, else the only GPU."""
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=index,uuid,pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=20).stdout.strip().splitlines()
    except (OSError, subprocess.SubprocessError):
        return local
    rows = [[c.strip() for c in ln.split(",")] for ln in out if ln.count(",") >= 2]
    if len(rows) == 1:
        return rows[0][0]
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", ""))
    for idx, u, bus in rows:
        if uuid and uuid in u:
            return idx
        pci = getattr(props, "pci_bus_id", None)
        if pci is not None and bus.lower().endswith(f"{int(pci):02x}:00.0"):
            return idx
    return local


# ------------------------------------------------------------ GPU arm ----
def make_inputs(torch, dev, frames, workload="default"):
    from synth import hd_stream
    w = hd_stream(accel=WORKLOADS[workload][1])
    ring = torch.from_numpy(np.stack([w.depth(k) for k in range(w.ring)])).to(dev)
    idx = torch.tensor([k % w.ring for k in range(frames)], device=dev)
    depth = ring[idx].contiguous()
    poses = torch.from_numpy(np.ascontiguousarray(w.poses[:frames])).to(dev)
    return w, poses, depth


def combine_ranks(torch, dist, ms_local, frames_local, world, dev):
    """Whole-job timing: the slowest rank's time, every rank's frames.

    Replicas process independent streams (no data exchange); the only
    collectives are this reduction and the barriers around the timed region.
    """
    ms = ms_local
    frames = frames_local
    if world > 1:
        t = torch.tensor([ms_local, float(frames_local)], device=dev, dtype=torch.float64)
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        ms = float(mx[0].item())
        frames = float(sm[1].item())
    return ms, frames / (ms / 1000.0)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2601_07154_gb300 as mf

    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    frames = args.frames
    w, poses, depth = make_inputs(torch, dev, frames, args.workload)
    K = w.K()
    M = torch.empty((frames, HEIGHT, WIDTH), dtype=torch.float32, device=dev)
    G = torch.empty_like(M)
    info = torch.empty(frames * 64, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)
    s = mf.MotionFocusStream(WIDTH, HEIGHT, window=WINDOW, smooth_len=SMOOTH, device=dev,
                             cuda_stream=stream, time_kernels=True, map_kernel=args.map_kernel,
                             mode=WORKLOADS[args.workload][0])
    h = s.handle
    Kh = np.ascontiguousarray(K)

    def step():
        mf.mf_reset_stream(h)
        mf.mf_push_frames(h, frames, poses, depth, Kh)
        got = mf.mf_get_maps(h, frames, M, G, info, None)
        assert got == frames

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    s0 = s.stats()
    l0 = mf.mf_total_kernel_launches()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(smi_index(torch, dev, local))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    launches = mf.mf_total_kernel_launches() - l0
    s1 = s.stats()
    map_ms = (s1.map_kernel_ms - s0.map_kernel_ms) / max(1, s1.map_launches - s0.map_launches)
    ms, value = combine_ranks(torch, dist, ms, frames * args.steps, world, dev)

    e2e = None
    if rank == 0 and not args.no_e2e:
        M = G = None
        e2e = run_e2e(torch, mf, w, depth, dev, args)
    prec = None
    if rank == 0 and not args.no_precision:
        prec = run_precision(torch, mf, w, poses, depth, dev, args, value / world)
    variants = None
    if rank == 0 and not args.no_variants:
        variants = run_variants(torch, mf, w, poses, depth, dev, args, value / world)
        if prec is not None:
            for name, dt in (("bf16_heading", torch.bfloat16), ("f16_heading", torch.float16)):
                prec[name] = run_leg(torch, mf, w, poses, depth, dev, args, dt, mode="heading")
                prec[name]["gain_vs_f32_heading"] = round(prec[name]["value"] /
                                                          variants["heading_f32"]["value"], 3)
    batched = served = None
    if rank == 0 and not args.no_serving:
        del M, G
        M = G = None
        pools32 = depth_pools(torch, dev, args.batch_frames, torch.float32)
        pools16 = {k: v.to(torch.bfloat16) for k, v in pools32.items()}
        # HEADING keeps the motion points in view, so every unit computes and
        # reads depth (the constant-speed ACCEL walkers' points mostly leave
        # the images); so does ACCEL on walkers that speed up and slow down
        legs = [("engine_f32", torch.float32, False, "accel", 0.0),
                ("engine_bf16", torch.bfloat16, False, "accel", 0.0),
                ("plain_f32", torch.float32, True, "accel", 0.0),
                ("engine_f32_heading", torch.float32, False, "heading", 0.0),
                ("engine_bf16_heading", torch.bfloat16, False, "heading", 0.0),
                ("plain_f32_heading", torch.float32, True, "heading", 0.0),
                ("engine_bf16_accel_in_view", torch.bfloat16, False, "accel", 1.5),
                ("plain_f32_accel_in_view", torch.float32, True, "accel", 1.5)]
        want = None if args.batch_legs == "all" else set(args.batch_legs.split(","))
        batched = {"workload": "64 streams, resolutions 640x480..3840x2160, windows 8..32, "
                               f"{args.batch_frames} frames per stream per step, own depth "
                               "planes per stream"}
        for name, dt, plain, mode, acc in legs:
            if want is None or name in want:
                batched[name] = run_batched(torch, mf, dev, args, pools32 if dt == torch.float32
                                            else pools16, dt, plain=plain, mode=mode, accel=acc)
        for k, base in (("engine_f32", "plain_f32"), ("engine_bf16", "plain_f32"),
                        ("engine_f32_heading", "plain_f32_heading"),
                        ("engine_bf16_heading", "plain_f32_heading"),
                        ("engine_bf16_accel_in_view", "plain_f32_accel_in_view")):
            if k in batched and base in batched:
                batched[k]["vs_" + base] = round(batched[k]["value"] / batched[base]["value"], 3)
        if not args.no_served:
            served = {"workload": "320 streams asking at start, then Poisson arrivals 4/s (mean "
                                  "life 32 s), cap 256 live, mixed resolutions 640x480..3840x2160, "
                                  "windows 8..32, ACCEL on walkers that speed up, slow down and "
                                  f"turn (points in view), admission by a {args.serve_budget_gb} GB "
                                  f"budget; levels of {list(SERVE_LEVELS)} frames/s per stream, "
                                  f"{args.serve_seconds} s each, until p99 > {P99_BOUND_MS} ms",
                      "server_bf16": run_served(torch, mf, dev, args, pools16, torch.bfloat16),
                      "server_f32": run_served(torch, mf, dev, args, pools32, torch.float32),
                      "plain_f32": run_served(torch, mf, dev, args, pools32, torch.float32,
                                              plain=True)}
            served["server_bf16_vs_plain_f32"] = round(
                served["server_bf16"]["max_sustained_fps"] /
                max(1e-9, served["plain_f32"]["max_sustained_fps"]), 3)
        del pools32, pools16
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, args.cpu_seconds)
    s.close()
    if rank == 0:
        peak, kind = hbm_peak()
        achieved = frames * FRAME_BYTES / (map_ms / 1000.0) / 1e9
        traffic = profiled_traffic(frames, map_kernel_name(s1), args.workload)
        all_work = None
        if variants is not None:
            hv = variants["heading_f32"]
            a_ach = frames * FRAME_BYTES / (hv["launch_ms"] / 1000.0) / 1e9
            a_tr = profiled_traffic(frames, hv["kernel"], "heading")
            all_work = {"workload": workload_config(frames, "heading")["workload"],
                        "bound": "hbm", "kernel": hv["kernel"], "achieved": round(a_ach, 1),
                        "peak": peak, "peak_kind": kind, "unit": "GB/s",
                        "frac": round(a_ach / peak, 4), "traffic": a_tr,
                        "dram_frac": (round(a_tr / (hv["launch_ms"] / 1000.0) / 1e9 / peak, 4)
                                      if a_tr else None),
                        "launch_ms": hv["launch_ms"], "value": hv["value"], "unit_value": "frames/s"}
        rec = {
            "metric": METRIC, "value": round(value, 2), "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "pose_dtype": "f64", "data": "synthetic (seeded walker poses, ray-cast depth)",
            "config": workload_config(frames, args.workload),
            "mpx_per_s": round(value * WIDTH * HEIGHT / 1e6, 1),
            "step_hbm_gbs": round(value / world * FRAME_BYTES / 1e9, 1),
            "roofline": {"bound": "hbm", "kernel": map_kernel_name(s1), "achieved": round(achieved, 1),
                         "peak": peak, "peak_kind": kind, "unit": "GB/s",
                         "frac": round(achieved / peak, 4),
                         "traffic": traffic,
                         "dram_frac": (round(traffic / (map_ms / 1000.0) / 1e9 / peak, 4)
                                       if traffic else None),
                         "algorithmic_bytes_per_launch": frames * FRAME_BYTES,
                         "launch_ms": round(map_ms, 4)},
            "roofline_all_work": all_work,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "precision": prec, "variants": variants, "batched": batched, "served": served,
        }
        print(json.dumps(rec), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_leg(torch, mf, w, poses, depth, dev, args, dt, mode="accel", normalize="count"):
    """The default workload with another storage type, mode or normalisation."""
    frames = int(depth.shape[0])
    steps = max(10, min(args.steps, 100))
    Kh = np.ascontiguousarray(w.K())
    din = depth if dt == torch.float32 else depth.to(dt)
    M = torch.empty((frames, HEIGHT, WIDTH), dtype=dt, device=dev)
    G = torch.empty_like(M)
    info = torch.empty(frames * 64, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)
    s = mf.MotionFocusStream(WIDTH, HEIGHT, window=WINDOW, smooth_len=SMOOTH, device=dev,
                             cuda_stream=stream, time_kernels=True, depth_dtype=dt,
                             map_dtype=dt, mode=mode, normalize=normalize)
    h = s.handle

    def step():
        mf.mf_reset_stream(h)
        mf.mf_push_frames(h, frames, poses, din, Kh)
        assert mf.mf_get_maps(h, frames, M, G, info, None) == frames

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    s0 = s.stats()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    ev1.synchronize()
    s1 = s.stats()
    ms = ev0.elapsed_time(ev1) / steps
    map_ms = (s1.map_kernel_ms - s0.map_kernel_ms) / max(1, s1.map_launches - s0.map_launches)
    bpp = 3 * din.element_size()
    kernel = map_kernel_name(s1)
    s.close()
    return {"value": round(frames / (ms / 1000.0), 2), "unit": "frames/s", "steps": steps,
            "map_gbs": round(frames * WIDTH * HEIGHT * bpp / (map_ms / 1000.0) / 1e9, 1),
            "map_frac": round(frames * WIDTH * HEIGHT * bpp / (map_ms / 1000.0) / 1e9 / hbm_peak()[0], 4),
            "bytes_per_px": bpp, "kernel": kernel, "launch_ms": round(map_ms, 4)}


def run_precision(torch, mf, w, poses, depth, dev, args, f32_value):
    """The same workload with 16-bit depth and map storage (FP32 arithmetic)."""
    out = {}
    for name, dt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        out[name] = run_leg(torch, mf, w, poses, depth, dev, args, dt)
        out[name]["gain_vs_f32"] = round(out[name]["value"] / f32_value, 3)
    return out


def run_variants(torch, mf, w, poses, depth, dev, args, f32_value):
    """HEADING mode and ACCEL with Z = the map maximum on the default frames,
    and ACCEL on a walker that speeds up and slows down (points in view), in
    FP32."""
    frames = int(depth.shape[0])
    w2, poses2, depth2 = make_inputs(torch, dev, frames, "accel_in_view")
    out = {"heading_f32": run_leg(torch, mf, w, poses, depth, dev, args, torch.float32,
                                  mode="heading"),
           "norm_max_f32": run_leg(torch, mf, w, poses, depth, dev, args, torch.float32,
                                   normalize="max"),
           "accel_in_view_f32": run_leg(torch, mf, w2, poses2, depth2, dev, args, torch.float32)}
    del depth2
    out["accel_in_view_f32"]["workload"] = workload_config(frames, "accel_in_view")["workload"]
    for v in out.values():
        v["vs_default"] = round(v["value"] / f32_value, 3)
    return out


def run_e2e(torch, mf, w, depth_dev, dev, args):
    """Same metric through the C ABI with pinned host inputs and outputs."""
    FR = int(depth_dev.shape[0])
    depth_h = torch.empty((FR, HEIGHT, WIDTH), dtype=torch.float32, pin_memory=True)
    depth_h.copy_(depth_dev)
    M_h = torch.empty_like(depth_h, pin_memory=True)
    G_h = torch.empty_like(depth_h, pin_memory=True)
    info_h = np.empty(FR, dtype=mf._mf.FRAME_INFO_DTYPE)
    poses_h = np.ascontiguousarray(w.poses[:FR])
    Kh = np.ascontiguousarray(w.K())
    s = mf.MotionFocusStream(WIDTH, HEIGHT, window=WINDOW, smooth_len=SMOOTH, device=dev)
    h = s.handle

    t_push = [0.0]

    def step():
        t0 = time.perf_counter()
        mf.mf_reset_stream(h)
        mf.mf_push_frames(h, FR, poses_h, depth_h, Kh)
        t_push[0] += time.perf_counter() - t0
        assert mf.mf_get_maps(h, FR, M_h, G_h, info_h, None) == FR

    for _ in range(2):
        step()
    n = max(3, args.e2e_steps)
    t_push[0] = 0.0
    laps = []
    t0 = time.perf_counter()
    for _ in range(n):
        step()
        laps.append(time.perf_counter())
    dt = time.perf_counter() - t0
    laps = np.diff([t0] + laps) * 1000.0
    s.close()
    h2d = FR * 96 + FR * WIDTH * HEIGHT * 4
    d2h = 2 * FR * WIDTH * HEIGHT * 4 + FR * 64
    return {"value": round(FR * n / dt, 2), "unit": "frames/s", "steps": n,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "host_link_gbs": round((h2d + d2h) * n / dt / 1e9, 1),
            "push_call_ms": round(1000 * t_push[0] / n, 2),
            "step_ms_min_median_max": [round(float(laps.min()), 2), round(float(np.median(laps)), 2),
                                       round(float(laps.max()), 2)],
            "path": "pinned host depth/maps; uploads and downloads on two copy streams in "
                    f"pieces of {PIECE_FRAMES} frames, overlapped with the map kernels"}


# ------------------------------------------------- batched and served --
MIX_RES = ((640, 480), (1280, 720), (1920, 1080), (3840, 2160))


def depth_pools(torch, dev, planes, dtype):
    """Per-resolution pools of ray-cast depth planes, shared read-only inputs."""
    from synth import hd_stream
    from synth.scene import render_depth
    w = hd_stream()
    pools = {}
    for width, height in MIX_RES:
        f = 0.9 * width
        intr = (f, f, width / 2.0, height / 2.0)
        imgs = [render_depth(w.boxes, w.traj.rot_c2w[(37 * k) % FRAMES],
                             w.traj.centres[(37 * k) % FRAMES], intr, width, height)
                for k in range(planes)]
        pools[(width, height)] = torch.from_numpy(np.stack(imgs)).to(dev).to(dtype)
    return pools


def run_batched(torch, mf, dev, args, pools, dtype, plain=False, mode="accel", accel=0.0):
    """64 mixed streams (640x480 .. 3840x2160, windows 8..32): every step
    pushes F frames of every stream; engine ticks or plain per-stream calls.
    ``accel`` > 0: walkers that also speed up and slow down."""
    from synth import mixed_streams
    F, n_streams = args.batch_frames, 64
    specs = mixed_streams(n_streams, cfg=4, accel=accel)
    steps, warm = args.batch_steps, 3
    need = (steps + warm) * F
    st = torch.cuda.Stream(dev)
    streams = []
    for sp in specs:
        P = sp.poses
        idx = np.arange(need) % len(P)
        streams.append(dict(
            w=sp.width, h=sp.height, win=sp.window, K=np.ascontiguousarray(sp.K()),
            poses=np.ascontiguousarray(P[idx]),
            M=torch.empty((F, sp.height, sp.width), dtype=dtype, device=dev),
            G=torch.empty((F, sp.height, sp.width), dtype=dtype, device=dev),
            info=torch.empty(F * 64, dtype=torch.uint8, device=dev),
            # every stream reads its own planes (a copy of the pool's), so
            # depth reads come from HBM as they would for distinct cameras
            depth=pools[(sp.width, sp.height)][:F].clone()))
    px = sum(s["w"] * s["h"] for s in streams) * F
    bpp = 3 * (4 if dtype == torch.float32 else 2)
    if plain:
        handles = []
        for s in streams:
            h = mf.MotionFocusStream(s["w"], s["h"], window=s["win"], smooth_len=SMOOTH, device=dev,
                                     mode=mode,
                                     cuda_stream=st, depth_dtype=dtype, map_dtype=dtype,
                                     max_pending=F)
            s["poses_dev"] = torch.from_numpy(s["poses"]).to(dev)
            handles.append(h)

        def step(k):
            for h, s in zip(handles, streams):
                mf.mf_push_frames(h.handle, F, s["poses_dev"][k * F:(k + 1) * F], s["depth"], s["K"])
                mf.mf_get_maps(h.handle, F, s["M"], s["G"], s["info"], None)
    else:
        eng = mf.MotionFocusEngine(max_streams=n_streams, max_tick_frames=n_streams * F,
                                   max_stream_frames=F, depth_dtype=dtype, map_dtype=dtype,
                                   device=dev, cuda_stream=st, tune=not args.no_tune)
        slots = [eng.add_stream(s["w"], s["h"], window=s["win"], smooth_len=SMOOTH, mode=mode)
                 for s in streams]
        rec = np.zeros(n_streams, dtype=mf.PUSH_DTYPE)
        rec["slot"] = slots
        rec["n"] = F
        rec["depth"] = [s["depth"].data_ptr() for s in streams]
        rec["K"] = [s["K"].ctypes.data for s in streams]
        rec["focus_map"] = [s["M"].data_ptr() for s in streams]
        rec["guided_depth"] = [s["G"].data_ptr() for s in streams]
        rec["info"] = [s["info"].data_ptr() for s in streams]
        pose_base = np.array([s["poses"].ctypes.data for s in streams], dtype=np.uint64)

        def step(k):
            rec["poses"] = pose_base + np.uint64(k * F * 96)
            mf.mf_engine_submit_batch(eng.handle, rec)
            eng.tick()
    for k in range(warm):
        step(k)
    st.synchronize()
    l0 = mf.mf_total_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record(st)
    for k in range(warm, warm + steps):
        step(k)
    ev1.record(st)
    ev1.synchronize()
    wall = time.perf_counter() - t0
    ms = ev0.elapsed_time(ev1)
    launches = mf.mf_total_kernel_launches() - l0
    frames = n_streams * F * steps
    out = {"value": round(frames / (ms / 1000.0), 1), "unit": "frames/s",
           "mpx_per_s": round(px * steps / (ms / 1000.0) / 1e6, 1),
           "hbm_gbs": round(px * steps * bpp / (ms / 1000.0) / 1e9, 1),
           "hbm_frac": round(px * steps * bpp / (ms / 1000.0) / 1e9 / hbm_peak()[0], 4),
           "ms_per_step": round(ms / steps, 3), "host_ms_per_step": round(1000 * wall / steps, 3),
           "frames_per_step": n_streams * F, "steps": steps, "kernel_launches_per_step": launches / steps}
    if not plain:
        est = eng.stats()
        out["graph_launches"] = int(est.graph_launches)
        eng.close()
    return out


SERVE_CAP = 256          # live streams at most (engine slots; the plain leg holds the same cap)
SERVE_R = 8              # planes per stream in the input pools and output rings
SERVE_LEVELS = (30, 60, 90, 120, 180, 240, 360, 480, 640, 800, 960, 1200)  # frames/s per stream
P99_BOUND_MS = 33.0      # the 30 FPS real-time bar as a per-frame latency bound


def serve_trajs():
    """Walkers that speed up and slow down (1.5 m/s^2) and turn, so ACCEL
    points land in view and every stream's maps are computed in full."""
    from synth import WalkerSpec, walk
    return [np.ascontiguousarray(walk(WalkerSpec(n_frames=900, seed=5100 + i, turns=True,
                                                 accel=1.5)).poses_w2c) for i in range(8)]


class ServeLeg:
    """One side of the served comparison, kept across the levels of the ramp:
    the continuous-batching server (one engine, native tick thread) or the
    plain per-stream path (one mf_stream per live stream, all on one CUDA
    stream, the caller's own loop).  Both are stamped the same way: a host
    function behind the GPU work records the completion time on
    mf_clock_ns()'s clock (the server's tick stamp; mf_probe_stamp for the
    plain path), and latency runs from each push's scheduled arrival."""

    def __init__(self, torch, mf, dev, args, pools, dtype, plain):
        self.torch, self.mf, self.dev, self.plain, self.dtype = torch, mf, dev, plain, dtype
        self.pools = pools
        self.esize = 4 if dtype == torch.float32 else 2
        self.budget = int(args.serve_budget_gb * 2 ** 30)
        self.st = torch.cuda.Stream(dev)
        self.rings = {}   # resolution -> free (M, G) output rings
        if plain:
            self.probe = mf._mf.mf_probe_open()
        else:
            self.srv = mf.MotionFocusServer(max_streams=SERVE_CAP, max_tick_frames=2048,
                                            max_stream_frames=SERVE_R, depth_dtype=dtype,
                                            map_dtype=dtype, memory_budget=self.budget,
                                            tick_us=args.tick_us, queue_limit=1024, device=dev)
            for width, height in MIX_RES:
                for win in (8, 16, 32):
                    self.srv.tune(width, height, win)
        self.reserved = 0
        self.open_streams = 0
        assert all(p.shape[0] >= SERVE_R for p in pools.values())

    def admit(self, s):
        """Admission: a free slot and room in the memory budget (the server
        decides by itself; the plain leg applies the same rule here)."""
        mf = self.mf
        plane = s["w"] * s["h"] * self.esize
        reserve = 2 * SERVE_R * plane
        if self.plain:
            if self.open_streams >= SERVE_CAP or self.reserved + reserve > self.budget:
                return False
            s["handle"] = mf.MotionFocusStream(s["w"], s["h"], window=s["win"], smooth_len=SMOOTH,
                                               device=self.dev, cuda_stream=self.st,
                                               depth_dtype=self.dtype, map_dtype=self.dtype,
                                               max_pending=SERVE_R)
            self.reserved += reserve
            self.open_streams += 1
        else:
            try:
                s["slot"] = self.srv.add_stream(s["w"], s["h"], window=s["win"], smooth_len=SMOOTH,
                                                reserve_bytes=reserve)
            except mf.MFError as e:
                if e.status == mf.MF_ERR_ADMISSION:
                    return False
                raise
        s["reserve"] = reserve
        free = self.rings.setdefault((s["w"], s["h"]), [])
        if free:
            s["M"], s["G"] = free.pop()
        else:
            s["M"] = self.torch.empty((SERVE_R, s["h"], s["w"]), dtype=self.dtype, device=self.dev)
            s["G"] = self.torch.empty_like(s["M"])
        s["plane"] = plane
        s["pool"] = self.pools[(s["w"], s["h"])].data_ptr()
        return True

    def done(self, s):
        """True once all the stream's pushed frames are complete on the GPU."""
        if self.plain:
            return s["event"] is not None and s["event"].query()
        return self.mf._mf.mf_server_frames_done(self.srv.handle, s["slot"]) >= s["sent"]

    def retire(self, s):
        if self.plain:
            s["handle"].close()
            self.reserved -= s["reserve"]
            self.open_streams -= 1
        else:
            self.srv.remove_stream(s["slot"])
        self.rings[(s["w"], s["h"])].append((s["M"], s["G"]))

    def finish(self, s):
        """The stream sent its last frame."""
        if self.plain:
            ev = self.torch.cuda.Event()
            ev.record(self.st)
            s["event"] = ev

    def submit(self, items, t0_ns):
        """items: (stream, n, first frame index, arrival s); returns how many
        of them were accepted (in order)."""
        mf = self.mf
        if not items:
            return 0
        if self.plain:
            arr = []
            for s, n, k, arrival in items:
                r = k % SERVE_R
                pk = (s["off"] + k) % 900
                h = s["handle"].handle
                mf.mf_push_frames(h, n, s["traj"].ctypes.data + pk * 96, s["pool"] + r * s["plane"],
                                  s["K"])
                mf.mf_get_maps(h, n, s["M"].data_ptr() + r * s["plane"],
                               s["G"].data_ptr() + r * s["plane"], None, None)
                arr.extend([t0_ns + int(arrival * 1e9)] * n)
            mf._mf.mf_probe_stamp(self.probe, self.st.cuda_stream, np.array(arr, dtype=np.int64))
            return len(items)
        rec = np.zeros(len(items), dtype=mf.PUSH_DTYPE)
        for j, (s, n, k, arrival) in enumerate(items):
            r = k % SERVE_R
            pk = (s["off"] + k) % 900
            rec[j] = (s["slot"], n, s["traj"].ctypes.data + pk * 96, s["pool"] + r * s["plane"],
                      s["K"].ctypes.data, s["M"].data_ptr() + r * s["plane"],
                      s["G"].data_ptr() + r * s["plane"], 0, t0_ns + int(arrival * 1e9))
        acc = mf._mf.ctypes.c_int32()
        rc = mf._mf.lib.mf_server_submit_batch(self.srv.handle, len(rec), rec.ctypes.data,
                                               mf._mf.ctypes.byref(acc))
        if rc not in (mf.MF_OK, mf.MF_ERR_NOT_READY):
            raise mf.MFError(rc, "mf_server_submit_batch")
        return acc.value

    def drain(self):
        if self.plain:
            self.st.synchronize()
        else:
            self.srv.drain()

    def latency(self):
        if self.plain:
            return self.mf._mf.mf_probe_latency(self.probe, reset=True)
        return self.srv.latency(reset=True)

    def close(self):
        if self.plain:
            self.mf._mf.mf_probe_close(self.probe)
        else:
            self.srv.close()


def serve_level(leg, mf, fps, seconds, demand0, seed, trajs):
    """One level of the ramp: `demand0` streams ask for admission at t = 0
    (more than the cap, so admission refuses some), then Poisson arrivals at
    4/s; each live stream sends `fps` frames/s on its schedule (mean stream
    life 32 s; mixed resolutions; windows 8..32) for `seconds`; frames due
    together on one stream go out as one push.  After the window, every
    frame is waited for, so frames still queued count in the latency."""
    from synth import Xoshiro256ss
    rng = Xoshiro256ss(seed)

    def new_stream(t_start):
        width, height = rng.choice(MIX_RES)
        win = int(rng.uniform(8, 33))
        length = max(30, int(-math.log(1.0 - rng.uniform()) * 32.0 * fps))
        f = rng.uniform(0.7, 1.2) * width
        return dict(w=width, h=height, win=win, length=length,
                    K=np.ascontiguousarray([f, f, width / 2, height / 2], dtype=np.float64),
                    traj=trajs[int(rng.uniform(0, len(trajs)))], off=int(rng.uniform(0, 900)),
                    t0=t_start, sent=0, event=None)

    counts = {"refused": 0, "waited": 0, "admitted": 0, "max_live": 0}
    active, waiting, finished = [], [], []

    def try_admit(s, now):
        if len(active) < SERVE_CAP and leg.admit(s):
            s["t0"] = max(s["t0"], now)
            active.append(s)
            counts["admitted"] += 1
            counts["max_live"] = max(counts["max_live"], len(active))
            return True
        counts["refused"] += 1
        if not s.get("waited"):
            s["waited"] = True
            counts["waited"] += 1
        return False

    for _ in range(demand0):
        s = new_stream(0.0)
        if not try_admit(s, 0.0):
            waiting.append(s)
    leg.torch.cuda.synchronize(leg.dev)
    next_arrival = -math.log(1.0 - rng.uniform()) / 4.0
    frames = 0
    t0_ns = mf.mf_clock_ns()
    t_begin = time.perf_counter()
    freed = False
    while True:
        now = time.perf_counter() - t_begin
        if now >= seconds:
            break
        while next_arrival <= now:
            waiting.append(new_stream(next_arrival))
            next_arrival += -math.log(1.0 - rng.uniform()) / 4.0
        # waiting streams retry when a slot was freed, new ones on arrival
        if waiting:
            still = []
            for s in waiting:
                if (freed or "waited" not in s) and try_admit(s, now):
                    continue
                still.append(s)
            waiting = still
        freed = False
        items = []
        for s in active:
            due = min(s["length"], int((now - s["t0"]) * fps) + 1) - s["sent"]
            if due <= 0:
                continue
            k = s["sent"]
            n = min(due, SERVE_R - k % SERVE_R, 900 - (s["off"] + k) % 900)
            items.append((s, n, k, s["t0"] + k / fps))
        acc = leg.submit(items, t0_ns)
        for s, n, k, _ in items[:acc]:
            s["sent"] += n
            frames += n
        keep = []
        for s in active:
            if s["sent"] >= s["length"]:
                leg.finish(s)
                finished.append(s)
            else:
                keep.append(s)
        active = keep
        still = []
        for s in finished:
            if leg.done(s):
                leg.retire(s)
                freed = True
            else:
                still.append(s)
        finished = still
    t_sub = time.perf_counter() - t_begin
    leg.drain()
    wall = time.perf_counter() - t_begin
    lat = leg.latency()
    for s in active + finished:   # all complete after the drain
        leg.retire(s)
    return {"fps_per_stream": fps, "frames": frames, "seconds": round(wall, 3),
            "value": round(frames / wall, 1), "unit": "frames/s",
            "offered_per_s": round(frames / t_sub, 1),
            "p50_ms": round(lat.p50_ms, 3), "p99_ms": round(lat.p99_ms, 3),
            "max_ms": round(lat.max_ms, 3), "latency_frames": int(lat.frames),
            "admitted": counts["admitted"], "max_live": counts["max_live"],
            "refused_admissions": counts["refused"], "streams_waited": counts["waited"],
            "sustained": bool(lat.p99_ms <= P99_BOUND_MS and lat.frames == frames)}


def run_served(torch, mf, dev, args, pools, dtype, plain=False):
    """Load ramp of the served form and of the plain per-stream path: levels
    of SERVE_LEVELS frames/s per stream, up to 256 live streams of the mixed
    resolutions (320 asking at the start), admission by a memory budget.
    The first level (30 fps) is the served workload itself; later levels
    raise the per-stream rate until p99 exceeds 33 ms.  Reports every level
    and the highest sustained frames/s (p99 <= 33 ms)."""
    trajs = serve_trajs()
    leg = ServeLeg(torch, mf, dev, args, pools, dtype, plain)
    levels, best = [], None
    try:
        for i, fps in enumerate(SERVE_LEVELS):
            lv = serve_level(leg, mf, fps, args.serve_seconds, 320, 5150 + i, trajs)
            levels.append(lv)
            if lv["sustained"]:
                best = lv
            else:
                break
    finally:
        leg.close()
    base = levels[0]
    out = {k: base[k] for k in ("p50_ms", "p99_ms", "max_ms", "value", "frames", "admitted",
                                "max_live", "refused_admissions", "streams_waited")}
    out.update({"unit": "frames/s",
                "latency": "scheduled frame arrival (per-stream fps schedule) -> GPU completion "
                           "stamped natively by a host function behind the work (server: its "
                           "tick; plain: mf_probe_stamp after each loop pass)",
                "max_sustained_fps": best["value"] if best else 0.0,
                "max_sustained_level_fps_per_stream": best["fps_per_stream"] if best else None,
                "levels": levels})
    return out


# ------------------------------------------------------------- CPU oracle --
# The oracle (test infrastructure, timed here as the CPU baseline) runs in a
# pool of worker processes started with "spawn", one per host core, each
# single-threaded: every worker renders whole rows of one frame (its motion
# points, the direct per-pixel Eq. 7 and the guided depth) and the rows of a
# frame are split evenly across the workers.
_ORACLE = {}


def _oracle_worker_init(accel):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import oracle as O
    from synth import hd_stream
    w = hd_stream(accel=accel)
    for k in range(w.ring):          # the depth ring is rendered before any timing
        w.depth(k)
    ref = O.OracleStream(O.Params(WIDTH, HEIGHT, window=WINDOW, smooth_len=SMOOTH))
    ref.push(w.poses, None, w.K())
    _ORACLE.update(O=O, w=w, ref=ref)


def _oracle_rows(task):
    """Motion points of frame n, then M and G over rows y0..y1-1."""
    n, y0, y1 = task
    O, w, ref = _ORACLE["O"], _ORACLE["w"], _ORACLE["ref"]
    pts = ref.points(n)
    ys = np.arange(y0, y1)
    yy = np.repeat(ys, WIDTH)
    xx = np.tile(np.arange(WIDTH), len(ys))
    M = O.focus_map(pts, WIDTH, HEIGHT, xx, yy)
    D = w.depth(n)[y0:y1, :].reshape(-1)
    O.guided_depth(M, D, 1.0)
    return y1 - y0


class OraclePool:
    """Worker processes over the host cores (spawn: safe after CUDA calls)."""

    def __init__(self, workers=None):
        import multiprocessing as mp
        self.workers = workers or os.cpu_count() or 1
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_oracle_worker_init,
                                                 initargs=(0.0,))
        # every worker builds its workload and renders its depth ring once
        # before any timing
        self.pool.map(_oracle_rows, [(450 + (k % 8), 0, 1) for k in range(4 * self.workers)])

    def frames(self, frames, rows):
        """Rows 0..rows-1 of every frame in `frames`, rows split across the
        workers; returns (frames credited, seconds)."""
        tasks = []
        per = max(1, -(-rows // self.workers))
        for n in frames:
            for y0 in range(0, rows, per):
                tasks.append((n, y0, min(rows, y0 + per)))
        t0 = time.perf_counter()
        done = sum(self.pool.map(_oracle_rows, tasks, chunksize=1))
        dt = time.perf_counter() - t0
        return done / HEIGHT, dt

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(w, seconds):
    pool = OraclePool()
    try:
        # calibrate on one frame per worker, then size the sample to ~`seconds`
        cred, dt = pool.frames(list(range(450 - pool.workers, 450)), HEIGHT)
        nframes = max(1, min(900 - 450, int(seconds * cred / dt)))
        frames = list(range(450, 450 + nframes))
        cred, dt = pool.frames(frames, HEIGHT)
    finally:
        pool.close()
    return {"value": round(cred / dt, 4), "unit": "frames/s", "cores": pool.workers, "kind": "oracle",
            "sample": f"{nframes} full 1920x1080 frames ({frames[0]}..{frames[-1]}) of the "
                      f"900-frame workload, FP64 numpy oracle, rows split over {pool.workers} "
                      f"single-threaded worker processes, {dt:.1f} s",
            "host": host_cpu(pool.workers)}


def host_cpu(threads=1):
    """CPU of the host the oracle ran on (model name when the OS reports it)."""
    import platform
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":")[0].strip().lower()
                if k in ("model name", "cpu part", "hardware"):
                    model = f"{platform.machine()} {ln.split(':', 1)[1].strip()}"
                    break
    except OSError:
        pass
    return {"model": model, "nproc": os.cpu_count(), "threads_used": threads}


def run_reference(args):
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    if rank != 0:
        return
    pool = OraclePool()
    try:
        budget = 150.0 / max(1, args.steps + args.warmup)
        cred, dt = pool.frames([450], 64)
        rows = int(max(pool.workers, min(HEIGHT, budget * cred / dt * HEIGHT)))
        for k in range(args.warmup):
            pool.frames([450 + k % 400], rows)
        credited, dt = 0.0, 0.0
        for k in range(args.steps):
            c, t = pool.frames([450 + k % 400], rows)
            credited += c
            dt += t
    finally:
        pool.close()
    value = credited / dt
    rec = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "frames/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1000 * dt / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(),
           "cpu_baseline": {"value": round(value, 5), "unit": "frames/s", "cores": pool.workers,
                            "kind": "oracle",
                            "sample": f"per step: one frame's motion points + {rows} of 1080 "
                                      f"map rows (credited as that fraction of a frame), rows "
                                      f"split over {pool.workers} worker processes"},
           "e2e": {"value": round(value, 5), "unit": "frames/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(rec), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the HEADING / Z=max legs")
    ap.add_argument("--map-kernel", default="auto", choices=["auto", "cuda_cores", "tensor_cores"],
                    help="map kernel of the default line (auto: the library's choice)")
    ap.add_argument("--no-serving", action="store_true", help="skip the batched and served legs")
    ap.add_argument("--no-served", action="store_true", help="skip the served leg")
    ap.add_argument("--no-tune", action="store_true", help="engine legs use the plain tile height")
    ap.add_argument("--batch-frames", type=int, default=8)
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--serve-seconds", type=float, default=2.5)
    ap.add_argument("--serve-budget-gb", type=float, default=32.0)
    ap.add_argument("--tick-us", type=int, default=200)
    ap.add_argument("--workload", default="default", choices=sorted(WORKLOADS),
                    help="frames of the 1080p line (default: the ACCEL config-2 walker; the others "
                         "only for profiling captures)")
    ap.add_argument("--batch-legs", default="all",
                    help="comma list of batched legs to run (default all; for profiling captures)")
    ap.add_argument("--frames", type=int, default=FRAMES,
                    help="frames per step (default: the full 900-frame workload; "
                         "smaller values only for profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
