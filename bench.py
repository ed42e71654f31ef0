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
    "map_stream_kernel": ("map_kernel_1080p_f32.txt", ("mf_map_kernel.cu", "mf_map_unit.cuh")),
    "map_tc_kernel": ("map_tc_kernel_1080p_f32.txt", ("mf_map_tc.cu", "mf_map_unit.cuh")),
}


PIECE_FRAMES = max(1, min(64, (128 << 20) // (12 * WIDTH * HEIGHT)))  # library transfer piece


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def workload_config(frames=FRAMES):
    return {"workload": f"1 stream, {frames} frames 1920x1080, window 16, K=15 fit, ACCEL, "
                        "FP32 depth+maps, walker with turns, ray-cast box scene",
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


def map_source_hash(kernel):
    h = hashlib.sha256()
    for f in PROFILES[kernel][1]:
        path = os.path.join(ROOT, "paper_2601_07154_gb300", "csrc", f)
        if os.path.exists(path):
            h.update(open(path, "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(frames, kernel):
    """DRAM bytes per launch from the committed ncu summary of `kernel`, if
    the summary was taken from the current sources."""
    if kernel not in PROFILES:
        return None
    try:
        text = open(os.path.join(ROOT, "profiles", PROFILES[kernel][0])).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256_16") != map_source_hash(kernel):
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
def make_inputs(torch, dev, frames):
    from synth import hd_stream
    w = hd_stream()
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
    w, poses, depth = make_inputs(torch, dev, frames)
    K = w.K()
    M = torch.empty((frames, HEIGHT, WIDTH), dtype=torch.float32, device=dev)
    G = torch.empty_like(M)
    info = torch.empty(frames * 64, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)
    s = mf.MotionFocusStream(WIDTH, HEIGHT, window=WINDOW, smooth_len=SMOOTH, device=dev,
                             cuda_stream=stream, time_kernels=True, map_kernel=args.map_kernel)
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
    batched = served = None
    if rank == 0 and not args.no_serving:
        del M, G
        M = G = None
        pools32 = depth_pools(torch, dev, args.batch_frames, torch.float32)
        pools16 = {k: v.to(torch.bfloat16) for k, v in pools32.items()}
        batched = {"workload": "64 streams, resolutions 640x480..3840x2160, windows 8..32, "
                               f"{args.batch_frames} frames per stream per step, own depth "
                               "planes per stream",
                   "engine_f32": run_batched(torch, mf, dev, args, pools32, torch.float32),
                   "engine_bf16": run_batched(torch, mf, dev, args, pools16, torch.bfloat16),
                   "plain_f32": run_batched(torch, mf, dev, args, pools32, torch.float32, plain=True),
                   # HEADING keeps the motion points in view, so every unit computes and
                   # reads depth (the ACCEL walkers' points mostly leave the images)
                   "engine_f32_heading": run_batched(torch, mf, dev, args, pools32, torch.float32,
                                                     mode="heading"),
                   "engine_bf16_heading": run_batched(torch, mf, dev, args, pools16, torch.bfloat16,
                                                      mode="heading"),
                   "plain_f32_heading": run_batched(torch, mf, dev, args, pools32, torch.float32,
                                                    plain=True, mode="heading")}
        for k in ("engine_f32", "engine_bf16"):
            batched[k]["vs_plain_f32"] = round(batched[k]["value"] / batched["plain_f32"]["value"], 3)
            batched[k + "_heading"]["vs_plain_f32"] = round(
                batched[k + "_heading"]["value"] / batched["plain_f32_heading"]["value"], 3)
        if not args.no_served:
            served = {"workload": "Poisson arrivals 4/s of 30 fps streams (mean 32 s), 128 live "
                                  "at start, cap 256, mixed resolutions, admission by memory "
                                  f"budget {args.serve_budget_gb} GB",
                      "server_bf16": run_served(torch, mf, dev, args, pools16, torch.bfloat16),
                      "server_f32": run_served(torch, mf, dev, args, pools32, torch.float32),
                      "plain_f32": run_served(torch, mf, dev, args, pools32, torch.float32,
                                              plain=True)}
        del pools32, pools16
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, args.cpu_seconds)
    s.close()
    if rank == 0:
        peak, kind = hbm_peak()
        achieved = frames * FRAME_BYTES / (map_ms / 1000.0) / 1e9
        traffic = profiled_traffic(frames, map_kernel_name(s1))
        rec = {
            "metric": METRIC, "value": round(value, 2), "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "pose_dtype": "f64", "data": "synthetic (seeded walker poses, ray-cast depth)",
            "config": workload_config(frames),
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
    s.close()
    return {"value": round(frames / (ms / 1000.0), 2), "unit": "frames/s", "steps": steps,
            "map_gbs": round(frames * WIDTH * HEIGHT * bpp / (map_ms / 1000.0) / 1e9, 1),
            "bytes_per_px": bpp}


def run_precision(torch, mf, w, poses, depth, dev, args, f32_value):
    """The same workload with 16-bit depth and map storage (FP32 arithmetic)."""
    out = {}
    for name, dt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        out[name] = run_leg(torch, mf, w, poses, depth, dev, args, dt)
        out[name]["gain_vs_f32"] = round(out[name]["value"] / f32_value, 3)
    return out


def run_variants(torch, mf, w, poses, depth, dev, args, f32_value):
    """HEADING mode, and ACCEL with Z = the map maximum (an extra in-place pass
    over both maps), on the default workload in FP32."""
    out = {"heading_f32": run_leg(torch, mf, w, poses, depth, dev, args, torch.float32,
                                  mode="heading"),
           "norm_max_f32": run_leg(torch, mf, w, poses, depth, dev, args, torch.float32,
                                   normalize="max")}
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


def run_batched(torch, mf, dev, args, pools, dtype, plain=False, mode="accel"):
    """64 mixed streams (640x480 .. 3840x2160, windows 8..32): every step
    pushes F frames of every stream; engine ticks or plain per-stream calls."""
    from synth import mixed_streams
    F, n_streams = args.batch_frames, 64
    specs = mixed_streams(n_streams, cfg=4)
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
           "ms_per_step": round(ms / steps, 3), "host_ms_per_step": round(1000 * wall / steps, 3),
           "frames_per_step": n_streams * F, "steps": steps, "kernel_launches_per_step": launches / steps}
    if not plain:
        est = eng.stats()
        out["graph_launches"] = int(est.graph_launches)
        eng.close()
    return out


def run_served(torch, mf, dev, args, pools, dtype, plain=False):
    """Poisson arrivals (4/s) of 30 fps streams (mean 32 s, resolutions of the
    mixed workload), 128 live at the start, up to 256; admission by memory.

    Every frame arrives on its stream's 30 fps schedule; latency runs from
    that arrival time to the GPU completion of the frame (native stamp for
    the server; host-observed event for the plain per-stream path).  The
    expected resolution classes are tuned and the first 128 streams admitted
    before the clock starts, as a deployment would warm up.
    """
    from synth import Xoshiro256ss, WalkerSpec, walk
    rng = Xoshiro256ss(5150)
    duration = args.serve_seconds if not plain else min(args.serve_seconds, 6.0)
    trajs = [np.ascontiguousarray(walk(WalkerSpec(n_frames=900, seed=5100 + i, turns=True)).poses_w2c)
             for i in range(8)]
    R = 8
    esize = 4 if dtype == torch.float32 else 2
    budget = int(args.serve_budget_gb * 2 ** 30)
    st = torch.cuda.Stream(dev)
    if not plain:
        srv = mf.MotionFocusServer(max_streams=256, max_tick_frames=1024, max_stream_frames=4,
                                   depth_dtype=dtype, map_dtype=dtype, memory_budget=budget,
                                   tick_us=args.tick_us, device=dev)
        for width, height in MIX_RES:
            for win in (8, 16, 32):
                srv.tune(width, height, win)
    rings = {}   # resolution -> free (M, G) output rings of the clients

    def new_stream(t_start):
        width, height = rng.choice(MIX_RES)
        win = int(rng.uniform(8, 33))
        length = max(30, int(-math.log(1.0 - rng.uniform()) * 32.0 * 30))
        f = rng.uniform(0.7, 1.2) * width
        return dict(w=width, h=height, win=win, length=length,
                    K=np.ascontiguousarray([f, f, width / 2, height / 2], dtype=np.float64),
                    traj=trajs[int(rng.uniform(0, len(trajs)))], off=int(rng.uniform(0, 900)),
                    t0=t_start, sent=0)

    counters = {"refused": 0, "admitted": 0}

    def admit(s, now):
        plane = s["w"] * s["h"] * esize
        try:
            if plain:
                s["handle"] = mf.MotionFocusStream(s["w"], s["h"], window=s["win"], smooth_len=SMOOTH,
                                                   device=dev, cuda_stream=st, depth_dtype=dtype,
                                                   map_dtype=dtype, max_pending=R)
            else:
                s["slot"] = srv.add_stream(s["w"], s["h"], window=s["win"], smooth_len=SMOOTH,
                                           reserve_bytes=2 * R * plane)
        except mf.MFError as e:
            if e.status == mf.MF_ERR_ADMISSION:
                counters["refused"] += 1
                return False
            raise
        free = rings.setdefault((s["w"], s["h"]), [])
        if free:
            s["M"], s["G"] = free.pop()
        else:
            s["M"] = torch.empty((R, s["h"], s["w"]), dtype=dtype, device=dev)
            s["G"] = torch.empty_like(s["M"])
        s["plane"] = plane
        s["pool"] = pools[(s["w"], s["h"])]
        s["t0"] = max(s["t0"], now)
        counters["admitted"] += 1
        return True

    def retire(s):
        if plain:
            s["handle"].close()
        else:
            srv.remove_stream(s["slot"])
        rings[(s["w"], s["h"])].append((s["M"], s["G"]))

    active = [s for s in (new_stream(0.0) for _ in range(128)) if admit(s, 0.0)]
    waiting, lags, lat_plain, pending_events, done = [], [], [], [], []
    torch.cuda.synchronize(dev)
    next_arrival = -math.log(1.0 - rng.uniform()) / 4.0
    served = 0
    t0_ns = mf.mf_clock_ns()
    t_begin = time.perf_counter()
    while True:
        now = time.perf_counter() - t_begin
        if now >= duration:
            break
        while next_arrival <= now:
            waiting.append(new_stream(next_arrival))
            next_arrival += -math.log(1.0 - rng.uniform()) / 4.0
        if waiting:
            still = []
            for s in waiting:
                if len(active) < 256 and admit(s, now):
                    active.append(s)
                else:
                    still.append(s)
            waiting = still
        keep, batch = [], []
        for s in active:
            due = min(s["length"], int((now - s["t0"]) * 30.0) + 1)
            while s["sent"] < due:
                k = s["sent"]
                r = k % R
                pk = (s["off"] + k) % 900
                if plain:
                    mf.mf_push_frames(s["handle"].handle, 1, s["traj"][pk][None], s["pool"][r], s["K"])
                    mf.mf_get_maps(s["handle"].handle, 1, s["M"][r], s["G"][r], None, None)
                    ev = torch.cuda.Event()
                    ev.record(st)
                    pending_events.append((ev, s["t0"] + k / 30.0))
                else:
                    batch.append((s["slot"], 1, s["traj"].ctypes.data + pk * 96,
                                  s["pool"].data_ptr() + r * s["plane"], s["K"].ctypes.data,
                                  s["M"].data_ptr() + r * s["plane"], s["G"].data_ptr() + r * s["plane"],
                                  0, t0_ns + int((s["t0"] + k / 30.0) * 1e9)))
                lags.append(now - (s["t0"] + k / 30.0))
                s["sent"] += 1
                served += 1
            (done if s["sent"] >= s["length"] else keep).append(s)
        active = keep
        if batch:
            mf.mf_server_submit_batch(srv.handle, np.array(batch, dtype=mf.PUSH_DTYPE))
        for s in done:
            retire(s)
        done.clear()
        if plain:
            while pending_events and pending_events[0][0].query():
                ev, due_t = pending_events.pop(0)
                lat_plain.append(1000.0 * (time.perf_counter() - t_begin - due_t))
    if plain:
        st.synchronize()
        for ev, due_t in pending_events:
            lat_plain.append(1000.0 * (time.perf_counter() - t_begin - due_t))
        lat = np.array(lat_plain)
        out = {"p50_ms": round(float(np.percentile(lat, 50)), 3),
               "p90_ms": round(float(np.percentile(lat, 90)), 3),
               "p99_ms": round(float(np.percentile(lat, 99)), 3),
               "max_ms": round(float(lat.max()), 3),
               "latency": "frame arrival (30 fps schedule) -> completion observed by the host"}
        for s in active:
            s["handle"].close()
    else:
        srv.drain()
        lat = srv.latency()
        est = srv.stats()
        out = {"p50_ms": round(lat.p50_ms, 3), "p90_ms": round(lat.p90_ms, 3),
               "p99_ms": round(lat.p99_ms, 3), "max_ms": round(lat.max_ms, 3),
               "latency": "frame arrival (30 fps schedule) -> GPU completion of its tick (native)",
               "ticks": int(est.ticks), "frames_per_tick": round(est.frames / max(1, est.ticks), 2)}
        for s in active:
            srv.remove_stream(s["slot"])
        srv.close()
    wall = time.perf_counter() - t_begin
    lagv = np.array(lags) * 1000.0
    out.update({"frames": served, "seconds": round(wall, 2), "value": round(served / wall, 1),
                "unit": "frames/s", "admitted": counters["admitted"],
                "refused_admissions": counters["refused"], "live_streams_end": len(active),
                "submit_lag_p99_ms": round(float(np.percentile(lagv, 99)), 3)})
    return out


# ------------------------------------------------------------- CPU oracle --
def oracle_sample(w, frames, rows):
    """Oracle frames/s on frames (full pose path) x rows of their maps."""
    import oracle as O
    p = O.Params(WIDTH, HEIGHT, window=WINDOW, smooth_len=SMOOTH)
    ref = O.OracleStream(p)
    ref.push(w.poses, None, w.K())
    ys_all = np.arange(HEIGHT)
    t0 = time.perf_counter()
    for n in frames:
        pts = ref.points(n)
        ys = ys_all[rows]
        yy = np.repeat(ys, WIDTH)
        xx = np.tile(np.arange(WIDTH), len(ys))
        M = O.focus_map(pts, WIDTH, HEIGHT, xx, yy)
        D = w.depth(n)[ys, :].reshape(-1)
        O.guided_depth(M, D, 1.0)
    dt = time.perf_counter() - t0
    credited = len(frames) * (len(range(HEIGHT)[rows]) / HEIGHT)
    return credited / dt, dt


def cpu_baseline(w, seconds):
    # calibrate on a 64-row band, then size the sample to ~`seconds`
    rate, dt = oracle_sample(w, [450], slice(0, 64))
    nframes = max(1, min(16, int(seconds * rate)))
    frames = list(range(450, 450 + nframes))
    rate, dt = oracle_sample(w, frames, slice(0, HEIGHT))
    return {"value": round(rate, 4), "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": f"{nframes} full 1920x1080 frames ({frames[0]}..{frames[-1]}) of the "
                      f"900-frame workload, FP64 numpy oracle, {dt:.1f} s",
            "host": host_cpu()}


def host_cpu():
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
    return {"model": model, "nproc": os.cpu_count(), "threads_used": 1}


def run_reference(args):
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    if rank != 0:
        return
    from synth import hd_stream
    w = hd_stream()
    budget = 150.0 / max(1, args.steps + args.warmup)
    rate0, _ = oracle_sample(w, [450], slice(0, 16))
    rows = int(max(1, min(HEIGHT, budget * rate0 * HEIGHT)))
    for k in range(args.warmup):
        oracle_sample(w, [450 + k % 400], slice(0, rows))
    t0 = time.perf_counter()
    credited = 0.0
    for k in range(args.steps):
        _, _ = oracle_sample(w, [450 + k % 400], slice(0, rows))
        credited += rows / HEIGHT
    dt = time.perf_counter() - t0
    value = credited / dt
    rec = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "frames/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1000 * dt / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(),
           "cpu_baseline": {"value": round(value, 5), "unit": "frames/s", "cores": 1,
                            "kind": "oracle",
                            "sample": f"per step: one frame's motion points + {rows} of 1080 "
                                      "map rows (credited as that fraction of a frame)"},
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
    ap.add_argument("--serve-seconds", type=float, default=12.0)
    ap.add_argument("--serve-budget-gb", type=float, default=32.0)
    ap.add_argument("--tick-us", type=int, default=200)
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
