"""Torch-facing wrapper of one libmf stream (allocation and marshalling only).

PyTorch supplies device memory (optionally through its caching allocator)
and the CUDA stream; every computation is a libmf kernel launched through
the C ABI.
"""
import numpy as np
import torch

from . import _mf

_DT = {torch.float32: _mf.MF_F32, torch.bfloat16: _mf.MF_BF16, torch.float16: _mf.MF_F16}
_NORMS = {"count": _mf.MF_NORM_COUNT, "max": _mf.MF_NORM_MAX}
_MAP_KERNELS = {"auto": 0, "cuda_cores": _mf.MF_FLAG_MAP_CUDA_CORES,
                "tensor_cores": _mf.MF_FLAG_MAP_TENSOR_CORES}
_MODES = {"accel": _mf.MF_MODE_ACCEL, "heading": _mf.MF_MODE_HEADING}
_FRAMES = {"world": _mf.MF_POSES_WORLD, "batch_local": _mf.MF_POSES_BATCH_LOCAL}


class MotionFocusStream:
    """One video stream: push pose/depth batches, get maps back.

    Maps come back as (n, height, width) tensors of ``map_dtype`` on the
    stream's device, with per-frame info and motion points as numpy
    structured arrays (layouts of ``mf_frame_info`` / ``mf_motion_point``).
    ``normalize`` picks Z of Eq. 7: "count" (the number of valid points) or
    "max" (the frame's map maximum, so that every non-empty map peaks at 1).
    ``map_kernel`` picks the CUDA-core ("cuda_cores", also what "auto"
    runs) or the tensor-core ("tensor_cores") map kernel.
    """

    def __init__(self, width, height, window=8, smooth_len=15, mode="accel",
                 pose_frame="world", overlap=0, depth_dtype=torch.float32,
                 map_dtype=torch.float32, calib=None, sigma_rel=0.1, s_lo=0.25, s_hi=4.0,
                 depth_ref_m=1.0, max_pending=1024, device=None, cuda_stream=None,
                 time_kernels=False, torch_allocator=True, normalize="count", map_kernel="auto",
                 depth_align=False):
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.width, self.height, self.window = int(width), int(height), int(window)
        self.map_dtype = map_dtype
        self.depth_dtype = depth_dtype
        with torch.cuda.device(self.device):
            self.torch_stream = cuda_stream or torch.cuda.current_stream(self.device)
            cw, ch = calib if calib is not None else (0, 0)
            fields = dict(width=self.width, height=self.height, calib_width=cw,
                          calib_height=ch, window=self.window, smooth_len=int(smooth_len),
                          mode=_MODES[mode], pose_frame=_FRAMES[pose_frame],
                          overlap=int(overlap), depth_dtype=_DT[depth_dtype],
                          map_dtype=_DT[map_dtype], max_pending=int(max_pending),
                          flags=(_mf.MF_FLAG_TIME_KERNELS if time_kernels else 0)
                          | _MAP_KERNELS[map_kernel]
                          | (_mf.MF_FLAG_DEPTH_ALIGN if depth_align else 0),
                          normalize=_NORMS[normalize],
                          sigma_rel=sigma_rel, s_lo=s_lo, s_hi=s_hi, depth_ref_m=depth_ref_m,
                          # torch's default stream has handle 0, which the ABI
                          # reads as "library-owned stream": pass the runtime's
                          # cudaStreamLegacy handle (0x1) for it instead
                          cuda_stream=self.torch_stream.cuda_stream or 1)
            self._cb = None
            if torch_allocator:
                dev, st = self.device, self.torch_stream

                def _alloc(nbytes, ctx):
                    try:
                        return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                    except RuntimeError:
                        return None

                def _free(p, ctx):
                    torch.cuda.caching_allocator_delete(p)

                self._cb = (_mf.ALLOC_FN(_alloc), _mf.FREE_FN(_free))
                fields.update(dev_alloc=self._cb[0], dev_free=self._cb[1])
            self.desc = _mf.mf_stream_desc_init(**fields)
            self.handle = _mf.mf_open_stream(self.desc)

    # -- ingestion ----------------------------------------------------------
    def push(self, poses, depth, K):
        """poses (n,3,4) or (n,12) FP64; depth (n,H,W) of depth_dtype or None;
        K = (fx, fy, cx, cy).  Tensors may live on the host or the device."""
        n = int(poses.shape[0])
        if isinstance(poses, torch.Tensor):
            assert poses.dtype == torch.float64 and poses.is_contiguous()
        else:
            poses = np.ascontiguousarray(poses, dtype=np.float64)
        if depth is not None:
            if isinstance(depth, torch.Tensor):
                assert depth.dtype == self.depth_dtype and depth.is_contiguous()
                assert tuple(depth.shape[1:]) == (self.height, self.width)
            else:
                depth = np.ascontiguousarray(depth)
        Kh = np.ascontiguousarray(np.asarray(K, dtype=np.float64).reshape(4))
        with torch.cuda.device(self.device):
            _mf.mf_push_frames(self.handle, n, poses, depth, Kh)
        self._keep = (poses, depth)  # device inputs must outlive their use

    def pending(self):
        return _mf.mf_pending_frames(self.handle)

    # -- results ------------------------------------------------------------
    def get_maps(self, max_frames=None, want_maps=True, want_points=True, out=None,
                 timeout_ns=-1):
        """Render pending frames; returns (M, G, info, points) for n frames."""
        n = self.pending() if max_frames is None else min(int(max_frames), self.pending())
        if n == 0:
            return None, None, np.zeros(0, _mf.FRAME_INFO_DTYPE), None
        if out is not None:
            M, G = out
        elif want_maps:
            M = torch.empty((n, self.height, self.width), dtype=self.map_dtype, device=self.device)
            G = torch.empty_like(M)
        else:
            M = G = None
        info = torch.empty(n * _mf.FRAME_INFO_DTYPE.itemsize, dtype=torch.uint8, device=self.device)
        pts = (torch.empty(n * self.window * _mf.MOTION_POINT_DTYPE.itemsize, dtype=torch.uint8,
                           device=self.device) if want_points else None)
        with torch.cuda.device(self.device):
            got = _mf.mf_get_maps(self.handle, n, M, G, info, pts, timeout_ns=timeout_ns)
        assert got == n
        self.torch_stream.synchronize()
        info_np = info.cpu().numpy().view(_mf.FRAME_INFO_DTYPE)
        pts_np = (pts.cpu().numpy().view(_mf.MOTION_POINT_DTYPE).reshape(n, self.window)
                  if pts is not None else None)
        return M, G, info_np, pts_np

    def snapshot(self):
        """Resident state as bytes (no pending frames): window history, frame
        counters, depth alignment state."""
        with torch.cuda.device(self.device):
            return _mf.mf_stream_snapshot(self.handle)

    def restore(self, blob):
        """Load a snapshot taken from a stream with the same options (this
        stream must not have taken a push yet, or must be reset)."""
        with torch.cuda.device(self.device):
            _mf.mf_stream_restore(self.handle, blob)

    def sync(self, timeout_ns=-1):
        _mf.mf_sync(self.handle, timeout_ns)

    def reset(self):
        _mf.mf_reset_stream(self.handle)

    def stats(self):
        return _mf.mf_stream_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            with torch.cuda.device(self.device):
                _mf.mf_close_stream(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MotionFocusEngine:
    """Many streams processed in batched ticks (the C ABI's mf_engine_*).

    ``add_stream`` admits a stream (its pose history lives on the GPU);
    ``submit`` queues one push of a stream with the device planes its maps
    go to; ``tick`` launches everything queued as one batch (a CUDA graph)
    without waiting.
    """

    def __init__(self, max_streams=256, max_tick_frames=4096, max_stream_frames=64,
                 depth_dtype=torch.float32, map_dtype=torch.float32, memory_budget=0,
                 graph=True, tune=True, time_kernels=False, device=None, cuda_stream=None):
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.depth_dtype, self.map_dtype = depth_dtype, map_dtype
        flags = 0 if graph else _mf.MF_ENGINE_NO_GRAPH
        flags |= 0 if tune else _mf.MF_ENGINE_NO_TUNE
        flags |= _mf.MF_FLAG_TIME_KERNELS if time_kernels else 0
        with torch.cuda.device(self.device):
            self.torch_stream = cuda_stream or torch.cuda.current_stream(self.device)
            self.desc = _mf.mf_engine_desc_init(
                max_streams=max_streams, max_tick_frames=max_tick_frames,
                max_stream_frames=max_stream_frames, depth_dtype=_DT[depth_dtype],
                map_dtype=_DT[map_dtype], flags=flags, memory_budget=int(memory_budget),
                cuda_stream=self.torch_stream.cuda_stream or 1)
            self.handle = _mf.mf_engine_open(self.desc)
        self.streams = {}

    def add_stream(self, width, height, window=8, smooth_len=15, mode="accel",
                   pose_frame="world", overlap=0, calib=None, reserve_bytes=0, sigma_rel=0.1,
                   s_lo=0.25, s_hi=4.0, depth_ref_m=1.0):
        cw, ch = calib if calib is not None else (0, 0)
        d = _mf.mf_stream_desc_init(
            width=int(width), height=int(height), calib_width=cw, calib_height=ch,
            window=int(window), smooth_len=int(smooth_len), mode=_MODES[mode],
            pose_frame=_FRAMES[pose_frame], overlap=int(overlap),
            depth_dtype=_DT[self.depth_dtype], map_dtype=_DT[self.map_dtype],
            sigma_rel=sigma_rel, s_lo=s_lo, s_hi=s_hi, depth_ref_m=depth_ref_m)
        with torch.cuda.device(self.device):
            slot = _mf.mf_engine_add_stream(self.handle, d, reserve_bytes)
        self.streams[slot] = (int(width), int(height), int(window))
        return slot

    def remove_stream(self, slot):
        with torch.cuda.device(self.device):
            _mf.mf_engine_remove_stream(self.handle, slot)
        self.streams.pop(slot, None)

    def submit(self, slot, poses, depth, K, focus_map=None, guided_depth=None, info=None):
        """poses: host (n,3,4) FP64; depth / maps / info: device tensors or None."""
        P = np.ascontiguousarray(np.asarray(poses, dtype=np.float64))
        Kh = np.ascontiguousarray(np.asarray(K, dtype=np.float64).reshape(4))
        with torch.cuda.device(self.device):
            _mf.mf_engine_submit(self.handle, slot, P.shape[0], P, depth, Kh, focus_map,
                                 guided_depth, info)

    def tick(self):
        with torch.cuda.device(self.device):
            return _mf.mf_engine_tick(self.handle)

    def done(self, tick):
        return _mf.mf_engine_query(self.handle, tick)

    def wait(self, tick, timeout_ns=-1):
        with torch.cuda.device(self.device):
            _mf.mf_engine_wait(self.handle, tick, timeout_ns)

    def tune(self, width, height, window):
        with torch.cuda.device(self.device):
            return _mf.mf_engine_tune(self.handle, width, height, window)

    def stats(self):
        return _mf.mf_engine_get_stats(self.handle)

    def latency(self, reset=False):
        """Per-frame submit-to-completion latency (ms) of the finished ticks."""
        return _mf.mf_engine_latency(self.handle, reset)

    def close(self):
        if getattr(self, "handle", None):
            with torch.cuda.device(self.device):
                _mf.mf_engine_close(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MotionFocusServer:
    """Continuous batching over an engine (the C ABI's mf_server_*).

    Streams are admitted with ``add_stream``; ``submit`` queues a push from
    any thread and returns at once; a native thread batches queued pushes of
    all streams into ticks while earlier ticks run on the GPU.
    """

    def __init__(self, max_streams=256, max_tick_frames=4096, max_stream_frames=64,
                 depth_dtype=torch.float32, map_dtype=torch.float32, memory_budget=0,
                 tick_us=200, queue_limit=64, graph=True, tune=True, device=None):
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.depth_dtype, self.map_dtype = depth_dtype, map_dtype
        flags = (0 if graph else _mf.MF_ENGINE_NO_GRAPH) | (0 if tune else _mf.MF_ENGINE_NO_TUNE)
        eng = _mf.mf_engine_desc_init(
            max_streams=max_streams, max_tick_frames=max_tick_frames,
            max_stream_frames=max_stream_frames, depth_dtype=_DT[depth_dtype],
            map_dtype=_DT[map_dtype], flags=flags, memory_budget=int(memory_budget))
        self.desc = _mf.mf_server_desc_init(engine=eng, tick_us=int(tick_us),
                                            queue_limit=int(queue_limit))
        with torch.cuda.device(self.device):
            self.handle = _mf.mf_server_open(self.desc)

    def add_stream(self, width, height, window=8, smooth_len=15, mode="accel",
                   pose_frame="world", overlap=0, calib=None, reserve_bytes=0):
        cw, ch = calib if calib is not None else (0, 0)
        d = _mf.mf_stream_desc_init(
            width=int(width), height=int(height), calib_width=cw, calib_height=ch,
            window=int(window), smooth_len=int(smooth_len), mode=_MODES[mode],
            pose_frame=_FRAMES[pose_frame], overlap=int(overlap),
            depth_dtype=_DT[self.depth_dtype], map_dtype=_DT[self.map_dtype])
        with torch.cuda.device(self.device):
            return _mf.mf_server_add_stream(self.handle, d, reserve_bytes)

    def submit(self, slot, poses, depth, K, focus_map=None, guided_depth=None, info=None):
        P = np.ascontiguousarray(np.asarray(poses, dtype=np.float64))
        Kh = np.ascontiguousarray(np.asarray(K, dtype=np.float64).reshape(4))
        _mf.mf_server_submit(self.handle, slot, P.shape[0], P, depth, Kh, focus_map,
                             guided_depth, info)

    def frames_done(self, slot):
        return _mf.mf_server_frames_done(self.handle, slot)

    def tune(self, width, height, window):
        with torch.cuda.device(self.device):
            return _mf.mf_server_tune(self.handle, width, height, window)

    def remove_stream(self, slot):
        _mf.mf_server_remove_stream(self.handle, slot)

    def drain(self, timeout_ns=-1):
        _mf.mf_server_drain(self.handle, timeout_ns)

    def latency(self, reset=False):
        return _mf.mf_server_latency(self.handle, reset)

    def stats(self):
        return _mf.mf_server_get_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            with torch.cuda.device(self.device):
                _mf.mf_server_close(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
