"""ctypes binding of libmf's C ABI (include/mf.h): argument marshalling only.

Every function here has the name of the C entry point it wraps and only
converts arguments (torch tensors, numpy arrays or raw integer addresses to
pointers; Python numbers to C scalars) and raises ``MFError`` on a non-zero
status.  All computation happens in the library's CUDA kernels.  Loading
fails loudly when libmf.so has not been built: there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MF_CHECKED=1 loads the checked debug library (bounds-checked map kernels)
LIB_PATH = os.path.join(_HERE, "libmf_checked.so" if os.environ.get("MF_CHECKED") == "1" else "libmf.so")

MF_F32, MF_BF16, MF_F16 = 0, 1, 2
MF_MODE_ACCEL, MF_MODE_HEADING = 0, 1
MF_POSES_WORLD, MF_POSES_BATCH_LOCAL = 0, 1
MF_FRAME_OK, MF_FRAME_EMPTY, MF_FRAME_BAD_POSE, MF_FRAME_TIMEOUT = 0, 1, 2, 3
MF_FLAG_TIME_KERNELS = 1
MF_FLAG_MAP_CUDA_CORES = 8
MF_FLAG_MAP_TENSOR_CORES = 16
MF_FLAG_DEPTH_ALIGN = 32
MF_NORM_COUNT, MF_NORM_MAX = 0, 1
(MF_OK, MF_ERR_INVALID_ARG, MF_ERR_INVALID_POSE, MF_ERR_OOM, MF_ERR_NOT_READY,
 MF_ERR_TIMEOUT, MF_ERR_CUDA, MF_ERR_ADMISSION, MF_ERR_NO_DEVICE) = range(9)

EXPORTED = ("mf_stream_desc_init", "mf_open_stream", "mf_push_frames", "mf_get_maps",
            "mf_sync", "mf_pending_frames", "mf_reset_stream", "mf_stream_stats",
            "mf_close_stream", "mf_status_string", "mf_version", "mf_total_kernel_launches",
            "mf_last_error", "mf_render_noalloc", "mf_engine_desc_init", "mf_engine_open",
            "mf_engine_add_stream", "mf_engine_remove_stream", "mf_engine_submit",
            "mf_engine_tick", "mf_engine_query", "mf_engine_wait", "mf_engine_tune",
            "mf_engine_get_stats", "mf_engine_close", "mf_engine_latency",
            "mf_server_desc_init", "mf_server_open", "mf_server_add_stream", "mf_server_submit",
            "mf_server_frames_done", "mf_server_remove_stream", "mf_server_drain",
            "mf_server_latency", "mf_server_get_stats", "mf_server_close", "mf_clock_ns",
            "mf_engine_submit_batch", "mf_server_submit_batch", "mf_server_tune",
            "mf_probe_open", "mf_probe_stamp", "mf_probe_latency", "mf_probe_close",
            "mf_set_fault", "mf_stream_snapshot", "mf_stream_restore")
MF_ENGINE_NO_GRAPH = 2
MF_ENGINE_NO_TUNE = 4
MF_NOALLOC_MAX_FRAMES = 256
MF_NOALLOC_MAX_POSES = MF_NOALLOC_MAX_FRAMES + 63

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class MFStreamDesc(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("calib_width", ctypes.c_int32), ("calib_height", ctypes.c_int32),
        ("window", ctypes.c_int32), ("smooth_len", ctypes.c_int32),
        ("mode", ctypes.c_int32), ("pose_frame", ctypes.c_int32),
        ("overlap", ctypes.c_int32), ("depth_dtype", ctypes.c_int32),
        ("map_dtype", ctypes.c_int32), ("max_pending", ctypes.c_int32),
        ("flags", ctypes.c_uint32), ("normalize", ctypes.c_int32),
        ("sigma_rel", ctypes.c_double), ("s_lo", ctypes.c_double),
        ("s_hi", ctypes.c_double), ("depth_ref_m", ctypes.c_double),
        ("cuda_stream", ctypes.c_void_p),
        ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
    ]


class MFStats(ctypes.Structure):
    _fields_ = [
        ("frames_pushed", ctypes.c_int64), ("frames_emitted", ctypes.c_int64),
        ("frames_rendered", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
        ("map_launches", ctypes.c_int64), ("map_kernel_ms", ctypes.c_double),
        ("device_bytes", ctypes.c_int64), ("last_map_kernel", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
    ]


class MFEngineDesc(ctypes.Structure):
    _fields_ = [
        ("max_streams", ctypes.c_int32), ("max_tick_frames", ctypes.c_int32),
        ("max_stream_frames", ctypes.c_int32), ("depth_dtype", ctypes.c_int32),
        ("map_dtype", ctypes.c_int32), ("flags", ctypes.c_uint32),
        ("memory_budget", ctypes.c_int64), ("cuda_stream", ctypes.c_void_p),
    ]


class MFEngineStats(ctypes.Structure):
    _fields_ = [
        ("ticks", ctypes.c_int64), ("frames", ctypes.c_int64), ("units", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64), ("graph_launches", ctypes.c_int64),
        ("streams", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("device_bytes", ctypes.c_int64), ("accounted_bytes", ctypes.c_int64),
        ("tick_gpu_ms", ctypes.c_double), ("frames_path", ctypes.c_int64 * 2),
    ]


class MFLatencyStats(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p90_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double)]


class MFServerDesc(ctypes.Structure):
    _fields_ = [("engine", MFEngineDesc), ("tick_us", ctypes.c_int32),
                ("queue_limit", ctypes.c_int32)]


# numpy views of the C result records (layouts of include/mf.h)
FRAME_INFO_DTYPE = np.dtype([
    ("frame_index", "<i8"), ("status", "<i4"), ("n_valid", "<i4"), ("valid_mask", "<u4"),
    ("focus_valid", "<i4"), ("focus_u", "<f8"), ("focus_v", "<f8"), ("focus_px_x", "<i4"),
    ("focus_px_y", "<i4"), ("argmax_x", "<i4"), ("argmax_y", "<i4"), ("map_max", "<f4"),
    ("depth_scale", "<f4")])
MOTION_POINT_DTYPE = np.dtype([("u", "<f8"), ("v", "<f8"), ("sigma", "<f8"), ("s", "<f8"),
                               ("valid", "<i4"), ("reserved", "<i4")])
PUSH_DTYPE = np.dtype([("slot", "<i4"), ("n", "<i4"), ("poses", "<u8"), ("depth", "<u8"),
                       ("K", "<u8"), ("focus_map", "<u8"), ("guided_depth", "<u8"),
                       ("info", "<u8"), ("arrival_ns", "<i8")])
assert FRAME_INFO_DTYPE.itemsize == 64 and MOTION_POINT_DTYPE.itemsize == 40
assert PUSH_DTYPE.itemsize == 64


class MFError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        msg = f"{where}: {status_name(status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.mf_stream_desc_init.argtypes = [ctypes.POINTER(MFStreamDesc)]
    lib.mf_stream_desc_init.restype = None
    lib.mf_open_stream.argtypes = [ctypes.POINTER(MFStreamDesc), ctypes.POINTER(vp)]
    lib.mf_push_frames.argtypes = [vp, i32, vp, vp, vp]
    lib.mf_get_maps.argtypes = [vp, i32, vp, vp, vp, vp, ctypes.POINTER(i32), i64]
    lib.mf_sync.argtypes = [vp, i64]
    lib.mf_pending_frames.argtypes = [vp, ctypes.POINTER(i32)]
    lib.mf_reset_stream.argtypes = [vp]
    lib.mf_stream_stats.argtypes = [vp, ctypes.POINTER(MFStats)]
    lib.mf_close_stream.argtypes = [vp]
    lib.mf_status_string.argtypes = [ctypes.c_int]
    lib.mf_status_string.restype = ctypes.c_char_p
    lib.mf_version.restype = ctypes.c_int
    lib.mf_total_kernel_launches.restype = i64
    lib.mf_last_error.restype = ctypes.c_char_p
    lib.mf_render_noalloc.argtypes = [ctypes.POINTER(MFStreamDesc), i32, vp, i32, vp, vp, vp, vp,
                                      vp]
    lib.mf_engine_desc_init.argtypes = [ctypes.POINTER(MFEngineDesc)]
    lib.mf_engine_desc_init.restype = None
    lib.mf_engine_open.argtypes = [ctypes.POINTER(MFEngineDesc), ctypes.POINTER(vp)]
    lib.mf_engine_add_stream.argtypes = [vp, ctypes.POINTER(MFStreamDesc), i64,
                                         ctypes.POINTER(i32)]
    lib.mf_engine_remove_stream.argtypes = [vp, i32]
    lib.mf_engine_submit.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.mf_engine_tick.argtypes = [vp, ctypes.POINTER(i64)]
    lib.mf_engine_query.argtypes = [vp, i64, ctypes.POINTER(i32)]
    lib.mf_engine_wait.argtypes = [vp, i64, i64]
    lib.mf_engine_tune.argtypes = [vp, i32, i32, i32, ctypes.POINTER(i32)]
    lib.mf_engine_get_stats.argtypes = [vp, ctypes.POINTER(MFEngineStats)]
    lib.mf_engine_close.argtypes = [vp]
    lib.mf_engine_latency.argtypes = [vp, ctypes.POINTER(MFLatencyStats), i32]
    lib.mf_server_desc_init.argtypes = [ctypes.POINTER(MFServerDesc)]
    lib.mf_server_desc_init.restype = None
    lib.mf_server_open.argtypes = [ctypes.POINTER(MFServerDesc), ctypes.POINTER(vp)]
    lib.mf_server_add_stream.argtypes = [vp, ctypes.POINTER(MFStreamDesc), i64,
                                         ctypes.POINTER(i32)]
    lib.mf_server_submit.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.mf_server_frames_done.argtypes = [vp, i32, ctypes.POINTER(i64)]
    lib.mf_server_remove_stream.argtypes = [vp, i32]
    lib.mf_server_drain.argtypes = [vp, i64]
    lib.mf_server_latency.argtypes = [vp, ctypes.POINTER(MFLatencyStats), i32]
    lib.mf_server_get_stats.argtypes = [vp, ctypes.POINTER(MFEngineStats)]
    lib.mf_server_close.argtypes = [vp]
    lib.mf_clock_ns.restype = i64
    lib.mf_engine_submit_batch.argtypes = [vp, i32, vp, ctypes.POINTER(i32)]
    lib.mf_server_submit_batch.argtypes = [vp, i32, vp, ctypes.POINTER(i32)]
    lib.mf_server_tune.argtypes = [vp, i32, i32, i32, ctypes.POINTER(i32)]
    lib.mf_probe_open.argtypes = [ctypes.POINTER(vp)]
    lib.mf_probe_stamp.argtypes = [vp, vp, i32, vp]
    lib.mf_probe_latency.argtypes = [vp, ctypes.POINTER(MFLatencyStats), i32]
    lib.mf_probe_close.argtypes = [vp]
    lib.mf_set_fault.argtypes = [ctypes.c_char_p]
    lib.mf_stream_snapshot.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
    lib.mf_stream_restore.argtypes = [vp, vp, i64]
    for name in ("mf_open_stream", "mf_push_frames", "mf_get_maps", "mf_sync",
                 "mf_pending_frames", "mf_reset_stream", "mf_stream_stats", "mf_close_stream",
                 "mf_render_noalloc", "mf_engine_open", "mf_engine_add_stream",
                 "mf_engine_remove_stream", "mf_engine_submit", "mf_engine_tick",
                 "mf_engine_query", "mf_engine_wait", "mf_engine_tune", "mf_engine_get_stats",
                 "mf_engine_close", "mf_engine_latency", "mf_server_open",
                 "mf_server_add_stream", "mf_server_submit", "mf_server_frames_done",
                 "mf_server_remove_stream", "mf_server_drain", "mf_server_latency",
                 "mf_server_get_stats", "mf_server_close", "mf_engine_submit_batch",
                 "mf_server_submit_batch", "mf_server_tune", "mf_probe_open", "mf_probe_stamp",
                 "mf_probe_latency", "mf_probe_close", "mf_set_fault", "mf_stream_snapshot",
                 "mf_stream_restore"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


lib = _load()


def status_name(status):
    return lib.mf_status_string(int(status)).decode()


def _check(rc, where):
    if rc != MF_OK:
        raise MFError(rc, where, lib.mf_last_error().decode(errors="replace"))


def ptr(x):
    """Address of a torch tensor, numpy array, ctypes object or int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return ctypes.addressof(x)


# ----------------------------------------------------------- entry points --
def mf_stream_desc_init(**fields):
    d = MFStreamDesc()
    lib.mf_stream_desc_init(ctypes.byref(d))
    for k, v in fields.items():
        if not hasattr(d, k):
            raise TypeError(f"unknown descriptor field {k}")
        setattr(d, k, v)
    return d


def mf_open_stream(desc):
    h = ctypes.c_void_p()
    _check(lib.mf_open_stream(ctypes.byref(desc), ctypes.byref(h)), "mf_open_stream")
    return h.value


def mf_push_frames(s, n, poses, depth, K):
    _check(lib.mf_push_frames(s, int(n), ptr(poses), ptr(depth), ptr(K)), "mf_push_frames")


def mf_get_maps(s, max_frames, focus_map=None, guided_depth=None, info=None, points=None,
                timeout_ns=-1):
    n = ctypes.c_int32()
    _check(lib.mf_get_maps(s, int(max_frames), ptr(focus_map), ptr(guided_depth), ptr(info),
                           ptr(points), ctypes.byref(n), int(timeout_ns)), "mf_get_maps")
    return n.value


def mf_sync(s, timeout_ns=-1):
    _check(lib.mf_sync(s, int(timeout_ns)), "mf_sync")


def mf_pending_frames(s):
    n = ctypes.c_int32()
    _check(lib.mf_pending_frames(s, ctypes.byref(n)), "mf_pending_frames")
    return n.value


def mf_reset_stream(s):
    _check(lib.mf_reset_stream(s), "mf_reset_stream")


def mf_stream_stats(s):
    st = MFStats()
    _check(lib.mf_stream_stats(s, ctypes.byref(st)), "mf_stream_stats")
    return st


def mf_close_stream(s):
    _check(lib.mf_close_stream(s), "mf_close_stream")


def mf_status_string(status):
    return status_name(status)


def mf_version():
    return lib.mf_version()


def mf_total_kernel_launches():
    return lib.mf_total_kernel_launches()


def mf_last_error():
    return lib.mf_last_error().decode(errors="replace")


def mf_render_noalloc(desc, n_poses, poses, n_render, depth, K, focus_map=None,
                      guided_depth=None, info=None):
    _check(lib.mf_render_noalloc(ctypes.byref(desc), int(n_poses), ptr(poses), int(n_render),
                                 ptr(depth), ptr(K), ptr(focus_map), ptr(guided_depth), ptr(info)),
           "mf_render_noalloc")


# ----------------------------------------------------------- engine --------
def mf_engine_desc_init(**fields):
    d = MFEngineDesc()
    lib.mf_engine_desc_init(ctypes.byref(d))
    for k, v in fields.items():
        if not hasattr(d, k):
            raise TypeError(f"unknown engine field {k}")
        setattr(d, k, v)
    return d


def mf_engine_open(desc):
    h = ctypes.c_void_p()
    _check(lib.mf_engine_open(ctypes.byref(desc), ctypes.byref(h)), "mf_engine_open")
    return h.value


def mf_engine_add_stream(e, stream_desc, reserve_bytes=0):
    slot = ctypes.c_int32()
    _check(lib.mf_engine_add_stream(e, ctypes.byref(stream_desc), int(reserve_bytes),
                                    ctypes.byref(slot)), "mf_engine_add_stream")
    return slot.value


def mf_engine_remove_stream(e, slot):
    _check(lib.mf_engine_remove_stream(e, int(slot)), "mf_engine_remove_stream")


def mf_engine_submit(e, slot, n, poses, depth, K, focus_map=None, guided_depth=None, info=None):
    _check(lib.mf_engine_submit(e, int(slot), int(n), ptr(poses), ptr(depth), ptr(K),
                                ptr(focus_map), ptr(guided_depth), ptr(info)), "mf_engine_submit")


def mf_engine_tick(e):
    t = ctypes.c_int64()
    _check(lib.mf_engine_tick(e, ctypes.byref(t)), "mf_engine_tick")
    return t.value


def mf_engine_query(e, tick):
    d = ctypes.c_int32()
    _check(lib.mf_engine_query(e, int(tick), ctypes.byref(d)), "mf_engine_query")
    return bool(d.value)


def mf_engine_wait(e, tick, timeout_ns=-1):
    _check(lib.mf_engine_wait(e, int(tick), int(timeout_ns)), "mf_engine_wait")


def mf_engine_tune(e, width, height, window):
    b = ctypes.c_int32()
    _check(lib.mf_engine_tune(e, int(width), int(height), int(window), ctypes.byref(b)),
           "mf_engine_tune")
    return b.value


def mf_engine_get_stats(e):
    st = MFEngineStats()
    _check(lib.mf_engine_get_stats(e, ctypes.byref(st)), "mf_engine_get_stats")
    return st


def mf_engine_close(e):
    _check(lib.mf_engine_close(e), "mf_engine_close")


def mf_engine_latency(e, reset=False):
    st = MFLatencyStats()
    _check(lib.mf_engine_latency(e, ctypes.byref(st), 1 if reset else 0), "mf_engine_latency")
    return st


# ----------------------------------------------------------- server --------
def mf_server_desc_init(engine=None, **fields):
    d = MFServerDesc()
    lib.mf_server_desc_init(ctypes.byref(d))
    if engine is not None:
        d.engine = engine
    for k, v in fields.items():
        if not hasattr(d, k):
            raise TypeError(f"unknown server field {k}")
        setattr(d, k, v)
    return d


def mf_server_open(desc):
    h = ctypes.c_void_p()
    _check(lib.mf_server_open(ctypes.byref(desc), ctypes.byref(h)), "mf_server_open")
    return h.value


def mf_server_add_stream(s, stream_desc, reserve_bytes=0):
    slot = ctypes.c_int32()
    _check(lib.mf_server_add_stream(s, ctypes.byref(stream_desc), int(reserve_bytes),
                                    ctypes.byref(slot)), "mf_server_add_stream")
    return slot.value


def mf_server_submit(s, slot, n, poses, depth, K, focus_map=None, guided_depth=None, info=None):
    _check(lib.mf_server_submit(s, int(slot), int(n), ptr(poses), ptr(depth), ptr(K),
                                ptr(focus_map), ptr(guided_depth), ptr(info)), "mf_server_submit")


def mf_server_frames_done(s, slot):
    n = ctypes.c_int64()
    _check(lib.mf_server_frames_done(s, int(slot), ctypes.byref(n)), "mf_server_frames_done")
    return n.value


def mf_server_remove_stream(s, slot):
    _check(lib.mf_server_remove_stream(s, int(slot)), "mf_server_remove_stream")


def mf_server_drain(s, timeout_ns=-1):
    _check(lib.mf_server_drain(s, int(timeout_ns)), "mf_server_drain")


def mf_server_latency(s, reset=False):
    st = MFLatencyStats()
    _check(lib.mf_server_latency(s, ctypes.byref(st), 1 if reset else 0), "mf_server_latency")
    return st


def mf_server_get_stats(s):
    st = MFEngineStats()
    _check(lib.mf_server_get_stats(s, ctypes.byref(st)), "mf_server_get_stats")
    return st


def mf_server_close(s):
    _check(lib.mf_server_close(s), "mf_server_close")


def mf_clock_ns():
    return lib.mf_clock_ns()


def mf_engine_submit_batch(e, pushes):
    """pushes: numpy array of PUSH_DTYPE records (addresses as integers)."""
    pushes = np.ascontiguousarray(pushes, dtype=PUSH_DTYPE)
    acc = ctypes.c_int32()
    _check(lib.mf_engine_submit_batch(e, len(pushes), pushes.ctypes.data, ctypes.byref(acc)),
           "mf_engine_submit_batch")
    return acc.value


def mf_server_submit_batch(s, pushes):
    pushes = np.ascontiguousarray(pushes, dtype=PUSH_DTYPE)
    acc = ctypes.c_int32()
    _check(lib.mf_server_submit_batch(s, len(pushes), pushes.ctypes.data, ctypes.byref(acc)),
           "mf_server_submit_batch")
    return acc.value


def mf_server_tune(s, width, height, window):
    b = ctypes.c_int32()
    _check(lib.mf_server_tune(s, int(width), int(height), int(window), ctypes.byref(b)),
           "mf_server_tune")
    return b.value


# ------------------------------------------------------------ latency probe --
def mf_probe_open():
    h = ctypes.c_void_p()
    _check(lib.mf_probe_open(ctypes.byref(h)), "mf_probe_open")
    return h.value


def mf_probe_stamp(p, cuda_stream, arrival_ns):
    """arrival_ns: int64 numpy array (mf_clock_ns clock); cuda_stream: handle or None."""
    a = np.ascontiguousarray(arrival_ns, dtype=np.int64)
    _check(lib.mf_probe_stamp(p, cuda_stream, len(a), a.ctypes.data if len(a) else None),
           "mf_probe_stamp")


def mf_probe_latency(p, reset=False):
    st = MFLatencyStats()
    _check(lib.mf_probe_latency(p, ctypes.byref(st), 1 if reset else 0), "mf_probe_latency")
    return st


def mf_probe_close(p):
    _check(lib.mf_probe_close(p), "mf_probe_close")


# ------------------------------------------------------- fault injection --
def mf_set_fault(spec=None):
    """Host-side fault injection rules (see include/mf.h); None clears them."""
    _check(lib.mf_set_fault(spec.encode() if spec else None), "mf_set_fault")


# ------------------------------------------------------- snapshot / restore --
def mf_stream_snapshot(s):
    """The stream's resident state as bytes (see include/mf.h)."""
    n = ctypes.c_int64()
    _check(lib.mf_stream_snapshot(s, None, 0, ctypes.byref(n)), "mf_stream_snapshot")
    buf = ctypes.create_string_buffer(n.value)
    _check(lib.mf_stream_snapshot(s, buf, n.value, ctypes.byref(n)), "mf_stream_snapshot")
    return buf.raw[:n.value]


def mf_stream_restore(s, blob):
    blob = bytes(blob)
    _check(lib.mf_stream_restore(s, blob, len(blob)), "mf_stream_restore")
