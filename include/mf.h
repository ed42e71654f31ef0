/*
 * mf.h -- C ABI of libmf, the GB300 (sm_103a) motion-focus library.
 *
 * The library implements the data-parallel path of "Motion Focus Recognition
 * in Fast-Moving Egocentric Video" (arXiv 2601.07154, Section 2.3): from a
 * stream of camera poses T_t^{w->c}, per-pixel depth maps D_t and pinhole
 * intrinsics K it produces, for every frame, the motion-focus map M of Eq. 7
 * and the motion-guided depth map of Fig. 1(iii) / Fig. 5.
 *
 * Conventions used by every entry point
 *   - Poses are world-to-camera rigid transforms stored as 3x4 row-major FP64
 *     matrices [R | t] (12 doubles, 96 bytes per frame); the implied bottom
 *     row is [0 0 0 1].  Camera axes: x right, y down, z forward (optical
 *     axis); the world y axis is gravity ("down").
 *   - Images (depth in, maps out) are height x width, row-major, one plane
 *     per frame, planes contiguous (frame stride = width*height elements).
 *     Pixel (x, y) -- column x, row y -- has its centre at image coordinates
 *     (x, y).  Depth is camera z-depth in metres; 0 or a non-finite value
 *     means "no depth".
 *   - Pointers may be host memory (pageable or pinned) or device memory of
 *     the stream's device; the library tells them apart with
 *     cudaPointerGetAttributes.  Managed memory counts as device memory.
 *     Device memory of another GPU is refused with MF_ERR_INVALID_ARG before
 *     any work is enqueued (the kernels run on the stream's device only).
 *   - Every entry point returns an mf_status (0 = MF_OK).  No exception or
 *     signal crosses the ABI.  Calls on one mf_stream are not reentrant;
 *     different mf_stream handles may be used from different threads.
 */
#ifndef MF_H
#define MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MF_VERSION 1
#define MF_MAX_WINDOW 32       /* N motion points per frame */
#define MF_MAX_HISTORY 64      /* window + smooth_len - 1 poses per frame */
#define MF_MAX_DIM 16384       /* largest width / height */

typedef struct mf_stream mf_stream; /* opaque, owned by the library */

typedef enum { MF_F32 = 0, MF_BF16 = 1, MF_F16 = 2 } mf_dtype;

/* Direction that is projected (Section 2.3):
 *   ACCEL   -- acceleration (Eqs. 2-3), the paper's motion focus;
 *   HEADING -- velocity: the projection of velocity that the paper compares
 *              its method against after Eq. 6. */
typedef enum { MF_MODE_ACCEL = 0, MF_MODE_HEADING = 1 } mf_mode;

/* Coordinate frame of pushed poses (Section 2.2):
 *   WORLD       -- poses already share one world frame;
 *   BATCH_LOCAL -- every push is one inference batch in its own local frame;
 *                  its first `overlap` frames repeat the previous batch's
 *                  last frames and are used for incremental anchoring. */
typedef enum { MF_POSES_WORLD = 0, MF_POSES_BATCH_LOCAL = 1 } mf_pose_frame;

typedef enum {
  MF_OK = 0,
  MF_ERR_INVALID_ARG = 1,  /* bad descriptor, size, pointer or call order */
  MF_ERR_INVALID_POSE = 2, /* reserved: poses are checked per frame, see MF_FRAME_BAD_POSE */
  MF_ERR_OOM = 3,          /* a device or pinned allocation failed */
  MF_ERR_NOT_READY = 4,    /* too many frames pending: call mf_get_maps first */
  MF_ERR_TIMEOUT = 5,      /* a bounded wait expired (see mf_get_maps / mf_sync) */
  MF_ERR_CUDA = 6,         /* a CUDA runtime call failed */
  MF_ERR_ADMISSION = 7,    /* a server could not admit a stream (budget) */
  MF_ERR_NO_DEVICE = 8     /* no usable CUDA device */
} mf_status;

/* Per-frame status reported in mf_frame_info.status. */
typedef enum {
  MF_FRAME_OK = 0,        /* at least one valid motion point */
  MF_FRAME_EMPTY = 1,     /* no valid motion point: M = G = 0 */
  MF_FRAME_BAD_POSE = 2,  /* the frame's own pose is not a rigid transform */
  MF_FRAME_TIMEOUT = 3    /* a bounded device wait of the tensor-core map kernel ran
                             out while rendering this frame: bands of its maps hold NaN
                             (the waiting call also returns MF_ERR_TIMEOUT) */
} mf_frame_status;

/* The normaliser Z of Eq. 7, which the paper leaves open:
 *   COUNT -- Z = number of valid points: M in [0, 1], 1 only where every
 *            point's Gaussian peaks (default);
 *   MAX   -- Z = the frame's largest point sum: the map is exactly 1 at
 *            its argmax (one extra in-place pass over M and G; map_max of
 *            mf_frame_info is then 1).  A frame whose count-normalised
 *            maximum is below 2^-20 (every point many sigma outside the
 *            image) keeps its count-normalised maps and map_max. */
typedef enum { MF_NORM_COUNT = 0, MF_NORM_MAX = 1 } mf_norm;

/* mf_stream_desc.flags */
#define MF_FLAG_TIME_KERNELS 1u /* time each map-kernel launch with CUDA events */
/* Map kernel choice.  Eq. 7 over a tile is a rank-N product of row and
 * column factor tables, so it can run on the CUDA cores (one FMA per point
 * and pixel) or on the tensor cores (tcgen05 with TMEM accumulators, three
 * TF32 products per FP32 term).  The map is HBM-bound, not a dense
 * contraction, so the library runs the CUDA-core kernel unless
 * MF_FLAG_MAP_TENSOR_CORES asks for the tensor cores; MF_FLAG_MAP_CUDA_CORES
 * names the default explicitly.  The flags are exclusive. */
#define MF_FLAG_MAP_CUDA_CORES 8u
#define MF_FLAG_MAP_TENSOR_CORES 16u
/* Depth alignment across batches (Section 2.2, Fig. 3), MF_POSES_BATCH_LOCAL
 * streams only: a monocular model returns every batch at its own scale, so
 * each batch after the first gets one scale s_b = s_{b-1} * m, where m is
 * the lower median of the single-precision ratios of the previous batch's
 * last `overlap` depth planes to this batch's first `overlap` planes, over
 * the pixels where both are finite and > 0 (no such pixel: m = 1; the first
 * batch, and the first batch after mf_reset_stream, has s = 1).  The
 * batch's translations are multiplied by s_b before anchoring, and its
 * depth by s_b in the motion-guided depth (G = M min(1, d0 / (s_b D))).
 * Needs every batch to hold at least `overlap` frames; the library keeps a
 * copy of the last `overlap` depth planes (device memory) between pushes.
 * The paper names the step but not its rule: this is the library's reading.
 * Not available in the batched engine or the serving loop
 * (MF_ERR_INVALID_ARG there). */
#define MF_FLAG_DEPTH_ALIGN 32u

/*
 * Stream descriptor.  Fill with mf_stream_desc_init() and override fields.
 *   width, height        map resolution == depth resolution (1..MF_MAX_DIM)
 *   calib_width/height   resolution the intrinsics K refer to; 0 = same as
 *                        the map.  K is rescaled to the map resolution
 *                        (the intrinsics K of Eq. 5, Section 1).
 *   window               W = N motion points per frame (Eq. 7), 1..32
 *   smooth_len           K samples of the causal least-squares fit that
 *                        generalises Eqs. 2-3 (3 reproduces Eq. 3 exactly);
 *                        >= 3 for ACCEL, >= 2 for HEADING;
 *                        window + smooth_len - 1 <= MF_MAX_HISTORY
 *   mode                 mf_mode
 *   pose_frame, overlap  mf_pose_frame and the shared frame count O of
 *                        Section 2.2 (BATCH_LOCAL: O >= 1; WORLD: O == 0)
 *   depth_dtype          storage type of pushed depth (mf_dtype)
 *   map_dtype            storage type of both output maps (mf_dtype)
 *   max_pending          frames that may wait between push and get_maps
 *   normalize            mf_norm (MF_NORM_MAX is not available to engine
 *                        streams)
 *   sigma_rel            sigma of Eq. 7 as a fraction of fx (default 0.1)
 *   s_lo, s_hi           clamp of the motion magnitude s_i (0.25, 4)
 *   depth_ref_m          d0 of the guided depth G = M min(1, d0/D) (1.0 m)
 *   cuda_stream          cudaStream_t to run on, including the runtime's
 *                        cudaStreamLegacy (0x1) and cudaStreamPerThread
 *                        (0x2) handles; NULL = a library-owned non-blocking
 *                        stream (not ordered with the legacy default stream)
 *   dev_alloc/dev_free   optional device allocator (e.g. PyTorch's caching
 *                        allocator); NULL = cudaMalloc / cudaFree
 */
typedef struct {
  int32_t width, height;
  int32_t calib_width, calib_height;
  int32_t window;
  int32_t smooth_len;
  int32_t mode;
  int32_t pose_frame;
  int32_t overlap;
  int32_t depth_dtype;
  int32_t map_dtype;
  int32_t max_pending;
  uint32_t flags;
  int32_t normalize;
  double sigma_rel, s_lo, s_hi, depth_ref_m;
  void* cuda_stream;
  void* (*dev_alloc)(size_t bytes, void* ctx);
  void (*dev_free)(void* ptr, void* ctx);
  void* alloc_ctx;
} mf_stream_desc;

/* Per-frame results (64 bytes). */
typedef struct {
  int64_t frame_index;   /* emitted-frame index within the stream, from 0 */
  int32_t status;        /* mf_frame_status */
  int32_t n_valid;       /* valid motion points = Z of Eq. 7 */
  uint32_t valid_mask;   /* bit s: slot s (frame n-W+1+s) is valid */
  int32_t focus_valid;   /* the newest point (slot W-1) is valid */
  double focus_u, focus_v;     /* Eq. 6 of the newest point, pixels; 0 if invalid */
  int32_t focus_px_x, focus_px_y; /* rint(focus) if inside the frame, else -1 */
  int32_t argmax_x, argmax_y;  /* largest M (ties: lowest y*width+x); -1 if empty */
  float map_max;               /* M at the argmax (FP32 arithmetic value, after
                                  the MF_NORM_MAX scaling when selected) */
  float depth_scale;           /* the frame's batch depth scale, rounded to FP32
                                  (1 without MF_FLAG_DEPTH_ALIGN) */
} mf_frame_info;

/* One motion point (slot s of a frame), FP64 (40 bytes). */
typedef struct {
  double u, v;      /* Eq. 6 projection at the map resolution */
  double sigma;     /* sigma * s_i of Eq. 7, pixels */
  double s;         /* motion magnitude s_i (clamped ratio to the mean) */
  int32_t valid;
  int32_t reserved;
} mf_motion_point;

typedef struct {
  int64_t frames_pushed;     /* poses received, overlap included */
  int64_t frames_emitted;    /* non-overlapping frames (Section 2.2) */
  int64_t frames_rendered;   /* frames whose maps were produced */
  int64_t kernel_launches;   /* this stream's kernel launches */
  int64_t map_launches;      /* map-kernel launches timed (MF_FLAG_TIME_KERNELS) */
  double map_kernel_ms;      /* summed CUDA-event time of those launches */
  int64_t device_bytes;      /* device memory the stream holds */
  uint32_t last_map_kernel;  /* MF_FLAG_MAP_CUDA_CORES or MF_FLAG_MAP_TENSOR_CORES:
                                the kernel of the last map launch (0 before any) */
  uint32_t reserved;
} mf_stats;

/* Fill *d with defaults (sigma_rel 0.1, s in [0.25, 4], d0 = 1 m, ACCEL,
 * WORLD poses, FP32 depth and maps, window 8, smooth_len 15,
 * max_pending 1024).  width/height stay 0 and must be set. */
void mf_stream_desc_init(mf_stream_desc* d);

/*
 * Open a stream: validates *d, allocates the pose history and the pending
 * frame records on the current CUDA device, and precomputes the
 * least-squares weights (Eqs. 2-3 generalised).  No kernel runs.
 * Returns MF_ERR_INVALID_ARG for an invalid descriptor, MF_ERR_OOM, or
 * MF_ERR_NO_DEVICE.  *out receives the handle (NULL on error).
 */
int mf_open_stream(const mf_stream_desc* d, mf_stream** out);

/*
 * Push one batch of n frames (Section 2.2; Eqs. 1-6 per frame).
 *   poses_w2c_3x4  n x 12 FP64 world-to-camera poses, host or device.
 *   depth          n depth planes of depth_dtype (height x width each),
 *                  host or device.  In BATCH_LOCAL mode after the first
 *                  push, planes 0..overlap-1 belong to overlap frames and
 *                  are not read (they may hold anything).  May be NULL:
 *                  then the guided-depth output of these frames is 0.
 *   K              host pointer to 4 FP64 values fx, fy, cx, cy at the
 *                  calibration resolution, in force for this batch.
 * Emits frames overlap..n-1 (all n on the first push or in WORLD mode):
 * anchors them (BATCH_LOCAL, gravity-locked yaw + translation), appends
 * them to the pose history and computes their motion points on the GPU.
 * Host poses and pageable host depth are copied before the call returns.
 * Pinned (page-locked) host depth is uploaded asynchronously by a copy
 * engine, in pieces that the map kernels consume as they arrive; device
 * inputs are read asynchronously on the stream, pose buffers before any
 * later push and depth buffers when the frames are rendered by mf_get_maps.
 * Keep pinned and device inputs unchanged until then.  A pose whose rotation is not orthonormal to 1e-6
 * (or not finite) makes its frame MF_FRAME_BAD_POSE and invalidates every
 * motion point whose fit uses it; a bad anchor makes the whole batch bad.
 * Errors: MF_ERR_INVALID_ARG (n < 1, n <= overlap on a later BATCH_LOCAL
 * push, NULL poses/K), MF_ERR_NOT_READY (more than max_pending frames would
 * wait), MF_ERR_OOM, MF_ERR_CUDA.  On error nothing is ingested.
 */
int mf_push_frames(mf_stream* s, int32_t n, const double* poses_w2c_3x4,
                   const void* depth, const double* K);

/*
 * Render up to max_frames pending frames, oldest first, into the caller's
 * buffers (Eq. 7 and the motion-guided depth), and report them.
 *   focus_map      n_out planes of map_dtype (height x width), or NULL
 *   guided_depth   n_out planes of map_dtype, or NULL
 *   info           n_out mf_frame_info records, or NULL
 *   points         n_out * window mf_motion_point records (slot-major per
 *                  frame), or NULL
 *   n_out          receives the number of frames returned (0 if none pend)
 *   timeout_ns     bound on the wait used when an output is host memory;
 *                  < 0 waits without bound.
 * If every non-NULL output is device memory the call only enqueues work on
 * the stream and returns; the results are ready once the stream reaches
 * that point (mf_sync).  If any output is host memory the call waits for
 * the copies.  Maps bound for host memory are rendered into a small device
 * ring in pieces of a few frames, and each piece is downloaded by a copy
 * engine while the next pieces render and the pinned-depth uploads of
 * mf_push_frames run, so both transfer directions overlap; on MF_ERR_TIMEOUT the frames count as returned but copies into
 * the caller's host buffers may still be in flight: keep those buffers
 * alive until mf_sync or mf_close_stream returns.
 */
int mf_get_maps(mf_stream* s, int32_t max_frames, void* focus_map, void* guided_depth,
                mf_frame_info* info, mf_motion_point* points, int32_t* n_out,
                int64_t timeout_ns);

/* Wait (bounded by timeout_ns; < 0 = no bound) until all work enqueued on
 * the stream has finished.  MF_ERR_TIMEOUT if the bound expires. */
int mf_sync(mf_stream* s, int64_t timeout_ns);

/* Number of emitted frames not yet returned by mf_get_maps. */
int mf_pending_frames(const mf_stream* s, int32_t* n);

/* Forget the pose history and pending frames (frame indices restart at 0);
 * keeps the allocations.  Does not wait: work already enqueued finishes in
 * stream order, and pending frames that were never returned are dropped. */
int mf_reset_stream(mf_stream* s);

/* Counters and, with MF_FLAG_TIME_KERNELS, map-kernel timings (waits for
 * the timed launches to finish). */
int mf_stream_stats(mf_stream* s, mf_stats* out);

/* Snapshot and restore of a stream's resident state, so that a live stream
 * can move to another process, GPU or server.  The paper has no
 * counterpart; the state is what the method carries between frames: the
 * last window + smooth_len - 1 world poses (Eqs. 1-4 look that far back)
 * with their bad-pose flags, the frame counters that place the next push's
 * anchoring (Section 2.2), and, with MF_FLAG_DEPTH_ALIGN, the batch scale
 * and the last `overlap` depth planes.
 *   mf_stream_snapshot  writes the snapshot to host memory buf (cap bytes);
 *                       buf = NULL only reports the size in *bytes.  Needs
 *                       no pending frames (MF_ERR_NOT_READY otherwise: call
 *                       mf_get_maps first); waits for the stream's work.
 *   mf_stream_restore   loads a snapshot into a stream opened with the same
 *                       descriptor fields (sizes, window, smooth_len, mode,
 *                       pose frame, overlap, dtypes, normalisation, sigma /
 *                       s / d0 parameters, depth alignment) that has taken no
 *                       push yet or was reset (MF_ERR_NOT_READY otherwise);
 *                       a different descriptor or a damaged snapshot gives
 *                       MF_ERR_INVALID_ARG.  Synchronous.
 * After a restore, the stream continues exactly as the snapshotted one
 * would: the same later pushes give bit-identical maps and records. */
int mf_stream_snapshot(mf_stream* s, void* buf, int64_t cap, int64_t* bytes);
int mf_stream_restore(mf_stream* s, const void* buf, int64_t bytes);

/* Wait for the stream's work, free everything the stream holds. */
int mf_close_stream(mf_stream* s);

/* Static description of a status code. */
const char* mf_status_string(int status);

/* MF_VERSION of the loaded library. */
int mf_version(void);

/* Kernel launches made by this process through the library (all streams). */
int64_t mf_total_kernel_launches(void);

/* Text of the last error raised on the calling thread ("" if none); valid
 * until the thread's next failing call. */
const char* mf_last_error(void);

/* Host-side fault injection, for testing how callers detect failures.  The
 * paper has no counterpart.  Every fault is made on the host at a chosen
 * call; none makes a GPU fault, trap or hang.  `spec` is a comma-separated
 * list of rules, each a name with an optional "@n" (the n-th occurrence
 * fails, counted from this call; without it every occurrence fails):
 *   alloc_fail      a device allocation of a stream or an engine returns
 *                   nothing (the call reports MF_ERR_OOM);
 *   bad_pose        a host pose of mf_push_frames is scaled so that it is no
 *                   rotation on its way to the device (its frame reports
 *                   MF_FRAME_BAD_POSE); occurrences count poses;
 *   drop_push       a serving push is accepted and then lost: its frames never
 *                   complete (mf_server_drain with a timeout returns
 *                   MF_ERR_TIMEOUT; mf_server_frames_done falls short);
 *   admission_full  an engine or server admission is refused (MF_ERR_ADMISSION);
 *   wait_timeout    a completed mf_sync / mf_get_maps wait reports a device
 *                   wait that ran out (MF_ERR_TIMEOUT), as the tensor-core map
 *                   kernel's bounded wait does when it expires.
 * NULL or "" removes every rule.  The environment variable MF_FAULT, read
 * at the first use, installs an initial spec.  Returns MF_ERR_INVALID_ARG for
 * a malformed spec (the rules in force are then unchanged). */
int mf_set_fault(const char* spec);

/* ---------------------------------------------------------------------------
 * Batched engine: many streams on one GPU, one batched launch per tick.
 *
 * The engine is the serving form of the same per-frame method (Sections
 * 2.2-2.3): each admitted stream keeps its pose history resident on the
 * GPU; frames submitted by any number of streams between two ticks are
 * processed by ONE batch -- a CUDA graph of one table upload and four kernels
 * (ingest + anchoring, motion points, the persistent map kernel over every
 * frame's tiles whatever its resolution and window, result records).  Ticks
 * are asynchronous and may overlap host-side preparation of the next one.
 * A frame's maps are identical whether its stream runs alone or among
 * others.  Tile heights are picked per resolution class by a built-in
 * autotuner (mf_engine_tune) unless MF_ENGINE_NO_TUNE is set.
 */
typedef struct mf_engine mf_engine;

#define MF_ENGINE_NO_GRAPH 2u /* launch the tick's kernels directly (no CUDA graph) */
#define MF_ENGINE_NO_TUNE 4u  /* use the plain path's tile height, never tune */

typedef struct {
  int32_t max_streams;       /* stream slots (default 256) */
  int32_t max_tick_frames;   /* emitted frames per tick over all streams (default 4096) */
  int32_t max_stream_frames; /* frames one stream may emit per tick (default 64) */
  int32_t depth_dtype;       /* storage type of all depth planes (mf_dtype) */
  int32_t map_dtype;         /* storage type of all output maps (mf_dtype) */
  uint32_t flags;            /* MF_ENGINE_* and MF_FLAG_TIME_KERNELS */
  int64_t memory_budget;     /* device bytes admitted streams may account for; 0 = no limit */
  void* cuda_stream;         /* as in mf_stream_desc */
} mf_engine_desc;

typedef struct {
  int64_t ticks;             /* ticks launched */
  int64_t frames;            /* frames processed */
  int64_t units;             /* map tiles processed */
  int64_t kernel_launches;   /* kernels run by the ticks (graph nodes included) */
  int64_t graph_launches;    /* CUDA graph launches */
  int32_t streams;           /* admitted streams */
  int32_t reserved;
  int64_t device_bytes;      /* device memory held by the engine */
  int64_t accounted_bytes;   /* engine memory + admitted streams' reservations */
  double tick_gpu_ms;        /* with MF_FLAG_TIME_KERNELS: summed GPU time of the ticks */
  int64_t frames_path[2];    /* frames rendered by the 32-point map path [0] (any window,
                                2 columns per lane) and by the 16-point path [1] (windows
                                up to 16 on widths divisible by its columns per lane) */
} mf_engine_stats;

/* Defaults: 256 streams, 4096 frames per tick, 64 per stream, FP32, no
 * budget, library-owned stream. */
void mf_engine_desc_init(mf_engine_desc* d);

/* Allocate the engine's tick tables (pinned + device, double-buffered), the
 * per-tick frame records and the stream slots.  MF_ERR_INVALID_ARG, MF_ERR_OOM. */
int mf_engine_open(const mf_engine_desc* d, mf_engine** out);

/* Admit a stream described by *d (its dtypes must equal the engine's, its
 * width must be even; its cuda_stream and allocator fields are ignored).
 * The stream's pose history (preallocated for every slot at open) stays
 * resident on the device until removal; admission allocates nothing and does
 * not wait, unless it must first tune a new resolution class (the
 * autotuner runs synchronously; mf_engine_tune can run it beforehand).
 * reserve_bytes: device memory the caller will hold for this stream (its
 * output planes, say), counted with the engine's own memory against
 * memory_budget.  On success *slot names the stream.  MF_ERR_ADMISSION when
 * every slot is taken or the budget would be exceeded; MF_ERR_INVALID_ARG for
 * a bad descriptor. */
int mf_engine_add_stream(mf_engine* e, const mf_stream_desc* d, int64_t reserve_bytes,
                         int32_t* slot);

/* Free a slot (waits for the ticks that used it).  Its frames must not be
 * pending (submitted after the last tick). */
int mf_engine_remove_stream(mf_engine* e, int32_t slot);

/* Queue one push of stream `slot` for the next tick (Section 2.2 semantics,
 * as mf_push_frames): n poses (host memory, n x 12 FP64, copied now), n depth
 * planes (device memory; planes of overlap frames are not read; NULL allowed),
 * K (host, fx fy cx cy).  The emitted frames' maps go to focus_map /
 * guided_depth (device planes, n_emit each, or NULL) and their records to
 * info (device, n_emit records, or NULL).  Device buffers are read and
 * written when the tick runs: keep them valid until it is done.
 * MF_ERR_NOT_READY if the stream already has a push in this tick or the tick
 * is full; MF_ERR_INVALID_ARG as mf_push_frames, or for planes not aligned
 * to two elements. */
int mf_engine_submit(mf_engine* e, int32_t slot, int32_t n, const double* poses_w2c_3x4,
                     const void* depth, const double* K, void* focus_map, void* guided_depth,
                     mf_frame_info* info);

/* One push for the batched submit calls below (64 bytes). */
typedef struct {
  int32_t slot, n;              /* stream and pose count, as mf_engine_submit */
  const double* poses_w2c_3x4;  /* host, n x 12 FP64 */
  const void* depth;            /* device planes or NULL */
  const double* K;              /* host, fx fy cx cy */
  void* focus_map;              /* device planes or NULL */
  void* guided_depth;           /* device planes or NULL */
  mf_frame_info* info;          /* device records or NULL */
  int64_t arrival_ns;           /* when the frames arrived, on mf_clock_ns()'s clock;
                                   0 = now.  Latency statistics start here. */
} mf_push;

/* The monotonic clock (nanoseconds) of arrival times and latency statistics. */
int64_t mf_clock_ns(void);

/* mf_engine_submit for n pushes in order; *accepted receives how many were
 * queued.  Stops at the first push that fails and returns its status. */
int mf_engine_submit_batch(mf_engine* e, int32_t n, const mf_push* pushes, int32_t* accepted);

/* Launch everything submitted since the previous tick as one batch.  Does
 * not wait.  *tick receives its id (-1 if nothing was submitted). */
int mf_engine_tick(mf_engine* e, int64_t* tick);

/* *done = 1 when tick `tick` (and every earlier one) has finished. */
int mf_engine_query(mf_engine* e, int64_t tick, int32_t* done);

/* Wait for tick `tick` (bounded by timeout_ns; < 0 = no bound). */
int mf_engine_wait(mf_engine* e, int64_t tick, int64_t timeout_ns);

/* Time the map kernel on a synthetic batch of width x height frames whose
 * points all reach the frame, with the window rounded up to 8, 16 or 32
 * points, for each candidate tile height, and keep the fastest for that
 * class (resolution, window bucket); *band_h receives it.  Synchronous. */
int mf_engine_tune(mf_engine* e, int32_t width, int32_t height, int32_t window, int32_t* band_h);

int mf_engine_get_stats(mf_engine* e, mf_engine_stats* out);

/* Per-frame latency of the ticks that have finished: from the frame's
 * mf_engine_submit call to the GPU completing its tick (stamped by a host
 * function enqueued behind the tick).  reset != 0 starts a new window. */
typedef struct {
  int64_t frames;   /* frames in the window */
  double p50_ms, p90_ms, p99_ms, max_ms, mean_ms;
} mf_latency_stats;

int mf_engine_latency(mf_engine* e, mf_latency_stats* out, int32_t reset);

/* Latency probe: the engine's completion stamp for work that is not an
 * engine tick, so that a caller's own per-stream loop (mf_push_frames /
 * mf_get_maps) is measured on the same clock and by the same mechanism as
 * the serving loop (the 30 FPS real-time bar of Section 2.2 is a per-frame
 * latency bound).
 *   mf_probe_stamp  enqueues on cuda_stream (a cudaStream_t; NULL: the legacy
 *                   default stream) a host function that records, when every
 *                   item queued on that stream before it has completed, the
 *                   latency of n frames: completion time minus each
 *                   arrival_ns[i] (mf_clock_ns() clock; host array, copied).
 *   mf_probe_latency  statistics of the stamps completed so far (reset != 0
 *                   starts a new window).
 * Stamps are held until read or the probe is closed; mf_probe_close waits
 * for the stamps still in flight.  A probe is not thread-safe. */
typedef struct mf_latency_probe mf_latency_probe;
int mf_probe_open(mf_latency_probe** out);
int mf_probe_stamp(mf_latency_probe* p, void* cuda_stream, int32_t n, const int64_t* arrival_ns);
int mf_probe_latency(mf_latency_probe* p, mf_latency_stats* out, int32_t reset);
int mf_probe_close(mf_latency_probe* p);

/* Wait for all ticks and free everything. */
int mf_engine_close(mf_engine* e);

/* ---------------------------------------------------------------------------
 * Serving loop: a thread-safe front end over an engine that batches frames
 * as they arrive (continuous batching).  Clients admit streams, submit
 * pushes from any thread and never call tick: a background thread launches
 * a tick as soon as work is queued (after at most tick_us of gathering)
 * while earlier ticks are still on the GPU (up to two in flight).  Pushes
 * that arrive while a stream's previous push is waiting are queued per
 * stream and go out in later ticks, in order.  Latency is measured from the
 * client's mf_server_submit to the completion of the frame's tick on the GPU.
 */
typedef struct mf_server mf_server;

typedef struct {
  mf_engine_desc engine;   /* engine limits, dtypes, budget, flags, stream */
  int32_t tick_us;         /* longest wait for more work before a tick (default 200) */
  int32_t queue_limit;     /* queued pushes per stream before NOT_READY (default 64) */
} mf_server_desc;

void mf_server_desc_init(mf_server_desc* d);
int mf_server_open(const mf_server_desc* d, mf_server** out);

/* Admission as mf_engine_add_stream (MF_ERR_ADMISSION when no slot or no
 * memory budget is left). */
int mf_server_add_stream(mf_server* s, const mf_stream_desc* d, int64_t reserve_bytes,
                         int32_t* slot);

/* Queue one push (arguments as mf_engine_submit; poses are copied now).
 * Thread-safe.  MF_ERR_NOT_READY when the stream's queue is full. */
int mf_server_submit(mf_server* s, int32_t slot, int32_t n, const double* poses_w2c_3x4,
                     const void* depth, const double* K, void* focus_map, void* guided_depth,
                     mf_frame_info* info);

/* mf_server_submit for n pushes under one lock; *accepted as in
 * mf_engine_submit_batch.  Latency statistics start at each push's
 * arrival_ns (0: the call's time). */
int mf_server_submit_batch(mf_server* s, int32_t n, const mf_push* pushes, int32_t* accepted);

/* Frames of the stream whose maps are complete on the GPU. */
int mf_server_frames_done(mf_server* s, int32_t slot, int64_t* frames);

/* Wait until every queued push of the stream is complete, then free its slot. */
int mf_server_remove_stream(mf_server* s, int32_t slot);

/* Wait until everything queued so far is complete (timeout_ns < 0: no bound). */
int mf_server_drain(mf_server* s, int64_t timeout_ns);

int mf_server_latency(mf_server* s, mf_latency_stats* out, int32_t reset);
int mf_server_get_stats(mf_server* s, mf_engine_stats* out);

/* mf_engine_tune on the server's engine (tune expected classes before
 * serving: tuning a new class at admission stalls the loop meanwhile). */
int mf_server_tune(mf_server* s, int32_t width, int32_t height, int32_t window, int32_t* band_h);

/* Stop the thread, wait for the GPU, free everything. */
int mf_server_close(mf_server* s);

/* ---------------------------------------------------------------------------
 * Allocation-free rendering.  The paper has no counterpart to this entry
 * point; it exists for callers that cannot let a library allocate device
 * memory: real-time loops that must never meet a cudaMalloc (it can
 * synchronise the device and has no latency bound), plugins running inside a
 * host framework that owns all device memory through its own pool, and
 * processes held to a fixed memory budget.
 *
 * It computes what a WORLD-pose stream would return for the last n_render of
 * n_poses consecutive poses (frames 0 .. n_poses-1; the earlier poses serve
 * as the window's history), with no mf_stream and no allocation: its
 * scratch (pose copies, rigidity flags, per-frame records and a work
 * counter, about 560 KB) is a static device array inside libmf that every
 * GPU loading the library holds until the process exits.  The caller passes and owns the inputs and
 * the outputs.
 *   d              stream descriptor: sizes, window, smooth_len, mode,
 *                  normalize, dtypes, sigma/s/d0 parameters and cuda_stream
 *                  are used; of the flags, MF_FLAG_MAP_CUDA_CORES and
 *                  MF_FLAG_MAP_TENSOR_CORES choose the map kernel as for a
 *                  stream, and the others are ignored; pose_frame must be
 *                  MF_POSES_WORLD; dev_alloc, dev_free and max_pending are
 *                  ignored.  A NULL cuda_stream here means the legacy default
 *                  stream -- unlike mf_open_stream, where NULL asks for a
 *                  library-owned stream, which this entry point would have to
 *                  create.
 *   poses_w2c_3x4  n_poses x 12 FP64 world-to-camera poses (device memory)
 *   depth          n_render depth planes of depth_dtype for frames
 *                  n_poses-n_render .. n_poses-1 (device memory) or NULL
 *   K              host pointer to fx, fy, cx, cy
 *   focus_map, guided_depth
 *                  n_render planes of map_dtype (device memory) or NULL
 *   info           n_render mf_frame_info records (device memory) or NULL
 * Limits: n_render <= MF_NOALLOC_MAX_FRAMES, n_poses <= MF_NOALLOC_MAX_POSES;
 * larger sizes, host pointers, pointers to another GPU's memory or
 * batch-local poses return MF_ERR_INVALID_ARG before any work is enqueued.  The call only enqueues
 * kernels on cuda_stream; results are ready when that stream reaches them.
 * It calls no cudaMalloc, cudaFree or other allocating routine.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call on a device shares the one array and
 * leaves its contents behind (each call rewrites all it reads), so calls whose
 * work overlaps on the GPU race: issue them on one stream, or synchronise
 * between them.
 */
#define MF_NOALLOC_MAX_FRAMES 256
#define MF_NOALLOC_MAX_POSES (MF_NOALLOC_MAX_FRAMES + MF_MAX_HISTORY - 1)

int mf_render_noalloc(const mf_stream_desc* d, int32_t n_poses, const double* poses_w2c_3x4,
                      int32_t n_render, const void* depth, const double* K, void* focus_map,
                      void* guided_depth, mf_frame_info* info);

#ifdef __cplusplus
}
#endif
#endif /* MF_H */
