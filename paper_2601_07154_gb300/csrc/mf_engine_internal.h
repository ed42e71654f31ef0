// Tick tables shared by the engine host code (mf_engine.cpp) and its batched
// kernels (mf_engine_kernels.cu).  Not part of the public ABI.
#pragma once

#include <vector>

#include "mf_internal.h"
#include "mf_pose_device.cuh"

namespace mf {

// Two map paths: every stream can take the 32-point path with 2 columns per
// lane; streams with windows up to 16 points and widths divisible by the
// 16-point path's columns per lane take that path (16-bit maps: 4 columns
// per lane, fewer instructions per pixel; FP32 maps: 2, whose smaller unit
// fits three CTAs per SM).
constexpr int kEngineCPT = 2;                           // columns per lane, 32-point path
constexpr int kEngineWideNMAX = 16;
__host__ __device__ constexpr int engine_wide_cpt(int map_bytes) { return map_bytes == 4 ? 2 : 4; }
constexpr int kEnginePaths = 2;                         // 0: 32-point, 1: 16-point

// Per admitted stream, written once at admission (device array by slot).
struct SlotParams {
  double* ring;            // resident pose history, ring_mask+1 slots x 12
  int32_t* ring_bad;
  int64_t ring_mask;
  FrameParams fp;
  float d0;
  int32_t pad;
  double w[kMaxHist];      // least-squares weights
};

// One push of one stream in a tick.
struct TickPush {
  int32_t slot;
  int32_t n;               // poses in the push
  int32_t first;           // first emitted pose (overlap or 0)
  int32_t anchor;          // gravity-locked anchoring against the history
  int64_t e0;              // stream's emitted count before the push
  int64_t pose_off;        // index of the push's first pose in the tick's pose block
  double K[4];
};

// One emitted frame of a tick (frames of a push are consecutive).
struct TickFrame {
  int32_t push;            // index into the tick's pushes
  int32_t k;               // emitted offset within the push
  int32_t bucket;          // window of the stream (informational)
  int32_t path;            // map path (0: 32-point, 1: 16-point wide)
  int32_t pad;
  int32_t band_h;          // tile height (autotuned per resolution class)
  int32_t groups_x;        // strip groups across the frame
  int32_t bands;
  int64_t unit_begin;      // first map unit of the frame
  const char* depth;       // depth plane (device) or NULL
  char* M;                 // focus-map plane (device) or NULL
  char* G;                 // guided-depth plane (device) or NULL
  mf_frame_info* info;     // record (device) or NULL
};

// Layout of one tick table (header, frames, path order, pushes, poses; each
// 256-B aligned).  The path order lists the frame indices of path 0, then
// those of path 1; unit_begin counts within the frame's path.
struct TickHeader {
  int32_t n_frames, n_pushes;
  int64_t n_units;                             // both paths
  int64_t frames_off, order_off, pushes_off, poses_off;  // byte offsets from the header
  int64_t n_units_path[kEnginePaths];
  int32_t n_frames_path[kEnginePaths];
};

// Persistent grid of each path's map kernel.
struct EngineGrids {
  int g[kEnginePaths];
};

struct EngineKernelArgs {
  const TickHeader* table;     // device tick table
  const SlotParams* slots;     // device slot parameters
  FrameRec* recs;              // max_tick_frames records
  int max_frames;              // capacity (grid sizes of the per-frame kernels)
  // one work counter per map path for the dynamic unit schedule (0 between
  // launches; the two paths run concurrently, so each has its own)
  unsigned int* sched;         // [kEnginePaths]
  unsigned int* fault;         // checked builds: set on an access outside a plane
};

// Kernel launches of one tick: ingest, points, the two map paths, finalize.
// The two map paths run concurrently: the 16-point path on `side`, forked
// from and joined back into `st` through the two events.
constexpr int kEngineTickLaunches = 5;
struct EngineFork {
  cudaStream_t side;
  cudaEvent_t fork, join;
};
cudaError_t launch_engine_tick(const EngineKernelArgs& a, int depth_dtype, int map_dtype,
                               const EngineGrids& grids, cudaStream_t st, const EngineFork& fk,
                               int64_t* launches);
// Resident CTAs per SM x SMs for each path's batched map kernel of a dtype pair.
EngineGrids engine_map_grids(int depth_dtype, int map_dtype);
// Runs both map paths over the given table (already on the device).
cudaError_t launch_engine_map_only(const EngineKernelArgs& a, int depth_dtype, int map_dtype,
                                   const EngineGrids& grids, cudaStream_t st);

// mf_engine_submit with an explicit submit time (steady-clock ns) for the
// latency statistics; the serving loop passes its clients' submit times.
int engine_submit_at(mf_engine* e, int32_t slot, int32_t n, const double* poses, const void* depth,
                     const double* K, void* focus_map, void* guided_depth, mf_frame_info* info,
                     int64_t submit_ns);
int64_t engine_now_ns();
// p50 / p90 / p99 / max / mean (nearest rank) of latencies in milliseconds.
void latency_summary(const std::vector<double>& latencies_ms, mf_latency_stats* out);

}  // namespace mf
