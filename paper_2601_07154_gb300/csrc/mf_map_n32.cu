// The per-pixel map kernels for windows of 17 to 32 points, every
// storage type pair (instantiated here so the build compiles the window
// buckets in parallel).
#include "mf_map_kernel.cuh"

namespace mf {
namespace mapk {
template cudaError_t launch_n<32>(const MapParams&, int, int, bool, cudaStream_t, int64_t*);
}  // namespace mapk
}  // namespace mf
