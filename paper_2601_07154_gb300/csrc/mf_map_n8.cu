// The per-pixel map kernels for windows of up to 8 points, every
// storage type pair (instantiated here so the build compiles the window
// buckets in parallel).
#include "mf_map_kernel.cuh"

namespace mf {
namespace mapk {
template cudaError_t launch_n<8>(const MapParams&, int, int, bool, cudaStream_t, int64_t*);
}  // namespace mapk
}  // namespace mf
