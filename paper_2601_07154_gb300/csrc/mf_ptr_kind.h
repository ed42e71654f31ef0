// Classification of a caller's pointer for work on one device, from the
// fields cudaPointerGetAttributes reports (kept free of CUDA headers so that
// host-only tests can compile it).
#pragma once

namespace mf {

// Where a pointer lives, for work launched on device `dev`.
constexpr int kPtrHost = 0;         // pageable or page-locked host memory
constexpr int kPtrDevice = 1;       // device memory of `dev`, or managed memory
constexpr int kPtrOtherDevice = 2;  // device memory of another GPU: refused

// memory_type: the cudaMemoryType value (0 unregistered, 1 host, 2 device,
// 3 managed); attr_device: the attribute's device ordinal.
inline int classify_pointer(int memory_type, int attr_device, int dev) {
  if (memory_type == 3) return kPtrDevice;
  if (memory_type == 2) return attr_device == dev ? kPtrDevice : kPtrOtherDevice;
  return kPtrHost;
}

}  // namespace mf
