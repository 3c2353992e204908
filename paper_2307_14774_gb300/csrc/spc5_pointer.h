// Where a vector argument lives, from the CUDA runtime's pointer attributes.
// Kept free of CUDA calls so the decision can be checked on a machine
// without a GPU.
#pragma once

namespace spc5 {

enum class Placement { kHost, kDevice, kOtherDevice };

// memory_type: cudaPointerAttributes::type (0 unregistered host memory,
// 1 page-locked host memory, 2 device memory, 3 managed memory), or -1 when
// the runtime did not recognise the pointer (plain host memory);
// attr_device: cudaPointerAttributes::device; want_device: the ordinal the
// matrix lives on.  Device memory of another GPU is rejected rather than
// read through a peer mapping that may not exist; managed memory is
// readable from any device.
inline Placement placement_of(int memory_type, int attr_device, int want_device) {
  if (memory_type == 2) return attr_device == want_device ? Placement::kDevice : Placement::kOtherDevice;
  if (memory_type == 3) return Placement::kDevice;
  return Placement::kHost;
}

}  // namespace spc5
