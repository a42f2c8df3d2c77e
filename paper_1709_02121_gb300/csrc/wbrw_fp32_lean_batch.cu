// FP32 instantiation for batches with the static potential and no event log.
#include "wbrw_device.cuh"

namespace wbrw {
const Driver* driver_fp32_lean_batch() { return DriverImpl<P32LB>::get(); }
}  // namespace wbrw
