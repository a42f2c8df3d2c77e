// FP32 instantiation in tangent mode for runs (plain or batched) with the
// static potential and no event log.
#include "wbrw_device.cuh"

namespace wbrw {
const Driver* driver_fp32_grad_lean() { return DriverImpl<P32GL>::get(); }
}  // namespace wbrw
