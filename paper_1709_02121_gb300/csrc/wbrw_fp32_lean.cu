// FP32 instantiation for runs with one instance, the static potential and no
// event log: the production path of the plain 2D workloads.
#include "wbrw_device.cuh"

namespace wbrw {
const Driver* driver_fp32_lean() { return DriverImpl<P32L>::get(); }
}  // namespace wbrw
