// FP32 instantiation of the WBRW kernels: the production path.
#include "wbrw_device.cuh"

namespace wbrw {
const Driver* driver_fp32() { return DriverImpl<P32>::get(); }
}  // namespace wbrw
