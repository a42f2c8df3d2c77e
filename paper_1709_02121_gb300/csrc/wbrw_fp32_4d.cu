// FP32 instantiation of the WBRW kernels for the 4D model (two electrons):
// the production path of the Helium-like system.
#include "wbrw_device.cuh"

namespace wbrw {
const Driver* driver_fp32_4d() { return DriverImpl<Q32>::get(); }
}  // namespace wbrw
