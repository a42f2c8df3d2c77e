// FP64 instantiation of the WBRW kernels for the 4D model (two electrons):
// the parity path of the Helium-like system.
#include "wbrw_device.cuh"

namespace wbrw {
const Driver* driver_fp64_4d() { return DriverImpl<Q64>::get(); }
}  // namespace wbrw
