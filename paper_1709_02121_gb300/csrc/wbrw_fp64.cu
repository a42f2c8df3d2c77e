// FP64 instantiation of the WBRW kernels: the parity path, whose arithmetic
// follows the oracle's operation order exactly.
#include "wbrw_device.cuh"

namespace wbrw {
const Driver* driver_fp64() { return DriverImpl<P64>::get(); }
}  // namespace wbrw
