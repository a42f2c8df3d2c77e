// FP64 instantiation of the WBRW kernels in tangent mode: the 2D model with
// likelihood-ratio tangent weights (d/dH, d/dw) on every particle.
#include "wbrw_device.cuh"

namespace wbrw {
const Driver* driver_fp64_grad() { return DriverImpl<P64G>::get(); }
}  // namespace wbrw
