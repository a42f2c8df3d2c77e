// FP32 instantiation of the WBRW kernels in tangent mode: the 2D model with
// likelihood-ratio tangent weights (d/dH, d/dw) on every particle.
#include "wbrw_device.cuh"

namespace wbrw {
const Driver* driver_fp32_grad() { return DriverImpl<P32G>::get(); }
}  // namespace wbrw
