// wbrw_probe.cu -- the integer-pipe ceiling of the hot path's random numbers.
//
// The flight and event kernels draw every random number from Philox4x32-10
// calls (philox_ks in wbrw_device.cuh) and spend most of their integer work
// there.  This kernel runs that same call in a dependent chain (each call's
// output is the next call's counter), with nothing else around it, on every
// resident thread of the GPU.  Its call rate is the most Philox calls per
// second the hot path could ever make, the denominator of the integer-bound
// kernels' roofline.
#include "wbrw_device.cuh"

namespace wbrw {
namespace {

__global__ void __launch_bounds__(kBlock) k_philox_chain(const KeySched ks, int iters,
                                                         unsigned long long nthreads,
                                                         uint32_t* out) {
  const unsigned long long t = (unsigned long long)blockIdx.x * kBlock + threadIdx.x;
  if (t >= nthreads) return;
  uint32_t c0 = (uint32_t)t, c1 = (uint32_t)(t >> 32), c2 = 0u, c3 = 0u;
  for (int i = 0; i < iters; ++i) {
    const uint4 r = philox_ks(ks, c0, c1, c2, c3);
    c0 = r.x;
    c1 = r.y;
    c2 = r.z;
    c3 = r.w;
  }
  out[t] = c0 ^ c1 ^ c2 ^ c3;  // keeps the chain live; 4 bytes per thread
}

}  // namespace
}  // namespace wbrw

extern "C" wbrw_status wbrw_philox_chain(unsigned long long seed, int iters,
                                         long long nthreads, unsigned int* out,
                                         void* cuda_stream) {
  if (iters < 1 || nthreads < 1 || nthreads > (1ll << 40) || !out) return WBRW_ERR_ARG;
  cudaPointerAttributes a;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WBRW_ERR_CUDA;
  if (cudaPointerGetAttributes(&a, out) != cudaSuccess) {
    cudaGetLastError();
    return WBRW_ERR_ARG;
  }
  if (!(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) || a.device != dev)
    return WBRW_ERR_ARG;
  wbrw::KeySched ks;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    ks.k0[r] = k0;
    ks.k1[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  const unsigned long long blocks = ((unsigned long long)nthreads + wbrw::kBlock - 1) / wbrw::kBlock;
  if (blocks > 0x7FFFFFFFull) return WBRW_ERR_ARG;
  wbrw::k_philox_chain<<<(unsigned)blocks, wbrw::kBlock, 0, (cudaStream_t)cuda_stream>>>(
      ks, iters, (unsigned long long)nthreads, out);
  return cudaGetLastError() == cudaSuccess ? WBRW_OK : WBRW_ERR_CUDA;
}
