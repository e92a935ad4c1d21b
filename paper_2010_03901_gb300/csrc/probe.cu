// FP64 throughput probe: independent fused multiply-add chains on every SM, for the
// measured FP64 peak that the Fourier Forwarding line's roofline divides by.  Not an
// operation of the method.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fc2d.h"
#include "plan_internal.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_probe_dfma(double* out, int64_t iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" fc2d_status fc2d_probe_fp64(double* out_dev, int blocks, int64_t iters,
                                       double* flops, void* stream) {
  if (!out_dev || blocks < 1 || iters < 1 || !flops)
    return fc2d::set_error(FC2D_ERR_ARG, "fc2d_probe_fp64: bad argument");
  k_probe_dfma<<<blocks, 256, 0, (cudaStream_t)stream>>>(out_dev, iters, 0.9999999, 1e-7);
  *flops = 2.0 * kChains * (double)iters * blocks * 256.0;
  return fc2d::cuda_check(cudaGetLastError(), "fc2d_probe_fp64");
}
