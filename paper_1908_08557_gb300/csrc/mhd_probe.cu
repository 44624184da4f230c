// mhd_probe.cu -- arithmetic throughput probe of the device (instrumentation
// for the rooflines of the ALU-bound kernels, not a step of the method): every
// thread runs eight independent fused multiply-add chains, so the FMA pipe of
// the precision R is kept busy without memory traffic.
#include "mhd_internal.h"

namespace mhd {

template <typename R>
__global__ void __launch_bounds__(256) fma_probe_kernel(R* out, int iters, R a, R b) {
  R x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = R(threadIdx.x + c) * R(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  R s = R(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  // the values stay finite and positive; the store keeps the chains alive
  if (s < R(0)) out[blockIdx.x] = s;
}

template <typename R>
void launch_fma_probe(R* out, int grid, int iters, cudaStream_t st) {
  fma_probe_kernel<R><<<grid, 256, 0, st>>>(out, iters, R(0.999999), R(1e-6));
}

template void launch_fma_probe<float>(float*, int, int, cudaStream_t);
template void launch_fma_probe<double>(double*, int, int, cudaStream_t);

}  // namespace mhd
