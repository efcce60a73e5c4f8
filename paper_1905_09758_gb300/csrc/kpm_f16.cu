// Chebyshev step kernels with __half probe-block storage (FP32 arithmetic).
#include "kpm_kernels.cuh"

namespace netdos {

template <>
int step_occupancy<__half>(const Plan& plan) {
  int blocks = 0;
  // the step kernels of one storage type share their register footprint
  // closely; the Q = 1, P = 1 DOS variant stands in for all of them
  (void)plan;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_cheb_step<__half, 1, 1, kModeDos>, kStepThreads, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 2;
  }
  return blocks > 0 ? blocks : 1;
}

template int launch_step<__half>(const Plan&, int, const StepParams&, cudaStream_t);
template int launch_init<__half>(const InitParams&, int, cudaStream_t);

}  // namespace netdos
