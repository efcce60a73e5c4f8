// Chebyshev step kernels with float probe-block storage (FP32 arithmetic).
#include "kpm_kernels.cuh"

namespace netdos {

template <>
int step_occupancy<float>(const Plan& plan) {
  int blocks = 0;
  // the step kernels of one storage type share their register footprint
  // closely; the Q = 1, P = 1 DOS variant stands in for all of them
  (void)plan;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_cheb_step<float, 1, 1, kModeDos>, kStepThreads, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 2;
  }
  return blocks > 0 ? blocks : 1;
}

template int launch_step<float>(const Plan&, int, const StepParams&, cudaStream_t);
template int launch_init<float>(const InitParams&, int, cudaStream_t);

}  // namespace netdos
