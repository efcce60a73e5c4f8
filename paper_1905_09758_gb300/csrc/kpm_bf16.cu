// Chebyshev step kernels with __nv_bfloat16 probe-block storage (FP32 arithmetic).
#include "kpm_kernels.cuh"

namespace netdos {

template <>
int step_occupancy<__nv_bfloat16>(const Plan& plan) {
  int blocks = 0;
  // the step kernels of one storage type share their register footprint
  // closely; the Q = 1, P = 1 DOS variant stands in for all of them
  (void)plan;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_cheb_step<__nv_bfloat16, 1, 1, kModeDos>, kStepThreads, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 2;
  }
  return blocks > 0 ? blocks : 1;
}

template int launch_step<__nv_bfloat16>(const Plan&, int, const StepParams&, cudaStream_t);
template int launch_init<__nv_bfloat16>(const InitParams&, int, cudaStream_t);

}  // namespace netdos
