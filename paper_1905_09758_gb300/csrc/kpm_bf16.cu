// Chebyshev step kernels with __nv_bfloat16 probe-block storage (FP32 arithmetic).
#include "kpm_kernels.cuh"

namespace netdos {

template int launch_step<__nv_bfloat16>(const Plan&, int, const StepParams&, cudaStream_t, const SideStreams&);
template int step_config<__nv_bfloat16>(int, int, int*, int*);
template int launch_init<__nv_bfloat16>(const InitParams&, int, cudaStream_t);

}  // namespace netdos
