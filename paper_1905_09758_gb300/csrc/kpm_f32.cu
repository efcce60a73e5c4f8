// Chebyshev step kernels with float probe-block storage (FP32 arithmetic).
#include "kpm_kernels.cuh"

namespace netdos {

template int launch_step<float>(const Plan&, int, const StepParams&, cudaStream_t, const SideStreams&);
template int step_config<float>(int, int, int*, int*);
template int launch_init<float>(const InitParams&, int, cudaStream_t);

}  // namespace netdos
