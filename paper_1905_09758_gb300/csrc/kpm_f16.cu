// Chebyshev step kernels with __half probe-block storage (FP32 arithmetic).
#include "kpm_kernels.cuh"

namespace netdos {

template int launch_step<__half>(const Plan&, int, const StepParams&, cudaStream_t, const SideStreams&);
template int step_config<__half>(int, int, int*, int*);
template int launch_init<__half>(const InitParams&, int, cudaStream_t);

}  // namespace netdos
