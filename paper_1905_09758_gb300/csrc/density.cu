// dos_density: damped spectral histogram from Chebyshev moments (§2.2
// spectral histogram, Eq. (7)-(8) dual basis and expansion, §4.1 Jackson
// damping), plus point masses for the filtered spikes.
#include <cmath>

#include "common.cuh"

namespace netdos {
namespace {

constexpr int kMaxSpikes = 16;

struct Spikes {
  int n;
  double lam[kMaxSpikes];
  double mass[kMaxSpikes];
};

// Jackson factor g_m for an M-term series (Jackson kernel of the KPM
// literature): [(M-m+1) cos(pi m/(M+1)) + sin(pi m/(M+1)) cot(pi/(M+1))]/(M+1)
__device__ double jackson_g(int m, int M) {
  const double a = M_PI / (M + 1.0);
  return ((M - m + 1.0) * cos(a * m) + sin(a * m) / tan(a)) / (M + 1.0);
}

// One CTA.  coef[m] folds the damping, the factor 2 of the m >= 1 terms and
// the 1/(m pi) of the bin integral; bin b then gets
//   coef[0] (theta_a - theta_b) + sum_{m>=1} coef[m] (sin(m theta_a) - sin(m theta_b)).
__global__ void k_density(const double* __restrict__ d, int M, int B, int kernel, double scale, Spikes sp,
                          double* __restrict__ h) {
  extern __shared__ double coef[];
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    const double g = kernel == DOS_KERNEL_JACKSON ? jackson_g(m, M) : 1.0;
    coef[m] = m == 0 ? g * d[0] / M_PI : 2.0 * g * d[m] / (m * M_PI);
  }
  __syncthreads();
  const double w = 2.0 / B;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double lo = -1.0 + w * b;
    const double hi = b + 1 == B ? 1.0 : -1.0 + w * (b + 1);
    const double ta = acos(lo), tb = acos(hi);
    double s = coef[0] * (ta - tb);
    for (int m = 1; m < M; ++m) s += coef[m] * (sin(m * ta) - sin(m * tb));
    s *= scale;
    for (int k = 0; k < sp.n; ++k) {
      const double x = fmin(fmax(sp.lam[k], -1.0), 1.0);
      const int e = static_cast<int>(rint((x + 1.0) / w));
      if (e > 0 && e < B && fabs(x - (-1.0 + w * e)) <= 1e-9) {
        if (b == e - 1 || b == e) s += 0.5 * sp.mass[k];
      } else {
        int bb = static_cast<int>(floor((x + 1.0) / w));
        bb = bb < 0 ? 0 : (bb >= B ? B - 1 : bb);
        if (b == bb) s += sp.mass[k];
      }
    }
    h[b] = s;
  }
}

}  // namespace
}  // namespace netdos

using namespace netdos;

extern "C" int dos_density(const double* d, int M, int n_bins, int kernel, double scale, const double* spikes,
                           int n_spikes, double* hist_out, void* stream) {
  clear_error();
  if (!d || !hist_out) return fail(DOS_EINVAL, "dos_density: null pointer");
  if (M < 1 || M > 16384) return fail(DOS_EINVAL, "dos_density: M must be in [1, 16384]");
  if (n_bins < 1 || n_bins > (1 << 20)) return fail(DOS_EINVAL, "dos_density: n_bins must be in [1, 2^20]");
  if (kernel != DOS_KERNEL_NONE && kernel != DOS_KERNEL_JACKSON) return fail(DOS_EINVAL, "dos_density: kernel");
  if (n_spikes < 0 || n_spikes > kMaxSpikes || (n_spikes > 0 && !spikes))
    return fail(DOS_EINVAL, "dos_density: at most 16 spikes");
  Spikes sp{};
  sp.n = n_spikes;
  for (int k = 0; k < n_spikes; ++k) {
    sp.lam[k] = spikes[2 * k];
    sp.mass[k] = spikes[2 * k + 1];
  }
  const size_t smem = sizeof(double) * static_cast<size_t>(M);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (smem > 48 * 1024) NDOS_CUDA(cudaFuncSetAttribute(k_density, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       static_cast<int>(smem)));
  k_density<<<1, 256, smem, s>>>(d, M, n_bins, kernel, scale, sp, hist_out);
  NDOS_LAUNCHED();
  return DOS_OK;
}
