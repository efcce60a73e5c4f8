// dos_density: damped spectral histogram from Chebyshev moments (§2.2
// spectral histogram, Eq. (7)-(8) dual basis and expansion, §4.1 Jackson
// damping), plus point masses for the filtered spikes.
#include <algorithm>
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"

namespace netdos {
namespace {

constexpr int kMaxSpikes = 64;

struct Spikes {
  int n;
  double lam[kMaxSpikes];
  double mass[kMaxSpikes];
};

// Mass that the point masses put into bin b of B equal bins over [-1, 1]: a
// point within 1e-9 of an interior edge splits evenly between the two bins,
// points at or beyond +-1 go to the end bins.
__device__ double spike_mass(const Spikes& sp, int b, int B) {
  const double w = 2.0 / B;
  double v = 0.0;
  for (int k = 0; k < sp.n; ++k) {
    const double x = fmin(fmax(sp.lam[k], -1.0), 1.0);
    const int e = static_cast<int>(rint((x + 1.0) / w));
    if (e > 0 && e < B && fabs(x - (-1.0 + w * e)) <= 1e-9) {
      if (b == e - 1 || b == e) v += 0.5 * sp.mass[k];
    } else {
      int bb = static_cast<int>(floor((x + 1.0) / w));
      bb = bb < 0 ? 0 : (bb >= B ? B - 1 : bb);
      if (b == bb) v += sp.mass[k];
    }
  }
  return v;
}

// hist[r][b] = scale * probs[r][b] + spike masses (learned densities)
__global__ void k_hist_assemble(const float* __restrict__ probs, int B, int64_t rows, double scale, Spikes sp,
                                double* __restrict__ h) {
  const int64_t total = rows * B;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    h[i] = scale * static_cast<double>(probs[i]) + spike_mass(sp, static_cast<int>(i % B), B);
}

// Jackson factor g_m for an M-term series (Jackson kernel of the KPM
// literature): [(M-m+1) cos(pi m/(M+1)) + sin(pi m/(M+1)) cot(pi/(M+1))]/(M+1)
__device__ double jackson_g(int m, int M) {
  const double a = M_PI / (M + 1.0);
  return ((M - m + 1.0) * cos(a * m) + sin(a * m) / tan(a)) / (M + 1.0);
}

// One CTA per bin b (and per graph blockIdx.y of a batch): thread i sums the terms m = i, i + blockDim, ... of
//   coef[m] (sin(m theta_a) - sin(m theta_b))   (m >= 1; theta_a - theta_b for m = 0),
// coef[m] folding the damping, the factor 2 of the m >= 1 terms and the
// 1/(m pi) of the exact bin integral; the partial sums are combined in a
// fixed tree order, so the result is deterministic.
__global__ void __launch_bounds__(256) k_density(const double* __restrict__ d, int M, int B, int kernel, double scale,
                                                 Spikes sp, double* __restrict__ h) {
  __shared__ double red[256];
  const int b = blockIdx.x;
  d += static_cast<size_t>(blockIdx.y) * M;  // graph blockIdx.y of a batch
  h += static_cast<size_t>(blockIdx.y) * B;
  const double w = 2.0 / B;
  const double lo = -1.0 + w * b;
  const double hi = b + 1 == B ? 1.0 : -1.0 + w * (b + 1);
  const double ta = acos(lo), tb = acos(hi);
  double s = 0.0;
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    const double g = kernel == DOS_KERNEL_JACKSON ? jackson_g(m, M) : 1.0;
    if (m == 0)
      s += g * d[0] / M_PI * (ta - tb);
    else
      s += 2.0 * g * d[m] / (m * M_PI) * (sin(m * ta) - sin(m * tb));
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) h[b] = scale * red[0] + spike_mass(sp, b, B);
}

}  // namespace
}  // namespace netdos

using namespace netdos;

static int read_spikes(const double* spikes, int n_spikes, Spikes* sp, const char* who) {
  if (n_spikes < 0 || n_spikes > kMaxSpikes || (n_spikes > 0 && !spikes))
    return fail(DOS_EINVAL, std::string(who) + ": at most 64 spikes");
  *sp = Spikes{};
  sp->n = n_spikes;
  for (int k = 0; k < n_spikes; ++k) {
    sp->lam[k] = spikes[2 * k];
    sp->mass[k] = spikes[2 * k + 1];
  }
  return DOS_OK;
}

static int density_launch(const double* d, int M, int n_bins, int kernel, double scale, const Spikes& sp,
                          double* hist_out, cudaStream_t s, const char* who) {
  if (!d || !hist_out) return fail(DOS_EINVAL, std::string(who) + ": null pointer");
  if (M < 1 || M > (1 << 20)) return fail(DOS_EINVAL, std::string(who) + ": M must be in [1, 2^20]");
  if (n_bins < 1 || n_bins > (1 << 20)) return fail(DOS_EINVAL, std::string(who) + ": n_bins must be in [1, 2^20]");
  if (kernel != DOS_KERNEL_NONE && kernel != DOS_KERNEL_JACKSON) return fail(DOS_EINVAL, std::string(who) + ": kernel");
  k_density<<<n_bins, 256, 0, s>>>(d, M, n_bins, kernel, scale, sp, hist_out);
  NDOS_LAUNCHED();
  return DOS_OK;
}

// Weight of the series part and the point masses of a whole-graph density
// (§3.4 filtered density; nodes without edges carry the eigenvalue 0):
//   N_total = N + n_isolated (counting isolated nodes) or N,
//   scale   = r / N_total, r = N - removed (N without a filter),
//   spikes  = every eigenvalue the filter removed, with isolated nodes added
//             at 0, as (lambda, count / N_total) in ascending lambda.
static int density_weights(const Graph* G, const Filter* F, uint32_t flags, double* scale,
                           std::vector<std::pair<double, int64_t>>* eigs, double* n_total) {
  if (F && !G) G = F->g;
  if (F && F->g != G) return fail(DOS_EINVAL, "dos_density: the filter belongs to another graph");
  if (flags & ~static_cast<uint32_t>(DOS_DENSITY_COUNT_ISOLATED)) return fail(DOS_EINVAL, "dos_density: unknown flags");
  eigs->clear();
  if (!G) {
    *scale = 1.0;
    *n_total = 0.0;
    return DOS_OK;
  }
  const int64_t iso = (flags & DOS_DENSITY_COUNT_ISOLATED) ? G->n_isolated : 0;
  const int64_t total = G->n + iso;
  if (total < 1) return fail(DOS_EINVAL, "dos_density: the graph has no nodes");
  const int64_t removed = F ? F->removed : 0;
  if (F) *eigs = F->spikes;  // ascending lambda
  if (iso > 0) {
    auto it = std::find_if(eigs->begin(), eigs->end(), [](const std::pair<double, int64_t>& e) { return e.first >= 0.0; });
    if (it != eigs->end() && it->first == 0.0)
      it->second += iso;
    else
      eigs->insert(it, {0.0, iso});
  }
  eigs->erase(std::remove_if(eigs->begin(), eigs->end(), [](const std::pair<double, int64_t>& e) { return e.second == 0; }),
              eigs->end());
  *scale = static_cast<double>(G->n - removed) / static_cast<double>(total);
  *n_total = static_cast<double>(total);
  return DOS_OK;
}

extern "C" int dos_density(const double* d, int M, int n_bins, int kernel, dos_graph_t g, dos_filter_t f,
                           uint32_t flags, double* hist_out, void* stream) {
  clear_error();
  double scale = 1.0, n_total = 0.0;
  std::vector<std::pair<double, int64_t>> eigs;
  NDOS_CHECK(density_weights(reinterpret_cast<const Graph*>(g), reinterpret_cast<const Filter*>(f), flags, &scale,
                             &eigs, &n_total));
  if (static_cast<int>(eigs.size()) > kMaxSpikes) return fail(DOS_EINVAL, "dos_density: more than 64 distinct spikes");
  Spikes sp{};
  sp.n = static_cast<int>(eigs.size());
  for (int k = 0; k < sp.n; ++k) {
    sp.lam[k] = eigs[k].first;
    sp.mass[k] = static_cast<double>(eigs[k].second) / n_total;
  }
  return density_launch(d, M, n_bins, kernel, scale, sp, hist_out, static_cast<cudaStream_t>(stream), "dos_density");
}

extern "C" int dos_density_weights(dos_graph_t g, dos_filter_t f, uint32_t flags, double* scale_out,
                                   double* spikes_out, int capacity, int* n_spikes) {
  clear_error();
  if (!g && !f) return fail(DOS_EINVAL, "dos_density_weights: no graph and no filter");
  if (capacity < 0 || (capacity > 0 && !spikes_out)) return fail(DOS_EINVAL, "dos_density_weights: bad buffer");
  double scale = 1.0, n_total = 0.0;
  std::vector<std::pair<double, int64_t>> eigs;
  NDOS_CHECK(density_weights(reinterpret_cast<const Graph*>(g), reinterpret_cast<const Filter*>(f), flags, &scale,
                             &eigs, &n_total));
  if (scale_out) *scale_out = scale;
  if (n_spikes) *n_spikes = static_cast<int>(eigs.size());
  for (int k = 0; k < static_cast<int>(eigs.size()) && k < capacity; ++k) {
    spikes_out[2 * k] = eigs[k].first;
    spikes_out[2 * k + 1] = static_cast<double>(eigs[k].second) / n_total;
  }
  return DOS_OK;
}

extern "C" int dos_density_raw(const double* d, int M, int n_bins, int kernel, double scale, const double* spikes,
                               int n_spikes, double* hist_out, void* stream) {
  clear_error();
  Spikes sp{};
  NDOS_CHECK(read_spikes(spikes, n_spikes, &sp, "dos_density_raw"));
  return density_launch(d, M, n_bins, kernel, scale, sp, hist_out, static_cast<cudaStream_t>(stream),
                        "dos_density_raw");
}

extern "C" int dos_density_batched(const double* d, int M, int64_t n_graphs, int n_bins, int kernel,
                                   double* hist_out, void* stream) {
  clear_error();
  if (!d || !hist_out) return fail(DOS_EINVAL, "dos_density_batched: null pointer");
  if (M < 1 || M > (1 << 20)) return fail(DOS_EINVAL, "dos_density_batched: M must be in [1, 2^20]");
  if (n_bins < 1 || n_bins > (1 << 20)) return fail(DOS_EINVAL, "dos_density_batched: n_bins must be in [1, 2^20]");
  if (n_graphs < 1) return fail(DOS_EINVAL, "dos_density_batched: n_graphs must be >= 1");
  if (kernel != DOS_KERNEL_NONE && kernel != DOS_KERNEL_JACKSON) return fail(DOS_EINVAL, "dos_density_batched: kernel");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  constexpr int64_t kMaxY = 65535;
  for (int64_t g0 = 0; g0 < n_graphs; g0 += kMaxY) {
    const int64_t ng = n_graphs - g0 < kMaxY ? n_graphs - g0 : kMaxY;
    k_density<<<dim3(n_bins, static_cast<unsigned>(ng)), 256, 0, s>>>(d + g0 * M, M, n_bins, kernel, 1.0, Spikes{},
                                                                       hist_out + g0 * n_bins);
    NDOS_LAUNCHED();
  }
  return DOS_OK;
}

extern "C" int dos_hist_assemble(const float* probs, int n_bins, int64_t rows, double scale, const double* spikes,
                                 int n_spikes, double* hist_out, void* stream) {
  clear_error();
  if (!probs || !hist_out) return fail(DOS_EINVAL, "dos_hist_assemble: null pointer");
  if (n_bins < 1 || n_bins > (1 << 20) || rows < 1) return fail(DOS_EINVAL, "dos_hist_assemble: bad sizes");
  Spikes sp{};
  NDOS_CHECK(read_spikes(spikes, n_spikes, &sp, "dos_hist_assemble"));
  const int64_t total = rows * n_bins;
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((total + 255) / 256, 152 * 16));
  k_hist_assemble<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(probs, n_bins, rows, scale, sp, hist_out);
  NDOS_LAUNCHED();
  return DOS_OK;
}
