// Traces and diagonals of matrix functions from (L)DOS moments (§6: the
// centralities and connectivity indices written as traces and diagonals of
// f(X); Eq. (5) shift and scale; Eq. (10)-(12) LDOS moments).
//
// With X~ = (X - c) / r on [-1, 1] and f(c + r x) = sum_m g_m T_m(x):
//   tr f(X)  = N sum_m g_m d_m  (+ f(0) = 1 per node without edges),
//   f(X)_kk  = sum_m g_m C[m][k].
// The coefficients g_m are Chebyshev interpolation coefficients at K =
// max(4M, 256) Chebyshev-Gauss points.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace netdos {
namespace {

__device__ __forceinline__ double fn_value(int fn, double p, double x) {
  return fn == DOS_FN_EXP ? exp(p * x) : 1.0 / (1.0 - p * x);
}

// g_m = (2 - [m = 0]) / K sum_j f(c + r cos t_j) cos(m t_j), t_j = pi (j + 1/2) / K;
// one thread per m, the sum in j order.  cos(m t_j) = cospi(m (2j + 1) / (2K))
// with the integer m (2j + 1) reduced modulo 4K first.
__global__ void k_fn_coeffs(int fn, double p, double c, double r, int m_count, int kpts, double* __restrict__ g) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= m_count) return;
  const int64_t period = 4LL * kpts;
  double s = 0.0;
  for (int j = 0; j < kpts; ++j) {
    const double x = cospi((2.0 * j + 1.0) / (2.0 * kpts));
    const int64_t a = (static_cast<int64_t>(m) * (2 * j + 1)) % period;
    s += fn_value(fn, p, c + r * x) * cospi(static_cast<double>(a) / (2.0 * kpts));
  }
  g[m] = (m == 0 ? 1.0 : 2.0) * s / kpts;
}

// out = n sum_m g_m d_m + n_iso: strided partial sums, then a fixed tree
__global__ void k_fn_trace(const double* __restrict__ g, const double* __restrict__ d, int m_count, double n,
                           double n_iso, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int m = threadIdx.x; m < m_count; m += blockDim.x) s += g[m] * d[m];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = n * red[0] + n_iso;
}

constexpr int kDiagThreads = 256;
constexpr int kDiagWarps = kDiagThreads / 32;
constexpr int kDiagChunk = 2048;  // coefficients staged in shared memory at a time
constexpr int kDiagUnroll = 4;    // independent row loads in flight per thread

// out[k] = s sum_m (g_m / s) C[m][k], s = max |g_m| (FP32 products and sums of
// the scaled coefficients: no overflow for large f, FP32 FMA throughput; the
// scale is applied in FP64).  Each thread owns VEC consecutive nodes (VEC = 4:
// 16-byte loads, n % 4 == 0 and C 16-byte aligned; VEC = 1: ragged n) and
// runs over all rows m, so a CTA reads 256 VEC contiguous floats of each row.
// At most 32 registers: eight CTAs per SM are resident, so n = 1.1M nodes
// (1074 CTAs) run in one wave.
template <int VEC>
__global__ void __launch_bounds__(kDiagThreads, 8) k_fn_diag(const float* __restrict__ C, int64_t n, int m_count,
                                                             const double* __restrict__ g, double* __restrict__ out) {
  __shared__ float gs[kDiagChunk];
  __shared__ double s_max[kDiagWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double mx = 0.0;
  for (int m = threadIdx.x; m < m_count; m += kDiagThreads) mx = fmax(mx, fabs(g[m]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_max[warp] = mx;
  __syncthreads();
  mx = 0.0;
#pragma unroll
  for (int w = 0; w < kDiagWarps; ++w) mx = fmax(mx, s_max[w]);
  const double scale = mx > 0.0 ? mx : 1.0;
  const int64_t k0 = (static_cast<int64_t>(blockIdx.x) * kDiagThreads + threadIdx.x) * VEC;
  const bool live = k0 < n;  // n % VEC == 0 when VEC = 4, so all VEC nodes exist
  float acc[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
  for (int m0 = 0; m0 < m_count; m0 += kDiagChunk) {
    const int cnt = min(kDiagChunk, m_count - m0);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += kDiagThreads) gs[i] = static_cast<float>(g[m0 + i] / scale);
    __syncthreads();
    if (!live) continue;
    const float* base = C + static_cast<size_t>(m0) * n + k0;
    int i = 0;
    for (; i + kDiagUnroll <= cnt; i += kDiagUnroll) {
      if constexpr (VEC == 4) {
        float4 r[kDiagUnroll];
#pragma unroll
        for (int u = 0; u < kDiagUnroll; ++u)
          r[u] = __ldcs(reinterpret_cast<const float4*>(base + static_cast<size_t>(i + u) * n));
#pragma unroll
        for (int u = 0; u < kDiagUnroll; ++u) {
          const float w = gs[i + u];
          acc[0] = fmaf(w, r[u].x, acc[0]);
          acc[1] = fmaf(w, r[u].y, acc[1]);
          acc[2] = fmaf(w, r[u].z, acc[2]);
          acc[3] = fmaf(w, r[u].w, acc[3]);
        }
      } else {
        float r[kDiagUnroll];
#pragma unroll
        for (int u = 0; u < kDiagUnroll; ++u) r[u] = __ldcs(base + static_cast<size_t>(i + u) * n);
#pragma unroll
        for (int u = 0; u < kDiagUnroll; ++u) acc[0] = fmaf(gs[i + u], r[u], acc[0]);
      }
    }
    for (; i < cnt; ++i) {
      const float w = gs[i];
      if constexpr (VEC == 4) {
        const float4 r = __ldcs(reinterpret_cast<const float4*>(base + static_cast<size_t>(i) * n));
        acc[0] = fmaf(w, r.x, acc[0]);
        acc[1] = fmaf(w, r.y, acc[1]);
        acc[2] = fmaf(w, r.z, acc[2]);
        acc[3] = fmaf(w, r.w, acc[3]);
      } else {
        acc[0] = fmaf(w, __ldcs(base + static_cast<size_t>(i) * n), acc[0]);
      }
    }
  }
  if (!live) return;
#pragma unroll
  for (int v = 0; v < VEC; ++v) out[k0 + v] = scale * static_cast<double>(acc[v]);
}

}  // namespace
}  // namespace netdos

using namespace netdos;

extern "C" int dos_fn_coeffs(int fn, double p, double lo, double hi, int M, double* coef_out, void* stream) {
  clear_error();
  if (!coef_out) return fail(DOS_EINVAL, "dos_fn_coeffs: null argument");
  if (fn != DOS_FN_EXP && fn != DOS_FN_RESOLVENT) return fail(DOS_EINVAL, "dos_fn_coeffs: unknown function");
  if (!(lo < hi) || !std::isfinite(lo) || !std::isfinite(hi) || !std::isfinite(p))
    return fail(DOS_EINVAL, "dos_fn_coeffs: need finite p and lo < hi");
  if (M < 1 || M > (1 << 20)) return fail(DOS_EINVAL, "dos_fn_coeffs: M must be in [1, 2^20]");
  if (fn == DOS_FN_RESOLVENT && !((1.0 - p * lo) * (1.0 - p * hi) > 0.0))
    return fail(DOS_EINVAL, "dos_fn_coeffs: 1 - p x vanishes on [lo, hi]");
  const int kpts = std::max(4 * M, 256);
  k_fn_coeffs<<<(M + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(fn, p, 0.5 * (lo + hi), 0.5 * (hi - lo),
                                                                             M, kpts, coef_out);
  NDOS_LAUNCHED();
  return DOS_OK;
}

extern "C" int dos_fn_trace(dos_graph_t g, const double* coef, const double* d, int M, double* out, void* stream) {
  clear_error();
  if (!g || !coef || !d || !out || M < 1) return fail(DOS_EINVAL, "dos_fn_trace: bad argument");
  const Graph* G = reinterpret_cast<const Graph*>(g);
  k_fn_trace<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(coef, d, M, static_cast<double>(G->n),
                                                                static_cast<double>(G->n_isolated), out);
  NDOS_LAUNCHED();
  return DOS_OK;
}

extern "C" int dos_fn_diag(const float* C, int64_t N, int M, const double* coef, double* out, void* stream) {
  clear_error();
  if (!C || !coef || !out || N < 1 || M < 1) return fail(DOS_EINVAL, "dos_fn_diag: bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool vec = N % 4 == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
  const int64_t per_cta = vec ? 4 * kDiagThreads : kDiagThreads;  // VEC nodes per thread
  const unsigned blocks = static_cast<unsigned>((N + per_cta - 1) / per_cta);
  if (vec)
    k_fn_diag<4><<<blocks, kDiagThreads, 0, s>>>(C, N, M, coef, out);
  else
    k_fn_diag<1><<<blocks, kDiagThreads, 0, s>>>(C, N, M, coef, out);
  NDOS_LAUNCHED();
  return DOS_OK;
}
