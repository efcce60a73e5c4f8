// Density-reconstruction MLP: a small fully connected network that maps a
// graph's noisy low-order Chebyshev moments and degree statistics to a
// B-bin spectral histogram (softmax output), with hand-written training
// (forward, backward, Adam) and inference kernels.  It has no counterpart in
// the paper; plain Jackson-damped KPM (dos_density) is its fallback and the
// judge of its L1 error.
//
//   z_l = a_{l-1} W_l^T + b_l,  a_l = relu(z_l) (hidden),  p = softmax(z_L),
//   loss = -(1/rows) sum t log p  against target histograms t.
//
// Parameters live in one flat FP32 buffer: for each layer W_l (out x in,
// row-major) then b_l.  Gradients, and Adam's first and second moments, use
// the same layout.  All reductions run in a fixed order (deterministic).
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "alloc_hook.h"
#include "common.cuh"

namespace netdos {
namespace {

constexpr int kTile = 64, kTk = 16;

// C[m][n] = sum_k A(m, k) B(k, n) (+ epilogue), A(m, k) = TA ? A[k][m] : A[m][k]
// (row stride lda), B(k, n) = TB ? B[n][k] : B[k][n] (row stride ldb); an
// optional row gather maps the row index of A (arow, when !TA) or of B
// (brow, when !TB) through an index list.  EPI 0: C = acc; 1: C = acc + bias,
// C2 = relu(C); 2: C = acc + bias.
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                              const float* __restrict__ B, int ldb, const int32_t* __restrict__ arow,
                                              const int32_t* __restrict__ brow, const float* __restrict__ bias,
                                              float* __restrict__ C, int ldc, float* __restrict__ C2) {
  __shared__ float As[kTk][kTile + 4], Bs[kTk][kTile + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kTk) {
    // each operand is read along its contiguous dimension (coalesced)
    for (int i = threadIdx.x; i < kTk * kTile; i += 256) {
      const int kk = TA ? i / kTile : i % kTk, mm = TA ? i % kTile : i / kTk;
      const int m = m0 + mm, k = k0 + kk;
      float a = 0.f;
      if (m < M && k < K) a = TA ? A[static_cast<size_t>(k) * lda + m] : A[static_cast<size_t>(arow ? arow[m] : m) * lda + k];
      As[kk][mm] = a;
    }
    for (int i = threadIdx.x; i < kTk * kTile; i += 256) {
      const int kk = TB ? i % kTk : i / kTile, nn = TB ? i / kTk : i % kTile;
      const int n = n0 + nn, k = k0 + kk;
      float b = 0.f;
      if (n < N && k < K) b = TB ? B[static_cast<size_t>(n) * ldb + k] : B[static_cast<size_t>(brow ? brow[k] : k) * ldb + n];
      Bs[kk][nn] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTk; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty * 4 + i];
        b[i] = Bs[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (EPI != 0) v += bias[n];
      C[static_cast<size_t>(m) * ldc + n] = v;
      if (EPI == 1) C2[static_cast<size_t>(m) * ldc + n] = v > 0.f ? v : 0.f;
    }
  }
}

// warp per row: softmax probabilities, per-row cross-entropy, and the
// logits' gradient (p - t) / rows
__global__ void k_softmax_xent(const float* __restrict__ z, const float* __restrict__ t,
                               const int32_t* __restrict__ trow, int rows, int n, float* __restrict__ p,
                               float* __restrict__ dz, float* __restrict__ rowloss) {
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= rows) return;
  const float* zr = z + static_cast<size_t>(r) * n;
  float mx = -INFINITY;
  for (int i = lane; i < n; i += 32) mx = fmaxf(mx, zr[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float s = 0.f;
  for (int i = lane; i < n; i += 32) s += expf(zr[i] - mx);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const float logs = logf(s);
  float loss = 0.f;
  const float* tr = t ? t + static_cast<size_t>(trow ? trow[r] : r) * n : nullptr;
  for (int i = lane; i < n; i += 32) {
    const float lp = zr[i] - mx - logs;
    const float pi = expf(lp);
    if (p) p[static_cast<size_t>(r) * n + i] = pi;
    if (tr) {
      loss -= tr[i] * lp;
      dz[static_cast<size_t>(r) * n + i] = (pi - tr[i]) / rows;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  if (lane == 0 && rowloss) rowloss[r] = loss;
}

// fixed-order sum of rowloss / rows into *out
__global__ void k_mean(const float* __restrict__ v, int n, float* __restrict__ out) {
  __shared__ double sh[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) a += v[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = static_cast<float>(sh[0] / n);
}

__global__ void k_relu_bwd(float* __restrict__ da, const float* __restrict__ z, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (z[i] <= 0.f) da[i] = 0.f;
}

// db[c] = sum over rows of dz[r][c], rows in order
__global__ void k_colsum(const float* __restrict__ dz, int rows, int cols, float* __restrict__ db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += dz[static_cast<size_t>(r) * cols + c];
  db[c] = s;
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// He-uniform weights from SplitMix64(seed)[i], zero biases
__global__ void k_init_params(float* __restrict__ w, int64_t n, int64_t w_end, float lim, uint64_t seed,
                              int64_t counter0) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < w_end) {
      const double u = static_cast<double>(splitmix64(seed, static_cast<uint64_t>(counter0 + i)) >> 11) * 0x1.0p-53;
      w[i] = static_cast<float>((2.0 * u - 1.0) * lim);
    } else {
      w[i] = 0.f;
    }
  }
}

// x[g] = [B * hist[g][0..B), d[g][1..K)] and, with stats (mean d, mean d^2,
// max d, N Nz per graph), [log(mean d), log(mean d^2)/2 - log(mean d),
// log(max d), log(N Nz)] / 10
__global__ void k_features(const double* __restrict__ hist, int B, const double* __restrict__ d, int ld_d, int K,
                           const double* __restrict__ stats, int64_t n_graphs, float* __restrict__ x) {
  const int F = B + K - 1 + (stats ? 4 : 0);
  const int64_t total = n_graphs * F;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = i / F;
    const int f = static_cast<int>(i - g * F);
    double v;
    if (f < B) {
      v = B * hist[g * B + f];
    } else if (f < B + K - 1) {
      v = d[g * ld_d + (f - B + 1)];
    } else {
      const double* st = stats + 4 * g;
      switch (f - (B + K - 1)) {
        case 0: v = log(st[0]); break;
        case 1: v = 0.5 * log(st[1]) - log(st[0]); break;
        case 2: v = log(st[2]); break;
        default: v = log(st[3]); break;
      }
      v /= 10.0;
    }
    x[i] = static_cast<float>(v);
  }
}

// degree statistics in two passes: every block reduces a grid-stride share
// of the degrees to (sum, sum of squares, max) -- exact in 64-bit integers,
// so the order of the additions does not matter -- and one block combines
// the blocks' triples into out = [sum / n, sumsq / n, max, n * nz]
__global__ void __launch_bounds__(1024) k_degree_partials(const int32_t* __restrict__ deg, int64_t n,
                                                          unsigned long long* __restrict__ part) {
  __shared__ unsigned long long s1[32], s2[32];
  __shared__ int smax[32];
  unsigned long long a = 0, b = 0;
  int mx = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long v = static_cast<unsigned long long>(deg[i]);
    a += v;
    b += v * v;
    mx = max(mx, deg[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    s1[w] = a;
    s2[w] = b;
    smax[w] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < static_cast<int>(blockDim.x >> 5); ++k) {
      s1[0] += s1[k];
      s2[0] += s2[k];
      smax[0] = max(smax[0], smax[k]);
    }
    part[3 * blockIdx.x] = s1[0];
    part[3 * blockIdx.x + 1] = s2[0];
    part[3 * blockIdx.x + 2] = static_cast<unsigned long long>(smax[0]);
  }
}

__global__ void k_degree_stats(const unsigned long long* __restrict__ part, int blocks, int64_t n, int nz,
                               double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  unsigned long long a = 0, b = 0, mx = 0;
  for (int k = 0; k < blocks; ++k) {
    a += part[3 * k];
    b += part[3 * k + 1];
    mx = part[3 * k + 2] > mx ? part[3 * k + 2] : mx;
  }
  out[0] = static_cast<double>(a) / static_cast<double>(n);
  out[1] = static_cast<double>(b) / static_cast<double>(n);
  out[2] = static_cast<double>(mx);
  out[3] = static_cast<double>(n) * static_cast<double>(nz);
}

// warp per graph: t[g][b] = max(h, 0) / sum max(h, 0), uniform if the sum is 0
__global__ void k_hist_normalize(const double* __restrict__ hist, int B, int64_t n_graphs, float* __restrict__ t) {
  const int lane = threadIdx.x & 31;
  const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (g >= n_graphs) return;
  const double* h = hist + g * B;
  double s = 0.0;
  for (int b = lane; b < B; b += 32) s += fmax(h[b], 0.0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  for (int b = lane; b < B; b += 32)
    t[g * B + b] = s > 0.0 ? static_cast<float>(fmax(h[b], 0.0) / s) : 1.f / B;
}

}  // namespace

struct Mlp {
  std::vector<int> sizes;  // [in, h1, ..., out]
  std::vector<int64_t> w_off, b_off;
  int64_t count = 0;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  int step = 0;
  int cap = 0;                      // batch capacity of the buffers below
  std::vector<float*> z, a;         // per layer l >= 1: pre-activation, activation [cap][sizes[l]]
  float *da = nullptr, *dz = nullptr, *rowloss = nullptr;
};

static void free_buffers(Mlp* h) {
  for (float* p : h->z) cudaFree(p);
  for (float* p : h->a) cudaFree(p);
  h->z.clear();
  h->a.clear();
  cudaFree(h->da);
  cudaFree(h->dz);
  cudaFree(h->rowloss);
  h->da = h->dz = h->rowloss = nullptr;
  h->cap = 0;
}

static int ensure(Mlp* h, int rows) {
  if (rows <= h->cap) return DOS_OK;
  free_buffers(h);
  int widest = 0;
  for (int s : h->sizes) widest = s > widest ? s : widest;
  const int L = static_cast<int>(h->sizes.size()) - 1;
  h->z.assign(L + 1, nullptr);
  h->a.assign(L + 1, nullptr);
  if (alloc_fault_injected()) return fail(DOS_ENOMEM, "injected allocation failure (dos_test_fail_alloc)");
  for (int l = 1; l <= L; ++l) {
    NDOS_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->z[l]), sizeof(float) * rows * h->sizes[l]));
    NDOS_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->a[l]), sizeof(float) * rows * h->sizes[l]));
  }
  NDOS_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->da), sizeof(float) * rows * widest));
  NDOS_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->dz), sizeof(float) * rows * widest));
  NDOS_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->rowloss), sizeof(float) * rows));
  h->cap = rows;
  return DOS_OK;
}

static dim3 gemm_grid(int M, int N) { return dim3((N + kTile - 1) / kTile, (M + kTile - 1) / kTile); }

// forward pass over `rows` inputs x (row r = x[idx ? idx[r] : r]); logits in z[L]
static int forward(Mlp* h, const float* x, const int32_t* idx, int rows, cudaStream_t s) {
  NDOS_CHECK(ensure(h, rows));
  const int L = static_cast<int>(h->sizes.size()) - 1;
  const float* in = x;
  for (int l = 1; l <= L; ++l) {
    const int fi = h->sizes[l - 1], fo = h->sizes[l];
    const float* W = h->params + h->w_off[l - 1];
    const float* b = h->params + h->b_off[l - 1];
    const int32_t* gather = l == 1 ? idx : nullptr;
    if (l < L)
      k_gemm<false, true, 1><<<gemm_grid(rows, fo), 256, 0, s>>>(rows, fo, fi, in, fi, W, fi, gather, nullptr, b,
                                                                 h->z[l], fo, h->a[l]);
    else
      k_gemm<false, true, 2><<<gemm_grid(rows, fo), 256, 0, s>>>(rows, fo, fi, in, fi, W, fi, gather, nullptr, b,
                                                                 h->z[l], fo, nullptr);
    NDOS_LAUNCHED();
    in = h->a[l];
  }
  return DOS_OK;
}

// loss and gradient (into h->grads) for targets t (row r = t[idx ? idx[r] : r])
static int loss_grad(Mlp* h, const float* x, const float* t, const int32_t* idx, int rows, float* loss,
                     cudaStream_t s) {
  NDOS_CHECK(forward(h, x, idx, rows, s));
  const int L = static_cast<int>(h->sizes.size()) - 1;
  const int out = h->sizes[L];
  k_softmax_xent<<<(rows * 32 + 255) / 256, 256, 0, s>>>(h->z[L], t, idx, rows, out, nullptr, h->dz, h->rowloss);
  NDOS_LAUNCHED();
  if (loss) {
    k_mean<<<1, 256, 0, s>>>(h->rowloss, rows, loss);
    NDOS_LAUNCHED();
  }
  for (int l = L; l >= 1; --l) {
    const int fi = h->sizes[l - 1], fo = h->sizes[l];
    const float* prev = l > 1 ? h->a[l - 1] : x;
    const int32_t* gather = l == 1 ? idx : nullptr;
    // dW = dz^T prev   (fo x fi)
    k_gemm<true, false, 0><<<gemm_grid(fo, fi), 256, 0, s>>>(fo, fi, rows, h->dz, fo, prev, fi, nullptr, gather,
                                                             nullptr, h->grads + h->w_off[l - 1], fi, nullptr);
    NDOS_LAUNCHED();
    k_colsum<<<(fo + 127) / 128, 128, 0, s>>>(h->dz, rows, fo, h->grads + h->b_off[l - 1]);
    NDOS_LAUNCHED();
    if (l > 1) {
      // da = dz W   (rows x fi), then dz = da * relu'(z_{l-1})
      k_gemm<false, false, 0><<<gemm_grid(rows, fi), 256, 0, s>>>(rows, fi, fo, h->dz, fo,
                                                                  h->params + h->w_off[l - 1], fi, nullptr, nullptr,
                                                                  nullptr, h->da, fi, nullptr);
      NDOS_LAUNCHED();
      const int64_t nn = static_cast<int64_t>(rows) * fi;
      k_relu_bwd<<<static_cast<unsigned>((nn + 255) / 256), 256, 0, s>>>(h->da, h->z[l - 1], nn);
      NDOS_LAUNCHED();
      std::swap(h->da, h->dz);
    }
  }
  return DOS_OK;
}

}  // namespace netdos

using namespace netdos;

extern "C" {

int dos_mlp_create(int n_layers, const int* sizes, uint64_t seed, dos_mlp_t* out) {
  clear_error();
  if (!out || !sizes || n_layers < 1 || n_layers > 16) return fail(DOS_EINVAL, "dos_mlp_create: 1..16 layers");
  *out = nullptr;
  for (int l = 0; l <= n_layers; ++l)
    if (sizes[l] < 1 || sizes[l] > 8192) return fail(DOS_EINVAL, "dos_mlp_create: layer sizes must be in [1, 8192]");
  Mlp* h = new Mlp();
  h->sizes.assign(sizes, sizes + n_layers + 1);
  for (int l = 0; l < n_layers; ++l) {
    h->w_off.push_back(h->count);
    h->count += static_cast<int64_t>(sizes[l]) * sizes[l + 1];
    h->b_off.push_back(h->count);
    h->count += sizes[l + 1];
  }
  float** bufs[] = {&h->params, &h->grads, &h->m, &h->v};
  for (float** b : bufs) {
    if (alloc_fault_injected()) {
      dos_mlp_destroy(reinterpret_cast<dos_mlp_t>(h));
      return fail(DOS_ENOMEM, "injected allocation failure (dos_test_fail_alloc)");
    }
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(b), sizeof(float) * h->count);
    if (e != cudaSuccess) {
      dos_mlp_destroy(reinterpret_cast<dos_mlp_t>(h));
      return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    }
  }
  cudaMemset(h->grads, 0, sizeof(float) * h->count);
  cudaMemset(h->m, 0, sizeof(float) * h->count);
  cudaMemset(h->v, 0, sizeof(float) * h->count);
  for (int l = 0; l < n_layers; ++l) {
    const int64_t n = static_cast<int64_t>(sizes[l]) * sizes[l + 1] + sizes[l + 1];
    const float lim = static_cast<float>(std::sqrt(6.0 / sizes[l]));
    k_init_params<<<static_cast<unsigned>((n + 255) / 256), 256>>>(h->params + h->w_off[l], n,
                                                                   static_cast<int64_t>(sizes[l]) * sizes[l + 1], lim,
                                                                   seed, h->w_off[l]);
    count_launch();
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    dos_mlp_destroy(reinterpret_cast<dos_mlp_t>(h));
    return cuda_fail(e, "dos_mlp_create", __FILE__, __LINE__);
  }
  *out = reinterpret_cast<dos_mlp_t>(h);
  return DOS_OK;
}

void dos_mlp_destroy(dos_mlp_t hh) {
  if (!hh) return;
  Mlp* h = reinterpret_cast<Mlp*>(hh);
  free_buffers(h);
  cudaFree(h->params);
  cudaFree(h->grads);
  cudaFree(h->m);
  cudaFree(h->v);
  delete h;
}

int dos_mlp_param_count(dos_mlp_t hh, int64_t* count) {
  if (!hh || !count) return fail(DOS_EINVAL, "dos_mlp_param_count: null argument");
  *count = reinterpret_cast<Mlp*>(hh)->count;
  return DOS_OK;
}

int dos_mlp_get_params(dos_mlp_t hh, float* out, void* stream) {
  if (!hh || !out) return fail(DOS_EINVAL, "dos_mlp_get_params: null argument");
  Mlp* h = reinterpret_cast<Mlp*>(hh);
  NDOS_CUDA(cudaMemcpyAsync(out, h->params, sizeof(float) * h->count, cudaMemcpyDeviceToDevice,
                            static_cast<cudaStream_t>(stream)));
  return DOS_OK;
}

int dos_mlp_set_params(dos_mlp_t hh, const float* in, void* stream) {
  if (!hh || !in) return fail(DOS_EINVAL, "dos_mlp_set_params: null argument");
  Mlp* h = reinterpret_cast<Mlp*>(hh);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NDOS_CUDA(cudaMemcpyAsync(h->params, in, sizeof(float) * h->count, cudaMemcpyDeviceToDevice, s));
  NDOS_CUDA(cudaMemsetAsync(h->m, 0, sizeof(float) * h->count, s));
  NDOS_CUDA(cudaMemsetAsync(h->v, 0, sizeof(float) * h->count, s));
  h->step = 0;
  return DOS_OK;
}

int dos_mlp_get_state(dos_mlp_t hh, float* params, float* m, float* v, int64_t* step, void* stream) {
  clear_error();
  if (!hh) return fail(DOS_EINVAL, "dos_mlp_get_state: null handle");
  Mlp* h = reinterpret_cast<Mlp*>(hh);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = sizeof(float) * h->count;
  if (params) NDOS_CUDA(cudaMemcpyAsync(params, h->params, bytes, cudaMemcpyDeviceToDevice, s));
  if (m) NDOS_CUDA(cudaMemcpyAsync(m, h->m, bytes, cudaMemcpyDeviceToDevice, s));
  if (v) NDOS_CUDA(cudaMemcpyAsync(v, h->v, bytes, cudaMemcpyDeviceToDevice, s));
  if (step) *step = h->step;
  return DOS_OK;
}

int dos_mlp_set_state(dos_mlp_t hh, const float* params, const float* m, const float* v, int64_t step,
                      void* stream) {
  clear_error();
  if (!hh || !params || !m || !v) return fail(DOS_EINVAL, "dos_mlp_set_state: null argument");
  if (step < 0 || step > 0x7fffffffLL) return fail(DOS_EINVAL, "dos_mlp_set_state: step out of range");
  Mlp* h = reinterpret_cast<Mlp*>(hh);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = sizeof(float) * h->count;
  NDOS_CUDA(cudaMemcpyAsync(h->params, params, bytes, cudaMemcpyDeviceToDevice, s));
  NDOS_CUDA(cudaMemcpyAsync(h->m, m, bytes, cudaMemcpyDeviceToDevice, s));
  NDOS_CUDA(cudaMemcpyAsync(h->v, v, bytes, cudaMemcpyDeviceToDevice, s));
  h->step = static_cast<int>(step);
  return DOS_OK;
}

int dos_mlp_forward(dos_mlp_t hh, const float* x, int rows, float* probs, void* stream) {
  clear_error();
  if (!hh || !x || !probs || rows < 1) return fail(DOS_EINVAL, "dos_mlp_forward: bad argument");
  Mlp* h = reinterpret_cast<Mlp*>(hh);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NDOS_CHECK(forward(h, x, nullptr, rows, s));
  const int L = static_cast<int>(h->sizes.size()) - 1;
  k_softmax_xent<<<(rows * 32 + 255) / 256, 256, 0, s>>>(h->z[L], nullptr, nullptr, rows, h->sizes[L], probs,
                                                         nullptr, nullptr);
  NDOS_LAUNCHED();
  return DOS_OK;
}

int dos_mlp_loss_grad(dos_mlp_t hh, const float* x, const float* t, int rows, float* loss, float* grad,
                      void* stream) {
  clear_error();
  if (!hh || !x || !t || rows < 1) return fail(DOS_EINVAL, "dos_mlp_loss_grad: bad argument");
  Mlp* h = reinterpret_cast<Mlp*>(hh);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NDOS_CHECK(loss_grad(h, x, t, nullptr, rows, loss, s));
  if (grad) NDOS_CUDA(cudaMemcpyAsync(grad, h->grads, sizeof(float) * h->count, cudaMemcpyDeviceToDevice, s));
  return DOS_OK;
}

int dos_mlp_train_step(dos_mlp_t hh, const float* x, const float* t, const int32_t* idx, int rows, float lr,
                       float* loss, void* stream) {
  clear_error();
  if (!hh || !x || !t || rows < 1 || !(lr > 0.f)) return fail(DOS_EINVAL, "dos_mlp_train_step: bad argument");
  Mlp* h = reinterpret_cast<Mlp*>(hh);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NDOS_CHECK(loss_grad(h, x, t, idx, rows, loss, s));
  h->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, static_cast<float>(h->step));
  const float c2 = 1.f - std::pow(b2, static_cast<float>(h->step));
  k_adam<<<static_cast<unsigned>(std::min<int64_t>((h->count + 255) / 256, 4096)), 256, 0, s>>>(
      h->params, h->grads, h->m, h->v, h->count, lr, b1, b2, 1e-8f, c1, c2);
  NDOS_LAUNCHED();
  return DOS_OK;
}

}  // extern "C"

extern "C" int dos_mlp_features(const double* hist, int n_bins, const double* d, int ld_d, int K,
                                const double* stats, int64_t n_graphs, float* x_out, void* stream) {
  clear_error();
  if (!hist || !d || !x_out) return fail(DOS_EINVAL, "dos_mlp_features: null pointer");
  if (n_bins < 1 || K < 1 || ld_d < K || n_graphs < 1 || n_bins + K - 1 > (1 << 20))
    return fail(DOS_EINVAL, "dos_mlp_features: bad sizes");
  const int64_t total = n_graphs * (n_bins + K - 1 + (stats ? 4 : 0));
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((total + 255) / 256, 152 * 16));
  k_features<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(hist, n_bins, d, ld_d, K, stats, n_graphs,
                                                                    x_out);
  NDOS_LAUNCHED();
  return DOS_OK;
}

extern "C" int dos_graph_stats(dos_graph_t g, int Nz, double* stats_out, void* stream) {
  clear_error();
  const Graph* G = reinterpret_cast<const Graph*>(g);
  if (!G || !stats_out) return fail(DOS_EINVAL, "dos_graph_stats: null argument");
  if (G->n < 1) return fail(DOS_EINVAL, "dos_graph_stats: graph has no edges");
  if (Nz < 1) return fail(DOS_EINVAL, "dos_graph_stats: Nz must be >= 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((G->n + 1023) / 1024, 2LL * num_sms())));
  Temps t(s);
  unsigned long long* part = nullptr;
  NDOS_CHECK(t.get(&part, static_cast<size_t>(3) * blocks));
  k_degree_partials<<<blocks, 1024, 0, s>>>(G->deg, G->n, part);
  NDOS_LAUNCHED();
  k_degree_stats<<<1, 32, 0, s>>>(part, blocks, G->n, Nz, stats_out);
  NDOS_LAUNCHED();
  return DOS_OK;
}

extern "C" int dos_hist_normalize(const double* hist, int n_bins, int64_t n_graphs, float* t_out, void* stream) {
  clear_error();
  if (!hist || !t_out) return fail(DOS_EINVAL, "dos_hist_normalize: null pointer");
  if (n_bins < 1 || n_graphs < 1) return fail(DOS_EINVAL, "dos_hist_normalize: bad sizes");
  const unsigned blocks = static_cast<unsigned>((n_graphs * 32 + 255) / 256);
  k_hist_normalize<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(hist, n_bins, n_graphs, t_out);
  NDOS_LAUNCHED();
  return DOS_OK;
}
