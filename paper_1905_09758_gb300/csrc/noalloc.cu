// dos_moments_noalloc: the FP32 DOS-moment path of dos_moments without any
// device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// moments: a process whose framework allocator (PyTorch's caching allocator,
// for instance) already holds nearly all device memory, where a fresh
// cudaMalloc fails or forces the framework to drop its cache; or a
// latency-bound caller for which cudaMalloc / cudaFree, which may synchronise
// the device, are not acceptable.  For them this entry point takes its
// scratch -- the two probe blocks and the FP64 moment partials -- from one
// file-scope device array of fixed size, kNoAllocScratchBytes, which every GPU
// that loads the library holds until the process exits.
//
// The array's host-side name is only a stand-in for the device symbol, so the
// host code looks up its device address with cudaGetSymbolAddress, once per
// device, with that device current, and passes the address to the kernels.
// The first call on a device does this look-up; that first call should come
// before any stream capture.
//
// All calls share the array and it keeps the previous call's contents: every
// region that must start at zero is cleared by this call.  Calls whose work
// overlaps on the GPU (other streams, other host threads) race on the array.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "kpm_kernels.cuh"

namespace netdos {

int make_plan(const Graph* G, int Nz, int prec, int mode, Plan* out);  // kpm.cu
int step_error_word(int** out);                                       // kpm.cu

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

int scratch_address(void** out) {
  int dev = 0;
  NDOS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(DOS_EINVAL, "dos_moments_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return DOS_OK;
}

inline size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// raw[s] = fixed-order sum of partial[s * width + i] (same order as dos_moments)
__global__ void __launch_bounds__(256) k_noalloc_reduce(const double* __restrict__ partial, int64_t width,
                                                        double* __restrict__ raw) {
  __shared__ double sh[256];
  const int s = blockIdx.x;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < width; i += blockDim.x) a += partial[static_cast<size_t>(s) * width + i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) raw[s] = sh[0];
}

// doubled moments from the dot slots: raw[0] = <V0,V0>, raw[1+2k] =
// <V_{k+1},V_{k+1}>, raw[2+2k] = <V_{k+1},V_k>
__global__ void k_noalloc_moments(const double* __restrict__ raw, int M, double norm, const int* __restrict__ err,
                                  double* __restrict__ d) {
  const bool failed = *err != 0;  // a bounded wait of the step kernel gave up
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    double mu;
    if (m == 0)
      mu = raw[0];
    else if (m == 1)
      mu = raw[2];
    else if ((m & 1) == 0)
      mu = 2.0 * raw[1 + 2 * (m / 2 - 1)] - raw[0];
    else
      mu = 2.0 * raw[2 + 2 * ((m - 1) / 2)] - raw[2];
    d[m] = failed ? __longlong_as_double(0x7ff8000000000000ll) : mu / norm;
  }
}

}  // namespace

static int moments_noalloc(const Graph* G, int M, int Nz, uint64_t seed, double* d_out, cudaStream_t s) {
  Plan plan;
  NDOS_CHECK(make_plan(G, Nz, DOS_FP32, kModeDos, &plan));
  const int64_t n = G->n;
  const int steps = M / 2;
  const int64_t width = plan.part_width;
  const int64_t n_raw = 1 + 2 * static_cast<int64_t>(steps);
  const size_t block_bytes = round256(sizeof(float) * static_cast<size_t>(n) * plan.nz_pad);
  const size_t partial_bytes = round256(sizeof(double) * static_cast<size_t>(n_raw) * width);
  const size_t raw_bytes = round256(sizeof(double) * static_cast<size_t>(n_raw));
  const size_t need = 2 * block_bytes + partial_bytes + raw_bytes;
  if (need > kNoAllocScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "dos_moments_noalloc: this graph, M and Nz need %zu bytes of scratch; the static scratch holds %zu "
             "bytes (use dos_moments)",
             need, kNoAllocScratchBytes);
    return fail(DOS_EINVAL, msg);
  }
  void* base = nullptr;
  NDOS_CHECK(scratch_address(&base));
  char* p = static_cast<char*>(base);
  float* ua = reinterpret_cast<float*>(p);
  float* ub = reinterpret_cast<float*>(p + block_bytes);
  double* partial = reinterpret_cast<double*>(p + 2 * block_bytes);
  double* raw = reinterpret_cast<double*>(p + 2 * block_bytes + partial_bytes);

  // the init kernel fills only part of slot 0; the rest must read as zero
  NDOS_CUDA(cudaMemsetAsync(partial, 0, sizeof(double) * width, s));

  InitParams ip{};
  ip.orig = G->p_orig;
  ip.compact = G->p_compact;
  ip.s32 = G->s32;
  ip.u0 = ua;
  ip.n = n;
  ip.t = plan.t;
  ip.nz = Nz;
  ip.nz_pad = plan.nz_pad;
  ip.seed = seed;
  ip.partial = partial;
  const int64_t chunks = n * (plan.nz_pad / VecT<float>::N);
  const int init_grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((chunks + 255) / 256, width)));
  NDOS_CHECK(launch_init<float>(ip, init_grid, s));

  StepParams prm{};
  prm.row_ptr = G->p_row_ptr;
  prm.col = G->p_col;
  prm.orig = G->p_orig;
  prm.compact = G->p_compact;
  prm.n = n;
  prm.n_heavy = G->n_heavy;
  prm.n_mid = G->n_mid;
  prm.tiles = plan.tiles;
  prm.part_width = plan.part_width;
  prm.mid_part_off = static_cast<int64_t>(plan.heavy_ctas) * plan.tiles;
  prm.light_part_off = static_cast<int64_t>(plan.heavy_ctas + plan.mid_ctas) * plan.tiles;
  NDOS_CHECK(step_error_word(&prm.err));
  prm.nz = Nz;
  prm.inv_nz = 1.0f / static_cast<float>(Nz);
  prm.seed = seed;
  for (int k = 0; k < steps; ++k) {
    prm.u_cur = (k & 1) ? ub : ua;
    prm.u_pn = (k & 1) ? ua : ub;
    prm.first = k == 0 ? 1 : 0;
    prm.partial = partial + static_cast<size_t>(1 + 2 * static_cast<int64_t>(k)) * width;
    NDOS_CHECK(launch_step<float>(plan, kModeDos, prm, s, SideStreams{}));
  }
  k_noalloc_reduce<<<static_cast<unsigned>(n_raw), 256, 0, s>>>(partial, width, raw);
  NDOS_LAUNCHED();
  k_noalloc_moments<<<1, 256, 0, s>>>(raw, M, static_cast<double>(n) * Nz, prm.err, d_out);
  NDOS_LAUNCHED();
  return DOS_OK;
}

}  // namespace netdos

using namespace netdos;

extern "C" int dos_moments_noalloc(dos_graph_t g, int M, int Nz, uint64_t seed, double* d_out, void* stream) {
  clear_error();
  if (!g) return fail(DOS_EINVAL, "dos_moments_noalloc: null graph");
  if (!d_out) return fail(DOS_EINVAL, "dos_moments_noalloc: d_out is NULL");
  const Graph* G = reinterpret_cast<const Graph*>(g);
  if (G->n < 1) return fail(DOS_EINVAL, "dos_moments_noalloc: graph has no edges");
  if (M < 1 || M > (1 << 20)) return fail(DOS_EINVAL, "dos_moments_noalloc: M must be in [1, 2^20]");
  if (Nz < 1 || Nz > 65536) return fail(DOS_EINVAL, "dos_moments_noalloc: Nz must be in [1, 65536]");
  return moments_noalloc(G, M, Nz, seed, d_out, static_cast<cudaStream_t>(stream));
}
