// dos_moments / ldos_moments: host driver of the stochastic Chebyshev
// recurrence (§3.1).  Plans the probe tiling, allocates the two probe blocks,
// runs the init kernel, floor(M/2) (DOS) or M-1 (LDOS) fused step launches
// and the deterministic FP64 reduction of the moment partials.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "kpm_kernels.cuh"

namespace netdos {

// class probe sums for the twin filter: csum[slot][j] = sum over members of z_j
// (integer-valued, so the float atomics are exact in any order)
__global__ void __launch_bounds__(256) k_class_sums(const int32_t* __restrict__ orig, const int32_t* __restrict__ slot,
                                                    int64_t n, int nz, int nz_pad, uint64_t seed,
                                                    float* __restrict__ csum) {
  const int words = (nz + 63) / 64;
  const int64_t total = n * words;
  for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < total;
       c += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t p = c / words;
    const int w = static_cast<int>(c % words);
    const int sl = slot[p];
    if (sl < 0) continue;
    const uint64_t word = probe_word(seed, static_cast<uint32_t>(orig[p]), static_cast<uint32_t>(w));
    const int jend = min(nz, 64 * (w + 1));
    for (int j = 64 * w; j < jend; ++j)
      atomicAdd(&csum[static_cast<size_t>(sl) * nz_pad + j], ((word >> (j & 63)) & 1ull) ? -1.f : 1.f);
  }
}

// raw[s] = sum of partial[s * width + i], i < width, in a fixed order
__global__ void __launch_bounds__(256) k_reduce_partials(const double* __restrict__ partial, int64_t width,
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

// raw dot slots -> normalised moments d_m = mu_m / norm.
// DOS (doubled): raw[0] = <V0,V0>, step k: raw[1+2k] = <V_{k+1},V_{k+1}>,
// raw[2+2k] = <V_{k+1},V_k>.  LDOS (direct): raw[m] = mu_m.
__global__ void k_moments_from_raw(const double* __restrict__ raw, int M, int doubled, double norm,
                                   const int* __restrict__ err, int negate_odd, double* __restrict__ d) {
  const bool failed = err && *err != 0;  // a bounded wait gave up: no valid moments
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
    if (failed) {
      d[m] = __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    double mu;
    if (!doubled) {
      mu = raw[m];
    } else if (m == 0) {
      mu = raw[0];
    } else if (m == 1) {
      mu = raw[2];
    } else if ((m & 1) == 0) {
      const int k = m / 2 - 1;
      mu = 2.0 * raw[1 + 2 * k] - raw[0];
    } else {
      const int k = (m - 1) / 2;
      mu = 2.0 * raw[2 + 2 * k] - raw[2];
    }
    d[m] = (negate_odd && (m & 1) ? -mu : mu) / norm;
  }
}

__global__ void k_fill_f32(float* __restrict__ p, int64_t n, int64_t stride, float v) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    p[i * stride] = v;
}

// LDOS output of a chunk of moments [m0, m0 + cnt) from the step scratch
// part[(m % ch) * tiles + t][p] (one row per tile, indexed by the position p
// of the degree-sorted order, so the steps' stores are coalesced); the
// tiles' values are summed in tile order.
// Moment-major (out[m * n + k]): a thread per (moment, position), reading
// the scratch rows in position order and writing at the node's compact id
// k = compact[p].
__global__ void __launch_bounds__(256) k_ldos_fold_mm(const float* __restrict__ part,
                                                      const int32_t* __restrict__ compact, int tiles, int ch,
                                                      int64_t n, int m0, int cnt, float* __restrict__ out) {
  const int64_t total = static_cast<int64_t>(cnt) * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(e / n);
    const int64_t p = e - static_cast<int64_t>(r) * n;
    const int m = m0 + r;
    const float* src = part + static_cast<size_t>(m % ch) * tiles * n + p;
    float v = 0.f;
    for (int t = 0; t < tiles; ++t) v += src[static_cast<size_t>(t) * n];
    out[static_cast<size_t>(m) * n + compact[p]] = v;
  }
}

// Node-major (out[k * M + m]): for every compact node k the value at
// p = pos[k], through a 32 x 32 shared-memory transpose so that each node's
// run of moments is one contiguous write.  Block (32, 8).
__global__ void __launch_bounds__(256) k_ldos_fold_nm(const float* __restrict__ part, const int32_t* __restrict__ pos,
                                                      int tiles, int ch, int64_t n, int m0, int cnt, int M,
                                                      float* __restrict__ out) {
  __shared__ float tile_s[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int64_t k0 = static_cast<int64_t>(blockIdx.x) * 32; k0 < n; k0 += static_cast<int64_t>(gridDim.x) * 32) {
    for (int r0 = 0; r0 < cnt; r0 += 32) {
      for (int r = ty; r < 32; r += 8) {
        const int64_t k = k0 + tx;
        float v = 0.f;
        if (k < n && r0 + r < cnt) {
          const int m = m0 + r0 + r;
          const float* src = part + static_cast<size_t>(m % ch) * tiles * n + pos[k];
          for (int t = 0; t < tiles; ++t) v += src[static_cast<size_t>(t) * n];
        }
        tile_s[r][tx] = v;
      }
      __syncthreads();
      for (int j = ty; j < 32; j += 8) {
        const int64_t k = k0 + j;
        if (k < n && r0 + tx < cnt) out[static_cast<size_t>(k) * M + m0 + r0 + tx] = tile_s[tx][j];
      }
      __syncthreads();
    }
  }
}

static std::mutex g_smem_mu;

int raise_smem_limit(const void* kernel, int* limits, int smem) {
  int dev = 0;
  NDOS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(DOS_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_smem_mu);
  if (smem > limits[dev]) {
    NDOS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    limits[dev] = smem;
  }
  return DOS_OK;
}

static int g_force_t = 0;  // 0 = planner's choice
static int g_force_ctas = 0;  // light-row CTAs per SM, 0 = as many as fit

static int elem_size(int prec) { return prec == DOS_FP32 ? 4 : 2; }

// device error word (one per device): set by a kernel that gives up on a
// bounded wait; the current step kernels have no such wait, so it stays 0
__device__ int g_step_err;
static std::mutex g_err_mu;
static int* g_err_addr[64] = {};

int step_error_word(int** out) {
  int dev = 0;
  NDOS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(DOS_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!g_err_addr[dev]) {
    void* p = nullptr;
    NDOS_CUDA(cudaGetSymbolAddress(&p, g_step_err));
    g_err_addr[dev] = static_cast<int*>(p);
  }
  *out = g_err_addr[dev];
  return DOS_OK;
}

// side streams and events of the step launches, one set per device
static std::mutex g_side_mu;
static SideStreams g_side[64];

int side_streams(SideStreams* out) {
  int dev = 0;
  NDOS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(DOS_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_side_mu);
  SideStreams& sd = g_side[dev];
  if (!sd.a) {
    NDOS_CUDA(cudaStreamCreateWithFlags(&sd.a, cudaStreamNonBlocking));
    NDOS_CUDA(cudaStreamCreateWithFlags(&sd.b, cudaStreamNonBlocking));
    NDOS_CUDA(cudaEventCreateWithFlags(&sd.fork, cudaEventDisableTiming));
    NDOS_CUDA(cudaEventCreateWithFlags(&sd.join_a, cudaEventDisableTiming));
    NDOS_CUDA(cudaEventCreateWithFlags(&sd.join_b, cudaEventDisableTiming));
  }
  *out = sd;
  return DOS_OK;
}

int side_streams_for_capture(SideStreams* out) { return side_streams(out); }

static int light_config(int prec, int q, int mode, int* smem, int* ctas) {
  switch (prec) {
    case DOS_BF16:
      return step_config<__nv_bfloat16>(q, mode, smem, ctas);
    case DOS_FP16:
      return step_config<__half>(q, mode, smem, ctas);
    default:
      return step_config<float>(q, mode, smem, ctas);
  }
}

// Probe tiling.  A tile of t probe columns is what concurrently running CTAs
// gather from, so t is chosen so that one tile of U_k (n * t elements) fits
// in a share of L2 when possible; among the tilings that fit, the one with
// the least modelled traffic per step (T re-reads of the CSR + three probe
// blocks including padding) wins.
int make_plan(const Graph* G, int Nz, int prec, int mode, Plan* out) {
  const int es = elem_size(prec);
  const int V = 16 / es;
  const int qmax = prec == DOS_FP32 ? 16 : 8;
  const double budget = 80.0e6;
  const double n = static_cast<double>(G->n), nnz = static_cast<double>(G->nnz);
  bool have = false, have_fit = false;
  double best = 0.0;
  Plan pl;
  // a plan forced process-wide wins over one tuned for this graph
  const bool tuned = G->tuned_t > 0 && G->tuned_nz == Nz && G->tuned_prec == prec;
  const int force_t = g_force_t ? g_force_t : (tuned ? G->tuned_t : 0);
  const int force_ctas = g_force_ctas ? g_force_ctas : (tuned ? G->tuned_ctas : 0);
  for (int q = 1; q <= qmax; q *= 2) {
    const int t = q * V;
    if (force_t && t != force_t) continue;
    const int tiles = (Nz + t - 1) / t;
    const int nz_pad = tiles * t;
    const double bytes = tiles * (4.0 * nnz + 8.0 * (n + 1) + 8.0 * n) + 3.0 * n * nz_pad * es;
    const bool fits = n * t * es <= budget;
    bool take = false;
    if (!have) take = true;
    else if (fits && !have_fit) take = true;
    else if (fits == have_fit && bytes < best) take = true;
    if (take) {
      have = true;
      have_fit = fits;
      best = bytes;
      pl.t = t;
      pl.q = q;
      pl.tiles = tiles;
      pl.nz_pad = nz_pad;
    }
  }
  if (!have) return fail(DOS_EINVAL, "no tile width matches the forced plan");
  const int sms = num_sms();
  int smem = 0, ctas = 0;
  NDOS_CHECK(light_config(prec, pl.q, mode, &smem, &ctas));
  pl.smem = smem;
  // at most three resident CTAs per SM (measured best on GB300 for t = 16
  // and 32: more shared memory per SM leaves less L1 for gathers in flight)
  ctas = std::min(ctas, force_ctas > 0 ? force_ctas : 3);
  const int64_t n_light = G->n - G->n_mid;
  const int64_t rounds = (n_light + 32 / pl.q - 1) / (32 / pl.q) * pl.tiles;
  pl.light_ctas = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(std::max(1, ctas)) * sms,
                                                     (rounds + kStepWarps - 1) / kStepWarps));
  pl.heavy_ctas = static_cast<int>(std::min<int64_t>(G->n_heavy, 4LL * sms));
  const int64_t n_mid_rows = G->n_mid - G->n_heavy;
  pl.mid_ctas = static_cast<int>(std::min<int64_t>((n_mid_rows + kStepWarps - 1) / kStepWarps, 4LL * sms));
  pl.part_width = static_cast<int64_t>(pl.heavy_ctas + pl.mid_ctas) * pl.tiles + pl.light_ctas;
  *out = pl;
  return DOS_OK;
}

// operator of a KPM run: kind (0 H, 1 A, 2 D - A), shift c and 1/r (Eq. (5)),
// and whether odd moments change sign (I - H = -(H) after the shift by 1)
struct OpSpec {
  int kind = 0;
  double c = 0.0, inv_r = 1.0;
  int negate_odd = 0;
};

template <typename T>
static int run_steps(const Graph* G, const Filter* F, const Plan& plan, int M, int Nz, uint64_t seed, int mode,
                     double* d_out, float* C_out, cudaStream_t s, const OpSpec& op = OpSpec(), int layout = 0) {
  constexpr int V = VecT<T>::N;
  const int64_t n = G->n;
  const bool ldos = mode == kModeLdos || mode == kModeLdosOp;
  const int steps = ldos ? M - 1 : M / 2;
  const int n_dots = ldos ? 1 : 2;
  const int64_t width = plan.part_width;
  const int64_t n_raw = 1 + static_cast<int64_t>(steps) * n_dots;
  const size_t elems = static_cast<size_t>(n) * plan.nz_pad;

  T *ua = nullptr, *ub = nullptr;
  double *partial = nullptr, *raw = nullptr;
  float *csum = nullptr, *lpart = nullptr;
  int st = DOS_OK;
  const auto cleanup = [&]() {
    dfree(ua, s);
    dfree(ub, s);
    dfree(partial, s);
    dfree(raw, s);
    dfree(csum, s);
    dfree(lpart, s);
  };
  if ((st = dalloc_t(&ua, elems, s)) || (st = dalloc_t(&ub, elems, s)) ||
      (st = dalloc_t(&partial, static_cast<size_t>(n_raw) * width, s)) || (st = dalloc_t(&raw, n_raw, s))) {
    cleanup();
    return st;
  }
  const auto cu = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == DOS_OK) st = cuda_fail(e, what, __FILE__, __LINE__);
  };
  cu(cudaMemsetAsync(partial, 0, sizeof(double) * width, s), "cudaMemsetAsync");

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
  ip.unscaled = op.kind != 0 ? 1 : 0;
  if (F && F->n_classes > 0 && st == DOS_OK) {
    if ((st = dalloc_t(&csum, static_cast<size_t>(F->n_classes) * plan.nz_pad, s)) == DOS_OK) {
      cu(cudaMemsetAsync(csum, 0, sizeof(float) * F->n_classes * plan.nz_pad, s), "cudaMemsetAsync");
      const int64_t work = n * ((Nz + 63) / 64);
      const unsigned g = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 8LL * num_sms())));
      k_class_sums<<<g, 256, 0, s>>>(G->p_orig, F->p_slot, n, Nz, plan.nz_pad, seed, csum);
      count_launch();
      cu(cudaGetLastError(), "k_class_sums");
      ip.slot = F->p_slot;
      ip.slot_size = F->slot_size;
      ip.csum = csum;
    }
  }
  const int64_t chunks = n * (plan.nz_pad / V);
  const int init_grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((chunks + 255) / 256, width)));
  if (st == DOS_OK) st = launch_init<T>(ip, init_grid, s);

  // LDOS output.  One tile and the moment-major layout: every step stores
  // its row of C_out directly.  Otherwise the steps store one row per tile
  // into a scratch of `ch` moments, and k_ldos_fold_* sum the tiles in a fixed
  // order into the requested layout once a chunk of moments is complete:
  // after every step for the moment-major layout (the scratch, tiles x N
  // floats, stays in L2 and its rows are written out coalesced), after up to
  // 32 steps for the node-major one (each node's run of moments is then one
  // contiguous write).
  const bool node_major = layout == 1;
  const bool fold = ldos && (plan.tiles > 1 || node_major);
  int ch = 1;
  if (fold && st == DOS_OK) {
    const double row = 4.0 * static_cast<double>(n) * plan.tiles;
    ch = node_major ? static_cast<int>(std::max(1.0, std::min(32.0, std::floor(256.0e6 / row)))) : 1;
    st = dalloc_t(&lpart, static_cast<size_t>(ch) * plan.tiles * n, s);
  }
  const auto fold_chunk = [&](int m0, int cnt) {
    if (node_major) {
      const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((n + 31) / 32, 16LL * num_sms()));
      k_ldos_fold_nm<<<blocks, dim3(32, 8), 0, s>>>(lpart, G->compact_to_p, plan.tiles, ch, n, m0, cnt, M, C_out);
    } else {
      const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((cnt * n + 255) / 256, 8LL * num_sms()));
      k_ldos_fold_mm<<<blocks, 256, 0, s>>>(lpart, G->p_compact, plan.tiles, ch, n, m0, cnt, C_out);
    }
    count_launch();
    cu(cudaGetLastError(), "k_ldos_fold");
  };
  if (ldos && st == DOS_OK) {
    // moment 0: C[0][k] = z_k . z_k / Nz = 1 for Rademacher probes
    k_fill_f32<<<std::min<unsigned>(4096, std::max<unsigned>(1, ceil_div(n, 256))), 256, 0, s>>>(
        C_out, n, node_major ? M : 1, 1.0f);
    count_launch();
    cu(cudaGetLastError(), "k_fill_f32");
  }

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
  if (st == DOS_OK) st = step_error_word(&prm.err);
  prm.nz = Nz;
  prm.inv_nz = 1.0f / static_cast<float>(Nz);
  prm.seed = seed;
  prm.ldos_tile_stride = fold && plan.tiles > 1 ? n : 0;
  prm.ldos_by_position = fold ? 1 : 0;
  prm.op = op.kind;
  prm.op_c = static_cast<float>(op.c);
  prm.op_inv_r = static_cast<float>(op.inv_r);
  const bool prof = profiling_on();
  SideStreams side;
  if (st == DOS_OK) st = side_streams(&side);
  for (int k = 0; k < steps && st == DOS_OK; ++k) {
    prm.u_cur = (k & 1) ? ub : ua;
    prm.u_pn = (k & 1) ? ua : ub;
    prm.first = k == 0 ? 1 : 0;
    prm.partial = partial + static_cast<size_t>(1 + static_cast<int64_t>(k) * n_dots) * width;
    const int m = k + 1;  // the LDOS moment this step produces
    prm.ldos = !ldos ? nullptr
                     : (fold ? lpart + static_cast<size_t>(m % ch) * plan.tiles * n : C_out + static_cast<size_t>(m) * n);
    if (prof) profile_begin(s);
    st = launch_step<T>(plan, op.kind == 0 ? (ldos ? kModeLdos : kModeDos) : (ldos ? kModeLdosOp : kModeDosOp), prm,
                        s, side);
    if (prof) profile_end(s);
    // a chunk is complete at its last moment or at M - 1 (moment 0 is filled above)
    if (fold && st == DOS_OK && ((m + 1) % ch == 0 || m == M - 1)) {
      const int m0 = std::max(1, (m / ch) * ch);
      fold_chunk(m0, m - m0 + 1);
    }
  }
  if (st == DOS_OK) {
    k_reduce_partials<<<static_cast<unsigned>(n_raw), 256, 0, s>>>(partial, width, raw);
    count_launch();
    cu(cudaGetLastError(), "k_reduce_partials");
  }
  if (st == DOS_OK && d_out) {
    const double r = F ? static_cast<double>(n - F->removed) : static_cast<double>(n);
    k_moments_from_raw<<<1, 256, 0, s>>>(raw, M, ldos ? 0 : 1, r * Nz, prm.err, op.negate_odd, d_out);
    count_launch();
    cu(cudaGetLastError(), "k_moments_from_raw");
  }
  cleanup();
  return st;
}

static int run_kpm(const Graph* G, const Filter* F, int M, int Nz, uint64_t seed, int prec, int mode,
                   double* d_out, float* C_out, cudaStream_t s, const OpSpec& op = OpSpec(), int layout = 0) {
  if (!G) return fail(DOS_EINVAL, "null graph");
  if (G->n < 1) return fail(DOS_EINVAL, "graph has no edges");
  if (M < 1 || M > (1 << 20)) return fail(DOS_EINVAL, "M must be in [1, 2^20]");
  if (Nz < 1 || Nz > 65536) return fail(DOS_EINVAL, "Nz must be in [1, 65536]");
  if (prec != DOS_FP32 && prec != DOS_BF16 && prec != DOS_FP16) return fail(DOS_EINVAL, "unknown precision");
  if (F && F->g != G) return fail(DOS_EINVAL, "filter belongs to another graph");
  if (mode == kModeLdos && op.kind != 0) {
    if (prec != DOS_FP32) return fail(DOS_EINVAL, "LDOS of A and D - A is computed in FP32 only");
    mode = kModeLdosOp;  // the light kernel's round layout carries both the own rows and the ids
  }
  Plan plan;
  NDOS_CHECK(make_plan(G, Nz, prec, mode, &plan));
  switch (prec) {
    case DOS_BF16:
      return run_steps<__nv_bfloat16>(G, F, plan, M, Nz, seed, mode, d_out, C_out, s, op, layout);
    case DOS_FP16:
      return run_steps<__half>(G, F, plan, M, Nz, seed, mode, d_out, C_out, s, op, layout);
    default:
      return run_steps<float>(G, F, plan, M, Nz, seed, mode, d_out, C_out, s, op, layout);
  }
}

// operator and interval of a KPM run on op (DOS_OP_*): H and I - H on
// their fixed intervals, A and D - A on [lo, hi] when lo < hi, else on the
// Gershgorin interval ([-d_max, d_max], [0, 2 d_max])
static int op_spec(const Graph* G, int op, double lo, double hi, OpSpec* spec, double* interval_out) {
  double a = -1.0, b = 1.0;
  switch (op) {
    case DOS_OP_NORMALIZED_ADJACENCY:
      break;
    case DOS_OP_NORMALIZED_LAPLACIAN:  // I - H on [0, 2]: (I - H) - 1 = -H
      a = 0.0;
      b = 2.0;
      spec->negate_odd = 1;
      break;
    case DOS_OP_ADJACENCY:
    case DOS_OP_LAPLACIAN: {
      spec->kind = op == DOS_OP_ADJACENCY ? 1 : 2;
      if (lo < hi) {
        a = lo;
        b = hi;
      } else {
        const double dmax = static_cast<double>(G->max_deg);
        a = op == DOS_OP_ADJACENCY ? -dmax : 0.0;
        b = op == DOS_OP_ADJACENCY ? dmax : 2.0 * dmax;
      }
      spec->c = 0.5 * (a + b);
      spec->inv_r = 2.0 / (b - a);
      break;
    }
    default:
      return fail(DOS_EINVAL, "unknown operator");
  }
  if (interval_out) {
    interval_out[0] = a;
    interval_out[1] = b;
  }
  return DOS_OK;
}

// rows m = 1, 3, 5, ... of a moment-major [M][n] matrix change sign
__global__ void k_negate_odd_rows(float* __restrict__ c, int M, int64_t n) {
  const int64_t total = static_cast<int64_t>(M / 2) * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / n;
    float* p = c + static_cast<size_t>(2 * r + 1) * n + (e - r * n);
    *p = -*p;
  }
}

}  // namespace netdos

using namespace netdos;

extern "C" {

int dos_moments(dos_graph_t g, dos_filter_t f, int M, int Nz, uint64_t seed, int prec, double* d_out,
                void* stream) {
  clear_error();
  if (!d_out) return fail(DOS_EINVAL, "dos_moments: d_out is NULL");
  return run_kpm(reinterpret_cast<const Graph*>(g), reinterpret_cast<const Filter*>(f), M, Nz, seed, prec,
                 kModeDos, d_out, nullptr, static_cast<cudaStream_t>(stream));
}

int ldos_moments(dos_graph_t g, int M, int Nz, uint64_t seed, int prec, float* C_out, double* d_out,
                 void* stream) {
  clear_error();
  if (!C_out) return fail(DOS_EINVAL, "ldos_moments: C_out is NULL");
  return run_kpm(reinterpret_cast<const Graph*>(g), nullptr, M, Nz, seed, prec, kModeLdos, d_out, C_out,
                 static_cast<cudaStream_t>(stream));
}

int ldos_moments_ex(dos_graph_t g, int M, int Nz, uint64_t seed, int prec, int layout, float* C_out,
                    double* d_out, void* stream) {
  clear_error();
  if (!C_out) return fail(DOS_EINVAL, "ldos_moments_ex: C_out is NULL");
  if (layout != DOS_MOMENT_MAJOR && layout != DOS_NODE_MAJOR) return fail(DOS_EINVAL, "ldos_moments_ex: layout");
  return run_kpm(reinterpret_cast<const Graph*>(g), nullptr, M, Nz, seed, prec, kModeLdos, d_out, C_out,
                 static_cast<cudaStream_t>(stream), OpSpec(), layout);
}

int dos_moments_op(dos_graph_t g, int op, double lo, double hi, int M, int Nz, uint64_t seed, int prec,
                   double* d_out, double* interval_out, void* stream) {
  clear_error();
  if (!g || !d_out) return fail(DOS_EINVAL, "dos_moments_op: null argument");
  const Graph* G = reinterpret_cast<const Graph*>(g);
  if (G->n < 1) return fail(DOS_EINVAL, "dos_moments_op: graph has no edges");
  OpSpec spec;
  NDOS_CHECK(op_spec(G, op, lo, hi, &spec, interval_out));
  return run_kpm(G, nullptr, M, Nz, seed, prec, kModeDos, d_out, nullptr, static_cast<cudaStream_t>(stream), spec);
}

int ldos_moments_op(dos_graph_t g, int op, double lo, double hi, int M, int Nz, uint64_t seed, float* C_out,
                    double* d_out, double* interval_out, void* stream) {
  clear_error();
  if (!g || !C_out) return fail(DOS_EINVAL, "ldos_moments_op: null argument");
  const Graph* G = reinterpret_cast<const Graph*>(g);
  if (G->n < 1) return fail(DOS_EINVAL, "ldos_moments_op: graph has no edges");
  OpSpec spec;
  NDOS_CHECK(op_spec(G, op, lo, hi, &spec, interval_out));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NDOS_CHECK(run_kpm(G, nullptr, M, Nz, seed, DOS_FP32, kModeLdos, d_out, C_out, s, spec));
  if (spec.negate_odd && M > 1) {  // I - H: T_m(-H) = (-1)^m T_m(H), row by row
    const int64_t work = static_cast<int64_t>(M / 2) * G->n;
    k_negate_odd_rows<<<static_cast<unsigned>(std::min<int64_t>((work + 255) / 256, 8LL * num_sms())), 256, 0, s>>>(
        C_out, M, G->n);
    NDOS_LAUNCHED();
  }
  return DOS_OK;
}

int dos_set_plan(int tile_width, int ctas_per_sm) {
  if (tile_width != 0 && (tile_width < 4 || tile_width > 64 || (tile_width & (tile_width - 1))))
    return fail(DOS_EINVAL, "dos_set_plan: tile width must be 0 or a power of two in [4, 64]");
  if (ctas_per_sm < 0 || ctas_per_sm > 32) return fail(DOS_EINVAL, "dos_set_plan: ctas_per_sm must be in [0, 32]");
  g_force_t = tile_width;
  g_force_ctas = ctas_per_sm;
  return DOS_OK;
}

int dos_get_plan(dos_graph_t g, int Nz, int prec, int* tile_width, int* ctas_per_sm, int* tiles, int* grid_x) {
  Plan pl;
  if (!g) return fail(DOS_EINVAL, "dos_get_plan: null graph");
  NDOS_CHECK(make_plan(reinterpret_cast<const Graph*>(g), Nz, prec, kModeDos, &pl));
  if (tile_width) *tile_width = pl.t;
  if (ctas_per_sm) *ctas_per_sm = (pl.light_ctas + num_sms() - 1) / num_sms();
  if (tiles) *tiles = pl.tiles;
  if (grid_x) *grid_x = pl.light_ctas;
  return DOS_OK;
}

int dos_device_status(void* stream, int* status) {
  int* err = nullptr;
  NDOS_CHECK(step_error_word(&err));
  int h = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NDOS_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  NDOS_CUDA(cudaStreamSynchronize(s));
  if (h != 0) NDOS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  if (status) *status = h;
  return h == 0 ? DOS_OK : fail(DOS_ETIMEOUT, "a bounded device wait of the step kernel gave up");
}

}  // extern "C"
