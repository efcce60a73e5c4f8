// Batches of graphs and plan tuning.
//
// dos_moments_batched: the DOS moments of every graph of a batch built by
// dos_build_csr_batched.  The batch's operator is the block-diagonal union of
// the graphs' normalized adjacencies, so one run of the fused Chebyshev step
// over the union advances every graph at once; the step kernels send each
// row's moment-dot contributions to its graph's FP64 accumulators.  The whole
// sequence (accumulator reset, probe init, floor(M/2) steps, moment
// assembly) is captured once into a CUDA graph, kept on the handle, and
// replayed with one cudaGraphLaunch per call.
//
// dos_autotune: times the candidate probe-tile widths and light-kernel CTA
// counts on the graph itself and keeps the fastest plan on the handle.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "alloc_hook.h"
#include "kpm_kernels.cuh"

namespace netdos {

int make_plan(const Graph* G, int Nz, int prec, int mode, Plan* out);  // kpm.cu
int step_error_word(int** out);                                       // kpm.cu
int side_streams_for_capture(SideStreams* out);                       // kpm.cu

struct Captured {
  int M = 0, Nz = 0, prec = -1, t = 0, ctas = 0;
  uint64_t seed = 0;
  double* d_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* ua = nullptr;
  void* ub = nullptr;
  double* gpartial = nullptr;
  double* init_partial = nullptr;
};

void destroy_captured(Captured* c) {
  if (!c) return;
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  void* ptrs[] = {c->ua, c->ub, c->gpartial, c->init_partial};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete c;
}

namespace {

// mu_0 of each graph: ||z||^2 summed over its Nz Rademacher probes
__global__ void k_batch_mu0(const int64_t* __restrict__ graph_n, int64_t n_graphs, int nz, double* __restrict__ raw0) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_graphs; g += (int64_t)gridDim.x * blockDim.x)
    raw0[g] = static_cast<double>(graph_n[g]) * nz;
}

// per graph: raw dot slots -> normalised moments (doubling identities as in
// dos_moments).  raw[slot * n_graphs + g]; d[g * M + m].
__global__ void k_batch_moments(const double* __restrict__ raw, int64_t n_graphs, int M, int nz,
                                const int64_t* __restrict__ graph_n, const int* __restrict__ err,
                                double* __restrict__ d) {
  const bool failed = *err != 0;
  const int64_t total = n_graphs * M;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = i / M;
    const int m = static_cast<int>(i % M);
    const auto r = [&](int64_t slot) { return raw[slot * n_graphs + g]; };
    double mu;
    if (m == 0)
      mu = r(0);
    else if (m == 1)
      mu = r(2);
    else if ((m & 1) == 0)
      mu = 2.0 * r(1 + 2 * (m / 2 - 1)) - r(0);
    else
      mu = 2.0 * r(2 + 2 * ((m - 1) / 2)) - r(2);
    const double norm = static_cast<double>(graph_n[g]) * nz;
    d[i] = (failed || norm == 0.0) ? __longlong_as_double(0x7ff8000000000000ll) : mu / norm;
  }
}

template <typename T>
int enqueue_batched(const Graph* G, const Plan& plan, Captured* c, cudaStream_t s, const SideStreams& side) {
  constexpr int V = VecT<T>::N;
  const int64_t n = G->n;
  const int steps = c->M / 2;
  const int64_t ng = G->n_graphs;
  const int64_t n_raw = 1 + 2 * static_cast<int64_t>(steps);
  NDOS_CUDA(cudaMemsetAsync(c->gpartial, 0, sizeof(double) * n_raw * ng, s));
  k_batch_mu0<<<ceil_div(ng, 256), 256, 0, s>>>(G->graph_n, ng, c->Nz, c->gpartial);
  NDOS_LAUNCHED();
  InitParams ip{};
  ip.orig = G->p_orig;
  ip.compact = G->p_compact;
  ip.s32 = G->s32;
  ip.u0 = c->ua;
  ip.n = n;
  ip.t = plan.t;
  ip.nz = c->Nz;
  ip.nz_pad = plan.nz_pad;
  ip.seed = c->seed;
  ip.partial = c->init_partial;
  const int64_t chunks = n * (plan.nz_pad / V);
  const int init_grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((chunks + 255) / 256, 4096)));
  NDOS_CHECK(launch_init<T>(ip, init_grid, s));
  StepParams prm{};
  prm.row_ptr = G->p_row_ptr;
  prm.col = G->p_col;
  prm.orig = G->p_orig;
  prm.compact = G->p_compact;
  prm.n = n;
  prm.n_heavy = G->n_heavy;
  prm.n_mid = G->n_mid;
  prm.gid = G->p_gid;
  prm.n_graphs = ng;
  prm.tiles = plan.tiles;
  prm.part_width = plan.part_width;
  prm.mid_part_off = static_cast<int64_t>(plan.heavy_ctas) * plan.tiles;
  prm.light_part_off = static_cast<int64_t>(plan.heavy_ctas + plan.mid_ctas) * plan.tiles;
  prm.partial = c->init_partial;  // per-CTA partials are not used with gid; a valid scratch target
  NDOS_CHECK(step_error_word(&prm.err));
  prm.nz = c->Nz;
  prm.inv_nz = 1.0f / static_cast<float>(c->Nz);
  prm.seed = c->seed;
  for (int k = 0; k < steps; ++k) {
    prm.u_cur = (k & 1) ? c->ub : c->ua;
    prm.u_pn = (k & 1) ? c->ua : c->ub;
    prm.first = k == 0 ? 1 : 0;
    prm.gpartial = c->gpartial + (1 + 2 * static_cast<int64_t>(k)) * ng;
    NDOS_CHECK(launch_step<T>(plan, kModeDos, prm, s, side));
  }
  k_batch_moments<<<std::min<unsigned>(4096, ceil_div(ng * c->M, 256)), 256, 0, s>>>(c->gpartial, ng, c->M, c->Nz,
                                                                                   G->graph_n, prm.err, c->d_out);
  NDOS_LAUNCHED();
  return DOS_OK;
}

int enqueue_any(int prec, const Graph* G, const Plan& plan, Captured* c, cudaStream_t s, const SideStreams& side) {
  switch (prec) {
    case DOS_BF16:
      return enqueue_batched<__nv_bfloat16>(G, plan, c, s, side);
    case DOS_FP16:
      return enqueue_batched<__half>(G, plan, c, s, side);
    default:
      return enqueue_batched<float>(G, plan, c, s, side);
  }
}

std::mutex g_cap_mu;
cudaStream_t g_cap_stream[64] = {};

int capture_stream(cudaStream_t* out) {
  int dev = 0;
  NDOS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(DOS_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_cap_mu);
  if (!g_cap_stream[dev]) NDOS_CUDA(cudaStreamCreateWithFlags(&g_cap_stream[dev], cudaStreamNonBlocking));
  *out = g_cap_stream[dev];
  return DOS_OK;
}

template <typename T>
int alloc_t(T** p, size_t count) {
  if (alloc_fault_injected()) return fail(DOS_ENOMEM, "injected allocation failure (dos_test_fail_alloc)");
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
  }
  return DOS_OK;
}

int build_captured(Graph* G, const Plan& plan, int M, int Nz, uint64_t seed, int prec, double* d_out) {
  Captured* c = new Captured();
  c->M = M;
  c->Nz = Nz;
  c->seed = seed;
  c->prec = prec;
  c->d_out = d_out;
  c->t = plan.t;
  c->ctas = plan.light_ctas;
  const size_t es = prec == DOS_FP32 ? 4 : 2;
  const size_t elems = static_cast<size_t>(G->n) * plan.nz_pad;
  const int64_t n_raw = 1 + 2 * static_cast<int64_t>(M / 2);
  int st = DOS_OK;
  if ((st = alloc_t(reinterpret_cast<char**>(&c->ua), elems * es)) ||
      (st = alloc_t(reinterpret_cast<char**>(&c->ub), elems * es)) ||
      (st = alloc_t(&c->gpartial, static_cast<size_t>(n_raw * G->n_graphs))) ||
      (st = alloc_t(&c->init_partial, std::max<size_t>(4096, static_cast<size_t>(2 * plan.part_width))))) {
    destroy_captured(c);
    return st;
  }
  cudaStream_t cs = nullptr;
  SideStreams side;
  if ((st = capture_stream(&cs)) || (st = side_streams_for_capture(&side))) {
    destroy_captured(c);
    return st;
  }
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    destroy_captured(c);
    return cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
  }
  st = enqueue_any(prec, G, plan, c, cs, side);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  if (st != DOS_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    destroy_captured(c);
    return st != DOS_OK ? st : cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  }
  c->graph = graph;
  e = cudaGraphInstantiate(&c->exec, graph, 0);
  if (e != cudaSuccess) {
    destroy_captured(c);
    return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
  }
  destroy_captured(G->captured);
  G->captured = c;
  return DOS_OK;
}

}  // namespace
}  // namespace netdos

using namespace netdos;

extern "C" {

int dos_batch_info(dos_graph_t g, int64_t* n_graphs, int64_t* graph_n, int64_t* graph_isolated) {
  if (!g) return fail(DOS_EINVAL, "dos_batch_info: null graph");
  const Graph* G = reinterpret_cast<const Graph*>(g);
  if (n_graphs) *n_graphs = G->n_graphs;
  for (int64_t i = 0; i < G->n_graphs; ++i) {
    if (graph_n) graph_n[i] = G->h_graph_n[i];
    if (graph_isolated) graph_isolated[i] = G->h_graph_iso[i];
  }
  return DOS_OK;
}

int dos_moments_batched(dos_graph_t g, int M, int Nz, uint64_t seed, int prec, double* d_out, void* stream) {
  clear_error();
  if (!g || !d_out) return fail(DOS_EINVAL, "dos_moments_batched: null argument");
  Graph* G = reinterpret_cast<Graph*>(g);
  if (G->n_graphs < 1) return fail(DOS_EINVAL, "dos_moments_batched: graph was not built by dos_build_csr_batched");
  if (G->n < 1) return fail(DOS_EINVAL, "dos_moments_batched: the batch has no edges");
  if (M < 2 || M > (1 << 20)) return fail(DOS_EINVAL, "dos_moments_batched: M must be in [2, 2^20]");
  if (Nz < 1 || Nz > 65536) return fail(DOS_EINVAL, "dos_moments_batched: Nz must be in [1, 65536]");
  if (prec != DOS_FP32 && prec != DOS_BF16 && prec != DOS_FP16) return fail(DOS_EINVAL, "unknown precision");
  Plan plan;
  NDOS_CHECK(make_plan(G, Nz, prec, kModeDos, &plan));
  const Captured* c = G->captured;
  const bool hit = c && c->M == M && c->Nz == Nz && c->seed == seed && c->prec == prec && c->d_out == d_out &&
                   c->t == plan.t && c->ctas == plan.light_ctas;
  if (!hit) NDOS_CHECK(build_captured(G, plan, M, Nz, seed, prec, d_out));
  count_launch();  // one graph launch (its kernels were counted when captured)
  NDOS_CUDA(cudaGraphLaunch(G->captured->exec, static_cast<cudaStream_t>(stream)));
  return DOS_OK;
}

int dos_autotune(dos_graph_t g, int Nz, int prec, void* stream, int* tile_width, int* ctas_per_sm) {
  clear_error();
  if (!g) return fail(DOS_EINVAL, "dos_autotune: null graph");
  Graph* G = reinterpret_cast<Graph*>(g);
  if (G->n < 1) return fail(DOS_EINVAL, "dos_autotune: graph has no edges");
  if (Nz < 1 || Nz > 65536) return fail(DOS_EINVAL, "dos_autotune: Nz must be in [1, 65536]");
  if (prec != DOS_FP32 && prec != DOS_BF16 && prec != DOS_FP16) return fail(DOS_EINVAL, "unknown precision");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int V = prec == DOS_FP32 ? 4 : 8;
  const int qmax = prec == DOS_FP32 ? 16 : 8;
  constexpr int kTuneM = 14;  // 7 fused steps per timing
  double* d = nullptr;
  NDOS_CHECK(dalloc_t(&d, kTuneM, s));
  cudaEvent_t a = nullptr, b = nullptr;
  NDOS_CUDA(cudaEventCreate(&a));
  NDOS_CUDA(cudaEventCreate(&b));
  G->tuned_t = 0;
  float best = 1e30f;
  int best_t = 0, best_c = 0;
  int st = DOS_OK;
  for (int q = 1; q <= qmax && st == DOS_OK; q *= 2) {
    const int t = q * V;
    if ((Nz + t - 1) / t > 16) continue;  // at most 16 tiles
    for (int ctas = 1; ctas <= 3 && st == DOS_OK; ++ctas) {
      G->tuned_t = t;
      G->tuned_ctas = ctas;
      G->tuned_nz = Nz;
      G->tuned_prec = prec;
      st = dos_moments(g, nullptr, kTuneM, Nz, 1, prec, d, stream);  // warm
      if (st != DOS_OK) break;
      cudaEventRecord(a, s);
      st = dos_moments(g, nullptr, kTuneM, Nz, 1, prec, d, stream);
      cudaEventRecord(b, s);
      if (cudaEventSynchronize(b) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "autotune", __FILE__, __LINE__);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (st == DOS_OK && ms < best) {
        best = ms;
        best_t = t;
        best_c = ctas;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  dfree(d, s);
  G->tuned_t = best_t;
  G->tuned_ctas = best_c;
  G->tuned_nz = Nz;
  G->tuned_prec = prec;
  if (st != DOS_OK) {
    G->tuned_t = 0;
    return st;
  }
  if (tile_width) *tile_width = best_t;
  if (ctas_per_sm) *ctas_per_sm = best_c;
  return DOS_OK;
}

}  // extern "C"
