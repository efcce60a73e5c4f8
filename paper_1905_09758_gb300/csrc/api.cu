// Library-wide ABI entry points: errors, version, handle queries and
// exports, launch accounting and step-kernel timing.
#include <cstdio>
#include <mutex>
#include <vector>

#include "alloc_hook.h"
#include "common.cuh"

namespace netdos {

// allocations left before the injected failure (-1: disarmed)
static std::atomic<int64_t> g_fail_after{-1};

bool alloc_fault_injected() {
  int64_t v = g_fail_after.load(std::memory_order_relaxed);
  while (v >= 0) {
    if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
  }
  return false;
}

static thread_local std::string t_last_error;
std::atomic<int64_t> g_launches{0};

void set_error(const std::string& msg) { t_last_error = msg; }
void clear_error() { t_last_error.clear(); }

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s) at %s:%d", what, cudaGetErrorName(e),
           cudaGetErrorString(e), file, line);
  set_error(buf);
  return e == cudaErrorMemoryAllocation ? DOS_ENOMEM : DOS_ECUDA;
}

int dalloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (alloc_fault_injected()) return fail(DOS_ENOMEM, "injected allocation failure (dos_test_fail_alloc)");
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "cudaMallocAsync", __FILE__, __LINE__);
  }
  return DOS_OK;
}

void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// ---------------------------------------------------------------------------
// step-kernel timing: event pairs recorded around each launch
// ---------------------------------------------------------------------------
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_events;
static std::vector<cudaEvent_t> g_prof_pool;
static thread_local cudaEvent_t t_pending = nullptr;

bool profiling_on() { return g_prof_on; }

static cudaEvent_t take_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void profile_begin(cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  t_pending = take_event();
  cudaEventRecord(t_pending, s);
}

void profile_end(cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t e = take_event();
  cudaEventRecord(e, s);
  g_prof_events.emplace_back(t_pending, e);
  t_pending = nullptr;
}

}  // namespace netdos

using namespace netdos;

extern "C" {

int dos_version(void) { return 100; }

const char* dos_last_error(void) { return t_last_error.c_str(); }

int64_t dos_launch_count(void) { return g_launches.load(); }

int dos_test_fail_alloc(int64_t after) {
  g_fail_after.store(after >= 0 ? after : -1);
  return DOS_OK;
}

int dos_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return DOS_OK;
}

int dos_profile_read(double* total_ms, int64_t* launches, int reset) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  double tot = 0.0;
  for (auto& pr : g_prof_events) {
    cudaError_t e = cudaEventSynchronize(pr.second);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize", __FILE__, __LINE__);
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, pr.first, pr.second);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime", __FILE__, __LINE__);
    tot += ms;
  }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = static_cast<int64_t>(g_prof_events.size());
  if (reset) {
    for (auto& pr : g_prof_events) {
      g_prof_pool.push_back(pr.first);
      g_prof_pool.push_back(pr.second);
    }
    g_prof_events.clear();
  }
  return DOS_OK;
}

int dos_graph_info(dos_graph_t g, int64_t* n, int64_t* nnz, int64_t* n_isolated,
                   int64_t* n_original) {
  if (!g) return fail(DOS_EINVAL, "dos_graph_info: null graph");
  const Graph* G = reinterpret_cast<const Graph*>(g);
  if (n) *n = G->n;
  if (nnz) *nnz = G->nnz;
  if (n_isolated) *n_isolated = G->n_isolated;
  if (n_original) *n_original = G->n_original;
  return DOS_OK;
}

int dos_graph_export(dos_graph_t g, int64_t* row_ptr, int32_t* col, int32_t* deg,
                     double* inv_sqrt_deg, float* inv_sqrt_deg32, int32_t* old_id,
                     void* stream) {
  if (!g) return fail(DOS_EINVAL, "dos_graph_export: null graph");
  const Graph* G = reinterpret_cast<const Graph*>(g);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const auto cp = [&](void* dst, const void* src, size_t bytes) -> int {
    if (dst && bytes) NDOS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
    return DOS_OK;
  };
  NDOS_CHECK(cp(row_ptr, G->row_ptr, sizeof(int64_t) * (G->n + 1)));
  NDOS_CHECK(cp(col, G->col, sizeof(int32_t) * G->nnz));
  NDOS_CHECK(cp(deg, G->deg, sizeof(int32_t) * G->n));
  NDOS_CHECK(cp(inv_sqrt_deg, G->s64, sizeof(double) * G->n));
  NDOS_CHECK(cp(inv_sqrt_deg32, G->s32, sizeof(float) * G->n));
  NDOS_CHECK(cp(old_id, G->old_id, sizeof(int32_t) * G->n));
  return DOS_OK;
}

void dos_graph_destroy(dos_graph_t g) {
  if (!g) return;
  Graph* G = reinterpret_cast<Graph*>(g);
  void* ptrs[] = {G->row_ptr, G->col,    G->deg,    G->s64,       G->s32,     G->old_id,
                  G->p_row_ptr, G->p_col, G->p_deg, G->p_orig, G->p_compact, G->compact_to_p, G->p_gid, G->graph_n};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  destroy_captured(G->captured);
  delete G;
}

int dos_filter_info(dos_filter_t f, int64_t* removed, int64_t* n_classes, int64_t* r) {
  if (!f) return fail(DOS_EINVAL, "dos_filter_info: null filter");
  const Filter* F = reinterpret_cast<const Filter*>(f);
  if (removed) *removed = F->removed;
  if (n_classes) *n_classes = F->n_classes;
  if (r) *r = F->g->n - F->removed;
  return DOS_OK;
}

int dos_filter_export(dos_filter_t f, int32_t* class_id, void* stream) {
  if (!f) return fail(DOS_EINVAL, "dos_filter_export: null filter");
  const Filter* F = reinterpret_cast<const Filter*>(f);
  if (class_id && F->g->n)
    NDOS_CUDA(cudaMemcpyAsync(class_id, F->class_id, sizeof(int32_t) * F->g->n,
                              cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
  return DOS_OK;
}

void dos_filter_destroy(dos_filter_t f) {
  if (!f) return;
  Filter* F = reinterpret_cast<Filter*>(f);
  // the buffers are pool allocations: wait for any work still using them,
  // then return them to the pool
  cudaDeviceSynchronize();
  void* ptrs[] = {F->class_id, F->p_slot, F->slot_size};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, 0);
  delete F;
}

}  // extern "C"
