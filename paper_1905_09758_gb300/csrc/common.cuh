// Shared infrastructure of the netdos CUDA library: status handling, the
// graph/filter handle layouts, the device-side SplitMix64 probe generator and
// launch accounting.  Everything here is internal; the ABI is include/netdos.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <utility>
#include <vector>

#include "netdos.h"

namespace netdos {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
void clear_error();

struct Status {
  int code = DOS_OK;
  bool ok() const { return code == DOS_OK; }
};

int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define NDOS_CUDA(call)                                                  \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess)                                               \
      return ::netdos::cuda_fail(e_, #call, __FILE__, __LINE__);         \
  } while (0)

#define NDOS_CHECK(call)                                                 \
  do {                                                                   \
    int s_ = (call);                                                     \
    if (s_ != DOS_OK) return s_;                                         \
  } while (0)

// ---------------------------------------------------------------------------
// launch accounting and step-kernel timing
// ---------------------------------------------------------------------------
extern std::atomic<int64_t> g_launches;
inline void count_launch(int64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }
#define NDOS_LAUNCHED()                                                  \
  do {                                                                   \
    ::netdos::count_launch();                                            \
    cudaError_t e_ = cudaGetLastError();                                 \
    if (e_ != cudaSuccess)                                               \
      return ::netdos::cuda_fail(e_, "kernel launch", __FILE__, __LINE__); \
  } while (0)

bool profiling_on();
// record a start event before / an end event after a step-kernel launch
void profile_begin(cudaStream_t s);
void profile_end(cudaStream_t s);

// ---------------------------------------------------------------------------
// device memory helpers (stream-ordered pool allocations)
// ---------------------------------------------------------------------------
int dalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);

template <typename T>
int dalloc_t(T** p, size_t count, cudaStream_t s) {
  return dalloc(reinterpret_cast<void**>(p), count * sizeof(T), s);
}

// temporaries of one call, released stream-ordered when the call returns
struct Temps {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Temps(cudaStream_t st) : s(st) {}
  ~Temps() {
    for (void* p : ptrs) dfree(p, s);
  }
  template <typename T>
  int get(T** p, size_t count) {
    int st = dalloc_t(p, count, s);
    if (st == DOS_OK) ptrs.push_back(*p);
    return st;
  }
};

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
// Two copies of the operator are kept:
//  * the CSR in compact-id order (the exported, bit-exact one), and
//  * a degree-sorted relabelling used by the Chebyshev kernels.  Rows are
//    ordered by degree (descending, ties by compact id), so heavy rows are a
//    prefix (load balancing) and the most-gathered rows share cache lines;
//    with DOS_ORDER_BY_CLASS only by degree class (heavy, medium, light),
//    compact-id order inside a class, which keeps a numbering's locality.
//    The spectrum is invariant under the relabelling.
struct Graph {
  int64_t n = 0, nnz = 0, n_isolated = 0, n_original = 0;
  int device = 0;
  // compact order
  int64_t* row_ptr = nullptr;   // [n+1]
  int32_t* col = nullptr;       // [nnz]
  int32_t* deg = nullptr;       // [n]
  double* s64 = nullptr;        // [n]
  float* s32 = nullptr;         // [n]
  int32_t* old_id = nullptr;    // [n]
  // degree-sorted order (k = position)
  int64_t* p_row_ptr = nullptr; // [n+1]
  int32_t* p_col = nullptr;     // [nnz]  neighbours as positions
  int32_t* p_deg = nullptr;     // [n]
  int32_t* p_orig = nullptr;    // [n]    original id of position k
  int32_t* p_compact = nullptr; // [n]    compact id of position k
  int32_t* compact_to_p = nullptr; // [n]
  int32_t max_deg = 0;          // largest degree
  int64_t n_heavy = 0;          // positions [0, n_heavy) have deg >= kHeavyDeg
  int64_t n_mid = 0;            // positions [n_heavy, n_mid) have kMediumDeg <= deg < kHeavyDeg
  // a batch of graphs (dos_build_csr_batched): the operator is their disjoint
  // union; n_graphs = 0 for a single graph
  int64_t n_graphs = 0;
  int32_t* p_gid = nullptr;     // [n] graph of position k
  int64_t* graph_n = nullptr;   // [n_graphs] non-isolated nodes per graph (device)
  std::vector<int64_t> h_graph_n, h_graph_iso;  // per graph: non-isolated / isolated nodes
  // plan chosen by dos_autotune (0 = none)
  int tuned_t = 0, tuned_ctas = 0, tuned_nz = 0, tuned_prec = -1;
  // captured batched-moment sequence (dos_moments_batched)
  struct Captured* captured = nullptr;
};

struct Captured;
void destroy_captured(Captured* c);  // batch.cu

struct Filter {
  const Graph* g = nullptr;
  int64_t removed = 0, n_classes = 0;
  int32_t* class_id = nullptr;  // [n] compact ids, smallest member
  // per position k of the degree-sorted order: slot of its nontrivial class
  // (-1 for singletons) and the class size
  int32_t* p_slot = nullptr;    // [n]
  int32_t* slot_size = nullptr; // [n_classes]
  // removed eigenvalues (lambda, count), ascending lambda: 0 for open twins,
  // -1/d for closed twins of degree d
  std::vector<std::pair<double, int64_t>> spikes;
};

constexpr int kHeavyDeg = 2048;  // rows at or above this degree get a whole CTA
constexpr int kMediumDeg = 64;   // rows at or above this degree (and below kHeavyDeg) get a warp

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): n-th output of the stream
// seeded with `seed` is mix(seed + (n + 1) * GAMMA).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// 64 probe sign bits (bit b -> probe 64*w + b; 1 means -1) of original node o
__host__ __device__ __forceinline__ uint64_t probe_word(uint64_t seed, uint32_t o, uint32_t w) {
  return splitmix64(seed, (static_cast<uint64_t>(w) << 32) | o);
}

inline unsigned ceil_div(int64_t a, int64_t b) { return static_cast<unsigned>((a + b - 1) / b); }

int num_sms();

}  // namespace netdos
