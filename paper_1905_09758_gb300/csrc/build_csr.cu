// dos_build_csr: undirected edge list -> CSR of A (compact ids), degrees,
// D^{-1/2} (§2.1), and the degree-sorted (or degree-class) relabelling used
// by the Chebyshev kernels.  Sorting and prefix sums use CUB's device primitives; every other
// step is a kernel of this file.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_select.cuh>

#include <string>
#include <vector>

#include "alloc_hook.h"
#include "common.cuh"

namespace netdos {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n, int per_block = kThreads) {
  int64_t b = (n + per_block - 1) / per_block;
  int64_t cap = static_cast<int64_t>(num_sms()) * 32;
  if (b > cap) b = cap;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}

inline int bits_for(uint64_t x) {
  int b = 0;
  while (b < 64 && (x >> b) != 0) ++b;
  return b;
}

// 2 directed keys (u << 32 | v) per undirected edge; self-loops and invalid
// endpoints become the sentinel n << 32 (sorted past every real key).
__global__ void k_make_keys(const int64_t* __restrict__ src, const int64_t* __restrict__ dst,
                            int64_t n_edges, int64_t n, uint64_t* __restrict__ keys,
                            int* __restrict__ bad) {
  const uint64_t sent = static_cast<uint64_t>(n) << 32;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_edges;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = src[e], v = dst[e];
    uint64_t k0 = sent, k1 = sent;
    if (u < 0 || u >= n || v < 0 || v >= n) {
      atomicOr(bad, 1);
    } else if (u != v) {
      k0 = (static_cast<uint64_t>(u) << 32) | static_cast<uint64_t>(v);
      k1 = (static_cast<uint64_t>(v) << 32) | static_cast<uint64_t>(u);
    }
    keys[2 * e] = k0;
    keys[2 * e + 1] = k1;
  }
}

__global__ void k_count_deg(const uint64_t* __restrict__ keys, int64_t nnz, int32_t* __restrict__ deg_full) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&deg_full[keys[k] >> 32], 1);
}

__global__ void k_keep_flag(const int32_t* __restrict__ deg_full, int64_t n, int32_t* __restrict__ keep) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n;
       o += (int64_t)gridDim.x * blockDim.x)
    keep[o] = deg_full[o] > 0 ? 1 : 0;
}

__global__ void k_compact_nodes(const int32_t* __restrict__ deg_full, const int32_t* __restrict__ new_id,
                                int64_t n, int32_t* __restrict__ old_id, int32_t* __restrict__ deg,
                                int64_t* __restrict__ deg64, double* __restrict__ s64,
                                float* __restrict__ s32) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = deg_full[o];
    if (d > 0) {
      const int32_t k = new_id[o];
      old_id[k] = static_cast<int32_t>(o);
      deg[k] = d;
      deg64[k] = d;
      // IEEE double sqrt and division are correctly rounded
      const double s = 1.0 / sqrt(static_cast<double>(d));
      s64[k] = s;
      s32[k] = static_cast<float>(s);
    }
  }
}

__global__ void k_fill_col(const uint64_t* __restrict__ keys, int64_t nnz, const int32_t* __restrict__ new_id,
                           int32_t* __restrict__ col) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    col[k] = new_id[keys[k] & 0xffffffffull];
}

__global__ void k_deg_sort_key(const int32_t* __restrict__ deg, int64_t n, uint32_t* __restrict__ key,
                               int32_t* __restrict__ idx) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    key[k] = 0x7fffffffu - static_cast<uint32_t>(deg[k]);
    idx[k] = static_cast<int32_t>(k);
  }
}

// Class order (DOS_ORDER_BY_CLASS): heavy, medium, light; the stable sort
// keeps compact-id order inside a class.
__global__ void k_class_sort_key(const int32_t* __restrict__ deg, int64_t n, uint32_t* __restrict__ key,
                                 int32_t* __restrict__ idx) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = deg[k];
    key[k] = d >= kHeavyDeg ? 0u : (d >= kMediumDeg ? 1u : 2u);
    idx[k] = static_cast<int32_t>(k);
  }
}

// Batch order: heavy rows (degree >= kHeavyDeg) first by degree, then medium
// and light rows, each class grouped by graph and degree-descending inside a
// graph.  Rows processed together then gather from one graph's block of U_k
// (a few MB, L2-resident) instead of from the whole batch.
__global__ void k_batch_sort_key(const int32_t* __restrict__ deg, const int32_t* __restrict__ old_id, int64_t n,
                                 const int64_t* __restrict__ node_off, int64_t n_graphs, uint64_t* __restrict__ key,
                                 int32_t* __restrict__ idx) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = old_id[k];
    int64_t lo = 0, hi = n_graphs - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (node_off[mid] <= o) lo = mid; else hi = mid - 1;
    }
    const uint64_t d = static_cast<uint64_t>(deg[k]);
    if (d >= static_cast<uint64_t>(kHeavyDeg))
      key[k] = 0x7fffffffull - d;
    else
      key[k] = ((d >= static_cast<uint64_t>(kMediumDeg) ? 1ull : 2ull) << 62) | (static_cast<uint64_t>(lo) << 11) |
               (2047ull - d);
    idx[k] = static_cast<int32_t>(k);
  }
}

__global__ void k_perm_nodes(const int32_t* __restrict__ p_compact, int64_t n, const int32_t* __restrict__ deg,
                             const int32_t* __restrict__ old_id, int32_t* __restrict__ compact_to_p,
                             int32_t* __restrict__ p_deg, int64_t* __restrict__ p_deg64,
                             int32_t* __restrict__ p_orig, unsigned long long* __restrict__ n_heavy,
                             unsigned long long* __restrict__ n_mid, unsigned long long* __restrict__ max_deg,
                             int heavy_deg, int mid_deg) {
  unsigned dmax = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = p_compact[p];
    compact_to_p[k] = static_cast<int32_t>(p);
    const int32_t d = deg[k];
    p_deg[p] = d;
    p_deg64[p] = d;
    p_orig[p] = old_id[k];
    if (d >= heavy_deg) atomicAdd(n_heavy, 1ull);
    if (d >= mid_deg) atomicAdd(n_mid, 1ull);
    dmax = max(dmax, static_cast<unsigned>(d));
  }
  dmax = __reduce_max_sync(0xffffffffu, dmax);
  if ((threadIdx.x & 31) == 0 && dmax > 0) atomicMax(max_deg, static_cast<unsigned long long>(dmax));
}

// relabelled nonzero keys (pos(u) << 32 | pos(v)) from the unique original keys
__global__ void k_perm_keys(const uint64_t* __restrict__ keys, int64_t nnz, const int32_t* __restrict__ new_id,
                            const int32_t* __restrict__ compact_to_p, uint64_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = keys[k];
    const uint64_t pu = static_cast<uint32_t>(compact_to_p[new_id[key >> 32]]);
    const uint64_t pv = static_cast<uint32_t>(compact_to_p[new_id[key & 0xffffffffull]]);
    out[k] = (pu << 32) | pv;
  }
}

// graph of each position (largest g with node_off[g] <= original id) and
// the non-isolated node count of each graph
__global__ void k_graph_of(const int32_t* __restrict__ p_orig, int64_t n, const int64_t* __restrict__ node_off,
                           int64_t n_graphs, int32_t* __restrict__ p_gid, unsigned long long* __restrict__ count) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = p_orig[p];
    int64_t lo = 0, hi = n_graphs - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (node_off[mid] <= o) lo = mid; else hi = mid - 1;
    }
    p_gid[p] = static_cast<int32_t>(lo);
    atomicAdd(&count[lo], 1ull);
  }
}

// every edge must join two nodes of the same graph (warp per row)
__global__ void k_check_within(const int64_t* __restrict__ p_row_ptr, const int32_t* __restrict__ p_col,
                               const int32_t* __restrict__ p_gid, int64_t n, int* __restrict__ bad) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = w0; p < n; p += nw) {
    const int32_t g = p_gid[p];
    for (int64_t e = p_row_ptr[p] + lane; e < p_row_ptr[p + 1]; e += 32)
      if (p_gid[p_col[e]] != g) atomicOr(bad, 1);
  }
}

__global__ void k_low_word(const uint64_t* __restrict__ keys, int64_t nnz, int32_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = static_cast<int32_t>(keys[k] & 0xffffffffull);
}


template <typename T>
int persistent_alloc(T** p, size_t count) {
  *p = nullptr;
  if (alloc_fault_injected()) return fail(DOS_ENOMEM, "injected allocation failure (dos_test_fail_alloc)");
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
  }
  return DOS_OK;
}

// exclusive prefix sum of int64 values into out[0..n], out[n] = total
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, Temps& t) {
  size_t bytes = 0;
  NDOS_CUDA(cub::DeviceScan::InclusiveSum(nullptr, bytes, in, out + 1, n, t.s));
  void* tmp = nullptr;
  NDOS_CHECK(t.get(reinterpret_cast<char**>(&tmp), bytes));
  NDOS_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), t.s));
  if (n > 0) NDOS_CUDA(cub::DeviceScan::InclusiveSum(tmp, bytes, in, out + 1, n, t.s));
  count_launch();
  return DOS_OK;
}

int sort_keys_u64(uint64_t*& keys, uint64_t*& alt, int64_t n, int end_bit, Temps& t) {
  if (n <= 1) return DOS_OK;
  cub::DoubleBuffer<uint64_t> db(keys, alt);
  size_t bytes = 0;
  NDOS_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, bytes, db, n, 0, end_bit, t.s));
  void* tmp = nullptr;
  NDOS_CHECK(t.get(reinterpret_cast<char**>(&tmp), bytes));
  NDOS_CUDA(cub::DeviceRadixSort::SortKeys(tmp, bytes, db, n, 0, end_bit, t.s));
  count_launch();
  if (db.Current() != keys) std::swap(keys, alt);
  return DOS_OK;
}

}  // namespace

// node_offset [host] (n_graphs + 1 entries) or NULL: with a batch, rows are
// ordered graph by graph inside the medium and light classes
static int build_csr_impl(const int64_t* src_in, const int64_t* dst_in, int64_t n_edges, int64_t n_nodes,
                          uint32_t flags, const int64_t* node_offset, int64_t n_graphs, cudaStream_t s, Graph* G) {
  Temps t(s);
  const int64_t* src = src_in;
  const int64_t* dst = dst_in;
  // host input: page-locked buffers are read in place by k_make_keys through
  // their device mapping (no 16-byte-per-edge device copy); pageable ones are
  // copied to temporaries first
  bool mapped = false;
  if ((flags & DOS_INPUT_HOST) && n_edges > 0) {
    cudaPointerAttributes as{}, ad{};
    if (cudaPointerGetAttributes(&as, src_in) == cudaSuccess && cudaPointerGetAttributes(&ad, dst_in) == cudaSuccess &&
        as.type == cudaMemoryTypeHost && ad.type == cudaMemoryTypeHost && as.devicePointer && ad.devicePointer) {
      src = static_cast<const int64_t*>(as.devicePointer);
      dst = static_cast<const int64_t*>(ad.devicePointer);
      mapped = true;
    }
    cudaGetLastError();  // an unregistered pointer is not an error here
  }
  if ((flags & DOS_INPUT_HOST) && n_edges > 0 && !mapped) {
    int64_t *ds = nullptr, *dd = nullptr;
    NDOS_CHECK(t.get(&ds, n_edges));
    NDOS_CHECK(t.get(&dd, n_edges));
    NDOS_CUDA(cudaMemcpyAsync(ds, src_in, sizeof(int64_t) * n_edges, cudaMemcpyHostToDevice, s));
    NDOS_CUDA(cudaMemcpyAsync(dd, dst_in, sizeof(int64_t) * n_edges, cudaMemcpyHostToDevice, s));
    src = ds;
    dst = dd;
  }
  const int64_t n_keys = 2 * n_edges;
  int* bad = nullptr;
  uint64_t *keys = nullptr, *alt = nullptr;
  NDOS_CHECK(t.get(&bad, 1));
  NDOS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  NDOS_CHECK(t.get(&keys, n_keys));
  NDOS_CHECK(t.get(&alt, n_keys));
  if (n_edges > 0) {
    k_make_keys<<<grid_for(n_edges), kThreads, 0, s>>>(src, dst, n_edges, n_nodes, keys, bad);
    NDOS_LAUNCHED();
  }
  const int end_bit = 32 + bits_for(static_cast<uint64_t>(n_nodes));
  NDOS_CHECK(sort_keys_u64(keys, alt, n_keys, end_bit, t));

  // unique (sorted) keys -> alt, count on device
  int64_t* n_uniq_d = nullptr;
  NDOS_CHECK(t.get(&n_uniq_d, 1));
  NDOS_CUDA(cudaMemsetAsync(n_uniq_d, 0, sizeof(int64_t), s));
  if (n_keys > 0) {
    size_t bytes = 0;
    NDOS_CUDA(cub::DeviceSelect::Unique(nullptr, bytes, keys, alt, n_uniq_d, n_keys, s));
    void* tmp = nullptr;
    NDOS_CHECK(t.get(reinterpret_cast<char**>(&tmp), bytes));
    NDOS_CUDA(cub::DeviceSelect::Unique(tmp, bytes, keys, alt, n_uniq_d, n_keys, s));
    count_launch();
  }
  int64_t n_uniq = 0;
  int h_bad = 0;
  NDOS_CUDA(cudaMemcpyAsync(&n_uniq, n_uniq_d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  NDOS_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  uint64_t last_key = 0;
  if (n_keys > 0) {
    NDOS_CUDA(cudaStreamSynchronize(s));
    if (n_uniq > 0)
      NDOS_CUDA(cudaMemcpyAsync(&last_key, alt + n_uniq - 1, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  }
  NDOS_CUDA(cudaStreamSynchronize(s));
  if (h_bad) return fail(DOS_EINVAL, "dos_build_csr: edge endpoint outside [0, n_nodes)");
  // drop the sentinel run (self-loops), which sorts last
  const uint64_t sent = static_cast<uint64_t>(n_nodes) << 32;
  const int64_t nnz = (n_uniq > 0 && last_key == sent) ? n_uniq - 1 : n_uniq;
  uint64_t* uk = alt;  // unique keys, CSR order

  int32_t *deg_full = nullptr, *keep = nullptr, *new_id = nullptr;
  NDOS_CHECK(t.get(&deg_full, n_nodes));
  NDOS_CHECK(t.get(&keep, n_nodes + 1));
  NDOS_CHECK(t.get(&new_id, n_nodes + 1));
  NDOS_CUDA(cudaMemsetAsync(deg_full, 0, sizeof(int32_t) * (n_nodes ? n_nodes : 1), s));
  if (nnz > 0) {
    k_count_deg<<<grid_for(nnz), kThreads, 0, s>>>(uk, nnz, deg_full);
    NDOS_LAUNCHED();
  }
  int32_t n_keep = 0;
  if (n_nodes > 0) {
    k_keep_flag<<<grid_for(n_nodes), kThreads, 0, s>>>(deg_full, n_nodes, keep);
    NDOS_LAUNCHED();
    size_t bytes = 0;
    NDOS_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, keep, new_id, n_nodes + 1, s));
    void* tmp = nullptr;
    NDOS_CHECK(t.get(reinterpret_cast<char**>(&tmp), bytes));
    NDOS_CUDA(cudaMemsetAsync(keep + n_nodes, 0, sizeof(int32_t), s));
    NDOS_CUDA(cub::DeviceScan::ExclusiveSum(tmp, bytes, keep, new_id, n_nodes + 1, s));
    count_launch();
    NDOS_CUDA(cudaMemcpyAsync(&n_keep, new_id + n_nodes, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    NDOS_CUDA(cudaStreamSynchronize(s));
  }
  const int64_t n = n_keep;
  G->n = n;
  G->nnz = nnz;
  G->n_original = n_nodes;
  G->n_isolated = n_nodes - n;

  NDOS_CHECK(persistent_alloc(&G->row_ptr, n + 1));
  NDOS_CHECK(persistent_alloc(&G->col, nnz));
  NDOS_CHECK(persistent_alloc(&G->deg, n));
  NDOS_CHECK(persistent_alloc(&G->s64, n));
  NDOS_CHECK(persistent_alloc(&G->s32, n));
  NDOS_CHECK(persistent_alloc(&G->old_id, n));
  // the hot-path arrays are padded: the step kernel's bulk copies round
  // their ranges out to 16-byte boundaries
  NDOS_CHECK(persistent_alloc(&G->p_row_ptr, n + 3));
  NDOS_CHECK(persistent_alloc(&G->p_col, nnz + 4));
  NDOS_CHECK(persistent_alloc(&G->p_deg, n));
  NDOS_CHECK(persistent_alloc(&G->p_orig, n + 4));
  NDOS_CHECK(persistent_alloc(&G->p_compact, n + 4));
  NDOS_CUDA(cudaMemsetAsync(G->p_row_ptr, 0, sizeof(int64_t) * (n + 3), s));
  NDOS_CUDA(cudaMemsetAsync(G->p_col, 0, sizeof(int32_t) * (nnz + 4), s));
  NDOS_CUDA(cudaMemsetAsync(G->p_orig, 0, sizeof(int32_t) * (n + 4), s));
  NDOS_CUDA(cudaMemsetAsync(G->p_compact, 0, sizeof(int32_t) * (n + 4), s));
  NDOS_CHECK(persistent_alloc(&G->compact_to_p, n));

  int64_t* deg64 = nullptr;
  NDOS_CHECK(t.get(&deg64, n + 1));
  if (n_nodes > 0) {
    k_compact_nodes<<<grid_for(n_nodes), kThreads, 0, s>>>(deg_full, new_id, n_nodes, G->old_id, G->deg, deg64,
                                                          G->s64, G->s32);
    NDOS_LAUNCHED();
  }
  NDOS_CHECK(exclusive_scan_i64(deg64, G->row_ptr, n, t));
  if (nnz > 0) {
    k_fill_col<<<grid_for(nnz), kThreads, 0, s>>>(uk, nnz, new_id, G->col);
    NDOS_LAUNCHED();
  }

  // ---- degree-sorted relabelling ----
  // [0] deg >= kHeavyDeg, [1] deg >= kMediumDeg, [2] the largest degree
  unsigned long long* n_heavy_d = nullptr;
  NDOS_CHECK(t.get(&n_heavy_d, 3));
  NDOS_CUDA(cudaMemsetAsync(n_heavy_d, 0, 3 * sizeof(unsigned long long), s));
  if (n > 0) {
    int32_t *idx = nullptr, *idx_alt = nullptr;
    NDOS_CHECK(t.get(&idx, n));
    NDOS_CHECK(t.get(&idx_alt, n));
    cub::DoubleBuffer<int32_t> vb(idx, idx_alt);
    size_t bytes = 0;
    void* tmp = nullptr;
    if (node_offset && n_graphs > 1) {
      uint64_t *bk = nullptr, *bk_alt = nullptr;
      int64_t* off = nullptr;
      NDOS_CHECK(t.get(&bk, n));
      NDOS_CHECK(t.get(&bk_alt, n));
      NDOS_CHECK(t.get(&off, n_graphs + 1));
      NDOS_CUDA(cudaMemcpyAsync(off, node_offset, sizeof(int64_t) * (n_graphs + 1), cudaMemcpyHostToDevice, s));
      k_batch_sort_key<<<grid_for(n), kThreads, 0, s>>>(G->deg, G->old_id, n, off, n_graphs, bk, idx);
      NDOS_LAUNCHED();
      cub::DoubleBuffer<uint64_t> kb(bk, bk_alt);
      NDOS_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, kb, vb, n, 0, 64, s));
      NDOS_CHECK(t.get(reinterpret_cast<char**>(&tmp), bytes));
      NDOS_CUDA(cub::DeviceRadixSort::SortPairs(tmp, bytes, kb, vb, n, 0, 64, s));
    } else {
      uint32_t *dk = nullptr, *dk_alt = nullptr;
      NDOS_CHECK(t.get(&dk, n));
      NDOS_CHECK(t.get(&dk_alt, n));
      const bool by_class = (flags & DOS_ORDER_BY_CLASS) != 0;
      if (by_class)
        k_class_sort_key<<<grid_for(n), kThreads, 0, s>>>(G->deg, n, dk, idx);
      else
        k_deg_sort_key<<<grid_for(n), kThreads, 0, s>>>(G->deg, n, dk, idx);
      NDOS_LAUNCHED();
      const int end_bit = by_class ? 2 : 31;
      cub::DoubleBuffer<uint32_t> kb(dk, dk_alt);
      NDOS_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, kb, vb, n, 0, end_bit, s));
      NDOS_CHECK(t.get(reinterpret_cast<char**>(&tmp), bytes));
      NDOS_CUDA(cub::DeviceRadixSort::SortPairs(tmp, bytes, kb, vb, n, 0, end_bit, s));
    }
    count_launch();
    NDOS_CUDA(cudaMemcpyAsync(G->p_compact, vb.Current(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    int64_t* pdeg64 = nullptr;
    NDOS_CHECK(t.get(&pdeg64, n));
    k_perm_nodes<<<grid_for(n), kThreads, 0, s>>>(G->p_compact, n, G->deg, G->old_id, G->compact_to_p, G->p_deg,
                                                 pdeg64, G->p_orig, n_heavy_d, n_heavy_d + 1, n_heavy_d + 2,
                                                 kHeavyDeg, kMediumDeg);
    NDOS_LAUNCHED();
    NDOS_CHECK(exclusive_scan_i64(pdeg64, G->p_row_ptr, n, t));
  } else {
    NDOS_CUDA(cudaMemsetAsync(G->row_ptr, 0, sizeof(int64_t), s));
    NDOS_CUDA(cudaMemsetAsync(G->p_row_ptr, 0, sizeof(int64_t), s));
  }
  if (nnz > 0) {
    // keys buffer (no longer needed) receives the relabelled keys
    k_perm_keys<<<grid_for(nnz), kThreads, 0, s>>>(uk, nnz, new_id, G->compact_to_p, keys);
    NDOS_LAUNCHED();
    uint64_t* k2 = keys;
    uint64_t* k2_alt = alt;  // unique keys are consumed by now
    NDOS_CHECK(sort_keys_u64(k2, k2_alt, nnz, 32 + bits_for(static_cast<uint64_t>(n)), t));
    k_low_word<<<grid_for(nnz), kThreads, 0, s>>>(k2, nnz, G->p_col);
    NDOS_LAUNCHED();
  }
  unsigned long long nh[3] = {0, 0, 0};
  NDOS_CUDA(cudaMemcpyAsync(nh, n_heavy_d, sizeof(nh), cudaMemcpyDeviceToHost, s));
  NDOS_CUDA(cudaStreamSynchronize(s));
  G->n_heavy = static_cast<int64_t>(nh[0]);
  G->n_mid = static_cast<int64_t>(nh[1]);
  G->max_deg = static_cast<int32_t>(nh[2]);

  return DOS_OK;
}

}  // namespace netdos

using namespace netdos;

static int build_graph(const int64_t* src, const int64_t* dst, int64_t n_edges, int64_t n_nodes, uint32_t flags,
                       const int64_t* node_offset, int64_t n_graphs, void* stream, dos_graph_t* out,
                       const char* who) {
  const std::string w(who);
  if (n_edges < 0 || n_nodes < 0) return fail(DOS_EINVAL, w + ": negative size");
  if (n_nodes > 0x7fffffffLL) return fail(DOS_EOVERFLOW, w + ": n_nodes exceeds 2^31 - 1");
  if (n_edges > (1LL << 40)) return fail(DOS_EOVERFLOW, w + ": n_edges exceeds 2^40");
  if (n_edges > 0 && (!src || !dst)) return fail(DOS_EINVAL, w + ": null edge arrays");
  if (flags & ~static_cast<uint32_t>(DOS_INPUT_HOST | DOS_ORDER_BY_CLASS)) return fail(DOS_EINVAL, w + ": unknown flags");
  if ((flags & DOS_ORDER_BY_CLASS) && node_offset)
    return fail(DOS_EINVAL, w + ": DOS_ORDER_BY_CLASS is for single graphs (a batch is grouped by graph)");
  Graph* G = new Graph();
  cudaGetDevice(&G->device);
  int st = build_csr_impl(src, dst, n_edges, n_nodes, flags, node_offset, n_graphs, static_cast<cudaStream_t>(stream),
                          G);
  if (st != DOS_OK) {
    dos_graph_destroy(reinterpret_cast<dos_graph_t>(G));
    return st;
  }
  *out = reinterpret_cast<dos_graph_t>(G);
  return DOS_OK;
}

static int tag_graphs(Graph* G, const int64_t* node_offset, int64_t n_graphs, cudaStream_t s) {
  Temps t(s);
  int64_t* off = nullptr;
  unsigned long long* cnt = nullptr;
  int* bad = nullptr;
  NDOS_CHECK(t.get(&off, n_graphs + 1));
  NDOS_CHECK(t.get(&cnt, n_graphs));
  NDOS_CHECK(t.get(&bad, 1));
  NDOS_CHECK(persistent_alloc(&G->p_gid, G->n));
  NDOS_CHECK(persistent_alloc(&G->graph_n, n_graphs));
  NDOS_CUDA(cudaMemcpyAsync(off, node_offset, sizeof(int64_t) * (n_graphs + 1), cudaMemcpyHostToDevice, s));
  NDOS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * n_graphs, s));
  NDOS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  if (G->n > 0) {
    k_graph_of<<<grid_for(G->n), kThreads, 0, s>>>(G->p_orig, G->n, off, n_graphs, G->p_gid, cnt);
    NDOS_LAUNCHED();
    k_check_within<<<grid_for(G->n * 32), kThreads, 0, s>>>(G->p_row_ptr, G->p_col, G->p_gid, G->n, bad);
    NDOS_LAUNCHED();
  }
  std::vector<unsigned long long> h(n_graphs);
  int h_bad = 0;
  NDOS_CUDA(cudaMemcpyAsync(h.data(), cnt, sizeof(unsigned long long) * n_graphs, cudaMemcpyDeviceToHost, s));
  NDOS_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  NDOS_CUDA(cudaStreamSynchronize(s));
  if (h_bad) return fail(DOS_EINVAL, "dos_build_csr_batched: an edge joins nodes of two different graphs");
  G->n_graphs = n_graphs;
  G->h_graph_n.resize(n_graphs);
  G->h_graph_iso.resize(n_graphs);
  for (int64_t g = 0; g < n_graphs; ++g) {
    G->h_graph_n[g] = static_cast<int64_t>(h[g]);
    G->h_graph_iso[g] = (node_offset[g + 1] - node_offset[g]) - G->h_graph_n[g];
  }
  NDOS_CUDA(cudaMemcpyAsync(G->graph_n, G->h_graph_n.data(), sizeof(int64_t) * n_graphs, cudaMemcpyHostToDevice, s));
  NDOS_CUDA(cudaStreamSynchronize(s));
  return DOS_OK;
}

extern "C" int dos_build_csr_batched(const int64_t* src, const int64_t* dst, int64_t n_edges,
                                     const int64_t* node_offset, int64_t n_graphs, uint32_t flags, void* stream,
                                     dos_graph_t* out) {
  clear_error();
  if (!out) return fail(DOS_EINVAL, "dos_build_csr_batched: out is NULL");
  *out = nullptr;
  if (!node_offset || n_graphs < 1) return fail(DOS_EINVAL, "dos_build_csr_batched: need node_offset and n_graphs >= 1");
  if (n_graphs > 0x7fffffffLL) return fail(DOS_EOVERFLOW, "dos_build_csr_batched: too many graphs");
  if (node_offset[0] != 0) return fail(DOS_EINVAL, "dos_build_csr_batched: node_offset[0] must be 0");
  for (int64_t g = 0; g < n_graphs; ++g)
    if (node_offset[g + 1] < node_offset[g]) return fail(DOS_EINVAL, "dos_build_csr_batched: node_offset decreases");
  dos_graph_t h = nullptr;
  NDOS_CHECK(build_graph(src, dst, n_edges, node_offset[n_graphs], flags, node_offset, n_graphs, stream, &h,
                         "dos_build_csr_batched"));
  Graph* G = reinterpret_cast<Graph*>(h);
  const int st = tag_graphs(G, node_offset, n_graphs, static_cast<cudaStream_t>(stream));
  if (st != DOS_OK) {
    dos_graph_destroy(h);
    return st;
  }
  *out = h;
  return DOS_OK;
}

extern "C" int dos_build_csr(const int64_t* src, const int64_t* dst, int64_t n_edges, int64_t n_nodes,
                             uint32_t flags, void* stream, dos_graph_t* out) {
  clear_error();
  if (!out) return fail(DOS_EINVAL, "dos_build_csr: out is NULL");
  *out = nullptr;
  return build_graph(src, dst, n_edges, n_nodes, flags, nullptr, 0, stream, out, "dos_build_csr");
}
