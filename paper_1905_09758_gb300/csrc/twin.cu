// dos_motif_filter / dos_motif_filter_ex: classes of nodes with identical
// neighbourhoods (§3.4, Fig. 3).
//   open twins    N(i) = N(j):  eigenvectors e_i - e_j with eigenvalue 0;
//   closed twins  N[i] = N[j] (N[i] = N(i) + {i}, so i ~ j and d_i = d_j = d):
//                 A (e_i - e_j) = e_j - e_i, eigenvalue -1/d of H.
//   pendant twins  nodes of degree d >= 2 with exactly one leaf neighbour and
//                 equal neighbourhoods apart from it: the nodes form one class
//                 and their leaves another; the vectors summing to zero over
//                 each carry c - 1 eigenvalues at each of +-1/sqrt(d) (d = 2:
//                 pendant 2-paths, +-1/sqrt 2; d = 4: the +-1/2 motif).
//   parallel paths  c >= 2 paths E - a - b - F through degree-2 nodes between
//                 the same hosts E != F of degree >= 3: the nodes next to the
//                 smaller host form one class and those next to the larger
//                 another; c - 1 eigenvalues at each of +-1/2.
// The relations are disjoint (no node is in two nontrivial classes), so one
// class id per node and one class-mean projection of the probes filters all.
//
// Detection follows the paper's hashing idea with an integer hash: each node
// gets h_i = mix(d_i) + sum_{j in N(i)} mix(j) (+ mix(i) for closed
// neighbourhoods; the leaf left out for pendant twins) (mod 2^64), an
// order-free function of the neighbour set, so
// twins always share a hash.  Nodes are sorted by hash (stable in the node
// id); inside each run of equal hashes the neighbour lists are compared
// exactly, so a hash collision never merges different neighbourhoods.  Class
// id = smallest member (compact id).
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "alloc_hook.h"
#include "common.cuh"

namespace netdos {
namespace {

__device__ __forceinline__ uint64_t mix_id(uint64_t x) { return splitmix64(0x5bd1e9955bd1e995ull, x); }

// pendant-twin eligibility: d >= 2 and exactly one leaf neighbour
__device__ __forceinline__ bool pendant_eligible(const int32_t* deg, const int32_t* nleaf, int64_t i) {
  return deg[i] >= 2 && nleaf[i] == 1;
}

// Order-free hash of the open (mode 0), closed (1) or leaf-reduced (2,
// pendant twins) neighbourhood of every row; a node that cannot be a pendant
// twin gets a hash of its own (mode 2).  Modes 0 and 1 fold the hash to 32
// bits (half the radix-sort passes; runs of equal keys are resolved by exact
// comparison, so a collision only costs a comparison); mode 2 keeps 64 bits,
// whose top bit marks the nodes that are not eligible.
__device__ __forceinline__ void row_hash_store(int mode, int64_t i, uint64_t h, const int32_t* __restrict__ deg,
                                               uint64_t* __restrict__ hash, int32_t* __restrict__ idx) {
  if (mode == 1) h += mix_id(static_cast<uint64_t>(i)) + 0x9e3779b97f4a7c15ull;
  if (mode == 2) h += 0x3c6ef372fe94f82bull;
  h += mix_id(0x8000000000000000ull | static_cast<uint64_t>(deg[i]));
  if (mode != 2) h = (h ^ (h >> 32)) & 0xffffffffull;
  hash[i] = h;
  idx[i] = static_cast<int32_t>(i);
}

// rows of degree >= 64 (degree-sorted positions [0, n_mid)): a warp per row,
// four independent column loads per lane in flight
__global__ void k_row_hash_wide(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const int32_t* __restrict__ deg, const int32_t* __restrict__ p_compact,
                                int64_t n_mid, int mode, const int32_t* __restrict__ nleaf,
                                const int32_t* __restrict__ leaf_of, uint64_t* __restrict__ hash,
                                int32_t* __restrict__ idx) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t k = w0; k < n_mid; k += nw) {
    const int64_t i = p_compact[k];
    if (mode == 2 && !pendant_eligible(deg, nleaf, i)) {  // warp-uniform
      if (lane == 0) {
        hash[i] = 0x8000000000000000ull | static_cast<uint64_t>(i);
        idx[i] = static_cast<int32_t>(i);
      }
      continue;
    }
    const int32_t skip = mode == 2 ? leaf_of[i] : -1;
    const int64_t e1 = row_ptr[i + 1];
    uint64_t h = 0;
    for (int64_t e0 = row_ptr[i] + lane; e0 < e1; e0 += 128) {
      int32_t c[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) c[u] = e0 + 32 * u < e1 ? col[e0 + 32 * u] : -1;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (c[u] >= 0 && c[u] != skip) h += mix_id(static_cast<uint64_t>(c[u]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if (lane == 0) row_hash_store(mode, i, h, deg, hash, idx);
  }
}

// rows of degree < kMediumDeg = 64 (positions [n_mid, n)): eight lanes per
// row, four rows per warp, each lane loading its (at most eight) columns at once
__global__ void k_row_hash_narrow(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                  const int32_t* __restrict__ deg, const int32_t* __restrict__ p_compact,
                                  int64_t n_mid, int64_t n, int mode, const int32_t* __restrict__ nleaf,
                                  const int32_t* __restrict__ leaf_of, uint64_t* __restrict__ hash,
                                  int32_t* __restrict__ idx) {
  const int lane = threadIdx.x & 31, sub = lane >> 3, sl = lane & 7;
  const int64_t w0 = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t k0 = n_mid + 4 * w0; k0 < n; k0 += 4 * nw) {  // warp-uniform bound
    const int64_t k = k0 + sub;
    const bool act = k < n;
    const int64_t i = act ? p_compact[k] : 0;
    const bool elig = act && (mode != 2 || pendant_eligible(deg, nleaf, i));
    uint64_t h = 0;
    if (elig) {
      const int32_t skip = mode == 2 ? leaf_of[i] : -1;
      const int64_t e0 = row_ptr[i] + sl, e1 = row_ptr[i + 1];
      static_assert(kMediumDeg <= 64, "eight lanes x eight loads cover a light row");
      int32_t c[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) c[u] = e0 + 8 * u < e1 ? col[e0 + 8 * u] : -1;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (c[u] >= 0 && c[u] != skip) h += mix_id(static_cast<uint64_t>(c[u]));
    }
    h += __shfl_xor_sync(0xffffffffu, h, 4);
    h += __shfl_xor_sync(0xffffffffu, h, 2);
    h += __shfl_xor_sync(0xffffffffu, h, 1);
    if (act && sl == 0) {
      if (elig) {
        row_hash_store(mode, i, h, deg, hash, idx);
      } else {
        hash[i] = 0x8000000000000000ull | static_cast<uint64_t>(i);
        idx[i] = static_cast<int32_t>(i);
      }
    }
  }
}

// after sorting: class_id = own id for nodes alone in their hash run, -1 for
// members of longer runs; record the start of each longer run
__global__ void k_mark_runs(const uint64_t* __restrict__ h, const int32_t* __restrict__ node, int64_t n,
                            int32_t* __restrict__ class_id, int64_t* __restrict__ run_start,
                            unsigned long long* __restrict__ n_runs) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const bool same_prev = k > 0 && h[k - 1] == h[k];
    const bool same_next = k + 1 < n && h[k + 1] == h[k];
    class_id[node[k]] = (same_prev || same_next) ? -1 : node[k];
    if (!same_prev && same_next) run_start[atomicAdd(n_runs, 1ull)] = k;
  }
}

__device__ __forceinline__ bool same_list(const int64_t* row_ptr, const int32_t* col, int32_t a, int32_t b) {
  const int64_t ba = row_ptr[a], bb = row_ptr[b];
  const int64_t la = row_ptr[a + 1] - ba;
  if (la != row_ptr[b + 1] - bb) return false;
  for (int64_t e = 0; e < la; ++e)
    if (col[ba + e] != col[bb + e]) return false;
  return true;
}

// N[a] = N[b] for a != b: a ~ b and N(a) - {b} = N(b) - {a} (sorted lists)
__device__ __forceinline__ bool same_closed_list(const int64_t* row_ptr, const int32_t* col, int32_t a, int32_t b) {
  const int64_t ba = row_ptr[a], bb = row_ptr[b];
  const int64_t la = row_ptr[a + 1] - ba, lb = row_ptr[b + 1] - bb;
  if (la != lb) return false;
  bool adjacent = false;
  int64_t i = 0, j = 0;
  while (i < la || j < lb) {
    if (i < la && col[ba + i] == b) {
      adjacent = true;
      ++i;
      continue;
    }
    if (j < lb && col[bb + j] == a) {
      ++j;
      continue;
    }
    if (i >= la || j >= lb || col[ba + i] != col[bb + j]) return false;
    ++i;
    ++j;
  }
  return adjacent;
}

// pendant twins: both eligible, N(a) - {leaf a} = N(b) - {leaf b}
__device__ __forceinline__ bool same_reduced_list(const int64_t* row_ptr, const int32_t* col, const int32_t* deg,
                                                  const int32_t* nleaf, const int32_t* leaf_of, int32_t a, int32_t b) {
  if (!pendant_eligible(deg, nleaf, a) || !pendant_eligible(deg, nleaf, b)) return false;
  const int64_t ba = row_ptr[a], bb = row_ptr[b];
  const int64_t la = row_ptr[a + 1] - ba, lb = row_ptr[b + 1] - bb;
  if (la != lb) return false;
  const int32_t sa = leaf_of[a], sb = leaf_of[b];
  int64_t i = 0, j = 0;
  while (i < la || j < lb) {
    if (i < la && col[ba + i] == sa) {
      ++i;
      continue;
    }
    if (j < lb && col[bb + j] == sb) {
      ++j;
      continue;
    }
    if (i >= la || j >= lb || col[ba + i] != col[bb + j]) return false;
    ++i;
    ++j;
  }
  return true;
}

// warp per run: repeated leader election in id order; every unassigned member
// equal to the leader joins its class
__global__ void k_resolve_runs(const uint64_t* __restrict__ h, const int32_t* __restrict__ node, int64_t n,
                               const int64_t* __restrict__ run_start, int64_t n_runs,
                               const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ deg, int mode, const int32_t* __restrict__ nleaf,
                               const int32_t* __restrict__ leaf_of, int32_t* class_id) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = w0; r < n_runs; r += nw) {
    const int64_t a = run_start[r];
    int64_t b = a + 1;
    while (b < n && h[b] == h[a]) ++b;
    for (int64_t lead = a; lead < b; ++lead) {
      const int32_t ln = node[lead];
      __syncwarp();
      if (*reinterpret_cast<volatile int32_t*>(class_id + ln) != -1) continue;  // warp-uniform
      if (lane == 0) class_id[ln] = ln;
      for (int64_t k = lead + 1 + lane; k < b; k += 32) {
        const int32_t m = node[k];
        if (*reinterpret_cast<volatile int32_t*>(class_id + m) != -1) continue;
        const bool same = mode == 0   ? same_list(row_ptr, col, ln, m)
                          : mode == 1 ? same_closed_list(row_ptr, col, ln, m)
                                      : same_reduced_list(row_ptr, col, deg, nleaf, leaf_of, ln, m);
        if (same) class_id[m] = ln;
      }
      __syncwarp();
    }
  }
}

__global__ void k_iota(int32_t* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    x[i] = static_cast<int32_t>(i);
}

// class sizes of one relation
__global__ void k_sizes(const int32_t* __restrict__ cid, int64_t n, int32_t* __restrict__ size) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    atomicAdd(&size[cid[i]], 1);
}

// merge the closed classes into the open ones (disjoint relations) and count
// the removed closed-twin eigenvalues -1/d per degree d
__global__ void k_merge_closed(int32_t* __restrict__ class_id, const int32_t* __restrict__ open_size,
                               const int32_t* __restrict__ closed_id, const int32_t* __restrict__ closed_size,
                               const int32_t* __restrict__ deg, int64_t n, unsigned long long* __restrict__ per_deg,
                               int* __restrict__ conflict) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t c = closed_id[i];
    if (closed_size[c] < 2) continue;
    if (open_size[class_id[i]] >= 2) atomicOr(conflict, 1);  // cannot happen (disjoint relations)
    class_id[i] = c;
    if (c != i) atomicAdd(&per_deg[deg[i]], 1ull);
  }
}

// leaves per node, and one leaf of each node (meaningful where the count is 1)
__global__ void k_leaf_info(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ deg, int64_t n, int32_t* __restrict__ nleaf,
                            int32_t* __restrict__ leaf_of) {
  for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < n;
       x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (deg[x] != 1) continue;
    const int32_t a = col[row_ptr[x]];
    atomicAdd(&nleaf[a], 1);
    leaf_of[a] = static_cast<int32_t>(x);
  }
}

// smallest leaf of each pendant-twin class (classes of size >= 2)
__global__ void k_leaf_min(const int32_t* __restrict__ pid, const int32_t* __restrict__ psize,
                           const int32_t* __restrict__ leaf_of, int64_t n, int32_t* __restrict__ leaf_min) {
  for (int64_t a = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; a < n;
       a += static_cast<int64_t>(gridDim.x) * blockDim.x)
    if (psize[pid[a]] >= 2) atomicMin(&leaf_min[pid[a]], leaf_of[a]);
}

// merge the pendant-twin classes (nodes, and their leaves as a second class)
// and count the removed pairs per degree
__global__ void k_merge_pendant(int32_t* __restrict__ class_id, const int32_t* __restrict__ size,
                                const int32_t* __restrict__ pid, const int32_t* __restrict__ psize,
                                const int32_t* __restrict__ leaf_of, const int32_t* __restrict__ leaf_min,
                                const int32_t* __restrict__ deg, int64_t n, unsigned long long* __restrict__ per_deg,
                                int* __restrict__ conflict) {
  for (int64_t a = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; a < n;
       a += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t c = pid[a];
    if (psize[c] < 2) continue;
    const int32_t x = leaf_of[a];
    // cannot happen (disjoint relations): either node already in a nontrivial class
    if (size[class_id[a]] >= 2 || size[class_id[x]] >= 2) atomicOr(conflict, 1);
    class_id[a] = c;
    class_id[x] = leaf_min[c];
    if (c != a) atomicAdd(&per_deg[deg[a]], 1ull);
  }
}

// parallel-path candidates: an edge (a, b), a < b, between degree-2 nodes
// whose other neighbours e (of a) and f (of b) differ and have degree >= 3;
// key = (min(e, f) << 32) | max(e, f), first = the node next to min(e, f)
__global__ void k_pp_candidates(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const int32_t* __restrict__ deg, int64_t n, uint64_t* __restrict__ key,
                                int32_t* __restrict__ idx, int32_t* __restrict__ first, int32_t* __restrict__ second,
                                unsigned long long* __restrict__ count) {
  for (int64_t a = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; a < n;
       a += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (deg[a] != 2) continue;
    const int32_t x0 = col[row_ptr[a]], x1 = col[row_ptr[a] + 1];
    for (int side = 0; side < 2; ++side) {
      const int32_t b = side == 0 ? x0 : x1, e = side == 0 ? x1 : x0;
      if (b <= a || deg[b] != 2) continue;
      const int32_t y0 = col[row_ptr[b]], y1 = col[row_ptr[b] + 1];
      const int32_t f = y0 == static_cast<int32_t>(a) ? y1 : y0;
      if (e == f || deg[e] < 3 || deg[f] < 3) continue;
      const unsigned long long k = atomicAdd(count, 1ull);
      const uint32_t lo = static_cast<uint32_t>(e < f ? e : f), hi = static_cast<uint32_t>(e < f ? f : e);
      key[k] = (static_cast<uint64_t>(lo) << 32) | hi;
      idx[k] = static_cast<int32_t>(k);
      first[k] = e < f ? static_cast<int32_t>(a) : b;
      second[k] = e < f ? b : static_cast<int32_t>(a);
    }
  }
}

// a thread per run of equal keys (sorted): c >= 2 paths form two classes
// (smallest members), c - 1 removed pairs
__global__ void k_pp_assign(const uint64_t* __restrict__ key, const int32_t* __restrict__ order, int64_t m,
                            const int32_t* __restrict__ first, const int32_t* __restrict__ second,
                            const int32_t* __restrict__ size, int32_t* __restrict__ class_id,
                            unsigned long long* __restrict__ pairs, int* __restrict__ conflict) {
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < m;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (p > 0 && key[p - 1] == key[p]) continue;  // not a run start
    int64_t q = p + 1;
    int32_t f1 = first[order[p]], f2 = second[order[p]];
    while (q < m && key[q] == key[p]) {
      f1 = min(f1, first[order[q]]);
      f2 = min(f2, second[order[q]]);
      ++q;
    }
    if (q - p < 2) continue;
    for (int64_t r = p; r < q; ++r) {
      const int32_t a = first[order[r]], b = second[order[r]];
      // cannot happen (disjoint relations): either node already in a nontrivial class
      if (size[class_id[a]] >= 2 || size[class_id[b]] >= 2) atomicOr(conflict, 1);
      class_id[a] = f1;
      class_id[b] = f2;
    }
    atomicAdd(pairs, static_cast<unsigned long long>(q - p - 1));
  }
}

__global__ void k_class_counts(const int32_t* __restrict__ class_id, int64_t n, int32_t* __restrict__ cnt,
                               unsigned long long* __restrict__ removed) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t c = class_id[i];
    atomicAdd(&cnt[c], 1);
    if (c != i) atomicAdd(removed, 1ull);
  }
}

__global__ void k_leader_flags(const int32_t* __restrict__ cnt, int64_t n, int32_t* __restrict__ flag) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    flag[i] = cnt[i] >= 2 ? 1 : 0;
}

// slot of each position's class (degree-sorted order) and class sizes
__global__ void k_slots(const int32_t* __restrict__ class_id, const int32_t* __restrict__ cnt,
                        const int32_t* __restrict__ slot_of_leader, const int32_t* __restrict__ p_compact, int64_t n,
                        int32_t* __restrict__ p_slot, int32_t* __restrict__ slot_size) {
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t c = class_id[p_compact[p]];
    const int32_t sz = cnt[c];
    if (sz >= 2) {
      const int32_t sl = slot_of_leader[c];
      p_slot[p] = sl;
      slot_size[sl] = sz;
    } else {
      p_slot[p] = -1;
    }
  }
}

inline unsigned grid_for(int64_t work, int per_block = 256) {
  int64_t b = (work + per_block - 1) / per_block;
  const int64_t cap = static_cast<int64_t>(num_sms()) * 32;
  if (b > cap) b = cap;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}


}  // namespace

// Classes of one relation (mode 0 open twins, 1 closed twins, 2 pendant
// twins, which need nleaf / leaf_of) into cid[n]: the smallest member of each
// node's class, its own id if it has no twin.
static int find_classes(const Graph* G, int mode, int32_t* cid, Temps& t, const int32_t* nleaf = nullptr,
                        const int32_t* leaf_of = nullptr) {
  const int64_t n = G->n;
  cudaStream_t s = t.s;
  uint64_t *h = nullptr, *h_alt = nullptr;
  int32_t *idx = nullptr, *idx_alt = nullptr;
  int64_t* run_start = nullptr;
  unsigned long long* n_runs_d = nullptr;
  NDOS_CHECK(t.get(&h, n));
  NDOS_CHECK(t.get(&h_alt, n));
  NDOS_CHECK(t.get(&idx, n));
  NDOS_CHECK(t.get(&idx_alt, n));
  NDOS_CHECK(t.get(&run_start, n));
  NDOS_CHECK(t.get(&n_runs_d, 1));
  NDOS_CUDA(cudaMemsetAsync(n_runs_d, 0, sizeof(unsigned long long), s));
  if (G->n_mid > 0) {
    k_row_hash_wide<<<grid_for(G->n_mid * 32), 256, 0, s>>>(G->row_ptr, G->col, G->deg, G->p_compact, G->n_mid,
                                                            mode, nleaf, leaf_of, h, idx);
    NDOS_LAUNCHED();
  }
  if (n > G->n_mid) {
    k_row_hash_narrow<<<grid_for((n - G->n_mid) * 8), 256, 0, s>>>(G->row_ptr, G->col, G->deg, G->p_compact,
                                                                   G->n_mid, n, mode, nleaf, leaf_of, h, idx);
    NDOS_LAUNCHED();
  }
  cub::DoubleBuffer<uint64_t> kb(h, h_alt);
  cub::DoubleBuffer<int32_t> vb(idx, idx_alt);
  const int key_bits = mode == 2 ? 64 : 32;
  size_t bytes = 0;
  NDOS_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, kb, vb, n, 0, key_bits, s));
  char* tmp = nullptr;
  NDOS_CHECK(t.get(&tmp, bytes));
  NDOS_CUDA(cub::DeviceRadixSort::SortPairs(tmp, bytes, kb, vb, n, 0, key_bits, s));
  count_launch();
  k_mark_runs<<<grid_for(n), 256, 0, s>>>(kb.Current(), vb.Current(), n, cid, run_start, n_runs_d);
  NDOS_LAUNCHED();
  unsigned long long n_runs = 0;
  NDOS_CUDA(cudaMemcpyAsync(&n_runs, n_runs_d, sizeof(n_runs), cudaMemcpyDeviceToHost, s));
  NDOS_CUDA(cudaStreamSynchronize(s));
  if (n_runs > 0) {
    k_resolve_runs<<<grid_for(static_cast<int64_t>(n_runs) * 32), 256, 0, s>>>(
        kb.Current(), vb.Current(), n, run_start, static_cast<int64_t>(n_runs), G->row_ptr, G->col, G->deg, mode, nleaf,
        leaf_of, cid);
    NDOS_LAUNCHED();
  }
  return DOS_OK;
}

static int motif_filter_impl(const Graph* G, uint32_t motifs, cudaStream_t s, Filter* F) {
  const int64_t n = G->n;
  Temps t(s);
  // the filter's own buffers come from the stream-ordered pool (a filter per
  // query would otherwise pay a cudaMalloc each time); dos_filter_destroy
  // synchronises the device before it returns them
  auto palloc = [s](int32_t** p, int64_t count) -> int {
    if (alloc_fault_injected()) return fail(DOS_ENOMEM, "injected allocation failure (dos_test_fail_alloc)");
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(p), sizeof(int32_t) * (count > 0 ? count : 1), s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "cudaMallocAsync", __FILE__, __LINE__);
    }
    return DOS_OK;
  };
  NDOS_CHECK(palloc(&F->class_id, n));
  NDOS_CHECK(palloc(&F->p_slot, n));
  if (n == 0) {
    NDOS_CHECK(palloc(&F->slot_size, 1));
    return DOS_OK;
  }
  int32_t *cnt = nullptr, *flag = nullptr, *slot_of = nullptr;
  unsigned long long* removed_d = nullptr;
  NDOS_CHECK(t.get(&cnt, n));
  NDOS_CHECK(t.get(&flag, n + 1));
  NDOS_CHECK(t.get(&slot_of, n + 1));
  NDOS_CHECK(t.get(&removed_d, 1));
  NDOS_CUDA(cudaMemsetAsync(removed_d, 0, sizeof(unsigned long long), s));
  NDOS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n, s));

  if (motifs & DOS_MOTIF_OPEN_TWINS) {
    NDOS_CHECK(find_classes(G, 0, F->class_id, t));
  } else {
    k_iota<<<grid_for(n), 256, 0, s>>>(F->class_id, n);
    NDOS_LAUNCHED();
  }
  int64_t removed_closed = 0;
  if (motifs & DOS_MOTIF_CLOSED_TWINS) {
    int32_t *closed_id = nullptr, *open_size = nullptr, *closed_size = nullptr;
    unsigned long long* per_deg = nullptr;
    int* conflict = nullptr;
    NDOS_CHECK(t.get(&closed_id, n));
    NDOS_CHECK(t.get(&open_size, n));
    NDOS_CHECK(t.get(&closed_size, n));
    NDOS_CHECK(t.get(&per_deg, n + 1));
    NDOS_CHECK(t.get(&conflict, 1));
    NDOS_CHECK(find_classes(G, 1, closed_id, t));
    NDOS_CUDA(cudaMemsetAsync(open_size, 0, sizeof(int32_t) * n, s));
    NDOS_CUDA(cudaMemsetAsync(closed_size, 0, sizeof(int32_t) * n, s));
    NDOS_CUDA(cudaMemsetAsync(per_deg, 0, sizeof(unsigned long long) * (n + 1), s));
    NDOS_CUDA(cudaMemsetAsync(conflict, 0, sizeof(int), s));
    k_sizes<<<grid_for(n), 256, 0, s>>>(F->class_id, n, open_size);
    NDOS_LAUNCHED();
    k_sizes<<<grid_for(n), 256, 0, s>>>(closed_id, n, closed_size);
    NDOS_LAUNCHED();
    k_merge_closed<<<grid_for(n), 256, 0, s>>>(F->class_id, open_size, closed_id, closed_size, G->deg, n, per_deg,
                                               conflict);
    NDOS_LAUNCHED();
    std::vector<unsigned long long> h_deg(static_cast<size_t>(n + 1));
    int h_conflict = 0;
    NDOS_CUDA(cudaMemcpyAsync(h_deg.data(), per_deg, sizeof(unsigned long long) * (n + 1), cudaMemcpyDeviceToHost, s));
    NDOS_CUDA(cudaMemcpyAsync(&h_conflict, conflict, sizeof(int), cudaMemcpyDeviceToHost, s));
    NDOS_CUDA(cudaStreamSynchronize(s));
    if (h_conflict) return fail(DOS_ECUDA, "dos_motif_filter: a node in both an open and a closed twin class");
    // one spike -1/d per degree d that has closed twins
    for (int64_t d = 1; d <= n; ++d)
      if (h_deg[d]) {
        F->spikes.push_back({-1.0 / static_cast<double>(d), static_cast<int64_t>(h_deg[d])});
        removed_closed += static_cast<int64_t>(h_deg[d]);
      }
  }
  int64_t removed_paths = 0;
  if (motifs & DOS_MOTIF_PENDANT_TWINS) {
    int32_t *nleaf = nullptr, *leaf_of = nullptr, *pid = nullptr, *psize = nullptr, *size = nullptr,
            *leaf_min = nullptr;
    unsigned long long* per_deg = nullptr;
    int* conflict = nullptr;
    NDOS_CHECK(t.get(&nleaf, n));
    NDOS_CHECK(t.get(&leaf_of, n));
    NDOS_CHECK(t.get(&pid, n));
    NDOS_CHECK(t.get(&psize, n));
    NDOS_CHECK(t.get(&size, n));
    NDOS_CHECK(t.get(&leaf_min, n));
    NDOS_CHECK(t.get(&per_deg, n + 1));
    NDOS_CHECK(t.get(&conflict, 1));
    NDOS_CUDA(cudaMemsetAsync(nleaf, 0, sizeof(int32_t) * n, s));
    NDOS_CUDA(cudaMemsetAsync(leaf_of, 0, sizeof(int32_t) * n, s));
    NDOS_CUDA(cudaMemsetAsync(psize, 0, sizeof(int32_t) * n, s));
    NDOS_CUDA(cudaMemsetAsync(size, 0, sizeof(int32_t) * n, s));
    NDOS_CUDA(cudaMemsetAsync(leaf_min, 0x7f, sizeof(int32_t) * n, s));  // 0x7f7f7f7f > any id
    NDOS_CUDA(cudaMemsetAsync(per_deg, 0, sizeof(unsigned long long) * (n + 1), s));
    NDOS_CUDA(cudaMemsetAsync(conflict, 0, sizeof(int), s));
    k_leaf_info<<<grid_for(n), 256, 0, s>>>(G->row_ptr, G->col, G->deg, n, nleaf, leaf_of);
    NDOS_LAUNCHED();
    NDOS_CHECK(find_classes(G, 2, pid, t, nleaf, leaf_of));
    k_sizes<<<grid_for(n), 256, 0, s>>>(pid, n, psize);
    NDOS_LAUNCHED();
    k_sizes<<<grid_for(n), 256, 0, s>>>(F->class_id, n, size);
    NDOS_LAUNCHED();
    k_leaf_min<<<grid_for(n), 256, 0, s>>>(pid, psize, leaf_of, n, leaf_min);
    NDOS_LAUNCHED();
    k_merge_pendant<<<grid_for(n), 256, 0, s>>>(F->class_id, size, pid, psize, leaf_of, leaf_min, G->deg, n, per_deg,
                                                conflict);
    NDOS_LAUNCHED();
    std::vector<unsigned long long> h_deg(static_cast<size_t>(n + 1));
    int h_conflict = 0;
    NDOS_CUDA(cudaMemcpyAsync(h_deg.data(), per_deg, sizeof(unsigned long long) * (n + 1), cudaMemcpyDeviceToHost, s));
    NDOS_CUDA(cudaMemcpyAsync(&h_conflict, conflict, sizeof(int), cudaMemcpyDeviceToHost, s));
    NDOS_CUDA(cudaStreamSynchronize(s));
    if (h_conflict) return fail(DOS_ECUDA, "dos_motif_filter: a pendant-twin node already in a twin class");
    for (int64_t d = 2; d <= n; ++d)
      if (h_deg[d]) {
        const double r = 1.0 / std::sqrt(static_cast<double>(d));
        F->spikes.push_back({-r, static_cast<int64_t>(h_deg[d])});
        F->spikes.push_back({r, static_cast<int64_t>(h_deg[d])});
        removed_paths += 2 * static_cast<int64_t>(h_deg[d]);
      }
  }
  int64_t removed_pp = 0;
  if (motifs & DOS_MOTIF_PARALLEL_PATHS) {
    uint64_t *key = nullptr, *key_alt = nullptr;
    int32_t *idx = nullptr, *idx_alt = nullptr, *first = nullptr, *second = nullptr, *size = nullptr;
    unsigned long long *count = nullptr, *pairs_d = nullptr;
    int* conflict = nullptr;
    NDOS_CHECK(t.get(&key, n));
    NDOS_CHECK(t.get(&key_alt, n));
    NDOS_CHECK(t.get(&idx, n));
    NDOS_CHECK(t.get(&idx_alt, n));
    NDOS_CHECK(t.get(&first, n));
    NDOS_CHECK(t.get(&second, n));
    NDOS_CHECK(t.get(&size, n));
    NDOS_CHECK(t.get(&count, 1));
    NDOS_CHECK(t.get(&pairs_d, 1));
    NDOS_CHECK(t.get(&conflict, 1));
    NDOS_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned long long), s));
    NDOS_CUDA(cudaMemsetAsync(pairs_d, 0, sizeof(unsigned long long), s));
    NDOS_CUDA(cudaMemsetAsync(conflict, 0, sizeof(int), s));
    NDOS_CUDA(cudaMemsetAsync(size, 0, sizeof(int32_t) * n, s));
    k_pp_candidates<<<grid_for(n), 256, 0, s>>>(G->row_ptr, G->col, G->deg, n, key, idx, first, second, count);
    NDOS_LAUNCHED();
    k_sizes<<<grid_for(n), 256, 0, s>>>(F->class_id, n, size);
    NDOS_LAUNCHED();
    unsigned long long m = 0;
    NDOS_CUDA(cudaMemcpyAsync(&m, count, sizeof(m), cudaMemcpyDeviceToHost, s));
    NDOS_CUDA(cudaStreamSynchronize(s));
    if (m > 0) {
      cub::DoubleBuffer<uint64_t> kb(key, key_alt);
      cub::DoubleBuffer<int32_t> vb(idx, idx_alt);
      size_t bytes = 0;
      NDOS_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, kb, vb, static_cast<int64_t>(m), 0, 64, s));
      char* tmp = nullptr;
      NDOS_CHECK(t.get(&tmp, bytes));
      NDOS_CUDA(cub::DeviceRadixSort::SortPairs(tmp, bytes, kb, vb, static_cast<int64_t>(m), 0, 64, s));
      count_launch();
      k_pp_assign<<<grid_for(static_cast<int64_t>(m)), 256, 0, s>>>(kb.Current(), vb.Current(), static_cast<int64_t>(m),
                                                                   first, second, size, F->class_id, pairs_d, conflict);
      NDOS_LAUNCHED();
    }
    unsigned long long pairs = 0;
    int h_conflict = 0;
    NDOS_CUDA(cudaMemcpyAsync(&pairs, pairs_d, sizeof(pairs), cudaMemcpyDeviceToHost, s));
    NDOS_CUDA(cudaMemcpyAsync(&h_conflict, conflict, sizeof(int), cudaMemcpyDeviceToHost, s));
    NDOS_CUDA(cudaStreamSynchronize(s));
    if (h_conflict) return fail(DOS_ECUDA, "dos_motif_filter: a parallel-path node already in another class");
    if (pairs) {
      F->spikes.push_back({-0.5, static_cast<int64_t>(pairs)});
      F->spikes.push_back({0.5, static_cast<int64_t>(pairs)});
    }
    removed_pp = 2 * static_cast<int64_t>(pairs);
  }
  k_class_counts<<<grid_for(n), 256, 0, s>>>(F->class_id, n, cnt, removed_d);
  NDOS_LAUNCHED();
  k_leader_flags<<<grid_for(n), 256, 0, s>>>(cnt, n, flag);
  NDOS_LAUNCHED();
  NDOS_CUDA(cudaMemsetAsync(flag + n, 0, sizeof(int32_t), s));
  size_t bytes = 0;
  NDOS_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, flag, slot_of, n + 1, s));
  char* tmp2 = nullptr;
  NDOS_CHECK(t.get(&tmp2, bytes));
  NDOS_CUDA(cub::DeviceScan::ExclusiveSum(tmp2, bytes, flag, slot_of, n + 1, s));
  count_launch();
  int32_t n_classes = 0;
  unsigned long long removed = 0;
  NDOS_CUDA(cudaMemcpyAsync(&n_classes, slot_of + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  NDOS_CUDA(cudaMemcpyAsync(&removed, removed_d, sizeof(removed), cudaMemcpyDeviceToHost, s));
  NDOS_CUDA(cudaStreamSynchronize(s));
  F->n_classes = n_classes;
  F->removed = static_cast<int64_t>(removed);
  const int64_t removed_open = F->removed - removed_closed - removed_paths - removed_pp;
  if (removed_open > 0) F->spikes.push_back({0.0, removed_open});
  std::sort(F->spikes.begin(), F->spikes.end(),
            [](const std::pair<double, int64_t>& x, const std::pair<double, int64_t>& y) { return x.first < y.first; });
  // equal eigenvalues of different motifs (e.g. -1/2) are one spike
  std::vector<std::pair<double, int64_t>> merged;
  for (const auto& sp : F->spikes) {
    if (!merged.empty() && merged.back().first == sp.first)
      merged.back().second += sp.second;
    else
      merged.push_back(sp);
  }
  F->spikes.swap(merged);
  NDOS_CHECK(palloc(&F->slot_size, n_classes));
  k_slots<<<grid_for(n), 256, 0, s>>>(F->class_id, cnt, slot_of, G->p_compact, n, F->p_slot, F->slot_size);
  NDOS_LAUNCHED();
  NDOS_CUDA(cudaStreamSynchronize(s));
  return DOS_OK;
}

}  // namespace netdos

using namespace netdos;

extern "C" int dos_motif_filter_ex(dos_graph_t g, uint32_t motifs, void* stream, dos_filter_t* out) {
  clear_error();
  if (!out) return fail(DOS_EINVAL, "dos_motif_filter: out is NULL");
  *out = nullptr;
  if (!g) return fail(DOS_EINVAL, "dos_motif_filter: null graph");
  const uint32_t known =
      DOS_MOTIF_OPEN_TWINS | DOS_MOTIF_CLOSED_TWINS | DOS_MOTIF_PENDANT_TWINS | DOS_MOTIF_PARALLEL_PATHS;
  if (motifs == 0 || (motifs & ~known)) return fail(DOS_EINVAL, "dos_motif_filter_ex: unknown or empty motif set");
  Filter* F = new Filter();
  F->g = reinterpret_cast<const Graph*>(g);
  int st = motif_filter_impl(F->g, motifs, static_cast<cudaStream_t>(stream), F);
  if (st != DOS_OK) {
    dos_filter_destroy(reinterpret_cast<dos_filter_t>(F));
    return st;
  }
  *out = reinterpret_cast<dos_filter_t>(F);
  return DOS_OK;
}

extern "C" int dos_motif_filter(dos_graph_t g, void* stream, dos_filter_t* out) {
  return dos_motif_filter_ex(g, DOS_MOTIF_OPEN_TWINS, stream, out);
}

extern "C" int dos_filter_spikes(dos_filter_t f, double* spikes, int capacity, int* n_spikes) {
  clear_error();
  if (!f) return fail(DOS_EINVAL, "dos_filter_spikes: null filter");
  if (capacity < 0 || (capacity > 0 && !spikes)) return fail(DOS_EINVAL, "dos_filter_spikes: bad buffer");
  const Filter* F = reinterpret_cast<const Filter*>(f);
  const int total = static_cast<int>(F->spikes.size());
  if (n_spikes) *n_spikes = total;
  for (int k = 0; k < total && k < capacity; ++k) {
    spikes[2 * k] = F->spikes[k].first;
    spikes[2 * k + 1] = static_cast<double>(F->spikes[k].second);
  }
  return DOS_OK;
}
