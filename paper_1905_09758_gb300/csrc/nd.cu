// Nested dissection for the PDOS (§3.3, Algorithm 1): the exact diagonal
// moments C[m][i] = T_m(H)_ii of every node, without probes, for graphs with
// small vertex separators.
//
// Partition tree (host).  A partition P with more than `leaf` nodes is split by
// a vertex separator S into two parts A, B with no edge between them; the
// recursion gives a tree whose node t holds its rows I_p = P and its columns
// I_s = S (a leaf holds I_s = I_p = P).  Separators are BFS level sets: a BFS
// on the subgraph induced by P from a far node (the last node of a first
// BFS) gives levels 0..L, and the level nearest the median by count splits
// the levels below it from the levels above it (edges only join equal or
// adjacent levels).  A disconnected P is split into one component and the
// rest with an empty separator; a P whose BFS has fewer than three levels
// becomes a leaf.  So every node of P is adjacent only to nodes of P and of
// the separators of t's ancestors, and every node is a column of exactly
// one tree node ("home").
//
// Recurrence (GPU).  With X_t^m = T_m(H)(I_p, I_s) for every tree node t,
//   X_t^{m+1} = 2 H(I_p, :) T_m(H)(:, I_s) - X_t^{m-1},
// where row i of H(I_p, :) reaches rows k of I_p (taken from X_t^m) and rows k
// of an ancestor's separator S_{t'} (T_m(H)(k, j) = T_m(H)(j, k) is entry
// (j, k) of X_{t'}^m, j in I_p(t')).  Every block needs only step-m values, so
// all blocks advance in parallel; the diagonal entry of node i is written
// where i is its home's column.  FP32 values, FP32 sums.
#include <algorithm>
#include <climits>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace netdos {
namespace {

struct NdTree {
  std::vector<int32_t> depth;     // per tree node
  std::vector<int64_t> row_off;   // [T+1] into rows
  std::vector<int64_t> col_off;   // [T+1] into cols
  std::vector<int32_t> rows, cols;
  int max_depth = 0;
};

// host partitioner: recursive BFS-level bisection (see the file comment)
void nd_partition(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci, int leaf, NdTree& tr) {
  struct Task {
    std::vector<int32_t> nodes;
    int depth;
  };
  std::vector<int32_t> stamp(static_cast<size_t>(n), -1), level(static_cast<size_t>(n), -1);
  std::vector<int32_t> queue;
  queue.reserve(static_cast<size_t>(n));
  std::vector<Task> stack;
  {
    Task root;
    root.nodes.resize(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) root.nodes[static_cast<size_t>(i)] = static_cast<int32_t>(i);
    root.depth = 0;
    stack.push_back(std::move(root));
  }
  int32_t task_id = 0;
  auto bfs = [&](int32_t src, int32_t id) {  // nodes of the task stamped `id`; levels in `level`
    queue.clear();
    queue.push_back(src);
    level[static_cast<size_t>(src)] = 0;
    stamp[static_cast<size_t>(src)] = id;
    for (size_t h = 0; h < queue.size(); ++h) {
      const int32_t v = queue[h];
      for (int64_t e = rp[static_cast<size_t>(v)]; e < rp[static_cast<size_t>(v) + 1]; ++e) {
        const int32_t w = ci[static_cast<size_t>(e)];
        if (stamp[static_cast<size_t>(w)] == id - 1) {  // in the task, not yet reached
          stamp[static_cast<size_t>(w)] = id;
          level[static_cast<size_t>(w)] = level[static_cast<size_t>(v)] + 1;
          queue.push_back(w);
        }
      }
    }
  };
  auto emit = [&](const std::vector<int32_t>& rws, const std::vector<int32_t>& cls, int depth) {
    tr.depth.push_back(depth);
    tr.row_off.push_back(static_cast<int64_t>(tr.rows.size()));
    tr.col_off.push_back(static_cast<int64_t>(tr.cols.size()));
    tr.rows.insert(tr.rows.end(), rws.begin(), rws.end());
    tr.cols.insert(tr.cols.end(), cls.begin(), cls.end());
    tr.max_depth = std::max(tr.max_depth, depth);
  };
  while (!stack.empty()) {
    Task tk = std::move(stack.back());
    stack.pop_back();
    std::vector<int32_t>& P = tk.nodes;
    if (static_cast<int64_t>(P.size()) <= leaf) {
      emit(P, P, tk.depth);
      continue;
    }
    // two fresh stamps per BFS: members carry id - 1, reached nodes id
    task_id += 2;
    for (int32_t v : P) stamp[static_cast<size_t>(v)] = task_id - 1;
    bfs(P[0], task_id);
    if (queue.size() < P.size()) {  // disconnected: one component and the rest, empty separator
      std::vector<int32_t> comp(queue.begin(), queue.end()), rest;
      std::sort(comp.begin(), comp.end());
      for (int32_t v : P)
        if (stamp[static_cast<size_t>(v)] != task_id) rest.push_back(v);
      emit(P, {}, tk.depth);
      stack.push_back({std::move(comp), tk.depth + 1});
      stack.push_back({std::move(rest), tk.depth + 1});
      continue;
    }
    const int32_t far = queue.back();
    task_id += 2;
    for (int32_t v : P) stamp[static_cast<size_t>(v)] = task_id - 1;
    bfs(far, task_id);
    const int levels = level[static_cast<size_t>(queue.back())] + 1;
    if (levels < 3) {
      emit(P, P, tk.depth);
      continue;
    }
    std::vector<int64_t> count(static_cast<size_t>(levels), 0);
    for (int32_t v : P) ++count[static_cast<size_t>(level[static_cast<size_t>(v)])];
    // separator level in [1, levels - 2] whose lower part is nearest half of P
    int sep = 1;
    int64_t below = count[0], best = INT64_MAX;
    for (int l = 1; l <= levels - 2; ++l) {
      const int64_t diff = std::llabs(2 * below - static_cast<int64_t>(P.size()));
      if (diff < best) {
        best = diff;
        sep = l;
      }
      below += count[static_cast<size_t>(l)];
    }
    std::vector<int32_t> S, A, B;
    for (int32_t v : P) {
      const int l = level[static_cast<size_t>(v)];
      (l == sep ? S : (l < sep ? A : B)).push_back(v);
    }
    emit(P, S, tk.depth);
    stack.push_back({std::move(A), tk.depth + 1});
    stack.push_back({std::move(B), tk.depth + 1});
  }
  tr.row_off.push_back(static_cast<int64_t>(tr.rows.size()));
  tr.col_off.push_back(static_cast<int64_t>(tr.cols.size()));
}

struct NdDev {
  const int64_t* row_ptr;  // compact CSR
  const int32_t* col;
  const float* s32;        // 1/sqrt(d)
  const int32_t* item_t;   // work item q: tree node and local row
  const int32_t* item_i;
  const int32_t* rows;     // flat rows of all tree nodes
  const int32_t* cols;     // flat columns
  const int64_t* row_off;  // [T+1]
  const int64_t* col_off;  // [T+1]
  const int64_t* val_off;  // [T+1] into the value blocks (row-major p_t x s_t)
  const int32_t* depth;    // [T]
  const int32_t* anc;      // [n][D]: tree node at each depth of the node's path (-1 past it)
  const int32_t* rowidx;   // [n][D]: local row index in that tree node
  const int32_t* home;     // [n]
  const int32_t* colidx;   // [n]: local column index in the home
  int D;
  int64_t n_items;
};

// X^0: identity restricted to each block; C[0][i] = 1
__global__ void k_nd_init(NdDev d, float* __restrict__ x0, float* __restrict__ c0) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t q = w0; q < d.n_items; q += nw) {
    const int32_t t = d.item_t[q], il = d.item_i[q];
    const int32_t i = d.rows[d.row_off[t] + il];
    const int64_t s_t = d.col_off[t + 1] - d.col_off[t];
    const int64_t base = d.val_off[t] + static_cast<int64_t>(il) * s_t;
    for (int64_t cj = lane; cj < s_t; cj += 32) x0[base + cj] = d.cols[d.col_off[t] + cj] == i ? 1.f : 0.f;
    if (lane == 0 && d.home[i] == t) c0[i] = 1.f;
  }
}

// one step: x_new = (first ? 1 : 2) H x_cur - (first ? 0 : x_prev), per block;
// a warp per work item (tree node t, row i of I_p(t)), lanes over the columns
__global__ void k_nd_step(NdDev d, int first, const float* __restrict__ x_cur, const float* __restrict__ x_prev,
                          float* __restrict__ x_new, float* __restrict__ c_out) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t q = w0; q < d.n_items; q += nw) {
    const int32_t t = d.item_t[q], il = d.item_i[q];
    const int64_t s_t = d.col_off[t + 1] - d.col_off[t];
    if (s_t == 0) continue;
    const int32_t i = d.rows[d.row_off[t] + il];
    const int dt = d.depth[t];
    const int64_t base = d.val_off[t];
    const float si = d.s32[i];
    const int64_t e0 = d.row_ptr[i], e1 = d.row_ptr[i + 1];
    const bool own_home = d.home[i] == t;
    const int32_t own_col = d.colidx[i];
    for (int64_t c0 = 0; c0 < s_t; c0 += 32) {
      const int64_t cj = c0 + lane;
      const bool active = cj < s_t;
      const int32_t j = active ? d.cols[d.col_off[t] + cj] : 0;
      float acc = 0.f;
      for (int64_t e = e0; e < e1; ++e) {
        const int32_t k = d.col[e];
        const float h = si * d.s32[k];
        float v = 0.f;
        if (d.anc[static_cast<int64_t>(k) * d.D + dt] == t) {
          // k in I_p(t): entry (k, j) of this block
          if (active) v = x_cur[base + static_cast<int64_t>(d.rowidx[static_cast<int64_t>(k) * d.D + dt]) * s_t + cj];
        } else {
          // k in the separator of an ancestor t2: entry (j, k) of that block
          const int32_t t2 = d.home[k];
          const int d2 = d.depth[t2];
          const int64_t s2 = d.col_off[t2 + 1] - d.col_off[t2];
          if (active)
            v = x_cur[d.val_off[t2] + static_cast<int64_t>(d.rowidx[static_cast<int64_t>(j) * d.D + d2]) * s2 +
                      d.colidx[k]];
        }
        acc = fmaf(h, v, acc);
      }
      if (active) {
        const int64_t off = base + static_cast<int64_t>(il) * s_t + cj;
        const float out = first ? acc : fmaf(2.f, acc, -x_prev[off]);
        x_new[off] = out;
        if (own_home && cj == own_col) c_out[i] = out;
      }
    }
  }
}

}  // namespace
}  // namespace netdos

using namespace netdos;

extern "C" int dos_pdos_nd(dos_graph_t g, int M, int leaf_size, double max_entries, float* C_out, int64_t* stats,
                           void* stream) {
  clear_error();
  if (!g || !C_out) return fail(DOS_EINVAL, "dos_pdos_nd: null argument");
  const Graph* G = reinterpret_cast<const Graph*>(g);
  const int64_t n = G->n;
  if (n < 1) return fail(DOS_EINVAL, "dos_pdos_nd: graph has no edges");
  if (M < 1 || M > (1 << 20)) return fail(DOS_EINVAL, "dos_pdos_nd: M must be in [1, 2^20]");
  if (leaf_size < 1) return fail(DOS_EINVAL, "dos_pdos_nd: leaf_size must be >= 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // compact CSR to the host, partition
  std::vector<int64_t> rp(static_cast<size_t>(n + 1));
  std::vector<int32_t> ci(static_cast<size_t>(G->nnz));
  NDOS_CUDA(cudaMemcpyAsync(rp.data(), G->row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
  if (G->nnz > 0) NDOS_CUDA(cudaMemcpyAsync(ci.data(), G->col, sizeof(int32_t) * G->nnz, cudaMemcpyDeviceToHost, s));
  NDOS_CUDA(cudaStreamSynchronize(s));
  NdTree tr;
  nd_partition(n, rp, ci, leaf_size, tr);
  const int T = static_cast<int>(tr.depth.size());
  const int D = tr.max_depth + 1;
  // value offsets, work items, per-node tables
  std::vector<int64_t> val_off(static_cast<size_t>(T) + 1, 0);
  int64_t max_sep = 0;
  for (int t = 0; t < T; ++t) {
    const int64_t p = tr.row_off[t + 1] - tr.row_off[t], sc = tr.col_off[t + 1] - tr.col_off[t];
    val_off[t + 1] = val_off[t] + p * sc;
    if (sc < p) max_sep = std::max(max_sep, sc);  // a separator (leaves have I_s = I_p)
  }
  const int64_t entries = val_off[T];
  if (stats) {
    stats[0] = T;
    stats[1] = D;
    stats[2] = entries;
    stats[3] = max_sep;
  }
  if (max_entries > 0.0 && static_cast<double>(entries) > max_entries)
    return fail(DOS_ENOMEM, "dos_pdos_nd: the separators are too large for this graph (" + std::to_string(entries) +
                                " block entries > max_entries)");
  std::vector<int32_t> item_t, item_i;
  item_t.reserve(tr.rows.size());
  item_i.reserve(tr.rows.size());
  std::vector<int32_t> anc(static_cast<size_t>(n) * D, -1), rowidx(static_cast<size_t>(n) * D, -1);
  std::vector<int32_t> home(static_cast<size_t>(n), -1), colidx(static_cast<size_t>(n), -1);
  for (int t = 0; t < T; ++t) {
    const int dt = tr.depth[t];
    for (int64_t r = tr.row_off[t]; r < tr.row_off[t + 1]; ++r) {
      const int32_t v = tr.rows[static_cast<size_t>(r)];
      anc[static_cast<size_t>(v) * D + dt] = t;
      rowidx[static_cast<size_t>(v) * D + dt] = static_cast<int32_t>(r - tr.row_off[t]);
      if (tr.col_off[t + 1] > tr.col_off[t]) {
        item_t.push_back(t);
        item_i.push_back(static_cast<int32_t>(r - tr.row_off[t]));
      }
    }
    for (int64_t c = tr.col_off[t]; c < tr.col_off[t + 1]; ++c) {
      const int32_t v = tr.cols[static_cast<size_t>(c)];
      home[static_cast<size_t>(v)] = t;
      colidx[static_cast<size_t>(v)] = static_cast<int32_t>(c - tr.col_off[t]);
    }
  }
  for (int64_t v = 0; v < n; ++v)
    if (home[static_cast<size_t>(v)] < 0) return fail(DOS_ECUDA, "dos_pdos_nd: a node without a home");
  // device copies
  Temps tm(s);
  auto up = [&](auto** dptr, const auto& vec) -> int {
    using E = typename std::remove_reference<decltype(vec)>::type::value_type;
    NDOS_CHECK(tm.get(reinterpret_cast<E**>(dptr), vec.size() ? vec.size() : 1));
    if (!vec.empty())
      NDOS_CUDA(cudaMemcpyAsync(*dptr, vec.data(), sizeof(E) * vec.size(), cudaMemcpyHostToDevice, s));
    return DOS_OK;
  };
  NdDev d{};
  int32_t *d_item_t = nullptr, *d_item_i = nullptr, *d_rows = nullptr, *d_cols = nullptr, *d_depth = nullptr,
          *d_anc = nullptr, *d_rowidx = nullptr, *d_home = nullptr, *d_colidx = nullptr;
  int64_t *d_row_off = nullptr, *d_col_off = nullptr, *d_val_off = nullptr;
  NDOS_CHECK(up(&d_item_t, item_t));
  NDOS_CHECK(up(&d_item_i, item_i));
  NDOS_CHECK(up(&d_rows, tr.rows));
  NDOS_CHECK(up(&d_cols, tr.cols));
  NDOS_CHECK(up(&d_depth, tr.depth));
  NDOS_CHECK(up(&d_anc, anc));
  NDOS_CHECK(up(&d_rowidx, rowidx));
  NDOS_CHECK(up(&d_home, home));
  NDOS_CHECK(up(&d_colidx, colidx));
  NDOS_CHECK(up(&d_row_off, tr.row_off));
  NDOS_CHECK(up(&d_col_off, tr.col_off));
  NDOS_CHECK(up(&d_val_off, val_off));
  d.row_ptr = G->row_ptr;
  d.col = G->col;
  d.s32 = G->s32;
  d.item_t = d_item_t;
  d.item_i = d_item_i;
  d.rows = d_rows;
  d.cols = d_cols;
  d.row_off = d_row_off;
  d.col_off = d_col_off;
  d.val_off = d_val_off;
  d.depth = d_depth;
  d.anc = d_anc;
  d.rowidx = d_rowidx;
  d.home = d_home;
  d.colidx = d_colidx;
  d.D = D;
  d.n_items = static_cast<int64_t>(item_t.size());
  float *xa = nullptr, *xb = nullptr, *xc = nullptr;
  NDOS_CHECK(tm.get(&xa, entries > 0 ? entries : 1));
  NDOS_CHECK(tm.get(&xb, entries > 0 ? entries : 1));
  NDOS_CHECK(tm.get(&xc, entries > 0 ? entries : 1));
  const unsigned grid = static_cast<unsigned>(std::max<int64_t>(
      1, std::min<int64_t>((d.n_items * 32 + 255) / 256, static_cast<int64_t>(num_sms()) * 64)));
  k_nd_init<<<grid, 256, 0, s>>>(d, xa, C_out);
  NDOS_LAUNCHED();
  // x_cur = T_m, x_prev = T_{m-1}; the new block overwrites T_{m-1}'s buffer
  float *x_prev = xc, *x_cur = xa, *x_new = xb;
  for (int m = 1; m < M; ++m) {
    k_nd_step<<<grid, 256, 0, s>>>(d, m == 1 ? 1 : 0, x_cur, x_prev, x_new, C_out + static_cast<size_t>(m) * n);
    NDOS_LAUNCHED();
    float* tmp = x_prev;
    x_prev = x_cur;
    x_cur = x_new;
    x_new = tmp;
  }
  return DOS_OK;
}
