// Kernels of the stochastic Chebyshev recurrence (§3.1): probe-block
// initialisation, the fused Chebyshev step, and the deterministic FP64
// reduction of the per-CTA moment partials.
//
// Scaled recurrence.  With V_k = T_k(H) Z and H = S A S (S = D^{-1/2}), the
// kernels carry U_k = S V_k:
//     U_{k+1} = 2 S^2 A U_k - U_{k-1},   U_1 = S^2 A U_0,   U_0 = S Z,
// so row i of a step is (2/d_i) * sum_{j in N(i)} U_k[j] - U_{k-1}[i] and a
// nonzero costs only its int32 column index (no stored or gathered values).
// Inner products of V are recovered with the degree: <V_a, V_b> = sum_i d_i
// <U_a[i], U_b[i]>, and (V_k)_i = sqrt(d_i) (U_k)_i.
//
// Block layout ("tile-major"): a block of Nz_pad = T * t probe columns over
// n rows is stored as T tiles of n x t, row-major inside a tile:
//     element (row p, probe j) at ((j / t) * n + p) * t + (j % t).
// Work is ordered tile-major, so the rows gathered by concurrently running
// CTAs come from one tile of U_k.
//
// Rows are relabelled by degree class: heavy rows (degree >= kHeavyDeg)
// first, then medium (>= kMediumDeg), then light rows, degree-descending
// inside a class (a batch of graphs groups the medium and light rows graph by
// graph; DOS_ORDER_BY_CLASS keeps the node numbering inside a class).  Heavy
// rows get a CTA each (k_cheb_heavy), medium rows a warp each
// (k_cheb_medium); light rows go to a persistent kernel in which every warp
// takes rounds of R = 32 / Q consecutive rows, Q lanes per row, each lane one
// 16-byte chunk of the row's tile (t = Q * VEC probes), and stages the next
// round's contiguous data in shared memory with cp.async (k_cheb_light).
#pragma once

#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace netdos {

constexpr int kStepThreads = 256;
constexpr int kStepWarps = kStepThreads / 32;

// DOS: fused moment dots on H; LDOS: per-node products on H; DOS_OP /
// LDOS_OP: the same on another operator (A or D - A, shifted and scaled),
// separate instances so that the H kernels carry no operator code
enum StepMode { kModeDos = 0, kModeLdos = 1, kModeDosOp = 2, kModeLdosOp = 3 };

template <int MODE>
struct ModeOf {
  static constexpr bool op = MODE == kModeDosOp || MODE == kModeLdosOp;  // X~ on unscaled vectors
  static constexpr bool ldos = MODE == kModeLdos || MODE == kModeLdosOp;  // per-node outputs, no dots
  static constexpr bool own = MODE != kModeLdos;  // the row's own U_k (dots or the X~ diagonal term)
};

template <typename T>
struct VecT;
template <>
struct VecT<float> {
  static constexpr int N = 4;
};
template <>
struct VecT<__nv_bfloat16> {
  static constexpr int N = 8;
};
template <>
struct VecT<__half> {
  static constexpr int N = 8;
};

// ---- 16-byte chunk <-> float[VEC] --------------------------------------------
template <typename T>
__device__ __forceinline__ void unpack16(const uint4& r, float* f);
template <>
__device__ __forceinline__ void unpack16<float>(const uint4& r, float* f) {
  f[0] = __uint_as_float(r.x);
  f[1] = __uint_as_float(r.y);
  f[2] = __uint_as_float(r.z);
  f[3] = __uint_as_float(r.w);
}
template <>
__device__ __forceinline__ void unpack16<__nv_bfloat16>(const uint4& r, float* f) {
  const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(w[i] << 16);
    f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}
template <>
__device__ __forceinline__ void unpack16<__half>(const uint4& r, float* f) {
  const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __half2 h;
    memcpy(&h, &w[i], 4);
    const float2 v = __half22float2(h);
    f[2 * i] = v.x;
    f[2 * i + 1] = v.y;
  }
}

template <typename T>
__device__ __forceinline__ uint4 pack16(const float* f);
template <>
__device__ __forceinline__ uint4 pack16<float>(const float* f) {
  return make_uint4(__float_as_uint(f[0]), __float_as_uint(f[1]), __float_as_uint(f[2]), __float_as_uint(f[3]));
}
template <>
__device__ __forceinline__ uint4 pack16<__nv_bfloat16>(const float* f) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    memcpy(&w[i], &h, 4);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}
template <>
__device__ __forceinline__ uint4 pack16<__half>(const float* f) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __half2 h = __floats2half2_rn(f[2 * i], f[2 * i + 1]);
    memcpy(&w[i], &h, 4);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// ---- memory access flavours --------------------------------------------------
// gathers of U_k rows: read-only path, kept in cache
__device__ __forceinline__ uint4 ld_gather(const uint4* p) { return __ldg(p); }
// U_{k-1} rows and the own row: read once per step, evict first
__device__ __forceinline__ uint4 ld_stream(const uint4* p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(uint4* p, const uint4& v) { __stcs(p, v); }
__device__ __forceinline__ int32_t ld_col(const int32_t* p) { return __ldcs(p); }

// ---- asynchronous global -> shared copies (cp.async, inline PTX) ------------
// Each lane copies 16-byte chunks straight into shared memory without going
// through registers; a warp commits one group per work item and waits with
// cp.async.wait_group, so no load of the CSR or of the streamed rows sits on
// the critical path and no thread spins on a flag.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// copy `chunks` 16-byte chunks src -> dst, spread over the warp's lanes
__device__ __forceinline__ void warp_copy16(unsigned char* dst, const unsigned char* src, int64_t chunks, int lane) {
  for (int64_t k = lane; k < chunks; k += 32) cp_async16(dst + 16 * k, src + 16 * k);
}

// Per-thread sum of FP32 terms kept as an unevaluated pair hi + lo (Knuth's
// TwoSum error-free transformation): about 48 significant bits from FP32
// instructions, where FP64 adds would occupy GB300's narrow FP64 pipe.
struct SumFF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
  }
  __device__ __forceinline__ double value() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};
struct SumD {
  double v = 0.0;
  __device__ __forceinline__ void add(float x) { v += static_cast<double>(x); }
  __device__ __forceinline__ double value() const { return v; }
};

struct StepParams {
  const int64_t* __restrict__ row_ptr;   // [n+1] degree-sorted CSR (allocation padded to n+3)
  const int32_t* __restrict__ col;       // [nnz] neighbour positions (padded to nnz+4)
  const int32_t* __restrict__ orig;      // [n] original ids (padded to n+4)
  const int32_t* __restrict__ compact;   // [n] compact ids (padded to n+4)
  const void* u_cur;                     // U_k
  void* u_pn;                            // U_{k-1} in, U_{k+1} out (in place)
  int64_t n;
  int64_t n_heavy;  // rows [0, n_heavy): k_cheb_heavy
  int64_t n_mid;    // rows [n_heavy, n_mid): k_cheb_medium; [n_mid, n): k_cheb_light
  // batch of graphs: gid[p] = graph of row p; the row's dot contributions go
  // to gpartial[dot * n_graphs + gid] (FP64 atomics) instead of the per-CTA
  // partials.  gid == nullptr for a single graph.
  const int32_t* __restrict__ gid;
  double* gpartial;
  int64_t n_graphs;
  int tiles;
  int first;        // 1: U_1 = S^2 A U_0 (no U_{k-1} term)
  int nz;           // real probe count (columns >= nz are zero padding)
  float inv_nz;
  uint64_t seed;
  double* partial;  // this step's partials: [n_dots][part_width]
  int64_t part_width;
  int64_t mid_part_off;    // medium CTAs write partial[mid_part_off + tile * grid + blockIdx.x]
  int64_t light_part_off;  // light CTAs write partial[light_part_off + blockIdx.x]
  // operator of the kModeDosOp instances: 1 the adjacency A, 2 the Laplacian
  // D - A, shifted and scaled to (X - op_c) * op_inv_r (Eq. (5)) on unscaled
  // vectors (U = V, dot weight 1); the other modes run on H (U = S V, dot
  // weight d_i)
  int op;
  float op_c, op_inv_r;
  float* ldos;      // LDOS: this step's output row
  int64_t ldos_tile_stride;  // tile j writes ldos + j * stride (0: a single tile)
  int ldos_by_position;      // 1: rows indexed by position (scratch, coalesced), 0: by compact id (C_out)
  int* err;         // device error word
};

// Epilogue of one row: recurrence update, store, fused dots / LDOS.
// Executed by all 32 lanes of a warp (the Q-lane reductions are warp
// shuffles); `active` lanes own a row whose neighbour sum is in acc.
template <typename T, int Q, int MODE, typename ACC>
__device__ __forceinline__ void step_epilogue(const StepParams& prm, bool active, int64_t p, int ql, int tile,
                                              const float* acc, const float* prev, const float* own, float fd,
                                              uint32_t orig, int32_t compact, bool owner, ACC& dd0, ACC& dd1) {
  constexpr int V = VecT<T>::N;
  constexpr int TW = Q * V;
  using MD = ModeOf<MODE>;
  float prod0 = 0.f, prod1 = 0.f;
  if (active) {
    const size_t off = (static_cast<size_t>(tile) * prm.n + p) * TW + ql * V;
    uint4* pn = reinterpret_cast<uint4*>(reinterpret_cast<T*>(prm.u_pn) + off);
    float u[V];
    if (!MD::op) {
      const float sc = (prm.first ? 1.0f : 2.0f) / fd;
#pragma unroll
      for (int v = 0; v < V; ++v) u[v] = fmaf(acc[v], sc, -prev[v]);
    } else {
      // X~ U = ca * (A U) + co * U row-wise: A: (1/r, -c/r); D - A: (-1/r, (d_i - c)/r)
      const float mult = prm.first ? 1.0f : 2.0f;
      const float ca = (prm.op == 1 ? prm.op_inv_r : -prm.op_inv_r) * mult;
      const float co = (prm.op == 1 ? -prm.op_c : fd - prm.op_c) * prm.op_inv_r * mult;
#pragma unroll
      for (int v = 0; v < V; ++v) u[v] = fmaf(acc[v], ca, fmaf(own[v], co, -prev[v]));
    }
    const uint4 packed = pack16<T>(u);
    st_stream(pn, packed);
    unpack16<T>(packed, u);  // the dots use the stored (rounded) values
    if (!MD::ldos) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        prod0 = fmaf(u[v], u[v], prod0);
        prod1 = fmaf(u[v], own[v], prod1);
      }
    } else {
      const int j0 = tile * TW + ql * V;
      const uint64_t word = probe_word(prm.seed, orig, static_cast<uint32_t>(j0 >> 6));
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int j = j0 + v;
        if (j < prm.nz) prod0 += ((word >> (j & 63)) & 1ull) ? -u[v] : u[v];
      }
    }
  }
  // reduce over the Q lanes that share a row
#pragma unroll
  for (int s = 1; s < Q; s <<= 1) {
    prod0 += __shfl_xor_sync(0xffffffffu, prod0, s);
    if (!MD::ldos) prod1 += __shfl_xor_sync(0xffffffffu, prod1, s);
  }
  if (!MD::ldos && prm.gid) {
    // batch: per-graph sums.  Rows are grouped by graph, so a warp's rows
    // nearly always share one graph: reduce in the warp and issue one atomic
    // per dot instead of one per row (the rows of a graph all hit the same
    // two addresses).
    const int32_t g = active ? prm.gid[p] : -1;
    const int32_t g0 = __shfl_sync(0xffffffffu, g, 0);
    const bool uniform = __all_sync(0xffffffffu, !active || g == g0);
    const float wd = MD::op ? 1.0f : fd;  // <V_a, V_b> = sum_i w_i <U_a, U_b>_i
    double a0 = active && owner ? static_cast<double>(wd * prod0) : 0.0;
    double a1 = active && owner ? static_cast<double>(wd * prod1) : 0.0;
    if (uniform) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      }
      if ((threadIdx.x & 31) == 0 && g0 >= 0) {
        atomicAdd(prm.gpartial + g0, a0);
        atomicAdd(prm.gpartial + prm.n_graphs + g0, a1);
      }
    } else if (active && owner) {
      atomicAdd(prm.gpartial + g, a0);
      atomicAdd(prm.gpartial + prm.n_graphs + g, a1);
    }
    return;
  }
  if (active && owner) {
    if (!MD::ldos) {
      const float wd = MD::op ? 1.0f : fd;  // <V_a, V_b> = sum_i w_i <U_a, U_b>_i
      dd0.add(wd * prod0);
      dd1.add(wd * prod1);
    } else {
      // sum_j z_j (V_{k+1})_j of this tile (V = S^{-1} U on H, U on X~)
      const float vsum = MD::op ? prod0 : prod0 * sqrtf(fd);
      dd0.add(vsum);
      // one plain store per (tile, node); several tiles are summed afterwards
      // in a fixed order (k_ldos_fold), so the result is reproducible
      const int64_t k = prm.ldos_by_position ? p : static_cast<int64_t>(compact);
      __stcs(prm.ldos + static_cast<size_t>(tile) * prm.ldos_tile_stride + k, vsum * prm.inv_nz);  // evict first
    }
  }
}

constexpr int kGatherBatch = 8;  // independent row gathers in flight per lane

// acc += chunk `ql` of U_k rows idx[s + STRIDE*u], u = 0, 1, ..., over the
// staged indices idx[0..cnt).  Loads are issued in batches of kGatherBatch
// independent requests; the early exit is warp-uniform.
template <typename T, int Q, int STRIDE>
__device__ __forceinline__ void gather_list(const uint4* __restrict__ ubase, const int32_t* idx, int cnt, int s,
                                            int ql, float* acc) {
  constexpr int V = VecT<T>::N;
#pragma unroll 1
  for (int u0 = 0;; u0 += kGatherBatch) {
    if (!__any_sync(0xffffffffu, s + STRIDE * u0 < cnt)) break;
    uint4 r[kGatherBatch];
#pragma unroll
    for (int v = 0; v < kGatherBatch; ++v) {
      const int j = s + STRIDE * (u0 + v);
      r[v] = j < cnt ? ld_gather(ubase + static_cast<size_t>(idx[j]) * Q + ql) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int v = 0; v < kGatherBatch; ++v) {
      float a[V];
      unpack16<T>(r[v], a);
#pragma unroll
      for (int w = 0; w < V; ++w) acc[w] += a[w];
    }
  }
}

// CTA-wide deterministic sum of two doubles over NW warps; thread 0 gets it
template <int NW>
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[NW], sb[NW];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    sa[warp] = a;
    sb[warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < NW; ++w) {
      x += sa[w];
      y += sb[w];
    }
    a = x;
    b = y;
  }
}

// ---------------------------------------------------------------------------
// Heavy rows (degree >= kHeavyDeg, a prefix of the degree-sorted order): a
// CTA per row, kStepThreads / Q neighbour slots, column indices staged in
// shared memory 2048 at a time.  Grid (heavy_ctas, T).
// ---------------------------------------------------------------------------
constexpr int kHeavyColsPerThread = 8;

template <typename T, int Q, int MODE>
__global__ void __launch_bounds__(kStepThreads) k_cheb_heavy(const StepParams prm) {
  constexpr int V = VecT<T>::N;
  constexpr int TW = Q * V;
  constexpr int PH = kStepThreads / Q;
  constexpr int BLK = kStepThreads * kHeavyColsPerThread;
  __shared__ int32_t s_col[BLK];
  __shared__ float red[kStepWarps][TW];
  const int tile = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int slot = tid / Q, ql = tid % Q;
  const uint4* ubase = reinterpret_cast<const uint4*>(prm.u_cur) + static_cast<size_t>(tile) * prm.n * Q;
  SumD dd0, dd1;
  for (int64_t p = blockIdx.x; p < prm.n_heavy; p += gridDim.x) {
    const int64_t beg = prm.row_ptr[p], end = prm.row_ptr[p + 1];
    // epilogue operands, loaded early by warp 0
    const int qv = lane % Q;
    const size_t off = (static_cast<size_t>(tile) * prm.n + p) * TW + qv * V;
    float prev[V], own[V];
#pragma unroll
    for (int v = 0; v < V; ++v) prev[v] = own[v] = 0.f;
    uint32_t orig = 0;
    int32_t compact = 0;
    if (warp == 0) {
      if (!prm.first)
        unpack16<T>(ld_stream(reinterpret_cast<const uint4*>(reinterpret_cast<const T*>(prm.u_pn) + off)), prev);
      if (ModeOf<MODE>::own)
        unpack16<T>(ld_gather(reinterpret_cast<const uint4*>(reinterpret_cast<const T*>(prm.u_cur) + off)), own);
      if (ModeOf<MODE>::ldos) {
        orig = static_cast<uint32_t>(prm.orig[p]);
        compact = prm.compact[p];
      }
    }
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.f;
    for (int64_t e0 = beg; e0 < end; e0 += BLK) {
      __syncthreads();
#pragma unroll
      for (int i = 0; i < kHeavyColsPerThread; ++i) {
        const int64_t e = e0 + tid + kStepThreads * i;
        s_col[tid + kStepThreads * i] = e < end ? ld_col(prm.col + e) : 0;
      }
      __syncthreads();
      const int cnt = static_cast<int>(end - e0 < BLK ? end - e0 : BLK);
      gather_list<T, Q, PH>(ubase, s_col, cnt, slot, ql, acc);
    }
#pragma unroll
    for (int o = Q; o < 32; o <<= 1)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
    if (lane < Q)
#pragma unroll
      for (int v = 0; v < V; ++v) red[warp][lane * V + v] = acc[v];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < kStepWarps; ++w) sum += red[w][qv * V + v];
        acc[v] = sum;
      }
      step_epilogue<T, Q, MODE>(prm, true, p, qv, tile, acc, prev, own, static_cast<float>(end - beg), orig, compact,
                                lane == 0, dd0, dd1);
    }
    __syncthreads();
  }
  double a0 = dd0.value(), a1 = dd1.value();
  block_sum2<kStepWarps>(a0, a1);
  if (threadIdx.x == 0) {
    const size_t i = static_cast<size_t>(tile) * gridDim.x + blockIdx.x;
    prm.partial[i] = a0;
    if (!ModeOf<MODE>::ldos) prm.partial[prm.part_width + i] = a1;
  }
}

// ---------------------------------------------------------------------------
// Medium rows (kMediumDeg <= degree < kHeavyDeg): a warp per row, 32/Q
// neighbour slots; each block of 256 column indices is staged in the warp's
// shared memory with coalesced loads before its gathers.  Grid (ctas, T).
// ---------------------------------------------------------------------------
constexpr int kMediumCols = 256;  // staged indices per warp per block

template <typename T, int Q, int MODE>
__global__ void __launch_bounds__(kStepThreads) k_cheb_medium(const StepParams prm) {
  constexpr int V = VecT<T>::N;
  constexpr int TW = Q * V;
  constexpr int PS = 32 / Q;  // neighbour slots per row
  __shared__ int32_t s_col[kStepWarps][kMediumCols];
  const int tile = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / Q, ql = lane % Q;
  const uint4* ubase = reinterpret_cast<const uint4*>(prm.u_cur) + static_cast<size_t>(tile) * prm.n * Q;
  SumD dd0, dd1;
  const int64_t w0 = static_cast<int64_t>(blockIdx.x) * kStepWarps + warp;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * kStepWarps;
  for (int64_t p = prm.n_heavy + w0; p < prm.n_mid; p += nw) {
    const int64_t beg = prm.row_ptr[p], end = prm.row_ptr[p + 1];
    const size_t off = (static_cast<size_t>(tile) * prm.n + p) * TW + ql * V;
    float prev[V], own[V];
#pragma unroll
    for (int v = 0; v < V; ++v) prev[v] = own[v] = 0.f;
    uint32_t orig = 0;
    int32_t compact = 0;
    if (!prm.first) unpack16<T>(ld_stream(reinterpret_cast<const uint4*>(reinterpret_cast<const T*>(prm.u_pn) + off)), prev);
    if (ModeOf<MODE>::own)
      unpack16<T>(ld_gather(reinterpret_cast<const uint4*>(reinterpret_cast<const T*>(prm.u_cur) + off)), own);
    if (ModeOf<MODE>::ldos) {
      orig = static_cast<uint32_t>(prm.orig[p]);
      compact = prm.compact[p];
    }
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.f;
    for (int64_t e0 = beg; e0 < end; e0 += kMediumCols) {
#pragma unroll
      for (int i = 0; i < kMediumCols / 32; ++i) {
        const int64_t e = e0 + lane + 32 * i;
        s_col[warp][lane + 32 * i] = e < end ? ld_col(prm.col + e) : 0;
      }
      __syncwarp();
      const int cnt = static_cast<int>(end - e0 < kMediumCols ? end - e0 : kMediumCols);
      gather_list<T, Q, PS>(ubase, s_col[warp], cnt, slot, ql, acc);
      __syncwarp();
    }
#pragma unroll
    for (int o = Q; o < 32; o <<= 1)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
    step_epilogue<T, Q, MODE>(prm, true, p, ql, tile, acc, prev, own, static_cast<float>(end - beg), orig, compact,
                              lane == 0, dd0, dd1);
  }
  double a0 = dd0.value(), a1 = dd1.value();
  block_sum2<kStepWarps>(a0, a1);
  if (threadIdx.x == 0) {
    const size_t i = static_cast<size_t>(prm.mid_part_off) + static_cast<size_t>(tile) * gridDim.x + blockIdx.x;
    prm.partial[i] = a0;
    if (!ModeOf<MODE>::ldos) prm.partial[prm.part_width + i] = a1;
  }
}

// ---------------------------------------------------------------------------
// Light rows (degree < kMediumDeg), the bulk of a sparse graph: every warp
// works through "rounds" of R = 32/Q consecutive rows (a group of Q lanes per
// row, one 16-byte chunk of the tile row each).  Work items (tile, round) are
// dealt to warps round-robin in tile-major order, so concurrently running
// warps gather from one tile of U_k.  Each warp double-buffers its items in
// shared memory: while it gathers for item i, its lanes have already issued
// cp.async copies of item i+1's row offsets, column indices, U_{k-1} rows and
// own U_k rows (DOS) or original / compact ids (LDOS) into the other slot,
// and lane 0 has loaded the CSR range of item i+2.  So only the gathers of
// neighbour rows of U_k are on the warp's critical path.
// ---------------------------------------------------------------------------
template <int Q, int ROWB, int MODE>
struct RoundLayout {
  static constexpr int R = 32 / Q;                                 // rows per round
  static constexpr int RP = (((R + 3) * 8) + 15) / 16 * 16;       // row offsets from an even row
  static constexpr int COL = ((R * (kMediumDeg - 1) + 8) * 4 + 15) / 16 * 16;
  static constexpr int BLK = R * ROWB;
  static constexpr int IDS = ((R + 8) * 4 + 15) / 16 * 16;
  static constexpr int off_rp = 0;
  static constexpr int off_col = off_rp + RP;
  static constexpr int off_prev = off_col + COL;
  static constexpr int off_aux = off_prev + BLK;                              // own U_k rows
  static constexpr int off_ids = off_aux + (ModeOf<MODE>::own ? BLK : 0);     // original / compact ids
  static constexpr int SLOT = off_ids + (ModeOf<MODE>::ldos ? 2 * IDS : 0);
  static constexpr int WARP = 2 * SLOT;  // two slots per warp
};

template <typename T, int Q, int MODE>
__global__ void __launch_bounds__(kStepThreads, 3) k_cheb_light(const StepParams prm) {
  constexpr int V = VecT<T>::N;
  constexpr int TW = Q * V;
  constexpr int ROWB = TW * static_cast<int>(sizeof(T));
  using L = RoundLayout<Q, ROWB, MODE>;
  using MD = ModeOf<MODE>;
  constexpr int R = L::R;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / Q, ql = lane % Q;
  unsigned char* wbuf = smem + warp * L::WARP;
  const int64_t light0 = prm.n_mid;
  const int64_t n_rounds = (prm.n - light0 + R - 1) / R;
  const int64_t nwarps = static_cast<int64_t>(gridDim.x) * kStepWarps;
  SumFF dd0, dd1;

  // item it = (tile, round) = (it / n_rounds, it % n_rounds); a warp takes
  // items wid, wid + nwarps, ...
  struct Cursor {
    int64_t round;
    int tile;
  };
  auto advance = [&](Cursor& c) {
    c.round += nwarps;
    while (c.round >= n_rounds) {
      c.round -= n_rounds;
      ++c.tile;
    }
  };
  auto rows_of = [&](const Cursor& c, int64_t& r0, int64_t& r1) {
    r0 = light0 + c.round * R;
    r1 = r0 + R < prm.n ? r0 + R : prm.n;
  };
  // the warp's lanes issue the copies of an item into slot s (e0, e1 = its CSR range)
  auto issue = [&](const Cursor& c, int s, int64_t e0, int64_t e1) {
    int64_t r0, r1;
    rows_of(c, r0, r1);
    unsigned char* sl = wbuf + s * L::SLOT;
    const int64_t r0a = r0 & ~int64_t(1), ea = e0 & ~int64_t(3), r0i = r0 & ~int64_t(3);
    warp_copy16(sl + L::off_rp, reinterpret_cast<const unsigned char*>(prm.row_ptr + r0a), (r1 + 2 - r0a) >> 1,
                lane);
    warp_copy16(sl + L::off_col, reinterpret_cast<const unsigned char*>(prm.col + ea),
                (((e1 + 3) & ~int64_t(3)) - ea) >> 2, lane);
    const size_t row_off = (static_cast<size_t>(c.tile) * prm.n + r0) * TW;
    const int64_t blk = (r1 - r0) * (ROWB / 16);
    if (!prm.first)
      warp_copy16(sl + L::off_prev, reinterpret_cast<const unsigned char*>(reinterpret_cast<const T*>(prm.u_pn) + row_off),
                  blk, lane);
    if (MD::own)
      warp_copy16(sl + L::off_aux, reinterpret_cast<const unsigned char*>(reinterpret_cast<const T*>(prm.u_cur) + row_off),
                  blk, lane);
    if (MD::ldos) {
      const int64_t ids = (((r1 + 3) & ~int64_t(3)) - r0i) >> 2;
      warp_copy16(sl + L::off_ids, reinterpret_cast<const unsigned char*>(prm.orig + r0i), ids, lane);
      warp_copy16(sl + L::off_ids + L::IDS, reinterpret_cast<const unsigned char*>(prm.compact + r0i), ids, lane);
    }
  };
  // CSR range of an item, loaded by lane 0 and broadcast (one iteration early)
  auto range_of = [&](const Cursor& c, int64_t& e0, int64_t& e1) {
    e0 = e1 = 0;
    if (lane == 0 && c.tile < prm.tiles) {
      int64_t r0, r1;
      rows_of(c, r0, r1);
      e0 = prm.row_ptr[r0];
      e1 = prm.row_ptr[r1];
    }
  };

  // cur = this iteration's item, nx1 = the next, nx2 = the one after
  Cursor cur{static_cast<int64_t>(blockIdx.x) * kStepWarps + warp, 0};
  if (n_rounds == 0) cur.tile = prm.tiles;
  while (cur.tile < prm.tiles && cur.round >= n_rounds) {
    cur.round -= n_rounds;
    ++cur.tile;
  }
  Cursor nx1 = cur;
  if (n_rounds > 0) advance(nx1);
  Cursor nx2 = nx1;
  if (n_rounds > 0) advance(nx2);
  int64_t nb0, nb1;  // CSR range of nx1 (lane 0)
  {
    int64_t e0, e1;
    range_of(cur, e0, e1);
    range_of(nx1, nb0, nb1);
    e0 = __shfl_sync(0xffffffffu, e0, 0);
    e1 = __shfl_sync(0xffffffffu, e1, 0);
    if (cur.tile < prm.tiles) issue(cur, 0, e0, e1);
    cp_async_commit();
  }
  for (int it = 0; cur.tile < prm.tiles; ++it) {
    const int s = it & 1;
    // issue nx1 into the other slot (its range was loaded one iteration ago),
    // and load the range of nx2; one group is committed per iteration
    {
      const int64_t e0 = __shfl_sync(0xffffffffu, nb0, 0), e1 = __shfl_sync(0xffffffffu, nb1, 0);
      if (nx1.tile < prm.tiles) issue(nx1, s ^ 1, e0, e1);
      cp_async_commit();
      range_of(nx2, nb0, nb1);
    }
    cp_async_wait<1>();  // this item's group has landed (only nx1's may be pending)
    __syncwarp();
    const int tile = cur.tile;
    int64_t r0, r1;
    rows_of(cur, r0, r1);
    const unsigned char* sl = wbuf + s * L::SLOT;
    const int64_t r0a = r0 & ~int64_t(1), r0i = r0 & ~int64_t(3);
    const int64_t* rp = reinterpret_cast<const int64_t*>(sl + L::off_rp) + (r0 - r0a);
    const int64_t ea = rp[0] & ~int64_t(3);
    const int32_t* cidx = reinterpret_cast<const int32_t*>(sl + L::off_col);
    const uint4* ubase = reinterpret_cast<const uint4*>(prm.u_cur) + static_cast<size_t>(tile) * prm.n * Q;
    const bool active = r0 + grp < r1;
    int64_t beg = 0, end = 0;
    if (active) {
      beg = rp[grp];
      end = rp[grp + 1];
    }
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.f;
    gather_list<T, Q, 1>(ubase, cidx + (beg - ea), static_cast<int>(end - beg), 0, ql, acc);
    float prev[V], own[V];
#pragma unroll
    for (int v = 0; v < V; ++v) prev[v] = own[v] = 0.f;
    uint32_t orig = 0;
    int32_t compact = 0;
    if (active) {
      if (!prm.first) unpack16<T>(*reinterpret_cast<const uint4*>(sl + L::off_prev + grp * ROWB + ql * 16), prev);
      if (MD::own) unpack16<T>(*reinterpret_cast<const uint4*>(sl + L::off_aux + grp * ROWB + ql * 16), own);
      if (MD::ldos) {
        orig = static_cast<uint32_t>(reinterpret_cast<const int32_t*>(sl + L::off_ids)[r0 + grp - r0i]);
        compact = reinterpret_cast<const int32_t*>(sl + L::off_ids + L::IDS)[r0 + grp - r0i];
      }
    }
    step_epilogue<T, Q, MODE>(prm, active, r0 + grp, ql, tile, acc, prev, own, static_cast<float>(end - beg), orig,
                              compact, ql == 0, dd0, dd1);
    __syncwarp();  // the slot is read; it is refilled next iteration
    cur = nx1;
    nx1 = nx2;
    if (n_rounds > 0) advance(nx2);
  }
  cp_async_wait<0>();  // the trailing groups are empty; nothing is left in flight
  double a0 = dd0.value(), a1 = dd1.value();
  block_sum2<kStepWarps>(a0, a1);
  if (threadIdx.x == 0) {
    const size_t i = static_cast<size_t>(prm.light_part_off) + blockIdx.x;
    prm.partial[i] = a0;
    if (!MD::ldos) prm.partial[prm.part_width + i] = a1;
  }
}

// ---- initialisation: U_0 = S Z (or S Z_r with the twin filter) -------------
struct InitParams {
  const int32_t* __restrict__ orig;     // [n] original ids
  const int32_t* __restrict__ compact;  // [n] compact ids
  const float* __restrict__ s32;        // [n_compact] 1/sqrt(d), compact order
  const int32_t* __restrict__ slot;     // [n] class slot or -1 (filter), or null
  const int32_t* __restrict__ slot_size;
  const float* __restrict__ csum;       // [n_classes][nz_pad] class probe sums
  void* u0;                             // block U_0
  int64_t n;
  int t;          // tile width
  int nz, nz_pad;
  uint64_t seed;
  double* partial;  // [gridDim.x]: sum of squares of V_0
  int unscaled;     // 1: U_0 = Z (operators A, D - A), else U_0 = S Z
};

__device__ __forceinline__ float probe_value(uint64_t word, int j, int nz) {
  return j < nz ? (((word >> (j & 63)) & 1ull) ? -1.f : 1.f) : 0.f;
}

template <typename T>
__global__ void __launch_bounds__(256) k_init_block(const InitParams prm) {
  constexpr int V = VecT<T>::N;
  const int chunks = prm.nz_pad / V;  // 16-byte chunks per row
  const int64_t total = prm.n * chunks;
  double acc = 0.0, dummy = 0.0;
  for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < total;
       c += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t p = c / chunks;
    const int j0 = static_cast<int>(c % chunks) * V;
    const uint64_t word = probe_word(prm.seed, static_cast<uint32_t>(prm.orig[p]), static_cast<uint32_t>(j0 >> 6));
    float z[V];
    const int sl = prm.slot ? prm.slot[p] : -1;
    if (sl >= 0) {
      const float inv = 1.0f / static_cast<float>(prm.slot_size[sl]);
#pragma unroll
      for (int v = 0; v < V; ++v) z[v] = prm.csum[static_cast<size_t>(sl) * prm.nz_pad + j0 + v] * inv;
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) z[v] = probe_value(word, j0 + v, prm.nz);
    }
    const float s = prm.unscaled ? 1.0f : prm.s32[prm.compact[p]];
    float u[V];
    float sq = 0.f;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      u[v] = s * z[v];
      sq = fmaf(z[v], z[v], sq);
    }
    acc += static_cast<double>(sq);
    const int tile = j0 / prm.t;
    const size_t off = (static_cast<size_t>(tile) * prm.n + p) * prm.t + (j0 % prm.t);
    *reinterpret_cast<uint4*>(reinterpret_cast<T*>(prm.u0) + off) = pack16<T>(u);
  }
  block_sum2<8>(acc, dummy);
  if (threadIdx.x == 0) prm.partial[blockIdx.x] = acc;
}

// ---- launch entry points (instantiated per storage type) -------------------
struct Plan {
  int t = 16;       // tile width (probes per tile)
  int q = 4;        // 16-byte chunks per tile row
  int tiles = 1;    // T
  int nz_pad = 16;
  int heavy_ctas = 0;
  int mid_ctas = 0;
  int light_ctas = 0;
  int smem = 0;     // dynamic shared memory of the light kernel
  int64_t part_width = 1;  // partial slots per dot
};

template <typename T, int Q, int MODE>
int light_smem() {
  return kStepWarps * RoundLayout<Q, Q * 16, MODE>::WARP + 128;
}

// Raise a kernel's dynamic shared-memory limit on the current device.  The
// attribute belongs to the device's context, so the raised limit is kept per
// device (and only grows, so earlier plans stay launchable).
int raise_smem_limit(const void* kernel, int* limits /* [64], per device */, int smem);

template <typename T, int Q, int MODE>
int light_config_q(int* smem, int* ctas_per_sm) {
  *smem = light_smem<T, Q, MODE>();
  static int s_limit[64] = {};
  const int st = raise_smem_limit(reinterpret_cast<const void*>(k_cheb_light<T, Q, MODE>), s_limit, *smem);
  if (st != DOS_OK) return st;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_cheb_light<T, Q, MODE>, kStepThreads, *smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor", __FILE__, __LINE__);
  return DOS_OK;
}

// Optional side streams: the heavy- and medium-row kernels run on them,
// forked from and joined back into the caller's stream, so they overlap the
// light-row kernel.  All null: everything runs on the caller's stream.
struct SideStreams {
  cudaStream_t a = nullptr, b = nullptr;
  cudaEvent_t fork = nullptr, join_a = nullptr, join_b = nullptr;
};

template <typename T, int Q, int MODE>
int launch_step_q(const Plan& plan, const StepParams& prm, cudaStream_t s, const SideStreams& side) {
  const bool heavy = prm.n_heavy > 0 && plan.heavy_ctas > 0;
  const bool mid = prm.n_mid > prm.n_heavy && plan.mid_ctas > 0;
  const bool fork = side.a && side.b && (heavy || mid);
  if (fork) NDOS_CUDA(cudaEventRecord(side.fork, s));
  if (heavy) {
    cudaStream_t hs = fork ? side.a : s;
    if (fork) NDOS_CUDA(cudaStreamWaitEvent(hs, side.fork, 0));
    k_cheb_heavy<T, Q, MODE><<<dim3(plan.heavy_ctas, plan.tiles), kStepThreads, 0, hs>>>(prm);
    NDOS_LAUNCHED();
    if (fork) NDOS_CUDA(cudaEventRecord(side.join_a, hs));
  }
  if (mid) {
    cudaStream_t ms = fork ? side.b : s;
    if (fork) NDOS_CUDA(cudaStreamWaitEvent(ms, side.fork, 0));
    k_cheb_medium<T, Q, MODE><<<dim3(plan.mid_ctas, plan.tiles), kStepThreads, 0, ms>>>(prm);
    NDOS_LAUNCHED();
    if (fork) NDOS_CUDA(cudaEventRecord(side.join_b, ms));
  }
  if (prm.n > prm.n_mid && plan.light_ctas > 0) {
    if (MODE == kModeDosOp) {  // the plan was made for kModeDos (same layout): raise this instance's limit
      int smem = 0, ctas = 0;
      const int st = light_config_q<T, Q, MODE>(&smem, &ctas);
      if (st != DOS_OK) return st;
    }
    k_cheb_light<T, Q, MODE><<<plan.light_ctas, kStepThreads, plan.smem, s>>>(prm);
    NDOS_LAUNCHED();
  }
  if (fork && heavy) NDOS_CUDA(cudaStreamWaitEvent(s, side.join_a, 0));
  if (fork && mid) NDOS_CUDA(cudaStreamWaitEvent(s, side.join_b, 0));
  return DOS_OK;
}

// dispatch on q to a template instance
#define NDOS_DISPATCH_Q(T, q, CALL)                   \
  switch (q) {                                        \
    case 1:                                           \
      return CALL(T, 1);                              \
    case 2:                                           \
      return CALL(T, 2);                              \
    case 4:                                           \
      return CALL(T, 4);                              \
    case 8:                                           \
      return CALL(T, 8);                              \
    case 16:                                          \
      if constexpr (VecT<T>::N == 4) return CALL(T, 16); \
      break;                                          \
    default:                                          \
      break;                                          \
  }

// one tile width, dispatch on the mode (LDOS on A / D - A: FP32 storage only)
template <typename T, int Q>
int launch_step_mode(const Plan& plan, int mode, const StepParams& prm, cudaStream_t s, const SideStreams& side) {
  switch (mode) {
    case kModeDos:
      return launch_step_q<T, Q, kModeDos>(plan, prm, s, side);
    case kModeLdos:
      return launch_step_q<T, Q, kModeLdos>(plan, prm, s, side);
    case kModeDosOp:
      return launch_step_q<T, Q, kModeDosOp>(plan, prm, s, side);
    default:
      if constexpr (std::is_same<T, float>::value) return launch_step_q<T, Q, kModeLdosOp>(plan, prm, s, side);
      return fail(DOS_EINVAL, "LDOS of A and D - A is computed in FP32 only");
  }
}

template <typename T, int Q>
int config_mode(int mode, int* smem, int* ctas) {
  switch (mode) {
    case kModeLdos:
      return light_config_q<T, Q, kModeLdos>(smem, ctas);
    case kModeLdosOp:
      if constexpr (std::is_same<T, float>::value) return light_config_q<T, Q, kModeLdosOp>(smem, ctas);
      return fail(DOS_EINVAL, "LDOS of A and D - A is computed in FP32 only");
    default:  // kModeDos; kModeDosOp has the same layout
      return light_config_q<T, Q, kModeDos>(smem, ctas);
  }
}

// Chebyshev step launch for storage type T (instantiated in kpm_<type>.cu)
template <typename T>
int launch_step(const Plan& plan, int mode, const StepParams& prm, cudaStream_t s, const SideStreams& side) {
#define NDOS_LAUNCH_CALL(TT, QQ) launch_step_mode<TT, QQ>(plan, mode, prm, s, side)
  NDOS_DISPATCH_Q(T, plan.q, NDOS_LAUNCH_CALL)
#undef NDOS_LAUNCH_CALL
  return fail(DOS_EINVAL, "unsupported tile width");
}

// dynamic shared memory and resident CTAs per SM of the light kernel
template <typename T>
int step_config(int q, int mode, int* smem, int* ctas) {
#define NDOS_CONFIG_CALL(TT, QQ) config_mode<TT, QQ>(mode, smem, ctas)
  NDOS_DISPATCH_Q(T, q, NDOS_CONFIG_CALL)
#undef NDOS_CONFIG_CALL
  return fail(DOS_EINVAL, "unsupported tile width");
}

template <typename T>
int launch_init(const InitParams& prm, int grid, cudaStream_t s) {
  k_init_block<T><<<grid, 256, 0, s>>>(prm);
  NDOS_LAUNCHED();
  return DOS_OK;
}

// The kernels are instantiated once, in kpm_<type>.cu.  Other translation
// units must not instantiate their own copies: each copy would be a separate
// device function, and attributes set on one (the shared-memory limit) would
// not apply to the other.
#define NDOS_EXTERN_STEP(T)                                                                           \
  extern template int launch_step<T>(const Plan&, int, const StepParams&, cudaStream_t, const SideStreams&); \
  extern template int step_config<T>(int, int, int*, int*);                                          \
  extern template int launch_init<T>(const InitParams&, int, cudaStream_t);
NDOS_EXTERN_STEP(float)
NDOS_EXTERN_STEP(__nv_bfloat16)
NDOS_EXTERN_STEP(__half)
#undef NDOS_EXTERN_STEP

}  // namespace netdos
