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
// One launch processes every tile (blockIdx.y = tile) of one step, so the
// rows gathered by concurrently running CTAs are one tile of U_k.
//
// Rows are in degree-sorted order (heavy rows first).  CTAs with
// blockIdx.x < heavy_ctas own whole heavy rows (all 256 threads on one row);
// the remaining CTAs give each light row a group of G = Q * P lanes: P
// neighbour slots, each slot Q lanes that read one 16-byte chunk of the
// neighbour's tile row (t = Q * VEC probes).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace netdos {

constexpr int kStepThreads = 256;
constexpr int kStepWarps = kStepThreads / 32;

enum StepMode { kModeDos = 0, kModeLdos = 1 };

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

struct StepParams {
  const int64_t* __restrict__ row_ptr;   // [n+1] degree-sorted CSR
  const int32_t* __restrict__ col;       // [nnz] neighbour positions
  const int32_t* __restrict__ deg;       // [n]
  const int32_t* __restrict__ orig;      // [n] original ids (LDOS probe signs)
  const int32_t* __restrict__ compact;   // [n] compact ids (LDOS output column)
  const void* u_cur;                     // U_k
  void* u_pn;                            // U_{k-1} in, U_{k+1} out (in place)
  int64_t n;
  int64_t n_heavy;
  int heavy_ctas;
  int first;        // 1: U_1 = S^2 A U_0 (no U_{k-1} term)
  int nz;           // real probe count (columns >= nz are zero padding)
  float inv_nz;
  uint64_t seed;
  double* partial;  // this step's partials: [n_dots][T][gridDim.x]
  float* ldos;      // LDOS: C_out + m * n_compact, indexed by compact id
  int ldos_atomic;  // 1 when several tiles add into the same C entry
};

// Epilogue of one row: recurrence update, store, fused dots / LDOS.
// Executed by all 32 lanes of a warp; `active` lanes own a row whose
// neighbour sum is in acc (ql = which 16-byte chunk of the tile row).
template <typename T, int Q, int MODE>
__device__ __forceinline__ void step_epilogue(const StepParams& prm, bool active, int64_t p, int ql, int tile,
                                              const float* acc, bool owner, double& dd0, double& dd1) {
  constexpr int V = VecT<T>::N;
  constexpr int TW = Q * V;  // tile width t
  float prod0 = 0.f, prod1 = 0.f;
  float fd = 1.f;
  if (active) {
    const int d = prm.deg[p];
    fd = static_cast<float>(d);
    const size_t off = (static_cast<size_t>(tile) * prm.n + p) * TW + ql * V;
    uint4* pn = reinterpret_cast<uint4*>(reinterpret_cast<T*>(prm.u_pn) + off);
    float u[V];
    if (prm.first) {
      const float sc = 1.0f / fd;
#pragma unroll
      for (int v = 0; v < V; ++v) u[v] = acc[v] * sc;
    } else {
      const float sc = 2.0f / fd;
      float prev[V];
      unpack16<T>(ld_stream(pn), prev);
#pragma unroll
      for (int v = 0; v < V; ++v) u[v] = fmaf(acc[v], sc, -prev[v]);
    }
    const uint4 packed = pack16<T>(u);
    st_stream(pn, packed);
    unpack16<T>(packed, u);  // the dots use the stored (rounded) values
    if (MODE == kModeDos) {
      float own[V];
      const uint4* cur = reinterpret_cast<const uint4*>(reinterpret_cast<const T*>(prm.u_cur) + off);
      unpack16<T>(ld_gather(cur), own);  // own row of U_k: also gathered by neighbours
#pragma unroll
      for (int v = 0; v < V; ++v) {
        prod0 = fmaf(u[v], u[v], prod0);
        prod1 = fmaf(u[v], own[v], prod1);
      }
    } else {
      const int j0 = tile * TW + ql * V;
      const uint64_t word = probe_word(prm.seed, static_cast<uint32_t>(prm.orig[p]), static_cast<uint32_t>(j0 >> 6));
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int j = j0 + v;
        if (j < prm.nz) prod0 += ((word >> (j & 63)) & 1ull) ? -u[v] : u[v];
      }
    }
  }
  // reduce over the Q lanes that share a row
#pragma unroll
  for (int o = 1; o < Q; o <<= 1) {
    prod0 += __shfl_xor_sync(0xffffffffu, prod0, o);
    if (MODE == kModeDos) prod1 += __shfl_xor_sync(0xffffffffu, prod1, o);
  }
  if (active && owner) {
    if (MODE == kModeDos) {
      dd0 += static_cast<double>(fd * prod0);
      dd1 += static_cast<double>(fd * prod1);
    } else {
      const float vsum = prod0 * sqrtf(fd);  // sum_j z_j (V_{k+1})_j of this tile
      dd0 += static_cast<double>(vsum);
      float* dst = prm.ldos + prm.compact[p];
      if (prm.ldos_atomic)
        atomicAdd(dst, vsum * prm.inv_nz);
      else
        *dst = vsum * prm.inv_nz;
    }
  }
}


// acc[0..V) += sum of the 16-byte chunk `ql` of U_k rows col[e], e = beg + slot,
// beg + slot + STRIDE, ... < end
template <typename T, int Q, int STRIDE>
__device__ __forceinline__ void gather_sum(const StepParams& prm, int64_t beg, int64_t end, int slot, int ql,
                                           int tile, float* acc) {
  constexpr int V = VecT<T>::N;
  const uint4* base = reinterpret_cast<const uint4*>(prm.u_cur) + static_cast<size_t>(tile) * prm.n * Q + ql;
  int64_t e = beg + slot;
  for (; e + 3 * STRIDE < end; e += 4 * STRIDE) {
    const int32_t j0 = ld_col(prm.col + e);
    const int32_t j1 = ld_col(prm.col + e + STRIDE);
    const int32_t j2 = ld_col(prm.col + e + 2 * STRIDE);
    const int32_t j3 = ld_col(prm.col + e + 3 * STRIDE);
    const uint4 r0 = ld_gather(base + static_cast<size_t>(j0) * Q);
    const uint4 r1 = ld_gather(base + static_cast<size_t>(j1) * Q);
    const uint4 r2 = ld_gather(base + static_cast<size_t>(j2) * Q);
    const uint4 r3 = ld_gather(base + static_cast<size_t>(j3) * Q);
    float a[V], b[V];
    unpack16<T>(r0, a);
    unpack16<T>(r1, b);
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] += a[v] + b[v];
    unpack16<T>(r2, a);
    unpack16<T>(r3, b);
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] += a[v] + b[v];
  }
  for (; e < end; e += STRIDE) {
    const int32_t j0 = ld_col(prm.col + e);
    float a[V];
    unpack16<T>(ld_gather(base + static_cast<size_t>(j0) * Q), a);
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] += a[v];
  }
}

// CTA-wide deterministic sum of two doubles; thread 0 gets the result
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[kStepWarps], sb[kStepWarps];
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
    for (int w = 0; w < kStepWarps; ++w) {
      x += sa[w];
      y += sb[w];
    }
    a = x;
    b = y;
  }
}

// One Chebyshev step over every tile: U_{k+1} = (2/d) A U_k - U_{k-1}, fused
// with the moment dots (DOS: <V_{k+1},V_{k+1}> and <V_{k+1},V_k>; LDOS:
// z o V_{k+1} per node and its sum).
template <typename T, int Q, int P, int MODE>
__global__ void __launch_bounds__(kStepThreads) k_cheb_step(const StepParams prm) {
  constexpr int V = VecT<T>::N;
  const int tile = blockIdx.y;
  double dd0 = 0.0, dd1 = 0.0;
  if (static_cast<int>(blockIdx.x) < prm.heavy_ctas) {
    // ---- heavy rows: a CTA per row ----
    constexpr int PH = kStepThreads / Q;
    __shared__ float red[kStepWarps][Q * V];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int slot = tid / Q, ql = tid % Q;
    for (int64_t p = blockIdx.x; p < prm.n_heavy; p += prm.heavy_ctas) {
      float acc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = 0.f;
      gather_sum<T, Q, PH>(prm, prm.row_ptr[p], prm.row_ptr[p + 1], slot, ql, tile, acc);
#pragma unroll
      for (int o = Q; o < 32; o <<= 1)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
      if (lane < Q)
#pragma unroll
        for (int v = 0; v < V; ++v) red[warp][lane * V + v] = acc[v];
      __syncthreads();
      if (warp == 0) {
        const int qv = lane % Q;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          float s = 0.f;
#pragma unroll
          for (int w = 0; w < kStepWarps; ++w) s += red[w][qv * V + v];
          acc[v] = s;
        }
        step_epilogue<T, Q, MODE>(prm, true, p, qv, tile, acc, lane == 0, dd0, dd1);
      }
      __syncthreads();
    }
  } else {
    // ---- light rows: G = Q * P lanes per row ----
    constexpr int G = Q * P;
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G, lig = lane % G, slot = lig / Q, ql = lig % Q;
    const int64_t light_n = prm.n - prm.n_heavy;
    const int64_t w_id = static_cast<int64_t>(blockIdx.x - prm.heavy_ctas) * kStepWarps + warp;
    const int64_t n_w = static_cast<int64_t>(gridDim.x - prm.heavy_ctas) * kStepWarps;
    for (int64_t base = w_id * RPW; base < light_n; base += n_w * RPW) {
      const bool active = base + grp < light_n;
      const int64_t p = prm.n_heavy + base + grp;
      float acc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = 0.f;
      if (active) gather_sum<T, Q, P>(prm, prm.row_ptr[p], prm.row_ptr[p + 1], slot, ql, tile, acc);
#pragma unroll
      for (int o = Q; o < G; o <<= 1)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
      step_epilogue<T, Q, MODE>(prm, active, p, ql, tile, acc, slot == 0 && ql == 0, dd0, dd1);
    }
  }
  block_sum2(dd0, dd1);
  if (threadIdx.x == 0) {
    const size_t w = static_cast<size_t>(gridDim.y) * gridDim.x;
    const size_t i = static_cast<size_t>(tile) * gridDim.x + blockIdx.x;
    prm.partial[i] = dd0;
    if (MODE == kModeDos) prm.partial[w + i] = dd1;
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
    const float s = prm.s32[prm.compact[p]];
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
  block_sum2(acc, dummy);
  if (threadIdx.x == 0) prm.partial[blockIdx.x] = acc;
}

// ---- launch entry points (instantiated per storage type) -------------------
struct Plan {
  int t = 16;      // tile width (probes per tile)
  int q = 4;       // lanes per 16-byte-chunked tile row
  int p = 2;       // neighbour slots per light row
  int tiles = 1;   // T
  int nz_pad = 16;
  int gx = 1;      // grid.x of a step (heavy + light CTAs)
  int heavy_ctas = 0;
};

template <typename T, int Q, int P>
int launch_step_qp(const Plan& plan, int mode, const StepParams& prm, cudaStream_t s) {
  const dim3 grid(plan.gx, plan.tiles);
  if (mode == kModeDos)
    k_cheb_step<T, Q, P, kModeDos><<<grid, kStepThreads, 0, s>>>(prm);
  else
    k_cheb_step<T, Q, P, kModeLdos><<<grid, kStepThreads, 0, s>>>(prm);
  NDOS_LAUNCHED();
  return DOS_OK;
}

template <typename T, int Q>
int launch_step_q(const Plan& plan, int mode, const StepParams& prm, cudaStream_t s) {
  switch (plan.p) {
    case 1:
      return launch_step_qp<T, Q, 1>(plan, mode, prm, s);
    case 2:
      if constexpr (Q * 2 <= 32) return launch_step_qp<T, Q, 2>(plan, mode, prm, s);
      break;
    case 4:
      if constexpr (Q * 4 <= 32) return launch_step_qp<T, Q, 4>(plan, mode, prm, s);
      break;
    default:
      break;
  }
  return fail(DOS_EINVAL, "unsupported neighbour-slot count");
}

// Chebyshev step launch for storage type T (instantiated in kpm_<type>.cu)
template <typename T>
int launch_step(const Plan& plan, int mode, const StepParams& prm, cudaStream_t s) {
  switch (plan.q) {
    case 1:
      return launch_step_q<T, 1>(plan, mode, prm, s);
    case 2:
      return launch_step_q<T, 2>(plan, mode, prm, s);
    case 4:
      return launch_step_q<T, 4>(plan, mode, prm, s);
    case 8:
      return launch_step_q<T, 8>(plan, mode, prm, s);
    case 16:
      if constexpr (VecT<T>::N == 4) return launch_step_q<T, 16>(plan, mode, prm, s);
      break;
    default:
      break;
  }
  return fail(DOS_EINVAL, "unsupported tile width");
}

template <typename T>
int launch_init(const InitParams& prm, int grid, cudaStream_t s) {
  k_init_block<T><<<grid, 256, 0, s>>>(prm);
  NDOS_LAUNCHED();
  return DOS_OK;
}

// occupancy (resident CTAs per SM) of the step kernel for a plan
template <typename T>
int step_occupancy(const Plan& plan);
}  // namespace netdos
