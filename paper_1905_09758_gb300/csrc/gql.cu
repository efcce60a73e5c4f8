// Gauss quadrature and Lanczos (GQL, §3.2): per-probe Lanczos on H (or on A
// and D - A, §2.1), the Gauss rule of each probe's spectral measure, its
// Chebyshev moments and its histogram, and a spectral interval from the
// extreme Ritz values.
//
// Lanczos runs on all Nz probes at once, FP32 vectors and FP64 reductions.
// On H it works in the scaled space of the Chebyshev kernels (U = S v,
// S = D^{-1/2}):
//     (S H v)_i = (1/d_i) sum_{j in N(i)} U_j,  u^T H u = sum_i d_i U_i (S H u)_i,
//     ||v||^2 = sum_i d_i U_i^2;
// on A and D - A the vectors are unscaled (S = I, unit dot weights) and the
// apply is sum_j U_j, resp. d_i U_i - sum_j U_j.
// The stored vectors are unnormalised: W_1 = S z, W_{k+1} = S (X u_k - alpha_k u_k
// - beta_{k-1} u_{k-1}) with u_k = S^{-1} W_k / beta_{k-1}, beta_0 = ||z||.  A
// step is two passes:
//   apply   Y = S X u_k (gather: a CTA per heavy row, a warp per other row,
//           in the degree-sorted row order) and the alpha_k partials;
//   update  W_{k+1} = Y - (alpha_k / beta_{k-1}) W_k - (beta_{k-1} / beta_{k-2}) W_{k-1}
//           (in place over W_{k-1}) and the ||w||^2 partials,
// each followed by a fixed-order FP64 reduction over CTAs, one thread per
// probe.  A probe stops when beta_k <= 1e-5 x (the Gershgorin bound of ||X||:
// 1 for H, d_max for A, 2 d_max for D - A): its Krylov space is exhausted and
// what is left is FP32 rounding noise (relative ~1e-7); its later vectors are
// zero and its rule keeps the steps it ran.
// No reorthogonalisation (the paper names none).
#include <algorithm>
#include <cmath>

#include "kpm_kernels.cuh"  // gather_list, cp.async staging helpers

namespace netdos {
namespace {

constexpr int kLzThreads = 256;
constexpr int kLzWarps = kLzThreads / 32;

// operator of a Lanczos run
enum LzOp { kLzH = 0, kLzA = 1, kLzL = 2 };

struct LanczosState {
  double* alpha;       // [nz][m] output
  double* beta;        // [nz][m] output (beta[p][k]: ||w_{k+1}||)
  int32_t* steps;      // [nz] output
  double* b_prev;      // beta_{k-1} per probe (beta_0 = ||z||)
  double* b_prev2;     // beta_{k-2} per probe
  float* inv_b;        // 1 / beta_{k-1}, 0 once stopped
  float* c1;           // alpha_k / beta_{k-1}
  float* c2;           // beta_{k-1} / beta_{k-2} (0 at k = 1)
  double* part;        // [grid][nzp] partial sums
};

// W_1 = S z in the degree-sorted row order (a symmetric relabelling leaves
// the Lanczos coefficients unchanged): row-major N x nzp, z_pj = +-1 from the
// probe hash keyed by the original id, 0 in the padding columns; S = I for
// A and D - A
__global__ void k_lz_init(const int32_t* __restrict__ p_orig, const int32_t* __restrict__ p_compact,
                          const float* __restrict__ s32, int op, int64_t n, int nz, int nzp, uint64_t seed,
                          float* __restrict__ w_cur, float* __restrict__ w_prev) {
  const int64_t total = n * nzp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / nzp;
    const int j = static_cast<int>(e - i * nzp);
    float v = 0.f;
    if (j < nz) {
      const uint64_t word = probe_word(seed, static_cast<uint32_t>(p_orig[i]), static_cast<uint32_t>(j >> 6));
      const float si = op == kLzH ? s32[p_compact[i]] : 1.0f;
      v = ((word >> (j & 63)) & 1ull) ? -si : si;
    }
    w_cur[e] = v;
    w_prev[e] = 0.f;
  }
}

__global__ void k_lz_state0(int nz, int nzp, double norm0, LanczosState st) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nzp) return;
  const bool real = p < nz;
  st.b_prev[p] = norm0;
  st.b_prev2[p] = 1.0;
  st.inv_b[p] = real ? static_cast<float>(1.0 / norm0) : 0.f;
  st.c2[p] = 0.f;
  if (real) st.steps[p] = 0;
}

// Gather of one row's neighbour rows, chunk `ch` of slot `slot`, over the
// neighbours [e_lo, e_hi) taken `stride` apart in batches of 32: column
// indices are loaded coalesced and handed to the slots by shuffles, so the
// gathers of a batch are independent loads.
template <int Q>
__device__ __forceinline__ void lz_gather(const int32_t* __restrict__ col, const float* __restrict__ w, int nzp,
                                          int64_t e_lo, int64_t e_hi, int64_t stride, int lane, int slot, int ch,
                                          float4& acc) {
  constexpr int P = 32 / Q;
  for (int64_t e0 = e_lo; e0 < e_hi; e0 += stride) {
    const int cnt = static_cast<int>(e_hi - e0 < 32 ? e_hi - e0 : 32);
    const int32_t mine = lane < cnt ? col[e0 + lane] : 0;
#pragma unroll
    for (int u = 0; u < 32 / P; ++u) {
      const int src = slot + u * P;
      const int32_t c = __shfl_sync(0xffffffffu, mine, src);
      if (src < cnt) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(w + static_cast<size_t>(c) * nzp) + ch);
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
      }
    }
  }
}

// Epilogue of one row (lanes of slot 0), acc = sum_j W_j over the neighbours:
//   H      Y = acc / d * inv_b,                  alpha weight d
//   A      Y = acc * inv_b,                      alpha weight 1
//   D - A  Y = (d W_own - acc) * inv_b,          alpha weight 1
// and the row's alpha contributions weight (W_own inv_b) Y.
__device__ __forceinline__ void lz_row_out(int op, int64_t i, float dd, const float4& acc, const float4& ib, int nzp,
                                           int ch, const float* __restrict__ w_cur, float* __restrict__ y, double& a0,
                                           double& a1, double& a2, double& a3) {
  const float4 own = reinterpret_cast<const float4*>(w_cur + static_cast<size_t>(i) * nzp)[ch];
  float4 v = acc;
  float wd = 1.0f;
  if (op == kLzH) {
    const float sc = 1.0f / dd;
    v = make_float4(acc.x * sc, acc.y * sc, acc.z * sc, acc.w * sc);
    wd = dd;
  } else if (op == kLzL) {
    v = make_float4(dd * own.x - acc.x, dd * own.y - acc.y, dd * own.z - acc.z, dd * own.w - acc.w);
  }
  const float4 out = make_float4(v.x * ib.x, v.y * ib.y, v.z * ib.z, v.w * ib.w);
  reinterpret_cast<float4*>(y + static_cast<size_t>(i) * nzp)[ch] = out;
  a0 += static_cast<double>(wd * (own.x * ib.x) * out.x);
  a1 += static_cast<double>(wd * (own.y * ib.y) * out.y);
  a2 += static_cast<double>(wd * (own.z * ib.z) * out.z);
  a3 += static_cast<double>(wd * (own.w * ib.w) * out.w);
}

// apply, rows [row0, n) (degree < kHeavyDeg): Y = S X u_k and the alpha
// partials.  A warp per row: Q = nzp / 4 lanes hold one 16-byte chunk each,
// 32 / Q neighbour slots.  Partials of CTA b go to part[b].
template <int Q>
__global__ void __launch_bounds__(kLzThreads) k_lz_apply(int op, const int64_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ col,
                                                         const int32_t* __restrict__ deg, int64_t row0, int64_t n,
                                                         int nzp, const float* __restrict__ w_cur,
                                                         const float* __restrict__ inv_b, float* __restrict__ y,
                                                         double* __restrict__ part) {
  __shared__ double red[kLzWarps][4 * Q];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / Q, ch = lane % Q;
  const float4 ib = reinterpret_cast<const float4*>(inv_b)[ch];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  const int64_t w0 = static_cast<int64_t>(blockIdx.x) * kLzWarps + warp;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * kLzWarps;
  for (int64_t i = row0 + w0; i < n; i += nw) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    lz_gather<Q>(col, w_cur, nzp, row_ptr[i], row_ptr[i + 1], 32, lane, slot, ch, acc);
#pragma unroll
    for (int o = Q; o < 32; o <<= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
      acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
    }
    if (slot == 0) lz_row_out(op, i, static_cast<float>(deg[i]), acc, ib, nzp, ch, w_cur, y, a0, a1, a2, a3);
  }
  if (slot == 0) {
    red[warp][4 * ch + 0] = a0;
    red[warp][4 * ch + 1] = a1;
    red[warp][4 * ch + 2] = a2;
    red[warp][4 * ch + 3] = a3;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < 4 * Q; p += kLzThreads) {
    double sum = 0.0;
    for (int w = 0; w < kLzWarps; ++w) sum += red[w][p];
    part[static_cast<size_t>(blockIdx.x) * nzp + p] = sum;
  }
}

// apply, light rows [row0, n) (degree < kMediumDeg): the staged pipeline of
// the Chebyshev step's light kernel.  Each warp takes rounds of R = 32 / Q
// consecutive rows (Q lanes per row, one 16-byte chunk each); while it
// gathers for one round its lanes have already issued cp.async copies of the
// next round's row offsets, column indices and own rows W_k into the other
// shared-memory slot, and lane 0 has loaded the CSR range of the round after.
template <int Q>
struct LzRound {
  static constexpr int R = 32 / Q;
  static constexpr int RP = (((R + 3) * 8) + 15) / 16 * 16;
  static constexpr int COL = ((R * (kMediumDeg - 1) + 8) * 4 + 15) / 16 * 16;
  static constexpr int OWN = R * Q * 16;
  static constexpr int off_col = RP, off_own = RP + COL;
  static constexpr int SLOT = RP + COL + OWN;
  static constexpr int WARP = 2 * SLOT;
};

template <int Q>
__global__ void __launch_bounds__(kLzThreads) k_lz_apply_light(int op, const int64_t* __restrict__ row_ptr,
                                                               const int32_t* __restrict__ col, int64_t row0,
                                                               int64_t n, int nzp, const float* __restrict__ w_cur,
                                                               const float* __restrict__ inv_b, float* __restrict__ y,
                                                               double* __restrict__ part) {
  using L = LzRound<Q>;
  constexpr int R = L::R;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red[kLzWarps][4 * Q];
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / Q, ch = lane % Q;
  unsigned char* wbuf = smem + warp * L::WARP;
  const float4 ib = reinterpret_cast<const float4*>(inv_b)[ch];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  const int64_t n_rounds = (n - row0 + R - 1) / R;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * kLzWarps;
  auto rows_of = [&](int64_t rd, int64_t& r0, int64_t& r1) {
    r0 = row0 + rd * R;
    r1 = r0 + R < n ? r0 + R : n;
  };
  auto issue = [&](int64_t rd, int sl_i, int64_t e0, int64_t e1) {
    int64_t r0, r1;
    rows_of(rd, r0, r1);
    unsigned char* sl = wbuf + sl_i * L::SLOT;
    const int64_t r0a = r0 & ~int64_t(1), ea = e0 & ~int64_t(3);
    warp_copy16(sl, reinterpret_cast<const unsigned char*>(row_ptr + r0a), (r1 + 2 - r0a) >> 1, lane);
    warp_copy16(sl + L::off_col, reinterpret_cast<const unsigned char*>(col + ea), (((e1 + 3) & ~int64_t(3)) - ea) >> 2,
                lane);
    warp_copy16(sl + L::off_own, reinterpret_cast<const unsigned char*>(w_cur + static_cast<size_t>(r0) * nzp),
                (r1 - r0) * Q, lane);
  };
  auto range_of = [&](int64_t rd, int64_t& e0, int64_t& e1) {
    e0 = e1 = 0;
    if (lane == 0 && rd < n_rounds) {
      int64_t r0, r1;
      rows_of(rd, r0, r1);
      e0 = row_ptr[r0];
      e1 = row_ptr[r1];
    }
  };
  int64_t cur = static_cast<int64_t>(blockIdx.x) * kLzWarps + warp;
  int64_t nb0, nb1;
  {
    int64_t e0, e1;
    range_of(cur, e0, e1);
    range_of(cur + nw, nb0, nb1);
    e0 = __shfl_sync(0xffffffffu, e0, 0);
    e1 = __shfl_sync(0xffffffffu, e1, 0);
    if (cur < n_rounds) issue(cur, 0, e0, e1);
    cp_async_commit();
  }
  for (int it = 0; cur < n_rounds; ++it, cur += nw) {
    const int s = it & 1;
    {
      const int64_t e0 = __shfl_sync(0xffffffffu, nb0, 0), e1 = __shfl_sync(0xffffffffu, nb1, 0);
      if (cur + nw < n_rounds) issue(cur + nw, s ^ 1, e0, e1);
      cp_async_commit();
      range_of(cur + 2 * nw, nb0, nb1);
    }
    cp_async_wait<1>();
    __syncwarp();
    int64_t r0, r1;
    rows_of(cur, r0, r1);
    const unsigned char* sl = wbuf + s * L::SLOT;
    const int64_t r0a = r0 & ~int64_t(1);
    const int64_t* rp = reinterpret_cast<const int64_t*>(sl) + (r0 - r0a);
    const int64_t ea = rp[0] & ~int64_t(3);
    const bool active = r0 + grp < r1;
    int64_t beg = 0, end = 0;
    if (active) {
      beg = rp[grp];
      end = rp[grp + 1];
    }
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    gather_list<float, Q, 1>(reinterpret_cast<const uint4*>(w_cur), reinterpret_cast<const int32_t*>(sl + L::off_col) +
                                                                         (beg - ea),
                             static_cast<int>(end - beg), 0, ch, acc);
    if (active) {
      const float4 own = *reinterpret_cast<const float4*>(sl + L::off_own + (grp * Q + ch) * 16);
      const float dd = static_cast<float>(end - beg);
      float4 v = make_float4(acc[0], acc[1], acc[2], acc[3]);
      float wd = 1.0f;
      if (op == kLzH) {
        const float sc = 1.0f / dd;
        v = make_float4(acc[0] * sc, acc[1] * sc, acc[2] * sc, acc[3] * sc);
        wd = dd;
      } else if (op == kLzL) {
        v = make_float4(dd * own.x - acc[0], dd * own.y - acc[1], dd * own.z - acc[2], dd * own.w - acc[3]);
      }
      const float4 out = make_float4(v.x * ib.x, v.y * ib.y, v.z * ib.z, v.w * ib.w);
      reinterpret_cast<float4*>(y + static_cast<size_t>(r0 + grp) * nzp)[ch] = out;
      a0 += static_cast<double>(wd * (own.x * ib.x) * out.x);
      a1 += static_cast<double>(wd * (own.y * ib.y) * out.y);
      a2 += static_cast<double>(wd * (own.z * ib.z) * out.z);
      a3 += static_cast<double>(wd * (own.w * ib.w) * out.w);
    }
    __syncwarp();
  }
  cp_async_wait<0>();
  // sum over the R row groups of the warp, then over the warps
#pragma unroll
  for (int o = Q; o < 32; o <<= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    a3 += __shfl_xor_sync(0xffffffffu, a3, o);
  }
  if (grp == 0) {
    red[warp][4 * ch + 0] = a0;
    red[warp][4 * ch + 1] = a1;
    red[warp][4 * ch + 2] = a2;
    red[warp][4 * ch + 3] = a3;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < 4 * Q; p += kLzThreads) {
    double sum = 0.0;
    for (int w = 0; w < kLzWarps; ++w) sum += red[w][p];
    part[static_cast<size_t>(blockIdx.x) * nzp + p] = sum;
  }
}

// apply, heavy rows [0, n_heavy): a CTA per row, the warps take interleaved
// batches of 32 neighbours; the warps' sums are added in warp order.
// Partials of row r go to part[r].
template <int Q>
__global__ void __launch_bounds__(kLzThreads) k_lz_apply_heavy(int op, const int64_t* __restrict__ row_ptr,
                                                               const int32_t* __restrict__ col,
                                                               const int32_t* __restrict__ deg, int nzp,
                                                               const float* __restrict__ w_cur,
                                                               const float* __restrict__ inv_b, float* __restrict__ y,
                                                               double* __restrict__ part) {
  __shared__ float4 wsum[kLzWarps][Q];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / Q, ch = lane % Q;
  const int64_t i = blockIdx.x;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  lz_gather<Q>(col, w_cur, nzp, row_ptr[i] + 32 * warp, row_ptr[i + 1], 32 * kLzWarps, lane, slot, ch, acc);
#pragma unroll
  for (int o = Q; o < 32; o <<= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
    acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
  }
  if (slot == 0) wsum[warp][ch] = acc;
  __syncthreads();
  if (warp == 0 && slot == 0) {
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int w = 0; w < kLzWarps; ++w) {
      t.x += wsum[w][ch].x;
      t.y += wsum[w][ch].y;
      t.z += wsum[w][ch].z;
      t.w += wsum[w][ch].w;
    }
    const float4 ib = reinterpret_cast<const float4*>(inv_b)[ch];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    lz_row_out(op, i, static_cast<float>(deg[i]), t, ib, nzp, ch, w_cur, y, a0, a1, a2, a3);
    double* o = part + static_cast<size_t>(i) * nzp + 4 * ch;
    o[0] = a0;
    o[1] = a1;
    o[2] = a2;
    o[3] = a3;
  }
}

// update: W_{k+1} = Y - c1 W_k - c2 W_{k-1} over W_{k-1}, ||w||^2 partials
// (weights d_i for H, 1 for A and D - A).
// Thread t handles chunk t % Q of rows t / Q, t / Q + stride, ...
template <int Q>
__global__ void __launch_bounds__(kLzThreads) k_lz_update(int op, const int32_t* __restrict__ deg, int64_t n, int nzp,
                                                          const float* __restrict__ y, const float* __restrict__ w_cur,
                                                          float* __restrict__ w_pn, const float* __restrict__ c1,
                                                          const float* __restrict__ c2, double* __restrict__ part) {
  constexpr int RPB = kLzThreads / Q;  // rows per block pass
  __shared__ double red[RPB][4 * Q];
  const int ch = threadIdx.x % Q, r = threadIdx.x / Q;
  const float4 a = reinterpret_cast<const float4*>(c1)[ch];
  const float4 b = reinterpret_cast<const float4*>(c2)[ch];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * RPB + r; i < n; i += static_cast<int64_t>(gridDim.x) * RPB) {
    const size_t off = static_cast<size_t>(i) * nzp;
    const float4 yy = reinterpret_cast<const float4*>(y + off)[ch];
    const float4 wc = reinterpret_cast<const float4*>(w_cur + off)[ch];
    float4* pn = reinterpret_cast<float4*>(w_pn + off) + ch;
    const float4 wp = *pn;
    const float4 o = make_float4(yy.x - a.x * wc.x - b.x * wp.x, yy.y - a.y * wc.y - b.y * wp.y,
                                 yy.z - a.z * wc.z - b.z * wp.z, yy.w - a.w * wc.w - b.w * wp.w);
    *pn = o;
    const float dd = op == kLzH ? static_cast<float>(deg[i]) : 1.0f;
    s0 += static_cast<double>(dd * o.x * o.x);
    s1 += static_cast<double>(dd * o.y * o.y);
    s2 += static_cast<double>(dd * o.z * o.z);
    s3 += static_cast<double>(dd * o.w * o.w);
  }
  red[r][4 * ch + 0] = s0;
  red[r][4 * ch + 1] = s1;
  red[r][4 * ch + 2] = s2;
  red[r][4 * ch + 3] = s3;
  __syncthreads();
  for (int p = threadIdx.x; p < 4 * Q; p += kLzThreads) {
    double s = 0.0;
    for (int rr = 0; rr < RPB; ++rr) s += red[rr][p];
    part[static_cast<size_t>(blockIdx.x) * nzp + p] = s;
  }
}

// sum over CTAs of one probe's partials: a warp per probe, lanes over CTAs,
// then a fixed shuffle tree (deterministic)
__device__ __forceinline__ double warp_sum_partials(const double* part, int grid, int nzp, int p, int lane) {
  double a = 0.0;
  for (int c = lane; c < grid; c += 32) a += part[static_cast<size_t>(c) * nzp + p];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}

// alpha_k = sum of the apply partials; coefficients of the update.  Grid:
// one 32-thread block per padded probe.
__global__ void k_lz_alpha(int nz, int nzp, int m, int k, int grid, LanczosState st) {
  const int p = blockIdx.x, lane = threadIdx.x;
  const double a = warp_sum_partials(st.part, grid, nzp, p, lane);
  if (lane != 0) return;
  if (p >= nz) {
    st.c1[p] = 0.f;
    st.c2[p] = 0.f;
    return;
  }
  const bool live = st.inv_b[p] != 0.f;
  if (live) st.alpha[static_cast<size_t>(p) * m + k] = a;
  st.c1[p] = live ? static_cast<float>(a / st.b_prev[p]) : 0.f;
  st.c2[p] = live && k > 0 ? static_cast<float>(st.b_prev[p] / st.b_prev2[p]) : 0.f;
}

// beta_k = ||w_{k+1}||; stop a probe whose Krylov space is exhausted
__global__ void k_lz_beta(int nz, int nzp, int m, int k, int grid, double stop, LanczosState st) {
  const int p = blockIdx.x, lane = threadIdx.x;
  if (p >= nz) return;
  const double s = warp_sum_partials(st.part, grid, nzp, p, lane);
  if (lane != 0 || st.inv_b[p] == 0.f) return;  // stopped earlier
  const double b = sqrt(s);
  st.beta[static_cast<size_t>(p) * m + k] = b;
  st.steps[p] = k + 1;
  st.b_prev2[p] = st.b_prev[p];
  st.b_prev[p] = b;
  st.inv_b[p] = b > stop ? static_cast<float>(1.0 / b) : 0.f;
}

// ---- the Gauss rule of each probe ---------------------------------------------
// Number of eigenvalues of tridiag(b; a; b) (size k) below x (Sturm sequence).
__device__ int sturm_below(const double* a, const double* b, int k, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int j = 0; j < k; ++j) {
    const double off = j > 0 ? b[j - 1] * b[j - 1] : 0.0;
    q = (a[j] - x) - (j > 0 ? off / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// eigenvalue i (ascending) of tridiag(b; a; b) of size k by bisection of the
// Sturm count, from the Gershgorin interval of the tridiagonal
__device__ double tridiag_eig(const double* a, const double* b, int k, int i) {
  double lo = a[0], hi = a[0];
  for (int j = 0; j < k; ++j) {
    const double r = (j > 0 ? fabs(b[j - 1]) : 0.0) + (j + 1 < k ? fabs(b[j]) : 0.0);
    lo = fmin(lo, a[j] - r);
    hi = fmax(hi, a[j] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * fmax(1.0, fabs(lo) + fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_below(a, b, k, mid) > i) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// one thread per (probe, node index i): node i by bisection (the point where
// the Sturm count passes i), its weight by the Christoffel number
// w_i = 1 / sum_j p_j(tau_i)^2 of the orthonormal polynomials of the rule
// (p_0 = 1, b_j p_{j+1} = (x - a_j) p_j - b_{j-1} p_{j-1}); slots past the
// probe's steps get node and weight 0
__global__ void k_gauss_rules(const double* __restrict__ alpha, const double* __restrict__ beta,
                              const int32_t* __restrict__ steps, int m, int nz, double* __restrict__ nodes,
                              double* __restrict__ weights) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= static_cast<int64_t>(nz) * m) return;
  const int p = static_cast<int>(t / m), i = static_cast<int>(t % m);
  const double* a = alpha + static_cast<size_t>(p) * m;
  const double* b = beta + static_cast<size_t>(p) * m;
  const int k = min(steps[p], m);
  if (i >= k) {
    nodes[t] = 0.0;
    weights[t] = 0.0;
    return;
  }
  const double x = tridiag_eig(a, b, k, i);
  double p_prev = 0.0, p_cur = 1.0, sum = 1.0;
  for (int j = 0; j + 1 < k; ++j) {
    const double nxt = ((x - a[j]) * p_cur - (j > 0 ? b[j - 1] * p_prev : 0.0)) / b[j];
    p_prev = p_cur;
    p_cur = nxt;
    sum += p_cur * p_cur;
  }
  nodes[t] = x;
  weights[t] = 1.0 / sum;
}

// extreme Ritz values of each probe widened by r: out[2p] = theta_min - r,
// out[2p + 1] = theta_max + r (one thread per (probe, end)), with
// r = beta_k (ritz = 0) or the Ritz pair's residual r = beta_k |s_k| (ritz =
// 1), s the unit eigenvector of the tridiagonal for theta.  Its components
// come from the three-term recurrence run backwards from s_k = 1,
//     b_{j-1} s_{j-1} = (theta - a_j) s_j - b_j s_{j+1},
// then |s_k| = 1 / ||s||: an extreme eigenvector decays toward its last
// component, which the backward direction computes stably (the forward one
// amplifies the rounding of theta into the tail).
__global__ void k_ritz_bounds(const double* __restrict__ alpha, const double* __restrict__ beta,
                              const int32_t* __restrict__ steps, int m, int nz, int ritz, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nz) return;
  const int p = t >> 1, end = t & 1;
  const double* a = alpha + static_cast<size_t>(p) * m;
  const double* b = beta + static_cast<size_t>(p) * m;
  const int k = min(max(steps[p], 1), m);
  const double theta = tridiag_eig(a, b, k, end ? k - 1 : 0);
  double r = fabs(b[k - 1]);
  if (ritz) {
    double s_next = 0.0, s_cur = 1.0, sum = 1.0;
    for (int j = k - 1; j > 0; --j) {
      const double prev = ((theta - a[j]) * s_cur - (j + 1 < k ? b[j] * s_next : 0.0)) / b[j - 1];
      s_next = s_cur;
      s_cur = prev;
      sum += s_cur * s_cur;
    }
    r /= sqrt(sum);
  }
  out[t] = end ? theta + r : theta - r;
}

// Chebyshev moments of the averaged rules, d_m = (1/nz) sum_p e_1^T T_m(G_p) e_1,
// by the Chebyshev recurrence on the tridiagonal G_p applied to e_1 (one
// thread per probe, per-probe results summed in probe order by k_sum_probes)
__global__ void k_gql_moments(const double* __restrict__ alpha, const double* __restrict__ beta,
                              const int32_t* __restrict__ steps, int m, int nz, int mc, double* __restrict__ scratch,
                              double* __restrict__ per_probe) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nz) return;
  const double* a = alpha + static_cast<size_t>(p) * m;
  const double* b = beta + static_cast<size_t>(p) * m;
  const int k = min(max(steps[p], 1), m);
  double* t_prev = scratch + static_cast<size_t>(p) * 2 * m;
  double* t_cur = t_prev + m;
  for (int j = 0; j < k; ++j) {
    t_prev[j] = 0.0;
    t_cur[j] = 0.0;
  }
  t_prev[0] = 1.0;  // T_0 e_1
  double* out = per_probe + static_cast<size_t>(p) * mc;
  out[0] = 1.0;
  if (mc > 1) {
    // T_1 e_1 = G e_1
    t_cur[0] = a[0];
    if (k > 1) t_cur[1] = b[0];
    out[1] = t_cur[0];
  }
  for (int mm = 2; mm < mc; ++mm) {
    // t_next = 2 G t_cur - t_prev, written over t_prev
    const int top = mm < k ? mm : k - 1;  // support of T_mm e_1
    for (int j = 0; j <= top; ++j) {
      const double gj =
          a[j] * t_cur[j] + (j > 0 ? b[j - 1] * t_cur[j - 1] : 0.0) + (j + 1 < k ? b[j] * t_cur[j + 1] : 0.0);
      t_prev[j] = 2.0 * gj - t_prev[j];
    }
    double* tmp = t_prev;
    t_prev = t_cur;
    t_cur = tmp;
    out[mm] = t_cur[0];
  }
}

__global__ void k_sum_probes(const double* __restrict__ per_probe, int nz, int mc, double* __restrict__ d) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= mc) return;
  double s = 0.0;
  for (int p = 0; p < nz; ++p) s += per_probe[static_cast<size_t>(p) * mc + m];
  d[m] = s / nz;
}

// histogram of the averaged rules' point masses: bin b sums, in node order,
// weight / nz of every node in it (a node within 1e-9 of an interior edge
// splits evenly, nodes at or beyond +-1 go to the end bins)
__global__ void k_gql_hist(const double* __restrict__ nodes, const double* __restrict__ weights, int64_t count,
                           int nz, int B, double* __restrict__ h) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double w = 2.0 / B;
  double v = 0.0;
  for (int64_t q = 0; q < count; ++q) {
    const double wt = weights[q];
    if (wt == 0.0) continue;
    const double x = fmin(fmax(nodes[q], -1.0), 1.0);
    const int e = static_cast<int>(rint((x + 1.0) / w));
    if (e > 0 && e < B && fabs(x - (-1.0 + w * e)) <= 1e-9) {
      if (b == e - 1 || b == e) v += 0.5 * wt;
    } else {
      int bb = static_cast<int>(floor((x + 1.0) / w));
      bb = bb < 0 ? 0 : (bb >= B ? B - 1 : bb);
      if (b == bb) v += wt;
    }
  }
  h[b] = v / nz;
}

inline unsigned blocks_for(int64_t work, int per = 256) {
  int64_t b = (work + per - 1) / per;
  const int64_t cap = static_cast<int64_t>(num_sms()) * 16;
  return static_cast<unsigned>(std::max<int64_t>(1, std::min(b, cap)));
}

template <int Q>
int lanczos_steps(const Graph* G, int op, int m, int nz, int nzp, float* w_cur, float* w_pn, float* y,
                  LanczosState st, int grid, double stop, cudaStream_t s) {
  const unsigned gp = static_cast<unsigned>(nzp);  // a warp per padded probe
  // light rows go through the staged kernel when a round has at most 16 rows
  // (Q >= 2); with one chunk per row its staging would not fit in shared memory
  const int64_t nh = G->n_heavy, nm = Q >= 2 ? G->n_mid : G->n;
  // apply partials: medium-row CTAs [0, grid), light-row CTAs [grid, 2 grid), heavy rows after
  const int parts = 2 * grid + static_cast<int>(nh);
  const int smem = kLzWarps * LzRound<Q>::WARP + 128;
  static int s_attr[64] = {};  // the shared-memory limit, raised once per device
  NDOS_CHECK(raise_smem_limit(reinterpret_cast<const void*>(k_lz_apply_light<Q>), s_attr, smem));
  for (int k = 0; k < m; ++k) {
    if (nh > 0) {
      k_lz_apply_heavy<Q><<<static_cast<unsigned>(nh), kLzThreads, 0, s>>>(
          op, G->p_row_ptr, G->p_col, G->p_deg, nzp, w_cur, st.inv_b, y,
          st.part + static_cast<size_t>(2 * grid) * nzp);
      NDOS_LAUNCHED();
    }
    k_lz_apply<Q><<<grid, kLzThreads, 0, s>>>(op, G->p_row_ptr, G->p_col, G->p_deg, nh, nm, nzp, w_cur, st.inv_b, y,
                                             st.part);
    NDOS_LAUNCHED();
    if (nm < G->n) {
      k_lz_apply_light<Q><<<grid, kLzThreads, smem, s>>>(op, G->p_row_ptr, G->p_col, nm, G->n, nzp, w_cur, st.inv_b,
                                                         y, st.part + static_cast<size_t>(grid) * nzp);
      NDOS_LAUNCHED();
    } else {
      NDOS_CUDA(cudaMemsetAsync(st.part + static_cast<size_t>(grid) * nzp, 0, sizeof(double) * grid * nzp, s));
    }
    k_lz_alpha<<<gp, 32, 0, s>>>(nz, nzp, m, k, parts, st);
    NDOS_LAUNCHED();
    k_lz_update<Q><<<grid, kLzThreads, 0, s>>>(op, G->p_deg, G->n, nzp, y, w_cur, w_pn, st.c1, st.c2, st.part);
    NDOS_LAUNCHED();
    k_lz_beta<<<gp, 32, 0, s>>>(nz, nzp, m, k, grid, stop, st);
    NDOS_LAUNCHED();
    std::swap(w_cur, w_pn);
  }
  return DOS_OK;
}

}  // namespace
}  // namespace netdos

using namespace netdos;

namespace netdos {
namespace {

// M Lanczos steps of operator op (kLzH, kLzA, kLzL) from Nz probes into
// alpha / beta / steps (device)
int run_lanczos(const Graph* G, int op, int M, int Nz, uint64_t seed, double* alpha_out, double* beta_out,
                int32_t* steps_out, cudaStream_t s) {
  // chunks per row: a power of two >= Nz / 4
  int q = 1;
  while (4 * q < Nz) q *= 2;
  const int nzp = 4 * q;
  const int64_t n = G->n;
  const int grid = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(num_sms()) * 8,
                                                      std::max<int64_t>(1, (n + kLzWarps - 1) / kLzWarps)));
  Temps t(s);
  float *w_cur = nullptr, *w_pn = nullptr, *y = nullptr, *fl = nullptr;
  double *dbl = nullptr, *part = nullptr;
  NDOS_CHECK(t.get(&w_cur, n * nzp));
  NDOS_CHECK(t.get(&w_pn, n * nzp));
  NDOS_CHECK(t.get(&y, n * nzp));
  NDOS_CHECK(t.get(&fl, 3 * nzp));
  NDOS_CHECK(t.get(&dbl, 2 * nzp));
  NDOS_CHECK(t.get(&part, (2 * static_cast<int64_t>(grid) + G->n_heavy) * nzp));
  LanczosState st{alpha_out, beta_out, steps_out, dbl, dbl + nzp, fl, fl + nzp, fl + 2 * nzp, part};
  NDOS_CUDA(cudaMemsetAsync(alpha_out, 0, sizeof(double) * Nz * M, s));
  NDOS_CUDA(cudaMemsetAsync(beta_out, 0, sizeof(double) * Nz * M, s));
  k_lz_init<<<blocks_for(n * nzp), 256, 0, s>>>(G->p_orig, G->p_compact, G->s32, op, n, Nz, nzp, seed, w_cur, w_pn);
  NDOS_LAUNCHED();
  const double norm0 = std::sqrt(static_cast<double>(n));  // ||z||^2 = N for +-1 probes
  k_lz_state0<<<(nzp + 127) / 128, 128, 0, s>>>(Nz, nzp, norm0, st);
  NDOS_LAUNCHED();
  // FP32 vectors: a residual below 1e-5 ||X|| is rounding noise
  const double x_norm = op == kLzH ? 1.0 : (op == kLzA ? 1.0 : 2.0) * G->max_deg;
  const double stop = 1e-5 * x_norm;
  int st_code = DOS_OK;
  switch (q) {
    case 1: st_code = lanczos_steps<1>(G, op, M, Nz, nzp, w_cur, w_pn, y, st, grid, stop, s); break;
    case 2: st_code = lanczos_steps<2>(G, op, M, Nz, nzp, w_cur, w_pn, y, st, grid, stop, s); break;
    case 4: st_code = lanczos_steps<4>(G, op, M, Nz, nzp, w_cur, w_pn, y, st, grid, stop, s); break;
    case 8: st_code = lanczos_steps<8>(G, op, M, Nz, nzp, w_cur, w_pn, y, st, grid, stop, s); break;
    case 16: st_code = lanczos_steps<16>(G, op, M, Nz, nzp, w_cur, w_pn, y, st, grid, stop, s); break;
    default: st_code = lanczos_steps<32>(G, op, M, Nz, nzp, w_cur, w_pn, y, st, grid, stop, s); break;
  }
  return st_code;
}

int lanczos_args(const char* who, dos_graph_t g, int M, int Nz, const void* a, const void* b, const void* st) {
  if (!g || !a || !b || !st) return fail(DOS_EINVAL, std::string(who) + ": null argument");
  if (reinterpret_cast<const Graph*>(g)->n == 0) return fail(DOS_EINVAL, std::string(who) + ": graph has no edges");
  if (M < 1 || M > 4096) return fail(DOS_EINVAL, std::string(who) + ": M must be in [1, 4096]");
  if (Nz < 1 || Nz > 128) return fail(DOS_EINVAL, std::string(who) + ": Nz must be in [1, 128]");
  return DOS_OK;
}

}  // namespace
}  // namespace netdos

extern "C" int dos_lanczos(dos_graph_t g, int M, int Nz, uint64_t seed, double* alpha_out, double* beta_out,
                           int32_t* steps_out, void* stream) {
  clear_error();
  NDOS_CHECK(lanczos_args("dos_lanczos", g, M, Nz, alpha_out, beta_out, steps_out));
  return run_lanczos(reinterpret_cast<const Graph*>(g), kLzH, M, Nz, seed, alpha_out, beta_out, steps_out,
                     static_cast<cudaStream_t>(stream));
}

extern "C" int dos_lanczos_op(dos_graph_t g, int op, int M, int Nz, uint64_t seed, double* alpha_out,
                              double* beta_out, int32_t* steps_out, void* stream) {
  clear_error();
  NDOS_CHECK(lanczos_args("dos_lanczos_op", g, M, Nz, alpha_out, beta_out, steps_out));
  int lz = 0;
  switch (op) {
    case DOS_OP_NORMALIZED_ADJACENCY: lz = kLzH; break;
    case DOS_OP_ADJACENCY: lz = kLzA; break;
    case DOS_OP_LAPLACIAN: lz = kLzL; break;
    default: return fail(DOS_EINVAL, "dos_lanczos_op: operator must be H, A or D - A");
  }
  return run_lanczos(reinterpret_cast<const Graph*>(g), lz, M, Nz, seed, alpha_out, beta_out, steps_out,
                     static_cast<cudaStream_t>(stream));
}

extern "C" int dos_ritz_bounds(const double* alpha, const double* beta, const int32_t* steps, int M, int Nz,
                               int bound, double* bounds_out, void* stream) {
  clear_error();
  if (!alpha || !beta || !steps || !bounds_out || M < 1 || Nz < 1)
    return fail(DOS_EINVAL, "dos_ritz_bounds: bad argument");
  if (bound != DOS_BOUND_RESIDUAL && bound != DOS_BOUND_RITZ)
    return fail(DOS_EINVAL, "dos_ritz_bounds: bound must be DOS_BOUND_RESIDUAL or DOS_BOUND_RITZ");
  k_ritz_bounds<<<(2 * Nz + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(
      alpha, beta, steps, M, Nz, bound == DOS_BOUND_RITZ, bounds_out);
  NDOS_LAUNCHED();
  return DOS_OK;
}

extern "C" int dos_spectral_interval(dos_graph_t g, int op, int M, int Nz, uint64_t seed, int bound, double pad,
                                     double* interval_out, void* stream) {
  clear_error();
  if (!g || !interval_out) return fail(DOS_EINVAL, "dos_spectral_interval: null argument");
  if (bound != DOS_BOUND_RESIDUAL && bound != DOS_BOUND_RITZ)
    return fail(DOS_EINVAL, "dos_spectral_interval: bound must be DOS_BOUND_RESIDUAL or DOS_BOUND_RITZ");
  if (!(pad >= 0.0 && pad <= 1.0)) return fail(DOS_EINVAL, "dos_spectral_interval: pad must be in [0, 1]");
  const Graph* G = reinterpret_cast<const Graph*>(g);
  if (G->n == 0) return fail(DOS_EINVAL, "dos_spectral_interval: graph has no edges");
  if (M < 1 || M > 4096) return fail(DOS_EINVAL, "dos_spectral_interval: M must be in [1, 4096]");
  if (Nz < 1 || Nz > 128) return fail(DOS_EINVAL, "dos_spectral_interval: Nz must be in [1, 128]");
  // the Lanczos operator and the Gershgorin interval; an end that is an
  // eigenvalue of every graph with an edge is taken exactly
  int lz = kLzH;
  double g_lo = -1.0, g_hi = 1.0;
  bool exact_lo = false, exact_hi = false;
  const double dmax = static_cast<double>(G->max_deg);
  switch (op) {
    case DOS_OP_NORMALIZED_ADJACENCY: exact_hi = true; break;  // lambda_max(H) = 1
    case DOS_OP_NORMALIZED_LAPLACIAN: g_lo = 0.0; g_hi = 2.0; exact_lo = true; break;  // from H: 1 - [lo, hi]
    case DOS_OP_ADJACENCY: lz = kLzA; g_lo = -dmax; g_hi = dmax; break;
    case DOS_OP_LAPLACIAN: lz = kLzL; g_lo = 0.0; g_hi = 2.0 * dmax; exact_lo = true; break;  // lambda_min = 0
    default: return fail(DOS_EINVAL, "dos_spectral_interval: unknown operator");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Temps t(s);
  double *alpha = nullptr, *beta = nullptr, *bounds = nullptr;
  int32_t* steps = nullptr;
  NDOS_CHECK(t.get(&alpha, static_cast<int64_t>(Nz) * M));
  NDOS_CHECK(t.get(&beta, static_cast<int64_t>(Nz) * M));
  NDOS_CHECK(t.get(&steps, Nz));
  NDOS_CHECK(t.get(&bounds, 2 * Nz));
  NDOS_CHECK(run_lanczos(G, lz, M, Nz, seed, alpha, beta, steps, s));
  NDOS_CHECK(dos_ritz_bounds(alpha, beta, steps, M, Nz, bound, bounds, s));
  std::vector<double> h(2 * Nz);
  NDOS_CUDA(cudaMemcpyAsync(h.data(), bounds, sizeof(double) * 2 * Nz, cudaMemcpyDeviceToHost, s));
  NDOS_CUDA(cudaStreamSynchronize(s));
  double lo = h[0], hi = h[1];
  for (int p = 1; p < Nz; ++p) {
    lo = std::min(lo, h[2 * p]);
    hi = std::max(hi, h[2 * p + 1]);
  }
  if (op == DOS_OP_NORMALIZED_LAPLACIAN) {  // spectrum of I - H = 1 - spectrum of H
    const double l = 1.0 - hi, u = 1.0 - lo;
    lo = l;
    hi = u;
  }
  const double w = hi - lo;
  lo -= pad * w;
  hi += pad * w;
  if (exact_lo) lo = g_lo;
  if (exact_hi) hi = g_hi;
  interval_out[0] = std::max(lo, g_lo);
  interval_out[1] = std::min(hi, g_hi);
  return DOS_OK;
}

extern "C" int dos_gauss_rules(const double* alpha, const double* beta, const int32_t* steps, int M, int Nz,
                               double* nodes_out, double* weights_out, void* stream) {
  clear_error();
  if (!alpha || !beta || !steps || !nodes_out || !weights_out || M < 1 || Nz < 1)
    return fail(DOS_EINVAL, "dos_gauss_rules: bad argument");
  const int64_t work = static_cast<int64_t>(Nz) * M;
  k_gauss_rules<<<static_cast<unsigned>((work + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
      alpha, beta, steps, M, Nz, nodes_out, weights_out);
  NDOS_LAUNCHED();
  return DOS_OK;
}

extern "C" int dos_gql_moments(const double* alpha, const double* beta, const int32_t* steps, int M, int Nz,
                               int m_count, double* d_out, void* stream) {
  clear_error();
  if (!alpha || !beta || !steps || !d_out || M < 1 || Nz < 1 || m_count < 1 || m_count > (1 << 20))
    return fail(DOS_EINVAL, "dos_gql_moments: bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Temps t(s);
  double *scratch = nullptr, *per = nullptr;
  NDOS_CHECK(t.get(&scratch, static_cast<int64_t>(Nz) * 2 * M));
  NDOS_CHECK(t.get(&per, static_cast<int64_t>(Nz) * m_count));
  k_gql_moments<<<(Nz + 63) / 64, 64, 0, s>>>(alpha, beta, steps, M, Nz, m_count, scratch, per);
  NDOS_LAUNCHED();
  k_sum_probes<<<(m_count + 127) / 128, 128, 0, s>>>(per, Nz, m_count, d_out);
  NDOS_LAUNCHED();
  return DOS_OK;
}

extern "C" int dos_gql_histogram(const double* nodes, const double* weights, int M, int Nz, int n_bins,
                                 double* hist_out, void* stream) {
  clear_error();
  if (!nodes || !weights || !hist_out || M < 1 || Nz < 1 || n_bins < 1 || n_bins > (1 << 20))
    return fail(DOS_EINVAL, "dos_gql_histogram: bad argument");
  k_gql_hist<<<(n_bins + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(
      nodes, weights, static_cast<int64_t>(M) * Nz, Nz, n_bins, hist_out);
  NDOS_LAUNCHED();
  return DOS_OK;
}
