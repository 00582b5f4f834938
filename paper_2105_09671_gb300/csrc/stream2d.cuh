// 2D streaming stencil with temporal blocking.
//
// Advances k explicit Euler steps of Eq. (pytorchACeq) per pass over HBM.
// Work unit: one warp owns a strip of SW = 32 * E columns (E cells per lane,
// 16-byte vectors) and a chunk of rows, and streams the rows in increasing y:
//   - rows of the input field arrive through a per-warp ring of shared-memory
//     stages filled by TMA tile loads (box SW x kRows, zero fill outside the
//     domain), signalled on one mbarrier per stage;
//   - time level l keeps its last three rows in registers; level l+1 of row
//     R is formed as soon as level l of row R+1 exists (a lag of one row per
//     level), so k levels are in flight at once and only level k is written;
//   - x neighbours come from the adjacent lane by warp shuffle, y neighbours
//     from the register rows;
//   - the zero-Neumann ghost of Section 2 is the clamp "neighbour outside
//     the domain = the boundary cell itself" at the current level: at
//     x = 0, nx-1 one select per vector when nx is a multiple of the vector
//     width (FASTX), else per element in strips that touch those faces; at
//     y = 0, ny-1 by copying the boundary row into the ghost slot, only in
//     the few row groups that touch them (a separate instantiation of the
//     loop body);
//   - each level invalidates one more column at the strip edges, so strips
//     overlap by a halo of HX >= k columns per side and write only their
//     interior (out_w = SW - 2 HX columns); chunks read k extra rows at each
//     end and write only their own rows.
#pragma once

#include <algorithm>

#include "kernels.h"

namespace ac {

constexpr int kS2Warps = 8;   // warps per CTA (independent strips)
constexpr int kS2Stages = 6;  // ring depth per warp
constexpr int kS2Rows = 2;    // rows per TMA box
constexpr int kS2Tiles = 2;   // strip widths (tile 0: S2Cfg::VPL vectors per lane, tile 1: two)

// VPL = 16-byte vectors per lane (tile 0).  FP32 also offers strips twice
// as wide (tile 1: two vectors, 8 cells per lane: half the shuffles and
// x-face selects per cell and half the strip-halo share, for more
// registers; depths up to KMAX_WIDE).
template <typename T> struct S2Cfg;
template <> struct S2Cfg<float> { static constexpr int VPL = 1, KMAX = 8, KMAX_WIDE = 6; };
template <> struct S2Cfg<double> { static constexpr int VPL = 2, KMAX = 8, KMAX_WIDE = 0; };
template <> struct S2Cfg<__half> { static constexpr int VPL = 1, KMAX = 6, KMAX_WIDE = 0; };

template <typename T, int K, int VPL_ = S2Cfg<T>::VPL>
struct S2Geom {
  static constexpr int V = Traits<T>::V;
  static constexpr int VPL = VPL_;
  static constexpr int E = V * VPL;                 // cells per lane
  static constexpr int SW = 32 * E;                 // strip width (cells)
  static constexpr int HX = V * ((K + V - 1) / V);  // halo per side, vector aligned
  static constexpr int OW = SW - 2 * HX;            // output columns per strip
  static constexpr int STAGE_ELEMS = SW * kS2Rows;
  static constexpr int RING_BYTES = kS2Stages * STAGE_ELEMS * (int)sizeof(T);
  static constexpr int SMEM = kS2Warps * (RING_BYTES + kS2Stages * 8);
};

// One strip item: the columns [xs, xs + SW) of rows [y0, y1) advanced by K
// steps, written for the columns [xs + hx, xs + SW - hx) of [y0, y1).
struct S2Item {
  int xs, y0, y1, hx;
  int nx, ny;
  int64_t pitch;
};

// Processes one item on the calling warp.  ring_smem / bars are the warp's
// TMA ring (mbarriers already initialised); u counts the ring groups this
// warp has consumed so far (stage u % D, phase (u / D) & 1) and is advanced
// past this item.  Returns false if a bounded wait expired (the status word
// is set and every copy this item issued has landed).
template <typename T, int K, bool FASTX, int VPL_ = S2Cfg<T>::VPL>
__device__ __forceinline__ bool s2_item(T *ring_smem, uint64_t *bars, uint32_t &u,
                                        const CUtensorMap *src_map, T *__restrict__ dst,
                                        const S2Item &it, typename Traits<T>::C alpha,
                                        typename Traits<T>::C beta, int *status) {
  using Gm = S2Geom<T, K, VPL_>;
  using C = typename Traits<T>::C;
  constexpr int E = Gm::E, V = Gm::V, VPL = Gm::VPL, D = kS2Stages;
  constexpr uint32_t kStageBytes = Gm::STAGE_ELEMS * sizeof(T);
  const int lane = threadIdx.x & 31;
  const int xs = it.xs, nx = it.nx, ny = it.ny, y0 = it.y0, y1 = it.y1;
  const int lo0 = max(0, y0 - K);
  const int hi0 = min(ny, y1 + K);
  const int n_in = hi0 - lo0;
  const int n_groups = (n_in + kS2Rows - 1) / kS2Rows;
  const int n_iter = y1 - lo0 + K;
  const uint32_t u0 = u;

  if (lane == 0) {
    for (int p = 0; p < D && p < n_groups; ++p) {
      const int s = (int)((u0 + p) % D);
      mbar_arrive_expect_tx(&bars[s], kStageBytes);
      tma_load_2d(ring_smem + s * Gm::STAGE_ELEMS, src_map, &bars[s], xs, lo0 + p * kS2Rows);
    }
  }
  __syncwarp();

  const int xl = xs + lane * E;  // column of this lane's first cell
  const int eL = -xl;            // element index holding x == 0 (if in [0, E))
  const int eR = nx - 1 - xl;    // element index holding x == nx-1
  const bool edge = (xs <= 0) || (xs + Gm::SW > nx - 1);
  bool lfix[VPL], rfix[VPL];  // vector v starts at x = 0 / ends at x = nx-1
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    lfix[v] = xl + v * V == 0;
    rfix[v] = xl + v * V + V - 1 == nx - 1;
  }
  const int out_lo = xs + it.hx, out_hi = xs + Gm::SW - it.hx;

  // Level l keeps its last three rows in a ring of register slots: at
  // iteration t slot t%3 holds row R+1 (newest), (t+2)%3 row R and (t+1)%3
  // row R-1 of the stencil that forms level l+1 of row R.  The row loop is
  // unrolled by three so that every slot index is a constant.
  C ring[K][3][E];
#pragma unroll
  for (int l = 0; l < K; ++l)
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int e = 0; e < E; ++e) ring[l][s][e] = C(0);

  auto body = [&]<int P, bool BND>(int t) -> bool {
    constexpr int SN = P, SB = (P + 2) % 3, SA = (P + 1) % 3;
    const int grp = t / kS2Rows;
    const int rr = t - grp * kS2Rows;
    const int stg = (int)((u0 + grp) % D);
    if (!BND || t < n_in) {
      if (rr == 0) {
        const bool ok = mbar_wait_bounded(&bars[stg], ((u0 + grp) / D) & 1u);
        if (!__all_sync(0xffffffffu, ok)) {
          // give up: record it, let every issued copy land, then leave
          if (lane == 0) {
            report_timeout(status);
            for (int q = grp + 1; q < n_groups && q < grp + D; ++q)
              mbar_wait_bounded(&bars[(u0 + q) % D], ((u0 + q) / D) & 1u);
          }
          __syncwarp();
          return false;
        }
      }
      const T *src = ring_smem + stg * Gm::STAGE_ELEMS + rr * Gm::SW + lane * E;
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const uint4 w = *reinterpret_cast<const uint4 *>(src + v * V);
        unpack16<T>(w, ring[0][SN] + v * V);
      }
    }

#pragma unroll
    for (int l = 0; l < K; ++l) {
      const int R = lo0 + t - (l + 1);  // row of level l+1 formed now
      // zero-Neumann ghosts: below row 0 and above row ny-1 the neighbour is
      // the boundary row itself (these slots are dead after this row)
      if constexpr (BND) {
        if (R == 0) {
#pragma unroll
          for (int e = 0; e < E; ++e) ring[l][SA][e] = ring[l][SB][e];
        }
        if (R == ny - 1) {
#pragma unroll
          for (int e = 0; e < E; ++e) ring[l][SN][e] = ring[l][SB][e];
        }
      }
      const C *mid = ring[l][SB];
      const C left = __shfl_up_sync(0xffffffffu, mid[E - 1], 1);
      const C right = __shfl_down_sync(0xffffffffu, mid[0], 1);
      C out[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const C p = mid[e];
        C w = (e == 0) ? left : mid[e - 1];
        C ea = (e == E - 1) ? right : mid[e + 1];
        if constexpr (FASTX) {
          if (e % V == 0) w = lfix[e / V] ? p : w;
          if (e % V == V - 1) ea = rfix[e / V] ? p : ea;
        } else {
          if (edge) {
            if (e == eL) w = p;
            if (e == eR) ea = p;
          }
        }
        out[e] = ac_update<C>(p, (w + ea) + (ring[l][SA][e] + ring[l][SN][e]), C(-4), alpha, beta);
      }
      if (l + 1 < K) {
#pragma unroll
        for (int e = 0; e < E; ++e) ring[l + 1 < K ? l + 1 : 0][SN][e] = out[e];
      } else {
        const int RK = R;
        if (RK >= y0 && RK < y1) {
          T *drow = dst + (int64_t)RK * it.pitch;
#pragma unroll
          for (int v = 0; v < VPL; ++v) {
            const int xv = xl + v * V;
            if (xv >= out_lo && xv < out_hi && xv < nx) {
              if (xv + V <= nx) {
                *reinterpret_cast<uint4 *>(drow + xv) = pack16<T>(out + v * V);
              } else {
#pragma unroll
                for (int e = 0; e < V; ++e)
                  if (xv + e < nx) drow[xv + e] = from_c<T>(out[v * V + e]);
              }
            }
          }
        }
      }
    }

    // the stage's last row has been consumed (its values used above): refill
    if (t < n_in && (rr == kS2Rows - 1 || t == n_in - 1)) {
      __syncwarp();
      const int nxt = grp + D;
      if (lane == 0 && nxt < n_groups) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bars[stg], kStageBytes);
        tma_load_2d(ring_smem + stg * Gm::STAGE_ELEMS, src_map, &bars[stg], xs, lo0 + nxt * kS2Rows);
      }
    }
    return true;
  };

  // Row groups that touch a y face (ghost copies) or run past the last input
  // row take the BND body: t in [1, K] when the chunk starts at y = 0, and
  // t >= ny - lo0 when it ends at the top face.
  const int bnd_lo_end = (lo0 == 0) ? K : -1;
  const int bnd_hi_begin = (hi0 == ny) ? ny - lo0 - 1 : n_iter;
  int t = 0;
  bool ok = true;
  for (; ok && t + 3 <= n_iter; t += 3) {
    const bool bnd = (t <= bnd_lo_end) || (t + 2 >= bnd_hi_begin);
    if (bnd) {
      ok = body.template operator()<0, true>(t) && body.template operator()<1, true>(t + 1) &&
           body.template operator()<2, true>(t + 2);
    } else {
      ok = body.template operator()<0, false>(t) && body.template operator()<1, false>(t + 1) &&
           body.template operator()<2, false>(t + 2);
    }
  }
  if (ok && t < n_iter) ok = body.template operator()<0, true>(t++);
  if (ok && t < n_iter) ok = body.template operator()<1, true>(t++);
  u = u0 + (uint32_t)n_groups;
  return ok;
}

// Per-warp TMA ring of the calling CTA: D stages and D mbarriers per warp.
template <typename T>
struct S2Ring {
  T *smem;
  uint64_t *bars;
};
template <typename T, int K, int VPL_ = S2Cfg<T>::VPL>
__device__ __forceinline__ S2Ring<T> s2_ring(unsigned char *smem, int warp) {
  using Gm = S2Geom<T, K, VPL_>;
  S2Ring<T> r;
  r.smem = reinterpret_cast<T *>(smem + warp * Gm::RING_BYTES);
  r.bars = reinterpret_cast<uint64_t *>(smem + kS2Warps * Gm::RING_BYTES) + warp * kS2Stages;
  return r;
}

template <typename T, int K, bool FASTX, int VPL_>
__global__ void __launch_bounds__(kS2Warps * 32, 1)
    stream2d_k(const __grid_constant__ CUtensorMap src_map, T *__restrict__ dst, GridParams g,
               int n_strips, int n_chunks, int chunk_rows) {
  using Gm = S2Geom<T, K, VPL_>;
  using C = typename Traits<T>::C;
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const S2Ring<T> ring = s2_ring<T, K, VPL_>(smem, warp);

  const int64_t gw = (int64_t)blockIdx.x * kS2Warps + warp;
  if (gw >= (int64_t)n_strips * n_chunks) return;  // no CTA-wide barrier in this kernel
  const int strip = (int)(gw % n_strips);
  const int chunk = (int)(gw / n_strips);
  S2Item it;
  it.xs = strip * Gm::OW - Gm::HX;  // first column of the strip (may be < 0)
  it.hx = Gm::HX;
  it.nx = (int)g.nx;
  it.ny = (int)g.ny;
  it.y0 = chunk * chunk_rows;
  it.y1 = min(it.ny, it.y0 + chunk_rows);
  it.pitch = g.pitch;

  if (lane == 0) {
    tma_prefetch_desc(&src_map);
    for (int s = 0; s < kS2Stages; ++s) mbar_init(&ring.bars[s], 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t u = 0;
  s2_item<T, K, FASTX, VPL_>(ring.smem, ring.bars, u, &src_map, dst, it, (C)g.alpha, (C)g.beta, g.status);
}

// ------------------------------------------------------------------ host ---

template <typename T, int K, int VPL_>
inline Stream2DGeom s2_geom_t() {
  using Gm = S2Geom<T, K, VPL_>;
  return Stream2DGeom{Gm::SW, kS2Rows, Gm::HX, Gm::OW};
}

template <typename T, int K, bool FASTX, int VPL_>
static cudaError_t s2_launch_t(const GridParams &g, const CUtensorMap *map, void *dst, int num_sms,
                               cudaStream_t s) {
  using Gm = S2Geom<T, K, VPL_>;
  static KernelSetup ks;
  int occ = 1;
  cudaError_t e = kernel_setup(ks, (const void *)stream2d_k<T, K, FASTX, VPL_>, kS2Warps * 32, Gm::SMEM, &occ);
  if (e != cudaSuccess) return e;
  const int n_strips = (int)((g.nx + Gm::OW - 1) / Gm::OW);
  // one wave of resident warps, but chunks of at least max(16, 3k) rows so
  // that the 2k halo rows per chunk stay a modest overhead
  const int64_t target_warps = (int64_t)std::max(1, num_sms) * occ * kS2Warps;
  int n_chunks = (int)std::max<int64_t>(1, target_warps / n_strips);
  const int min_rows = std::max(16, 3 * K);
  n_chunks = std::min<int>(n_chunks, (int)std::max<int64_t>(1, g.ny / min_rows));
  const int chunk_rows = (int)((g.ny + n_chunks - 1) / n_chunks);
  n_chunks = (int)((g.ny + chunk_rows - 1) / chunk_rows);
  const int64_t warps = (int64_t)n_strips * n_chunks;
  const unsigned blocks = (unsigned)((warps + kS2Warps - 1) / kS2Warps);
  stream2d_k<T, K, FASTX, VPL_><<<blocks, kS2Warps * 32, Gm::SMEM, s>>>(*map, (T *)dst, g, n_strips,
                                                                        n_chunks, chunk_rows);
  return cudaGetLastError();
}

// Depths available for a storage type and tile (0: VPL of S2Cfg, 1: twice as wide).
template <typename T>
constexpr int s2_kmax(int tile) {
  return tile == 0 ? S2Cfg<T>::KMAX : tile == 1 ? S2Cfg<T>::KMAX_WIDE : 0;
}

template <typename T, int VPL_>
cudaError_t s2_dispatch(int k, const GridParams &g, const CUtensorMap *map, void *dst, int num_sms,
                        cudaStream_t s) {
  constexpr int KMAX = VPL_ == S2Cfg<T>::VPL ? S2Cfg<T>::KMAX : S2Cfg<T>::KMAX_WIDE;
  const bool fastx = g.nx % Traits<T>::V == 0;
  switch (k) {
#define AC_CASE(KK)                                                                \
  case KK:                                                                         \
    if constexpr (KK <= KMAX)                                                      \
      return fastx ? s2_launch_t<T, KK, true, VPL_>(g, map, dst, num_sms, s)       \
                   : s2_launch_t<T, KK, false, VPL_>(g, map, dst, num_sms, s);     \
    break;
    AC_CASE(1) AC_CASE(2) AC_CASE(3) AC_CASE(4) AC_CASE(5) AC_CASE(6) AC_CASE(7) AC_CASE(8)
#undef AC_CASE
  }
  return cudaErrorInvalidValue;
}

template <typename T, int VPL_>
Stream2DGeom s2_geom(int k) {
  constexpr int KMAX = VPL_ == S2Cfg<T>::VPL ? S2Cfg<T>::KMAX : S2Cfg<T>::KMAX_WIDE;
  switch (k) {
#define AC_CASE(KK) \
  case KK:          \
    if constexpr (KK <= KMAX) return s2_geom_t<T, KK, VPL_>(); \
    break;
    AC_CASE(1) AC_CASE(2) AC_CASE(3) AC_CASE(4) AC_CASE(5) AC_CASE(6) AC_CASE(7) AC_CASE(8)
#undef AC_CASE
  }
  return Stream2DGeom{0, 0, 0, 0};
}

cudaError_t stream2d_launch_f64(int k, const GridParams &g, const CUtensorMap *map, void *dst, int num_sms, cudaStream_t s);
cudaError_t stream2d_launch_f32(int k, const GridParams &g, const CUtensorMap *map, void *dst, int num_sms, cudaStream_t s);
cudaError_t stream2d_launch_f32_wide(int k, const GridParams &g, const CUtensorMap *map, void *dst, int num_sms, cudaStream_t s);
cudaError_t stream2d_launch_f16(int k, const GridParams &g, const CUtensorMap *map, void *dst, int num_sms, cudaStream_t s);

}  // namespace ac
