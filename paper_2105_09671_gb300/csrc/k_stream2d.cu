// 2D streaming stencil with temporal blocking.
//
// Advances k explicit Euler steps of Eq. (pytorchACeq) per pass over HBM.
// Work unit: one warp owns a strip of SW = 32 * E columns (E cells per lane,
// 16-byte vectors) and a chunk of rows, and streams the rows in increasing y:
//   - rows of the input field arrive through a per-warp ring of shared-memory
//     stages filled by TMA tile loads (box SW x kRows, zero fill outside the
//     domain), signalled on one mbarrier per stage;
//   - time level l keeps its last two rows in registers; level l+1 of row R
//     is formed as soon as level l of row R+1 exists (a lag of one row per
//     level), so k levels are in flight at once and only level k is written;
//   - x neighbours come from the adjacent lane by warp shuffle, y neighbours
//     from the register rows;
//   - the zero-Neumann ghost of Section 2 is the clamp "neighbour outside
//     the domain = the boundary cell itself" at the current level, applied
//     per element at x = 0, nx-1 and per row at y = 0, ny-1;
//   - each level invalidates one more column at the strip edges, so strips
//     overlap by a halo of HX >= k columns per side and write only their
//     interior (out_w = SW - 2 HX columns); chunks read k extra rows at each
//     end and write only their own rows.
#include <algorithm>

#include "kernels.h"

namespace ac {

constexpr int kS2Warps = 8;   // warps per CTA (independent strips)
constexpr int kS2Stages = 8;  // ring depth per warp
constexpr int kS2Rows = 2;    // rows per TMA box

template <typename T> struct S2Cfg;
template <> struct S2Cfg<float> { static constexpr int VPL = 1, KMAX = 8; };
template <> struct S2Cfg<double> { static constexpr int VPL = 2, KMAX = 8; };
template <> struct S2Cfg<__half> { static constexpr int VPL = 1, KMAX = 6; };

template <typename T, int K>
struct S2Geom {
  static constexpr int V = Traits<T>::V;
  static constexpr int VPL = S2Cfg<T>::VPL;
  static constexpr int E = V * VPL;                 // cells per lane
  static constexpr int SW = 32 * E;                 // strip width (cells)
  static constexpr int HX = V * ((K + V - 1) / V);  // halo per side, vector aligned
  static constexpr int OW = SW - 2 * HX;            // output columns per strip
  static constexpr int STAGE_ELEMS = SW * kS2Rows;
  static constexpr int RING_BYTES = kS2Stages * STAGE_ELEMS * (int)sizeof(T);
  static constexpr int SMEM = kS2Warps * (RING_BYTES + kS2Stages * 8);
};

template <typename T, int K>
__global__ void __launch_bounds__(kS2Warps * 32)
    stream2d_k(const __grid_constant__ CUtensorMap src_map, T *__restrict__ dst, GridParams g,
               int n_strips, int n_chunks, int chunk_rows) {
  using Gm = S2Geom<T, K>;
  using C = typename Traits<T>::C;
  constexpr int E = Gm::E, V = Gm::V, VPL = Gm::VPL;
  constexpr uint32_t kStageBytes = Gm::STAGE_ELEMS * sizeof(T);
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T *ring = reinterpret_cast<T *>(smem + warp * Gm::RING_BYTES);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kS2Warps * Gm::RING_BYTES) + warp * kS2Stages;

  const int64_t gw = (int64_t)blockIdx.x * kS2Warps + warp;
  if (gw >= (int64_t)n_strips * n_chunks) return;  // no CTA-wide barrier in this kernel
  const int strip = (int)(gw % n_strips);
  const int chunk = (int)(gw / n_strips);
  const int xs = strip * Gm::OW - Gm::HX;  // first column of the strip (may be < 0)
  const int ny = (int)g.ny, nx = (int)g.nx;
  const int y0 = chunk * chunk_rows;
  const int y1 = min(ny, y0 + chunk_rows);
  const int lo0 = max(0, y0 - K);
  const int hi0 = min(ny, y1 + K);
  const int n_in = hi0 - lo0;
  const int n_groups = (n_in + kS2Rows - 1) / kS2Rows;
  const int n_iter = y1 - lo0 + K;

  if (lane == 0) {
    tma_prefetch_desc(&src_map);
    for (int s = 0; s < kS2Stages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
    for (int s = 0; s < kS2Stages && s < n_groups; ++s) {
      mbar_arrive_expect_tx(&bars[s], kStageBytes);
      tma_load_2d(ring + s * Gm::STAGE_ELEMS, &src_map, &bars[s], xs, lo0 + s * kS2Rows);
    }
  }
  __syncwarp();

  const int xl = xs + lane * E;  // column of this lane's first cell
  const int eL = -xl;            // element index holding x == 0 (if in [0, E))
  const int eR = nx - 1 - xl;    // element index holding x == nx-1
  const bool edge = (xs <= 0) || (xs + Gm::SW > nx - 1);
  const C alpha = (C)g.alpha, beta = (C)g.beta;

  C wa[K][E], wb[K][E];  // level l rows R-1 and R (produced two and one rows ago)
#pragma unroll
  for (int l = 0; l < K; ++l)
#pragma unroll
    for (int e = 0; e < E; ++e) { wa[l][e] = C(0); wb[l][e] = C(0); }

  for (int t = 0; t < n_iter; ++t) {
    C nw[E];  // newest row of the level being processed
    const int grp = t / kS2Rows;
    const int rr = t - grp * kS2Rows;
    const int stg = grp % kS2Stages;
    if (t < n_in) {
      if (rr == 0) {
        bool ok = mbar_wait_bounded(&bars[stg], (uint32_t)(grp / kS2Stages) & 1u);
        if (!__all_sync(0xffffffffu, ok)) {
          // give up: record it, let every issued copy land, then leave
          if (lane == 0) {
            report_timeout(g.status);
            for (int q = grp + 1; q < n_groups && q < grp + kS2Stages; ++q)
              mbar_wait_bounded(&bars[q % kS2Stages], (uint32_t)(q / kS2Stages) & 1u);
          }
          __syncwarp();
          return;
        }
      }
      const T *src = ring + stg * Gm::STAGE_ELEMS + rr * Gm::SW + lane * E;
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const uint4 w = *reinterpret_cast<const uint4 *>(src + v * V);
        unpack16<T>(w, nw + v * V);
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) nw[e] = wb[0][e];  // past the last row: never stored
    }

#pragma unroll
    for (int l = 0; l < K; ++l) {
      // level l+1 of row R from level l rows R-1 (wa), R (wb), R+1 (nw)
      const int R = lo0 + t - (l + 1);
      const bool at_lo = (R == 0), at_hi = (R == ny - 1);
      C out[E];
      const C left = __shfl_up_sync(0xffffffffu, wb[l][E - 1], 1);
      const C right = __shfl_down_sync(0xffffffffu, wb[l][0], 1);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const C p = wb[l][e];
        C w = (e == 0) ? left : wb[l][e - 1];
        C ea = (e == E - 1) ? right : wb[l][e + 1];
        if (edge) {
          if (e == eL) w = p;
          if (e == eR) ea = p;
        }
        const C s = at_lo ? p : wa[l][e];
        const C n = at_hi ? p : nw[e];
        out[e] = ac_update<C>(p, (w + ea) + (s + n), C(-4), alpha, beta);
      }
#pragma unroll
      for (int e = 0; e < E; ++e) {
        wa[l][e] = wb[l][e];
        wb[l][e] = nw[e];
        nw[e] = out[e];
      }
    }

    // nw now holds level K of row RK
    const int RK = lo0 + t - K;
    if (RK >= y0 && RK < y1) {
      T *drow = dst + (int64_t)RK * g.pitch;
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const int xv = xl + v * V;
        if (xv >= xs + Gm::HX && xv < xs + Gm::SW - Gm::HX && xv < nx) {
          if (xv + V <= nx) {
            *reinterpret_cast<uint4 *>(drow + xv) = pack16<T>(nw + v * V);
          } else {
#pragma unroll
            for (int e = 0; e < V; ++e)
              if (xv + e < nx) drow[xv + e] = from_c<T>(nw[v * V + e]);
          }
        }
      }
    }

    // the stage's last row has been consumed (its values used above): refill
    if (t < n_in && (rr == kS2Rows - 1 || t == n_in - 1)) {
      __syncwarp();
      const int nxt = grp + kS2Stages;
      if (lane == 0 && nxt < n_groups) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bars[stg], kStageBytes);
        tma_load_2d(ring + stg * Gm::STAGE_ELEMS, &src_map, &bars[stg], xs, lo0 + nxt * kS2Rows);
      }
    }
  }
}

// ------------------------------------------------------------------ host ---

template <typename T, int K>
static Stream2DGeom geom_t() {
  using Gm = S2Geom<T, K>;
  return Stream2DGeom{Gm::SW, kS2Rows, Gm::HX, Gm::OW};
}

template <typename T, int K>
static cudaError_t launch_t(const GridParams &g, const CUtensorMap *map, void *dst, int num_sms,
                            cudaStream_t s) {
  using Gm = S2Geom<T, K>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(stream2d_k<T, K>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, Gm::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int n_strips = (int)((g.nx + Gm::OW - 1) / Gm::OW);
  // enough warps to keep ~8 rings per SM busy, but chunks of >= 4k (and 32) rows
  const int target_warps = std::max(1, num_sms) * 8;
  int n_chunks = std::max(1, target_warps / n_strips);
  const int min_rows = std::max(32, 4 * K);
  n_chunks = std::min<int>(n_chunks, (int)std::max<int64_t>(1, g.ny / min_rows));
  const int chunk_rows = (int)((g.ny + n_chunks - 1) / n_chunks);
  n_chunks = (int)((g.ny + chunk_rows - 1) / chunk_rows);
  const int64_t warps = (int64_t)n_strips * n_chunks;
  const unsigned blocks = (unsigned)((warps + kS2Warps - 1) / kS2Warps);
  stream2d_k<T, K><<<blocks, kS2Warps * 32, Gm::SMEM, s>>>(*map, (T *)dst, g, n_strips, n_chunks,
                                                          chunk_rows);
  return cudaGetLastError();
}

#define AC_S2_CASES(T, MAC) \
  MAC(T, 1) MAC(T, 2) MAC(T, 3) MAC(T, 4) MAC(T, 5) MAC(T, 6)
#define AC_S2_CASES8(T, MAC) AC_S2_CASES(T, MAC) MAC(T, 7) MAC(T, 8)

template <typename T>
static cudaError_t dispatch(int k, const GridParams &g, const CUtensorMap *map, void *dst,
                            int num_sms, cudaStream_t s) {
  switch (k) {
#define AC_CASE(TT, KK) \
  case KK:              \
    if constexpr (KK <= S2Cfg<TT>::KMAX) return launch_t<TT, KK>(g, map, dst, num_sms, s); \
    break;
    AC_S2_CASES8(T, AC_CASE)
#undef AC_CASE
  }
  return cudaErrorInvalidValue;
}

template <typename T>
static Stream2DGeom geom_dispatch(int k) {
  switch (k) {
#define AC_CASE(TT, KK) \
  case KK:              \
    if constexpr (KK <= S2Cfg<TT>::KMAX) return geom_t<TT, KK>(); \
    break;
    AC_S2_CASES8(T, AC_CASE)
#undef AC_CASE
  }
  return Stream2DGeom{0, 0, 0, 0};
}

bool stream2d_supported(int dtype, int k) {
  if (k < 1) return false;
  switch (dtype) {
    case AC_F64: return k <= S2Cfg<double>::KMAX;
    case AC_F32: return k <= S2Cfg<float>::KMAX;
    case AC_F16S: return k <= S2Cfg<__half>::KMAX;
  }
  return false;
}

Stream2DGeom stream2d_geom(int dtype, int k) {
  switch (dtype) {
    case AC_F64: return geom_dispatch<double>(k);
    case AC_F32: return geom_dispatch<float>(k);
    case AC_F16S: return geom_dispatch<__half>(k);
  }
  return Stream2DGeom{0, 0, 0, 0};
}

cudaError_t launch_stream2d(int dtype, int k, const GridParams &g, const CUtensorMap *src_map,
                            void *dst, int num_sms, cudaStream_t s) {
  switch (dtype) {
    case AC_F64: return dispatch<double>(k, g, src_map, dst, num_sms, s);
    case AC_F32: return dispatch<float>(k, g, src_map, dst, num_sms, s);
    case AC_F16S: return dispatch<__half>(k, g, src_map, dst, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ac
