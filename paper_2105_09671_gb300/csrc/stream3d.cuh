// 3D streaming stencil with temporal blocking (7-point Laplacian).
//
// Advances k explicit Euler steps of Eq. (pytorchACeq) per pass over HBM.
// Work unit: one CTA owns an xy tile (out_x x out_y cells plus a halo of HX
// columns and k rows per side) and a chunk of z planes, and streams the
// planes in increasing z:
//   - input planes arrive through a ring of shared-memory stages, each one
//     TMA tile load of the whole halo tile (zero fill outside the domain),
//     signalled on one mbarrier per stage;
//   - time level l of plane Z is formed once level l-1 of plane Z+1 exists
//     (a lag of one plane per level); each thread keeps, for its own 16-byte
//     vectors, the last three planes of every level in a ring of registers
//     (the z neighbours), and levels 1..k-1 also publish their newest plane
//     in shared memory (double buffered) for the x/y neighbours of others;
//   - x neighbours come from the adjacent lane by warp shuffle (lanes own
//     consecutive vectors of a row), the two warp-edge lanes read them from
//     shared memory; y neighbours are shared-memory reads;
//   - zero-Neumann ghosts (Section 2) are clamps at the current level: a
//     neighbour across a domain face is the boundary cell itself.  y faces
//     are clamped shared-memory offsets; z faces copy the boundary plane into
//     the ghost slot in the few iterations that touch them (a separate
//     instantiation of the loop body); x faces are one select per vector
//     when nx is a multiple of the vector width (FASTX), else per element;
//   - only level k inside the tile interior and the chunk's own planes is
//     written; the halo cells computed on the way are discarded.
// One __syncthreads per plane; persistent CTAs loop over (tile, z-chunk)
// items.
#pragma once

#include <algorithm>

#include "kernels.h"

namespace ac {

// Tile shapes (the autotuner picks one): TILE 0 = 32 output rows, the default
// vectors per thread; TILE 1 = 16 output rows (several CTAs per SM, each with
// its own barrier); TILE 2 = 32 rows with two vectors per thread (more warps).
constexpr int kS3Tiles = 3;
template <typename T, int TILE> struct S3Cfg;
template <int TILE> struct S3Cfg<float, TILE> {
  static constexpr int OX = 128, OY = TILE == 1 ? 16 : 32, VPT = TILE == 2 ? 2 : 3, D = 4, KMAX = 3;
};
template <int TILE> struct S3Cfg<double, TILE> {
  static constexpr int OX = 64, OY = TILE == 1 ? 16 : 32, VPT = TILE == 2 ? 2 : 3, D = 4, KMAX = 2;
};
template <int TILE> struct S3Cfg<__half, TILE> {
  static constexpr int OX = 128, OY = TILE == 1 ? 16 : 32, VPT = TILE == 2 ? 1 : 2, D = 4, KMAX = 3;
};

template <typename T, int K, int TILE = 0>
struct S3Geom {
  using Cfg = S3Cfg<T, TILE>;
  using C = typename Traits<T>::C;
  static constexpr int V = Traits<T>::V;
  static constexpr int HX = V * ((K + V - 1) / V);
  static constexpr int OX = Cfg::OX, OY = Cfg::OY;
  static constexpr int TX = OX + 2 * HX, TXV = TX / V, TY = OY + 2 * K;
  static constexpr int NVEC = TXV * TY;
  static constexpr int VPT = Cfg::VPT;
  static constexpr int NT = ((NVEC + VPT - 1) / VPT + 31) / 32 * 32;
  static constexpr int D = Cfg::D;
  static constexpr int MINB = TILE == 1 ? 2 : 1;  // resident CTAs the register budget targets
  static constexpr int STAGE_BYTES = TX * TY * (int)sizeof(T);
  static constexpr int STAGE_STRIDE = (STAGE_BYTES + 127) / 128 * 128;  // TMA dst alignment
  static constexpr int LVL_BYTES = TX * TY * (int)sizeof(C);
  static constexpr int LVL_TOTAL = (K > 1 ? 2 * (K - 1) * LVL_BYTES : 0);
  static constexpr int SMEM = D * STAGE_STRIDE + LVL_TOTAL + D * 8 + 16;
  static_assert(NT <= 1024, "tile too large for one CTA");
  static_assert(VPT * NT >= NVEC, "vector slots");
};

template <typename T, int V>
__device__ __forceinline__ void ld_vec(const T *buf, int idx, typename Traits<T>::C *out) {
  unpack16<T>(*reinterpret_cast<const uint4 *>(buf + idx), out);
}
template <int V>
__device__ __forceinline__ void ld_vec_c(const float *buf, int idx, float *out) {
#pragma unroll
  for (int i = 0; i < V; i += 4) {
    const float4 f = *reinterpret_cast<const float4 *>(buf + idx + i);
    out[i] = f.x; out[i + 1] = f.y; out[i + 2] = f.z; out[i + 3] = f.w;
  }
}
template <int V>
__device__ __forceinline__ void ld_vec_c(const double *buf, int idx, double *out) {
#pragma unroll
  for (int i = 0; i < V; i += 2) {
    const double2 f = *reinterpret_cast<const double2 *>(buf + idx + i);
    out[i] = f.x; out[i + 1] = f.y;
  }
}
template <int V>
__device__ __forceinline__ void st_vec_c(float *buf, int idx, const float *in) {
#pragma unroll
  for (int i = 0; i < V; i += 4)
    *reinterpret_cast<float4 *>(buf + idx + i) = make_float4(in[i], in[i + 1], in[i + 2], in[i + 3]);
}
template <int V>
__device__ __forceinline__ void st_vec_c(double *buf, int idx, const double *in) {
#pragma unroll
  for (int i = 0; i < V; i += 2)
    *reinterpret_cast<double2 *>(buf + idx + i) = make_double2(in[i], in[i + 1]);
}

template <typename T, int K, bool FASTX, int TILE>
__global__ void __launch_bounds__(S3Geom<T, K, TILE>::NT, S3Geom<T, K, TILE>::MINB)
    stream3d_k(const __grid_constant__ CUtensorMap src_map, T *__restrict__ dst, GridParams g,
               int tiles_x, int tiles_y, int nzc, int zchunk) {
  using Gm = S3Geom<T, K, TILE>;
  using C = typename Traits<T>::C;
  constexpr int V = Gm::V, VPT = Gm::VPT, TXV = Gm::TXV, TY = Gm::TY, TX = Gm::TX, D = Gm::D;
  constexpr int NT = Gm::NT, NVEC = Gm::NVEC;
  constexpr int PLANE = TX * TY;  // elements per plane buffer
  extern __shared__ __align__(128) unsigned char smem[];
  // stage s of the TMA ring starts at byte s * STAGE_STRIDE
  auto stage_ptr = [&](int s) { return reinterpret_cast<T *>(smem + s * Gm::STAGE_STRIDE); };
  C *lvl = reinterpret_cast<C *>(smem + D * Gm::STAGE_STRIDE);  // [K-1][2][TY][TX]
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + D * Gm::STAGE_STRIDE + Gm::LVL_TOTAL);
  volatile int &abort_flag = *reinterpret_cast<int *>(bars + D);

  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    tma_prefetch_desc(&src_map);
    for (int s = 0; s < D; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
    abort_flag = 0;
  }
  __syncthreads();

  // this thread's vector slots: q = tid + j*NT -> tile row qr, vector column qc
  int qr[VPT], qc[VPT];
  bool qv[VPT];
#pragma unroll
  for (int j = 0; j < VPT; ++j) {
    const int q = tid + j * NT;
    qv[j] = q < NVEC;
    const int qq = qv[j] ? q : NVEC - 1;
    qr[j] = qq / TXV;
    qc[j] = qq - qr[j] * TXV;
  }
  const int nx = (int)g.nx, ny = (int)g.ny, nz = (int)g.nz;
  const int64_t plane_stride = g.pitch * g.ny;
  const C alpha = (C)g.alpha, beta = (C)g.beta;

  // Level l keeps its last three planes in a ring of register slots: at
  // iteration t slot t%3 holds plane Z+1 (newest), (t+2)%3 plane Z and
  // (t+1)%3 plane Z-1 of the stencil that forms level l+1 of plane Z.  The
  // plane loop is unrolled by three so that every slot index is a constant.
  C ring[K][3][VPT][V];
#pragma unroll
  for (int l = 0; l < K; ++l)
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int j = 0; j < VPT; ++j)
#pragma unroll
        for (int e = 0; e < V; ++e) ring[l][s][j][e] = C(0);

  uint32_t slot = 0;  // planes consumed so far by this CTA: ring position and phase
  const int items = tiles_x * tiles_y * nzc;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int tx = item % tiles_x;
    const int rem = item / tiles_x;
    const int ty = rem % tiles_y;
    const int zc = rem / tiles_y;
    const int x0 = tx * Gm::OX, y0 = ty * Gm::OY;
    const int z0 = zc * zchunk, z1 = min(nz, z0 + zchunk);
    const int lo0 = max(0, z0 - K), hi0 = min(nz, z1 + K);
    const int n_in = hi0 - lo0, n_iter = z1 - lo0 + K;
    const int bx = x0 - Gm::HX, by = y0 - K;

    if (tid == 0) {
      for (int p = 0; p < D && p < n_in; ++p) {
        const int s = (int)((slot + p) % D);
        mbar_arrive_expect_tx(&bars[s], Gm::STAGE_BYTES);
        tma_load_3d(stage_ptr(s), &src_map, &bars[s], bx, by, lo0 + p);
      }
    }

    // Per-item facts of this thread's vectors.  y neighbours are read at
    // shared-memory offsets clamped to the domain (row gy = 0 reads itself
    // as its lower neighbour, gy = ny-1 as its upper one: the zero-Neumann
    // ghost) and to the tile.
    const int rlo = max(0, -by), rhi = min(TY - 1, ny - 1 - by);
    const bool xedge = (bx <= 0) || (bx + TX > nx - 1);
    int own[VPT], ysn[VPT], ynn[VPT], lnb[VPT], rnb[VPT], gxv[VPT];
    bool st_ok[VPT], st_full[VPT], lfix[VPT], rfix[VPT];
    int64_t goff[VPT];
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      const int r = qr[j], c = qc[j];
      own[j] = r * TX + c * V;
      ysn[j] = max(r - 1, rlo) * TX + c * V;
      ynn[j] = min(r + 1, rhi) * TX + c * V;
      lnb[j] = (lane == 0 && c > 0) ? own[j] - 1 : -1;
      rnb[j] = (lane == 31 && c < TXV - 1) ? own[j] + V : -1;
      const int gy = by + r, gx = bx + c * V;
      gxv[j] = gx;
      lfix[j] = gx == 0;               // element 0 is the x = 0 face
      rfix[j] = gx + V - 1 == nx - 1;  // element V-1 is the x = nx-1 face
      st_ok[j] = qv[j] && r >= K && r < K + Gm::OY && c >= Gm::HX / V &&
                 c < (Gm::HX + Gm::OX) / V && gy < ny && gx < nx;
      st_full[j] = gx + V <= nx;
      goff[j] = (int64_t)gy * g.pitch + gx;
    }

    auto body = [&]<int P, bool BND>(int t) -> bool {
      constexpr int SN = P, SB = (P + 2) % 3, SA = (P + 1) % 3;
      if (!BND || t < n_in) {
        const uint32_t u = slot + t;
        const int s = (int)(u % D);
        if (!mbar_wait_bounded(&bars[s], (u / D) & 1u)) abort_flag = 1;
        const T *stage = stage_ptr(s);
#pragma unroll
        for (int j = 0; j < VPT; ++j) ld_vec<T, V>(stage, own[j], ring[0][SN][j]);
      }
#pragma unroll
      for (int l = 0; l < K; ++l) {
        const int Z = lo0 + t - (l + 1);  // plane of level l+1 formed now
        if constexpr (BND) {
          if (Z == 0) {                   // ghost below the bottom face
#pragma unroll
            for (int j = 0; j < VPT; ++j)
#pragma unroll
              for (int e = 0; e < V; ++e) ring[l][SA][j][e] = ring[l][SB][j][e];
          }
          if (Z == nz - 1) {              // ghost above the top face
#pragma unroll
            for (int j = 0; j < VPT; ++j)
#pragma unroll
              for (int e = 0; e < V; ++e) ring[l][SN][j][e] = ring[l][SB][j][e];
          }
        }
        const int ZK = lo0 + t - K;
        const bool store = (l == K - 1) && ZK >= z0 && ZK < z1;
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
          const C *mid = ring[l][SB][j];
          C sv[V], nv[V], wl, er;
          const C sh_l = __shfl_up_sync(0xffffffffu, mid[V - 1], 1);
          const C sh_r = __shfl_down_sync(0xffffffffu, mid[0], 1);
          if (l == 0) {
            const T *cb = stage_ptr((int)((slot + t + D - 1) % D));
            ld_vec<T, V>(cb, ysn[j], sv);
            ld_vec<T, V>(cb, ynn[j], nv);
            wl = lnb[j] >= 0 ? to_c(cb[lnb[j]]) : sh_l;
            er = rnb[j] >= 0 ? to_c(cb[rnb[j]]) : sh_r;
          } else {
            const C *cb = lvl + ((l - 1) * 2 + ((t + 1) & 1)) * PLANE;
            ld_vec_c<V>(cb, ysn[j], sv);
            ld_vec_c<V>(cb, ynn[j], nv);
            wl = lnb[j] >= 0 ? cb[lnb[j]] : sh_l;
            er = rnb[j] >= 0 ? cb[rnb[j]] : sh_r;
          }
          if constexpr (FASTX) {
            wl = lfix[j] ? mid[0] : wl;
            er = rfix[j] ? mid[V - 1] : er;
          }
          C out[V];
#pragma unroll
          for (int e = 0; e < V; ++e) {
            const C p = mid[e];
            C w = (e == 0) ? wl : mid[e - 1];
            C ea = (e == V - 1) ? er : mid[e + 1];
            if constexpr (!FASTX) {
              if (xedge) {
                const int gx = gxv[j] + e;
                if (gx == 0) w = p;
                if (gx == nx - 1) ea = p;
              }
            }
            const C nsum = ((w + ea) + (sv[e] + nv[e])) + (ring[l][SA][j][e] + ring[l][SN][j][e]);
            out[e] = ac_update<C>(p, nsum, C(-6), alpha, beta);
          }
          if (l + 1 < K) {
#pragma unroll
            for (int e = 0; e < V; ++e) ring[l + 1 < K ? l + 1 : 0][SN][j][e] = out[e];
            if (qv[j]) st_vec_c<V>(lvl + (l * 2 + (t & 1)) * PLANE, own[j], out);
          } else if (store && st_ok[j]) {
            T *d = dst + (int64_t)ZK * plane_stride + goff[j];
            if (st_full[j]) {
              *reinterpret_cast<uint4 *>(d) = pack16<T>(out);
            } else {
#pragma unroll
              for (int e = 0; e < V; ++e)
                if (gxv[j] + e < nx) d[e] = from_c<T>(out[e]);
            }
          }
        }
      }

      __syncthreads();
      if (abort_flag) {
        if (tid == 0) {
          report_timeout(g.status);
          for (int p = t + 1; p < n_in && p < t + D; ++p) {
            const uint32_t u = slot + p;
            mbar_wait_bounded(&bars[u % D], (u / D) & 1u);
          }
        }
        return false;
      }
      // the stage of plane t-1 is no longer read: refill it with plane t-1+D
      if (tid == 0 && t >= 1 && t - 1 + D < n_in) {
        const uint32_t u = slot + t - 1;
        const int s = (int)(u % D);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bars[s], Gm::STAGE_BYTES);
        tma_load_3d(stage_ptr(s), &src_map, &bars[s], bx, by, lo0 + t - 1 + D);
      }
      return true;
    };

    // Iterations that touch a z face (ghost copies) or run past the last
    // input plane take the BND body: t in [1, K] when the chunk starts at
    // z = 0, and t >= nz - lo0 when it ends at the top face.
    const int bnd_lo_end = (lo0 == 0) ? K : -1;
    const int bnd_hi_begin = (hi0 == nz) ? nz - lo0 - 1 : n_iter;
    int t = 0;
    for (; t + 3 <= n_iter; t += 3) {
      const bool bnd = (t <= bnd_lo_end) || (t + 2 >= bnd_hi_begin);
      if (bnd) {
        if (!body.template operator()<0, true>(t)) return;
        if (!body.template operator()<1, true>(t + 1)) return;
        if (!body.template operator()<2, true>(t + 2)) return;
      } else {
        if (!body.template operator()<0, false>(t)) return;
        if (!body.template operator()<1, false>(t + 1)) return;
        if (!body.template operator()<2, false>(t + 2)) return;
      }
    }
    if (t < n_iter && !body.template operator()<0, true>(t++)) return;
    if (t < n_iter && !body.template operator()<1, true>(t++)) return;
    slot += (uint32_t)n_in;
  }
}

// ------------------------------------------------------------------ host ---

template <typename T, int K, int TILE>
inline Stream3DGeom s3_geom_t() {
  using Gm = S3Geom<T, K, TILE>;
  return Stream3DGeom{Gm::TX, Gm::TY, Gm::HX, Gm::OX, Gm::OY, Gm::NT, Gm::SMEM};
}

template <typename T, int K, bool FASTX, int TILE>
static cudaError_t s3_launch_t(const GridParams &g, const CUtensorMap *map, void *dst, int num_sms,
                               cudaStream_t s) {
  using Gm = S3Geom<T, K, TILE>;
  int dev = 0;
  cudaGetDevice(&dev);
  static unsigned attr_mask = 0;
  static int occ_cache[32] = {0};
  if (dev < 32 && !(attr_mask & (1u << dev))) {
    cudaError_t e = cudaFuncSetAttribute(stream3d_k<T, K, FASTX, TILE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, Gm::SMEM);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, stream3d_k<T, K, FASTX, TILE>, Gm::NT, Gm::SMEM);
    if (e != cudaSuccess) return e;
    occ_cache[dev] = std::max(1, occ);
    attr_mask |= 1u << dev;
  }
  const int occ = dev < 32 ? occ_cache[dev] : 1;
  const int tiles_x = (int)((g.nx + Gm::OX - 1) / Gm::OX);
  const int tiles_y = (int)((g.ny + Gm::OY - 1) / Gm::OY);
  const int64_t tiles = (int64_t)tiles_x * tiles_y;
  const int64_t slots = (int64_t)std::max(1, num_sms) * occ;
  // z-chunk count: minimise (rounds of items over the resident CTAs) x
  // (planes streamed per item, including the 2k halo planes)
  int best_nzc = 1;
  double best_cost = 1e300;
  const int max_nzc = (int)std::max<int64_t>(1, g.nz / std::max(4, 2 * K));
  for (int nzc = 1; nzc <= max_nzc; ++nzc) {
    const int64_t items = tiles * nzc;
    const int64_t rounds = (items + slots - 1) / slots;
    const int64_t chunk = (g.nz + nzc - 1) / nzc;
    const double cost = (double)rounds * (double)(chunk + 2 * K);
    if (cost < best_cost - 1e-9) { best_cost = cost; best_nzc = nzc; }
  }
  const int zchunk = (int)((g.nz + best_nzc - 1) / best_nzc);
  const int nzc = (int)((g.nz + zchunk - 1) / zchunk);
  const int64_t items = tiles * nzc;
  const unsigned blocks = (unsigned)std::min<int64_t>(items, slots);
  stream3d_k<T, K, FASTX, TILE><<<blocks, Gm::NT, Gm::SMEM, s>>>(*map, (T *)dst, g, tiles_x, tiles_y,
                                                           nzc, zchunk);
  return cudaGetLastError();
}

// Dispatch over the supported depths and tiles of one storage type.
template <typename T, int TILE>
cudaError_t s3_dispatch_tile(int k, const GridParams &g, const CUtensorMap *map, void *dst,
                             int num_sms, cudaStream_t s) {
  const bool fastx = g.nx % Traits<T>::V == 0;
  switch (k) {
    case 1:
      return fastx ? s3_launch_t<T, 1, true, TILE>(g, map, dst, num_sms, s)
                   : s3_launch_t<T, 1, false, TILE>(g, map, dst, num_sms, s);
    case 2:
      if constexpr (S3Cfg<T, TILE>::KMAX >= 2)
        return fastx ? s3_launch_t<T, 2, true, TILE>(g, map, dst, num_sms, s)
                     : s3_launch_t<T, 2, false, TILE>(g, map, dst, num_sms, s);
      break;
    case 3:
      if constexpr (S3Cfg<T, TILE>::KMAX >= 3)
        return fastx ? s3_launch_t<T, 3, true, TILE>(g, map, dst, num_sms, s)
                     : s3_launch_t<T, 3, false, TILE>(g, map, dst, num_sms, s);
      break;
  }
  return cudaErrorInvalidValue;
}

template <typename T, int TILE>
Stream3DGeom s3_geom_tile(int k) {
  switch (k) {
    case 1: return s3_geom_t<T, 1, TILE>();
    case 2:
      if constexpr (S3Cfg<T, TILE>::KMAX >= 2) return s3_geom_t<T, 2, TILE>();
      break;
    case 3:
      if constexpr (S3Cfg<T, TILE>::KMAX >= 3) return s3_geom_t<T, 3, TILE>();
      break;
  }
  return Stream3DGeom{0, 0, 0, 0, 0, 0, 0};
}

template <typename T>
Stream3DGeom s3_geom(int k, int tile) {
  switch (tile) {
    case 0: return s3_geom_tile<T, 0>(k);
    case 1: return s3_geom_tile<T, 1>(k);
    case 2: return s3_geom_tile<T, 2>(k);
  }
  return Stream3DGeom{0, 0, 0, 0, 0, 0, 0};
}

// Launch of one (storage type, tile): defined and explicitly instantiated in
// k_stream3d_<type>.cu, which is compiled once per tile (AC_S3_TILE) so that
// the kernel instantiations spread over parallel compiler processes.
template <typename T, int TILE>
cudaError_t stream3d_launch_tile(int k, const GridParams &g, const CUtensorMap *map, void *dst,
                                 int num_sms, cudaStream_t s);

}  // namespace ac
