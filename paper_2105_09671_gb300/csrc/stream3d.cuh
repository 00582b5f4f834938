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
//     (a lag of one plane per level);
//   - a thread owns R vertically adjacent 16-byte vectors (one column of R
//     rows) and keeps, for each, the last three planes of every level in a
//     ring of registers (the z neighbours); levels 1..k-1 also publish their
//     newest plane in shared memory (three buffers) for the x/y
//     neighbours of others;
//   - x neighbours come from the adjacent lane by warp shuffle (lanes own
//     consecutive columns of a row group), the two warp-edge lanes read
//     theirs from shared memory; at k = 2 the output columns of each row
//     group fill one warp's lanes and the halo slots whole warps after
//     them, which form levels 1..k-1 only; y neighbours inside the thread's own rows
//     are registers, the rows above and below its group are shared-memory
//     reads.  The reads of level 0 (the previous input plane's stage) are
//     issued at the start of an iteration, ahead of the wait for the new
//     plane; those of level l >= 1 right before level l is formed, which
//     spreads the iteration's shared-memory traffic instead of issuing it
//     in one burst after the barrier;
//   - zero-Neumann ghosts (Section 2) are clamps at the current level: a
//     neighbour across a domain face is the boundary cell itself.  y faces
//     are clamped shared-memory offsets and, inside a row group, a select
//     (only in tiles that hold a y face); z faces copy the boundary plane
//     into the ghost slot in the few iterations that touch them; those
//     iterations and y-face tiles run a separate instantiation of the loop
//     body.  x faces are one select per vector when nx is a multiple of the
//     vector width (FASTX), else per element;
//   - only level k inside the tile interior and the chunk's own planes is
//     written; the halo cells computed on the way are discarded.
// One CTA barrier per plane (__syncthreads_or, which also tells every
// thread whether any bounded wait expired); persistent CTAs loop over
// (tile, z-chunk) items.
#pragma once

#include <algorithm>
#include <type_traits>

#include "kernels.h"

namespace ac {

// Tile shapes (the autotuner picks one), out_x x out_y outputs per CTA and
// R rows per thread: TILE 0 = 128 x 32, R = 2; TILE 1 = 128 x 16, R = 2,
// several CTAs per SM; TILE 2 = 128 x 32, R = 4 (twice the work per thread
// and iteration, half the threads; FP16 storage: R = 1).  FP64 tiles are
// half as wide in x.  MINB = resident CTAs the register budget targets.  The
// TMA box (the halo tile) is at most 256 elements in x.
constexpr int kS3Tiles = 3;
template <typename T, int TILE> struct S3Cfg;
// VL = cells per thread vector: one 16-byte vector (FP16 storage: 8
// cells).  Half vectors for FP16 storage (VL = 4, 8-byte loads, FP32's
// thread count and registers) were measured slower on GB300 at 512^3 (k = 2
// tile 0: 995 against 1054 Gcell-updates/s): more threads repeat the
// per-plane work, and the 16-byte TMA alignment widens the x halo to 8.
template <int TILE> struct S3Cfg<float, TILE> {
  static constexpr int OX = 128, OY = TILE == 1 ? 16 : 32;
  static constexpr int R = TILE == 2 ? 4 : 2, KMAX = 3, MINB = TILE == 1 ? 2 : 1;
  static constexpr int DK = TILE == 0 ? 6 : 3;  // TMA stages at k >= 2
  static constexpr int VL = 4;
};
template <int TILE> struct S3Cfg<double, TILE> {
  static constexpr int OX = 64, OY = TILE == 1 ? 16 : 32;
  static constexpr int R = TILE == 2 ? 4 : 2, KMAX = 2, MINB = TILE == 1 ? 2 : 1;
  static constexpr int DK = 3;
  static constexpr int VL = 2;
};
template <int TILE> struct S3Cfg<__half, TILE> {
  static constexpr int OX = 128, OY = TILE == 1 ? 16 : 32;
  static constexpr int R = TILE == 2 ? 1 : 2, KMAX = 3, MINB = TILE == 1 ? 2 : 1;
  static constexpr int DK = 3;
  static constexpr int VL = 8;
};

template <typename T, int K, int TILE = 0>
struct S3Geom {
  using Cfg = S3Cfg<T, TILE>;
  using C = typename Traits<T>::C;
  static constexpr int V = Cfg::VL;                       // cells per thread vector
  static constexpr int VA = 16 / (int)sizeof(T);          // TMA x alignment (elements)
  static constexpr int HA = V > VA ? V : VA;
  static constexpr int R = Cfg::R, MINB = Cfg::MINB;
  static constexpr int HX = HA * ((K + HA - 1) / HA);     // halo columns, both alignments
  static constexpr int OX = Cfg::OX, OY = Cfg::OY;
  static constexpr int TX = OX + 2 * HX, TXV = TX / V;
  static constexpr int TY = (OY + 2 * K + R - 1) / R * R;  // rows, whole groups of R
  static constexpr int NSLOT = TXV * (TY / R);             // (column, row group) slots
  // Output slots: the columns of the out_x cells in the row groups that hold
  // an output row.  When they fill whole warps (SPLIT) they take the first
  // NA threads, row group by row group, and the halo slots the warps after
  // them, which skip the last level (a warp-uniform branch in the same
  // code).  Measured on GB300 at 512^3 (FP32, 256^3 FP64): +2.7 % FP32,
  // +5.5 % FP16 storage, +4.4 % FP64 at k = 2; at k = 3 (more registers,
  // spills) and at k = 1 (no halo warp work to save; 17 warps instead of
  // 19) it was slower, so only k = 2 takes it.
  static constexpr int OXV = OX / V, HXV = HX / V;
  static constexpr int GA0 = K / R, GA1 = (K + OY + R - 1) / R;  // row groups with output rows
  static constexpr int NA = (GA1 - GA0) * OXV;
  static constexpr bool SPLIT = K == 2 && NA % 32 == 0 && NA < NSLOT && HXV == 1;
  static constexpr int NT = (NSLOT + 31) / 32 * 32;        // one slot per thread
  static constexpr int STAGE_BYTES = TX * TY * (int)sizeof(T);
  static constexpr int STAGE_STRIDE = (STAGE_BYTES + 127) / 128 * 128;  // TMA dst alignment
  static constexpr int LVL_BYTES = TX * TY * (int)sizeof(C);
  // Level buffers of 8-cell vectors (FP16 storage) are split in two regions
  // of 4-value halves (LHALF elements apart, LROW elements per row), so that
  // each lane's 16-byte read or write is one of 32 consecutive 16-byte words
  // (the 32-byte vectors side by side conflict two ways in shared memory).
  static constexpr bool LSPLIT = V == 8 && std::is_same_v<C, float>;
  static constexpr int LROW = LSPLIT ? TX / 2 : TX, LHALF = LSPLIT ? TX * TY / 2 : 0;
  static constexpr int LVL_TOTAL = (K > 1 ? 3 * (K - 1) * LVL_BYTES : 0);  // 3 planes per level
  // D TMA stages (3 or 6; the planes in flight hide HBM latency): 6 at
  // k = 1, else per type and tile as measured on GB300 at 512^3 (six pay
  // for the FP32 128 x 32 tile, +5 % at k = 2, and cost elsewhere, where
  // the twice-unrolled plane loop outgrows the instruction cache).  The
  // plane loop is unrolled by U = lcm(3, D) so that every stage,
  // register-ring slot and level buffer index is a constant.
  static constexpr bool FITS6 = 6 * STAGE_STRIDE + LVL_TOTAL + 6 * 8 + 16 <= 227 * 1024;
  static constexpr int D = K == 1 ? 6 : (Cfg::DK == 6 && FITS6 ? 6 : 3);
  static constexpr int U = D == 6 ? 6 : 3;
  static_assert(D == 3 || D == 6, "stages");
  static constexpr int SMEM = D * STAGE_STRIDE + LVL_TOTAL + D * 8;  // + the stage barriers
  static_assert(NT <= 1024, "tile too large for one CTA");
  static_assert(SMEM <= 227 * 1024, "tile too large for shared memory");
  static_assert(TY <= 256 && TX <= 256, "TMA box limits");
};

// V storage elements (16 or 8 bytes) <-> V compute values.
template <typename T, int V>
__device__ __forceinline__ void ld_vec(const T *buf, int idx, typename Traits<T>::C *out) {
  if constexpr (sizeof(T) * V == 16) {
    unpack16<T>(*reinterpret_cast<const uint4 *>(buf + idx), out);
  } else {
    static_assert(std::is_same_v<T, __half> && V == 4, "8-byte vectors are FP16 storage");
    const uint2 w = *reinterpret_cast<const uint2 *>(buf + idx);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&w.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&w.y));
    out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
  }
}
template <typename T, int V>
__device__ __forceinline__ void st_vec_g(T *p, const typename Traits<T>::C *in, bool pred) {
  if constexpr (sizeof(T) * V == 16) {
    const uint4 pk = pack16<T>(in);
    if (pred) *reinterpret_cast<uint4 *>(p) = pk;
  } else {
    static_assert(std::is_same_v<T, __half> && V == 4, "8-byte vectors are FP16 storage");
    const __half2 a = __floats2half2_rn(in[0], in[1]), b = __floats2half2_rn(in[2], in[3]);
    uint2 pk;
    pk.x = *reinterpret_cast<const uint32_t *>(&a);
    pk.y = *reinterpret_cast<const uint32_t *>(&b);
    if (pred) *reinterpret_cast<uint2 *>(p) = pk;
  }
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

// A vector of V compute values in a level buffer (split layout: two halves
// Gm::LHALF elements apart).
template <typename Gm, typename C>
__device__ __forceinline__ void ld_lvl(const C *buf, int idx, C *out) {
  if constexpr (Gm::LSPLIT) {
    ld_vec_c<Gm::V / 2>(buf, idx, out);
    ld_vec_c<Gm::V / 2>(buf + Gm::LHALF, idx, out + Gm::V / 2);
  } else {
    ld_vec_c<Gm::V>(buf, idx, out);
  }
}
template <typename Gm, typename C>
__device__ __forceinline__ void st_lvl(C *buf, int idx, const C *in) {
  if constexpr (Gm::LSPLIT) {
    st_vec_c<Gm::V / 2>(buf, idx, in);
    st_vec_c<Gm::V / 2>(buf + Gm::LHALF, idx, in + Gm::V / 2);
  } else {
    st_vec_c<Gm::V>(buf, idx, in);
  }
}

template <typename T, int K, bool FASTX, int TILE>
__global__ void __launch_bounds__(S3Geom<T, K, TILE>::NT, S3Geom<T, K, TILE>::MINB)
    stream3d_k(const __grid_constant__ CUtensorMap src_map, T *__restrict__ dst, GridParams g,
               int tiles_x, int tiles_y, int nzc, int zchunk) {
  using Gm = S3Geom<T, K, TILE>;
  using C = typename Traits<T>::C;
  constexpr int V = Gm::V, R = Gm::R, TXV = Gm::TXV, TY = Gm::TY, TX = Gm::TX, D = Gm::D, U = Gm::U;
  constexpr int NSLOT = Gm::NSLOT;
  constexpr int PLANE = TX * TY;  // elements per plane buffer
  extern __shared__ __align__(128) unsigned char smem[];
  // stage s of the TMA ring starts at byte s * STAGE_STRIDE
  auto stage_ptr = [&](int s) { return reinterpret_cast<T *>(smem + s * Gm::STAGE_STRIDE); };
  C *lvl = reinterpret_cast<C *>(smem + D * Gm::STAGE_STRIDE);  // [K-1][3][TY][TX]
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + D * Gm::STAGE_STRIDE + Gm::LVL_TOTAL);

  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    tma_prefetch_desc(&src_map);
    for (int s = 0; s < D; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // this thread's slot: vector column qc of rows R*qg .. R*qg + R-1 (threads
  // past the last slot duplicate it and store nothing)
  const bool qv = tid < NSLOT;
  const int qq = qv ? tid : NSLOT - 1;
  // x neighbours come from the adjacent lane (shuffles) where it holds the
  // adjacent column of the same rows; lsm / rsm: the left / right one is
  // read from shared memory instead (never both)
  int qg, qc;
  bool lsm, rsm;
  if constexpr (Gm::SPLIT) {
    constexpr int OXV = Gm::OXV, HXV = Gm::HXV, GA0 = Gm::GA0, GA1 = Gm::GA1;
    const int top = GA0 * TXV, bot = (Gm::TY / R - GA1) * TXV;
    if (qq < Gm::NA) {
      // output slots, OXV consecutive lanes per row group; the first and
      // last column's outer neighbours are halo slots
      qg = GA0 + qq / OXV;
      const int ic = qq % OXV;
      qc = HXV + ic;
      lsm = ic == 0;
      rsm = ic == OXV - 1;
    } else if (const int h = qq - Gm::NA; h < top + bot) {
      // whole halo rows (above, then below the output row groups), columns
      // in consecutive lanes: the warp-edge lanes read across the warp edge
      qg = h < top ? h / TXV : GA1 + (h - top) / TXV;
      qc = h < top ? h % TXV : (h - top) % TXV;
      lsm = lane == 0 && qc > 0;
      rsm = lane == 31 && qc < TXV - 1;
    } else {
      // the HXV halo columns each side of the output row groups: the one
      // neighbour that matters (towards the output columns) is read
      const int j = (h - top - bot) % (2 * HXV);
      qg = GA0 + (h - top - bot) / (2 * HXV);
      qc = j < HXV ? j : OXV + j;
      lsm = qc >= HXV + OXV;
      rsm = qc < HXV;
    }
  } else {
    qg = qq / TXV;
    qc = qq - qg * TXV;
    // the two warp-edge lanes read across the warp edge unless the
    // neighbour lies outside the tile
    lsm = lane == 0 && qc > 0;
    rsm = lane == 31 && qc < TXV - 1;
  }
  // a halo warp (warp-uniform: the output slots fill whole warps)
  const bool hw = Gm::SPLIT && tid >= Gm::NA;
  const int r0 = R * qg;
  const int nx = (int)g.nx, ny = (int)g.ny, nz = (int)g.nz;
  const int64_t plane_stride = g.pitch * g.ny;
  const C alpha = (C)g.alpha, beta = (C)g.beta;
  const bool esm = lsm || rsm;

  // Level l keeps its last three planes in a ring of register slots: at
  // iteration t slot t%3 holds plane Z+1 (newest), (t+2)%3 plane Z and
  // (t+1)%3 plane Z-1 of the stencil that forms level l+1 of plane Z.  The
  // plane loop is unrolled by U (a multiple of three) so that every slot
  // index is a constant.
  C ring[K][3][R][V];
#pragma unroll
  for (int l = 0; l < K; ++l)
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int e = 0; e < V; ++e) ring[l][s][i][e] = C(0);

  // Every item starts the TMA ring at stage 0 (the previous item consumed
  // all its loads), so plane t of an item sits in stage t % D; bit s of ph
  // is the parity of stage s's next completion.
  uint32_t ph = 0;
  // The next launch on the stream may start its setup now; this one touches
  // global memory only once the previous launch (whose output it reads and
  // whose input it overwrites) has completed.
  pdl_launch_dependents();
  pdl_wait();
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
        mbar_arrive_expect_tx(&bars[p], Gm::STAGE_BYTES);
        tma_load_3d(stage_ptr(p), &src_map, &bars[p], bx, by, lo0 + p);
      }
    }

    // Per-item facts of this slot.  Rows rlo / rhi of the tile are the
    // domain's y = 0 / y = ny-1 rows (clamped to the tile): their outer
    // neighbour is the row itself, the zero-Neumann ghost.
    const int rlo = max(0, -by), rhi = min(TY - 1, ny - 1 - by);
    const bool yface = rlo > 0 || rhi < TY - 1;
    const bool xedge = (bx <= 0) || (bx + TX > nx - 1);
    const int own = r0 * TX + qc * V;                 // row i at own + i * TX
    const int ysn = max(r0 - 1, rlo) * TX + qc * V;   // row below the group
    const int ynn = min(r0 + R, rhi) * TX + qc * V;   // row above the group
    const int eoff = esm ? own + (lsm ? -1 : V) : own;  // the x neighbour read from shared memory
    // The same places in the level buffers' layout.  Split layout: a
    // vector's first LV values in region 0, its last LV in region 1; the
    // left neighbour cell (last of the vector on the left) is the last value
    // of that vector's region-1 half, the right one (first of the vector on
    // the right) the first value of its region-0 half.
    constexpr int LROW = Gm::LROW, LHALF = Gm::LHALF, LV = Gm::LSPLIT ? V / 2 : V;
    const int lown = r0 * LROW + qc * LV;
    const int lysn = max(r0 - 1, rlo) * LROW + qc * LV;
    const int lynn = min(r0 + R, rhi) * LROW + qc * LV;
    int leoff = eoff;
    if constexpr (Gm::LSPLIT) leoff = !esm ? lown : lsm ? LHALF + lown - 1 : lown + LV;
    const int gx0 = bx + qc * V;
    const bool lfix = gx0 == 0;               // element 0 is the x = 0 face
    const bool rfix = gx0 + V - 1 == nx - 1;  // element V-1 is the x = nx-1 face
    const bool st_full = gx0 + V <= nx;
    const bool st_col = qv && qc >= Gm::HX / V && qc < (Gm::HX + Gm::OX) / V && gx0 < nx;
    bool st_row[R];
#pragma unroll
    for (int i = 0; i < R; ++i)
      st_row[i] = st_col && r0 + i >= K && r0 + i < K + Gm::OY && by + r0 + i < ny;
    const int64_t goff = (int64_t)(by + r0) * g.pitch + gx0;

    auto body = [&]<int P, bool BND>(int t) -> bool {
      // t % U == P: register-ring slots, TMA stages and level buffers
      constexpr int SN = P % 3, SB = (P + 2) % 3, SA = (P + 1) % 3;
      constexpr int SCUR = P % D, SPREV = (P + D - 1) % D;
      constexpr int LW = P % 3, LR = (P + 2) % 3;
      // Shared-memory reads of level 0: the stage of plane t-1 (level l >= 1
      // reads the level-l plane of the previous iteration in its own turn).
      // At t == 0 there is no plane t-1: that stage may still be receiving
      // the prologue's TMA load, so it is not read (the values would only
      // feed plane lo0-1, which lies outside every output cone).
      C ys[K][V], yn[K][V], ev[K][R];
      if (P != 0 || t > 0) {
        const T *cb = stage_ptr(SPREV);
        ld_vec<T, V>(cb, ysn, ys[0]);
        ld_vec<T, V>(cb, ynn, yn[0]);
#pragma unroll
        for (int i = 0; i < R; ++i) ev[0][i] = esm ? to_c(cb[eoff + i * TX]) : C(0);
      } else {
#pragma unroll
        for (int e = 0; e < V; ++e) ys[0][e] = yn[0][e] = C(0);
#pragma unroll
        for (int i = 0; i < R; ++i) ev[0][i] = C(0);
      }
      bool ok = true;
      if (!BND || t < n_in) {
        ok = mbar_wait_bounded(&bars[SCUR], (ph >> SCUR) & 1u);
        if (ok) ph ^= 1u << SCUR;  // (an expired wait keeps the parity for the drain)
        const T *stage = stage_ptr(SCUR);
#pragma unroll
        for (int i = 0; i < R; ++i) ld_vec<T, V>(stage, own + i * TX, ring[0][SN][i]);
      }
#pragma unroll
      for (int l = 0; l < K; ++l) {
        if (l == K - 1 && hw) break;  // halo warps: no last level
        if (l > 0) {
          const C *cb = lvl + ((l - 1) * 3 + LR) * PLANE;
          ld_lvl<Gm>(cb, lysn, ys[l]);
          ld_lvl<Gm>(cb, lynn, yn[l]);
#pragma unroll
          for (int i = 0; i < R; ++i) ev[l][i] = esm ? cb[leoff + i * LROW] : C(0);
        }
        const int Z = lo0 + t - (l + 1);  // plane of level l+1 formed now
        if constexpr (BND) {
          if (Z == 0) {                   // ghost below the bottom face
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
              for (int e = 0; e < V; ++e) ring[l][SA][i][e] = ring[l][SB][i][e];
          }
          if (Z == nz - 1) {              // ghost above the top face
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
              for (int e = 0; e < V; ++e) ring[l][SN][i][e] = ring[l][SB][i][e];
          }
        }
        const int ZK = lo0 + t - K;
        const bool store = (l == K - 1) && ZK >= z0 && ZK < z1;
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const C *mid = ring[l][SB][i];
          const C *sp = i == 0 ? ys[l] : ring[l][SB][i - 1];
          const C *np = i == R - 1 ? yn[l] : ring[l][SB][i + 1];
          // inside the group a domain y face is a select (y-face tiles only)
          const bool sself = BND && i > 0 && r0 + i == rlo;
          const bool nself = BND && i < R - 1 && r0 + i == rhi;
          const C sh_l = __shfl_up_sync(0xffffffffu, mid[V - 1], 1);
          const C sh_r = __shfl_down_sync(0xffffffffu, mid[0], 1);
          C wl = lsm ? ev[l][i] : sh_l;
          C er = rsm ? ev[l][i] : sh_r;
          if constexpr (FASTX) {
            wl = lfix ? mid[0] : wl;
            er = rfix ? mid[V - 1] : er;
          }
          C out[V];
#pragma unroll
          for (int e = 0; e < V; ++e) {
            const C p = mid[e];
            C w = (e == 0) ? wl : mid[e - 1];
            C ea = (e == V - 1) ? er : mid[e + 1];
            if constexpr (!FASTX) {
              if (xedge) {
                const int gx = gx0 + e;
                if (gx == 0) w = p;
                if (gx == nx - 1) ea = p;
              }
            }
            C sv = sp[e], nv = np[e];
            if constexpr (BND) {
              sv = sself ? p : sv;
              nv = nself ? p : nv;
            }
            const C nsum = ((w + ea) + (sv + nv)) + (ring[l][SA][i][e] + ring[l][SN][i][e]);
            out[e] = ac_update<C>(p, nsum, C(-6), alpha, beta);
          }
          if (l + 1 < K) {
#pragma unroll
            for (int e = 0; e < V; ++e) ring[l + 1 < K ? l + 1 : 0][SN][i][e] = out[e];
            if (qv) st_lvl<Gm>(lvl + (l * 3 + LW) * PLANE, lown + i * LROW, out);
          } else {
            // the address is formed by every thread and only the store is
            // predicated (one predicated 16-byte store, no branch)
            T *d = dst + (int64_t)ZK * plane_stride + goff + (int64_t)i * g.pitch;
            const bool sv = store && st_row[i];
            if (FASTX || st_full) {  // (FASTX: nx % V == 0, every vector is whole)
              st_vec_g<T, V>(d, out, sv);
            } else if (sv) {
#pragma unroll
              for (int e = 0; e < V; ++e)
                if (gx0 + e < nx) d[e] = from_c<T>(out[e]);
            }
          }
        }
      }

      // the plane barrier, which also tells every thread whether any
      // thread's wait expired
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          report_timeout(g.status);
          // loads that may be in flight: from plane t (t + 1 if thread 0
          // saw it land) up to D-1 (the prologue's) or t+D-2 (the last
          // refill; this iteration's was not issued)
          const int last = max(D - 1, t + D - 2);
          for (int p = ok ? t + 1 : t; p < n_in && p <= last; ++p)
            mbar_wait_bounded(&bars[p % D], (ph >> (p % D)) & 1u);
        }
        return false;
      }
      // the stage of plane t-1 is no longer read: refill it with plane t-1+D
      if (tid == 0 && t >= 1 && t - 1 + D < n_in) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bars[SPREV], Gm::STAGE_BYTES);
        tma_load_3d(stage_ptr(SPREV), &src_map, &bars[SPREV], bx, by, lo0 + t - 1 + D);
      }
      return true;
    };

    // Iterations that touch a z face (ghost copies) or run past the last
    // input plane take the BND body: t in [1, K] when the chunk starts at
    // z = 0, and t >= nz - lo0 when it ends at the top face; so does every
    // iteration of a tile that holds a y face.
    const int bnd_lo_end = (lo0 == 0) ? K : -1;
    const int bnd_hi_begin = (hi0 == nz) ? nz - lo0 - 1 : n_iter;
    int t = 0;
    for (; t + U <= n_iter; t += U) {
      const bool bnd = yface || (t <= bnd_lo_end) || (t + U - 1 >= bnd_hi_begin);
      if (bnd) {
        if (!body.template operator()<0, true>(t)) return;
        if (!body.template operator()<1, true>(t + 1)) return;
        if (!body.template operator()<2, true>(t + 2)) return;
        if constexpr (U == 6) {
          if (!body.template operator()<3, true>(t + 3)) return;
          if (!body.template operator()<4, true>(t + 4)) return;
          if (!body.template operator()<5, true>(t + 5)) return;
        }
      } else {
        if (!body.template operator()<0, false>(t)) return;
        if (!body.template operator()<1, false>(t + 1)) return;
        if (!body.template operator()<2, false>(t + 2)) return;
        if constexpr (U == 6) {
          if (!body.template operator()<3, false>(t + 3)) return;
          if (!body.template operator()<4, false>(t + 4)) return;
          if (!body.template operator()<5, false>(t + 5)) return;
        }
      }
    }
    // the remaining t % U planes (t is a multiple of U here)
    if (t < n_iter && !body.template operator()<0, true>(t++)) return;
    if (t < n_iter && !body.template operator()<1, true>(t++)) return;
    if constexpr (U == 6) {
      if (t < n_iter && !body.template operator()<2, true>(t++)) return;
      if (t < n_iter && !body.template operator()<3, true>(t++)) return;
      if (t < n_iter && !body.template operator()<4, true>(t++)) return;
    }
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
  static KernelSetup ks;
  int occ = 1;
  cudaError_t e = kernel_setup(ks, (const void *)stream3d_k<T, K, FASTX, TILE>, Gm::NT, Gm::SMEM, &occ);
  if (e != cudaSuccess) return e;
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
  // programmatic stream serialization (one CTA per SM only): the launch
  // overlaps the tail of the previous stencil launch on the stream (see
  // pdl_wait in the kernel).  Measured on GB300 at 512^3: +1.1 % for launches
  // issued one by one (FP32 tile 0), no change under graph replay, and -2.7 %
  // for the two-CTA FP16 tile 1, which therefore launches without it.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(Gm::NT);
  cfg.dynamicSmemBytes = Gm::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = Gm::MINB == 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, stream3d_k<T, K, FASTX, TILE>, *map, (T *)dst, g, tiles_x, tiles_y,
                            nzc, zchunk);
}

// Dispatch over the supported depths and tiles of one storage type.
template <typename T, int TILE>
cudaError_t s3_dispatch_tile(int k, const GridParams &g, const CUtensorMap *map, void *dst,
                             int num_sms, cudaStream_t s) {
  const bool fastx = g.nx % S3Cfg<T, TILE>::VL == 0;
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
