// Row-streaming tensor-core convolution of the jump network (the 32 -> 32
// layers, forward and data gradient):
//
//   out[p][n] = sum_{t < T} sum_{c < 32} in[p + t][c] * Wx[n][t*32 + c]
//
// Work item: 128 consecutive x positions of a run of output rows (one z, one
// image).  The input rows reach shared memory once each, by TMA, and stay in
// a ring while the three output rows that use them are formed:
//   - layout of one padded input row: 4 planes of 8 channels, each plane the
//     130 pixels x0-1 .. x0+128 at 16 bytes per pixel (one 2D TMA box of
//     8 channels x 130 pixels), so that pixel m sits at 16 m bytes; an x
//     offset of a tap is then +16 bytes on the descriptor's start address
//     (canonical K-major layout without swizzle: LBO = plane stride between
//     the K-adjacent 8-channel core matrices, SBO = 128 bytes between 8-pixel
//     groups);
//   - warp 0 (one thread) issues the TMA loads into a ring of row sets (the
//     1 or 3 rows of one y at every needed z), each set on a full / empty
//     mbarrier pair;
//   - warps 1 and 6 (one thread each, alternate output rows) issue T x 2
//     tcgen05.mma (M = 128 pixels, N = 32, K = 16) per output row into one
//     of their two TMEM accumulators and commit to the accumulator's
//     barrier and to the empty barriers of the sets this issuer no longer
//     reads (each set is released once by each issuer);
//   - warps 2..5 read the accumulator (tcgen05.ld, lanes 32 (w % 4) ..),
//     release it, and run the epilogue: bias, pre-activation store, GELU
//     (tanh form, hardware tanh approximation) and the store with its
//     replicated ghost ring; or the raw FP32 store of the data gradient.
// Every wait is bounded; a timeout sets the status word and the roles wind
// down without leaving copies or MMAs in flight.
#include "kernels.h"
#include "net.cuh"
#include "tc.cuh"

namespace ac {

namespace {

constexpr int kCvPix = 130;                // 128 outputs + 2 halo columns
constexpr int kCvPlane = 136 * 16;         // bytes of one 8-channel plane (rows padded to 136)
constexpr int kCvRow = 4 * kCvPlane;       // one padded input row (32 channels)
constexpr int kCvBox = 8 * kCvPix * 2;     // bytes of one TMA box
constexpr int kCvThreads = 224;  // TMA warp, 2 MMA warps, 4 epilogue warps
constexpr int kCvIssuers = 2;    // MMA-issuing warps (alternate output rows)

template <int NDIM>
struct CvGeom {
  static constexpr int NZ = NDIM == 3 ? 3 : 1;       // rows per set (z - 1, z, z + 1)
  static constexpr int NS = NDIM == 3 ? 6 : 8;       // sets in the ring
  static constexpr int MINB = NDIM == 3 ? 1 : 2;     // CTAs per SM
  static constexpr int NACC = 4;                      // TMEM accumulators (2 per issuer)
  static constexpr int T = net_taps(NDIM);
  static constexpr int KB = T * kNetC;                // GEMM K
  static constexpr int KCB = KB / 8;                  // 8-element K chunks of B
  static constexpr int SET = NZ * kCvRow;
  static constexpr int OFF_A = (64 * KB + 1023) / 1024 * 1024;
  static constexpr int OFF_BAR = OFF_A + NS * SET;
  // full[NS], empty[NS], accf[NACC], acce[NACC], fin; the TMEM slot and
  // abort word; the 32 biases
  static constexpr int OFF_BIAS = OFF_BAR + (2 * NS + 2 * NACC + 1) * 8 + 16;
  static constexpr int SMEM = OFF_BIAS + 32 * 4;
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

struct CvItem {
  int b, z, x0, ya, nrows;
};

__device__ __forceinline__ CvItem cv_item(int64_t item, const NetShape &sh, int tiles_x, int nchunk,
                                          int chunk) {
  CvItem it;
  const int tx = (int)(item % tiles_x);
  int64_t r = item / tiles_x;
  const int yc = (int)(r % nchunk);
  r /= nchunk;
  it.z = (int)(r % sh.nz);
  it.b = (int)(r / sh.nz);
  it.x0 = tx * 128;
  it.ya = yc * chunk;
  it.nrows = min(chunk, sh.ny - it.ya);
  return it;
}

}  // namespace

// MODE 0: forward epilogue (bias, zout, GELU, replicated store into outpad);
// MODE 1: raw FP32 output (the data gradient before its finishing pass).
template <int NDIM, int MODE>
__global__ void __launch_bounds__(kCvThreads, CvGeom<NDIM>::MINB)
    net_conv_rows_k(const __grid_constant__ CUtensorMap in_map, const bf16 *__restrict__ Wx,
                    const float *__restrict__ bias, NetShape sh, int chunk, bf16 *__restrict__ zout,
                    bf16 *__restrict__ outpad, float *__restrict__ outraw, int *status) {
  using Gm = CvGeom<NDIM>;
  constexpr int NS = Gm::NS, NZ = Gm::NZ, T = Gm::T, KCB = Gm::KCB, KB = Gm::KB;
  constexpr int NACC = Gm::NACC;
  constexpr uint32_t idesc = tc_idesc_bf16_f32(128, 32);
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char *sB = sm;
  unsigned char *sA = sm + Gm::OFF_A;
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + Gm::OFF_BAR);
  uint64_t *empty = full + NS;
  uint64_t *accf = empty + NS;
  uint64_t *acce = accf + NACC;
  uint64_t *fin = acce + NACC;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(fin + 1);
  volatile int &abort_flag = *reinterpret_cast<volatile int *>(tslot + 1);
  float *sbias = reinterpret_cast<float *>(sm + Gm::OFF_BIAS);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < 32) sbias[tid] = MODE == 0 ? bias[tid] : 0.0f;

  // B operand (32 x KB, canonical K-major) for the CTA's lifetime
  for (int i = tid; i < 32 * KCB; i += kCvThreads) {
    const int n = i / KCB, c = i - n * KCB;
    *reinterpret_cast<uint4 *>(sB + tc_kmajor_off(n, c * 8, KCB)) =
        *reinterpret_cast<const uint4 *>(Wx + (int64_t)n * KB + c * 8);
  }
  if (tid == 0) {
    tma_prefetch_desc(&in_map);
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kCvIssuers);  // each issuer releases every set once
    }
    for (int a = 0; a < NACC; ++a) {
      mbar_init(&accf[a], 1);
      mbar_init(&acce[a], 4);
    }
    mbar_init(fin, kCvIssuers);
    fence_mbar_init();
    abort_flag = 0;
  }
  if (warp == 1) {
    tmem_alloc(tslot, 32 * NACC);
    tmem_relinquish();
  }
  fence_proxy_async_smem();  // B (generic writes) before the MMAs read it
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const int tiles_x = (sh.nx + 127) / 128;
  const int nchunk = (sh.ny + chunk - 1) / chunk;
  const int64_t items = (int64_t)sh.batch * sh.nz * nchunk * tiles_x;

  if (warp == 0) {
    // ---------------------------------------------------------- TMA loads --
    if (lane == 0) {
      uint32_t i = 0;  // row sets issued
      bool ok = true;
      for (int64_t item = blockIdx.x; item < items && ok; item += gridDim.x) {
        const CvItem it = cv_item(item, sh, tiles_x, nchunk, chunk);
        for (int r = 0; r < it.nrows + 2 && ok; ++r, ++i) {
          const int s = (int)(i % NS);
          if (i >= (uint32_t)NS && !mbar_wait_bounded(&empty[s], ((i / NS) - 1) & 1u)) {
            ok = false;
            break;
          }
          if (abort_flag) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[s], NZ * 4 * kCvBox);
          for (int dz = 0; dz < NZ; ++dz) {
            // padded row (z + dz, ya + r) from padded column x0 (= cell x0 - 1)
            const int64_t p0 = sh.p(it.b, NDIM == 3 ? it.z + dz : 0, it.ya + r, it.x0);
            for (int kc = 0; kc < 4; ++kc)
              tma_load_2d(sA + s * Gm::SET + dz * kCvRow + kc * kCvPlane, &in_map, &full[s],
                          kc * 8, (int)p0);
          }
        }
      }
      if (!ok && !abort_flag) {
        report_timeout(status);
        abort_flag = 1;
      }
      // never leave with a copy in flight
      for (uint32_t v = i > (uint32_t)NS ? i - NS : 0; v < i; ++v)
        mbar_wait_bounded(&full[v % NS], (v / NS) & 1u);
    }
  } else if (warp == 1 || warp == 6) {
    // ------------------------------------------------------------- MMAs --
    // Issuer p takes the item's output rows j = p, p + 2, ...; its k-th row
    // goes to accumulator p + 2 (k % 2).  It releases set j and j + 1 after
    // row j (their last use by this issuer); the item's other sets are
    // released before its first row (those it never reads) or after its
    // last row (the rest).
    const int p = warp == 6 ? 1 : 0;
    if (lane == 0) {
      const uint64_t a_desc0 = tc_smem_desc(sA, kCvPlane, 128);       // A rows: LBO plane, SBO 8 px
      const uint64_t b_desc0 = tc_smem_desc(sB, 128, KCB * 128);      // B: canonical K-major
      uint32_t i = 0, kq = 0;  // row sets consumed (CTA), rows formed by this issuer
      bool ok = true;
      for (int64_t item = blockIdx.x; item < items && ok; item += gridDim.x) {
        const CvItem it = cv_item(item, sh, tiles_x, nchunk, chunk);
        const uint32_t base = i;
        const bool had = it.nrows > p;
        // sets this issuer never reads are released before its first row:
        // those below it (all of them if it has no row in this item), so
        // the producer can refill their slots while the other issuer works.
        // Each release waits for the set to be loaded first: only then has
        // the slot's previous phase completed, so the arrival counts for
        // this set and not for the slot's previous occupant.
        for (int r = 0; r <= it.nrows + 1 && ok; ++r)
          if (!had || r < p) {
            const uint32_t k = base + r;
            if (!mbar_wait_bounded(&full[k % NS], (k / NS) & 1u)) ok = false;
            else mbar_arrive(&empty[k % NS]);
          }
        for (int j = p; j < it.nrows && ok; j += kCvIssuers, ++kq) {
          for (uint32_t k = base + j; k <= base + j + 2; ++k)
            if (!mbar_wait_bounded(&full[k % NS], (k / NS) & 1u)) ok = false;
          const uint32_t buf = p + kCvIssuers * (kq % 2);
          if (kq >= 2 && !mbar_wait_bounded(&acce[buf], ((kq / 2) - 1) & 1u)) ok = false;
          if (!ok || abort_flag) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + buf * 32;
          // descriptors: the start-address field is addr >> 4 in the low 14
          // bits, so a byte offset off (16-byte multiple, inside shared
          // memory) is + off >> 4 on the base descriptor
          uint32_t srow[3];
#pragma unroll
          for (int dy = 0; dy < 3; ++dy) srow[dy] = ((base + j + dy) % NS) * (Gm::SET >> 4);
#pragma unroll
          for (int t = 0; t < T; ++t) {
            const int ox = t % 3 - 1, oy = (t / 3) % 3 - 1, dz = NDIM == 3 ? t / 9 : 0;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              const uint64_t da = a_desc0 + srow[oy + 1] +
                                  (uint32_t)((dz * kCvRow + (ox + 1) * 16 + 2 * kk * kCvPlane) >> 4);
              const uint64_t db = b_desc0 + (uint32_t)(((t * 4 + kk * 2) * 128) >> 4);
              tc_mma_bf16(d, da, db, idesc, (t | kk) != 0);
            }
          }
          tc_commit(&accf[buf]);
          tc_commit(&empty[(base + j) % NS]);      // this issuer's last use of set j
          tc_commit(&empty[(base + j + 1) % NS]);  // and of set j + 1
        }
        if (!ok) break;
        // the sets above its last row + 1, once that row's MMAs completed
        // (and, as above, once the set is loaded)
        if (had) {
          const int last = it.nrows - 1 - ((it.nrows - 1 - p) % kCvIssuers + kCvIssuers) % kCvIssuers;
          for (int r = last + 2; r <= it.nrows + 1 && ok; ++r) {
            const uint32_t k = base + r;
            if (!mbar_wait_bounded(&full[k % NS], (k / NS) & 1u)) ok = false;
            else tc_commit(&empty[k % NS]);
          }
        }
        if (!ok) break;
        i = base + it.nrows + 2;
      }
      if (!ok && !abort_flag) {
        report_timeout(status);
        abort_flag = 1;
      }
      // every MMA issued has completed before the accumulator is freed
      tc_commit(fin);
      mbar_wait_bounded(fin, 0);
    }
  } else {
    // -------------------------------------------------------- epilogue --
    const int q = warp & 3;  // TMEM lane quarter of this warp
    uint32_t kq[kCvIssuers] = {};  // rows formed so far by each issuer
    bool ok = true;
    for (int64_t item = blockIdx.x; item < items && ok; item += gridDim.x) {
      const CvItem it = cv_item(item, sh, tiles_x, nchunk, chunk);
      for (int j = 0; j < it.nrows; ++j) {
        const int ip = j % kCvIssuers;  // the issuer of this row and its accumulator
        const uint32_t buf = ip + kCvIssuers * (kq[ip] % 2);
        const uint32_t par = (kq[ip] / 2) & 1u;
        ++kq[ip];
        const bool got = mbar_wait_bounded(&accf[buf], par);
        if (__any_sync(0xffffffffu, !got || abort_flag)) {  // the warp leaves together
          ok = false;
          break;
        }
        tc_fence_after();
        float v[32];
        tmem_ld32(tmem + buf * 32 + ((uint32_t)(q * 32) << 16), v);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[buf]);
        const int x = it.x0 + q * 32 + lane;
        const int y = it.ya + j;
        if (x < sh.nx) {
          const int64_t pu = sh.u(it.b, it.z, y, x);
          if (MODE == 0) {
#pragma unroll
            for (int c = 0; c < 32; ++c) v[c] += sbias[c];
            if (zout) {
              uint4 *dz = reinterpret_cast<uint4 *>(zout + pu * kNetC);
#pragma unroll
              for (int c = 0; c < 4; ++c) dz[c] = pack8_bf16(v + 8 * c);
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) v[c] = net_gelu_fast(v[c]);
            store_replicated<NDIM>(outpad, sh, it.b, it.z, y, x, v);
          } else {
            float4 *d = reinterpret_cast<float4 *>(outraw + pu * kNetC);
#pragma unroll
            for (int c = 0; c < 8; ++c)
              d[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
          }
        }
      }
    }
    if (!ok && lane == 0 && !abort_flag) {
      report_timeout(status);
      abort_flag = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 32 * NACC);
}

// ------------------------------------------------------------------ host ---
template <int NDIM, int MODE>
static cudaError_t conv_rows_t(const bf16 *in, const bf16 *Wx, const float *bias,
                               const NetShape &sh, bf16 *zout, bf16 *outpad, float *outraw,
                               int *status, int num_sms, cudaStream_t s) {
  using Gm = CvGeom<NDIM>;
  static KernelSetup ks;
  int occ = 1;
  cudaError_t e0 = kernel_setup(ks, (const void *)net_conv_rows_k<NDIM, MODE>, kCvThreads, Gm::SMEM,
                                &occ, 100);
  if (e0 != cudaSuccess) return e0;
  // the register budget of __launch_bounds__ guarantees MINB CTAs per SM
  // (the shared memory fits as well); the query may report fewer
  occ = std::max(occ, Gm::MINB);
  // the padded activations as a 2D tensor {32 channels, padded pixels}
  const int64_t P = sh.padded_cells();
  if (P + 2 * kCvPix >= (int64_t)INT32_MAX) return cudaErrorInvalidValue;
  EncodeTiledFn fn = ac_encode_fn();
  if (!fn) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)kNetC, (cuuint64_t)P};
  const cuuint64_t strides[1] = {(cuuint64_t)kNetC * 2};
  const cuuint32_t box[2] = {8, (cuuint32_t)kCvPix}, es[2] = {1, 1};
  if (fn(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(in), dims, strides, box, es,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  // rows per item: about two items per resident CTA, at least 4 rows (each
  // item loads its rows + 2)
  const int64_t slots = (int64_t)std::max(1, num_sms) * occ;
  const int64_t columns = (int64_t)sh.batch * sh.nz * ((sh.nx + 127) / 128);
  int chunk = (int)std::min<int64_t>(sh.ny, std::max<int64_t>(4, (columns * sh.ny + 2 * slots - 1) / (2 * slots)));
  const int nchunk = (sh.ny + chunk - 1) / chunk;
  const int64_t items = columns * nchunk;
  const int grid = (int)std::min<int64_t>(items, slots);
  net_conv_rows_k<NDIM, MODE><<<grid, kCvThreads, Gm::SMEM, s>>>(map, Wx, bias, sh, chunk, zout,
                                                                  outpad, outraw, status);
  return cudaGetLastError();
}

cudaError_t net_conv_rows(int mode, const bf16 *in, const bf16 *Wx, const float *bias,
                          const NetShape &sh, bf16 *zout, bf16 *outpad, float *outraw, int *status,
                          int num_sms, cudaStream_t s) {
  if (sh.ndim == 3)
    return mode == 0 ? conv_rows_t<3, 0>(in, Wx, bias, sh, zout, outpad, outraw, status, num_sms, s)
                     : conv_rows_t<3, 1>(in, Wx, bias, sh, zout, outpad, outraw, status, num_sms, s);
  return mode == 0 ? conv_rows_t<2, 0>(in, Wx, bias, sh, zout, outpad, outraw, status, num_sms, s)
                   : conv_rows_t<2, 1>(in, Wx, bias, sh, zout, outpad, outraw, status, num_sms, s);
}

}  // namespace ac
