// Float64-accurate rank-32 update C -= D E^T on the tensor cores, for the
// trailing update of the SPD inverse of the Dyson solve.
//
// Every row of D and of E (32 float64 values) is scaled by a power of two,
// x = 2^e a with |a| < 1/2, and cut into integer slices
//   a = sum_{t=1..7} 2^(-8 t) s_t   (base-256 digits of round(a 2^56)),
// |s_t| <= 128: each slice is exact in bf16 and the representation error is
// at most 2^-56 2^e (oz_slice.cuh).  The products of the 28 slice pairs with
// t + u <= 8 are issued as bf16 tcgen05 MMAs (K = 32, two K16 steps each) into
// seven fp32 accumulators in TMEM, one per level t + u.  A level sum is an
// integer of magnitude at most 7 * 32 * 2^14 < 2^22, hence exact in fp32.
// The epilogue combines the levels as 64-bit integers, rounds the product to
// float64 with integer instructions (oz_combine.cuh) and subtracts it from C.
// The dropped pairs (t + u >= 9) bound the error by about 6e-16 |D|max |E|max
// per element, on a par with a float64 dot product of 32 terms; the update
// runs at tensor-core speed instead of the 2 DFMA per SM per clock of the
// float64 pipe.
//
// Tiles of 128 x 64 elements of the lower triangle; elements in the rows or
// columns of the excluded pivot blocks (the side stream of the SPD inverse
// updates those) are left untouched.
#include <cuda_bf16.h>

#include <cmath>

#include "lrs_internal.h"
#include "oz_combine.cuh"
#include "oz_slice.cuh"
#include "tc_common.cuh"

namespace lrs {
using namespace tc;

constexpr int OZ_SLICES = OZ_SLICE_COUNT;
constexpr int OZ_PLANES = OZ_PLANE_COUNT;      // two slices per 128-byte row (the last half of plane 3 is zero)
constexpr int OZ_LEVELS = 7;                   // t + u = 2 .. 8
constexpr int OZ_TM = 128, OZ_TN = 64;
constexpr int OZ_A_PLANE = OZ_TM * 128;        // bytes of one A plane tile
constexpr int OZ_B_PLANE = OZ_TN * 128;
constexpr int OZ_STAGE = OZ_PLANES * (OZ_A_PLANE + OZ_B_PLANE);
constexpr int OZ_STAGES = 1;
constexpr int OZ_EPI_WARPS = 16;               // four per TMEM lane quarter, 16 columns each
constexpr int OZ_EPI_COLS = OZ_TN / (OZ_EPI_WARPS / 4);
constexpr int OZ_STG_LD = OZ_EPI_COLS + 1;      // padded row of a warp's staging tile
constexpr int OZ_STAGE_EPI = OZ_EPI_WARPS * 32 * OZ_STG_LD * 8;   // per-warp [32][17] float64 staging of C
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE + OZ_STAGE_EPI + 1024;
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;   // producer, MMA issuer, epilogue warps
constexpr int OZ_TMEM_COLS = 512;              // 7 levels x 64 columns used

struct OzUpdate {
  double* C;
  int n, ldc;
  const int* ed;        // row exponents of D (output rows)
  const int* ee;        // row exponents of E (output columns)
  int x0, x1;           // rows / columns in [x0, x1) are left to the side stream
  int row_tiles, col_tiles;
  int a_plane_rows, b_plane_rows;   // padded rows of one plane (row offset between planes)
};

__device__ __forceinline__ bool oz_decode(const OzUpdate& p, int u, int& bi, int& bj) {
  bi = u / p.col_tiles;
  bj = u % p.col_tiles;
  return bj * OZ_TN <= bi * OZ_TM + OZ_TM - 1;   // tile reaches the lower triangle
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_update_kernel(const __grid_constant__ CUtensorMap tmD, const __grid_constant__ CUtensorMap tmE,
                     const OzUpdate p, int* status) {
  __shared__ __align__(8) uint64_t full_bar[OZ_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[OZ_STAGES];
  __shared__ __align__(8) uint64_t accf_bar;
  __shared__ __align__(8) uint64_t acce_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  extern __shared__ uint8_t oz_smem_raw[];
  const uint32_t smem_base = (smem_u32(oz_smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = p.row_tiles * p.col_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&accf_bar, 1);
    mbar_init(&acce_bar, OZ_EPI_WARPS);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_map(&tmD);
    tma_prefetch_map(&tmE);
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base, OZ_TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer: all slice planes of a tile
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      for (int u = blockIdx.x; u < units; u += gridDim.x) {
        int bi, bj;
        if (!oz_decode(p, u, bi, bj)) continue;
        if (!mbar_wait(&empty_bar[stage], phase ^ 1u, &abort_flag)) {
          abort_flag = 1;
          atomicCAS(status, 0, TC_TIMEOUT_PRODUCER);
          break;
        }
        mbar_arrive_expect_tx(&full_bar[stage], OZ_STAGE);
        const uint32_t s = smem_base + stage * OZ_STAGE;
        for (int q = 0; q < OZ_PLANES; ++q) {
          tma_load_2d(s + q * OZ_A_PLANE, &tmD, &full_bar[stage], 0, q * p.a_plane_rows + bi * OZ_TM);
          tma_load_2d(s + OZ_PLANES * OZ_A_PLANE + q * OZ_B_PLANE, &tmE, &full_bar[stage], 0,
                      q * p.b_plane_rows + bj * OZ_TN);
        }
        if (++stage == OZ_STAGES) { stage = 0; phase ^= 1u; }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issue: 28 slice pairs x 2 K16 steps
    if (lane == 0) {
      constexpr uint32_t ID = idesc_f16(OZ_TM, OZ_TN, 1, false);
      int stage = 0;
      uint32_t phase = 0, acc_phase = 0;
      for (int u = blockIdx.x; u < units; u += gridDim.x) {
        int bi, bj;
        if (!oz_decode(p, u, bi, bj)) continue;
        if (!mbar_wait(&acce_bar, acc_phase ^ 1u, &abort_flag) || !mbar_wait(&full_bar[stage], phase, &abort_flag)) {
          abort_flag = 1;
          atomicCAS(status, 0, TC_TIMEOUT_MMA);
          break;
        }
        tc_fence_after();
        const uint32_t s = smem_base + stage * OZ_STAGE;
        const uint32_t sa = s, sb = s + OZ_PLANES * OZ_A_PLANE;
#pragma unroll
        for (int t = 0; t < OZ_SLICES; ++t) {
#pragma unroll
          for (int v = 0; v < OZ_SLICES; ++v) {
            if (t + v > OZ_SLICES - 1) continue;                 // keep t + u <= 8 (1-based)
            const uint32_t d = tbase + (t + v) * OZ_TN;
            const uint32_t ao = sa + (t >> 1) * OZ_A_PLANE + (t & 1) * 64;
            const uint32_t bo = sb + (v >> 1) * OZ_B_PLANE + (v & 1) * 64;
            // pairs are issued t-major, so (0, level) is the first product into each level
            const uint32_t first = (t == 0) ? 0u : 1u;
            mma_f16(d, sw128_desc(ao), sw128_desc(bo), ID, first);
            mma_f16(d, sw128_desc(ao + 32), sw128_desc(bo + 32), ID, 1u);
          }
        }
        mma_commit(&empty_bar[stage]);
        mma_commit(&accf_bar);
        if (++stage == OZ_STAGES) { stage = 0; phase ^= 1u; }
        acc_phase ^= 1u;
      }
    }
  } else {
    // ------------------------------------------------ epilogue: combine the levels, C -= D E^T
    // Each warp owns 32 rows (its TMEM lane quarter) x 16 columns of the tile.  Its
    // share of C is copied into a [32][17] shared-memory stage (cp.async) before the
    // accumulators are ready, so the memory latency overlaps the MMAs.  Level sums S_L
    // (integers of magnitude below 2^22 in fp32, read as int32 by one fp32 add each)
    // are combined into one 64-bit integer in units of 2^-56 of the scaled product,
    //   V = S_0 2^40 + S_1 2^32 + S_2 2^24 + S_3 2^16 + S_4 2^8 + S_5 + floor(S_6 / 2^8)
    // (|V| < 2^60; the floor drops less than 2^-56 of the row scales' product), so
    // the product is 2^(e_i + f_j - 56) V, rounded to float64 with integer
    // instructions and subtracted from the staged C (the only float64 operation per
    // element).  TMEM is then released to the next tile's MMAs, and the stage is
    // written back, two rows of 16 columns per instruction.
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int cg = ew >> 2;                      // column group of 16
    const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
    double* stg = reinterpret_cast<double*>(oz_smem_raw + (smem_base - smem_u32(oz_smem_raw)) +
                                            OZ_STAGES * OZ_STAGE) + ew * 32 * OZ_STG_LD;
    const uint32_t stg_s = smem_u32(stg);
    const int wc = lane & 15, wr = lane >> 4;    // this lane's column and row parity when C moves
    uint32_t acc_phase = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
      int bi, bj;
      if (!oz_decode(p, u, bi, bj)) continue;
      const int row0 = bi * OZ_TM + quarter * 32;
      const int col0 = bj * OZ_TN + cg * OZ_EPI_COLS;
      const int j = col0 + wc;
      const bool col_ok = j < p.n && !(j >= p.x0 && j < p.x1);
      // rows r of this warp's 32 that this lane's column takes: inside the matrix, outside the
      // pivot blocks [x0, x1), and on or below the diagonal (row0 + r >= j)
      const int my_i = row0 + lane;
      const unsigned rows_in = __ballot_sync(0xffffffffu, my_i < p.n && !(my_i >= p.x0 && my_i < p.x1));
      const int rmin = j - row0;
      const unsigned lower = rmin <= 0 ? 0xffffffffu : (rmin >= 32 ? 0u : (0xffffffffu << rmin));
      const unsigned take = col_ok ? (rows_in & lower) : 0u;
#pragma unroll 4
      for (int r = wr; r < 32; r += 2) {
        if ((take >> r) & 1u)
          cp_async8(stg_s + (uint32_t)(r * OZ_STG_LD + wc) * 8u, p.C + (size_t)(row0 + r) * p.ldc + j);
      }
      cp_async_commit();
      // the row scale of this lane's TMEM row and the column scales of the 16 columns
      const int my_row = row0 + lane;
      const int ei = my_row < p.n ? p.ed[my_row] : 0;
      const int fj_lane = (col0 + wc) < p.n ? p.ee[col0 + wc] : 0;
      int got = 1;
      if (lane == 0) got = mbar_wait(&accf_bar, acc_phase, &abort_flag) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      if (!got) {
        cp_async_wait_all();
        if (lane == 0) {
          abort_flag = 1;
          atomicCAS(status, 0, TC_TIMEOUT_EPILOGUE);
        }
        break;
      }
      tc_fence_after();
      cp_async_wait_all();
      __syncwarp();
#pragma unroll
      for (int ch = 0; ch < OZ_EPI_COLS / 8; ++ch) {
        float a[OZ_LEVELS][8];
#pragma unroll
        for (int lv = 0; lv < OZ_LEVELS; ++lv)
          tmem_ld8(tbase + lane_off + lv * OZ_TN + cg * OZ_EPI_COLS + ch * 8, a[lv]);
        tmem_ld_wait();
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          // |S_L| < 2^22: pairs of levels combine exactly in int32 before one 64-bit assembly
          const int t3 = oz_pair<8>(oz_level_bits(a[0][c]), oz_level_bits(a[1][c]));
          const int t2 = oz_pair<8>(oz_level_bits(a[2][c]), oz_level_bits(a[3][c]));
          const int t1 = oz_pair<8>(oz_level_bits(a[4][c]), oz_level_bits(a[5][c])) +
                         oz_level_shr<8>(oz_level_bits(a[6][c]));
          const long long V = ((long long)t3 << 32) + ((long long)t2 << 16) + (long long)t1;
          const int fj = __shfl_sync(0xffffffffu, fj_lane, ch * 8 + c);
          double* q = stg + lane * OZ_STG_LD + ch * 8 + c;
          // entries of the stage outside the update hold stale values and are not written back
          *q = *q - oz_i64_times_pow2(V, ei + fj - 56);
        }
      }
      // the accumulators have been read: the next tile's MMAs may start
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce_bar);
      acc_phase ^= 1u;
#pragma unroll 4
      for (int r = wr; r < 32; r += 2) {
        if ((take >> r) & 1u) p.C[(size_t)(row0 + r) * p.ldc + j] = stg[r * OZ_STG_LD + wc];
      }
      __syncwarp();
    }
  }
  // teardown: every role has finished or given up; wait for the others before freeing TMEM
  tc_fence_before();
  __syncthreads();
  if (abort_flag) {
    // let copies and MMAs already issued land before the shared memory and TMEM go away
    const uint64_t t0 = global_timer_ns();
    while (global_timer_ns() - t0 < 200000ull) {
    }
  }
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, OZ_TMEM_COLS);
  }
}

int oz_make_maps(lrs_ctx* ctx, const uint16_t* dplanes, const uint16_t* eplanes, int rows_pad, CUtensorMap* md,
                 CUtensorMap* me) {
  LRS_TRY(make_operand_map(md, dplanes, 64, (uint64_t)OZ_PLANES * rows_pad, OZ_TM));
  return make_operand_map(me, eplanes, 64, (uint64_t)OZ_PLANES * rows_pad, OZ_TN);
}

int oz_update(lrs_ctx* ctx, const CUtensorMap& md, const CUtensorMap& me, double* C, int n, int ldc,
              const int* ed, const int* ee, int x0, int x1, int rows_pad, cudaStream_t stream) {
  OzUpdate p;
  p.C = C;
  p.n = n;
  p.ldc = ldc;
  p.ed = ed;
  p.ee = ee;
  p.x0 = x0;
  p.x1 = x1;
  p.row_tiles = (n + OZ_TM - 1) / OZ_TM;
  p.col_tiles = (n + OZ_TN - 1) / OZ_TN;
  p.a_plane_rows = rows_pad;
  p.b_plane_rows = rows_pad;
  if (!ctx->capturing)
    LRS_CUDA_TRY(cudaFuncSetAttribute(oz_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
  const int grid = std::min(p.row_tiles * p.col_tiles, ctx->num_sms);
  oz_update_kernel<<<grid, OZ_THREADS, OZ_SMEM, stream>>>(md, me, p, ctx->ws.status.ptr + 8);
  return after_launch(ctx, "oz_update_kernel");
}

int oz_rows_pad(int n) { return (n + OZ_TM - 1) / OZ_TM * OZ_TM; }
size_t oz_plane_elems(int n) { return (size_t)OZ_PLANES * oz_rows_pad(n) * 64; }

}  // namespace lrs
