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
// Tiles of 64 rows x 128 columns of C, transposed on the tensor cores: the MMA's M
// side (the 128 TMEM lanes) runs along the columns j (rows of E) and its N side (64
// TMEM columns per level) along the rows i (rows of D).  A warp's 32 lanes then hold
// 32 consecutive columns of one row of the row-major C and read and write it in
// 256-byte lines, with no staging of the result.  Every level accumulator starts with
// one product of constant tiles (1.0 times 1.5 2^19 over K = 16), so it holds the level
// sum plus 1.5 2^23 and its bits are read directly as a biased integer.  The epilogue
// packs the seven levels of its elements into 64-bit integers and releases TMEM before
// rounding them, so the next tile's MMAs run under the rounding and the float64
// subtractions.  Elements in the rows or columns of the excluded pivot blocks (the
// side stream of the SPD inverse updates those) and above the diagonal are left
// untouched.
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
constexpr int OZ_TJ = 128, OZ_TI = 64;         // columns (MMA M, TMEM lanes) and rows (MMA N) of a tile
constexpr int OZ_A_PLANE = OZ_TJ * 128;        // bytes of one E plane tile (the A operand)
constexpr int OZ_B_PLANE = OZ_TI * 128;        // bytes of one D plane tile (the B operand)
constexpr int OZ_STAGE = OZ_PLANES * (OZ_A_PLANE + OZ_B_PLANE);
constexpr int OZ_BIAS = OZ_A_PLANE + OZ_B_PLANE;   // the constant tiles of the bias product
constexpr int OZ_EPI_WARPS = 16;               // four per TMEM lane quarter
constexpr int OZ_EPI_ROWS = OZ_TI / (OZ_EPI_WARPS / 4);   // 16 rows of C per warp
constexpr int OZ_HALF = OZ_EPI_ROWS / 2;       // C is fetched in two halves of 8 rows
constexpr int OZ_STAGE_EPI = OZ_EPI_WARPS * OZ_EPI_ROWS * 32 * 8;   // per-warp [16][32] float64 copy of C
constexpr int OZ_SMEM = OZ_STAGE + OZ_BIAS + OZ_STAGE_EPI + 1024;
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;   // producer, MMA issuer, epilogue warps
constexpr int OZ_TMEM_COLS = 512;              // 7 levels x 64 columns used
constexpr uint32_t OZ_BF16_ONE2 = 0x3F803F80u;     // two bf16 1.0
constexpr uint32_t OZ_BF16_BIAS2 = 0x49404940u;    // two bf16 1.5 2^19 (16 of them sum to 1.5 2^23)

struct OzUpdate {
  double* C;
  int n, ldc;
  const int* ed;        // row exponents of D (rows i of C)
  const int* ee;        // row exponents of E (columns j of C)
  int x0, x1;           // rows / columns in [x0, x1) are left to the side stream
  int ti_tiles, tiles;                // tiles of 64 rows; tiles reaching the lower triangle
  int d_plane_rows, e_plane_rows;     // padded rows of one plane (row offset between planes)
};

// The tiles that reach the lower triangle, numbered row by row: row tile ti holds
// tj = 0 .. floor(ti / 2) (a tile of 64 rows and 128 columns reaches the diagonal when
// tj 128 <= ti 64 + 63), so the rows before ti hold m (m + 1) tiles for ti = 2m and
// (m + 1)^2 for ti = 2m + 1.  Numbering only these tiles gives every CTA of the grid
// the same count to within one.
__host__ __device__ inline int oz_tile_count(int ti_tiles) {
  const int m = ti_tiles >> 1;
  return (ti_tiles & 1) ? (m + 1) * (m + 1) : m * (m + 1);
}

__device__ __forceinline__ void oz_tile(int L, int& ti, int& tj) {
  int s = (int)sqrtf((float)L);
  while (s * s > L) --s;
  while ((s + 1) * (s + 1) <= L) ++s;
  if (L < s * s + s) {
    ti = 2 * s - 1;
    tj = L - s * s;
  } else {
    ti = 2 * s;
    tj = L - s * s - s;
  }
}

// An epilogue warp's share of a tile: its lane's column j, the first of its 16 rows, and
// which rows this lane's element takes (inside the matrix, outside the pivot blocks, on
// or below the diagonal).  Warp-collective (a ballot).
struct OzRows {
  double* at;          // C at (row i0, column j); dereferenced only where `take` says so
  int i0, j;
  unsigned take;       // bit c: row i0 + c
};

__device__ __forceinline__ OzRows oz_rows(const OzUpdate& p, int ti, int tj, int quarter, int cg, int lane) {
  OzRows r;
  r.i0 = ti * OZ_TI + cg * OZ_EPI_ROWS;
  r.j = tj * OZ_TJ + quarter * 32 + lane;
  const int i = r.i0 + lane;
  const unsigned rows_in =
      __ballot_sync(0xffffffffu, lane < OZ_EPI_ROWS && i < p.n && !(i >= p.x0 && i < p.x1)) & 0xFFFFu;
  const int rmin = r.j - r.i0;   // rows c >= rmin are on or below the diagonal
  const unsigned lower = rmin <= 0 ? 0xFFFFu : (rmin >= OZ_EPI_ROWS ? 0u : ((0xFFFFu << rmin) & 0xFFFFu));
  const bool col_ok = r.j < p.n && !(r.j >= p.x0 && r.j < p.x1);
  r.take = col_ok ? (rows_in & lower) : 0u;
  r.at = p.C + ((size_t)r.i0 * p.ldc + r.j);
  return r;
}

// Copies rows [8H, 8H + 8) of the warp's share of C into its stage (one copy group).
// FULL: every lane takes every row (a tile inside the lower triangle), no tests.
template <int H, bool FULL>
__device__ __forceinline__ void oz_fetch(const OzRows& r, int ldc, uint32_t stg_s, int lane) {
#pragma unroll
  for (int c = H * OZ_HALF; c < (H + 1) * OZ_HALF; ++c)
    if (FULL || ((r.take >> c) & 1u)) cp_async8(stg_s + (uint32_t)(c * 32 + lane) * 8u, r.at + (size_t)c * ldc);
  cp_async_commit();
}

template <int H>
__device__ __forceinline__ void oz_fetch_any(const OzRows& r, bool full, int ldc, uint32_t stg_s, int lane) {
  if (full) oz_fetch<H, true>(r, ldc, stg_s, lane);
  else oz_fetch<H, false>(r, ldc, stg_s, lane);
}

// C - 2^(e_i + f_j - 56) V for rows [8H, 8H + 8): rounds each V to float64, subtracts it
// from the staged C and writes the row back.  Returns the rows whose product leaves the
// directly assembled exponent range (left unwritten here).
template <int H, bool FULL>
__device__ __forceinline__ unsigned oz_finish(const OzRows& r, int ldc, const double* stg,
                                              const long long (&V)[OZ_EPI_ROWS], int ei_lane, int fjm, int lane) {
  double x[OZ_HALF];   // the staged C (stale where this lane's element is not taken)
#pragma unroll
  for (int c = 0; c < OZ_HALF; ++c) x[c] = stg[(H * OZ_HALF + c) * 32 + lane];
  unsigned bad = 0u;
#pragma unroll
  for (int c = H * OZ_HALF; c < (H + 1) * OZ_HALF; ++c) {
    const int k = __shfl_sync(0xffffffffu, ei_lane, c) + fjm;
    bool ok;
    const double prod = oz_round_pow2(V[c], k, ok);
    if (FULL || ((r.take >> c) & 1u)) {
      if (ok) r.at[(size_t)c * ldc] = x[c - H * OZ_HALF] - prod;
      else bad |= 1u << c;
    }
  }
  return bad;
}

template <int H>
__device__ __forceinline__ unsigned oz_finish_any(const OzRows& r, bool full, int ldc, const double* stg,
                                                  const long long (&V)[OZ_EPI_ROWS], int ei_lane, int fjm, int lane) {
  return full ? oz_finish<H, true>(r, ldc, stg, V, ei_lane, fjm, lane)
              : oz_finish<H, false>(r, ldc, stg, V, ei_lane, fjm, lane);
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_update_kernel(const __grid_constant__ CUtensorMap tmD, const __grid_constant__ CUtensorMap tmE,
                     const OzUpdate p, int* status) {
  __shared__ __align__(8) uint64_t full_bar;
  __shared__ __align__(8) uint64_t empty_bar;
  __shared__ __align__(8) uint64_t accf_bar;
  __shared__ __align__(8) uint64_t acce_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  extern __shared__ uint8_t oz_smem_raw[];
  const uint32_t smem_base = (smem_u32(oz_smem_raw) + 1023u) & ~1023u;
  uint8_t* const smem = oz_smem_raw + (smem_base - smem_u32(oz_smem_raw));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = p.tiles;

  // the constant tiles of the bias product, written once and handed to the tensor cores
  uint32_t* const bias_w = reinterpret_cast<uint32_t*>(smem + OZ_STAGE);
  for (int w = threadIdx.x; w < OZ_BIAS / 4; w += blockDim.x)
    bias_w[w] = w < OZ_A_PLANE / 4 ? OZ_BF16_ONE2 : OZ_BF16_BIAS2;
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(&full_bar, 1);
    mbar_init(&empty_bar, 1);
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
      uint32_t phase = 0;
      for (int u = blockIdx.x; u < units; u += gridDim.x) {
        int ti, tj;
        oz_tile(u, ti, tj);
        if (!mbar_wait(&empty_bar, phase ^ 1u, &abort_flag)) {
          abort_flag = 1;
          atomicCAS(status, 0, TC_TIMEOUT_PRODUCER);
          break;
        }
        mbar_arrive_expect_tx(&full_bar, OZ_STAGE);
        for (int q = 0; q < OZ_PLANES; ++q) {
          tma_load_2d(smem_base + q * OZ_A_PLANE, &tmE, &full_bar, 0, q * p.e_plane_rows + tj * OZ_TJ);
          tma_load_2d(smem_base + OZ_PLANES * OZ_A_PLANE + q * OZ_B_PLANE, &tmD, &full_bar, 0,
                      q * p.d_plane_rows + ti * OZ_TI);
        }
        phase ^= 1u;
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issue: 7 bias products, then 28 slice pairs x 2 K16 steps
    if (lane == 0) {
      constexpr uint32_t ID = idesc_f16(OZ_TJ, OZ_TI, 1, false);
      const uint32_t sa = smem_base, sb = smem_base + OZ_PLANES * OZ_A_PLANE;
      const uint64_t bias_a = sw128_desc(smem_base + OZ_STAGE), bias_b = sw128_desc(smem_base + OZ_STAGE + OZ_A_PLANE);
      uint32_t phase = 0, acc_phase = 0;
      for (int u = blockIdx.x; u < units; u += gridDim.x) {
        if (!mbar_wait(&acce_bar, acc_phase ^ 1u, &abort_flag) || !mbar_wait(&full_bar, phase, &abort_flag)) {
          abort_flag = 1;
          atomicCAS(status, 0, TC_TIMEOUT_MMA);
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int L = 0; L < OZ_LEVELS; ++L) mma_f16(tbase + L * OZ_TI, bias_a, bias_b, ID, 0u);
#pragma unroll
        for (int t = 0; t < OZ_SLICES; ++t) {
#pragma unroll
          for (int v = 0; v < OZ_SLICES; ++v) {
            if (t + v > OZ_SLICES - 1) continue;                 // keep t + u <= 8 (1-based)
            const uint32_t d = tbase + (t + v) * OZ_TI;
            const uint32_t ao = sa + (t >> 1) * OZ_A_PLANE + (t & 1) * 64;
            const uint32_t bo = sb + (v >> 1) * OZ_B_PLANE + (v & 1) * 64;
            mma_f16(d, sw128_desc(ao), sw128_desc(bo), ID, 1u);
            mma_f16(d, sw128_desc(ao + 32), sw128_desc(bo + 32), ID, 1u);
          }
        }
        mma_commit(&empty_bar);
        mma_commit(&accf_bar);
        phase ^= 1u;
        acc_phase ^= 1u;
      }
    }
  } else {
    // ------------------------------------------------ epilogue: combine the levels, C -= D E^T
    // Each warp owns 32 columns (its TMEM lane quarter) x 16 rows of the tile.  Its share
    // of C is copied into a [16][32] stage in two halves of 8 rows, each half of the next
    // tile as soon as this tile's half has been consumed, so the copies run under the
    // MMAs and the rounding.  The biased level sums b_L = S_L + 1.5 2^23 are combined
    // into one 64-bit integer in units of 2^-56 of the scaled product,
    //   V = S_0 2^40 + S_1 2^32 + S_2 2^24 + S_3 2^16 + S_4 2^8 + S_5 + floor(S_6 / 2^8)
    // (|V| < 2^60; the floor drops less than 2^-56 of the row scales' product), after
    // which TMEM goes back to the MMAs.  The product 2^(e_i + f_j - 56) V is rounded to
    // float64 with integer instructions and subtracted from C (the only float64
    // operation per element).
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int cg = ew >> 2;                      // group of 16 rows
    const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
    const double* stg = reinterpret_cast<const double*>(smem + OZ_STAGE + OZ_BIAS) + ew * OZ_EPI_ROWS * 32;
    const uint32_t stg_s = smem_base + OZ_STAGE + OZ_BIAS + ew * OZ_EPI_ROWS * 32 * 8;
    uint32_t acc_phase = 0;
    int u = blockIdx.x;
    OzRows cur;
    cur.take = 0u;
    if (u < units) {
      int ti, tj;
      oz_tile(u, ti, tj);
      cur = oz_rows(p, ti, tj, quarter, cg, lane);
    }
    bool cur_full = __all_sync(0xffffffffu, cur.take == 0xFFFFu);
    oz_fetch_any<0>(cur, cur_full, p.ldc, stg_s, lane);
    oz_fetch_any<1>(cur, cur_full, p.ldc, stg_s, lane);
    while (u < units) {
      // the column scale of this lane and the row scales of the warp's 16 rows
      const int fjm = (cur.j < p.n ? p.ee[cur.j] : 0) - 56;
      const int ei_lane = (lane < OZ_EPI_ROWS && cur.i0 + lane < p.n) ? p.ed[cur.i0 + lane] : 0;
      int got = 1;
      if (lane == 0) got = mbar_wait(&accf_bar, acc_phase, &abort_flag) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      if (!got) {
        if (lane == 0) {
          abort_flag = 1;
          atomicCAS(status, 0, TC_TIMEOUT_EPILOGUE);
        }
        break;
      }
      tc_fence_after();
      long long V[OZ_EPI_ROWS];
#pragma unroll
      for (int q = 0; q < OZ_EPI_ROWS / 4; ++q) {
        float a[OZ_LEVELS][4];
#pragma unroll
        for (int lv = 0; lv < OZ_LEVELS; ++lv)
          tmem_ld4(tbase + lane_off + lv * OZ_TI + cg * OZ_EPI_ROWS + q * 4, a[lv]);
        tmem_ld_wait();
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          // |S_L| < 2^22: pairs of levels combine exactly in int32 before one 64-bit assembly
          const int t3 = oz_pair<8>(__float_as_uint(a[0][c]), __float_as_uint(a[1][c]));
          const int t2 = oz_pair<8>(__float_as_uint(a[2][c]), __float_as_uint(a[3][c]));
          const int t1 = oz_pair<8>(__float_as_uint(a[4][c]), __float_as_uint(a[5][c])) +
                         oz_level_shr<8>(__float_as_uint(a[6][c]));
          V[q * 4 + c] = ((long long)t3 << 32) + ((long long)t2 << 16) + (long long)t1;
        }
      }
      // the accumulators have been read: the next tile's MMAs may start
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce_bar);
      acc_phase ^= 1u;
      const int u2 = u + gridDim.x;
      OzRows nxt;
      nxt.take = 0u;
      if (u2 < units) {
        int ti2, tj2;
        oz_tile(u2, ti2, tj2);
        nxt = oz_rows(p, ti2, tj2, quarter, cg, lane);
      }
      const bool nxt_full = __all_sync(0xffffffffu, nxt.take == 0xFFFFu);
      cp_async_wait_group<1>();                  // this tile's first half has landed
      unsigned bad = oz_finish_any<0>(cur, cur_full, p.ldc, stg, V, ei_lane, fjm, lane);
      oz_fetch_any<0>(nxt, nxt_full, p.ldc, stg_s, lane);
      cp_async_wait_group<1>();                  // and its second half
      bad |= oz_finish_any<1>(cur, cur_full, p.ldc, stg, V, ei_lane, fjm, lane);
      oz_fetch_any<1>(nxt, nxt_full, p.ldc, stg_s, lane);
      if (__any_sync(0xffffffffu, bad != 0u)) {
        // products outside the directly assembled exponent range (C itself is still unwritten there)
#pragma unroll
        for (int c = 0; c < OZ_EPI_ROWS; ++c) {
          const int k = __shfl_sync(0xffffffffu, ei_lane, c) + fjm;
          if ((bad >> c) & 1u) {
            double* q = cur.at + (size_t)c * p.ldc;
            *q = *q - oz_i64_times_pow2_slow(V[c], k);
          }
        }
      }
      cur = nxt;
      cur_full = nxt_full;
      u = u2;
    }
    cp_async_wait_all();
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
  LRS_TRY(make_operand_map(md, dplanes, 64, (uint64_t)OZ_PLANES * rows_pad, OZ_TI));
  return make_operand_map(me, eplanes, 64, (uint64_t)OZ_PLANES * rows_pad, OZ_TJ);
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
  p.ti_tiles = (n + OZ_TI - 1) / OZ_TI;
  p.tiles = oz_tile_count(p.ti_tiles);
  p.d_plane_rows = rows_pad;
  p.e_plane_rows = rows_pad;
  if (!ctx->capturing)
    LRS_CUDA_TRY(cudaFuncSetAttribute(oz_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
  const int grid = std::min(p.tiles, ctx->num_sms);
  oz_update_kernel<<<grid, OZ_THREADS, OZ_SMEM, stream>>>(md, me, p, ctx->ws.status.ptr + 8);
  return after_launch(ctx, "oz_update_kernel");
}

int oz_rows_pad(int n) { return (n + OZ_TJ - 1) / OZ_TJ * OZ_TJ; }
size_t oz_plane_elems(int n) { return (size_t)OZ_PLANES * oz_rows_pad(n) * 64; }

}  // namespace lrs
