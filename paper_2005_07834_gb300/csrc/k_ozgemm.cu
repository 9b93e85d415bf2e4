// Float64-accurate batched GEMM on the tensor cores,
//   C_b = alpha op(A_b) diag(ks_b) op(B_b) + beta C_b,
// for the basis changes of the lm-basis Dyson solve (Sec. VI.E: T = chi0 Q Y,
// X = Y^T Q T, U = Y Z, W = U Y^T, one batch entry per radial shell) and the
// radial-block products of its SPD form (F^T X F, F M^-1 F^T: one batch entry
// per lm, operands and results addressed through arbitrary strides).
//
// Packing (oz_pack_kernel): every row of op(A) diag(ks) and of op(B)^T is
// scaled by a power of two, x = 2^e a with |a| < 1/2 (e from the largest
// exponent of the row), and written as the integer N = round(a 2^56) in base
// 128 with balanced digits,
//   a = sum_{t=0..7} s_t 128^-(t+1),  |s_t| <= 64,
// each digit exact in bf16; the representation error is at most 2^-56 2^e.
// Slices 2q and 2q + 1 share one 128-byte row of plane q (the [hi | lo]
// layout the swizzled operand tiles use), per K chunk of 32.  Integer and
// fp32 instructions only (oz_combine.cuh), apart from the product with ks.
//
// Products (oz_gemm_kernel): the 36 slice pairs with t + u <= 7 are issued as
// bf16 tcgen05 MMAs into eight fp32 accumulators in TMEM, one per level
// t + u.  Over a K segment of 128 a level sum is an integer of magnitude at
// most 128 * 8 * 64 * 64 = 2^22, so the tensor cores accumulate it exactly.
// The epilogue combines the levels of a segment into one 64-bit integer and
// rounds the product to float64 with integer instructions (oz_combine.cuh);
// segments add in float64.  The dropped pairs (t + u >= 8) and the
// representation errors bound the error by about 2^-54 K |A|row max |B|row max
// per element, the bound of a float64 dot product of K terms.
//
// Tiles of 128 x 64 outputs, one persistent CTA per SM: a TMA producer warp,
// an MMA-issuing warp and sixteen epilogue warps; two pipeline stages of one K
// chunk (four A and four B planes, 96 KB) each.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "lrs_internal.h"
#include "oz_combine.cuh"
#include "tc_common.cuh"

namespace lrs {
using namespace tc;

constexpr int OG_SLICES = 8;                   // base-128 digits per value
constexpr int OG_PLANES = 4;                   // two slices per 128-byte row
constexpr int OG_LEVELS = 8;                   // t + u = 0 .. 7
constexpr int OG_TM = 128, OG_TN = 64;
constexpr int OG_A_PLANE = OG_TM * 128;        // bytes of one A plane tile (one K chunk of 32)
constexpr int OG_B_PLANE = OG_TN * 128;
constexpr int OG_STAGE = OG_PLANES * (OG_A_PLANE + OG_B_PLANE);
constexpr int OG_STAGES = 2;
constexpr int OG_SEG = 4;                      // K chunks of 32 per exact accumulation segment
constexpr int OG_EPI_WARPS = 16;               // four per TMEM lane quarter, 16 columns each
constexpr int OG_EPI_COLS = OG_TN / (OG_EPI_WARPS / 4);
constexpr int OG_STG_LD = 33;                  // per-warp [8 columns][33] float64 staging
constexpr int OG_STAGE_EPI = OG_EPI_WARPS * 8 * OG_STG_LD * 8;
constexpr int OG_SMEM = OG_STAGES * OG_STAGE + OG_STAGE_EPI + 1024;
constexpr int OG_THREADS = 64 + 32 * OG_EPI_WARPS;   // producer, MMA issuer, epilogue warps
constexpr int OG_TMEM_COLS = 512;              // 8 levels x 64 columns
constexpr int OG_BAD_EXP = 1 << 20;            // row exponent of a row holding a NaN or an infinity

static_assert(OG_SMEM <= 227 * 1024, "shared memory of one CTA");

// ---------------------------------------------------------------- slicing
// Operand X (rows x k, logical) with X[i][kk] = x[i si + kk sk] ks[kk]
// into planes[b][q][kc][rows_pad][64] and expo[b][rows_pad].  One CTA: 32 rows, all of K,
// read through 32 x 32 shared-memory tiles so that both layouts are read coalesced.
struct OgPack {
  const double* x;
  long long si, sk;        // element (i, kk) of batch b at x + b stride + i si + kk sk
  long long stride;
  const double* ks;
  long long stride_ks;
  int trans;               // the tile is walked with i fastest (si is the short stride)
  int rows, k, rows_pad, nchunks;
  uint16_t* planes;
  int* expo;
};

__device__ __forceinline__ void og_load_tile(const OgPack& p, const double* x, const double* ks, int i0, int k0,
                                             double (*t)[33]) {
  for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
    int ii, kk;
    if (p.trans) { kk = idx >> 5; ii = idx & 31; } else { ii = idx >> 5; kk = idx & 31; }
    const int i = i0 + ii, k = k0 + kk;
    double v = 0.0;
    if (i < p.rows && k < p.k) {
      v = x[i * p.si + k * p.sk];
      if (ks) v *= ks[k];
    }
    t[kk][ii] = v;
  }
}

// Digits of one value (lane k of a row with scale e): planes[(s / 2) nchunks + kc][row][(s % 2) 32 + k].
__device__ __forceinline__ void og_put_digits(double v, int e, uint16_t* base, size_t chunk_elems, int nchunks,
                                              int kc, int row, int lane) {
  // N = round(v 2^(56 - e)), |N| <= 2^55; balanced base-128 digits s_7 .. s_1 in [-64, 63], leading s_0
  long long N = oz_fixed56(v, e);
  int dig[OG_SLICES];
#pragma unroll
  for (int s = OG_SLICES - 1; s > 0; --s) {
    const long long d = ((N + 64) & 127) - 64;
    dig[s] = (int)d;
    N = (N - d) >> 7;                          // exact
  }
  dig[0] = (int)N;
#pragma unroll
  for (int s = 0; s < OG_SLICES; ++s)
    base[((size_t)(s >> 1) * nchunks + kc) * chunk_elems + (size_t)row * 64 + (s & 1) * 32 + lane] =
        oz_int_to_bf16_bits(dig[s]);
}

// One CTA: 32 rows (warp w holds rows w, w + 8, w + 16, w + 24, lane = K index within a chunk).
// Up to HOLD chunks stay in registers between the row scale and the digits; longer rows are
// read twice (the second time from L2).  HOLD follows K (2 or 4 chunks; 1 = read twice), so
// that few registers are held and several CTAs reside on an SM to cover the memory latency.
template <int HOLD>
__global__ void __launch_bounds__(256, HOLD <= 2 ? 4 : 3) oz_pack_kernel(const OgPack p) {
  constexpr int OG_HOLD = HOLD;
  __shared__ double t[32][33];
  const int b = blockIdx.y;
  const double* x = p.x + p.stride * b;
  const double* ks = p.ks ? p.ks + p.stride_ks * b : nullptr;
  const int i0 = blockIdx.x * 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool hold = p.nchunks <= OG_HOLD;
  double v[OG_HOLD][4];
  int emax[4] = {0, 0, 0, 0};
  // pass 1: largest exponent field per row
  for (int kc = 0; kc < p.nchunks; ++kc) {
    og_load_tile(p, x, ks, i0, kc * 32, t);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const double y = t[lane][warp + 8 * r];
      emax[r] = max(emax[r], oz_exp_field(y));
#pragma unroll
      for (int c = 0; c < OG_HOLD; ++c)
        if (c == kc) v[c][r] = y;
    }
    __syncthreads();
  }
  int e[4];
  bool bad[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int E = (int)__reduce_max_sync(0xffffffffu, (unsigned)emax[r]);
    bad[r] = E == 0x7FF;                       // an infinity or a NaN in the row
    e[r] = bad[r] ? OG_BAD_EXP : oz_row_scale(E);
    if (lane == 0) p.expo[(size_t)b * p.rows_pad + i0 + warp + 8 * r] = e[r];
  }
  // pass 2: digits
  const size_t chunk_elems = (size_t)p.rows_pad * 64;
  uint16_t* base = p.planes + (size_t)b * OG_PLANES * p.nchunks * chunk_elems;
  if (hold) {
#pragma unroll
    for (int c = 0; c < OG_HOLD; ++c) {
      if (c >= p.nchunks) break;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        og_put_digits(bad[r] ? 0.0 : v[c][r], bad[r] ? 0 : e[r], base, chunk_elems, p.nchunks, c,
                      i0 + warp + 8 * r, lane);
    }
  } else {
    for (int kc = 0; kc < p.nchunks; ++kc) {
      og_load_tile(p, x, ks, i0, kc * 32, t);
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 4; ++r)
        og_put_digits(bad[r] ? 0.0 : t[lane][warp + 8 * r], bad[r] ? 0 : e[r], base, chunk_elems, p.nchunks, kc,
                      i0 + warp + 8 * r, lane);
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- products
struct OgGemm {
  double* C;
  long long rs, cs;        // element (i, j) of C_b at C + b stride_c + i rs + j cs
  long long stride_c;
  int m, n;
  double alpha, beta;
  int alpha_mode;          // 0: alpha = 1, 1: alpha = -1 (a sign flip), 2: a float64 product
  int beta_zero;           // beta == 0: C is not read in the first segment
  int dI, dJ, dB;          // dadd is added where i dI + j dJ + b dB == 0 (a diagonal), if has_diag
  int has_diag;
  double dadd;
  const int* ea;           // [a batches][a_rows_pad]
  const int* eb;           // [b batches][b_rows_pad]
  int a_shared, b_shared;  // one packed operand serves every batch entry
  int b_sqrt;              // B of batch entry b is packed batch floor(sqrt(b))
  int a_rows_pad, b_rows_pad, nchunks;
  int row_tiles, col_tiles, batch;
  int batch_fastest;       // units run batch entry fastest (neighbouring entries write neighbouring words)
  int lower_col;           // > 0: C_b is column block b * lower_col of a symmetric matrix (lower tiles only)
};

__device__ __forceinline__ bool og_decode(const OgGemm& p, int u, int& b, int& bi, int& bj) {
  const int per = p.row_tiles * p.col_tiles;
  int rem;
  if (p.batch_fastest) {
    rem = u / p.batch;
    b = u - rem * p.batch;
  } else {
    b = u / per;
    rem = u - b * per;
  }
  bi = rem / p.col_tiles;
  bj = rem - bi * p.col_tiles;
  return p.lower_col <= 0 || bi * OG_TM + OG_TM - 1 >= b * p.lower_col + bj * OG_TN;
}

__device__ __forceinline__ int og_b_batch(const OgGemm& p, int b) {
  if (p.b_shared) return 0;
  if (!p.b_sqrt) return b;
  int l = (int)sqrtf((float)b);
  while (l * l > b) --l;
  while ((l + 1) * (l + 1) <= b) ++l;
  return l;
}

// ROWWISE: C is row-major (cs == 1) and a warp stores 4 rows x 8 columns per step; otherwise each
// lane stores its own row (consecutive words when rs == 1).
// One 64-bit integer per element from the eight level sums of an epilogue step, in units of
// 2^-56 of the scaled product: V = sum_L S_L 2^(42 - 7 L) with floor(S_7 / 2^7) (|V| < 2^62; the
// floor drops less than 2^-56 of the row scales' product).
__device__ __forceinline__ long long og_level_value(const float (&a)[OG_LEVELS][8], int c) {
  const int ta = oz_pair<7>(oz_level_bits(a[1][c]), oz_level_bits(a[2][c]));
  const int tb = oz_pair<7>(oz_level_bits(a[3][c]), oz_level_bits(a[4][c]));
  const int tc = oz_pair<7>(oz_level_bits(a[5][c]), oz_level_bits(a[6][c])) + oz_level_shr<7>(oz_level_bits(a[7][c]));
  return ((long long)oz_level_int(a[0][c]) << 42) + ((long long)ta << 28) + ((long long)tb << 14) + (long long)tc;
}

// Writes one staged step of 8 columns into C (alpha times the product, plus beta C, plus the
// diagonal term), with the launch's uniform options as template arguments so that the loop over
// the elements tests none of them.  neg flips the sign (alpha = -1) with an integer instruction.
template <bool ROWWISE, bool READ_C, bool GEN_ALPHA, bool DIAG>
__device__ __forceinline__ void og_write_step(const OgGemm& p, double* C, const double* stg, int row0, int colc,
                                              int lane, long long neg, double cscale, int b) {
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const int r = ROWWISE ? it * 4 + (lane >> 3) : lane, c = ROWWISE ? lane & 7 : it;
    const int i = row0 + r, j = colc + c;
    if (i < p.m && j < p.n) {
      double v = __longlong_as_double(__double_as_longlong(stg[c * OG_STG_LD + r]) ^ neg);
      if (GEN_ALPHA) v *= p.alpha;
      if (READ_C) v = fma(cscale, C[i * p.rs + j * p.cs], v);
      if (DIAG && i * p.dI + j * p.dJ + b * p.dB == 0) v += p.dadd;
      C[i * p.rs + j * p.cs] = v;
    }
  }
}

template <bool ROWWISE, bool READ_C>
__device__ __forceinline__ void og_write_step_any(const OgGemm& p, double* C, const double* stg, int row0, int colc,
                                                  int lane, long long neg, bool gen_alpha, bool diag, double cscale,
                                                  int b) {
  if (gen_alpha) {
    if (diag) og_write_step<ROWWISE, READ_C, true, true>(p, C, stg, row0, colc, lane, neg, cscale, b);
    else og_write_step<ROWWISE, READ_C, true, false>(p, C, stg, row0, colc, lane, neg, cscale, b);
  } else {
    if (diag) og_write_step<ROWWISE, READ_C, false, true>(p, C, stg, row0, colc, lane, neg, cscale, b);
    else og_write_step<ROWWISE, READ_C, false, false>(p, C, stg, row0, colc, lane, neg, cscale, b);
  }
}

template <bool ROWWISE>
__global__ void __launch_bounds__(OG_THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const OgGemm p, int* status) {
  __shared__ __align__(8) uint64_t full_bar[OG_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[OG_STAGES];
  __shared__ __align__(8) uint64_t accf_bar;
  __shared__ __align__(8) uint64_t acce_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  extern __shared__ uint8_t og_smem_raw[];
  const uint32_t smem_base = (smem_u32(og_smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = p.batch * p.row_tiles * p.col_tiles;
  const int nseg = (p.nchunks + OG_SEG - 1) / OG_SEG;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OG_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&accf_bar, 1);
    mbar_init(&acce_bar, OG_EPI_WARPS);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_map(&tmA);
    tma_prefetch_map(&tmB);
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base, OG_TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer: all slice planes of one K chunk per stage
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool stop = false;
      for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
        int b, bi, bj;
        if (!og_decode(p, u, b, bi, bj)) continue;
        const int ab = p.a_shared ? 0 : b, bb = og_b_batch(p, b);
        for (int kc = 0; kc < p.nchunks; ++kc) {
          if (!mbar_wait(&empty_bar[stage], phase ^ 1u, &abort_flag)) {
            abort_flag = 1;
            atomicCAS(status, 0, TC_TIMEOUT_PRODUCER);
            stop = true;
            break;
          }
          mbar_arrive_expect_tx(&full_bar[stage], OG_STAGE);
          const uint32_t s = smem_base + stage * OG_STAGE;
          for (int q = 0; q < OG_PLANES; ++q) {
            tma_load_2d(s + q * OG_A_PLANE, &tmA, &full_bar[stage], 0,
                        ((ab * OG_PLANES + q) * p.nchunks + kc) * p.a_rows_pad + bi * OG_TM);
            tma_load_2d(s + OG_PLANES * OG_A_PLANE + q * OG_B_PLANE, &tmB, &full_bar[stage], 0,
                        ((bb * OG_PLANES + q) * p.nchunks + kc) * p.b_rows_pad + bj * OG_TN);
          }
          if (++stage == OG_STAGES) { stage = 0; phase ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issue: 36 slice pairs x 2 K16 steps per chunk
    if (lane == 0) {
      constexpr uint32_t ID = idesc_f16(OG_TM, OG_TN, 1, false);
      int stage = 0;
      uint32_t phase = 0, acc_phase = 0;
      bool stop = false;
      for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
        int b, bi, bj;
        if (!og_decode(p, u, b, bi, bj)) continue;
        for (int sg = 0; sg < nseg && !stop; ++sg) {
          if (!mbar_wait(&acce_bar, acc_phase ^ 1u, &abort_flag)) {
            abort_flag = 1;
            atomicCAS(status, 0, TC_TIMEOUT_MMA);
            stop = true;
            break;
          }
          tc_fence_after();
          const int kc1 = min(p.nchunks, (sg + 1) * OG_SEG);
          for (int kc = sg * OG_SEG; kc < kc1; ++kc) {
            if (!mbar_wait(&full_bar[stage], phase, &abort_flag)) {
              abort_flag = 1;
              atomicCAS(status, 0, TC_TIMEOUT_MMA);
              stop = true;
              break;
            }
            tc_fence_after();
            const uint32_t s = smem_base + stage * OG_STAGE;
            const uint32_t sa = s, sb = s + OG_PLANES * OG_A_PLANE;
            const uint32_t seg_first = (kc == sg * OG_SEG) ? 1u : 0u;
#pragma unroll
            for (int t = 0; t < OG_SLICES; ++t) {
#pragma unroll
              for (int v = 0; v < OG_SLICES; ++v) {
                if (t + v > OG_LEVELS - 1) continue;
                const uint32_t d = tbase + (t + v) * OG_TN;
                const uint32_t ao = sa + (t >> 1) * OG_A_PLANE + (t & 1) * 64;
                const uint32_t bo = sb + (v >> 1) * OG_B_PLANE + (v & 1) * 64;
                // pairs are issued t-major, so (0, level) is the first product into each level
                const uint32_t acc = (seg_first && t == 0) ? 0u : 1u;
                mma_f16(d, sw128_desc(ao), sw128_desc(bo), ID, acc);
                mma_f16(d, sw128_desc(ao + 32), sw128_desc(bo + 32), ID, 1u);
              }
            }
            mma_commit(&empty_bar[stage]);
            if (++stage == OG_STAGES) { stage = 0; phase ^= 1u; }
          }
          if (stop) break;
          mma_commit(&accf_bar);
          acc_phase ^= 1u;
        }
      }
    }
  } else {
    // ------------------------------------------------ epilogue: combine the levels, C = alpha sum + beta C
    // Level sums S_0 .. S_7 (integers of magnitude at most 2^22 in fp32, read as int32 by one
    // fp32 add each) are combined into one 64-bit integer V, the segment's product being
    // 2^(e_i + f_j - 56) V, rounded to float64 with integer instructions: with alpha = 1 and
    // beta = 0 the epilogue issues no float64 operation.  Sixteen warps, four per TMEM lane
    // quarter with 16 columns each (two steps of 8), keep enough independent work in flight to
    // cover the latency of these integer chains.  Each step is staged in shared memory and, for
    // row-major C, written row-wise (coalesced).
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int cg = ew >> 2;                      // column group of OG_EPI_COLS
    const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
    double* stg = reinterpret_cast<double*>(og_smem_raw + (smem_base - smem_u32(og_smem_raw)) +
                                            OG_STAGES * OG_STAGE) + ew * 8 * OG_STG_LD;
    uint32_t acc_phase = 0;
    bool stop = false;
    for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
      int b, bi, bj;
      if (!og_decode(p, u, b, bi, bj)) continue;
      const int ab = p.a_shared ? 0 : b, bb = og_b_batch(p, b);
      double* C = p.C + p.stride_c * b;
      const int row0 = bi * OG_TM + quarter * 32;
      const int col0 = bj * OG_TN + cg * OG_EPI_COLS;
      const int ei = p.ea[(size_t)ab * p.a_rows_pad + row0 + lane];   // padded rows hold 0
      for (int sg = 0; sg < nseg; ++sg) {
        int got = 1;
        if (lane == 0) got = mbar_wait(&accf_bar, acc_phase, &abort_flag) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) {
          if (lane == 0) {
            abort_flag = 1;
            atomicCAS(status, 0, TC_TIMEOUT_EPILOGUE);
          }
          stop = true;
          break;
        }
        tc_fence_after();
        const bool read_c = sg > 0 || !p.beta_zero;
        const double cscale = sg > 0 ? 1.0 : p.beta;
        const bool gen_alpha = p.alpha_mode == 2, diag = p.has_diag && sg == 0;
        const long long neg = p.alpha_mode == 1 ? (long long)0x8000000000000000ull : 0ll;
        constexpr bool rowwise = ROWWISE;
#pragma unroll 1
        for (int ch = 0; ch < OG_EPI_COLS / 8; ++ch) {
          if (col0 + ch * 8 >= p.n) break;       // warp-uniform: nothing to store past column n
          float a[OG_LEVELS][8];
#pragma unroll
          for (int lv = 0; lv < OG_LEVELS; ++lv)
            tmem_ld8(tbase + lane_off + lv * OG_TN + cg * OG_EPI_COLS + ch * 8, a[lv]);
          tmem_ld_wait();
          unsigned badm = 0u;   // columns whose product leaves the directly assembled exponent range
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const long long V = og_level_value(a, c);
            const int j = col0 + ch * 8 + c;
            const int fj = p.eb[(size_t)bb * p.b_rows_pad + j];   // padded rows hold 0
            bool ok;
            const double prod = oz_round_pow2(V, ei + fj - 56, ok);
            badm |= ok ? 0u : (1u << c);
            stg[c * OG_STG_LD + lane] = (ei == OG_BAD_EXP || fj == OG_BAD_EXP)
                                            ? __longlong_as_double(0x7ff8000000000000ll)   // NaN, as in float64
                                            : prod;
          }
          if (__any_sync(0xffffffffu, badm != 0u)) {
            // rare: those products again from the levels (still in TMEM), through float64
            float a2[OG_LEVELS][8];
#pragma unroll
            for (int lv = 0; lv < OG_LEVELS; ++lv)
              tmem_ld8(tbase + lane_off + lv * OG_TN + cg * OG_EPI_COLS + ch * 8, a2[lv]);
            tmem_ld_wait();
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              if ((badm >> c) & 1u) {
                const int fj = p.eb[(size_t)bb * p.b_rows_pad + col0 + ch * 8 + c];
                stg[c * OG_STG_LD + lane] = (ei == OG_BAD_EXP || fj == OG_BAD_EXP)
                                                ? __longlong_as_double(0x7ff8000000000000ll)
                                                : oz_i64_times_pow2_slow(og_level_value(a2, c), ei + fj - 56);
              }
            }
          }
          __syncwarp();
          if (read_c) og_write_step_any<rowwise, true>(p, C, stg, row0, col0 + ch * 8, lane, neg, gen_alpha, diag, cscale, b);
          else og_write_step_any<rowwise, false>(p, C, stg, row0, col0 + ch * 8, lane, neg, gen_alpha, diag, cscale, b);
          __syncwarp();
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce_bar);
        acc_phase ^= 1u;
      }
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
    tmem_dealloc(tbase, OG_TMEM_COLS);
  }
}

static int og_pack(lrs_ctx* ctx, const double* x, long long si, long long sk, long long stride, const double* ks,
                   long long stride_ks, int rows, int k, int rows_pad, int nchunks, int batches, uint16_t* planes,
                   int* expo) {
  OgPack p;
  p.x = x;
  p.si = si;
  p.sk = sk;
  p.stride = stride;
  p.ks = ks;
  p.stride_ks = stride_ks;
  p.trans = (si < sk) ? 1 : 0;
  p.rows = rows;
  p.k = k;
  p.rows_pad = rows_pad;
  p.nchunks = nchunks;
  p.planes = planes;
  p.expo = expo;
  const dim3 grid(rows_pad / 32, batches);
  if (nchunks <= 2) oz_pack_kernel<2><<<grid, 256, 0, ctx->stream>>>(p);
  else if (nchunks <= 4) oz_pack_kernel<4><<<grid, 256, 0, ctx->stream>>>(p);
  else oz_pack_kernel<1><<<grid, 256, 0, ctx->stream>>>(p);
  return after_launch(ctx, "oz_pack_kernel");
}

int oz_gemm_strided(lrs_ctx* ctx, int m, int n, int k, int batch, const OzOperand& a, const double* ks,
                    long long stride_ks, const OzOperand& b, const OzStore& c) {
  if (m <= 0 || n <= 0 || batch <= 0) return LRS_OK;
  if (k <= 0) return set_error(LRS_ERR_ARG, "oz_gemm_strided: empty contraction");
  if (a.sqrt_batch) return set_error(LRS_ERR_ARG, "oz_gemm_strided: sqrt batch mapping is for B only");
  const int nchunks = (k + 31) / 32;
  const int a_rows_pad = (m + OG_TM - 1) / OG_TM * OG_TM;
  const int b_rows_pad = (n + OG_TN - 1) / OG_TN * OG_TN;
  const bool a_shared = a.sb == 0 && (ks == nullptr || stride_ks == 0);
  const bool b_shared = b.sb == 0;
  int b_distinct = batch;
  if (b.sqrt_batch) {
    int l = 0;
    while ((l + 1) * (l + 1) <= batch - 1) ++l;
    b_distinct = l + 1;
  }
  const int a_batches = a_shared ? 1 : batch, b_batches = b_shared ? 1 : b_distinct;
  const size_t a_elems = (size_t)a_batches * OG_PLANES * nchunks * a_rows_pad * 64;
  const size_t b_elems = (size_t)b_batches * OG_PLANES * nchunks * b_rows_pad * 64;
  LRS_TRY(ensure(ctx, ctx->ws.og_planes, a_elems + b_elems));
  LRS_TRY(ensure(ctx, ctx->ws.og_expo, (size_t)a_batches * a_rows_pad + (size_t)b_batches * b_rows_pad));
  uint16_t* pa = ctx->ws.og_planes.ptr;
  uint16_t* pb = pa + a_elems;
  int* xa = ctx->ws.og_expo.ptr;
  int* xb = xa + (size_t)a_batches * a_rows_pad;
  // A diag(ks): rows i, K index kk; B: rows j (output columns), K index kk
  LRS_TRY(og_pack(ctx, a.x, a.si, a.sk, a_shared ? 0 : a.sb, ks, a_shared ? 0 : stride_ks, m, k, a_rows_pad, nchunks,
                  a_batches, pa, xa));
  LRS_TRY(og_pack(ctx, b.x, b.si, b.sk, b_shared ? 0 : b.sb, nullptr, 0, n, k, b_rows_pad, nchunks, b_batches, pb,
                  xb));
  CUtensorMap ma, mb;
  LRS_TRY(make_operand_map(&ma, pa, 64, (uint64_t)a_batches * OG_PLANES * nchunks * a_rows_pad, OG_TM));
  LRS_TRY(make_operand_map(&mb, pb, 64, (uint64_t)b_batches * OG_PLANES * nchunks * b_rows_pad, OG_TN));
  OgGemm p;
  p.C = c.c;
  p.rs = c.rs;
  p.cs = c.cs;
  p.stride_c = c.sb;
  p.m = m;
  p.n = n;
  p.alpha = c.alpha;
  p.beta = c.beta;
  p.alpha_mode = c.alpha == 1.0 ? 0 : (c.alpha == -1.0 ? 1 : 2);
  p.beta_zero = c.beta == 0.0 ? 1 : 0;
  p.dI = c.dI;
  p.dJ = c.dJ;
  p.dB = c.dB;
  p.has_diag = c.dadd != 0.0 ? 1 : 0;
  p.dadd = c.dadd;
  p.ea = xa;
  p.eb = xb;
  p.a_shared = a_shared ? 1 : 0;
  p.b_shared = b_shared ? 1 : 0;
  p.b_sqrt = (b.sqrt_batch && !b_shared) ? 1 : 0;
  p.a_rows_pad = a_rows_pad;
  p.b_rows_pad = b_rows_pad;
  p.nchunks = nchunks;
  p.row_tiles = a_rows_pad / OG_TM;
  p.col_tiles = b_rows_pad / OG_TN;
  p.batch = batch;
  p.batch_fastest = c.batch_fastest ? 1 : 0;
  p.lower_col = c.lower_col;
  const long long units = (long long)batch * p.row_tiles * p.col_tiles;
  const int grid = (int)std::min<long long>(units, ctx->num_sms);
  if (c.cs == 1) {
    if (!ctx->capturing)
      LRS_CUDA_TRY(cudaFuncSetAttribute(oz_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, OG_SMEM));
    oz_gemm_kernel<true><<<grid, OG_THREADS, OG_SMEM, ctx->stream>>>(ma, mb, p, ctx->ws.status.ptr + 8);
  } else {
    if (!ctx->capturing)
      LRS_CUDA_TRY(cudaFuncSetAttribute(oz_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, OG_SMEM));
    oz_gemm_kernel<false><<<grid, OG_THREADS, OG_SMEM, ctx->stream>>>(ma, mb, p, ctx->ws.status.ptr + 8);
  }
  return after_launch(ctx, "oz_gemm_kernel");
}

int oz_gemm_batched(lrs_ctx* ctx, bool ta, bool tb, int m, int n, int k, double alpha, const double* a, int lda,
                    long long stride_a, const double* ks, long long stride_ks, const double* b, int ldb,
                    long long stride_b, double beta, double* c, int ldc, long long stride_c, int batch,
                    int lower_col) {
  if (m <= 0 || n <= 0 || batch <= 0) return LRS_OK;
  if (k <= 0)   // C = beta C: nothing for the tensor cores to do
    return dgemm_batched(ctx, ta, tb, m, n, 0, alpha, a, lda, stride_a, ks, stride_ks, b, ldb, stride_b, nullptr,
                         beta, c, ldc, stride_c, batch);
  // op(A)[i][kk] and op(B)^T[j][kk] = op(B)[kk][j]
  const OzOperand A{a, ta ? 1 : (long long)lda, ta ? (long long)lda : 1, stride_a, false};
  const OzOperand B{b, tb ? (long long)ldb : 1, tb ? 1 : (long long)ldb, stride_b, false};
  OzStore C;
  C.c = c;
  C.rs = ldc;
  C.cs = 1;
  C.sb = stride_c;
  C.alpha = alpha;
  C.beta = beta;
  C.lower_col = lower_col;
  return oz_gemm_strided(ctx, m, n, k, batch, A, ks, stride_ks, B, C);
}

}  // namespace lrs
