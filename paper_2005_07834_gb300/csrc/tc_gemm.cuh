// Generic split-precision complex GEMM on tcgen05 (sm_103a): D = A B^T with
// A [M][K], B [N][K] stored as 16-bit hi/lo planes (re and im separately).
//   Re D = Ar Br - Ai Bi,  Im D = Ar Bi + Ai Br,
// each real product as hi*hi + hi*lo + lo*hi (12 MMAs of 128 x TN x 16 per
// 16-wide K step).  Tiles are staged by TMA with the 128-byte swizzle through
// an mbarrier pipeline.
//
// Segmented accumulation.  The tensor cores add every MMA result into their
// fp32 accumulator with a rounding that is biased toward zero, so the error of
// one long accumulation grows linearly with K (measured: relative 4.5e-5 at
// K = 5120).  The K loop is therefore cut into segments of `seg` chunks of 32:
// each segment is accumulated from zero into one of two TMEM buffers, and the
// epilogue warps fold the finished buffer into fp32 register sums with
// round-to-nearest additions while the tensor cores fill the other buffer.
// The tensor-core error is then bounded by one segment.
//
// NPHASE = 2 (chi0) splits K into two contractions with separate sums: the
// first `nchunk0` chunks (occupied bands, Go) and the rest (unoccupied, Gu^T).
//
// Roles (320 threads, one CTA per SM, persistent over work units):
//   warp 0      TMA producer (one lane)
//   warp 1      TMEM allocation and MMA issue (one lane)
//   warps 2..9  epilogue: two warps per TMEM lane quarter, each owning TN/2
//               columns of its 32 rows
// Every wait is bounded in time; a timeout raises a status code and the CTA
// drains and frees its TMEM before returning.
#pragma once

#include "lrs_internal.h"
#include "tc_common.cuh"

namespace lrs {

using namespace tc;

constexpr int TC_THREADS = 320;
constexpr int TC_EPI_WARPS = 8;
constexpr int MAX_K_POINTS = 64;

struct TcShape {
  int m_tiles, n_tiles, batches;
  int nchunk;        // K chunks of 32
  int nchunk0;       // chunks of the first contraction (NPHASE = 2)
  int seg;           // chunks per accumulation segment
  int a_batch_rows;  // row offset of batch b in A (0 = shared)
  int b_batch_rows;  // row offset of batch b in B (0 = shared)
  int a_im_rows;     // row offset of the imaginary planes in A
  int b_im_rows;     // row offset of the imaginary planes in B
  int units;         // total work units
  const struct SiteTile* sites;   // multi-site table (NULL: one problem)
  int nsites;
  int real_b;        // 1: B is real (its imaginary planes are neither loaded nor multiplied)
  int tri;           // 1 (site-table launches): only the tiles that reach the lower triangle of each output
};

struct Unit {
  int tm, tn, b;     // row tile, column tile, batch (frequency or k-point)
  int ya, yb;        // first operand rows of the unit in A and B
  int site;
  long long slab0;   // output offset of the site (multi-site launches)
  int ld;            // output leading dimension (multi-site launches)
  int m_valid, n_valid;   // extent of the output (multi-site launches)
};

// Units of a launch.  With a site table the units of all sites are numbered
// site after site (every unit has the same K, hence the same cost, so the
// static round-robin over CTAs stays balanced for uneven sites).
template <int TN>
__device__ __forceinline__ Unit decode_unit(const TcShape& sh, const SiteTile* __restrict__ sites, int nsites,
                                            int u) {
  Unit x;
  if (sites) {
    int lo = 0, hi = nsites - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sites[mid].unit0 <= u) lo = mid;
      else hi = mid - 1;
    }
    const SiteTile st = sites[lo];
    const int lu = u - st.unit0;
    x.b = lu % sh.batches;
    const int t = lu / sh.batches;
    if (sh.tri) {
      // row tile tm holds the q (tm + 1) column tiles that reach the diagonal; it starts at
      // unit q tm (tm + 1) / 2
      constexpr int q = TILE_M / TN;
      int tm = (int)((sqrtf(8.f * (float)t / q + 1.f) - 1.f) * 0.5f);
      while (tm > 0 && q * tm * (tm + 1) / 2 > t) --tm;
      while (q * (tm + 1) * (tm + 2) / 2 <= t) ++tm;
      x.tm = tm;
      x.tn = t - q * tm * (tm + 1) / 2;
    } else {
      x.tm = t / st.n_tiles;
      x.tn = t % st.n_tiles;
    }
    x.ya = st.a_row0 + x.b * st.np + x.tm * TILE_M;
    x.yb = st.b_row0 + x.tn * TN;
    x.site = lo;
    x.slab0 = st.slab0;
    x.ld = st.ldc;
    x.m_valid = st.m_valid;
    x.n_valid = st.n_valid;
  } else {
    x.b = u % sh.batches;
    const int t = u / sh.batches;
    x.tm = t / sh.n_tiles;
    x.tn = t % sh.n_tiles;
    x.ya = x.b * sh.a_batch_rows + x.tm * TILE_M;
    x.yb = x.b * sh.b_batch_rows + x.tn * TN;
    x.site = 0;
    x.slab0 = 0;
    x.ld = sh.m_tiles * TILE_M;
    x.m_valid = x.ld;
    x.n_valid = sh.n_tiles * TN;
  }
  return x;
}

// Segments of a unit: phase 0 covers chunks [0, c0), phase 1 [c0, nchunk).
template <int NPHASE>
struct SegPlan {
  int c0, nchunk, seg;
  __device__ __forceinline__ int count() const {
    if (NPHASE == 1) return (nchunk + seg - 1) / seg;
    return (c0 + seg - 1) / seg + (nchunk - c0 + seg - 1) / seg;
  }
  __device__ __forceinline__ int count_phase0() const { return (c0 + seg - 1) / seg; }
  // first chunk, chunk count and phase of segment i
  __device__ __forceinline__ void get(int i, int& first, int& len, int& phase) const {
    const int n0 = (NPHASE == 1) ? count() : (c0 + seg - 1) / seg;
    if (i < n0) {
      phase = 0;
      first = i * seg;
      const int end = (NPHASE == 1) ? nchunk : c0;
      len = min(seg, end - first);
    } else {
      phase = 1;
      first = c0 + (i - n0) * seg;
      len = min(seg, nchunk - first);
    }
  }
};

template <int TN>
__host__ __device__ constexpr int tc_stage_bytes() {
  return 2 * TILE_BYTES + 2 * (TN * 128);   // A re, A im (128 rows) + B re, B im (TN rows)
}

template <int TN>
__host__ __device__ constexpr int tc_stages() {
  return (200 * 1024) / tc_stage_bytes<TN>() > 6 ? 6 : (200 * 1024) / tc_stage_bytes<TN>();
}

template <int TN>
__host__ __device__ constexpr int tc_smem_bytes() {
  return tc_stages<TN>() * tc_stage_bytes<TN>() + 1024;
}

// One K16 step of a complex product D = A B^T from hi/lo split planes (offsets hi, lo within
// the 128-byte rows):  Re += Ar Br - Ai Bi, Im += Ar Bi + Ai Br, each real product as the three
// split terms hi hi + hi lo + lo hi.  The two products of one A hi tile into the same accumulator
// are issued back to back with A kept in the collector buffer (8 reads of A instead of 12); the
// minus sign of Ai Bi is the A negation bit.  a0 = 0 starts both accumulators.
template <uint32_t FMT, int TN>
__device__ __forceinline__ void cplx_products(uint32_t dre, uint32_t dim, uint32_t aR, uint32_t aI, uint32_t bR,
                                              uint32_t bI, uint32_t hi, uint32_t lo, uint32_t a0) {
  constexpr uint32_t P = idesc_f16(TILE_M, TN, FMT, false);
  constexpr uint32_t N = idesc_f16(TILE_M, TN, FMT, true);
  mma_f16a<A_FILL>(dre, sw128_desc(aR + hi), sw128_desc(bR + hi), P, a0);
  mma_f16a<A_LAST>(dre, sw128_desc(aR + hi), sw128_desc(bR + lo), P, 1u);
  mma_f16a<A_ONCE>(dre, sw128_desc(aR + lo), sw128_desc(bR + hi), P, 1u);
  mma_f16a<A_FILL>(dre, sw128_desc(aI + hi), sw128_desc(bI + hi), N, 1u);
  mma_f16a<A_LAST>(dre, sw128_desc(aI + hi), sw128_desc(bI + lo), N, 1u);
  mma_f16a<A_ONCE>(dre, sw128_desc(aI + lo), sw128_desc(bI + hi), N, 1u);
  mma_f16a<A_FILL>(dim, sw128_desc(aR + hi), sw128_desc(bI + hi), P, a0);
  mma_f16a<A_LAST>(dim, sw128_desc(aR + hi), sw128_desc(bI + lo), P, 1u);
  mma_f16a<A_ONCE>(dim, sw128_desc(aR + lo), sw128_desc(bI + hi), P, 1u);
  mma_f16a<A_FILL>(dim, sw128_desc(aI + hi), sw128_desc(bR + hi), P, 1u);
  mma_f16a<A_LAST>(dim, sw128_desc(aI + hi), sw128_desc(bR + lo), P, 1u);
  mma_f16a<A_ONCE>(dim, sw128_desc(aI + lo), sw128_desc(bR + hi), P, 1u);
}

// The same step with B real: Re += Ar Br, Im += Ai Br.
template <uint32_t FMT, int TN>
__device__ __forceinline__ void cplx_products_real_b(uint32_t dre, uint32_t dim, uint32_t aR, uint32_t aI,
                                                     uint32_t bR, uint32_t hi, uint32_t lo, uint32_t a0) {
  constexpr uint32_t P = idesc_f16(TILE_M, TN, FMT, false);
  mma_f16a<A_FILL>(dre, sw128_desc(aR + hi), sw128_desc(bR + hi), P, a0);
  mma_f16a<A_LAST>(dre, sw128_desc(aR + hi), sw128_desc(bR + lo), P, 1u);
  mma_f16a<A_ONCE>(dre, sw128_desc(aR + lo), sw128_desc(bR + hi), P, 1u);
  mma_f16a<A_FILL>(dim, sw128_desc(aI + hi), sw128_desc(bR + hi), P, a0);
  mma_f16a<A_LAST>(dim, sw128_desc(aI + hi), sw128_desc(bR + lo), P, 1u);
  mma_f16a<A_ONCE>(dim, sw128_desc(aI + lo), sw128_desc(bR + hi), P, 1u);
}

// ---------------------------------------------------------------- the kernel
template <int TN, int NPHASE, uint32_t FMT, class Epi, bool DIRECT = false>
__global__ void __launch_bounds__(TC_THREADS, 1)
    zgemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const TcShape sh, const Epi epi, int* status) {
  constexpr int STAGES = tc_stages<TN>();
  constexpr int STAGE_BYTES = tc_stage_bytes<TN>();
  constexpr int B_TILE = TN * 128;
  constexpr uint32_t SET_COLS = 2 * TN;             // re + im of one complex accumulator
  constexpr uint32_t TMEM_COLS = 2 * SET_COLS < 32 ? 32 : 2 * SET_COLS;
  constexpr int COLS = TN / 2;                       // columns per epilogue thread
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = sh.units;
  const SegPlan<NPHASE> plan{sh.nchunk0, sh.nchunk, sh.seg};

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], TC_EPI_WARPS);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_map(&tmA);
    tma_prefetch_map(&tmB);
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const Unit x = decode_unit<TN>(sh, sh.sites, sh.nsites, u);
        const int ya = x.ya, yb = x.yb;
        for (int c = 0; c < sh.nchunk; ++c) {
          if (!mbar_wait(&empty_bar[stage], phase ^ 1u, &abort_flag)) {
            abort_flag = 1;
            atomicCAS(status, 0, TC_TIMEOUT_PRODUCER);
            goto producer_done;
          }
          mbar_arrive_expect_tx(&full_bar[stage], sh.real_b ? STAGE_BYTES - B_TILE : STAGE_BYTES);
          const uint32_t s = smem_base + stage * STAGE_BYTES;
          tma_load_2d(s, &tmA, &full_bar[stage], c * 64, ya);
          tma_load_2d(s + TILE_BYTES, &tmA, &full_bar[stage], c * 64, ya + sh.a_im_rows);
          tma_load_2d(s + 2 * TILE_BYTES, &tmB, &full_bar[stage], c * 64, yb);
          if (!sh.real_b)
            tma_load_2d(s + 2 * TILE_BYTES + B_TILE, &tmB, &full_bar[stage], c * 64, yb + sh.b_im_rows);
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
      }
    producer_done:;
    }
  } else if (DIRECT && warp == 1) {
    // ------------------------------------------------ MMA issue, short K: Go whole into set 0, Gu^T into set 1
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, unit_phase = 0;
      const bool real_b = sh.real_b != 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        // both sets free: the epilogue has read the previous unit
        if (!mbar_wait(&acce_bar[0], unit_phase ^ 1u, &abort_flag)) {
          abort_flag = 1;
          atomicCAS(status, 0, TC_TIMEOUT_MMA);
          break;
        }
        tc_fence_after();
        for (int c = 0; c < sh.nchunk; ++c) {
          if (!mbar_wait(&full_bar[stage], phase, &abort_flag)) {
            abort_flag = 1;
            atomicCAS(status, 0, TC_TIMEOUT_MMA);
            ok = false;
            break;
          }
          tc_fence_after();
          const int set = c < sh.nchunk0 ? 0 : 1;
          const int cl = set ? c - sh.nchunk0 : c;              // chunk within its contraction
          const uint32_t dre = tbase + set * SET_COLS, dim = dre + TN;
          const uint32_t s = smem_base + stage * STAGE_BYTES;
          const uint32_t aR = s, aI = s + TILE_BYTES, bR = s + 2 * TILE_BYTES, bI = bR + B_TILE;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint32_t a0 = (cl == 0 && ks == 0) ? 0u : 1u;
            if (real_b) cplx_products_real_b<FMT, TN>(dre, dim, aR, aI, bR, 32 * ks, 64 + 32 * ks, a0);
            else cplx_products<FMT, TN>(dre, dim, aR, aI, bR, bI, 32 * ks, 64 + 32 * ks, a0);
          }
          mma_commit(&empty_bar[stage]);
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(&accf_bar[1]);   // completes once every product of the unit has landed
        unit_phase ^= 1u;
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issue
    if (lane == 0) {
      int stage = 0, set = 0;
      uint32_t phase = 0, set_phase = 0;
      const int nseg = plan.count();
      const bool real_b = sh.real_b != 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        for (int sg = 0; sg < nseg && ok; ++sg) {
          int first, len, ph;
          plan.get(sg, first, len, ph);
          (void)first;
          (void)ph;
          if (!mbar_wait(&acce_bar[set], set_phase ^ 1u, &abort_flag)) {
            abort_flag = 1;
            atomicCAS(status, 0, TC_TIMEOUT_MMA);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dre = tbase + set * SET_COLS, dim = dre + TN;
          for (int c = 0; c < len; ++c) {
            if (!mbar_wait(&full_bar[stage], phase, &abort_flag)) {
              abort_flag = 1;
              atomicCAS(status, 0, TC_TIMEOUT_MMA);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t s = smem_base + stage * STAGE_BYTES;
            const uint32_t aR = s, aI = s + TILE_BYTES, bR = s + 2 * TILE_BYTES, bI = bR + B_TILE;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint32_t a0 = (c == 0 && ks == 0) ? 0u : 1u;
              // real B (Gamma-point real orbitals): Re = Ar Br, Im = Ai Br
              if (real_b) cplx_products_real_b<FMT, TN>(dre, dim, aR, aI, bR, 32 * ks, 64 + 32 * ks, a0);
              else cplx_products<FMT, TN>(dre, dim, aR, aI, bR, bI, 32 * ks, 64 + 32 * ks, a0);
            }
            mma_commit(&empty_bar[stage]);
            if (++stage == STAGES) { stage = 0; phase ^= 1u; }
          }
          if (!ok) break;
          mma_commit(&accf_bar[set]);
          set ^= 1;
          if (set == 0) set_phase ^= 1u;
        }
      }
    }
  } else if (DIRECT) {
    // ------------------------------------------------ epilogue, short K: both contractions read from TMEM
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
    const int lrow = quarter * 32 + lane, lcol0 = half * COLS;
    uint32_t unit_phase = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
      const Unit x = decode_unit<TN>(sh, sh.sites, sh.nsites, u);
      int got = 1;
      if (lane == 0) got = mbar_wait(&accf_bar[1], unit_phase, &abort_flag) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      __syncwarp();
      if (!got) {
        if (lane == 0) {
          abort_flag = 1;
          atomicCAS(status, 0, TC_TIMEOUT_EPILOGUE);
        }
        break;
      }
      tc_fence_after();
      const uint32_t tb = tbase + lane_off + lcol0;
#pragma unroll 1
      for (int j = 0; j < COLS / 16; ++j) {
        float gr[16], gi[16], ur[16], ui[16];
        tmem_ld16(tb + 16 * j, gr);                     // Go re, im (set 0)
        tmem_ld16(tb + TN + 16 * j, gi);
        tmem_ld16(tb + SET_COLS + 16 * j, ur);          // Gu^T re, im (set 1)
        tmem_ld16(tb + SET_COLS + TN + 16 * j, ui);
        tmem_ld_wait();
        epi.store_direct16(gr, gi, ur, ui, x, x.tm * TILE_M + lrow, x.tn * TN + lcol0 + 16 * j);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce_bar[0]);
      unit_phase ^= 1u;
    }
  } else {
    // ------------------------------------------------ epilogue (warps 2..9)
    const int quarter = warp & 3;                 // TMEM lanes 32*quarter .. +31
    const int half = (warp - 2) >> 2;             // column half of the tile
    const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
    // Register sums (re, im) of the contraction in progress.  For NPHASE = 2 the
    // occupied sums are parked in the epilogue's scratch at the phase switch.
    float sum[2][COLS];
    int set = 0;
    uint32_t set_phase = 0;
    const int nseg = plan.count();
    const int lrow = quarter * 32 + lane, lcol0 = half * COLS;
    bool ok = true;
    for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const Unit x = decode_unit<TN>(sh, sh.sites, sh.nsites, u);
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int i = 0; i < COLS; ++i) sum[q][i] = 0.f;
      for (int sg = 0; sg < nseg; ++sg) {
        int first, len, ph;
        plan.get(sg, first, len, ph);
        (void)first;
        (void)len;
        if (NPHASE == 2 && ph == 1 && (sg == 0 || sg == plan.count_phase0())) {
          epi.template save_phase0<COLS>(sum, lrow, lcol0);
#pragma unroll
          for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int i = 0; i < COLS; ++i) sum[q][i] = 0.f;
        }
        int got = 1;
        if (lane == 0) got = mbar_wait(&accf_bar[set], set_phase, &abort_flag) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        __syncwarp();
        if (!got) {
          if (lane == 0) {
            abort_flag = 1;
            atomicCAS(status, 0, TC_TIMEOUT_EPILOGUE);
          }
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tb = tbase + lane_off + set * SET_COLS + half * COLS;
#pragma unroll
        for (int j = 0; j < COLS / 16; ++j) {
#pragma unroll
          for (int part = 0; part < 2; ++part) {   // re, then im: 16 registers in flight
            float v[16];
            tmem_ld16(tb + part * TN + 16 * j, v);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i) sum[part][16 * j + i] += v[i];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce_bar[set]);
        set ^= 1;
        if (set == 0) set_phase ^= 1u;
      }
      if (!ok) break;
      epi.template store<COLS>(sum, x, x.tm * TILE_M + lrow, lrow, x.tn * TN + lcol0, lcol0);
    }
  }

  __syncthreads();
  if (abort_flag) {
    // let copies and MMAs already issued land before the shared memory and TMEM go away
    const uint64_t t0 = global_timer_ns();
    while (global_timer_ns() - t0 < 200000ull) {
    }
  }
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, TMEM_COLS);
  }
}

template <int TN, int NPHASE, uint32_t FMT, class Epi, bool DIRECT = false>
int launch_tc(lrs_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb, const TcShape& sh, const Epi& epi,
              const char* name) {
  static_assert(!DIRECT || (NPHASE == 2 && Epi::kDirect), "short-K mode: two contractions, chi0 epilogue");
  constexpr int smem = tc_smem_bytes<TN>();
  if (!ctx->capturing)
    LRS_CUDA_TRY(cudaFuncSetAttribute(zgemm_tc_kernel<TN, NPHASE, FMT, Epi, DIRECT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int grid = std::min(sh.units, ctx->num_sms);
  if (grid <= 0) return LRS_OK;
  // The persistent tensor-core CTAs take the highest launch priority, so that on
  // SMs shared with FP64 kernels of another build (or stream) they are placed
  // first and the smaller FP64 CTAs fill the remaining shared memory.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = ctx->prio_greatest;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, zgemm_tc_kernel<TN, NPHASE, FMT, Epi, DIRECT>, ma, mb, sh, epi,
                                     ctx->ws.status.ptr + 8);
  if (e != cudaSuccess) return set_error(LRS_ERR_CUDA, "%s launch: %s", name, cudaGetErrorString(e));
  return after_launch(ctx, name);
}

// Index of element (row, col) in one frequency's fp32 slab of a site padded to Np (a multiple of
// 128): each 128-row band is stored as [col / 4][row % 128][4], so that a warp writing (or
// reading) one float4 of columns for 32 consecutive rows covers 512 consecutive bytes.
__host__ __device__ __forceinline__ size_t slab_index(int Np, int row, int col) {
  return (size_t)(row >> 7) * 128 * Np + (size_t)(col >> 2) * 512 + (size_t)(row & 127) * 4 + (col & 3);
}

// ---------------------------------------------------------------- epilogue stores
// Slot of a parked value in a CTA's scratch ([2][128][2 COLS] floats): the 256 epilogue threads
// (row lrow of the tile, column half lcol0 / COLS) keep their float4 chunks interleaved, chunk c
// of part p of thread t at ((p COLS / 4 + c) 256 + t) float4s, so that a warp's 32 lanes touch
// 512 consecutive bytes per access; each thread reads back only what it wrote.
template <int COLS>
__device__ __forceinline__ float* park_slot(float* scratch, int lrow, int lcol0, int part, int i) {
  const int t = lrow + (lcol0 / COLS) * 128;
  return scratch + (size_t)blockIdx.x * 2 * 128 * (2 * COLS) +
         ((size_t)(part * (COLS / 4) + (i >> 2)) * 256 + t) * 4;
}
// chi0: X = Re[Go o Gu^T] of one frequency into its fp32 slab (layout of slab_index).
// The occupied sums Go of a unit are parked in `scratch` (per CTA
// [2][128][tile_n] fp32, L2 resident) while the unoccupied sums accumulate in
// registers; each thread reads back only what it wrote.
struct Chi0Store {
  static constexpr bool kDirect = true;
  float* slab;      // [batches][ld][ld]
  float* scratch;   // [gridDim.x][2][128][tile_n]
  int ld, tile_n;
  // Short K: both contractions of 16 columns of this thread's row, read straight from TMEM.
  __device__ void store_direct16(const float (&gr)[16], const float (&gi)[16], const float (&ur)[16],
                                 const float (&ui)[16], const Unit& x, int row, int col) const {
    float* plane = slab + x.slab0 + (size_t)x.b * x.ld * x.ld;
#pragma unroll
    for (int i = 0; i < 16; i += 4) {
      float4 v;
      v.x = fmaf(-gi[i + 0], ui[i + 0], gr[i + 0] * ur[i + 0]);
      v.y = fmaf(-gi[i + 1], ui[i + 1], gr[i + 1] * ur[i + 1]);
      v.z = fmaf(-gi[i + 2], ui[i + 2], gr[i + 2] * ur[i + 2]);
      v.w = fmaf(-gi[i + 3], ui[i + 3], gr[i + 3] * ur[i + 3]);
      *reinterpret_cast<float4*>(plane + slab_index(x.ld, row, col + i)) = v;
    }
  }
  template <int COLS>
  __device__ void save_phase0(const float (&s)[2][COLS], int lrow, int lcol0) const {
#pragma unroll
    for (int part = 0; part < 2; ++part)
#pragma unroll
      for (int i = 0; i < COLS; i += 4)
        *reinterpret_cast<float4*>(park_slot<COLS>(scratch, lrow, lcol0, part, i)) =
            make_float4(s[part][i], s[part][i + 1], s[part][i + 2], s[part][i + 3]);
  }
  template <int COLS>
  __device__ void store(const float (&s)[2][COLS], const Unit& x, int row, int lrow, int col0, int lcol0) const {
    float* plane = slab + x.slab0 + (size_t)x.b * x.ld * x.ld;
#pragma unroll
    for (int i = 0; i < COLS; i += 4) {
      const float4 r = *reinterpret_cast<const float4*>(park_slot<COLS>(scratch, lrow, lcol0, 0, i));
      const float4 m = *reinterpret_cast<const float4*>(park_slot<COLS>(scratch, lrow, lcol0, 1, i));
      float4 v;
      v.x = fmaf(-m.x, s[1][i + 0], r.x * s[0][i + 0]);
      v.y = fmaf(-m.y, s[1][i + 1], r.y * s[0][i + 1]);
      v.z = fmaf(-m.z, s[1][i + 2], r.z * s[0][i + 2]);
      v.w = fmaf(-m.w, s[1][i + 3], r.w * s[0][i + 3]);
      *reinterpret_cast<float4*>(plane + slab_index(x.ld, row, col0 + i)) = v;
    }
  }
};

// Adjoint: the Green's functions themselves, Go and Gu^T of one frequency,
// as complex fp32 [np][np] (ld = unit.ld).
struct GStore {
  static constexpr bool kDirect = false;
  __device__ void store_direct16(const float (&)[16], const float (&)[16], const float (&)[16], const float (&)[16],
                                 const Unit&, int, int) const {}
  float2* go;
  float2* gu;
  float* scratch;   // [gridDim.x][2][128][tile_n]
  int tile_n;
  template <int COLS>
  __device__ void save_phase0(const float (&s)[2][COLS], int lrow, int lcol0) const {
#pragma unroll
    for (int part = 0; part < 2; ++part)
#pragma unroll
      for (int i = 0; i < COLS; i += 4)
        *reinterpret_cast<float4*>(park_slot<COLS>(scratch, lrow, lcol0, part, i)) =
            make_float4(s[part][i], s[part][i + 1], s[part][i + 2], s[part][i + 3]);
  }
  template <int COLS>
  __device__ void store(const float (&s)[2][COLS], const Unit& x, int row, int lrow, int col0, int lcol0) const {
    float2* po = go + x.slab0 + (size_t)row * x.ld + col0;
    float2* pu = gu + x.slab0 + (size_t)row * x.ld + col0;
#pragma unroll
    for (int i = 0; i < COLS; i += 2) {
      const float* g0 = park_slot<COLS>(scratch, lrow, lcol0, 0, i & ~3) + (i & 3);
      const float* g1 = park_slot<COLS>(scratch, lrow, lcol0, 1, i & ~3) + (i & 3);
      const float2 r = *reinterpret_cast<const float2*>(g0);
      const float2 m = *reinterpret_cast<const float2*>(g1);
      *reinterpret_cast<float4*>(po + i) = make_float4(r.x, m.x, r.y, m.y);
      *reinterpret_cast<float4*>(pu + i) = make_float4(s[0][i], s[1][i], s[0][i + 1], s[1][i + 1]);
    }
  }
};

// Adjoint: a plain complex product D (fp32 re, im) into out + unit.slab0,
// rows < m_valid, columns < n_valid.
struct ZStore {
  static constexpr bool kDirect = false;
  __device__ void store_direct16(const float (&)[16], const float (&)[16], const float (&)[16], const float (&)[16],
                                 const Unit&, int, int) const {}
  float2* out;
  template <int COLS>
  __device__ void save_phase0(const float (&)[2][COLS], int, int) const {}
  template <int COLS>
  __device__ void store(const float (&s)[2][COLS], const Unit& x, int row, int lrow, int col0, int lcol0) const {
    (void)lrow;
    (void)lcol0;
    if (row >= x.m_valid) return;
    float2* dst = out + x.slab0 + (size_t)row * x.ld + col0;
#pragma unroll
    for (int i = 0; i < COLS; ++i)
      if (col0 + i < x.n_valid) dst[i] = make_float2(s[0][i], s[1][i]);
  }
};

// projection: psi(p, b) = e^{ik.R_p}/sqrt(Omega) * unscale * D(p, b), scattered
// into the occupied / unoccupied orbital blocks.
struct ProjStore {
  static constexpr bool kDirect = false;
  __device__ void store_direct16(const float (&)[16], const float (&)[16], const float (&)[16], const float (&)[16],
                                 const Unit&, int, int) const {}
  const double2* kph;     // [nk][npts]
  const float* unscale;   // device scalar
  int npts, nb;
  double2* psi_o;
  double2* psi_u;
  int Ko, Ku;
  int nocc[MAX_K_POINTS], oofs[MAX_K_POINTS], uofs[MAX_K_POINTS];
  template <int COLS>
  __device__ void save_phase0(const float (&)[2][COLS], int, int) const {}
  template <int COLS>
  __device__ void store(const float (&s)[2][COLS], const Unit& x, int row, int lrow, int col0, int lcol0) const {
    (void)lrow;
    (void)lcol0;
    const int k = x.b;
    if (row >= npts) return;
    const double us = (double)*unscale;
    const double2 ph = kph[(size_t)k * npts + row];
    const float pr = (float)(ph.x * us), pi = (float)(ph.y * us);
    const int no = nocc[k];
#pragma unroll
    for (int i = 0; i < COLS; ++i) {
      const int band = col0 + i;
      if (band >= nb) continue;
      const float a = s[0][i], c = s[1][i];
      // widened with integer instructions (GB300 converts on its float64 pipe)
      const double2 v = make_double2(f32_to_f64_exact(pr * a - pi * c), f32_to_f64_exact(pr * c + pi * a));
      if (band < no) psi_o[(size_t)row * Ko + oofs[k] + band] = v;
      else psi_u[(size_t)row * Ku + uofs[k] + band - no] = v;
    }
  }
};

}  // namespace lrs
