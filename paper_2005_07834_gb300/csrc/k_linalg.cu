// Float64 dense linear algebra of the Dyson step (Sec. VI.E; Eq. (eq-reducible)
// and (eq-W) give (I - v Q chi0 Q) W = v on the grid):
//   dgemm         C = alpha op(A) diag(ks) op(B) diag(cs) + beta C
//   lu_panel      unblocked LU with partial pivoting of a column panel
//   laswp         row interchanges outside the panel
//   trsm          triangular solves with a jb x jb diagonal block
// and the right-looking blocked LU plus forward/backward substitution that
// solve for W with all npts right-hand sides.  The FP64 pipe of GB300 retires
// about two DFMA per SM clock, so every kernel here is bound by DFMA issue;
// the tiling only has to keep all SMs busy.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>

#include "lrs_internal.h"
#include "oz_slice.cuh"

namespace lrs {

constexpr int GT = 64;   // dgemm tile edge
constexpr int GKC = 16;  // dgemm k chunk
constexpr int NB = 32;   // LU panel width

// Element offsets between the matrices of consecutive batch entries (blockIdx.z).
struct BatchStrides {
  long long a = 0, ks = 0, b = 0, c = 0;
  // > 0: C is the column block blockIdx.z * lower_col of a symmetric matrix and
  // only tiles holding an element on or below its diagonal are computed
  int lower_col = 0;
};

// C tile of GT rows x TNW columns per CTA (TNW = 64, 96 or 112: the 81- and
// 110-wide products of the lm-basis change fit one tile), 256 threads, each
// 4 rows x TNW/16 columns.
template <bool TA, bool TB, int TNW>
__global__ void __launch_bounds__(256) dgemm_kernel(int m, int n, int k, double alpha,
                                                    const double* __restrict__ A, int lda,
                                                    const double* __restrict__ ks,
                                                    const double* __restrict__ B, int ldb,
                                                    const double* __restrict__ cs, double beta,
                                                    double* __restrict__ C, int ldc, BatchStrides bs) {
  constexpr int CJ = TNW / 16;
  __shared__ double As[GKC][GT + 1];
  __shared__ double Bs[GKC][TNW + 1];
  A += bs.a * blockIdx.z;
  B += bs.b * blockIdx.z;
  C += bs.c * blockIdx.z;
  if (ks) ks += bs.ks * blockIdx.z;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * GT, j0 = blockIdx.x * TNW;
  if (bs.lower_col > 0 && i0 + GT <= (int)blockIdx.z * bs.lower_col + j0) return;
  double acc[4][CJ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CJ; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < k; k0 += GKC) {
    for (int idx = threadIdx.x; idx < GKC * GT; idx += 256) {
      int r, kk;
      if (TA) { kk = idx / GT; r = idx % GT; } else { r = idx / GKC; kk = idx % GKC; }
      int gi = i0 + r, gk = k0 + kk;
      double a = 0.0;
      if (gi < m && gk < k) {
        a = TA ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk];
        if (ks) a *= ks[gk];
      }
      As[kk][r] = a;
    }
    for (int idx = threadIdx.x; idx < GKC * TNW; idx += 256) {
      int c, kk;
      if (TB) { c = idx / GKC; kk = idx % GKC; } else { kk = idx / TNW; c = idx % TNW; }
      int gj = j0 + c, gk = k0 + kk;
      double b = 0.0;
      if (gj < n && gk < k) b = TB ? B[(size_t)gj * ldb + gk] : B[(size_t)gk * ldb + gj];
      Bs[kk][c] = b;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GKC; ++kk) {
      double a[4], b[CJ];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < CJ; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CJ; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gi = i0 + ty + 16 * i;
    if (gi >= m) continue;
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
      int gj = j0 + tx + 16 * j;
      if (gj >= n) continue;
      double v = alpha * acc[i][j];
      if (cs) v *= cs[gj];
      double* c = &C[(size_t)gi * ldc + gj];
      *c = (beta == 0.0) ? v : fma(beta, *c, v);
    }
  }
}

template <int TNW>
static void launch_dgemm(lrs_ctx* ctx, bool ta, bool tb, dim3 grid, int m, int n, int k, double alpha,
                         const double* a, int lda, const double* ks, const double* b, int ldb, const double* cs,
                         double beta, double* c, int ldc, const BatchStrides& bs) {
  if (!ta && !tb)
    dgemm_kernel<false, false, TNW><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, a, lda, ks, b, ldb, cs, beta, c, ldc, bs);
  else if (ta && !tb)
    dgemm_kernel<true, false, TNW><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, a, lda, ks, b, ldb, cs, beta, c, ldc, bs);
  else if (!ta && tb)
    dgemm_kernel<false, true, TNW><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, a, lda, ks, b, ldb, cs, beta, c, ldc, bs);
  else
    dgemm_kernel<true, true, TNW><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, a, lda, ks, b, ldb, cs, beta, c, ldc, bs);
}

int dgemm_batched(lrs_ctx* ctx, bool ta, bool tb, int m, int n, int k, double alpha, const double* a, int lda,
                  long long stride_a, const double* ks, long long stride_ks, const double* b, int ldb,
                  long long stride_b, const double* cs, double beta, double* c, int ldc, long long stride_c,
                  int batch) {
  if (m <= 0 || n <= 0 || batch <= 0) return LRS_OK;
  ctx->fp64_flops += 2.0 * m * (double)n * (k > 0 ? k : 0) * batch;
  // tile width: one tile for 64 < n <= 112 (less padding than two 64-wide tiles)
  const int tnw = (n > 64 && n <= 96) ? 96 : (n > 96 && n <= 112) ? 112 : 64;
  dim3 grid((n + tnw - 1) / tnw, (m + GT - 1) / GT, batch);
  if (k <= 0) k = 0;
  BatchStrides bs;
  bs.a = stride_a;
  bs.ks = stride_ks;
  bs.b = stride_b;
  bs.c = stride_c;
  if (tnw == 96) launch_dgemm<96>(ctx, ta, tb, grid, m, n, k, alpha, a, lda, ks, b, ldb, cs, beta, c, ldc, bs);
  else if (tnw == 112) launch_dgemm<112>(ctx, ta, tb, grid, m, n, k, alpha, a, lda, ks, b, ldb, cs, beta, c, ldc, bs);
  else launch_dgemm<64>(ctx, ta, tb, grid, m, n, k, alpha, a, lda, ks, b, ldb, cs, beta, c, ldc, bs);
  return after_launch(ctx, "dgemm_kernel");
}

int dgemm_batched_lower(lrs_ctx* ctx, bool ta, bool tb, int m, int n, int k, const double* a, int lda,
                        long long stride_a, const double* ks, long long stride_ks, const double* b, int ldb,
                        double* c, int ldc, int batch) {
  if (m <= 0 || n <= 0 || batch <= 0) return LRS_OK;
  ctx->fp64_flops += 1.0 * m * (double)n * (k > 0 ? k : 0) * batch;   // about half the tiles
  const int tnw = (n > 64 && n <= 96) ? 96 : (n > 96 && n <= 112) ? 112 : 64;
  dim3 grid((n + tnw - 1) / tnw, (m + GT - 1) / GT, batch);
  BatchStrides bs;
  bs.a = stride_a;
  bs.ks = stride_ks;
  bs.c = n;
  bs.lower_col = n;
  if (tnw == 96) launch_dgemm<96>(ctx, ta, tb, grid, m, n, k, 1.0, a, lda, ks, b, ldb, nullptr, 0.0, c, ldc, bs);
  else if (tnw == 112) launch_dgemm<112>(ctx, ta, tb, grid, m, n, k, 1.0, a, lda, ks, b, ldb, nullptr, 0.0, c, ldc, bs);
  else launch_dgemm<64>(ctx, ta, tb, grid, m, n, k, 1.0, a, lda, ks, b, ldb, nullptr, 0.0, c, ldc, bs);
  return after_launch(ctx, "dgemm_kernel");
}

// Upper triangle of a symmetric matrix from its lower triangle (32 x 32 tiles).
__global__ void __launch_bounds__(256) mirror_lower_kernel(double* __restrict__ a, int n, int lda) {
  __shared__ double t[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;   // destination tile (bi, bj), bi <= bj
  if (bi > bj) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {   // source tile (bj, bi), row bj*32 + r
    const int i = bj * 32 + r, j = bi * 32 + tx;
    t[r][tx] = (i < n && j < n) ? a[(size_t)i * lda + j] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = bi * 32 + r, j = bj * 32 + tx;
    if (i < n && j < n && j > i) a[(size_t)i * lda + j] = t[tx][r];
  }
}

int mirror_lower(lrs_ctx* ctx, double* a, int n, int lda) {
  if (n <= 0) return LRS_OK;
  const int nb = (n + 31) / 32;
  mirror_lower_kernel<<<dim3(nb, nb), 256, 0, ctx->stream>>>(a, n, lda);
  return after_launch(ctx, "mirror_lower_kernel");
}

int dgemm_t(lrs_ctx* ctx, bool ta, bool tb, int m, int n, int k, double alpha, const double* a, int lda,
            const double* ks, const double* b, int ldb, const double* cs, double beta, double* c, int ldc) {
  return dgemm_batched(ctx, ta, tb, m, n, k, alpha, a, lda, 0, ks, 0, b, ldb, 0, cs, beta, c, ldc, 0, 1);
}

int dgemm(lrs_ctx* ctx, int m, int n, int k, double alpha, const double* a, int lda, const double* kscale,
          const double* b, int ldb, const double* cscale, double beta, double* c, int ldc) {
  return dgemm_t(ctx, false, false, m, n, k, alpha, a, lda, kscale, b, ldb, cscale, beta, c, ldc);
}

__global__ void add_identity_kernel(double* __restrict__ a, int n, int lda, double s) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[(size_t)i * lda + i] += s;
}

// Unblocked LU with partial pivoting of rows [j0, n) x columns [j0, j0+jb).
// One CTA; the panel stays in L2.  status[0] = 1 on a zero or non-finite
// pivot column (status[1] = that column), left for the host to report.
__global__ void __launch_bounds__(1024) lu_panel_kernel(double* __restrict__ A, int lda, int n, int j0, int jb,
                                                        int* __restrict__ ipiv, int* __restrict__ status) {
  __shared__ double s_val[32];
  __shared__ int s_idx[32];
  __shared__ int s_bad[32];
  __shared__ double urow[NB];
  __shared__ int s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  for (int c = 0; c < jb; ++c) {
    const int col = j0 + c;
    double best = -1.0;
    int bi = n;
    int bad = 0;
    for (int r = col + tid; r < n; r += blockDim.x) {
      double a = A[(size_t)r * lda + col];
      if (!isfinite(a)) bad = 1;
      double m = fabs(a);
      if (m > best) { best = m; bi = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_down_sync(0xffffffffu, best, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      bad |= __shfl_down_sync(0xffffffffu, bad, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; s_bad[warp] = bad; }
    __syncthreads();
    if (warp == 0) {
      best = lane < nwarp ? s_val[lane] : -1.0;
      bi = lane < nwarp ? s_idx[lane] : n;
      bad = lane < nwarp ? s_bad[lane] : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_down_sync(0xffffffffu, best, o);
        int oi = __shfl_down_sync(0xffffffffu, bi, o);
        bad |= __shfl_down_sync(0xffffffffu, bad, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        if (bi >= n) bi = col;
        s_piv = bi;
        ipiv[col] = bi;
        if ((bad || !(best > 0.0)) && atomicCAS(&status[0], 0, 1) == 0) status[1] = col;
      }
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != col) {
      for (int j = tid; j < jb; j += blockDim.x) {
        double t = A[(size_t)col * lda + j0 + j];
        A[(size_t)col * lda + j0 + j] = A[(size_t)piv * lda + j0 + j];
        A[(size_t)piv * lda + j0 + j] = t;
      }
    }
    __syncthreads();
    if (tid < jb) urow[tid] = A[(size_t)col * lda + j0 + tid];
    __syncthreads();
    const double d = urow[c];
    const double inv = (d != 0.0) ? 1.0 / d : 0.0;
    for (int r = col + 1 + tid; r < n; r += blockDim.x) {
      double* row = A + (size_t)r * lda + j0;
      double l = row[c] * inv;
      row[c] = l;
      for (int j = c + 1; j < jb; ++j) row[j] = fma(-l, urow[j], row[j]);
    }
    __syncthreads();
  }
}

// Applies the interchanges ipiv[r0 .. r0+cnt) (in order) to every column
// except [skip0, skip0+skipn).  One thread per column.
__global__ void laswp_kernel(double* __restrict__ A, int lda, int ncols, const int* __restrict__ ipiv, int r0,
                             int cnt, int skip0, int skipn) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int col = t < skip0 ? t : t + skipn;
  if (t >= ncols - skipn || col >= ncols) return;
  for (int i = r0; i < r0 + cnt; ++i) {
    int p = ipiv[i];
    if (p != i) {
      double a = A[(size_t)i * lda + col];
      A[(size_t)i * lda + col] = A[(size_t)p * lda + col];
      A[(size_t)p * lda + col] = a;
    }
  }
}

// X = T^-1 B for a jb x jb triangular block T (lower unit or upper non-unit)
// and a jb x ncols block B, in place.  One thread per column of B.
template <bool kLowerUnit>
__global__ void trsm_kernel(const double* __restrict__ T, int ldt, int jb, double* __restrict__ B, int ldb,
                            int ncols) {
  __shared__ double Ts[NB][NB + 1];
  for (int idx = threadIdx.x; idx < jb * jb; idx += blockDim.x) {
    int i = idx / jb, j = idx % jb;
    Ts[i][j] = T[(size_t)i * ldt + j];
  }
  __syncthreads();
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncols) return;
  double x[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) x[i] = (i < jb) ? B[(size_t)i * ldb + col] : 0.0;
  if (kLowerUnit) {
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      if (i >= jb) break;
      double s = x[i];
#pragma unroll
      for (int k = 0; k < NB; ++k)
        if (k < i) s = fma(-Ts[i][k], x[k], s);
      x[i] = s;
    }
  } else {
#pragma unroll
    for (int ii = NB - 1; ii >= 0; --ii) {
      if (ii >= jb) continue;
      double s = x[ii];
#pragma unroll
      for (int k = 0; k < NB; ++k)
        if (k > ii && k < jb) s = fma(-Ts[ii][k], x[k], s);
      x[ii] = s / Ts[ii][ii];
    }
  }
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < jb) B[(size_t)i * ldb + col] = x[i];
}

// Panel LU held in the shared memory of one thread-block cluster.  The rows
// [j0, n) of the jb-wide panel are split into CS contiguous chunks, one per
// CTA.  Per column: each CTA finds its local pivot candidate; after a cluster
// barrier every CTA reads all candidates through distributed shared memory
// and agrees on the pivot (largest |a|, lowest row on ties); the owners of
// the pivot row and of the diagonal row publish them; after a second barrier
// the rows are exchanged and every CTA applies the rank-1 update to its rows.
// Same arithmetic and pivot choice as lu_panel_kernel, on-chip.
constexpr int PANEL_CS = 16;         // CTAs per cluster
constexpr int PANEL_THREADS = 512;

__global__ void __launch_bounds__(PANEL_THREADS) lu_panel_cluster_kernel(double* __restrict__ A, int lda, int n,
                                                                         int j0, int jb, int rows_per_cta,
                                                                         int* __restrict__ ipiv,
                                                                         int* __restrict__ status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ double panel[];                 // [rows_per_cta][NB]
  __shared__ double cand_val;
  __shared__ int cand_idx, cand_bad;
  __shared__ double prow[NB], crow[NB], urow[NB];
  __shared__ double w_val[PANEL_THREADS / 32];
  __shared__ int w_idx[PANEL_THREADS / 32], w_bad[PANEL_THREADS / 32];
  __shared__ int s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = j0 + rank * rows_per_cta;                       // first global row of this CTA
  const int nloc = max(0, min(rows_per_cta, n - r0));            // rows held here
  for (int i = tid; i < nloc * NB; i += PANEL_THREADS) {
    const int r = i / NB, c = i % NB;
    panel[i] = c < jb ? A[(size_t)(r0 + r) * lda + j0 + c] : 0.0;
  }
  __syncthreads();
  for (int c = 0; c < jb; ++c) {
    const int col = j0 + c;
    // 1. local candidate over rows >= col
    double best = -1.0;
    int bi = n, bad = 0;
    for (int r = tid; r < nloc; r += PANEL_THREADS) {
      if (r0 + r < col) continue;
      const double a = panel[r * NB + c];
      if (!isfinite(a)) bad = 1;
      const double m = fabs(a);
      if (m > best) { best = m; bi = r0 + r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      bad |= __shfl_down_sync(0xffffffffu, bad, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { w_val[warp] = best; w_idx[warp] = bi; w_bad[warp] = bad; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < PANEL_THREADS / 32; ++w) {
        if (w_val[w] > best || (w_val[w] == best && w_idx[w] < bi)) { best = w_val[w]; bi = w_idx[w]; }
        bad |= w_bad[w];
      }
      cand_val = best;
      cand_idx = bi;
      cand_bad = bad;
    }
    cluster.sync();
    // 2. agree on the pivot
    if (warp == 0) {
      double v = -1.0;
      int ix = n, bd = 0;
      if (lane < PANEL_CS) {
        v = *cluster.map_shared_rank(&cand_val, lane);
        ix = *cluster.map_shared_rank(&cand_idx, lane);
        bd = *cluster.map_shared_rank(&cand_bad, lane);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v, o);
        const int oi = __shfl_down_sync(0xffffffffu, ix, o);
        bd |= __shfl_down_sync(0xffffffffu, bd, o);
        if (ov > v || (ov == v && oi < ix)) { v = ov; ix = oi; }
      }
      if (lane == 0) {
        if (ix >= n) ix = col;
        s_piv = ix;
        if (rank == 0) {
          ipiv[col] = ix;
          if ((bd || !(v > 0.0)) && atomicCAS(&status[0], 0, 1) == 0) status[1] = col;
        }
      }
    }
    __syncthreads();
    const int piv = s_piv;
    const int own_p = (piv - j0) / rows_per_cta, own_c = (col - j0) / rows_per_cta;
    // 3. publish the pivot row and the diagonal row
    if (rank == own_p && tid < NB) prow[tid] = panel[(piv - r0) * NB + tid];
    if (rank == own_c && tid < NB) crow[tid] = panel[(col - r0) * NB + tid];
    cluster.sync();
    // 4. exchange and take the pivot row as the U row of this column
    if (tid < NB) {
      const double u = *cluster.map_shared_rank(&prow[tid], own_p);
      urow[tid] = u;
      if (rank == own_c) panel[(col - r0) * NB + tid] = u;
      if (rank == own_p && piv != col) panel[(piv - r0) * NB + tid] = *cluster.map_shared_rank(&crow[tid], own_c);
    }
    __syncthreads();
    // 5. rank-1 update of this CTA's rows below the diagonal
    const double d = urow[c];
    const double inv = (d != 0.0) ? 1.0 / d : 0.0;
    const int rbeg = max(0, col + 1 - r0);
    for (int r = rbeg + tid; r < nloc; r += PANEL_THREADS) panel[r * NB + c] *= inv;
    __syncthreads();
    const int w = jb - c - 1;
    for (int i = tid; i < (nloc - rbeg) * w; i += PANEL_THREADS) {
      const int r = rbeg + i / w, cc = c + 1 + i % w;
      panel[r * NB + cc] = fma(-panel[r * NB + c], urow[cc], panel[r * NB + cc]);
    }
    __syncthreads();
  }
  for (int i = tid; i < nloc * NB; i += PANEL_THREADS) {
    const int r = i / NB, c = i % NB;
    if (c < jb) A[(size_t)(r0 + r) * lda + j0 + c] = panel[i];
  }
  cluster.sync();   // no CTA leaves while others may still read its shared memory
}

static int launch_panel_cluster(lrs_ctx* ctx, double* A, int n, int j0, int jb, int* ipiv, int* status,
                                bool* used) {
  *used = false;
  const int m = n - j0;
  const int rows = (m + PANEL_CS - 1) / PANEL_CS;
  const size_t smem = (size_t)rows * NB * sizeof(double);
  if (smem > 200 * 1024) return LRS_OK;   // taller panels: single-CTA kernel
  // configured once, also when contexts on several host threads get here together
  static std::atomic<bool> usable{true};
  static std::once_flag configured;
  std::call_once(configured, [] {
    if (cudaFuncSetAttribute(lu_panel_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess ||
        cudaFuncSetAttribute(lu_panel_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess) {
      cudaGetLastError();
      usable = false;
    }
  });
  if (!usable) return LRS_OK;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(PANEL_CS);
  cfg.blockDim = dim3(PANEL_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = PANEL_CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, lu_panel_cluster_kernel, A, n, n, j0, jb, rows, ipiv, status);
  if (e != cudaSuccess) {
    cudaGetLastError();
    usable = false;   // e.g. cluster size not supported: fall back for good
    return LRS_OK;
  }
  *used = true;
  return after_launch(ctx, "lu_panel_cluster_kernel");
}

// In-place LU with partial pivoting of the n x n matrix A (row-major).
int lu_factor(lrs_ctx* ctx, double* A, int n, int* ipiv, int* status) {
  for (int j0 = 0; j0 < n; j0 += NB) {
    int jb = std::min(NB, n - j0);
    bool used = false;
    // panel rank-1 updates plus the triangular solve of the U row block
    ctx->fp64_flops += (double)(n - j0) * jb * jb + (double)jb * jb * (n - j0 - jb);
    LRS_TRY(launch_panel_cluster(ctx, A, n, j0, jb, ipiv, status, &used));
    if (!used) {
      lu_panel_kernel<<<1, 1024, 0, ctx->stream>>>(A, n, n, j0, jb, ipiv, status);
      LRS_TRY(after_launch(ctx, "lu_panel_kernel"));
    }
    if (n - jb > 0) {
      laswp_kernel<<<(n - jb + 255) / 256, 256, 0, ctx->stream>>>(A, n, n, ipiv, j0, jb, j0, jb);
      LRS_TRY(after_launch(ctx, "laswp_kernel"));
    }
    int rest = n - j0 - jb;
    if (rest > 0) {
      trsm_kernel<true><<<(rest + 127) / 128, 128, 0, ctx->stream>>>(A + (size_t)j0 * n + j0, n, jb,
                                                                      A + (size_t)j0 * n + j0 + jb, n, rest);
      LRS_TRY(after_launch(ctx, "trsm_kernel"));
      LRS_TRY(dgemm_t(ctx, false, false, rest, rest, jb, -1.0, A + (size_t)(j0 + jb) * n + j0, n, nullptr,
                      A + (size_t)j0 * n + j0 + jb, n, nullptr, 1.0, A + (size_t)(j0 + jb) * n + j0 + jb, n));
    }
  }
  return LRS_OK;
}

// Solves (LU) X = P B for the n x nrhs matrix B in place (row-major, ldb).
int lu_solve(lrs_ctx* ctx, const double* LU, int n, const int* ipiv, double* B, int nrhs, int ldb) {
  laswp_kernel<<<(nrhs + 255) / 256, 256, 0, ctx->stream>>>(B, ldb, nrhs, ipiv, 0, n, nrhs, 0);
  LRS_TRY(after_launch(ctx, "laswp_kernel"));
  for (int j0 = 0; j0 < n; j0 += NB) {
    int jb = std::min(NB, n - j0);
    trsm_kernel<true><<<(nrhs + 127) / 128, 128, 0, ctx->stream>>>(LU + (size_t)j0 * n + j0, n, jb,
                                                                    B + (size_t)j0 * ldb, ldb, nrhs);
    LRS_TRY(after_launch(ctx, "trsm_kernel"));
    int rest = n - j0 - jb;
    if (rest > 0)
      LRS_TRY(dgemm_t(ctx, false, false, rest, nrhs, jb, -1.0, LU + (size_t)(j0 + jb) * n + j0, n, nullptr,
                      B + (size_t)j0 * ldb, ldb, nullptr, 1.0, B + (size_t)(j0 + jb) * ldb, ldb));
  }
  int last = ((n - 1) / NB) * NB;
  for (int j0 = last; j0 >= 0; j0 -= NB) {
    int jb = std::min(NB, n - j0);
    trsm_kernel<false><<<(nrhs + 127) / 128, 128, 0, ctx->stream>>>(LU + (size_t)j0 * n + j0, n, jb,
                                                                     B + (size_t)j0 * ldb, ldb, nrhs);
    LRS_TRY(after_launch(ctx, "trsm_kernel"));
    if (j0 > 0)
      LRS_TRY(dgemm_t(ctx, false, false, j0, nrhs, jb, -1.0, LU + j0, n, nullptr, B + (size_t)j0 * ldb, ldb,
                      nullptr, 1.0, B, ldb));
  }
  return LRS_OK;
}

// Inverses of the jb x jb diagonal blocks of an LU factor (unit lower or
// upper), one CTA per block, thread c solving for column c.  out: [blocks][NB][NB].
template <bool kLowerUnit>
__global__ void invert_diag_blocks_kernel(const double* __restrict__ LU, int n, double* __restrict__ out) {
  __shared__ double T[NB][NB + 1];
  const int b = blockIdx.x, j0 = b * NB, jb = min(NB, n - j0);
  for (int i = threadIdx.x; i < jb * jb; i += blockDim.x) T[i / jb][i % jb] = LU[(size_t)(j0 + i / jb) * n + j0 + i % jb];
  __syncthreads();
  const int c = threadIdx.x;
  double x[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) x[i] = 0.0;
  if (c < jb) {
    if (kLowerUnit) {
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        if (i >= jb) break;
        double s = (i == c) ? 1.0 : 0.0;
#pragma unroll
        for (int k = 0; k < NB; ++k)
          if (k < i) s = fma(-T[i][k], x[k], s);
        x[i] = s;
      }
    } else {
#pragma unroll
      for (int ii = NB - 1; ii >= 0; --ii) {
        if (ii >= jb) continue;
        double s = (ii == c) ? 1.0 : 0.0;
#pragma unroll
        for (int k = 0; k < NB; ++k)
          if (k > ii && k < jb) s = fma(-T[ii][k], x[k], s);
        x[ii] = s / T[ii][ii];
      }
    }
  }
  double* o = out + (size_t)b * NB * NB;
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (c < NB) o[i * NB + c] = (c < jb && i < jb) ? x[i] : 0.0;
}

// B[0:jb, :] <- Tinv B[0:jb, :] in place, 16 columns per CTA (all of a CTA's
// columns are read before any is written, and no other CTA touches them).
constexpr int TA_COLS = 16;
__global__ void __launch_bounds__(256) trsm_apply_kernel(const double* __restrict__ Tinv, int jb,
                                                         double* __restrict__ B, int ldb, int ncols) {
  __shared__ double Ts[NB][NB + 1];
  __shared__ double Bs[NB][TA_COLS + 1];
  const int c0 = blockIdx.x * TA_COLS;
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) Ts[i / NB][i % NB] = Tinv[i];
  for (int i = threadIdx.x; i < NB * TA_COLS; i += blockDim.x) {
    const int r = i / TA_COLS, c = i % TA_COLS;
    Bs[r][c] = (r < jb && c0 + c < ncols) ? B[(size_t)r * ldb + c0 + c] : 0.0;
  }
  __syncthreads();
  // 256 threads: row r = tid / 8, columns (tid % 8) and (tid % 8) + 8
  const int r = threadIdx.x >> 3, ca = threadIdx.x & 7;
  double s0 = 0.0, s1 = 0.0;
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const double t = Ts[r][k];
    s0 = fma(t, Bs[k][ca], s0);
    s1 = fma(t, Bs[k][ca + 8], s1);
  }
  if (r < jb) {
    if (c0 + ca < ncols) B[(size_t)r * ldb + c0 + ca] = s0;
    if (c0 + ca + 8 < ncols) B[(size_t)r * ldb + c0 + ca + 8] = s1;
  }
}

// lu_solve with the diagonal blocks inverted once (tinv: 2 * ceil(n/NB) * NB * NB doubles).
int lu_solve_inv(lrs_ctx* ctx, const double* LU, int n, const int* ipiv, double* B, int nrhs, int ldb,
                 double* tinv) {
  const int nblk = (n + NB - 1) / NB;
  double* linv = tinv;
  double* uinv = tinv + (size_t)nblk * NB * NB;
  invert_diag_blocks_kernel<true><<<nblk, NB, 0, ctx->stream>>>(LU, n, linv);
  LRS_TRY(after_launch(ctx, "invert_diag_blocks_kernel"));
  invert_diag_blocks_kernel<false><<<nblk, NB, 0, ctx->stream>>>(LU, n, uinv);
  LRS_TRY(after_launch(ctx, "invert_diag_blocks_kernel"));
  laswp_kernel<<<(nrhs + 255) / 256, 256, 0, ctx->stream>>>(B, ldb, nrhs, ipiv, 0, n, nrhs, 0);
  LRS_TRY(after_launch(ctx, "laswp_kernel"));
  const int tgrid = (nrhs + TA_COLS - 1) / TA_COLS;
  ctx->fp64_flops += 2.0 * 2.0 * NB * (double)n * nrhs;   // diagonal-block products, both sweeps
  for (int b = 0; b < nblk; ++b) {
    const int j0 = b * NB, jb = std::min(NB, n - j0);
    trsm_apply_kernel<<<tgrid, 256, 0, ctx->stream>>>(linv + (size_t)b * NB * NB, jb, B + (size_t)j0 * ldb, ldb,
                                                       nrhs);
    LRS_TRY(after_launch(ctx, "trsm_apply_kernel"));
    const int rest = n - j0 - jb;
    if (rest > 0)
      LRS_TRY(dgemm_t(ctx, false, false, rest, nrhs, jb, -1.0, LU + (size_t)(j0 + jb) * n + j0, n, nullptr,
                      B + (size_t)j0 * ldb, ldb, nullptr, 1.0, B + (size_t)(j0 + jb) * ldb, ldb));
  }
  for (int b = nblk - 1; b >= 0; --b) {
    const int j0 = b * NB, jb = std::min(NB, n - j0);
    trsm_apply_kernel<<<tgrid, 256, 0, ctx->stream>>>(uinv + (size_t)b * NB * NB, jb, B + (size_t)j0 * ldb, ldb,
                                                       nrhs);
    LRS_TRY(after_launch(ctx, "trsm_apply_kernel"));
    if (j0 > 0)
      LRS_TRY(dgemm_t(ctx, false, false, j0, nrhs, jb, -1.0, LU + j0, n, nullptr, B + (size_t)j0 * ldb, ldb,
                      nullptr, 1.0, B, ldb));
  }
  return LRS_OK;
}

int dyson_solve(lrs_ctx* ctx, Site& s) {
  const int n = s.npts;
  const size_t nn = (size_t)n * n;
  LRS_TRY(ensure(ctx, s.v, nn));
  LRS_TRY(ensure(ctx, s.w, nn));
  LRS_TRY(ensure(ctx, ctx->ws.dyson_a, nn));
  LRS_TRY(ensure(ctx, ctx->ws.ipiv, n));
  const int L2 = (s.lmax + 1) * (s.lmax + 1);
  if (ctx->dyson_basis == LRS_DYSON_LM && !s.product)
    return set_error(LRS_ERR_ARG, "lm-basis Dyson solve needs a radial x angular product grid");
  if (s.product && (ctx->dyson_basis == LRS_DYSON_LM ||
                    (ctx->dyson_basis == LRS_DYSON_AUTO && (long long)s.nrad * L2 < n)))
    return dyson_solve_lm(ctx, s);   // the full-grid v is built only on request
  LRS_TRY(coulomb_build(ctx, s, s.v.ptr));
  s.has_v = true;
  double* A = ctx->ws.dyson_a.ptr;
  // A = I - (v Q)(chi0 Q)
  LRS_TRY(dgemm_t(ctx, false, false, n, n, n, -1.0, s.v.ptr, n, s.wts.ptr, s.response_chi(), n, s.wts.ptr, 0.0, A, n));
  add_identity_kernel<<<(n + 255) / 256, 256, 0, ctx->stream>>>(A, n, n, 1.0);
  LRS_TRY(after_launch(ctx, "add_identity_kernel"));
  LRS_TRY(lu_factor(ctx, A, n, ctx->ws.ipiv.ptr, ctx->ws.status.ptr));
  LRS_CUDA_TRY(cudaMemcpyAsync(s.w.ptr, s.v.ptr, nn * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  LRS_TRY(ensure(ctx, ctx->ws.tinv, 2 * (size_t)((n + NB - 1) / NB) * NB * NB));
  return lu_solve_inv(ctx, A, n, ctx->ws.ipiv.ptr, s.w.ptr, n, n, ctx->ws.tinv.ptr);
}

// ---------------------------------------------------------------- SPD inverse
// In-place inverse of a symmetric positive definite matrix by blocked
// Gauss-Jordan exchange steps.  Exchanging block k (pivot P = A_kk) maps
//   A_kk -> P^-1,  A_ik -> A_ik P^-1,  A_kj -> -P^-1 A_kj,  A_ij -> A_ij - A_ik P^-1 A_kj,
// and after every block has been exchanged the matrix is A^-1.  Every pivot
// block of an SPD matrix is SPD (a Schur complement), so no pivoting is needed.
// Only the lower triangle is stored: blocks (i, j) and (j, i) stay transposes
// of each other up to the sign s = -1 when exactly one of the two block
// indices has been exchanged.  Cost n^3 flop (lower-triangle rank-nb updates),
// against 8/3 n^3 for LU plus n right-hand sides.
constexpr int GJ_NB = 32;               // pivot block width
constexpr int GJ_PR = 256 / GJ_NB;       // row groups of the 256-thread pivot and apply kernels

// Column block k of the current matrix from the lower triangle, C (n x kb,
// leading dimension GJ_NB): element (i, j), j in block k, is stored at
// (max(i, j), min(i, j)); rows i < k0 take it with the sign -1 (one of the two
// blocks exchanged).  E = sigma C with sigma = -1 on rows i < k0, so that
// A_kj = E_j^T for every j != k.
//
// The exchange of the previous block kp (= k - 1, D_p = C_p P^-1, E_p) has not
// been applied to block k (the bulk update leaves blocks kp and k out): the
// gather applies it on the fly, stored(r, s) - D_p[r] . E_p[s], except on the
// rows of block kp, where the exchange itself writes D_p (read here from D_p,
// so the gather does not wait for gj_fix_kernel).  Block k of A is rewritten
// by its own exchange, so the updated values are not stored.
// GJ_GR rows per CTA, one warp per row (lane = column in the block); the CTAs
// cover rows row_base + GJ_GR blockIdx.x, and groups starting in [skip_lo,
// skip_hi) are left out (ranges are multiples of GJ_GR, or end at n).
constexpr int GJ_GR = 8;
__global__ void __launch_bounds__(256) gj_gather_kernel(const double* __restrict__ A, int n, int lda, int k0, int kb,
                                                        const double* __restrict__ Dp, const double* __restrict__ Ep,
                                                        int kp0, int kpb, double* __restrict__ C,
                                                        double* __restrict__ E, uint16_t* __restrict__ eplanes,
                                                        size_t plane_stride, int* __restrict__ eexp, int row_base,
                                                        int skip_lo, int skip_hi) {
  __shared__ double dr[GJ_GR][GJ_NB + 1], er[GJ_GR][GJ_NB + 1];   // D_p, E_p rows of this CTA's rows
  __shared__ double dk[GJ_NB][GJ_NB + 1], ek[GJ_NB][GJ_NB + 1];   // D_p, E_p rows of block k
  const int i0 = row_base + blockIdx.x * GJ_GR;
  if (i0 >= skip_lo && i0 < skip_hi) return;   // the whole CTA, before any barrier
  const int r = threadIdx.x >> 5, c = threadIdx.x & 31;
  if (Dp) {
    for (int idx = threadIdx.x; idx < GJ_GR * GJ_NB; idx += blockDim.x) {
      const int rr = idx / GJ_NB, cc = idx % GJ_NB, i = i0 + rr;
      dr[rr][cc] = (i < n && cc < kpb) ? Dp[(size_t)i * GJ_NB + cc] : 0.0;
      er[rr][cc] = (i < n && cc < kpb) ? Ep[(size_t)i * GJ_NB + cc] : 0.0;
    }
    for (int idx = threadIdx.x; idx < GJ_NB * GJ_NB; idx += blockDim.x) {
      const int rr = idx / GJ_NB, cc = idx % GJ_NB, j = k0 + rr;
      dk[rr][cc] = (rr < kb && cc < kpb) ? Dp[(size_t)j * GJ_NB + cc] : 0.0;
      ek[rr][cc] = (rr < kb && cc < kpb) ? Ep[(size_t)j * GJ_NB + cc] : 0.0;
    }
    __syncthreads();
  }
  const int i = i0 + r;
  if (i >= n) return;                          // whole warp: one row per warp
  const int j = k0 + c;
  double v = 0.0;
  if (c < kb) {
    if (Dp && i >= kp0 && i < kp0 + kpb) {
      // stored (j, i) in the column block of kp below its diagonal: the exchange of kp
      // writes D_p there (gj_fix_kernel, which may still be running)
      v = dk[c][i - kp0];
    } else {
      v = (i >= j) ? A[(size_t)i * lda + j] : A[(size_t)j * lda + i];
    }
    if (Dp && !(i >= kp0 && i < kp0 + kpb)) {
      // stored (max, min): D_p of the larger index, E_p of the smaller
      const double* d = (i >= j) ? dr[r] : dk[c];
      const double* e = (i >= j) ? ek[c] : er[r];
      // four partial sums: a 32-long chain of dependent float64 FMAs would pay their
      // latency 32 times
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int kk = 0; kk < GJ_NB; ++kk) acc[kk & 3] = fma(d[kk], e[kk], acc[kk & 3]);
      v -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    const bool flip = i < k0;
    C[(size_t)i * GJ_NB + c] = flip ? -v : v;
    E[(size_t)i * GJ_NB + c] = v;
  }
  // slices of the row of E for the tensor-core update
  if (eplanes) oz_slice_row(c < kb ? v : 0.0, c, i, plane_stride, eplanes, eexp);
}

constexpr int GJ_PM = GJ_NB / GJ_PR;     // pivot rows per thread
// Pinv = P^-1 for the kb x kb pivot block P = C[k0, k0 + kb) by scalar
// exchange steps; a ragged block is padded with the identity.  (Variants with
// one barrier per step, the reciprocal on a separate warp, the lower triangle
// only, or a division-free scaled form all measured slower on GB300: the
// float64 latency of each step's dependent operations, not the FMA count,
// sets the pace, and here the division runs while the FP64 units are idle.)  Thread t holds
// column t % GJ_NB of rows t / GJ_NB + GJ_PR m in registers; per step the
// owners of column p publish it divided by the pivot and the owners of row p
// publish that row, then every element takes one FMA.  One SM retires two
// DFMA per clock, so an nb x nb inverse is about nb^3 / 2 clocks.  A pivot
// that is not positive and finite sets status[0] = 2, status[1] = its column
// (the matrix is not SPD).
__global__ void __launch_bounds__(256) gj_pivot_kernel(const double* __restrict__ C, int k0, int kb,
                                                       double* __restrict__ Pinv, int* __restrict__ status) {
  __shared__ double colv[GJ_NB];   // column p, then column p / pivot
  __shared__ double roww[GJ_NB];   // row p
  __shared__ double dinv;
  const int j = threadIdx.x % GJ_NB, ib = threadIdx.x / GJ_NB;
  double a[GJ_PM];
#pragma unroll
  for (int m = 0; m < GJ_PM; ++m) {
    const int i = ib + GJ_PR * m;
    a[m] = (i < kb && j < kb) ? C[(size_t)(k0 + i) * GJ_NB + j] : (i == j ? 1.0 : 0.0);
  }
  for (int p = 0; p < GJ_NB; ++p) {
    if (j == p) {
#pragma unroll
      for (int m = 0; m < GJ_PM; ++m) colv[ib + GJ_PR * m] = a[m];
    }
#pragma unroll
    for (int m = 0; m < GJ_PM; ++m)
      if (ib + GJ_PR * m == p) roww[j] = a[m];
    __syncthreads();
    const double piv = colv[p];
    if (!(piv > 0.0) || !isfinite(piv)) {   // same value in every thread: uniform exit
      if (threadIdx.x == 0 && atomicCAS(&status[0], 0, 2) == 0) status[1] = k0 + p;
      break;
    }
    __syncthreads();
    if (threadIdx.x < GJ_NB) {
      const double d = 1.0 / piv;
      colv[threadIdx.x] *= d;
      if (threadIdx.x == 0) dinv = d;
    }
    __syncthreads();
    const double rj = roww[j], d = dinv;
#pragma unroll
    for (int m = 0; m < GJ_PM; ++m) {
      const int i = ib + GJ_PR * m;
      const double ci = colv[i];
      if (i == p) a[m] = (j == p) ? d : -rj * d;
      else if (j == p) a[m] = ci;
      else a[m] = fma(-ci, rj, a[m]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < GJ_PM; ++m) {
    const int i = ib + GJ_PR * m;
    if (i < kb && j < kb) Pinv[(size_t)i * GJ_NB + j] = a[m];
  }
}

// D = C Pinv (n x kb), 8 rows per CTA so that every SM takes part; rows as in
// gj_gather_kernel (row_base, groups starting in [skip_lo, skip_hi) left out).
constexpr int GJ_DR = 8;
__global__ void __launch_bounds__(256) gj_apply_kernel(const double* __restrict__ C, int n, int kb,
                                                       const double* __restrict__ Pinv, double* __restrict__ D,
                                                       uint16_t* __restrict__ dplanes, size_t plane_stride,
                                                       int* __restrict__ dexp, int row_base, int skip_lo,
                                                       int skip_hi) {
  __shared__ double pv[GJ_NB][GJ_NB + 1];
  __shared__ double cr[GJ_DR][GJ_NB + 1];
  const int r0 = row_base + blockIdx.x * GJ_DR;
  if (r0 >= skip_lo && r0 < skip_hi) return;   // the whole CTA, before any barrier
  // zero beyond kb, so that the product can run over all GJ_NB terms
  for (int idx = threadIdx.x; idx < GJ_NB * GJ_NB; idx += blockDim.x) {
    const int i = idx / GJ_NB, j = idx % GJ_NB;
    pv[i][j] = (i < kb && j < kb) ? Pinv[(size_t)i * GJ_NB + j] : 0.0;
  }
  for (int idx = threadIdx.x; idx < GJ_DR * GJ_NB; idx += blockDim.x) {
    const int i = idx / GJ_NB, j = idx % GJ_NB;
    cr[i][j] = (r0 + i < n && j < kb) ? C[(size_t)(r0 + i) * GJ_NB + j] : 0.0;
  }
  __syncthreads();
  const int j = threadIdx.x % GJ_NB, ib = threadIdx.x / GJ_NB;   // rows ib + GJ_PR m (a warp per row group)
  // four partial sums per element: a kb-long chain of dependent float64 FMAs would pay
  // their latency kb times (entries beyond kb are zero)
  double acc[GJ_DR / GJ_PR][4];
#pragma unroll
  for (int m = 0; m < GJ_DR / GJ_PR; ++m) acc[m][0] = acc[m][1] = acc[m][2] = acc[m][3] = 0.0;
  if (j < kb) {
#pragma unroll
    for (int k = 0; k < GJ_NB; ++k) {
      const double b = pv[k][j];
#pragma unroll
      for (int m = 0; m < GJ_DR / GJ_PR; ++m) acc[m][k & 3] = fma(cr[ib + GJ_PR * m][k], b, acc[m][k & 3]);
    }
  }
#pragma unroll
  for (int m = 0; m < GJ_DR / GJ_PR; ++m) {
    const int r = r0 + ib + GJ_PR * m;
    const double dv = (acc[m][0] + acc[m][1]) + (acc[m][2] + acc[m][3]);
    if (r < n && j < kb) D[(size_t)r * GJ_NB + j] = dv;
    // slices of the row of D for the tensor-core update (the warp holds the whole row)
    if (dplanes && r < n) oz_slice_row(dv, j, r, plane_stride, dplanes, dexp);
  }
}

// After the trailing update: pivot block <- Pinv, column block k below it <- D
// (= C Pinv), row block k left of it <- D^T (the exchanged A_kj = -P^-1 A_kj).
__global__ void __launch_bounds__(256) gj_fix_kernel(double* __restrict__ A, int n, int lda, int k0, int kb,
                                                     const double* __restrict__ D, const double* __restrict__ Pinv) {
  __shared__ double t[GJ_NB][GJ_NB + 1];
  const int i0 = blockIdx.x * GJ_NB;
  if (i0 < k0) {
    for (int idx = threadIdx.x; idx < GJ_NB * kb; idx += blockDim.x) {
      const int ii = idx / kb, c = idx % kb;
      t[c][ii] = D[(size_t)(i0 + ii) * GJ_NB + c];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kb * GJ_NB; idx += blockDim.x) {
      const int c = idx / GJ_NB, ii = idx % GJ_NB;
      A[(size_t)(k0 + c) * lda + i0 + ii] = t[c][ii];
    }
  } else if (i0 == k0) {
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
      const int i = idx / kb, j = idx % kb;
      A[(size_t)(k0 + i) * lda + k0 + j] = Pinv[(size_t)i * GJ_NB + j];
    }
  } else {
    for (int idx = threadIdx.x; idx < GJ_NB * kb; idx += blockDim.x) {
      const int ii = idx / kb, c = idx % kb, i = i0 + ii;
      if (i < n) A[(size_t)i * lda + k0 + c] = D[(size_t)i * GJ_NB + c];
    }
  }
}

// Trailing update A_ij -= D_i E_j^T of the exchange of block k on 32 x 32
// tiles of the lower triangle (a pivot block spans GJ_TB x GJ_TB tiles), on the
// float64 pipe.  The FP64 pipe of one SM is saturated by a few warps, so small
// tiles cost no throughput and balance the SMs: a step has thousands of equal
// tiles.  1-D grid over the lower-triangle tiles; tiles in pivot blocks k and
// k + 1 (rows or columns) are left out (the exchange of block k rewrites its
// own, and the gather of block k + 1 applies this update to that block).
constexpr int UT = 32;
constexpr int GJ_TB = GJ_NB / UT;   // update tiles per pivot block and dimension
__global__ void __launch_bounds__(128) gj_update_kernel(double* __restrict__ A, int n, int lda, int kb, int k,
                                                        const double* __restrict__ D,
                                                        const double* __restrict__ E) {
  __shared__ double Ds[GJ_NB][UT + 1];
  __shared__ double Es[GJ_NB][UT + 1];
  int ti, tj;
  {
    const long long t = blockIdx.x;
    ti = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)(ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while ((long long)ti * (ti + 1) / 2 > t) --ti;
    tj = (int)(t - (long long)ti * (ti + 1) / 2);
    const int bi = ti / GJ_TB, bj = tj / GJ_TB;
    if (bi == k || bi == k + 1 || bj == k || bj == k + 1) return;
  }
  const int i0 = ti * UT, j0 = tj * UT;
  for (int idx = threadIdx.x; idx < UT * kb; idx += blockDim.x) {
    const int r = idx / kb, c = idx % kb;
    Ds[c][r] = (i0 + r < n) ? D[(size_t)(i0 + r) * GJ_NB + c] : 0.0;
    Es[c][r] = (j0 + r < n) ? E[(size_t)(j0 + r) * GJ_NB + c] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;   // rows ty, ty + 16; columns tx + 8 c
  double acc[2][4] = {{0.0, 0.0, 0.0, 0.0}, {0.0, 0.0, 0.0, 0.0}};
  for (int kk = 0; kk < kb; ++kk) {
    const double a0 = Ds[kk][ty], a1 = Ds[kk][ty + 16];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double b = Es[kk][tx + 8 * c];
      acc[0][c] = fma(a0, b, acc[0][c]);
      acc[1][c] = fma(a1, b, acc[1][c]);
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = i0 + ty + 16 * h;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx + 8 * c;
      if (j < n) A[(size_t)i * lda + j] -= acc[h][c];
    }
  }
}

// Schedule.  Streams: s1 (the context stream) runs the bulk of each trailing
// update (every tile away from blocks p and p + 1); three side streams of
// higher priority prepare the panels in two alternating buffer sets.  Panel p
// on rows R_p = [32 p, 32 p + kb):
//   s2: gather of rows R_p -> 32 x 32 pivot inverse -> D_p on rows R_{p+1}
//       (all that the next gather of the diagonal block needs): the chain of
//       dependent steps, kept as short as possible;
//   s4: gather of the other rows -> D_p on the other rows;
//   s3: write-back of the exchanged block p (fix).
// Events (pairs alternate with the block parity):
//   gather R_p        <- D_{p-1} on R_p (s2 order), gather rest p-1, bulk p-2, fix p-2 (buffer set);
//   gather rest p     <- D_{p-1} rest (s4 order), D_{p-1} on R_p, bulk p-2;
//   D_p on R_{p+1}    <- pivot p (s2 order), gather rest p;
//   D_p rest          <- gather rest p (s4 order), pivot p;
//   fix p, bulk p     <- both parts of D_p; bulk p also <- fix p-1.
// The serial pivot inverse (one SM) thereby overlaps the bulk update and the
// row-parallel parts of the panels.
int spd_inverse(lrs_ctx* ctx, double* A, int n, int lda, int* status) {
  static_assert(GJ_NB % UT == 0 && GJ_TB >= 1, "a pivot block spans whole update tiles");
  static_assert(GJ_NB % GJ_GR == 0 && GJ_GR == GJ_DR, "row groups of the gather and apply kernels tile a block");
  if (n <= 0) return LRS_OK;
  const size_t set = 3 * (size_t)n * GJ_NB + GJ_NB * GJ_NB;
  LRS_TRY(ensure(ctx, ctx->ws.gj, 2 * set));
  LRS_TRY(aux_stream_ready(ctx));
  SpdStreams& sp = ctx->spd;
  cudaStream_t s1 = ctx->stream, s2 = sp.s2, s3 = sp.s3, s4 = sp.s4;
  double *Cb[2], *Eb[2], *Db[2], *Pb[2];
  for (int q = 0; q < 2; ++q) {
    Cb[q] = ctx->ws.gj.ptr + q * set;
    Eb[q] = Cb[q] + (size_t)n * GJ_NB;
    Db[q] = Eb[q] + (size_t)n * GJ_NB;
    Pb[q] = Db[q] + (size_t)n * GJ_NB;
  }
  const int nblk = (n + GJ_NB - 1) / GJ_NB;
  const long long nt = (n + UT - 1) / UT;   // 32-wide update tiles per dimension
  // bulk updates on the tensor cores (float64-accurate slices) or the FP64 pipe
  const bool tc = ctx->dyson_update == LRS_UPDATE_TC ||
                  (ctx->dyson_update == LRS_UPDATE_AUTO && ctx->precision != LRS_FP64);
  const int rows_pad = oz_rows_pad(n);
  const size_t pe = oz_plane_elems(n);
  const size_t stride = (size_t)rows_pad * 64;
  uint16_t* dpl[2] = {nullptr, nullptr};
  uint16_t* epl[2] = {nullptr, nullptr};
  int* dsc[2] = {nullptr, nullptr};
  int* esc[2] = {nullptr, nullptr};
  CUtensorMap md[2], me[2];
  if (tc) {
    LRS_TRY(ensure(ctx, ctx->ws.oz_planes, 4 * pe));
    LRS_TRY(ensure(ctx, ctx->ws.oz_expo, 4 * (size_t)rows_pad));
    for (int q = 0; q < 2; ++q) {
      dpl[q] = ctx->ws.oz_planes.ptr + (2 * q) * pe;
      epl[q] = ctx->ws.oz_planes.ptr + (2 * q + 1) * pe;
      dsc[q] = ctx->ws.oz_expo.ptr + (2 * q) * (size_t)rows_pad;
      esc[q] = ctx->ws.oz_expo.ptr + (2 * q + 1) * (size_t)rows_pad;
      LRS_TRY(oz_make_maps(ctx, dpl[q], epl[q], rows_pad, &md[q], &me[q]));
    }
    // rows beyond n stay zero; rows below n are rewritten by every panel
    LRS_CUDA_TRY(cudaMemsetAsync(ctx->ws.oz_planes.ptr, 0, 4 * pe * sizeof(uint16_t), s1));
  }
  auto ev = [&](int base, int p) { return sp.ev[base + (p & 1)]; };
  auto wait = [&](cudaStream_t st, int base, int p) { return cudaStreamWaitEvent(st, ev(base, p), 0); };
  auto record = [&](cudaStream_t st, int base, int p) { return cudaEventRecord(ev(base, p), st); };
  const int pr = ctx->prio_greatest;   // side-chain launches: highest priority, also as graph nodes
  auto rows_of = [&](int p, int& lo, int& hi) {   // rows of block p ([0, 0) beyond the last block)
    lo = p < nblk ? p * GJ_NB : 0;
    hi = p < nblk ? std::min(n, lo + GJ_NB) : 0;
  };
  auto gather = [&](int p, cudaStream_t st, int row_base, int nrows, int skip_lo, int skip_hi) -> int {
    const int q = p & 1, qp = q ^ 1, k0 = p * GJ_NB, kb = std::min(GJ_NB, n - k0);
    const bool prev = p > 0;   // the exchange of block p - 1 is applied to block p on the fly
    const double* dprev = prev ? Db[qp] : nullptr;
    const double* eprev = prev ? Eb[qp] : nullptr;
    LRS_CUDA_TRY(launch_with_priority(gj_gather_kernel, dim3((nrows + GJ_GR - 1) / GJ_GR), dim3(256), 0, st, pr,
                                      (const double*)A, n, lda, k0, kb, dprev, eprev, k0 - GJ_NB, (int)GJ_NB, Cb[q],
                                      Eb[q], epl[q], stride, esc[q], row_base, skip_lo, skip_hi));
    return after_launch(ctx, "gj_gather_kernel");
  };
  auto apply = [&](int p, cudaStream_t st, int row_base, int nrows, int skip_lo, int skip_hi) -> int {
    const int q = p & 1, k0 = p * GJ_NB, kb = std::min(GJ_NB, n - k0);
    if (nrows <= 0) return LRS_OK;
    LRS_CUDA_TRY(launch_with_priority(gj_apply_kernel, dim3((nrows + GJ_DR - 1) / GJ_DR), dim3(256), 0, st, pr,
                                      (const double*)Cb[q], n, kb, (const double*)Pb[q], Db[q], dpl[q], stride,
                                      dsc[q], row_base, skip_lo, skip_hi));
    return after_launch(ctx, "gj_apply_kernel");
  };
  auto panel = [&](int p) -> int {
    const int q = p & 1, k0 = p * GJ_NB, kb = std::min(GJ_NB, n - k0);
    int lo, hi, nlo, nhi;
    rows_of(p, lo, hi);
    rows_of(p + 1, nlo, nhi);
    // s2: the diagonal block and its inverse
    if (p >= 2) {
      LRS_CUDA_TRY(wait(s2, SPD_BULK, p - 2));
      LRS_CUDA_TRY(wait(s2, SPD_FIX, p - 2));
    }
    LRS_TRY(gather(p, s2, lo, hi - lo, 0, 0));
    LRS_CUDA_TRY(launch_with_priority(gj_pivot_kernel, dim3(1), dim3(256), 0, s2, pr, (const double*)Cb[q], k0, kb,
                                      Pb[q], status));
    LRS_TRY(after_launch(ctx, "gj_pivot_kernel"));
    LRS_CUDA_TRY(record(s2, SPD_PIVOT, p));
    // s4: the other rows of the panel, then their D.  The rows of block p - 2 read stored
    // (j, i), j in block p, from the column block that the exchange write-back of p - 2
    // (gj_fix_kernel on s3) rewrites: wait for it too
    if (p >= 1) LRS_CUDA_TRY(wait(s4, SPD_ADIAG, p - 1));
    if (p >= 2) {
      LRS_CUDA_TRY(wait(s4, SPD_BULK, p - 2));
      LRS_CUDA_TRY(wait(s4, SPD_FIX, p - 2));
    }
    LRS_TRY(gather(p, s4, 0, n, lo, hi));
    LRS_CUDA_TRY(record(s4, SPD_GREST, p));
    LRS_CUDA_TRY(wait(s4, SPD_PIVOT, p));
    LRS_TRY(apply(p, s4, 0, n, nlo, nhi));
    LRS_CUDA_TRY(record(s4, SPD_AREST, p));
    // s2: D on the rows of the next block
    LRS_CUDA_TRY(wait(s2, SPD_GREST, p));
    LRS_TRY(apply(p, s2, nlo, nhi - nlo, 0, 0));
    LRS_CUDA_TRY(record(s2, SPD_ADIAG, p));
    if (p > 0) ctx->fp64_flops += 2.0 * n * kb * GJ_NB;
    ctx->fp64_flops += 2.0 * n * kb * kb;
    return LRS_OK;
  };
  // fork the side streams from the context stream (also inside a graph capture)
  LRS_CUDA_TRY(cudaEventRecord(sp.ev[SPD_FORK], s1));
  for (cudaStream_t st : {s2, s3, s4}) LRS_CUDA_TRY(cudaStreamWaitEvent(st, sp.ev[SPD_FORK], 0));
  LRS_TRY(panel(0));
  for (int k = 0; k < nblk; ++k) {
    const int q = k & 1, k0 = k * GJ_NB, kb = std::min(GJ_NB, n - k0);
    // bulk of the trailing update on the context stream
    LRS_CUDA_TRY(wait(s1, SPD_ADIAG, k));
    LRS_CUDA_TRY(wait(s1, SPD_AREST, k));
    if (k >= 1) LRS_CUDA_TRY(wait(s1, SPD_FIX, k - 1));   // bulk k updates block k - 1, just written back
    // the trailing updates of an inverse nested in the blocked one are not its main updates
    const bool main = !ctx->spd_inner;
    if (main) LRS_TRY(stage_begin(ctx, ST_W_MAIN));
    if (tc) {
      LRS_TRY(oz_update(ctx, md[q], me[q], A, n, lda, dsc[q], esc[q], k0, std::min(n, k0 + 2 * GJ_NB), rows_pad,
                        s1));
    } else {
      gj_update_kernel<<<(unsigned)(nt * (nt + 1) / 2), 128, 0, s1>>>(A, n, lda, kb, k, Db[q], Eb[q]);
      LRS_TRY(after_launch(ctx, "gj_update_kernel"));
    }
    if (main) LRS_TRY(stage_end(ctx, ST_W_MAIN));
    if (main) {
      // lower-triangle elements outside the rows and columns of blocks k and k + 1
      const double b0 = k0, b1 = std::min(n, k0 + 2 * GJ_NB), nn = n;
      const double rows_in = (b1 * (b1 + 1) - b0 * (b0 + 1)) / 2.0;   // sum of (i + 1), i in [b0, b1)
      const double elems = nn * (nn + 1) / 2.0 - rows_in - (b1 - b0) * (nn - b1);
      ctx->w_main_flop += 2.0 * kb * elems;
      ctx->w_main_elems += elems;
      ++ctx->w_main_launches;
    }
    if (!tc) ctx->fp64_flops += (double)n * n * kb;
    LRS_CUDA_TRY(record(s1, SPD_BULK, k));
    // write-back of the exchanged block k on the third stream
    LRS_CUDA_TRY(wait(s3, SPD_ADIAG, k));
    LRS_CUDA_TRY(wait(s3, SPD_AREST, k));
    LRS_CUDA_TRY(launch_with_priority(gj_fix_kernel, dim3(nblk), dim3(256), 0, s3, pr, A, n, lda, k0, kb,
                                      (const double*)Db[q], (const double*)Pb[q]));
    LRS_TRY(after_launch(ctx, "gj_fix_kernel"));
    LRS_CUDA_TRY(record(s3, SPD_FIX, k));
    if (k + 1 < nblk) LRS_TRY(panel(k + 1));
  }
  // join the side streams
  LRS_CUDA_TRY(cudaEventRecord(sp.ev[SPD_JOIN2], s2));
  LRS_CUDA_TRY(cudaEventRecord(sp.ev[SPD_JOIN3], s3));
  LRS_CUDA_TRY(cudaEventRecord(sp.ev[SPD_JOIN4], s4));
  for (int e : {SPD_JOIN2, SPD_JOIN3, SPD_JOIN4}) LRS_CUDA_TRY(cudaStreamWaitEvent(s1, sp.ev[e], 0));
  return LRS_OK;
}

}  // namespace lrs
