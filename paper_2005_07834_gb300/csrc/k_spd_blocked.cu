// Symmetric positive definite inverse of the lm-basis Dyson matrix with
// 128-wide pivot blocks (Sec. VI.E; the solve of (I - C X) Z = C in its
// symmetric form Z = F (I - F^T X F)^-1 F^T).
//
// The in-place Gauss-Jordan exchange of spd_inverse (k_linalg.cu) applied to
// a pivot block K of 128 indices at once: with the column block read from the
// stored lower triangle, C = sigma A[:, K] (sigma = -1 on the rows before K),
// E = A[:, K], P = (C_KK)^-1,
//   D = C P,   A_ij -= D_i . E_j  (i >= j, i and j outside K),
//   A_KK <- P, A[i, K] <- D_i (i after K), A[K, j] <- D_j^T (j before K).
// Exchanging K at once equals exchanging its four 32-wide sub-blocks one
// after the other (the sweep of a block is the product of the sweeps of its
// parts); here the 128 x 128 inverse is itself the 32-wide spd_inverse, and
// D = C P and the rank-128 trailing update run float64-accurate on the tensor
// cores (oz_gemm_batched: eight exact bf16 slices per row, one 128-long
// accumulation segment).  The trailing update then passes over the matrix
// once per 128 pivots instead of once per 32, with four times the tensor-core
// work per pass, so its epilogue (level combination, rounding, the float64
// subtraction) runs a quarter as often.
#include <algorithm>

#include "lrs_internal.h"

namespace lrs {

constexpr int BB = SPD_OUTER_BLOCK;

// C = sigma A[:, K], E = A[:, K] (columns c >= kb zero) for every row, and the pivot block
// into Pd (kb x kb, row stride BB).  32 x 32 tiles: below the diagonal the stored rows are read
// directly, above it the stored rows of the block are read and transposed in shared memory.
__global__ void __launch_bounds__(256) spdb_gather_kernel(const double* __restrict__ A, int n, int lda, int k0,
                                                          int kb, double* __restrict__ C, double* __restrict__ E,
                                                          double* __restrict__ Pd) {
  __shared__ double t[32][33];
  const int i0 = blockIdx.x * 32, c0 = blockIdx.y * 32;   // rows i0.., block columns c0..
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j0 = k0 + c0;
  // t[r][c] = A_sym(i0 + r, j0 + c)
  for (int r = ty; r < 32; r += 8) {
    // stored element of (i0 + r, j0 + tx) when i >= j, read row-wise
    const int i = i0 + r, j = j0 + tx;
    if (i < n && c0 + tx < kb && i >= j) t[r][tx] = A[(size_t)i * lda + j];
  }
  for (int r = ty; r < 32; r += 8) {
    // stored element (j0 + r, i0 + tx) for i < j: row j of the block, read row-wise, transposed
    const int j = j0 + r, i = i0 + tx;
    if (i < n && c0 + r < kb && i < j) t[tx][r] = A[(size_t)j * lda + i];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, c = c0 + tx;
    if (i >= n) continue;
    const double v = c < kb ? t[r][tx] : 0.0;
    C[(size_t)i * BB + c] = i < k0 ? -v : v;
    E[(size_t)i * BB + c] = v;
    if (i >= k0 && i < k0 + kb && c < kb) Pd[(size_t)(i - k0) * BB + c] = v;
  }
}

// After the trailing update: A_KK <- P (lower), A[i, K] <- D_i for i after K, A[K, j] <- D_j^T
// for j before K (32 x 32 tiles, the transposed ones through shared memory).
__global__ void __launch_bounds__(256) spdb_fix_kernel(double* __restrict__ A, int n, int lda, int k0, int kb,
                                                       const double* __restrict__ D, const double* __restrict__ P) {
  __shared__ double t[32][33];
  const int i0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (c0 >= kb) return;
  if (i0 + 32 <= k0) {
    // rows before the block: A[k0 + c][i] = D[i][c]
    for (int r = ty; r < 32; r += 8) t[r][tx] = D[(size_t)(i0 + r) * BB + c0 + tx];
    __syncthreads();
    for (int r = ty; r < 32; r += 8)
      if (c0 + r < kb) A[(size_t)(k0 + c0 + r) * lda + i0 + tx] = t[tx][r];
    return;
  }
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, c = c0 + tx;
    if (i >= n || c >= kb) continue;
    if (i >= k0 + kb) A[(size_t)i * lda + k0 + c] = D[(size_t)i * BB + c];
    else if (i >= k0 && i - k0 >= c) A[(size_t)i * lda + k0 + c] = P[(size_t)(i - k0) * BB + c];
  }
}

int spd_inverse_blocked(lrs_ctx* ctx, double* A, int n, int lda, int* status) {
  if (n <= 0) return LRS_OK;
  static_assert(BB % 32 == 0, "the outer block is a whole number of 32-wide tiles");
  // C, E, D [n][BB] and the pivot block [BB][BB]
  LRS_TRY(ensure(ctx, ctx->ws.gjb, 3 * (size_t)n * BB + (size_t)BB * BB));
  double* C = ctx->ws.gjb.ptr;
  double* E = C + (size_t)n * BB;
  double* D = E + (size_t)n * BB;
  double* P = D + (size_t)n * BB;
  const int nblk = (n + BB - 1) / BB;
  for (int kk = 0; kk < nblk; ++kk) {
    const int k0 = kk * BB, kb = std::min(BB, n - k0);
    spdb_gather_kernel<<<dim3((n + 31) / 32, BB / 32), 256, 0, ctx->stream>>>(A, n, lda, k0, kb, C, E, P);
    LRS_TRY(after_launch(ctx, "spdb_gather_kernel"));
    // P <- (C_KK)^-1 (lower triangle), then the full symmetric P for the product
    ctx->spd_inner = true;
    const int rc = spd_inverse(ctx, P, kb, BB, status);
    ctx->spd_inner = false;
    LRS_TRY(rc);
    LRS_TRY(mirror_lower(ctx, P, kb, BB));
    // D = C P
    LRS_TRY(oz_gemm_batched(ctx, false, false, n, kb, kb, 1.0, C, BB, 0, nullptr, 0, P, BB, 0, 0.0, D, BB, 0, 1, 0));
    // A -= D E^T on the tiles that reach the lower triangle (block K's rows and columns are
    // rewritten below; the upper triangle is never read)
    LRS_TRY(stage_begin(ctx, ST_W_MAIN));
    LRS_TRY(oz_gemm_batched(ctx, false, true, n, n, kb, -1.0, D, BB, 0, nullptr, 0, E, BB, 0, 1.0, A, lda, 0, 1,
                            n));
    LRS_TRY(stage_end(ctx, ST_W_MAIN));
    {
      // lower-triangle elements outside the rows and columns of block K
      const double nn = n, b0 = k0, b1 = k0 + kb;
      const double rows_in = (b1 * (b1 + 1) - b0 * (b0 + 1)) / 2.0;
      const double elems = nn * (nn + 1) / 2.0 - rows_in - (b1 - b0) * (nn - b1);
      ctx->w_main_flop += 2.0 * kb * elems;
      ctx->w_main_elems += elems;
      ++ctx->w_main_launches;
    }
    spdb_fix_kernel<<<dim3((n + 31) / 32, BB / 32), 256, 0, ctx->stream>>>(A, n, lda, k0, kb, D, P);
    LRS_TRY(after_launch(ctx, "spdb_fix_kernel"));
  }
  return LRS_OK;
}

}  // namespace lrs
