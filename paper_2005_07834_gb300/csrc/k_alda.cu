// ALDA vertex correction (Sec. VII, Eq. (chi-alda) and (kxc_alda)):
//   chi~ = (1 - chi0 (v + f_xc))^-1 chi0,  f_xc(r, r') = delta(r - r') f(r).
// On the grid (integrals weighted by Q = diag(w)) the contact term is
// D = diag(f w), and chi~ = (I - chi0 Q v Q - chi0 D)^-1 chi0 is the RPA
// Dyson chain of the dressed polarizability
//   chi_eff = (I - chi0 D)^-1 chi0,
// since (I - chi0 D)^-1 (I - chi0 Q v Q - chi0 D) = I - chi_eff Q v Q.  So the
// ALDA screened interaction W~ = v + v Q chi~ Q v is the Dyson solve (either
// basis) of chi_eff, which this file forms with an FP64 LU (n right-hand
// sides).  f is given per grid point or, for the exchange-only ALDA, computed
// from the site density n = 2 sum_k w_k sum_occ |psi|^2 as
// f_x(n) = -(1/3) (3/pi)^(1/3) n^(-2/3) (Dirac exchange of the uniform gas).
#include <cmath>

#include "lrs_internal.h"

namespace lrs {

// n(r_p) = 2 sum_c w_c |psi_o[p, c]|^2, one CTA per point.
__global__ void density_kernel(const double2* __restrict__ psi_o, const double* __restrict__ w_o, int Ko,
                               double* __restrict__ n) {
  const int p = blockIdx.x;
  double s = 0.0;
  for (int c = threadIdx.x; c < Ko; c += blockDim.x) {
    const double2 v = psi_o[(size_t)p * Ko + c];
    s = fma(w_o[c], v.x * v.x + v.y * v.y, s);
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    n[p] = 2.0 * s;
  }
}

__global__ void exchange_kernel_kernel(const double* __restrict__ n, int npts, double* __restrict__ f) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npts) return;
  const double c = cbrt(3.0 / 3.14159265358979323846);   // (3/pi)^(1/3)
  const double t = cbrt(n[p]);
  f[p] = -c / (3.0 * t * t);
}

// B = I - chi0 diag(f w).
__global__ void alda_matrix_kernel(const double* __restrict__ chi0, const double* __restrict__ f,
                                   const double* __restrict__ w, int n, double* __restrict__ B) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y;
  if (col >= n) return;
  B[(size_t)row * n + col] = (row == col ? 1.0 : 0.0) - chi0[(size_t)row * n + col] * f[col] * w[col];
}

// m <- (m + m^T) / 2.
__global__ void average_transpose_kernel(double* __restrict__ m, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (q >= n || q < p) return;
  const double s = 0.5 * (m[(size_t)p * n + q] + m[(size_t)q * n + p]);
  m[(size_t)p * n + q] = s;
  m[(size_t)q * n + p] = s;
}

int site_density(lrs_ctx* ctx, Site& s, double* n_dev) {
  if (!s.has_psi) return set_error(LRS_ERR_STATE, "the site has no orbitals (project first)");
  density_kernel<<<s.npts, 256, 0, ctx->stream>>>(s.psi_o.ptr, ctx->w_o.ptr, ctx->Ko, n_dev);
  return after_launch(ctx, "density_kernel");
}

// The kernel f used for the site: the caller's values, or f_x of the current density.
int site_fxc(lrs_ctx* ctx, Site& s) {
  if (s.fxc_kind == LRS_FXC_USER) return LRS_OK;   // uploaded by lrs_set_fxc
  LRS_TRY(ensure(ctx, s.fxc, (size_t)s.npts));
  LRS_TRY(ensure(ctx, ctx->ws.alda_n, (size_t)s.npts));
  LRS_TRY(site_density(ctx, s, ctx->ws.alda_n.ptr));
  exchange_kernel_kernel<<<(s.npts + 255) / 256, 256, 0, ctx->stream>>>(ctx->ws.alda_n.ptr, s.npts, s.fxc.ptr);
  return after_launch(ctx, "exchange_kernel_kernel");
}

int alda_dress(lrs_ctx* ctx, Site& s) {
  const int n = s.npts;
  const size_t nn = (size_t)n * n;
  Workspace& ws = ctx->ws;
  LRS_TRY(site_fxc(ctx, s));
  LRS_TRY(ensure(ctx, s.chi_eff, nn));
  LRS_TRY(ensure(ctx, ws.dyson_a, nn));   // scratch: the Dyson solve that follows rebuilds it
  LRS_TRY(ensure(ctx, ws.ipiv, (size_t)n));
  double* B = ws.dyson_a.ptr;
  alda_matrix_kernel<<<dim3((n + 127) / 128, n), 128, 0, ctx->stream>>>(s.chi0.ptr, s.fxc.ptr, s.wts.ptr, n, B);
  LRS_TRY(after_launch(ctx, "alda_matrix_kernel"));
  LRS_CUDA_TRY(cudaMemcpyAsync(s.chi_eff.ptr, s.chi0.ptr, nn * sizeof(double), cudaMemcpyDeviceToDevice,
                               ctx->stream));
  LRS_TRY(lu_factor(ctx, B, n, ws.ipiv.ptr, ws.status.ptr));
  LRS_TRY(lu_solve(ctx, B, n, ws.ipiv.ptr, s.chi_eff.ptr, n, n));
  // chi_eff is symmetric (chi0 and D are): remove the rounding asymmetry of the solve
  average_transpose_kernel<<<dim3((n + 127) / 128, n), 128, 0, ctx->stream>>>(s.chi_eff.ptr, n);
  return after_launch(ctx, "average_transpose_kernel");
}

}  // namespace lrs
