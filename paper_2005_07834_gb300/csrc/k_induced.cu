// Response to a spherical short-range potential in the (radial shell, l, m)
// basis: the induced density and potential of Sec. VI.E (the core-hole
// screening of the paper), with v1 of Eq. (eq-partition) for v_ext = q / r:
//   v1(r) = q (1/r - 1/R_S) inside the shell radius R_S, 0 outside.
//
// On a product grid p = j * nang + a, with Y[(j,a),(j,lm)] = Y_lm(Omega_a)
// restricted to l <= l_resp, Q = diag(w) and X = Y^T Q chi0 Q Y, the paper's
// S = I - chi0_lm v (radial integrals by quadrature) and chi = S^-1 chi0_lm give
//   z = (I - X C)^-1 X u,   u[(j,00)] = sqrt(4 pi) v1(r_j),
//   rho_lm(r_j) = z[(j,lm)] / w_r(j),   v_ind_lm(r_j) = (C z)[(j,lm)],
// C the block-diagonal radial Coulomb matrix 4 pi/(2l+1) r_<^l / r_>^(l+1) and
// w_r(j) = sum_a w[(j,a)] / 4 pi the radial weights.  With l_resp = L this is
// the full lm-basis response (v_ind = v Q chi Q v1 on the grid); l_resp = 0 is
// the paper's default.
#include <cmath>

#include "lrs_internal.h"

namespace lrs {

// Per shell: radial weight, and u = sqrt(4 pi) v1(r_j).
__global__ void induced_shell_kernel(const double* __restrict__ pts, const double* __restrict__ wts, int nrad,
                                     int nang, double q, double rs, double* __restrict__ wr,
                                     double* __restrict__ u) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nrad) return;
  const double four_pi = 12.566370614359172953850573533118;
  double s = 0.0;
  for (int a = 0; a < nang; ++a) s += wts[(size_t)j * nang + a];
  wr[j] = s / four_pi;
  const double* p = pts + 3 * (size_t)j * nang;
  const double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  u[j] = r < rs ? sqrt(four_pi) * q * (1.0 / r - 1.0 / rs) : 0.0;
}

// y = X u (only the l = 0 columns of X meet u).
__global__ void induced_rhs_kernel(const double* __restrict__ X, int nrad, int L2s, const double* __restrict__ u,
                                   double* __restrict__ y) {
  const int d = nrad * L2s;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= d) return;
  double s = 0.0;
  for (int jp = 0; jp < nrad; ++jp) s = fma(X[(size_t)row * d + (size_t)jp * L2s], u[jp], s);
  y[row] = s;
}

// B = I - X C: B[row, (j', lm)] = delta - sum_x X[row, (x, lm)] c_l(x, j').
__global__ void induced_matrix_kernel(const double* __restrict__ X, const double* __restrict__ rl, int nrad,
                                      int L2s, double* __restrict__ B) {
  const int d = nrad * L2s;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y;
  if (col >= d || row >= d) return;
  const int jp = col / L2s, lm = col % L2s;
  int l = 0;
  while ((l + 1) * (l + 1) <= lm) ++l;
  const double* c = rl + (size_t)l * nrad * nrad;
  const double* x = X + (size_t)row * d + lm;
  double s = 0.0;
  for (int k = 0; k < nrad; ++k) s = fma(x[(size_t)k * L2s], c[(size_t)k * nrad + jp], s);
  B[(size_t)row * d + col] = (row == col ? 1.0 : 0.0) - s;
}

// rho = z / w_r, v_ind = C z.
__global__ void induced_out_kernel(const double* __restrict__ z, const double* __restrict__ rl,
                                   const double* __restrict__ wr, int nrad, int L2s, double* __restrict__ rho,
                                   double* __restrict__ vind) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrad * L2s) return;
  const int j = i / L2s, lm = i % L2s;
  int l = 0;
  while ((l + 1) * (l + 1) <= lm) ++l;
  const double* c = rl + ((size_t)l * nrad + j) * nrad;
  double s = 0.0;
  for (int jp = 0; jp < nrad; ++jp) s = fma(c[jp], z[(size_t)jp * L2s + lm], s);
  rho[i] = z[i] / wr[j];
  vind[i] = s;
}

// v_ind on the grid: sum_{lm < L2s} v_ind_lm(r_j) Y_lm(Omega_a).
__global__ void induced_grid_kernel(const double* __restrict__ vind, const double* __restrict__ yang, int nrad,
                                    int nang, int L2, int L2s, double* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nrad * nang) return;
  const int j = p / nang, a = p % nang;
  double s = 0.0;
  for (int lm = 0; lm < L2s; ++lm) s = fma(vind[(size_t)j * L2s + lm], yang[(size_t)a * L2 + lm], s);
  out[p] = s;
}

int induced_potential(lrs_ctx* ctx, Site& s, double q, double rs, int lresp, double* rho_h, double* vind_h,
                      double* grid_h) {
  const int n = s.npts, nrad = s.nrad, nang = s.nang;
  const int L2 = (s.lmax + 1) * (s.lmax + 1), L2s = (lresp + 1) * (lresp + 1), d = nrad * L2s;
  Workspace& ws = ctx->ws;
  // T [n][d] | X [d][d] | B [d][d] | y [d] | wr, u [nrad] | rho, vind [d] | grid [n]
  const size_t need = (size_t)n * d + 2 * (size_t)d * d + 3 * (size_t)d + 2 * (size_t)nrad + n;
  LRS_TRY(ensure(ctx, ws.induced, need));
  LRS_TRY(ensure(ctx, ws.ipiv, std::max(d, n)));
  double* T = ws.induced.ptr;
  double* X = T + (size_t)n * d;
  double* B = X + (size_t)d * d;
  double* y = B + (size_t)d * d;
  double* wr = y + d;
  double* u = wr + nrad;
  double* rho = u + nrad;
  double* vind = rho + d;
  double* grid = vind + d;
  // T[:, (j, lm)] = chi0[:, shell j] diag(w_j) Y_sub;  X[(j, lm), :] = Y_sub^T diag(w_j) T[shell j, :]
  LRS_TRY(dgemm_batched(ctx, false, false, n, L2s, nang, 1.0, s.response_chi(), n, nang, s.wts.ptr, nang, s.yang.ptr, L2,
                        0, nullptr, 0.0, T, d, L2s, nrad));
  LRS_TRY(dgemm_batched(ctx, true, false, L2s, d, nang, 1.0, s.yang.ptr, L2, 0, s.wts.ptr, nang, T, d,
                        (long long)nang * d, nullptr, 0.0, X, d, (long long)L2s * d, nrad));
  induced_shell_kernel<<<(nrad + 127) / 128, 128, 0, ctx->stream>>>(s.pts.ptr, s.wts.ptr, nrad, nang, q, rs, wr, u);
  LRS_TRY(after_launch(ctx, "induced_shell_kernel"));
  induced_rhs_kernel<<<(d + 127) / 128, 128, 0, ctx->stream>>>(X, nrad, L2s, u, y);
  LRS_TRY(after_launch(ctx, "induced_rhs_kernel"));
  induced_matrix_kernel<<<dim3((d + 127) / 128, d), 128, 0, ctx->stream>>>(X, s.rl.ptr, nrad, L2s, B);
  LRS_TRY(after_launch(ctx, "induced_matrix_kernel"));
  LRS_TRY(lu_factor(ctx, B, d, ws.ipiv.ptr, ws.status.ptr));
  LRS_TRY(lu_solve(ctx, B, d, ws.ipiv.ptr, y, 1, 1));
  induced_out_kernel<<<(d + 127) / 128, 128, 0, ctx->stream>>>(y, s.rl.ptr, wr, nrad, L2s, rho, vind);
  LRS_TRY(after_launch(ctx, "induced_out_kernel"));
  induced_grid_kernel<<<(n + 127) / 128, 128, 0, ctx->stream>>>(vind, s.yang.ptr, nrad, nang, L2, L2s, grid);
  LRS_TRY(after_launch(ctx, "induced_grid_kernel"));
  if (rho_h) LRS_CUDA_TRY(cudaMemcpyAsync(rho_h, rho, d * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (vind_h) LRS_CUDA_TRY(cudaMemcpyAsync(vind_h, vind, d * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (grid_h) LRS_CUDA_TRY(cudaMemcpyAsync(grid_h, grid, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  int status[2] = {0, 0};
  LRS_CUDA_TRY(cudaMemcpyAsync(status, ws.status.ptr, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (status[0] != 0) {
    cudaMemsetAsync(ws.status.ptr, 0, 4 * sizeof(int), ctx->stream);
    return set_error(LRS_ERR_NUMERIC, "induced response: zero or non-finite pivot (column %d)", status[1]);
  }
  return LRS_OK;
}

}  // namespace lrs
