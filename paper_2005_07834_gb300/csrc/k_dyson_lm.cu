// Dyson equation in the (radial shell, l, m) basis on product grids (Sec. VI.E).
//
// On a grid p = j * nang + a (shell radius r_j, direction Omega_a, the same
// angular set on every shell) the multipole Coulomb operator factorises
// exactly through the addition theorem P_l(u.u') = 4pi/(2l+1) sum_m Y_lm(u) Y_lm(u'):
//   v = Y C Y^T,  Y[(j,a),(j',lm)] = delta_jj' Y_lm(Omega_a),
//   C[(j,lm),(j',l'm')] = delta_{lm,l'm'} 4pi/(2l+1) r_<^l / r_>^(l+1),
// so (I - v Q chi0 Q) W = v becomes, with X = Y^T Q chi0 Q Y and the
// push-through identity (I - U V)^-1 U = U (I - V U)^-1,
//   W = Y Z Y^T,   (I - C X) Z = C,
// an LU of size r = nrad (L+1)^2 instead of npts.  This is the basis in which
// the paper forms chi = S^-1 chi0; here it is used to obtain the full-grid W.
#include <cmath>
#include <vector>

#include "lrs_internal.h"

namespace lrs {

// Real spherical harmonics Y_lm (orthonormal on the sphere) at unit vector u,
// l = 0..L, ordered l*l + l + m for m = -l..l.  Associated Legendre functions
// by the standard upward recurrences in l at fixed m.
static void real_sph_harm(int L, double x, double y, double z, double* out) {
  const double pi = 3.14159265358979323846;
  const double ct = std::max(-1.0, std::min(1.0, z));
  const double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
  const double phi = std::atan2(y, x);
  std::vector<double> P((L + 1) * (L + 1), 0.0);   // P[l][m], m >= 0
  auto Pl = [&](int l, int m) -> double& { return P[l * (L + 1) + m]; };
  Pl(0, 0) = 1.0;
  for (int m = 1; m <= L; ++m) Pl(m, m) = -(2.0 * m - 1.0) * st * Pl(m - 1, m - 1);
  for (int m = 0; m < L; ++m) Pl(m + 1, m) = (2.0 * m + 1.0) * ct * Pl(m, m);
  for (int m = 0; m <= L; ++m)
    for (int l = m + 2; l <= L; ++l)
      Pl(l, m) = ((2.0 * l - 1.0) * ct * Pl(l - 1, m) - (l + m - 1.0) * Pl(l - 2, m)) / (l - m);
  for (int l = 0; l <= L; ++l) {
    for (int m = 0; m <= l; ++m) {
      double ratio = 1.0;   // (l-m)!/(l+m)!
      for (int k = l - m + 1; k <= l + m; ++k) ratio /= k;
      const double norm = std::sqrt((2.0 * l + 1.0) / (4.0 * pi) * ratio);
      if (m == 0) {
        out[l * l + l] = norm * Pl(l, 0);
      } else {
        out[l * l + l + m] = std::sqrt(2.0) * norm * Pl(l, m) * std::cos(m * phi);
        out[l * l + l - m] = std::sqrt(2.0) * norm * Pl(l, m) * std::sin(m * phi);
      }
    }
  }
}

int site_detect_product(lrs_ctx* ctx, Site& s, const double* pts) {
  s.product = false;
  const int n = s.npts;
  auto radius = [&](int p) {
    return std::sqrt(pts[3 * p] * pts[3 * p] + pts[3 * p + 1] * pts[3 * p + 1] + pts[3 * p + 2] * pts[3 * p + 2]);
  };
  const double r0 = radius(0);
  int nang = 1;
  while (nang < n && std::fabs(radius(nang) - r0) <= 1e-12 * r0) ++nang;
  if (n % nang != 0 || nang < 2) return LRS_OK;
  const int nrad = n / nang;
  std::vector<double> rad(nrad);
  for (int j = 0; j < nrad; ++j) {
    const double rj = radius(j * nang);
    rad[j] = rj;
    for (int a = 0; a < nang; ++a) {
      const int p = j * nang + a;
      const double rp = radius(p);
      if (std::fabs(rp - rj) > 1e-12 * rj) return LRS_OK;
      for (int d = 0; d < 3; ++d)
        if (std::fabs(pts[3 * p + d] / rp - pts[3 * a + d] / r0) > 1e-12) return LRS_OK;
    }
  }
  const int L = s.lmax, L2 = (L + 1) * (L + 1);
  std::vector<double> yang((size_t)nang * L2);
  for (int a = 0; a < nang; ++a)
    real_sph_harm(L, pts[3 * a] / r0, pts[3 * a + 1] / r0, pts[3 * a + 2] / r0, &yang[(size_t)a * L2]);
  const double pi = 3.14159265358979323846;
  std::vector<double> rl((size_t)(L + 1) * nrad * nrad);
  for (int l = 0; l <= L; ++l)
    for (int j = 0; j < nrad; ++j)
      for (int k = 0; k < nrad; ++k) {
        const double lo = std::min(rad[j], rad[k]), hi = std::max(rad[j], rad[k]);
        rl[((size_t)l * nrad + j) * nrad + k] = 4.0 * pi / (2.0 * l + 1.0) * std::pow(lo / hi, l) / hi;
      }
  // Cholesky factor of each radial block (positive definite: it is the
  // Coulomb kernel of the l-th multipole on distinct radii)
  std::vector<double> fl(rl.size(), 0.0);
  bool spd = true;
  for (int l = 0; l <= L && spd; ++l) {
    const double* a = &rl[(size_t)l * nrad * nrad];
    double* f = &fl[(size_t)l * nrad * nrad];
    for (int j = 0; j < nrad && spd; ++j) {
      for (int k = 0; k <= j; ++k) {
        double t = a[(size_t)j * nrad + k];
        for (int m = 0; m < k; ++m) t -= f[(size_t)j * nrad + m] * f[(size_t)k * nrad + m];
        if (k == j) {
          if (!(t > 0.0)) { spd = false; break; }
          f[(size_t)j * nrad + j] = std::sqrt(t);
        } else {
          f[(size_t)j * nrad + k] = t / f[(size_t)k * nrad + k];
        }
      }
    }
  }
  LRS_TRY(ensure(ctx, s.yang, yang.size()));
  LRS_TRY(ensure(ctx, s.rl, rl.size()));
  LRS_TRY(h2d_sync(ctx, s.yang.ptr, yang.data(), yang.size() * sizeof(double)));
  LRS_TRY(h2d_sync(ctx, s.rl.ptr, rl.data(), rl.size() * sizeof(double)));
  s.spd = spd;
  if (spd) {
    LRS_TRY(ensure(ctx, s.fl, fl.size()));
    LRS_TRY(h2d_sync(ctx, s.fl.ptr, fl.data(), fl.size() * sizeof(double)));
  }
  s.product = true;
  s.nrad = nrad;
  s.nang = nang;
  return LRS_OK;
}

// B = I - C X on the (j, lm) index: b[(j,lm), c] = delta - sum_j' rl[l][j][j'] X[(j',lm), c].
__global__ void lm_dyson_matrix_kernel(const double* __restrict__ X, const double* __restrict__ rl, int nrad,
                                       int L2, double* __restrict__ B) {
  const int r = nrad * L2;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y;            // (j, lm)
  if (col >= r || row >= r) return;
  const int j = row / L2, lm = row % L2;
  int l = 0;
  while ((l + 1) * (l + 1) <= lm) ++l;
  const double* rlj = rl + ((size_t)l * nrad + j) * nrad;
  double s = 0.0;
  for (int jp = 0; jp < nrad; ++jp) s = fma(rlj[jp], X[(size_t)(jp * L2 + lm) * r + col], s);
  B[(size_t)row * r + col] = (row == col ? 1.0 : 0.0) - s;
}

// Dense C (right-hand side of (I - C X) Z = C).
__global__ void lm_coulomb_kernel(const double* __restrict__ rl, int nrad, int L2, double* __restrict__ Cm) {
  const int r = nrad * L2;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y;
  if (col >= r || row >= r) return;
  const int j = row / L2, lm = row % L2, jp = col / L2, lmp = col % L2;
  double v = 0.0;
  if (lm == lmp) {
    int l = 0;
    while ((l + 1) * (l + 1) <= lm) ++l;
    v = rl[((size_t)l * nrad + j) * nrad + jp];
  }
  Cm[(size_t)row * r + col] = v;
}

// Radial-block products on the (j, lm) index, F given per l as [nrad][nrad]:
//   left:  out[(j,lm), c] = add_i delta + alpha sum_j' f_l(j, j') in[(j',lm), c]
//   right: out[c, (j,lm)] = add_i delta + alpha sum_j' in[c, (j',lm)] f_l(j', j)
// with f_l(a, b) = F_l[b][a] when TF, else F_l[a][b].  F_l is lower triangular
// (a Cholesky factor), so only j' >= j (TF) or j' <= j (not TF) contribute.
// SYM_IN reads `in` from its lower triangle only (a symmetric matrix stored
// that way).
template <bool TF, bool SYM_IN>
__global__ void lm_left_kernel(const double* __restrict__ in, const double* __restrict__ F, int nrad, int L2,
                               double alpha, double add_i, double* __restrict__ out) {
  const int r = nrad * L2;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y;
  if (col >= r || row >= r) return;
  const int j = row / L2, lm = row % L2;
  int l = 0;
  while ((l + 1) * (l + 1) <= lm) ++l;
  const double* f = F + (size_t)l * nrad * nrad;
  double s = 0.0;
  const int lo = TF ? j : 0, hi = TF ? nrad : j + 1;
  for (int jp = lo; jp < hi; ++jp) {
    const double c = TF ? f[(size_t)jp * nrad + j] : f[(size_t)j * nrad + jp];
    const int src = jp * L2 + lm;
    const double x = (!SYM_IN || src >= col) ? in[(size_t)src * r + col] : in[(size_t)col * r + src];
    s = fma(c, x, s);
  }
  out[(size_t)row * r + col] = (row == col ? add_i : 0.0) + alpha * s;
}

template <bool TF>
__global__ void lm_right_kernel(const double* __restrict__ in, const double* __restrict__ F, int nrad, int L2,
                                double alpha, double add_i, double* __restrict__ out) {
  const int r = nrad * L2;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;   // (j, lm)
  const int row = blockIdx.y;
  if (col >= r || row >= r) return;
  const int j = col / L2, lm = col % L2;
  int l = 0;
  while ((l + 1) * (l + 1) <= lm) ++l;
  const double* f = F + (size_t)l * nrad * nrad;
  const double* x = in + (size_t)row * r + lm;
  double s = 0.0;
  const int lo = TF ? 0 : j, hi = TF ? j + 1 : nrad;
  for (int jp = lo; jp < hi; ++jp) {
    const double c = TF ? f[(size_t)j * nrad + jp] : f[(size_t)jp * nrad + j];
    s = fma(x[(size_t)jp * L2], c, s);
  }
  out[(size_t)row * r + col] = (row == col ? add_i : 0.0) + alpha * s;
}

int dyson_solve_lm(lrs_ctx* ctx, Site& s) {
  const int n = s.npts, nrad = s.nrad, nang = s.nang;
  const int L2 = (s.lmax + 1) * (s.lmax + 1), r = nrad * L2;
  const size_t nn = (size_t)n * n, rr = (size_t)r * r;
  // workspace: T / U [n][r], X, B, Z [r][r]
  LRS_TRY(ensure(ctx, ctx->ws.dyson_a, std::max(nn, 3 * rr + (size_t)n * r)));
  LRS_TRY(ensure(ctx, ctx->ws.ipiv, std::max(n, r)));
  double* T = ctx->ws.dyson_a.ptr;        // [n][r]
  double* X = T + (size_t)n * r;          // [r][r]
  double* B = X + rr;                     // [r][r]
  double* Z = B + rr;                     // [r][r]
  const double* Yang = s.yang.ptr;        // [nang][L2]
  // The four basis changes (T, X, U, W) run on the tensor cores from exact bf16
  // slices (float64-accurate, k_ozgemm.cu) wherever the trailing updates of the
  // SPD inverse do, else with float64 FMAs.
  const bool tc = ctx->dyson_update == LRS_UPDATE_TC ||
                  (ctx->dyson_update == LRS_UPDATE_AUTO && ctx->precision != LRS_FP64);
  // T[:, j' block] = chi0[:, shell j'] diag(Q_j') Yang        (one launch, batch = shell)
  if (tc)
    LRS_TRY(oz_gemm_batched(ctx, false, false, n, L2, nang, 1.0, s.response_chi(), n, nang, s.wts.ptr, nang, Yang,
                            L2, 0, 0.0, T, r, L2, nrad, 0));
  else
    LRS_TRY(dgemm_batched(ctx, false, false, n, L2, nang, 1.0, s.response_chi(), n, nang, s.wts.ptr, nang, Yang, L2,
                          0, nullptr, 0.0, T, r, L2, nrad));
  // X = Y^T Q T is symmetric; its transpose is formed, X^T[:, j block] = T[shell j, :]^T diag(Q_j) Yang,
  // so that the 81- (generally (L+1)^2-) wide side of the product is a tile column.  The SPD
  // route reads only its lower triangle.
  const bool use_spd = ctx->dyson_solver == LRS_SOLVER_SPD || (ctx->dyson_solver == LRS_SOLVER_AUTO && s.spd);
  if (use_spd && !s.spd) return set_error(LRS_ERR_STATE, "SPD Dyson solver: a radial Coulomb block has no Cholesky factor");
  if (tc)
    LRS_TRY(oz_gemm_batched(ctx, true, false, r, L2, nang, 1.0, T, r, (long long)nang * r, s.wts.ptr, nang, Yang,
                            L2, 0, 0.0, X, r, L2, nrad, use_spd ? L2 : 0));
  else if (use_spd)
    LRS_TRY(dgemm_batched_lower(ctx, true, false, r, L2, nang, T, r, (long long)nang * r, s.wts.ptr, nang, Yang,
                                L2, X, r, nrad));
  else
    LRS_TRY(dgemm_batched(ctx, true, false, r, L2, nang, 1.0, T, r, (long long)nang * r, s.wts.ptr, nang, Yang,
                          L2, 0, nullptr, 0.0, X, r, L2, nrad));
  dim3 g((r + 127) / 128, r);
  // 128-wide pivot blocks on request (LRS_OPT_DYSON_PANEL); the default keeps the 32-wide
  // exchange, whose trailing update overlaps the pivot chain
  const bool blocked = ctx->dyson_panel == SPD_OUTER_BLOCK;
  if (use_spd && tc) {
    // The same four radial-block products as below, each a GEMM over the radial index per lm
    // (rows c, columns j, contraction j'), float64-accurate on the tensor cores.  With
    // Fh = blockdiag_lm F_l (Fh[(j', lm), (j, lm)] = F_l[j'][j]):
    //   B = X Fh,  M = I - B^T Fh = I - Fh^T X Fh,  Y = M^-1 Fh^T,  Z = Y^T Fh^T = Fh M^-1 Fh^T.
    // A product whose operand is a symmetric matrix S reads S[(j', lm), c] for S[c, (j', lm)]
    // (consecutive c, consecutive words); M and Z are symmetric, so they are stored at the
    // transposed position, again with consecutive c in consecutive words.
    const long long R = r, LR = (long long)L2 * r;
    const OzOperand Fjpj{s.fl.ptr, 1, nrad, (long long)nrad * nrad, true};    // (j, j') -> F_l[j'][j]
    const OzOperand Fjjp{s.fl.ptr, nrad, 1, (long long)nrad * nrad, true};    // (j, j') -> F_l[j][j']
    OzStore to_rows;           // [c][(j, lm)]: row c, column j L2 + lm
    to_rows.rs = R;
    to_rows.cs = L2;
    to_rows.sb = 1;
    to_rows.batch_fastest = true;   // entries lm, lm + 1, ... fill the same sectors together
    OzStore to_cols = to_rows;      // [(j, lm)][c]
    to_cols.rs = 1;
    to_cols.cs = LR;
    to_cols.sb = R;
    to_cols.batch_fastest = false;
    LRS_TRY(mirror_lower(ctx, X, r, r));
    to_rows.c = B;
    LRS_TRY(oz_gemm_strided(ctx, r, nrad, nrad, L2, OzOperand{X, 1, LR, R, false}, nullptr, 0, Fjpj, to_rows));
    OzStore m = to_cols;
    m.c = Z;
    m.alpha = -1.0;
    m.dI = 1;                  // diagonal: c == j L2 + lm
    m.dJ = -L2;
    m.dB = -1;
    m.dadd = 1.0;
    LRS_TRY(oz_gemm_strided(ctx, r, nrad, nrad, L2, OzOperand{B, 1, LR, R, false}, nullptr, 0, Fjpj, m));
    if (blocked) LRS_TRY(spd_inverse_blocked(ctx, Z, r, r, ctx->ws.status.ptr));
    else LRS_TRY(spd_inverse(ctx, Z, r, r, ctx->ws.status.ptr));
    LRS_TRY(mirror_lower(ctx, Z, r, r));
    to_rows.c = X;
    LRS_TRY(oz_gemm_strided(ctx, r, nrad, nrad, L2, OzOperand{Z, 1, LR, R, false}, nullptr, 0, Fjjp, to_rows));
    to_cols.c = Z;
    LRS_TRY(oz_gemm_strided(ctx, r, nrad, nrad, L2, OzOperand{X, 1, LR, R, false}, nullptr, 0, Fjjp, to_cols));
  } else if (use_spd) {
    // M = I - F^T X F (in Z), inverted in place; Z = F M^-1 F^T
    lm_left_kernel<true, true><<<g, 128, 0, ctx->stream>>>(X, s.fl.ptr, nrad, L2, 1.0, 0.0, B);
    LRS_TRY(after_launch(ctx, "lm_left_kernel"));
    lm_right_kernel<false><<<g, 128, 0, ctx->stream>>>(B, s.fl.ptr, nrad, L2, -1.0, 1.0, Z);
    LRS_TRY(after_launch(ctx, "lm_right_kernel"));
    if (blocked) LRS_TRY(spd_inverse_blocked(ctx, Z, r, r, ctx->ws.status.ptr));
    else LRS_TRY(spd_inverse(ctx, Z, r, r, ctx->ws.status.ptr));
    lm_left_kernel<false, true><<<g, 128, 0, ctx->stream>>>(Z, s.fl.ptr, nrad, L2, 1.0, 0.0, X);
    LRS_TRY(after_launch(ctx, "lm_left_kernel"));
    lm_right_kernel<true><<<g, 128, 0, ctx->stream>>>(X, s.fl.ptr, nrad, L2, 1.0, 0.0, Z);
    LRS_TRY(after_launch(ctx, "lm_right_kernel"));
    ctx->fp64_flops += 4.0 * (double)r * r * nrad;   // four triangular radial-block products
  } else {
    lm_dyson_matrix_kernel<<<g, 128, 0, ctx->stream>>>(X, s.rl.ptr, nrad, L2, B);
    LRS_TRY(after_launch(ctx, "lm_dyson_matrix_kernel"));
    lm_coulomb_kernel<<<g, 128, 0, ctx->stream>>>(s.rl.ptr, nrad, L2, Z);
    LRS_TRY(after_launch(ctx, "lm_coulomb_kernel"));
    LRS_TRY(lu_factor(ctx, B, r, ctx->ws.ipiv.ptr, ctx->ws.status.ptr));
    LRS_TRY(ensure(ctx, ctx->ws.tinv, 2 * (size_t)((r + 31) / 32) * 32 * 32));
    LRS_TRY(lu_solve_inv(ctx, B, r, ctx->ws.ipiv.ptr, Z, r, r, ctx->ws.tinv.ptr));
  }
  // U[shell j, :] = Yang Z[j block, :]   (reuses T)
  double* U = T;
  if (tc)
    LRS_TRY(oz_gemm_batched(ctx, false, false, nang, r, L2, 1.0, Yang, L2, 0, nullptr, 0, Z, r, (long long)L2 * r,
                            0.0, U, r, (long long)nang * r, nrad, 0));
  else
    LRS_TRY(dgemm_batched(ctx, false, false, nang, r, L2, 1.0, Yang, L2, 0, nullptr, 0, Z, r, (long long)L2 * r,
                          nullptr, 0.0, U, r, (long long)nang * r, nrad));
  // W[:, shell j'] = U[:, j' block] Yang^T on and below the diagonal, then mirrored (W is symmetric)
  if (tc)
    LRS_TRY(oz_gemm_batched(ctx, false, true, n, nang, L2, 1.0, U, r, L2, nullptr, 0, Yang, L2, 0, 0.0, s.w.ptr, n,
                            nang, nrad, nang));
  else
    LRS_TRY(dgemm_batched_lower(ctx, false, true, n, nang, L2, U, r, L2, nullptr, 0, Yang, L2, s.w.ptr, n, nrad));
  return mirror_lower(ctx, s.w.ptr, n, n);
}

}  // namespace lrs
