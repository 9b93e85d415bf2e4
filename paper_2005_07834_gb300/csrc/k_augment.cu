// All-electron augmentation of the site orbitals (Sec. VI.C, Eq. (eq-aug1)
// and (eq-aug2)):
//   psi_ae = psi_ps + sum_lm sum_{nu,nu'} Y_lm [phi_ae_{nu l} - phi_ps_{nu l}]
//                     (A_l^-1)_{nu nu'} <phi_ps_{nu' l} Y_lm | psi_ps>,
//   A_{nu nu'; l} = int_0^{r_a} dr r^2 phi_ps_{nu l} phi_ps_{nu' l},
// on the site's product grid: radial integrals by the grid's radial weights
// over the shells with r_j <= r_a, projections with the point weights.  The
// host forms A_l, inverts it and folds it into the correction functions
//   E_{nu' l}(r_j) = sum_nu [phi_ae - phi_ps]_{nu l}(r_j) (A_l^-1)_{nu nu'};
// the device computes c = <phi_ps Y_lm | psi> for every orbital column and
// adds sum E Y_lm c in place, in float64.
#include <cmath>
#include <vector>

#include "lrs_internal.h"

namespace lrs {

// c[proj][col] = sum_p w_p P_{l nu}(r_j) Y_lm(a) psi[p][col], proj = (l^2 + l + m) nnu + nu.
__global__ void augment_project_kernel(const double2* __restrict__ psi, int ncol, const double* __restrict__ wts,
                                       const double* __restrict__ pf, const double* __restrict__ yang, int L2,
                                       int nrad, int nang, int nnu, double2* __restrict__ c) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int proj = blockIdx.y;
  if (col >= ncol) return;
  const int lm = proj / nnu, nu = proj % nnu;
  int l = 0;
  while ((l + 1) * (l + 1) <= lm) ++l;
  const double* f = pf + ((size_t)l * nnu + nu) * nrad;
  double sr = 0.0, si = 0.0;
  for (int j = 0; j < nrad; ++j) {
    const double fj = f[j];
    if (fj == 0.0) continue;   // shells beyond the augmentation radius
    for (int a = 0; a < nang; ++a) {
      const size_t p = (size_t)j * nang + a;
      const double g = wts[p] * fj * yang[(size_t)a * L2 + lm];
      const double2 v = psi[p * ncol + col];
      sr = fma(g, v.x, sr);
      si = fma(g, v.y, si);
    }
  }
  c[(size_t)proj * ncol + col] = make_double2(sr, si);
}

// psi[p][col] += sum_proj E_{l nu}(r_j) Y_lm(a) c[proj][col] on shells inside the radius.
__global__ void augment_apply_kernel(double2* __restrict__ psi, int ncol, const double* __restrict__ ef,
                                     const unsigned char* __restrict__ inside, const double* __restrict__ yang,
                                     int L2, int nrad, int nang, int nnu, int nproj,
                                     const double2* __restrict__ c) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (col >= ncol) return;
  const int j = p / nang, a = p % nang;
  if (!inside[j]) return;
  double sr = 0.0, si = 0.0;
  for (int proj = 0; proj < nproj; ++proj) {
    const int lm = proj / nnu, nu = proj % nnu;
    int l = 0;
    while ((l + 1) * (l + 1) <= lm) ++l;
    const double g = ef[((size_t)l * nnu + nu) * nrad + j] * yang[(size_t)a * L2 + lm];
    const double2 v = c[(size_t)proj * ncol + col];
    sr = fma(g, v.x, sr);
    si = fma(g, v.y, si);
  }
  double2 o = psi[(size_t)p * ncol + col];
  o.x += sr;
  o.y += si;
  psi[(size_t)p * ncol + col] = o;
}

// In-place inverse of a small matrix (Gauss-Jordan with partial pivoting); false if singular.
static bool invert_small(std::vector<double>& a, int n) {
  std::vector<double> inv(n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[r * n + c]) > std::fabs(a[piv * n + c])) piv = r;
    if (!(std::fabs(a[piv * n + c]) > 0.0) || !std::isfinite(a[piv * n + c])) return false;
    for (int k = 0; k < n; ++k) {
      std::swap(a[c * n + k], a[piv * n + k]);
      std::swap(inv[c * n + k], inv[piv * n + k]);
    }
    const double d = 1.0 / a[c * n + c];
    for (int k = 0; k < n; ++k) {
      a[c * n + k] *= d;
      inv[c * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[r * n + k] -= f * a[c * n + k];
        inv[r * n + k] -= f * inv[c * n + k];
      }
    }
  }
  a = inv;
  return true;
}

int augment_site(lrs_ctx* ctx, Site& s, int lmax_aug, int nnu, double r_aug, const double* phi_ae,
                 const double* phi_ps) {
  const int n = s.npts, nrad = s.nrad, nang = s.nang;
  const int L2 = (s.lmax + 1) * (s.lmax + 1), nproj = (lmax_aug + 1) * (lmax_aug + 1) * nnu;
  // shell radii and radial weights from the grid (host copies of the site's points and weights)
  std::vector<double> pts((size_t)n * 3), wts(n);
  LRS_CUDA_TRY(cudaMemcpyAsync(pts.data(), s.pts.ptr, pts.size() * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
  LRS_CUDA_TRY(cudaMemcpyAsync(wts.data(), s.wts.ptr, wts.size() * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  const double four_pi = 12.566370614359172953850573533118;
  std::vector<double> wr(nrad);
  std::vector<unsigned char> inside(nrad);
  for (int j = 0; j < nrad; ++j) {
    const double* p = &pts[3 * (size_t)j * nang];
    const double r = std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double sw = 0.0;
    for (int a = 0; a < nang; ++a) sw += wts[(size_t)j * nang + a];
    wr[j] = sw / four_pi;
    inside[j] = r <= r_aug ? 1 : 0;
  }
  // pseudo partial waves inside the radius, and the corrections with A_l^-1 folded in
  std::vector<double> pf((size_t)(lmax_aug + 1) * nnu * nrad, 0.0), ef(pf.size(), 0.0);
  for (int l = 0; l <= lmax_aug; ++l) {
    const double* ps = phi_ps + (size_t)l * nnu * nrad;
    const double* ae = phi_ae + (size_t)l * nnu * nrad;
    std::vector<double> A((size_t)nnu * nnu, 0.0);
    for (int u = 0; u < nnu; ++u)
      for (int v = 0; v < nnu; ++v)
        for (int j = 0; j < nrad; ++j)
          if (inside[j]) A[u * nnu + v] += wr[j] * ps[(size_t)u * nrad + j] * ps[(size_t)v * nrad + j];
    if (!invert_small(A, nnu))
      return set_error(LRS_ERR_NUMERIC, "overlap of the pseudo partial waves for l = %d is singular", l);
    for (int v = 0; v < nnu; ++v)
      for (int j = 0; j < nrad; ++j) {
        if (!inside[j]) continue;
        pf[((size_t)l * nnu + v) * nrad + j] = ps[(size_t)v * nrad + j];
        double e = 0.0;
        for (int u = 0; u < nnu; ++u) e += (ae[(size_t)u * nrad + j] - ps[(size_t)u * nrad + j]) * A[u * nnu + v];
        ef[((size_t)l * nnu + v) * nrad + j] = e;
      }
  }
  Workspace& ws = ctx->ws;
  const int K = std::max(ctx->Ko, ctx->Ku);
  const size_t tab = pf.size();
  LRS_TRY(ensure(ctx, ws.aug_tab, 2 * tab + (nrad + 7) / 8));
  LRS_TRY(ensure(ctx, ws.aug_coef, (size_t)nproj * K));
  double* d_pf = ws.aug_tab.ptr;
  double* d_ef = d_pf + tab;
  unsigned char* d_in = reinterpret_cast<unsigned char*>(d_ef + tab);
  LRS_CUDA_TRY(cudaMemcpyAsync(d_pf, pf.data(), tab * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  LRS_CUDA_TRY(cudaMemcpyAsync(d_ef, ef.data(), tab * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  LRS_CUDA_TRY(cudaMemcpyAsync(d_in, inside.data(), nrad, cudaMemcpyHostToDevice, ctx->stream));
  for (int blk = 0; blk < 2; ++blk) {
    double2* psi = blk == 0 ? s.psi_o.ptr : s.psi_u.ptr;
    const int ncol = blk == 0 ? ctx->Ko : ctx->Ku;
    augment_project_kernel<<<dim3((ncol + 127) / 128, nproj), 128, 0, ctx->stream>>>(
        psi, ncol, s.wts.ptr, d_pf, s.yang.ptr, L2, nrad, nang, nnu, ws.aug_coef.ptr);
    LRS_TRY(after_launch(ctx, "augment_project_kernel"));
    augment_apply_kernel<<<dim3((ncol + 127) / 128, n), 128, 0, ctx->stream>>>(
        psi, ncol, d_ef, d_in, s.yang.ptr, L2, nrad, nang, nnu, nproj, ws.aug_coef.ptr);
    LRS_TRY(after_launch(ctx, "augment_apply_kernel"));
  }
  // the host tables above are read by copies in flight: finish before they go out of scope
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return LRS_OK;
}

}  // namespace lrs
