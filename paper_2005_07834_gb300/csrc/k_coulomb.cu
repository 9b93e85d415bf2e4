// Coulomb operator on a site grid in multipole form (Sec. VI.E): the expansion
// v = sum_lm 4pi/(2l+1) r_<^l/r_>^(l+1) Y_lm Y*_lm, summed over m with the
// addition theorem, gives v(p,q) = (1/r_>) sum_{l<=L} (r_</r_>)^l P_l(u_p . u_q),
// evaluated with the Legendre recurrence (l+1) P_{l+1} = (2l+1) x P_l - l P_{l-1}.
#include "lrs_internal.h"

namespace lrs {

__global__ void radial_unit_kernel(const double* __restrict__ pts, int n, RadialUnit* __restrict__ ru) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double x = pts[3 * p], y = pts[3 * p + 1], z = pts[3 * p + 2];
  double r = sqrt(x * x + y * y + z * z);
  double inv = 1.0 / r;
  ru[p] = RadialUnit{x * inv, y * inv, z * inv, r};
}

__global__ void coulomb_kernel(const RadialUnit* __restrict__ ru, int n, int lmax, double* __restrict__ v) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  int p = blockIdx.y;
  if (p >= n || q >= n) return;
  RadialUnit a = ru[p], b = ru[q];
  double x = a.x * b.x + a.y * b.y + a.z * b.z;
  x = fmin(1.0, fmax(-1.0, x));
  double rl = fmin(a.r, b.r), rg = fmax(a.r, b.r);
  double rho = rl / rg;
  double p0 = 1.0, p1 = x, sum = 1.0, rp = 1.0;
  for (int l = 1; l <= lmax; ++l) {
    rp *= rho;
    sum = fma(rp, p1, sum);
    double p2 = ((2.0 * l + 1.0) * x * p1 - l * p0) / (l + 1.0);
    p0 = p1;
    p1 = p2;
  }
  v[(size_t)p * n + q] = sum / rg;
}

int coulomb_build(lrs_ctx* ctx, Site& s, double* v) {
  LRS_TRY(ensure(ctx, ctx->ws.ru, (size_t)s.npts));
  RadialUnit* ru = ctx->ws.ru.ptr;
  radial_unit_kernel<<<(s.npts + 127) / 128, 128, 0, ctx->stream>>>(s.pts.ptr, s.npts, ru);
  LRS_TRY(after_launch(ctx, "radial_unit_kernel"));
  dim3 grid((s.npts + 127) / 128, s.npts);
  coulomb_kernel<<<grid, 128, 0, ctx->stream>>>(ru, s.npts, s.lmax, v);
  return after_launch(ctx, "coulomb_kernel");
}

}  // namespace lrs
