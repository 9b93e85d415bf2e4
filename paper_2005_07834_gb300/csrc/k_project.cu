// Projection of Bloch orbitals onto a site grid (Sec. VI.B, method 1,
// Eq. (bloch)):  psi_kb(tau + r_p) = Omega^-1/2 e^{i k.R_p} sum_G C_kb(G) e^{i G.R_p}.
//
// The phase matrix P_k(p, G) is never stored: G.R = n1 (b1.R) + n2 (b2.R) +
// n3 (b3.R), so e^{i G.R} is the product of three entries of small per-point
// tables T_i[p][n] = e^{i n (b_i.R_p)}, generated once per site and read from
// L1/L2 while the contraction tiles are staged in shared memory.
#include <cmath>

#include <algorithm>

#include "lrs_internal.h"

namespace lrs {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// tab layout: [3][npts][width_i] with width_i = 2*nmax_i + 1, offsets off_i.
__global__ void phase_tables_kernel(const double* __restrict__ pts, int npts, double cx, double cy,
                                    double cz, double3 b1, double3 b2, double3 b3, int3 nmax,
                                    double2* __restrict__ tab, int off1, int off2) {
  int p = blockIdx.x;
  if (p >= npts) return;
  double rx = cx + pts[3 * p], ry = cy + pts[3 * p + 1], rz = cz + pts[3 * p + 2];
  double th[3] = {b1.x * rx + b1.y * ry + b1.z * rz, b2.x * rx + b2.y * ry + b2.z * rz,
                  b3.x * rx + b3.y * ry + b3.z * rz};
  int nm[3] = {nmax.x, nmax.y, nmax.z};
  int off[3] = {0, off1, off2};
  for (int i = 0; i < 3; ++i) {
    int width = 2 * nm[i] + 1;
    for (int j = threadIdx.x; j < width; j += blockDim.x) {
      double s, c;
      sincos((double)(j - nm[i]) * th[i], &s, &c);
      tab[off[i] + (size_t)p * width + j] = make_double2(c, s);
    }
  }
}

__global__ void kphase_kernel(const double* __restrict__ pts, int npts, double cx, double cy, double cz,
                              const double* __restrict__ kpts, int nk, double inv_sqrt_omega,
                              double2* __restrict__ out) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  if (p >= npts || k >= nk) return;
  double rx = cx + pts[3 * p], ry = cy + pts[3 * p + 1], rz = cz + pts[3 * p + 2];
  double th = kpts[3 * k] * rx + kpts[3 * k + 1] * ry + kpts[3 * k + 2] * rz;
  double s, c;
  sincos(th, &s, &c);
  out[(size_t)k * npts + p] = make_double2(c * inv_sqrt_omega, s * inv_sqrt_omega);
}

constexpr int GK = 16;   // plane waves per chunk

// Column offsets of the k-points of one launch (blockIdx.z = k - k0).
constexpr int PROJ_KMAX = 64;
struct ProjK {
  int k0;
  int nocc[PROJ_KMAX], oofs[PROJ_KMAX], uofs[PROJ_KMAX];
};

// psi[p][b] of k-point k0 + blockIdx.z for a T x T tile (T = 64 or 32), complex FP64, (T/16)^2
// outputs per thread (every k-point of a launch at once, so that small sites still fill the GPU).
template <int T>
__global__ void __launch_bounds__(256) project_fp64_kernel(
    const double2* __restrict__ tab, int npts, int3 nmax, int off1, int off2,
    const int* __restrict__ gvec, int ng, const double2* __restrict__ coeff, int nb,
    const double2* __restrict__ kphase, const ProjK pk, double2* __restrict__ psi_o, int Ko,
    double2* __restrict__ psi_u, int Ku) {
  const int kz = blockIdx.z, k = pk.k0 + kz;
  const double2* __restrict__ coeff_k = coeff + (size_t)k * ng * nb;
  const double2* __restrict__ kph = kphase + (size_t)k * npts;
  const int nocc = pk.nocc[kz], oofs = pk.oofs[kz], uofs = pk.uofs[kz];
  __shared__ double2 As[GK][T + 1];
  __shared__ double2 Bs[GK][T + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int p0 = blockIdx.y * T, b0 = blockIdx.x * T;
  const int w1 = 2 * nmax.x + 1, w2 = 2 * nmax.y + 1, w3 = 2 * nmax.z + 1;
  constexpr int R = T / 16;
  double2 acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int g0 = 0; g0 < ng; g0 += GK) {
    // A: phases for T points x 16 plane waves
    for (int idx = threadIdx.x; idx < GK * T; idx += 256) {
      int kk = idx / T, r = idx % T;
      int g = g0 + kk, p = p0 + r;
      double2 val = make_double2(0.0, 0.0);
      if (g < ng && p < npts) {
        int n1 = gvec[3 * g] + nmax.x, n2 = gvec[3 * g + 1] + nmax.y, n3 = gvec[3 * g + 2] + nmax.z;
        double2 t1 = tab[(size_t)p * w1 + n1];
        double2 t2 = tab[off1 + (size_t)p * w2 + n2];
        double2 t3 = tab[off2 + (size_t)p * w3 + n3];
        val = cmul(cmul(t1, t2), t3);
      }
      As[kk][r] = val;
    }
    // B: coefficients for 16 plane waves x T bands
    for (int idx = threadIdx.x; idx < GK * T; idx += 256) {
      int kk = idx / T, c = idx % T;
      int g = g0 + kk, b = b0 + c;
      Bs[kk][c] = (g < ng && b < nb) ? coeff_k[(size_t)g * nb + b] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      double2 a[R], b[R];
#pragma unroll
      for (int i = 0; i < R; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < R; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int p = p0 + ty + 16 * i;
    if (p >= npts) continue;
    double2 ph = kph[p];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      int b = b0 + tx + 16 * j;
      if (b >= nb) continue;
      double2 v = cmul(ph, acc[i][j]);
      if (b < nocc) psi_o[(size_t)p * Ko + oofs + b] = v;
      else psi_u[(size_t)p * Ku + uofs + (b - nocc)] = v;
    }
  }
}

// Builds the phase tables and e^{ik.R}/sqrt(Omega) of one site into the workspace.
int phase_setup(lrs_ctx* ctx, Site& s, int* off1, int* off2) {
  const int* nm = ctx->gmax_idx;
  int w1 = 2 * nm[0] + 1, w2 = 2 * nm[1] + 1, w3 = 2 * nm[2] + 1;
  size_t n_tab = (size_t)s.npts * (w1 + w2 + w3);
  LRS_TRY(ensure(ctx, ctx->ws.phase_tab, n_tab));
  LRS_TRY(ensure(ctx, ctx->ws.kphase, (size_t)ctx->nk * s.npts));
  *off1 = s.npts * w1;
  *off2 = s.npts * (w1 + w2);
  const double* r = ctx->recip;
  double3 b1 = make_double3(r[0], r[1], r[2]), b2 = make_double3(r[3], r[4], r[5]),
          b3 = make_double3(r[6], r[7], r[8]);
  phase_tables_kernel<<<s.npts, 64, 0, ctx->stream>>>(s.pts.ptr, s.npts, s.center[0], s.center[1],
                                                        s.center[2], b1, b2, b3,
                                                        make_int3(nm[0], nm[1], nm[2]),
                                                        ctx->ws.phase_tab.ptr, *off1, *off2);
  LRS_TRY(after_launch(ctx, "phase_tables_kernel"));
  dim3 grid((s.npts + 127) / 128, ctx->nk);
  kphase_kernel<<<grid, 128, 0, ctx->stream>>>(s.pts.ptr, s.npts, s.center[0], s.center[1], s.center[2],
                                                ctx->d_kpts.ptr, ctx->nk, 1.0 / std::sqrt(ctx->omega),
                                                ctx->ws.kphase.ptr);
  int rc = after_launch(ctx, "kphase_kernel");
  return rc;
}

int project_fp64(lrs_ctx* ctx, Site& s) {
  int off1, off2;
  LRS_TRY(phase_setup(ctx, s, &off1, &off2));
  const int* nm = ctx->gmax_idx;
  int oofs = 0, uofs = 0;
  for (int k0 = 0; k0 < ctx->nk; k0 += PROJ_KMAX) {
    const int nks = std::min(PROJ_KMAX, ctx->nk - k0);
    ProjK pk;
    pk.k0 = k0;
    for (int j = 0; j < nks; ++j) {
      pk.nocc[j] = ctx->nocc[k0 + j];
      pk.oofs[j] = oofs;
      pk.uofs[j] = uofs;
      oofs += ctx->nocc[k0 + j];
      uofs += ctx->nb - ctx->nocc[k0 + j];
    }
    // 32-wide tiles when 64-wide ones would leave most SMs idle (the FP64 pipe of one SM is slow)
    const long long big = (long long)((ctx->nb + 63) / 64) * ((s.npts + 63) / 64) * nks;
    if (big < 2LL * ctx->num_sms) {
      dim3 grid((ctx->nb + 31) / 32, (s.npts + 31) / 32, nks);
      project_fp64_kernel<32><<<grid, 256, 0, ctx->stream>>>(
          ctx->ws.phase_tab.ptr, s.npts, make_int3(nm[0], nm[1], nm[2]), off1, off2, ctx->d_gvec.ptr, ctx->ng,
          ctx->coeff.ptr, ctx->nb, ctx->ws.kphase.ptr, pk, s.psi_o.ptr, ctx->Ko, s.psi_u.ptr, ctx->Ku);
    } else {
      dim3 grid((ctx->nb + 63) / 64, (s.npts + 63) / 64, nks);
      project_fp64_kernel<64><<<grid, 256, 0, ctx->stream>>>(
          ctx->ws.phase_tab.ptr, s.npts, make_int3(nm[0], nm[1], nm[2]), off1, off2, ctx->d_gvec.ptr, ctx->ng,
          ctx->coeff.ptr, ctx->nb, ctx->ws.kphase.ptr, pk, s.psi_o.ptr, ctx->Ko, s.psi_u.ptr, ctx->Ku);
    }
    LRS_TRY(after_launch(ctx, "project_fp64_kernel"));
  }
  return LRS_OK;
}

}  // namespace lrs
