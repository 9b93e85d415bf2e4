// Float64 polarizability of one site (Eq. (chi1) with the Green's functions of
// Sec. VI.D and the single-grid quadrature of App. D.1).
//
// For each output tile (I, J) of 64 x 64 grid points and each frequency t_f:
//   Go(p,p')   = sum_v conj psi_v(p) d_v(t_f) psi_v(p')       (occupied columns)
//   GuT(p,p')  = sum_c psi_c(p) d_c(t_f) conj psi_c(p')       (unoccupied columns)
//   S(p,p')   += W_f Re[Go(p,p') GuT(p,p')]
// with d = w_k / (mu + i t - eps).  G is never written to memory.  The grid is
// (tiles x frequencies) so that small sites still fill every SM; the per-
// frequency contributions meet in S through float64 atomics.  Finally
// chi0 = (2/pi)(S + S^T) (spin 2 and the 1/2pi of Eq. (chi1) folded with the
// t -> -t symmetry of the integrand).
#include "lrs_internal.h"

namespace lrs {

__global__ void denominators_kernel(const double* __restrict__ e, const double* __restrict__ w, int ncol,
                                    const double* __restrict__ t, int nf, double mu,
                                    double2* __restrict__ d) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int f = blockIdx.y;
  if (c >= ncol || f >= nf) return;
  // w / (alpha + i t) = w (alpha - i t) / (alpha^2 + t^2),  alpha = mu - eps
  double alpha = mu - e[c], tf = t[f];
  double den = alpha * alpha + tf * tf;
  d[(size_t)f * ncol + c] = make_double2(w[c] * alpha / den, -w[c] * tf / den);
}

int build_denominators(lrs_ctx* ctx) {
  LRS_TRY(ensure(ctx, ctx->ws.denom_o, (size_t)ctx->nf * ctx->Ko));
  LRS_TRY(ensure(ctx, ctx->ws.denom_u, (size_t)ctx->nf * ctx->Ku));
  dim3 go((ctx->Ko + 255) / 256, ctx->nf), gu((ctx->Ku + 255) / 256, ctx->nf);
  denominators_kernel<<<go, 256, 0, ctx->stream>>>(ctx->e_o.ptr, ctx->w_o.ptr, ctx->Ko, ctx->d_t.ptr, ctx->nf,
                                                    ctx->mu, ctx->ws.denom_o.ptr);
  LRS_TRY(after_launch(ctx, "denominators_kernel"));
  denominators_kernel<<<gu, 256, 0, ctx->stream>>>(ctx->e_u.ptr, ctx->w_u.ptr, ctx->Ku, ctx->d_t.ptr, ctx->nf,
                                                    ctx->mu, ctx->ws.denom_u.ptr);
  LRS_TRY(after_launch(ctx, "denominators_kernel"));
  return LRS_OK;
}

constexpr int TT = 64;   // tile edge (points)
constexpr int KC = 16;   // columns per chunk

__device__ __forceinline__ double2 cmul64(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Accumulates acc(p,p') += sum_k A(p,k) B(p',k) over one column set where
//   A(p,k) = conjA ? conj(psi(p,k)) d(k) : psi(p,k) d(k)
//   B(p',k)= conjA ? psi(p',k)          : conj(psi(p',k))
template <bool kOcc>
__device__ __forceinline__ void tile_green(const double2* __restrict__ psi, int K, const double2* __restrict__ d,
                                           int n, int i0, int j0, double2 (&As)[KC][TT + 1],
                                           double2 (&Bs)[KC][TT + 1], double2 (&acc)[4][4]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int k0 = 0; k0 < K; k0 += KC) {
    for (int idx = threadIdx.x; idx < KC * TT; idx += 256) {
      int r = idx / KC, kk = idx % KC;
      int k = k0 + kk;
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
      if (k < K) {
        double2 dk = d[k];
        if (i0 + r < n) {
          double2 v = psi[(size_t)(i0 + r) * K + k];
          if (kOcc) v.y = -v.y;
          a = cmul64(v, dk);
        }
        if (j0 + r < n) {
          b = psi[(size_t)(j0 + r) * K + k];
          if (!kOcc) b.y = -b.y;
        }
      }
      As[kk][r] = a;
      Bs[kk][r] = b;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) chi0_fp64_kernel(
    const double2* __restrict__ psi_o, int Ko, const double2* __restrict__ psi_u, int Ku,
    const double2* __restrict__ denom_o, const double2* __restrict__ denom_u, const double* __restrict__ Wf,
    int n, double* __restrict__ S) {
  __shared__ double2 As[KC][TT + 1];
  __shared__ double2 Bs[KC][TT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * TT, j0 = blockIdx.x * TT, f = blockIdx.z;
  double2 go[4][4], gu[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) go[i][j] = gu[i][j] = make_double2(0.0, 0.0);
  tile_green<true>(psi_o, Ko, denom_o + (size_t)f * Ko, n, i0, j0, As, Bs, go);
  tile_green<false>(psi_u, Ku, denom_u + (size_t)f * Ku, n, i0, j0, As, Bs, gu);
  const double wf = Wf[f];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int p = i0 + ty + 16 * i;
    if (p >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int q = j0 + tx + 16 * j;
      if (q >= n) continue;
      double re = go[i][j].x * gu[i][j].x - go[i][j].y * gu[i][j].y;
      S[((size_t)f * n + p) * n + q] = wf * re;   // this frequency's slab: no atomics, fixed sum order
    }
  }
}

// chi0 = (2/pi)(S + S^T), in place (each thread owns one (p, q) pair with p <= q).
__global__ void symmetrize_kernel(double* __restrict__ m, int n) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  int p = blockIdx.y;
  if (p >= n || q >= n || q < p) return;
  const double c = 0.63661977236758134308;  // 2/pi
  double a = m[(size_t)p * n + q], b = m[(size_t)q * n + p];
  double s = c * (a + b);
  m[(size_t)p * n + q] = s;
  m[(size_t)q * n + p] = s;
}

int symmetrize_chi0(lrs_ctx* ctx, double* chi0, int n) {
  dim3 grid((n + 127) / 128, n);
  symmetrize_kernel<<<grid, 128, 0, ctx->stream>>>(chi0, n);
  return after_launch(ctx, "symmetrize_kernel");
}

// chi0 = (2/pi) sum_f (S_f + S_f^T), frequencies summed in order (deterministic).
__global__ void reduce_slabs_kernel(const double* __restrict__ slab, int n, int nf, double* __restrict__ chi0) {
  __shared__ double t[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int f = 0; f < nf; ++f) {
    const double* s = slab + (size_t)f * n * n;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = c0 + ty + 8 * i, c = r0 + tx;
      t[ty + 8 * i][tx] = (r < n && c < n) ? s[(size_t)r * n + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + ty + 8 * i, c = c0 + tx;
      const double direct = (r < n && c < n) ? s[(size_t)r * n + c] : 0.0;
      acc[i] += direct + t[tx][ty + 8 * i];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty + 8 * i, c = c0 + tx;
    if (r < n && c < n) chi0[(size_t)r * n + c] = 0.63661977236758134308 * acc[i];
  }
}

int chi0_fp64(lrs_ctx* ctx, Site& s) {
  const int n = s.npts;
  LRS_TRY(ensure(ctx, ctx->ws.slab64, (size_t)ctx->nf * n * n));
  LRS_TRY(stage_begin(ctx, ST_CHI0_MAIN));
  dim3 grid((n + TT - 1) / TT, (n + TT - 1) / TT, ctx->nf);
  chi0_fp64_kernel<<<grid, 256, 0, ctx->stream>>>(s.psi_o.ptr, ctx->Ko, s.psi_u.ptr, ctx->Ku,
                                                   ctx->ws.denom_o.ptr, ctx->ws.denom_u.ptr, ctx->d_W.ptr, n,
                                                   ctx->ws.slab64.ptr);
  LRS_TRY(after_launch(ctx, "chi0_fp64_kernel"));
  LRS_TRY(stage_end(ctx, ST_CHI0_MAIN));
  dim3 rg((n + 31) / 32, (n + 31) / 32);
  reduce_slabs_kernel<<<rg, dim3(32, 8), 0, ctx->stream>>>(ctx->ws.slab64.ptr, n, ctx->nf, s.chi0.ptr);
  return after_launch(ctx, "reduce_slabs_kernel");
}

}  // namespace lrs
