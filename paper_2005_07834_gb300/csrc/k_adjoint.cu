// Adjoint of (band energies, site-grid orbitals) -> chi0 -> W for one site.
// The paper has no gradients; this is the derivative of the computation it
// defines (Eq. (chi1) with the single-grid quadrature, Eq. (eq-W)).
//
// With A = I - v Q chi0 Q and W = A^-1 v,  dW = W Q dchi0 Q W, so
//   dL/dchi0 = Q W^T G_W W^T Q (+ any direct dL/dchi0),
// and with chi0 = (2/pi)(S + S^T), dL/dS = G_S = (2/pi)(G + G^T).
// Per frequency t_f (mu and the quadrature held fixed) the Green's functions
//   Go(p,p')   = sum_b conj psi(p,b) d_b psi(p',b)     (occupied)
//   GuT(p,p')  = sum_c psi(p,c) d_c conj psi(p',c)     (unoccupied)
// are recomputed (never stored across frequencies), S_f = W_f Re[Go o GuT],
// and with Ho = W_f G_S o GuT, Hu = W_f G_S o Go:
//   Yo = Ho psi_o,  Zo = Ho^T conj psi_o,  Yu = Hu conj psi_u,  Zu = Hu^T psi_u,
//   dL/dpsi_o += d Yo + conj(d Zo),        dL/dpsi_u += conj(d Yu) + d Zu,
//   dL/deps_b += Re[(d_b^2 / w_b) sum_p conj psi(p,b) Yo(p,b)]   (occupied)
//   dL/deps_c += Re[(d_c^2 / w_c) sum_p psi(p,c) Yu(p,c)]        (unoccupied)
// in the dL/dRe + i dL/dIm convention.  All arithmetic is float64.
#include <algorithm>

#include "lrs_internal.h"

namespace lrs {

constexpr int ZK = 16;    // k chunk

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }

// C[m][n] = sum_k opA(m,k) s_k opB(k,n)  (+ beta C), complex float64, row-major.
// opA(m,k) = (TA ? A[k][m] : A[m][k]), conjugated if CA; opB likewise.  Batch z
// (blockIdx.z) offsets A, s, B and C by z times their batch strides (0: shared).
struct ZBatch {
  long long a, s, b, c;
};
// T x T output tile (T = 64 or 32), 256 threads of (T/16) x (T/16) outputs each.
template <bool TA, bool CA, bool TB, bool CB, int T>
__global__ void __launch_bounds__(256) zgemm64_kernel(int m, int n, int k, const double2* __restrict__ A, int lda,
                                                      const double2* __restrict__ s, const double2* __restrict__ B,
                                                      int ldb, double beta, double2* __restrict__ C, int ldc,
                                                      ZBatch bs) {
  A += blockIdx.z * bs.a;
  if (s) s += blockIdx.z * bs.s;
  B += blockIdx.z * bs.b;
  C += blockIdx.z * bs.c;
  constexpr int R = T / 16;   // outputs per thread and dimension
  __shared__ double2 As[ZK][T + 1];
  __shared__ double2 Bs[ZK][T + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * T, j0 = blockIdx.x * T;
  double2 acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < k; k0 += ZK) {
    for (int idx = threadIdx.x; idx < ZK * T; idx += 256) {
      int r, kk;
      if (TA) { kk = idx / T; r = idx % T; } else { r = idx / ZK; kk = idx % ZK; }
      const int gi = i0 + r, gk = k0 + kk;
      double2 a = make_double2(0.0, 0.0);
      if (gi < m && gk < k) {
        a = TA ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk];
        if (CA) a = zconj(a);
        if (s) a = zmul(a, s[gk]);
      }
      As[kk][r] = a;
    }
    for (int idx = threadIdx.x; idx < ZK * T; idx += 256) {
      int c, kk;
      if (TB) { c = idx / ZK; kk = idx % ZK; } else { kk = idx / T; c = idx % T; }
      const int gj = j0 + c, gk = k0 + kk;
      double2 b = make_double2(0.0, 0.0);
      if (gj < n && gk < k) {
        b = TB ? B[(size_t)gj * ldb + gk] : B[(size_t)gk * ldb + gj];
        if (CB) b = zconj(b);
      }
      Bs[kk][c] = b;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < ZK; ++kk) {
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
    const int gi = i0 + ty + 16 * i;
    if (gi >= m) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int gj = j0 + tx + 16 * j;
      if (gj >= n) continue;
      double2* c = &C[(size_t)gi * ldc + gj];
      if (beta == 0.0) {
        *c = acc[i][j];
      } else {
        const double2 o = *c;
        *c = make_double2(fma(beta, o.x, acc[i][j].x), fma(beta, o.y, acc[i][j].y));
      }
    }
  }
}

template <bool TA, bool CA, bool TB, bool CB>
static int zgemm64(lrs_ctx* ctx, int m, int n, int k, const double2* A, int lda, const double2* s,
                   const double2* B, int ldb, double beta, double2* C, int ldc, int batch = 1,
                   ZBatch bs = ZBatch{0, 0, 0, 0}) {
  // 32-wide tiles when 64-wide ones would leave most SMs idle (the FP64 pipe of one SM is slow)
  const long long big = (long long)((n + 63) / 64) * ((m + 63) / 64) * batch;
  if (big < 2LL * ctx->num_sms) {
    dim3 grid((n + 31) / 32, (m + 31) / 32, batch);
    zgemm64_kernel<TA, CA, TB, CB, 32><<<grid, 256, 0, ctx->stream>>>(m, n, k, A, lda, s, B, ldb, beta, C, ldc, bs);
  } else {
    dim3 grid((n + 63) / 64, (m + 63) / 64, batch);
    zgemm64_kernel<TA, CA, TB, CB, 64><<<grid, 256, 0, ctx->stream>>>(m, n, k, A, lda, s, B, ldb, beta, C, ldc, bs);
  }
  return after_launch(ctx, "zgemm64_kernel");
}

// G_S = (2/pi) [Q_p Q_q (T[p][q] + T[q][p]) + gc[p][q] + gc[q][p]]
__global__ void gamma_s_kernel(const double* __restrict__ T, const double* __restrict__ gc,
                               const double* __restrict__ q, int n, double* __restrict__ G) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (c >= n || r >= n) return;
  double v = 0.0;
  if (T) v = q[r] * q[c] * (T[(size_t)r * n + c] + T[(size_t)c * n + r]);
  if (gc) v += gc[(size_t)r * n + c] + gc[(size_t)c * n + r];
  G[(size_t)r * n + c] = 0.63661977236758134308 * v;
}

// In place, for nb frequencies f stored one after the other (nn elements each):
// go <- W_f G_S o gu (= Ho), gu <- W_f G_S o go (= Hu).
__global__ void hadamard_kernel(const double* __restrict__ G, const double* __restrict__ wf, size_t nn, int nb,
                                double2* __restrict__ go, double2* __restrict__ gu) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= nn * nb) return;
  const double g = wf[i / nn] * G[i % nn];
  const double2 a = go[i], b = gu[i];
  go[i] = make_double2(g * b.x, g * b.y);
  gu[i] = make_double2(g * a.x, g * a.y);
}

// Accumulates the orbital and energy gradients of one column set and frequency.
// occupied: gpsi += d Y + conj(d Z),  e_b = sum_p conj psi(p,b) Y(p,b)
// unoccupied: gpsi += conj(d Y) + d Z, e_c = sum_p psi(p,c) Y(p,c)
// A CTA covers 32 columns (one per lane, so rows are read coalesced) and GA_ROWS
// rows (eight row groups); the column sums e of its rows go to part[chunk][b]
// and grad_energy_kernel adds the chunks in a fixed order (no atomics: the
// result does not depend on the schedule).
constexpr int GA_ROWS = 256;
template <bool kOcc>
__global__ void __launch_bounds__(256) grad_accum_kernel(const double2* __restrict__ psi,
                                                         const double2* __restrict__ Y,
                                                         const double2* __restrict__ Z,
                                                         const double2* __restrict__ d, int n, int K,
                                                         double2* __restrict__ gpsi, double2* __restrict__ part) {
  __shared__ double2 red[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int b = blockIdx.x * 32 + tx;
  const int p0 = blockIdx.y * GA_ROWS;
  double er = 0.0, ei = 0.0;
  if (b < K) {
    const double2 db = d[b];
    const int p1 = min(n, p0 + GA_ROWS);
    for (int p = p0 + ty; p < p1; p += 8) {
      const size_t ix = (size_t)p * K + b;
      const double2 y = Y[ix], z = Z[ix], ps = psi[ix];
      const double2 dy = zmul(db, y), dz = zmul(db, z);
      double2 g = gpsi[ix];
      g.x += dy.x + dz.x;
      g.y += kOcc ? (dy.y - dz.y) : (-dy.y + dz.y);
      gpsi[ix] = g;
      const double2 t = kOcc ? zmul(zconj(ps), y) : zmul(ps, y);
      er += t.x;
      ei += t.y;
    }
  }
  red[ty][tx] = make_double2(er, ei);
  __syncthreads();
  if (ty == 0 && b < K) {
    double2 s = red[0][tx];
    for (int r = 1; r < 8; ++r) { s.x += red[r][tx].x; s.y += red[r][tx].y; }
    part[(size_t)blockIdx.y * K + b] = s;
  }
}

// ge[b] += Re[e_b d_b^2 / w_b] with e_b the sum of the row chunks' partial sums (in chunk order).
__global__ void grad_energy_kernel(const double2* __restrict__ part, int chunks, const double2* __restrict__ d,
                                   const double* __restrict__ w, int K, double* __restrict__ ge) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= K) return;
  double er = 0.0, ei = 0.0;
  for (int c = 0; c < chunks; ++c) {
    const double2 v = part[(size_t)c * K + b];
    er += v.x;
    ei += v.y;
  }
  const double2 db = d[b];
  const double2 d2 = zmul(db, db);
  ge[b] += (er * d2.x - ei * d2.y) / w[b];
}

int grad_energy(lrs_ctx* ctx, const double2* part, int chunks, const double2* d, const double* w, int K,
                double* ge) {
  grad_energy_kernel<<<(K + 255) / 256, 256, 0, ctx->stream>>>(part, chunks, d, w, K, ge);
  return after_launch(ctx, "grad_energy_kernel");
}

// Scatter of the internal (occupied | unoccupied) columns to the public (k, band) order.
__global__ void scatter_grad_kernel(const double2* __restrict__ go, const double2* __restrict__ gu, int n, int Ko,
                                    int Ku, const int* __restrict__ col_o, const int* __restrict__ col_u, int ncol,
                                    double2* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (p >= n || j >= Ko + Ku) return;
  if (j < Ko) out[(size_t)p * ncol + col_o[j]] = go[(size_t)p * Ko + j];
  else out[(size_t)p * ncol + col_u[j - Ko]] = gu[(size_t)p * Ku + (j - Ko)];
}

__global__ void scatter_energy_kernel(const double* __restrict__ ge, int Ko, int Ku, const int* __restrict__ col_o,
                                      const int* __restrict__ col_u, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Ko + Ku) return;
  if (j < Ko) out[col_o[j]] = ge[j];
  else out[col_u[j - Ko]] = ge[j];
}

// G_S = (2/pi)(G + G^T), G = Q W^T G_W W^T Q + dL/dchi0, into ws.gamma_s.
int gamma_s_build(lrs_ctx* ctx, Site& s, const double* grad_w, const double* grad_chi0) {
  const int n = s.npts;
  const size_t nn = (size_t)n * n;
  Workspace& ws = ctx->ws;
  LRS_TRY(ensure(ctx, ws.gamma_s, nn));
  double* T = nullptr;
  if (grad_w) {
    LRS_TRY(ensure(ctx, ws.tmp_nn, 2 * nn));
    double* T1 = ws.tmp_nn.ptr;
    T = ws.tmp_nn.ptr + nn;
    // the two n^3 products run float64-accurate on the tensor cores wherever the Dyson products do
    const bool tc = ctx->dyson_update == LRS_UPDATE_TC ||
                    (ctx->dyson_update == LRS_UPDATE_AUTO && ctx->precision != LRS_FP64);
    if (tc) {
      LRS_TRY(oz_gemm_batched(ctx, false, true, n, n, n, 1.0, grad_w, n, 0, nullptr, 0, s.w.ptr, n, 0, 0.0, T1, n, 0,
                              1, 0));
      LRS_TRY(oz_gemm_batched(ctx, true, false, n, n, n, 1.0, s.w.ptr, n, 0, nullptr, 0, T1, n, 0, 0.0, T, n, 0, 1,
                              0));
    } else {
      LRS_TRY(dgemm_t(ctx, false, true, n, n, n, 1.0, grad_w, n, nullptr, s.w.ptr, n, nullptr, 0.0, T1, n));
      LRS_TRY(dgemm_t(ctx, true, false, n, n, n, 1.0, s.w.ptr, n, nullptr, T1, n, nullptr, 0.0, T, n));
    }
  }
  dim3 g2((n + 127) / 128, n);
  gamma_s_kernel<<<g2, 128, 0, ctx->stream>>>(T, grad_chi0, s.wts.ptr, n, ws.gamma_s.ptr);
  return after_launch(ctx, "gamma_s_kernel");
}

int backward_site(lrs_ctx* ctx, Site& s, const double* grad_w, const double* grad_chi0, double* grad_e,
                  double2* grad_psi) {
  if (ctx->precision != LRS_FP64) return backward_site_mixed(ctx, s, grad_w, grad_chi0, grad_e, grad_psi);
  const int n = s.npts, Ko = ctx->Ko, Ku = ctx->Ku, K = Ko + Ku, nf = ctx->nf;
  const size_t nn = (size_t)n * n;
  Workspace& ws = ctx->ws;
  // frequencies per batch: the Green's functions and Y, Z of a batch held at once (up to ~1 GB),
  // so that the small problems of small sites still fill the GPU
  const size_t per_f = (2 * nn + 2 * (size_t)n * K) * sizeof(double2);
  const int fb = (int)std::max<size_t>(1, std::min<size_t>((size_t)nf, ((size_t)1 << 30) / per_f));
  LRS_TRY(ensure(ctx, ws.gbuf_o, nn * fb));
  LRS_TRY(ensure(ctx, ws.gbuf_u, nn * fb));
  LRS_TRY(ensure(ctx, ws.ybuf, 2 * (size_t)n * K * fb));
  LRS_TRY(ensure(ctx, ws.gpsi, (size_t)n * K));
  LRS_TRY(ensure(ctx, ws.ge, (size_t)K));
  const int chunks = (n + GA_ROWS - 1) / GA_ROWS;
  LRS_TRY(ensure(ctx, ws.gpart, (size_t)chunks * K));
  // denominators of the current quadrature (held fixed)
  LRS_TRY(build_denominators(ctx));
  LRS_TRY(gamma_s_build(ctx, s, grad_w, grad_chi0));
  LRS_CUDA_TRY(cudaMemsetAsync(ws.gpsi.ptr, 0, (size_t)n * K * sizeof(double2), ctx->stream));
  LRS_CUDA_TRY(cudaMemsetAsync(ws.ge.ptr, 0, (size_t)K * sizeof(double), ctx->stream));
  double2* go = ws.gbuf_o.ptr;
  double2* gu = ws.gbuf_u.ptr;
  // per frequency of the batch: Y = [Yo | Yu], Z = [Zo | Zu], each [n][Kx]
  const long long yz = 2LL * n * K;
  double2* gpo = ws.gpsi.ptr;
  double2* gpu = ws.gpsi.ptr + (size_t)n * Ko;
  for (int f0 = 0; f0 < nf; f0 += fb) {
    const int nb = std::min(fb, nf - f0);
    const double2* dof = ws.denom_o.ptr + (size_t)f0 * Ko;
    const double2* duf = ws.denom_u.ptr + (size_t)f0 * Ku;
    double2* Yo = ws.ybuf.ptr;
    double2* Yu = Yo + (size_t)n * Ko;
    double2* Zo = Yo + (size_t)n * K;
    double2* Zu = Zo + (size_t)n * Ko;
    const long long snn = (long long)nn;
    // Go = (conj psi_o d) psi_o^T,  GuT = (psi_u d) conj(psi_u)^T  (one launch per batch of frequencies)
    LRS_TRY((zgemm64<false, true, true, false>(ctx, n, n, Ko, s.psi_o.ptr, Ko, dof, s.psi_o.ptr, Ko, 0.0, go, n, nb,
                                               ZBatch{0, Ko, 0, snn})));
    LRS_TRY((zgemm64<false, false, true, true>(ctx, n, n, Ku, s.psi_u.ptr, Ku, duf, s.psi_u.ptr, Ku, 0.0, gu, n, nb,
                                               ZBatch{0, Ku, 0, snn})));
    hadamard_kernel<<<(unsigned)((nn * nb + 255) / 256), 256, 0, ctx->stream>>>(ws.gamma_s.ptr, ctx->d_W.ptr + f0,
                                                                               nn, nb, go, gu);
    LRS_TRY(after_launch(ctx, "hadamard_kernel"));
    // now go = Ho, gu = Hu
    LRS_TRY((zgemm64<false, false, false, false>(ctx, n, Ko, n, go, n, nullptr, s.psi_o.ptr, Ko, 0.0, Yo, Ko, nb,
                                                 ZBatch{snn, 0, 0, yz})));
    LRS_TRY((zgemm64<true, false, false, true>(ctx, n, Ko, n, go, n, nullptr, s.psi_o.ptr, Ko, 0.0, Zo, Ko, nb,
                                               ZBatch{snn, 0, 0, yz})));
    LRS_TRY((zgemm64<false, false, false, true>(ctx, n, Ku, n, gu, n, nullptr, s.psi_u.ptr, Ku, 0.0, Yu, Ku, nb,
                                                ZBatch{snn, 0, 0, yz})));
    LRS_TRY((zgemm64<true, false, false, false>(ctx, n, Ku, n, gu, n, nullptr, s.psi_u.ptr, Ku, 0.0, Zu, Ku, nb,
                                                ZBatch{snn, 0, 0, yz})));
    for (int j = 0; j < nb; ++j) {
      const double2* dj_o = dof + (size_t)j * Ko;
      const double2* dj_u = duf + (size_t)j * Ku;
      const size_t o = (size_t)j * yz;
      grad_accum_kernel<true><<<dim3((Ko + 31) / 32, chunks), 256, 0, ctx->stream>>>(s.psi_o.ptr, Yo + o, Zo + o,
                                                                                     dj_o, n, Ko, gpo, ws.gpart.ptr);
      LRS_TRY(after_launch(ctx, "grad_accum_kernel"));
      LRS_TRY(grad_energy(ctx, ws.gpart.ptr, chunks, dj_o, ctx->w_o.ptr, Ko, ws.ge.ptr));
      grad_accum_kernel<false><<<dim3((Ku + 31) / 32, chunks), 256, 0, ctx->stream>>>(s.psi_u.ptr, Yu + o, Zu + o,
                                                                                      dj_u, n, Ku, gpu, ws.gpart.ptr);
      LRS_TRY(after_launch(ctx, "grad_accum_kernel"));
      LRS_TRY(grad_energy(ctx, ws.gpart.ptr, chunks, dj_u, ctx->w_u.ptr, Ku, ws.ge.ptr + Ko));
    }
  }
  return scatter_gradients(ctx, n, gpo, gpu, ws.ge.ptr, grad_e, grad_psi);
}

// Internal (occupied | unoccupied) gradient columns to the public (k, band) order.
int scatter_gradients(lrs_ctx* ctx, int n, const double2* gpo, const double2* gpu, const double* ge,
                      double* grad_e, double2* grad_psi) {
  const int Ko = ctx->Ko, Ku = ctx->Ku, K = Ko + Ku;
  const int ncol = ctx->nk * ctx->nb;
  dim3 gs((K + 255) / 256, n);
  scatter_grad_kernel<<<gs, 256, 0, ctx->stream>>>(gpo, gpu, n, Ko, Ku, ctx->d_col_o.ptr, ctx->d_col_u.ptr, ncol,
                                                   grad_psi);
  LRS_TRY(after_launch(ctx, "scatter_grad_kernel"));
  scatter_energy_kernel<<<(K + 255) / 256, 256, 0, ctx->stream>>>(ge, Ko, Ku, ctx->d_col_o.ptr, ctx->d_col_u.ptr,
                                                                   grad_e);
  return after_launch(ctx, "scatter_energy_kernel");
}

}  // namespace lrs
