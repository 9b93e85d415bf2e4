// Projection by Sec. VI.B, method 2: the periodic parts u_kb are carried to a
// real-space grid over the cell by an inverse FFT of their plane-wave
// coefficients, interpolated to the site points with 3rd-degree Lagrange
// polynomials (nodes i0 - 1 .. i0 + 2 in each lattice direction, periodic),
// and multiplied by the Bloch phase exp(i k.r) / sqrt(Omega).
//
// Grid layout per k-point: [N1][N2][N3][nb] complex, bands innermost, so that
// every transform line and every interpolation stencil row is a contiguous
// run of bands (coalesced).  The transform is pruned: the z pass runs only on
// (x, y) columns that hold a G vector (fused with the scatter of the
// coefficients), the y pass only on x-planes that hold one, the x pass on all
// lines.  Each 1-D transform is a mixed-radix (3, 2) Stockham inverse DFT in
// shared memory over BC interleaved band columns.  Mixed-precision contexts
// transform in fp32 (the interpolation error of the method, 1e-3..1e-2, is
// far above fp32 rounding); FP64 contexts in float64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lrs_internal.h"

namespace lrs {

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

template <typename T> struct FftBands;                       // band columns per CTA
template <> struct FftBands<float> { static constexpr int BC = 32; };
template <> struct FftBands<double> { static constexpr int BC = 16; };

constexpr int FFT_THREADS = 256;

bool fft_length_ok(int n) {
  if (n < 1 || n > LRS_FFT_MAX_N) return false;
  while (n % 3 == 0) n /= 3;
  while (n % 2 == 0) n /= 2;
  return n == 1;
}

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// Inverse DFT (exponent +2 pi i) of length N of BC interleaved sequences,
// element i of sequence b at X[i * BC + b].  Stage with radix R on sub-length
// n and stride s (n s = N, m = n / R):
//   y[q + s (R p + t)] = w_n^{p t} sum_{r < R} x[q + s (p + r m)] w_R^{r t},
// w_n = exp(2 pi i / n), for p < m, q < s, t < R; the output of the last
// stage is in natural order.  tw[j] = exp(2 pi i j / N).  Returns the buffer
// holding the result.
template <typename T>
__device__ typename Cplx<T>::type* stockham_inverse(typename Cplx<T>::type* X, typename Cplx<T>::type* Y,
                                                    const typename Cplx<T>::type* __restrict__ tw, int N, int BC) {
  using C = typename Cplx<T>::type;
  const T h3 = (T)0.866025403784438646763723170752936183;   // sin(2 pi / 3)
  int n = N, s = 1;
  while (n > 1) {
    const int R = (n % 3 == 0) ? 3 : 2;
    const int m = n / R;
    const int total = m * s * BC;
    const int tstep = N / n;
    const size_t in_step = (size_t)s * m * BC, out_step = (size_t)s * BC;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int b = idx % BC, rest = idx / BC, q = rest % s, p = rest / s;
      const C* src = X + (size_t)(q + s * p) * BC + b;
      C* dst = Y + (size_t)(q + s * R * p) * BC + b;
      if (R == 2) {
        const C a0 = src[0], a1 = src[in_step];
        dst[0] = C{a0.x + a1.x, a0.y + a1.y};
        dst[out_step] = cmul(C{a0.x - a1.x, a0.y - a1.y}, tw[p * tstep]);
      } else {
        const C a0 = src[0], a1 = src[in_step], a2 = src[2 * in_step];
        const C sum = C{a1.x + a2.x, a1.y + a2.y};
        const C rot = C{-h3 * (a1.y - a2.y), h3 * (a1.x - a2.x)};   // i sin(2pi/3) (a1 - a2)
        const C base = C{a0.x - (T)0.5 * sum.x, a0.y - (T)0.5 * sum.y};
        dst[0] = C{a0.x + sum.x, a0.y + sum.y};
        dst[out_step] = cmul(C{base.x + rot.x, base.y + rot.y}, tw[p * tstep]);
        dst[2 * out_step] = cmul(C{base.x - rot.x, base.y - rot.y}, tw[2 * p * tstep]);
      }
    }
    __syncthreads();
    C* t = X;
    X = Y;
    Y = t;
    n = m;
    s *= R;
  }
  return X;
}

// Coefficients of one populated (x, y) column placed at z = n3 mod N3, then
// the z transform; written to grid[(x N2 + y) N3 + z][band].
template <typename T>
__global__ void __launch_bounds__(FFT_THREADS) fft_z_kernel(const double2* __restrict__ coeff, int nb,
                                                            const int* __restrict__ col_xy,
                                                            const int* __restrict__ col_ptr,
                                                            const int* __restrict__ ent_g,
                                                            const int* __restrict__ ent_z, int ncol, int N3,
                                                            const double2* __restrict__ tw_d,
                                                            typename Cplx<T>::type* __restrict__ grid) {
  using C = typename Cplx<T>::type;
  constexpr int BC = FftBands<T>::BC;
  extern __shared__ __align__(16) unsigned char fft_smem[];
  C* X = reinterpret_cast<C*>(fft_smem);
  C* Y = X + N3 * BC;
  C* tw = Y + N3 * BC;
  // band chunk fastest: neighbouring CTAs read adjacent bands of the same rows
  const int c = blockIdx.y + blockIdx.z * gridDim.y, b0 = blockIdx.x * BC;
  if (c >= ncol) return;
  for (int i = threadIdx.x; i < N3 * BC; i += blockDim.x) X[i] = C{(T)0, (T)0};
  for (int i = threadIdx.x; i < N3; i += blockDim.x) tw[i] = C{(T)tw_d[i].x, (T)tw_d[i].y};
  __syncthreads();
  const int e0 = col_ptr[c], e1 = col_ptr[c + 1];
  for (int idx = threadIdx.x; idx < (e1 - e0) * BC; idx += blockDim.x) {
    const int e = e0 + idx / BC, b = idx % BC;
    if (b0 + b < nb) {
      const double2 v = coeff[(size_t)ent_g[e] * nb + b0 + b];
      X[ent_z[e] * BC + b] = C{(T)v.x, (T)v.y};
    }
  }
  __syncthreads();
  const C* R = stockham_inverse<T>(X, Y, tw, N3, BC);
  const size_t base = (size_t)col_xy[c] * N3 * nb;
  for (int idx = threadIdx.x; idx < N3 * BC; idx += blockDim.x) {
    const int z = idx / BC, b = idx % BC;
    if (b0 + b < nb) grid[base + (size_t)z * nb + b0 + b] = R[idx];
  }
}

// In-place transform of length N along one axis.  Line (ai, ci) =
// (blockIdx.y, blockIdx.z): a = a_list[ai] (or ai), elements at
// a sa + ci sc + i stride; blockIdx.x is the band chunk.
template <typename T>
__global__ void __launch_bounds__(FFT_THREADS) fft_line_kernel(typename Cplx<T>::type* __restrict__ grid, int nb,
                                                               int N, long long stride,
                                                               const int* __restrict__ a_list, long long sa,
                                                               long long sc,
                                                               const double2* __restrict__ tw_d) {
  using C = typename Cplx<T>::type;
  constexpr int BC = FftBands<T>::BC;
  extern __shared__ __align__(16) unsigned char fft_smem[];
  C* X = reinterpret_cast<C*>(fft_smem);
  C* Y = X + N * BC;
  C* tw = Y + N * BC;
  const int ai = blockIdx.y, ci = blockIdx.z, b0 = blockIdx.x * BC;
  const long long a = a_list ? a_list[ai] : ai;
  const size_t base = (size_t)(a * sa + ci * sc);
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = C{(T)tw_d[i].x, (T)tw_d[i].y};
  for (int idx = threadIdx.x; idx < N * BC; idx += blockDim.x) {
    const int i = idx / BC, b = idx % BC;
    X[idx] = (b0 + b < nb) ? grid[base + (size_t)i * stride + b0 + b] : C{(T)0, (T)0};
  }
  __syncthreads();
  const C* R = stockham_inverse<T>(X, Y, tw, N, BC);
  for (int idx = threadIdx.x; idx < N * BC; idx += blockDim.x) {
    const int i = idx / BC, b = idx % BC;
    if (b0 + b < nb) grid[base + (size_t)i * stride + b0 + b] = R[idx];
  }
}

struct LagrangeGeom {
  double center[3];
  double inv[9];      // inverse of the cell matrix (rows a1..a3): fractional f = r inv
  double k[3];
  double scale;       // Omega^-1/2
  int n[3];
};

// psi(p, (k, b)) = exp(i k.r) Omega^-1/2 sum_{a,b,c < 4} L_a(t1) L_b(t2) L_c(t3) u[i0 + (a, b, c) - 1][band],
// written to the occupied (b < nocc) or unoccupied block.
template <typename T>
__global__ void __launch_bounds__(FFT_THREADS) lagrange_kernel(const typename Cplx<T>::type* __restrict__ grid,
                                                               int nb, const double* __restrict__ pts,
                                                               LagrangeGeom g, int nocc, int oofs, int uofs,
                                                               int Ko, int Ku, double2* __restrict__ psi_o,
                                                               double2* __restrict__ psi_u) {
  using C = typename Cplx<T>::type;
  __shared__ T wt[64];
  __shared__ long long off[64];
  __shared__ double2 phase;
  const int p = blockIdx.x;
  if (threadIdx.x < 64) {
    double r[3], s[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) r[d] = g.center[d] + pts[3 * (size_t)p + d];
#pragma unroll
    for (int d = 0; d < 3; ++d) s[d] = (r[0] * g.inv[d] + r[1] * g.inv[3 + d] + r[2] * g.inv[6 + d]) * g.n[d];
    const int tid = (int)threadIdx.x;   // stencil point (a, b, c) = (tid / 16, tid / 4 % 4, tid % 4)
    double w = 1.0;
    long long lin = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double fl = floor(s[d]);
      const double t = s[d] - fl;
      const int m = (d == 0 ? tid >> 4 : d == 1 ? (tid >> 2) & 3 : tid & 3) - 1;   // node offset -1 .. 2
      double l;
      if (m == -1) l = -t * (t - 1.0) * (t - 2.0) / 6.0;
      else if (m == 0) l = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;
      else if (m == 1) l = -(t + 1.0) * t * (t - 2.0) / 2.0;
      else l = (t + 1.0) * t * (t - 1.0) / 6.0;
      w *= l;
      long long idx = ((long long)fl + m) % g.n[d];
      if (idx < 0) idx += g.n[d];
      lin = lin * g.n[d] + idx;
    }
    wt[threadIdx.x] = (T)w;
    off[threadIdx.x] = lin * nb;
    if (threadIdx.x == 0) {
      const double kr = g.k[0] * r[0] + g.k[1] * r[1] + g.k[2] * r[2];
      double sn, cs;
      sincos(kr, &sn, &cs);
      phase = make_double2(cs * g.scale, sn * g.scale);
    }
  }
  __syncthreads();
  const double2 ph = phase;
  for (int b = blockIdx.y * blockDim.x + threadIdx.x; b < nb; b += gridDim.y * blockDim.x) {
    T ar = (T)0, ai = (T)0;
#pragma unroll 8
    for (int j = 0; j < 64; ++j) {
      const C v = grid[off[j] + b];
      ar = fma(wt[j], v.x, ar);
      ai = fma(wt[j], v.y, ai);
    }
    const double2 o = make_double2(ph.x * (double)ar - ph.y * (double)ai, ph.x * (double)ai + ph.y * (double)ar);
    if (b < nocc) psi_o[(size_t)p * Ko + oofs + b] = o;
    else psi_u[(size_t)p * Ku + uofs + (b - nocc)] = o;
  }
}

// ---------------------------------------------------------------- host

// Grid actually used: the explicit sizes, or per direction the smallest
// 2^a 3^b >= 2 (2 max|n_i| + 1) (oversampling 2).
int fft_grid_dims(lrs_ctx* ctx, int n[3]) {
  for (int d = 0; d < 3; ++d) {
    const int need = 2 * ctx->gmax_idx[d] + 1;
    if (ctx->fft_n[d] > 0) {
      if (ctx->fft_n[d] < need)
        return set_error(LRS_ERR_ARG, "FFT grid %d along direction %d holds |n| <= %d, the G set needs %d points",
                         ctx->fft_n[d], d, (ctx->fft_n[d] - 1) / 2, need);
      n[d] = ctx->fft_n[d];
    } else {
      int best = 0;
      for (int c = 2 * need; c <= LRS_FFT_MAX_N && !best; ++c)
        if (fft_length_ok(c)) best = c;
      if (!best)
        return set_error(LRS_ERR_UNSUPPORTED, "no 2^a 3^b FFT length <= %d holds twice %d points", LRS_FFT_MAX_N, need);
      n[d] = best;
    }
  }
  return LRS_OK;
}

static int build_plan(lrs_ctx* ctx, const int n[3]) {
  Workspace& ws = ctx->ws;
  if (ws.fft_plan_ok && ws.fft_plan_n[0] == n[0] && ws.fft_plan_n[1] == n[1] && ws.fft_plan_n[2] == n[2])
    return LRS_OK;
  const int ng = ctx->ng;
  // populated (x, y) columns, their (G, z) entries, populated x-planes
  std::vector<int> key(ng);
  for (int gi = 0; gi < ng; ++gi) {
    const int* v = &ctx->gvec[3 * (size_t)gi];
    const int x = ((v[0] % n[0]) + n[0]) % n[0], y = ((v[1] % n[1]) + n[1]) % n[1];
    key[gi] = x * n[1] + y;
  }
  std::vector<int> order(ng);
  for (int i = 0; i < ng; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
  std::vector<int> col_xy, col_ptr, ent_g, ent_z, xs;
  for (int i = 0; i < ng; ++i) {
    const int gi = order[i];
    if (col_xy.empty() || col_xy.back() != key[gi]) {
      col_xy.push_back(key[gi]);
      col_ptr.push_back(i);
    }
    ent_g.push_back(gi);
    ent_z.push_back(((ctx->gvec[3 * (size_t)gi + 2] % n[2]) + n[2]) % n[2]);
  }
  col_ptr.push_back(ng);
  for (int c : col_xy) {
    const int x = c / n[1];
    if (xs.empty() || xs.back() != x) xs.push_back(x);
  }
  std::vector<int> all;
  ws.fft_off[0] = 0;
  all.insert(all.end(), col_xy.begin(), col_xy.end());
  ws.fft_off[1] = (int)all.size();
  all.insert(all.end(), col_ptr.begin(), col_ptr.end());
  ws.fft_off[2] = (int)all.size();
  all.insert(all.end(), ent_g.begin(), ent_g.end());
  ws.fft_off[3] = (int)all.size();
  all.insert(all.end(), ent_z.begin(), ent_z.end());
  ws.fft_off[4] = (int)all.size();
  all.insert(all.end(), xs.begin(), xs.end());
  ws.fft_ncol = (int)col_xy.size();
  ws.fft_nx = (int)xs.size();
  // twiddles exp(2 pi i j / N) for the three lengths
  std::vector<double2> tw;
  const double two_pi = 6.283185307179586476925286766559;
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < n[d]; ++j) tw.push_back(make_double2(std::cos(two_pi * j / n[d]), std::sin(two_pi * j / n[d])));
  LRS_TRY(ensure(ctx, ws.fft_index, all.size()));
  LRS_TRY(ensure(ctx, ws.fft_tw, tw.size()));
  LRS_TRY(h2d_sync(ctx, ws.fft_index.ptr, all.data(), all.size() * sizeof(int)));
  LRS_TRY(h2d_sync(ctx, ws.fft_tw.ptr, tw.data(), tw.size() * sizeof(double2)));
  for (int d = 0; d < 3; ++d) ws.fft_plan_n[d] = n[d];
  ws.fft_plan_ok = true;
  return LRS_OK;
}

template <typename T>
static size_t fft_smem_bytes(int N) {
  return (2 * (size_t)N * FftBands<T>::BC + N) * sizeof(typename Cplx<T>::type);
}

template <typename T>
static int project_fft_t(lrs_ctx* ctx, const std::vector<int>& list, const int n[3]) {
  using C = typename Cplx<T>::type;
  constexpr int BC = FftBands<T>::BC;
  Workspace& ws = ctx->ws;
  const int nb = ctx->nb;
  const size_t cells = (size_t)n[0] * n[1] * n[2];
  const size_t grid_bytes = cells * nb * sizeof(C);
  LRS_TRY(ensure(ctx, ws.fft_grid, (grid_bytes + sizeof(double2) - 1) / sizeof(double2)));
  C* grid = reinterpret_cast<C*>(ws.fft_grid.ptr);
  const int* col_xy = ws.fft_index.ptr + ws.fft_off[0];
  const int* col_ptr = ws.fft_index.ptr + ws.fft_off[1];
  const int* ent_g = ws.fft_index.ptr + ws.fft_off[2];
  const int* ent_z = ws.fft_index.ptr + ws.fft_off[3];
  const int* xs = ws.fft_index.ptr + ws.fft_off[4];
  const double2* tw1 = ws.fft_tw.ptr;
  const double2* tw2 = tw1 + n[0];
  const double2* tw3 = tw2 + n[1];
  const size_t smax = fft_smem_bytes<T>(LRS_FFT_MAX_N);
  if (!ctx->capturing) {
    LRS_CUDA_TRY(cudaFuncSetAttribute(fft_z_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
    LRS_CUDA_TRY(cudaFuncSetAttribute(fft_line_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
  }
  const unsigned nchunk = (unsigned)((nb + BC - 1) / BC);
  LagrangeGeom geo;
  // inverse of the cell matrix (rows a1..a3) from the reciprocal vectors: inv = recip^T / (2 pi)
  const double two_pi = 6.283185307179586476925286766559;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) geo.inv[i * 3 + j] = ctx->recip[j * 3 + i] / two_pi;
  geo.scale = 1.0 / std::sqrt(ctx->omega);
  for (int d = 0; d < 3; ++d) geo.n[d] = n[d];
  int oofs = 0, uofs = 0;
  for (int k = 0; k < ctx->nk; ++k) {
    const int nocc = ctx->nocc[k];
    LRS_CUDA_TRY(cudaMemsetAsync(grid, 0, grid_bytes, ctx->stream));
    const double2* ck = ctx->coeff.ptr + (size_t)k * ctx->ng * nb;
    const unsigned cy = (unsigned)std::min(ws.fft_ncol, 32768), cz = (unsigned)((ws.fft_ncol + cy - 1) / cy);
    fft_z_kernel<T><<<dim3(nchunk, cy, cz), FFT_THREADS, fft_smem_bytes<T>(n[2]), ctx->stream>>>(
        ck, nb, col_xy, col_ptr, ent_g, ent_z, ws.fft_ncol, n[2], tw3, grid);
    LRS_TRY(after_launch(ctx, "fft_z_kernel"));
    // y: lines (populated x, z), stride N3 nb
    fft_line_kernel<T><<<dim3(nchunk, (unsigned)ws.fft_nx, (unsigned)n[2]), FFT_THREADS, fft_smem_bytes<T>(n[1]),
                         ctx->stream>>>(grid, nb, n[1], (long long)n[2] * nb, xs, (long long)n[1] * n[2] * nb,
                                        (long long)nb, tw2);
    LRS_TRY(after_launch(ctx, "fft_line_kernel"));
    // x: lines (y, z), stride N2 N3 nb
    fft_line_kernel<T><<<dim3(nchunk, (unsigned)n[1], (unsigned)n[2]), FFT_THREADS, fft_smem_bytes<T>(n[0]),
                         ctx->stream>>>(grid, nb, n[0], (long long)n[1] * n[2] * nb, nullptr, (long long)n[2] * nb,
                                        (long long)nb, tw1);
    LRS_TRY(after_launch(ctx, "fft_line_kernel"));
    for (int d = 0; d < 3; ++d) geo.k[d] = ctx->kpts[3 * (size_t)k + d];
    for (int i : list) {
      Site& s = ctx->sites[i];
      for (int d = 0; d < 3; ++d) geo.center[d] = s.center[d];
      const unsigned by = (unsigned)std::min(16, (nb + FFT_THREADS - 1) / FFT_THREADS);
      lagrange_kernel<T><<<dim3(s.npts, by), FFT_THREADS, 0, ctx->stream>>>(
          grid, nb, s.pts.ptr, geo, nocc, oofs, uofs, ctx->Ko, ctx->Ku, s.psi_o.ptr, s.psi_u.ptr);
      LRS_TRY(after_launch(ctx, "lagrange_kernel"));
    }
    oofs += nocc;
    uofs += nb - nocc;
  }
  return LRS_OK;
}

int project_fft(lrs_ctx* ctx, const std::vector<int>& list) {
  int n[3];
  LRS_TRY(fft_grid_dims(ctx, n));
  for (int d = 0; d < 3; ++d)
    if (!fft_length_ok(n[d])) return set_error(LRS_ERR_ARG, "FFT length %d is not 2^a 3^b <= %d", n[d], LRS_FFT_MAX_N);
  LRS_TRY(build_plan(ctx, n));
  if (ctx->precision == LRS_FP64) return project_fft_t<double>(ctx, list, n);
  return project_fft_t<float>(ctx, list, n);
}

}  // namespace lrs
