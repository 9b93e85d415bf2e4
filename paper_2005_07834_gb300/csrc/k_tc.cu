// Mixed-precision projection and chi0 on the tcgen05 tensor cores.
//
// Projection (Sec. VI.B method 1): psi_k = e^{ik.R}/sqrt(Omega) (P C_k) with
// the k-independent phase operand P(p, G) = e^{i G.R_p} and the coefficient
// operand C_k(G, b), both of modulus <= 1.  It is always computed with fp16
// hi/lo planes (11-bit significands, scaled by powers of two into the normal
// fp16 range), whose split residual is 2^-22.
//
// chi0 (Sec. VI.D, Eq. (chi1), single-grid quadrature of App. D.1): per
// frequency t_f the tensor cores form
//   Go(p,p')   = sum_v [conj psi_v(p) d_v] psi_v(p'),
//   Gu^T(p,p') = sum_c [psi_c(p) d_c] conj psi_c(p'),
// (A planes per frequency, B planes shared), the epilogue writes the fp32
// product X_f = Re[Go o Gu^T] of each frequency to its own slab, and the
// reduction forms chi0 = (2/pi) sum_f W_f (X_f + X_f^T) in float64.  The
// denominators d = w_k/(mu + i t - eps) are float64 (k_chi0_fp64.cu); the
// split is bf16 (LRS_MIXED_BF16X3) or scaled fp16 (LRS_MIXED_FP16X3).
#include <cmath>
#include <cstring>

#include "tc_gemm.cuh"

namespace lrs {

int make_operand_map(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
  // looked up once (a function-local static is initialised once even when contexts on several
  // host threads get here together)
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode) return set_error(LRS_ERR_CUDA, "cuTensorMapEncodeTiled not available from the driver");
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (cols * 2) % 16 != 0 || cols % 64 != 0 || rows % 128 != 0)
    return set_error(LRS_ERR_ARG, "operand map: misaligned base or shape (%llu x %llu)",
                     (unsigned long long)rows, (unsigned long long)cols);
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(LRS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return LRS_OK;
}

// ---------------------------------------------------------------- operand preparation
template <uint32_t FMT>
__device__ __forceinline__ void put_split(uint16_t* plane_row, int k, float x) {
  uint16_t h, l;
  split16<FMT>(x, h, l);
  const int col = (k >> 5) * 64 + (k & 31);
  plane_row[col] = h;
  plane_row[col + 32] = l;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned int* dst, float v) {
  atomicMax(dst, __float_as_uint(v));   // non-negative floats order like their bit patterns
}

// max |z| over a complex float64 array (result as float bits, pre-zeroed).
__global__ void max_abs_kernel(const double2* __restrict__ a, size_t n, unsigned int* __restrict__ out) {
  float m = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = a[i];
    m = fmaxf(m, (float)sqrt(v.x * v.x + v.y * v.y));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

// scales[f] for the A planes of frequency f (|conj psi d_f| <= max|psi| max|d_f|),
// scales[nf] for the B planes.  One block per frequency.
__global__ void chi0_scales_kernel(const double2* __restrict__ d_o, int Ko, const double2* __restrict__ d_u, int Ku,
                                   int nf, const unsigned int* __restrict__ psi_max_bits, float* __restrict__ scales) {
  const int f = blockIdx.x;
  float m = 0.f;
  for (int k = threadIdx.x; k < Ko + Ku; k += blockDim.x) {
    const double2 d = k < Ko ? d_o[(size_t)f * Ko + k] : d_u[(size_t)f * Ku + (k - Ko)];
    m = fmaxf(m, (float)sqrt(d.x * d.x + d.y * d.y));
  }
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    const float pm = __uint_as_float(*psi_max_bits);
    scales[f] = pow2_scale(pm * m);
    if (f == 0) scales[nf] = pow2_scale(pm);
  }
}

// B planes (frequency independent):  occupied columns psi, unoccupied conj(psi).
// A planes per frequency:            occupied conj(psi) d_f, unoccupied psi d_f.
// Planes: [2 (re, im)][rows][2*Kp] with rows = Np (B) or nf*Np (A).  `scales`
// (NULL = 1) multiplies the A planes of frequency f by scales[f] and the B
// planes by scales[nf].
// The denominators of the A planes in fp32, dtab[f][k] = d_f(k) scales[f] (0 on padded
// columns), formed once per launch: GB300 converts float64 at the FP64 rate, so converting them
// per grid point (N times) dominated the operand preparation.
__global__ void denom32_kernel(const double2* __restrict__ d_o, int Ko, const double2* __restrict__ d_u, int Ku,
                               int Kop, int Kp, int nf, const float* __restrict__ scales, float2* __restrict__ dtab) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (k >= Kp) return;
  const bool occ = k < Kop;
  const int kk = occ ? k : k - Kop;
  float2 v = make_float2(0.f, 0.f);
  if (occ ? kk < Ko : kk < Ku) {
    const double2 d = occ ? d_o[(size_t)f * Ko + kk] : d_u[(size_t)f * Ku + kk];
    const float sa = scales ? scales[f] : 1.f;
    v = make_float2((float)d.x * sa, (float)d.y * sa);
  }
  dtab[(size_t)f * Kp + k] = v;
}

template <uint32_t FMT>
__global__ void chi0_prep_kernel(const double2* __restrict__ psi_o, int Ko, const double2* __restrict__ psi_u,
                                 int Ku, int n, int Np, int Kop, int Kp, const float2* __restrict__ dtab, int nf,
                                 const float* __restrict__ scales, uint16_t* __restrict__ A, size_t aplane,
                                 uint16_t* __restrict__ B, size_t bplane) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (k >= Kp || p >= Np) return;
  const bool occ = k < Kop;
  const int kk = occ ? k : k - Kop;
  const bool live = p < n && (occ ? kk < Ko : kk < Ku);
  float xr = 0.f, xi = 0.f;
  if (live) {
    double2 v = occ ? psi_o[(size_t)p * Ko + kk] : psi_u[(size_t)p * Ku + kk];
    xr = (float)v.x;
    xi = (float)v.y;
  }
  const size_t ld = 2 * (size_t)Kp;
  const float sb = scales ? scales[nf] : 1.f;
  put_split<FMT>(B + (size_t)p * ld, k, sb * xr);
  put_split<FMT>(B + bplane + (size_t)p * ld, k, sb * (occ ? xi : -xi));
  const float cr = xr, ci = occ ? -xi : xi;   // conj for occupied
  for (int f = 0; f < nf; ++f) {
    float ar = 0.f, ai = 0.f;
    if (live) {
      const float2 d = dtab[(size_t)f * Kp + k];
      ar = cr * d.x - ci * d.y;
      ai = cr * d.y + ci * d.x;
    }
    const size_t row = (size_t)f * Np + p;
    put_split<FMT>(A + row * ld, k, ar);
    put_split<FMT>(A + aplane + row * ld, k, ai);
  }
}

// chi0 = (2/pi) sum_f W_f (X_f + X_f^T) / (scales[f] scales[nf])^2, float64 accumulation.
// The result is symmetric: one CTA per pair of 32 x 32 tiles (bi <= bj) reads tiles (bi, bj) and
// (bj, bi) of every frequency once, accumulates their symmetric sum once and writes both output
// tiles through shared memory (coalesced rows), so that each slab element is read once and each
// float64 accumulation is done once.  The slabs are in the chi0 kernel's layout (slab_index:
// 128-row bands stored as [column / 4][row][4]); thread (w, lane) reads row lane of a block as
// the float4 of columns 4 w .. 4 w + 3, so that a warp reads 512 consecutive bytes.  With sym,
// X_f is itself symmetric (real orbitals: both Green's functions are symmetric in r, r') and only
// the tiles reaching its lower triangle were computed: X_f + X_f^T = 2 X_f is read from the lower
// element of each pair (the tile (bj, bi), and within a diagonal tile whichever of the two
// elements lies on or below the diagonal), so that chi0 comes out exactly symmetric.
__global__ void __launch_bounds__(256) chi0_reduce_kernel(const float* __restrict__ slab, int Np, int nf,
                                                          const double* __restrict__ Wf,
                                                          const float* __restrict__ scales, int n, int sym,
                                                          double* __restrict__ chi0) {
  constexpr int FB = 4;          // frequencies per pair of barriers: all their tiles in flight at once
  __shared__ float tb[FB][32][33];   // tb[h][a][b] = X_f(c0 + b, r0 + a) of frequency f + h
  __shared__ double o[32][33];
  __shared__ double wsm[128];   // per-frequency weights W_f / (scales[f] scales[nf])^2 (x 2 with sym)
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bi > bj) return;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8: lane, and the column group of 4
  const int tid = ty * 32 + tx;
  const int r0 = bi * 32, c0 = bj * 32;
  for (int f = tid; f < nf; f += 256) {
    double w = Wf[f];
    if (scales) {
      const double sc = (double)scales[f] * (double)scales[nf];
      w /= sc * sc;
    }
    wsm[f] = sym ? 2.0 * w : w;
  }
  // this thread's outputs: row R = r0 + tx, columns q = c0 + 4 ty + j
  const bool need_direct = !(sym && bi != bj);
  const size_t off_direct = slab_index(Np, r0 + tx, c0 + 4 * ty);
  const size_t off_trans = slab_index(Np, c0 + tx, r0 + 4 * ty);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int f = 0; f < nf; f += FB) {
    const int nb = min(FB, nf - f);
    float4 direct[FB];
#pragma unroll
    for (int h = 0; h < FB; ++h) {
      if (h >= nb) break;
      const float* s = slab + (size_t)(f + h) * Np * Np;
      const float4 tv = *reinterpret_cast<const float4*>(s + off_trans);   // X(c0 + tx, r0 + 4 ty + j)
      tb[h][4 * ty + 0][tx] = tv.x;
      tb[h][4 * ty + 1][tx] = tv.y;
      tb[h][4 * ty + 2][tx] = tv.z;
      tb[h][4 * ty + 3][tx] = tv.w;
      direct[h] = need_direct ? *reinterpret_cast<const float4*>(s + off_direct) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < FB; ++h) {
      if (h >= nb) break;
      const double w = wsm[f + h];
      const float d[4] = {direct[h].x, direct[h].y, direct[h].z, direct[h].w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        // output (R, q) = (r0 + tx, c0 + 4 ty + j): tb holds X_f(q, R), d X_f(R, q)
        const float tq = tb[h][tx][4 * ty + j];
        const float v = sym ? ((c0 + 4 * ty + j >= r0 + tx) ? tq : d[j]) : d[j] + tq;
        acc[j] = fma(w, f32_to_f64_exact(v), acc[j]);
      }
    }
    __syncthreads();
  }
  const double c = 0.63661977236758134308;   // 2/pi
#pragma unroll
  for (int j = 0; j < 4; ++j) o[tx][4 * ty + j] = c * acc[j];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty + 8 * i, q = c0 + tx;
    if (r < n && q < n) chi0[(size_t)r * n + q] = o[ty + 8 * i][tx];
  }
  if (bi == bj) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = c0 + ty + 8 * i, q = r0 + tx;   // output tile (bj, bi): element (q', r') of o transposed
    if (r < n && q < n) chi0[(size_t)r * n + q] = o[tx][ty + 8 * i];
  }
}

// Projection B operand: C_k(G, b) * scale -> planes [2][nk*nbp][2*NGp] (rows = k*nbp + b, K = G).
template <uint32_t FMT>
__global__ void coeff_prep_kernel(const double2* __restrict__ coeff, int ng, int nb, int NGp, int nbp,
                                  const float* __restrict__ scale, uint16_t* __restrict__ B, size_t im_off) {
  __shared__ float2 t[32][33];
  const int k = blockIdx.z;
  const int g0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  const float sc = *scale;
  for (int i = ty; i < 32; i += 8) {
    const int g = g0 + i, b = b0 + tx;
    float2 v = make_float2(0.f, 0.f);
    if (g < ng && b < nb) {
      const double2 c = coeff[((size_t)k * ng + g) * nb + b];
      v = make_float2((float)c.x * sc, (float)c.y * sc);
    }
    t[i][tx] = v;
  }
  __syncthreads();
  const size_t ld = 2 * (size_t)NGp;
  for (int i = ty; i < 32; i += 8) {
    const int b = b0 + i, g = g0 + tx;
    if (b >= nbp || g >= NGp) continue;
    const float2 v = t[tx][i];
    uint16_t* row = B + ((size_t)k * nbp + b) * ld;
    put_split<FMT>(row, g, v.x);
    put_split<FMT>(row + im_off, g, v.y);
  }
}

// The phase tables in fp32 (converted once: GB300 converts float64 at the FP64 rate).
__global__ void tab32_kernel(const double2* __restrict__ tab, size_t n, float2* __restrict__ out) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float2((float)tab[i].x, (float)tab[i].y);
}

// Projection A operand: e^{i G.R_p} = T1 T2 T3 (times `scale`) -> planes [2][Np][2*NGp].
template <uint32_t FMT>
__global__ void phase_prep_kernel(const float2* __restrict__ tab, int npts, int3 nmax, int off1, int off2,
                                  const int* __restrict__ gvec, int ng, int Np, int NGp, float scale,
                                  uint16_t* __restrict__ A, size_t im_off) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (g >= NGp || p >= Np) return;
  float re = 0.f, im = 0.f;
  if (g < ng && p < npts) {
    const int w1 = 2 * nmax.x + 1, w2 = 2 * nmax.y + 1, w3 = 2 * nmax.z + 1;
    const float2 t1 = tab[(size_t)p * w1 + gvec[3 * g] + nmax.x];
    const float2 t2 = tab[off1 + (size_t)p * w2 + gvec[3 * g + 1] + nmax.y];
    const float2 t3 = tab[off2 + (size_t)p * w3 + gvec[3 * g + 2] + nmax.z];
    const float ar = t1.x, ai = t1.y, br = t2.x, bi = t2.y;
    const float cr = ar * br - ai * bi, ci = ar * bi + ai * br;
    const float dr = t3.x, di = t3.y;
    re = (cr * dr - ci * di) * scale;
    im = (cr * di + ci * dr) * scale;
  }
  uint16_t* row = A + (size_t)p * 2 * NGp;
  put_split<FMT>(row, g, re);
  put_split<FMT>(row + im_off, g, im);
}

// unscale = 1 / (phase_scale * coefficient scale), the coefficient scale from max |C|.
__global__ void coeff_scale_kernel(const unsigned int* __restrict__ cmax_bits, float phase_scale,
                                   float* __restrict__ scale, float* __restrict__ unscale) {
  const float s = pow2_scale(__uint_as_float(*cmax_bits));
  *scale = s;
  *unscale = 1.f / (s * phase_scale);
}

static inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

constexpr int CHI0_TN = 128;   // chi0 tile columns
constexpr int PROJ_TN = 128;   // projection tile columns

int phase_setup(lrs_ctx* ctx, Site& s, int* off1, int* off2);

// chi0 of several sites in one persistent tensor-core launch.  The operand
// planes of all sites are stacked (A: [2][sum_s nf Np_s][2Kp], B: [2][sum_s
// Np_s][2Kp]) so that one pair of tensor maps covers every unit; a site table
// maps the global unit index to (site, tile, tile, frequency).
template <uint32_t FMT, int TN>
static int chi0_mixed_t(lrs_ctx* ctx, const std::vector<int>& list, int toff) {
  const int nf = ctx->nf;
  const int Kop = round_up(ctx->Ko, 32), Kup = round_up(ctx->Ku, 32), Kp = Kop + Kup;
  const size_t ld = 2 * (size_t)Kp;
  const int ns = (int)list.size();
  // Gamma-point real orbitals: B = [psi_o | conj psi_u] is real, both Green's functions are
  // symmetric in (r, r'), and so is each frequency's product: only the tiles that reach the
  // lower triangle are computed
  const bool real = ctx->real_orbitals && ctx->real_mode == LRS_REAL_AUTO;
  std::vector<SiteTile> table(ns);
  long long ra = 0, rb = 0, slab = 0, units = 0;
  for (int i = 0; i < ns; ++i) {
    const int np = round_up(ctx->sites[list[i]].npts, TILE_M);
    SiteTile& t = table[i];
    t.unit0 = (int)units;
    t.m_tiles = np / TILE_M;
    t.n_tiles = np / TN;
    t.ldc = np;
    t.m_valid = np;
    t.n_valid = np;
    t.np = np;
    t.a_row0 = (int)ra;
    t.b_row0 = (int)rb;
    t.slab0 = slab;
    const long long q = TILE_M / TN;
    units += (real ? q * t.m_tiles * (t.m_tiles + 1) / 2 : (long long)t.m_tiles * t.n_tiles) * nf;
    ra += (long long)nf * np;
    rb += np;
    slab += (long long)nf * np * np;
  }
  if (2 * ra > INT32_MAX || units > INT32_MAX) return set_error(LRS_ERR_ARG, "too many sites for one launch");
  LRS_TRY(ensure(ctx, ctx->ws.planes_a, 2 * (size_t)ra * ld));
  LRS_TRY(ensure(ctx, ctx->ws.planes_b, 2 * (size_t)rb * ld));
  LRS_TRY(ensure(ctx, ctx->ws.slab, (size_t)slab));
  LRS_TRY(ensure(ctx, ctx->ws.site_tiles, (size_t)toff + ns));
  LRS_TRY(ensure(ctx, ctx->ws.tc_scratch, (size_t)ctx->num_sms * 2 * TILE_M * TN));
  const size_t sstride = (size_t)nf + 8;    // fp16 operand scales of one site
  if (FMT == 0) LRS_TRY(ensure(ctx, ctx->ws.scales, sstride * ns));
  // the unit table goes to the device only when it changes (never while a graph is recorded)
  if (ctx->site_tiles_dev_ptr != ctx->ws.site_tiles.ptr) ctx->site_tiles_dev.clear();   // buffer was replaced
  const bool same = ctx->site_tiles_dev.size() >= (size_t)toff + ns &&
                    std::memcmp(ctx->site_tiles_dev.data() + toff, table.data(), ns * sizeof(SiteTile)) == 0;
  if (!same) {
    if (ctx->capturing) return set_error(LRS_ERR_STATE, "site table changed during graph capture");
    drop_graph(ctx);   // a recorded build reads this table
    LRS_CUDA_TRY(cudaMemcpyAsync(ctx->ws.site_tiles.ptr + toff, table.data(), ns * sizeof(SiteTile),
                                 cudaMemcpyHostToDevice, ctx->stream));
    LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (ctx->site_tiles_dev.size() < (size_t)toff + ns) ctx->site_tiles_dev.resize((size_t)toff + ns);
    std::memcpy(ctx->site_tiles_dev.data() + toff, table.data(), ns * sizeof(SiteTile));
    ctx->site_tiles_dev_ptr = ctx->ws.site_tiles.ptr;
  }
  for (int i = 0; i < ns; ++i) {
    Site& s = ctx->sites[list[i]];
    const SiteTile& t = table[i];
    const int n = s.npts;
    float* scales = nullptr;
    if (FMT == 0) {
      scales = ctx->ws.scales.ptr + sstride * i;
      unsigned int* pmax = reinterpret_cast<unsigned int*>(scales + nf + 4);
      LRS_CUDA_TRY(cudaMemsetAsync(pmax, 0, sizeof(unsigned int), ctx->stream));
      max_abs_kernel<<<ctx->num_sms * 4, 256, 0, ctx->stream>>>(s.psi_o.ptr, (size_t)n * ctx->Ko, pmax);
      LRS_TRY(after_launch(ctx, "max_abs_kernel"));
      max_abs_kernel<<<ctx->num_sms * 4, 256, 0, ctx->stream>>>(s.psi_u.ptr, (size_t)n * ctx->Ku, pmax);
      LRS_TRY(after_launch(ctx, "max_abs_kernel"));
      chi0_scales_kernel<<<nf, 256, 0, ctx->stream>>>(ctx->ws.denom_o.ptr, ctx->Ko, ctx->ws.denom_u.ptr, ctx->Ku,
                                                       nf, pmax, scales);
      LRS_TRY(after_launch(ctx, "chi0_scales_kernel"));
    }
    LRS_TRY(ensure(ctx, ctx->ws.denom32, (size_t)nf * Kp));
    denom32_kernel<<<dim3((Kp + 255) / 256, nf), 256, 0, ctx->stream>>>(
        ctx->ws.denom_o.ptr, ctx->Ko, ctx->ws.denom_u.ptr, ctx->Ku, Kop, Kp, nf, scales, ctx->ws.denom32.ptr);
    LRS_TRY(after_launch(ctx, "denom32_kernel"));
    dim3 pg((Kp + 127) / 128, t.np);
    chi0_prep_kernel<FMT><<<pg, 128, 0, ctx->stream>>>(
        s.psi_o.ptr, ctx->Ko, s.psi_u.ptr, ctx->Ku, n, t.np, Kop, Kp, ctx->ws.denom32.ptr, nf, scales,
        ctx->ws.planes_a.ptr + (size_t)t.a_row0 * ld, (size_t)ra * ld, ctx->ws.planes_b.ptr + (size_t)t.b_row0 * ld,
        (size_t)rb * ld);
    LRS_TRY(after_launch(ctx, "chi0_prep_kernel"));
  }
  CUtensorMap ma, mb;
  LRS_TRY(make_operand_map(&ma, ctx->ws.planes_a.ptr, ld, 2 * (uint64_t)ra, TILE_M));
  LRS_TRY(make_operand_map(&mb, ctx->ws.planes_b.ptr, ld, 2 * (uint64_t)rb, TN));
  TcShape sh{};
  sh.batches = nf;
  sh.nchunk = Kp / 32;
  sh.nchunk0 = Kop / 32;
  sh.seg = ctx->seg_chunks;
  sh.a_im_rows = (int)ra;
  sh.b_im_rows = (int)rb;
  sh.units = (int)units;
  sh.sites = ctx->ws.site_tiles.ptr + toff;
  sh.nsites = ns;
  sh.real_b = real ? 1 : 0;
  sh.tri = real ? 1 : 0;
  // short K (each contraction at most two accumulation segments long): both contractions of a
  // unit accumulate whole in their own TMEM set and the epilogue multiplies them straight from
  // TMEM, with no folding of segments and no parking of the occupied sums
  const bool direct = sh.nchunk0 <= 2 * sh.seg && sh.nchunk - sh.nchunk0 <= 2 * sh.seg;
  Chi0Store epi{ctx->ws.slab.ptr, ctx->ws.tc_scratch.ptr, 0, TN};
  LRS_TRY(stage_begin(ctx, ST_CHI0_MAIN));
  if (direct) LRS_TRY((launch_tc<TN, 2, FMT, Chi0Store, true>(ctx, ma, mb, sh, epi, "zgemm_tc_kernel<chi0, short K>")));
  else LRS_TRY((launch_tc<TN, 2, FMT, Chi0Store>(ctx, ma, mb, sh, epi, "zgemm_tc_kernel<chi0>")));
  LRS_TRY(stage_end(ctx, ST_CHI0_MAIN));
  for (int i = 0; i < ns; ++i) {
    Site& s = ctx->sites[list[i]];
    const SiteTile& t = table[i];
    dim3 rg(t.np / 32, t.np / 32);
    chi0_reduce_kernel<<<rg, dim3(32, 8), 0, ctx->stream>>>(ctx->ws.slab.ptr + t.slab0, t.np, nf, ctx->d_W.ptr,
                                                            FMT == 0 ? ctx->ws.scales.ptr + sstride * i : nullptr,
                                                            s.npts, real ? 1 : 0, s.chi0.ptr);
    LRS_TRY(after_launch(ctx, "chi0_reduce_kernel"));
  }
  return LRS_OK;
}

int chi0_mixed(lrs_ctx* ctx, const std::vector<int>& list, int toff) {
  const bool fp16 = ctx->precision == LRS_MIXED_FP16X3;
  if (ctx->chi0_tn == 64) return fp16 ? chi0_mixed_t<0, 64>(ctx, list, toff) : chi0_mixed_t<1, 64>(ctx, list, toff);
  return fp16 ? chi0_mixed_t<0, 128>(ctx, list, toff) : chi0_mixed_t<1, 128>(ctx, list, toff);
}

int project_mixed(lrs_ctx* ctx, Site& s) {
  constexpr uint32_t FMT = 0;               // fp16 hi/lo: operands are bounded by 1
  constexpr float PHASE_SCALE = 16384.f;    // |e^{iG.R}| = 1
  if (ctx->nk > MAX_K_POINTS)
    return set_error(LRS_ERR_UNSUPPORTED, "mixed projection supports at most %d k-points", MAX_K_POINTS);
  const int n = s.npts;
  const int Np = round_up(n, TILE_M);
  const int NGp = round_up(ctx->ng, 32);
  const int nbp = round_up(ctx->nb, PROJ_TN);
  const size_t ld = 2 * (size_t)NGp;
  LRS_TRY(ensure(ctx, ctx->ws.proj_scale, 4));
  float* cscale = ctx->ws.proj_scale.ptr;      // [0] coefficient scale, [1] unscale, [2] max bits
  // coefficient planes depend only on the orbitals: rebuilt when they change
  const size_t bsz = 2 * (size_t)ctx->nk * nbp * ld;
  if (!ctx->ws.coeff_planes_valid || ctx->ws.proj_b.count < bsz) {
    LRS_TRY(ensure(ctx, ctx->ws.proj_b, bsz));
    unsigned int* cmax = reinterpret_cast<unsigned int*>(cscale + 2);
    LRS_CUDA_TRY(cudaMemsetAsync(cmax, 0, sizeof(unsigned int), ctx->stream));
    max_abs_kernel<<<ctx->num_sms * 4, 256, 0, ctx->stream>>>(ctx->coeff.ptr, (size_t)ctx->nk * ctx->ng * ctx->nb,
                                                               cmax);
    LRS_TRY(after_launch(ctx, "max_abs_kernel"));
    coeff_scale_kernel<<<1, 1, 0, ctx->stream>>>(cmax, PHASE_SCALE, cscale, cscale + 1);
    LRS_TRY(after_launch(ctx, "coeff_scale_kernel"));
    dim3 cg((NGp + 31) / 32, (nbp + 31) / 32, ctx->nk);
    coeff_prep_kernel<FMT><<<cg, dim3(32, 8), 0, ctx->stream>>>(ctx->coeff.ptr, ctx->ng, ctx->nb, NGp, nbp, cscale,
                                                                  ctx->ws.proj_b.ptr, (size_t)ctx->nk * nbp * ld);
    LRS_TRY(after_launch(ctx, "coeff_prep_kernel"));
    ctx->ws.coeff_planes_valid = true;
  }
  int off1, off2;
  LRS_TRY(phase_setup(ctx, s, &off1, &off2));
  LRS_TRY(ensure(ctx, ctx->ws.proj_a, 2 * (size_t)Np * ld));
  const int* nm = ctx->gmax_idx;
  const size_t n_tab = (size_t)n * ((2 * nm[0] + 1) + (2 * nm[1] + 1) + (2 * nm[2] + 1));
  LRS_TRY(ensure(ctx, ctx->ws.phase_tab32, n_tab));
  tab32_kernel<<<(unsigned)((n_tab + 255) / 256), 256, 0, ctx->stream>>>(ctx->ws.phase_tab.ptr, n_tab,
                                                                          ctx->ws.phase_tab32.ptr);
  LRS_TRY(after_launch(ctx, "tab32_kernel"));
  dim3 pg((NGp + 127) / 128, Np);
  phase_prep_kernel<FMT><<<pg, 128, 0, ctx->stream>>>(ctx->ws.phase_tab32.ptr, n, make_int3(nm[0], nm[1], nm[2]),
                                                       off1, off2, ctx->d_gvec.ptr, ctx->ng, Np, NGp, PHASE_SCALE,
                                                       ctx->ws.proj_a.ptr, (size_t)Np * ld);
  LRS_TRY(after_launch(ctx, "phase_prep_kernel"));
  CUtensorMap ma, mb;
  LRS_TRY(make_operand_map(&ma, ctx->ws.proj_a.ptr, ld, 2 * (uint64_t)Np, TILE_M));
  LRS_TRY(make_operand_map(&mb, ctx->ws.proj_b.ptr, ld, 2 * (uint64_t)ctx->nk * nbp, PROJ_TN));
  TcShape sh{};
  sh.m_tiles = Np / TILE_M;
  sh.n_tiles = nbp / PROJ_TN;
  sh.batches = ctx->nk;
  sh.nchunk = NGp / 32;
  sh.nchunk0 = sh.nchunk;
  sh.seg = ctx->proj_seg_chunks;
  sh.a_batch_rows = 0;
  sh.b_batch_rows = nbp;
  sh.a_im_rows = Np;
  sh.b_im_rows = ctx->nk * nbp;
  sh.units = sh.m_tiles * sh.n_tiles * sh.batches;
  sh.sites = nullptr;
  sh.nsites = 0;
  ProjStore epi;
  epi.kph = ctx->ws.kphase.ptr;
  epi.unscale = cscale + 1;
  epi.npts = n;
  epi.nb = ctx->nb;
  epi.psi_o = s.psi_o.ptr;
  epi.psi_u = s.psi_u.ptr;
  epi.Ko = ctx->Ko;
  epi.Ku = ctx->Ku;
  int oo = 0, uo = 0;
  for (int k = 0; k < ctx->nk; ++k) {
    epi.nocc[k] = ctx->nocc[k];
    epi.oofs[k] = oo;
    epi.uofs[k] = uo;
    oo += ctx->nocc[k];
    uo += ctx->nb - ctx->nocc[k];
  }
  return launch_tc<PROJ_TN, 1, FMT, ProjStore>(ctx, ma, mb, sh, epi, "zgemm_tc_kernel<project>");
}

}  // namespace lrs

// ============================================================================
// Adjoint on the tensor cores (mixed precisions).  Same mathematics as the
// float64 adjoint (k_adjoint.cu): per frequency the Green's functions are
// recomputed with the chi0 operand planes and stored as fp32 (GStore), then
//   Ho = W_f G_S o Gu^T,  Hu = W_f G_S o Go   (bf16 hi/lo planes, and their transposes)
//   Yo = Ho psi_o, Zo = Ho^T conj psi_o, Yu = Hu conj psi_u, Zu = Hu^T psi_u
// run as one tensor-core launch with four problems (ZStore), and the
// gradients accumulate over frequencies in float64.
// ============================================================================
namespace lrs {

// Transposed orbital planes for the B operand of the Y/Z products.  Rows:
// [psi_o^T | conj psi_o^T | conj psi_u^T | psi_u^T] (band rows, padded to
// 128 per block), K = grid point.  blockIdx.z: 0 occupied, 1 unoccupied.
__global__ void psiT_prep_kernel(const double2* __restrict__ psi_o, int Ko, const double2* __restrict__ psi_u,
                                 int Ku, int n, int Np, int Ko128, int Ku128, uint16_t* __restrict__ T,
                                 size_t im_off) {
  __shared__ float2 tile[32][33];
  const bool occ = blockIdx.z == 0;
  const int Kx = occ ? Ko : Ku, Kx128 = occ ? Ko128 : Ku128;
  const double2* psi = occ ? psi_o : psi_u;
  const int p0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  if (b0 >= Kx128) return;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int i = ty; i < 32; i += 8) {
    const int p = p0 + i, b = b0 + tx;
    float2 v = make_float2(0.f, 0.f);
    if (p < n && b < Kx) {
      const double2 d = psi[(size_t)p * Kx + b];
      v = make_float2((float)d.x, (float)d.y);
    }
    tile[i][tx] = v;
  }
  __syncthreads();
  const size_t ld = 2 * (size_t)Np;
  const int rplain = occ ? 0 : 2 * Ko128 + Ku128;
  const int rconj = occ ? Ko128 : 2 * Ko128;
  for (int i = ty; i < 32; i += 8) {
    const int b = b0 + i, p = p0 + tx;
    if (p >= Np) continue;
    const float2 v = tile[tx][i];
    uint16_t* rp = T + (size_t)(rplain + b) * ld;
    uint16_t* rc = T + (size_t)(rconj + b) * ld;
    put_split<1>(rp, p, v.x);
    put_split<1>(rp + im_off, p, v.y);
    put_split<1>(rc, p, v.x);
    put_split<1>(rc + im_off, p, -v.y);
  }
}

// H planes for one frequency: rows [Ho | Ho^T | Hu | Hu^T] (Np each), K = grid point.
__global__ void hprep_kernel(const float2* __restrict__ go, const float2* __restrict__ gu,
                             const double* __restrict__ gs, int n, int Np, double wf, uint16_t* __restrict__ H,
                             size_t im_off) {
  __shared__ float2 to[32][33], tu[32][33];
  const int q0 = blockIdx.x * 32, p0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  const size_t ld = 2 * (size_t)Np;
  for (int i = ty; i < 32; i += 8) {
    const int p = p0 + i, q = q0 + tx;
    float2 ho = make_float2(0.f, 0.f), hu = make_float2(0.f, 0.f);
    if (p < n && q < n) {
      const float g = (float)(wf * gs[(size_t)p * n + q]);
      const float2 a = go[(size_t)p * Np + q], b = gu[(size_t)p * Np + q];
      ho = make_float2(g * b.x, g * b.y);
      hu = make_float2(g * a.x, g * a.y);
    }
    to[i][tx] = ho;
    tu[i][tx] = hu;
    uint16_t* r0 = H + (size_t)p * ld;                    // Ho row p, K = q
    uint16_t* r2 = H + (size_t)(2 * Np + p) * ld;         // Hu row p
    put_split<1>(r0, q, ho.x);
    put_split<1>(r0 + im_off, q, ho.y);
    put_split<1>(r2, q, hu.x);
    put_split<1>(r2 + im_off, q, hu.y);
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int q = q0 + i, p = p0 + tx;                    // transposed: row q, K = p
    const float2 ho = to[tx][i], hu = tu[tx][i];
    uint16_t* r1 = H + (size_t)(Np + q) * ld;
    uint16_t* r3 = H + (size_t)(3 * Np + q) * ld;
    put_split<1>(r1, p, ho.x);
    put_split<1>(r1 + im_off, p, ho.y);
    put_split<1>(r3, p, hu.x);
    put_split<1>(r3 + im_off, p, hu.y);
  }
}

// psi (float64 complex) -> fp32 complex, once per adjoint.
__global__ void psi_to_f32_kernel(const double2* __restrict__ psi, size_t count, float2* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = psi[i];
    out[i] = make_float2((float)v.x, (float)v.y);
  }
}

// Same update as the float64 adjoint's grad_accum_kernel, from fp32 Y, Z.
constexpr int GA32_ROWS = 256;
template <bool kOcc>
__global__ void __launch_bounds__(256) grad_accum32_kernel(const float2* __restrict__ psi,
                                                           const float2* __restrict__ Y,
                                                           const float2* __restrict__ Z,
                                                           const double2* __restrict__ d, int n, int K,
                                                           double2* __restrict__ gpsi, double2* __restrict__ part) {
  // 32 columns per CTA (one per lane: coalesced rows), GA32_ROWS rows in eight row groups.
  // The products with d and psi are formed in fp32 (Y and Z are fp32 tensor-core results);
  // each element's contribution is added to the float64 gradient once per frequency, and the
  // column sums of the energy gradient leave the CTA as float64 partial sums.  psi arrives as
  // fp32 (converted once per adjoint) and the fp32 terms are widened with integer instructions:
  // GB300 converts between fp32 and float64 on its float64 pipe, which the sums already use.
  __shared__ double2 red[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int b = blockIdx.x * 32 + tx;
  const int p0 = blockIdx.y * GA32_ROWS;
  float er = 0.f, ei = 0.f;
  if (b < K) {
    const double2 dd = d[b];
    const float dx = (float)dd.x, dy = (float)dd.y;
    const int p1 = min(n, p0 + GA32_ROWS);
    for (int p = p0 + ty; p < p1; p += 8) {
      const size_t ix = (size_t)p * K + b;
      const float2 y = Y[ix], z = Z[ix];
      const float2 ps = psi[ix];
      const float sx = y.x + z.x, sy = y.y + z.y;                       // y + z
      const float tx_ = kOcc ? y.x - z.x : z.x - y.x, ty_ = kOcc ? y.y - z.y : z.y - y.y;
      double2 g = gpsi[ix];
      g.x += f32_to_f64_exact(fmaf(dx, sx, -dy * sy));                 // Re d (y + z)
      g.y += f32_to_f64_exact(fmaf(dx, ty_, dy * tx_));                // Im d (y -+ z)
      gpsi[ix] = g;
      const float px = ps.x, py = ps.y;
      if (kOcc) {                                                       // conj(psi) y
        er += fmaf(px, y.x, py * y.y);
        ei += fmaf(px, y.y, -py * y.x);
      } else {                                                          // psi y
        er += fmaf(px, y.x, -py * y.y);
        ei += fmaf(px, y.y, py * y.x);
      }
    }
  }
  red[ty][tx] = make_double2((double)er, (double)ei);
  __syncthreads();
  if (ty == 0 && b < K) {
    double2 s = red[0][tx];
    for (int r = 1; r < 8; ++r) { s.x += red[r][tx].x; s.y += red[r][tx].y; }
    part[(size_t)blockIdx.y * K + b] = s;
  }
}

int backward_site_mixed(lrs_ctx* ctx, Site& s, const double* grad_w, const double* grad_chi0, double* grad_e,
                        double2* grad_psi) {
  const int n = s.npts, nf = ctx->nf, Ko = ctx->Ko, Ku = ctx->Ku, K = Ko + Ku;
  const int Np = round_up(n, TILE_M);
  const int Kop = round_up(Ko, 32), Kup = round_up(Ku, 32), Kp = Kop + Kup;
  const int Ko128 = round_up(Ko, 128), Ku128 = round_up(Ku, 128);
  const int RB = 2 * Ko128 + 2 * Ku128;
  const size_t ldg = 2 * (size_t)Kp, ldn = 2 * (size_t)Np;
  Workspace& ws = ctx->ws;
  if (ctx->capturing) return set_error(LRS_ERR_STATE, "the adjoint cannot be recorded in a graph");
  LRS_TRY(build_denominators(ctx));
  LRS_TRY(gamma_s_build(ctx, s, grad_w, grad_chi0));
  LRS_TRY(ensure(ctx, ws.planes_a, 2 * (size_t)nf * Np * ldg));
  LRS_TRY(ensure(ctx, ws.planes_b, 2 * (size_t)Np * ldg));
  LRS_TRY(ensure(ctx, ws.planes_t, 2 * (size_t)RB * ldn));
  LRS_TRY(ensure(ctx, ws.planes_h, 2 * (size_t)4 * Np * ldn));
  LRS_TRY(ensure(ctx, ws.g32, 2 * (size_t)Np * Np));
  LRS_TRY(ensure(ctx, ws.yz32, 2 * (size_t)n * K));
  LRS_TRY(ensure(ctx, ws.gpsi, (size_t)n * K));
  LRS_TRY(ensure(ctx, ws.psi32, (size_t)n * K));
  LRS_TRY(ensure(ctx, ws.ge, (size_t)K));
  const int chunks = (n + GA32_ROWS - 1) / GA32_ROWS;
  LRS_TRY(ensure(ctx, ws.gpart, (size_t)chunks * K));
  LRS_TRY(ensure(ctx, ws.tc_scratch, (size_t)ctx->num_sms * 2 * TILE_M * 128));
  LRS_TRY(ensure(ctx, ws.adj_tiles, (size_t)nf + 4));
  LRS_CUDA_TRY(cudaMemsetAsync(ws.gpsi.ptr, 0, (size_t)n * K * sizeof(double2), ctx->stream));
  float2* psi32_o = ws.psi32.ptr;
  float2* psi32_u = ws.psi32.ptr + (size_t)n * Ko;
  psi_to_f32_kernel<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(s.psi_o.ptr, (size_t)n * Ko, psi32_o);
  LRS_TRY(after_launch(ctx, "psi_to_f32_kernel"));
  psi_to_f32_kernel<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(s.psi_u.ptr, (size_t)n * Ku, psi32_u);
  LRS_TRY(after_launch(ctx, "psi_to_f32_kernel"));
  LRS_CUDA_TRY(cudaMemsetAsync(ws.ge.ptr, 0, (size_t)K * sizeof(double), ctx->stream));
  // operands of the Green's functions (all frequencies) and of the Y/Z products
  LRS_TRY(ensure(ctx, ws.denom32, (size_t)nf * Kp));
  denom32_kernel<<<dim3((Kp + 255) / 256, nf), 256, 0, ctx->stream>>>(ws.denom_o.ptr, Ko, ws.denom_u.ptr, Ku, Kop,
                                                                       Kp, nf, nullptr, ws.denom32.ptr);
  LRS_TRY(after_launch(ctx, "denom32_kernel"));
  dim3 pg((Kp + 127) / 128, Np);
  chi0_prep_kernel<1><<<pg, 128, 0, ctx->stream>>>(s.psi_o.ptr, Ko, s.psi_u.ptr, Ku, n, Np, Kop, Kp,
                                                    ws.denom32.ptr, nf, nullptr, ws.planes_a.ptr,
                                                    (size_t)nf * Np * ldg, ws.planes_b.ptr, (size_t)Np * ldg);
  LRS_TRY(after_launch(ctx, "chi0_prep_kernel"));
  dim3 tg(Np / 32, std::max(Ko128, Ku128) / 32, 2);
  psiT_prep_kernel<<<tg, dim3(32, 8), 0, ctx->stream>>>(s.psi_o.ptr, Ko, s.psi_u.ptr, Ku, n, Np, Ko128, Ku128,
                                                        ws.planes_t.ptr, (size_t)RB * ldn);
  LRS_TRY(after_launch(ctx, "psiT_prep_kernel"));
  // unit tables: nf single-frequency Green's-function problems, then the four Y/Z products
  std::vector<SiteTile> tbl(nf + 4);
  for (int f = 0; f < nf; ++f) {
    SiteTile& t = tbl[f];
    t.unit0 = 0;
    t.m_tiles = Np / TILE_M;
    t.n_tiles = Np / 128;
    t.np = Np;
    t.a_row0 = f * Np;
    t.b_row0 = 0;
    t.slab0 = 0;
    t.ldc = Np;
    t.m_valid = Np;
    t.n_valid = Np;
  }
  const int kx[4] = {Ko, Ko, Ku, Ku}, kx128[4] = {Ko128, Ko128, Ku128, Ku128};
  const int brow[4] = {0, Ko128, 2 * Ko128, 2 * Ko128 + Ku128};
  const long long yoff[4] = {0, (long long)n * Ko, 2LL * n * Ko, 2LL * n * Ko + (long long)n * Ku};
  int units = 0;
  for (int j = 0; j < 4; ++j) {
    SiteTile& t = tbl[nf + j];
    t.unit0 = units;
    t.m_tiles = Np / TILE_M;
    t.n_tiles = kx128[j] / 128;
    t.np = Np;
    t.a_row0 = j * Np;
    t.b_row0 = brow[j];
    t.slab0 = yoff[j];
    t.ldc = kx[j];
    t.m_valid = n;
    t.n_valid = kx[j];
    units += t.m_tiles * t.n_tiles;
  }
  LRS_CUDA_TRY(cudaMemcpyAsync(ws.adj_tiles.ptr, tbl.data(), tbl.size() * sizeof(SiteTile), cudaMemcpyHostToDevice,
                               ctx->stream));
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  CUtensorMap ma_g, mb_g, ma_h, mb_t;
  LRS_TRY(make_operand_map(&ma_g, ws.planes_a.ptr, ldg, 2 * (uint64_t)nf * Np, TILE_M));
  LRS_TRY(make_operand_map(&mb_g, ws.planes_b.ptr, ldg, 2 * (uint64_t)Np, 128));
  LRS_TRY(make_operand_map(&ma_h, ws.planes_h.ptr, ldn, 2 * (uint64_t)4 * Np, TILE_M));
  LRS_TRY(make_operand_map(&mb_t, ws.planes_t.ptr, ldn, 2 * (uint64_t)RB, 128));
  float2* go = ws.g32.ptr;
  float2* gu = ws.g32.ptr + (size_t)Np * Np;
  float2* Y = ws.yz32.ptr;
  GStore gst{go, gu, ws.tc_scratch.ptr, 128};
  ZStore zst{Y};
  for (int f = 0; f < nf; ++f) {
    TcShape sg{};
    sg.batches = 1;
    sg.nchunk = Kp / 32;
    sg.nchunk0 = Kop / 32;
    sg.seg = ctx->seg_chunks;
    sg.a_im_rows = nf * Np;
    sg.b_im_rows = Np;
    sg.units = (Np / TILE_M) * (Np / 128);
    sg.sites = ws.adj_tiles.ptr + f;
    sg.nsites = 1;
    LRS_TRY((launch_tc<128, 2, 1, GStore>(ctx, ma_g, mb_g, sg, gst, "zgemm_tc_kernel<green>")));
    dim3 hg(Np / 32, Np / 32);
    hprep_kernel<<<hg, dim3(32, 8), 0, ctx->stream>>>(go, gu, ws.gamma_s.ptr, n, Np, ctx->W[f], ws.planes_h.ptr,
                                                      (size_t)4 * Np * ldn);
    LRS_TRY(after_launch(ctx, "hprep_kernel"));
    TcShape sy{};
    sy.batches = 1;
    sy.nchunk = Np / 32;
    sy.nchunk0 = sy.nchunk;
    sy.seg = ctx->seg_chunks;
    sy.a_im_rows = 4 * Np;
    sy.b_im_rows = RB;
    sy.units = units;
    sy.sites = ws.adj_tiles.ptr + nf;
    sy.nsites = 4;
    LRS_TRY((launch_tc<128, 1, 1, ZStore>(ctx, ma_h, mb_t, sy, zst, "zgemm_tc_kernel<adjoint>")));
    const double2* dof = ws.denom_o.ptr + (size_t)f * Ko;
    const double2* duf = ws.denom_u.ptr + (size_t)f * Ku;
    grad_accum32_kernel<true><<<dim3((Ko + 31) / 32, chunks), 256, 0, ctx->stream>>>(
        psi32_o, Y + yoff[0], Y + yoff[1], dof, n, Ko, ws.gpsi.ptr, ws.gpart.ptr);
    LRS_TRY(after_launch(ctx, "grad_accum32_kernel"));
    LRS_TRY(grad_energy(ctx, ws.gpart.ptr, chunks, dof, ctx->w_o.ptr, Ko, ws.ge.ptr));
    grad_accum32_kernel<false><<<dim3((Ku + 31) / 32, chunks), 256, 0, ctx->stream>>>(
        psi32_u, Y + yoff[2], Y + yoff[3], duf, n, Ku, ws.gpsi.ptr + (size_t)n * Ko, ws.gpart.ptr);
    LRS_TRY(after_launch(ctx, "grad_accum32_kernel"));
    LRS_TRY(grad_energy(ctx, ws.gpart.ptr, chunks, duf, ctx->w_u.ptr, Ku, ws.ge.ptr + Ko));
  }
  return scatter_gradients(ctx, n, ws.gpsi.ptr, ws.gpsi.ptr + (size_t)n * Ko, ws.ge.ptr, grad_e, grad_psi);
}

}  // namespace lrs
