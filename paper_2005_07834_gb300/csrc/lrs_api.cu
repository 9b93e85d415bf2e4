// C-ABI entry points of liblrs (declared in include/lrs.h): argument checks,
// device-memory ownership, the frequency quadrature of App. D.1 and the
// dispatch of each stage to the kernels of the k_*.cu translation units.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <unordered_map>

#include "lrs_internal.h"

namespace lrs {

static thread_local std::string g_last_error;

int set_error(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

void clear_error() { g_last_error.clear(); }

int h2d_sync(lrs_ctx* ctx, void* dst, const void* src, size_t bytes) {
  LRS_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return LRS_OK;
}

int after_launch(lrs_ctx* ctx, const char* what, int n) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_error(LRS_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
  ctx->stats.kernel_launches += n;
  return LRS_OK;
}

int dev_alloc_bytes(lrs_ctx* ctx, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_error(LRS_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  ctx->stats.device_bytes += (int64_t)bytes;
  ctx->stats.device_bytes_peak = std::max(ctx->stats.device_bytes_peak, ctx->stats.device_bytes);
  return LRS_OK;
}

void drop_graph(lrs_ctx* ctx) {
  if (!ctx->graph_exec) return;
  cudaGraphExecDestroy(ctx->graph_exec);
  ctx->graph_exec = nullptr;
}

void dev_free_temp(lrs_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  ctx->stats.device_bytes -= (int64_t)bytes;
}

void dev_free_bytes(lrs_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  drop_graph(ctx);
  dev_free_temp(ctx, p, bytes);
}

static int spd_streams_create(SpdStreams& sp, int priority) {
  for (cudaStream_t* st : {&sp.s2, &sp.s3, &sp.s4})
    LRS_CUDA_TRY(cudaStreamCreateWithPriority(st, cudaStreamNonBlocking, priority));
  for (cudaEvent_t& e : sp.ev) LRS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return LRS_OK;
}

static void spd_streams_destroy(SpdStreams& sp) {
  for (cudaEvent_t e : sp.ev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t st : {sp.s2, sp.s3, sp.s4})
    if (st) cudaStreamDestroy(st);
  sp = SpdStreams{};
}

int aux_stream_ready(lrs_ctx* ctx) {
  if (ctx->spd.s2) return LRS_OK;
  int lo = 0, hi = 0;
  LRS_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  ctx->prio_greatest = hi;
  return spd_streams_create(ctx->spd, hi);
}

// Lanes 1 .. n - 1 of lrs_solve_w (lane 0 is the context): streams (the first
// at the lowest priority, the panel streams at the highest), events.
static int lanes_ready(lrs_ctx* ctx, int n) {
  LRS_TRY(aux_stream_ready(ctx));
  if (!ctx->ev_lanes) LRS_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_lanes, cudaEventDisableTiming));
  int lo = 0, hi = 0;
  LRS_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  while ((int)ctx->lanes.size() < n - 1) {
    ctx->lanes.emplace_back();
    DysonLane& l = ctx->lanes.back();
    LRS_CUDA_TRY(cudaStreamCreateWithPriority(&l.s1, cudaStreamNonBlocking, lo));
    LRS_TRY(spd_streams_create(l.spd, hi));
    LRS_CUDA_TRY(cudaEventCreateWithFlags(&l.ev_done, cudaEventDisableTiming));
  }
  return LRS_OK;
}

// Exchanges the context's streams, events and Dyson workspace with a lane's
// (host-side enqueueing of one lane's solves; called again to swap back).
static void lane_swap(lrs_ctx* ctx, DysonLane& l) {
  std::swap(ctx->stream, l.s1);
  std::swap(ctx->spd, l.spd);
  Workspace& w = ctx->ws;
  std::swap(w.dyson_a, l.dyson_a);
  std::swap(w.tinv, l.tinv);
  std::swap(w.gj, l.gj);
  std::swap(w.gjb, l.gjb);
  std::swap(w.alda_n, l.alda_n);
  std::swap(w.ipiv, l.ipiv);
  std::swap(w.oz_expo, l.oz_expo);
  std::swap(w.og_expo, l.og_expo);
  std::swap(w.oz_planes, l.oz_planes);
  std::swap(w.og_planes, l.og_planes);
  std::swap(w.ru, l.ru);
}

static void release_lane_buffers(lrs_ctx* ctx, DysonLane& l) {
  release(ctx, l.dyson_a); release(ctx, l.tinv); release(ctx, l.gj); release(ctx, l.gjb); release(ctx, l.alda_n);
  release(ctx, l.ipiv); release(ctx, l.oz_expo); release(ctx, l.og_expo);
  release(ctx, l.oz_planes); release(ctx, l.og_planes); release(ctx, l.ru);
}

// A top-level stage starts a new measurement; ST_CHI0_MAIN (ST_W_MAIN)
// intervals add up until the next ST_CHI0 (ST_W) begins.
int stage_begin(lrs_ctx* ctx, Stage s) {
  if (ctx->capturing) return LRS_OK;   // stage timings are not part of a recorded graph
  if (s != ST_CHI0_MAIN && s != ST_W_MAIN) ctx->ev_used[s] = 0;
  if (s == ST_CHI0) ctx->ev_used[ST_CHI0_MAIN] = 0;
  if (s == ST_W) ctx->ev_used[ST_W_MAIN] = 0;
  const size_t i = ctx->ev_used[s];
  if (i >= ctx->ev_begin[s].size()) {
    cudaEvent_t b = nullptr, e = nullptr;
    LRS_CUDA_TRY(cudaEventCreate(&b));
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) {
      cudaEventDestroy(b);
      return set_error(LRS_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(err));
    }
    ctx->ev_begin[s].push_back(b);
    ctx->ev_end[s].push_back(e);
  }
  LRS_CUDA_TRY(cudaEventRecord(ctx->ev_begin[s][i], ctx->stream));
  return LRS_OK;
}

int stage_end(lrs_ctx* ctx, Stage s) {
  if (ctx->capturing) return LRS_OK;
  LRS_CUDA_TRY(cudaEventRecord(ctx->ev_end[s][ctx->ev_used[s]], ctx->stream));
  ++ctx->ev_used[s];
  ctx->ev_pending[s] = true;
  return LRS_OK;
}

// Switches to the context's device for the duration of an API call.
struct DeviceGuard {
  int prev = -1;
  int rc = LRS_OK;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) rc = set_error(LRS_ERR_CUDA, "cudaSetDevice(%d): %s", dev, cudaGetErrorString(e));
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Gauss-Legendre nodes (ascending) and weights on [-1, 1] by Newton iteration
// on the three-term recurrence (l+1) P_{l+1} = (2l+1) x P_l - l P_{l-1}.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int l = 1; l < n; ++l) {
        double p2 = ((2.0 * l + 1.0) * z * p1 - l * p0) / (l + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      // P_n = p1, P_{n-1} = p0;  P_n' = n (z P_n - P_{n-1}) / (z^2 - 1)
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        // one more evaluation of the derivative at the converged node
        p0 = 1.0; p1 = z;
        for (int l = 1; l < n; ++l) {
          double p2 = ((2.0 * l + 1.0) * z * p1 - l * p0) / (l + 1.0);
          p0 = p1;
          p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    double wi = 2.0 / ((1.0 - z * z) * dp * dp);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = wi;
    w[n - 1 - i] = wi;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

static bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Gamma-point real orbitals (Sec. VI.F): one k-point at k = 0 and, for every
// G, -G in the set with C_b(-G) = conj C_b(G) (to 1e-12 of the largest |C|).
// Gamma-point real orbitals (Sec. VI.F): one k-point at Gamma and C(-G) = conj C(G) for every
// band and G (to 1e-12 of the largest coefficient component).  The host pairs each G with -G
// (false if a partner is missing); the device compares the coefficients.
static bool gamma_partners(int nk, const double* kpts, int ng, const int* gvec, std::vector<int>& partner) {
  if (nk != 1 || kpts[0] != 0.0 || kpts[1] != 0.0 || kpts[2] != 0.0) return false;
  auto key = [](int a, int b, int c) {
    return ((long long)(a + (1 << 20)) << 42) | ((long long)(b + (1 << 20)) << 21) | (long long)(c + (1 << 20));
  };
  std::unordered_map<long long, int> index;
  index.reserve((size_t)ng * 2);
  for (int g = 0; g < ng; ++g) index[key(gvec[3 * g], gvec[3 * g + 1], gvec[3 * g + 2])] = g;
  partner.resize(ng);
  for (int g = 0; g < ng; ++g) {
    const auto it = index.find(key(-gvec[3 * g], -gvec[3 * g + 1], -gvec[3 * g + 2]));
    if (it == index.end()) return false;
    partner[g] = it->second;
  }
  return true;
}

// Largest |Re| or |Im| of n complex values as float64 bits (non-negative doubles order as
// their bit patterns).
__global__ void coeff_absmax_kernel(const double2* __restrict__ c, size_t n, unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fmax(fabs(c[i].x), fabs(c[i].y)));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// bad = 1 if some C(G, b) differs from conj C(-G, b) by more than 1e-12 of the largest component.
__global__ void gamma_real_check_kernel(const double2* __restrict__ c, const int* __restrict__ partner, int ng,
                                        int nb, const unsigned long long* __restrict__ maxbits,
                                        int* __restrict__ bad) {
  const double tol = 1e-12 * __longlong_as_double((long long)*maxbits);
  const size_t n = (size_t)ng * nb;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(i / nb), b = (int)(i % nb);
    const double2 x = c[i], y = c[(size_t)partner[g] * nb + b];
    if (fabs(x.x - y.x) > tol || fabs(x.y + y.y) > tol) *bad = 1;
  }
}

// Public-order energies [nk][nb] -> the per-column arrays of the occupied and unoccupied sets.
__global__ void gather_energies_kernel(const double* __restrict__ e, const int* __restrict__ col_o,
                                       const int* __restrict__ col_u, int Ko, int Ku, double* __restrict__ eo,
                                       double* __restrict__ eu) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < Ko) eo[j] = e[col_o[j]];
  else if (j < Ko + Ku) eu[j - Ko] = e[col_u[j - Ko]];
}

// Public-order site orbitals [npts][ncol] -> psi_o [npts][Ko], psi_u [npts][Ku].
__global__ void gather_psi_kernel(const double2* __restrict__ psi, int npts, int ncol, const int* __restrict__ col_o,
                                  const int* __restrict__ col_u, int Ko, int Ku, double2* __restrict__ po,
                                  double2* __restrict__ pu) {
  const size_t total = (size_t)npts * (Ko + Ku);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i / (Ko + Ku);
    const int j = (int)(i % (Ko + Ku));
    if (j < Ko) po[p * Ko + j] = psi[p * ncol + col_o[j]];
    else pu[p * Ku + (j - Ko)] = psi[p * ncol + col_u[j - Ko]];
  }
}

// After lrs_set_energies_dev the host copy of the energies is rebuilt from the
// per-column device arrays the first time host code needs it.
static int host_energies(lrs_ctx* ctx) {
  if (!ctx->energies_on_device_only) return LRS_OK;
  std::vector<double> eo(ctx->Ko), eu(ctx->Ku);
  LRS_CUDA_TRY(cudaMemcpyAsync(eo.data(), ctx->e_o.ptr, ctx->Ko * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(cudaMemcpyAsync(eu.data(), ctx->e_u.ptr, ctx->Ku * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  for (int j = 0; j < ctx->Ko; ++j) ctx->energies[ctx->col_o[j]] = eo[j];
  for (int j = 0; j < ctx->Ku; ++j) ctx->energies[ctx->col_u[j]] = eu[j];
  ctx->energies_on_device_only = false;
  return LRS_OK;
}

static int check_site(lrs_ctx* ctx, int site) {
  if (site < 0 || site >= (int)ctx->sites.size())
    return set_error(LRS_ERR_ARG, "site %d out of range (have %zu)", site, ctx->sites.size());
  return LRS_OK;
}

static int site_list(lrs_ctx* ctx, int nsite, const int* sites, std::vector<int>& out) {
  out.clear();
  if (ctx->sites.empty()) return set_error(LRS_ERR_STATE, "no sites defined");
  if (sites == nullptr) {
    for (int i = 0; i < (int)ctx->sites.size(); ++i) out.push_back(i);
    return LRS_OK;
  }
  if (nsite < 0) return set_error(LRS_ERR_ARG, "nsite < 0");
  for (int i = 0; i < nsite; ++i) {
    LRS_TRY(check_site(ctx, sites[i]));
    out.push_back(sites[i]);
  }
  return LRS_OK;
}

static void free_site(lrs_ctx* ctx, Site& s) {
  release(ctx, s.pts);
  release(ctx, s.wts);
  s.has_v = false;
  release(ctx, s.psi_o);
  release(ctx, s.psi_u);
  release(ctx, s.chi0);
  release(ctx, s.w);
  release(ctx, s.v);
  release(ctx, s.yang);
  release(ctx, s.rl);
  release(ctx, s.fl);
  s.spd = false;
  release(ctx, s.fxc);
  release(ctx, s.chi_eff);
  s.fxc_kind = LRS_FXC_NONE;
  s.product = false;
  s.has_psi = s.has_chi0 = s.has_w = false;
}

static void free_workspace(lrs_ctx* ctx) {
  Workspace& w = ctx->ws;
  release(ctx, w.denom_o); release(ctx, w.denom_u); release(ctx, w.dyson_a); release(ctx, w.ipiv); release(ctx, w.tinv);
  release(ctx, w.status); release(ctx, w.phase_tab); release(ctx, w.kphase); release(ctx, w.ru);
  release(ctx, w.gamma_s); release(ctx, w.gbuf_o); release(ctx, w.gbuf_u); release(ctx, w.ybuf);
  release(ctx, w.ge); release(ctx, w.gpsi); release(ctx, w.gpart); release(ctx, w.tmp_nn);
  release(ctx, w.planes_a); release(ctx, w.planes_b); release(ctx, w.slab); release(ctx, w.denom32); release(ctx, w.phase_tab32); release(ctx, w.tc_scratch); release(ctx, w.slab64);
  release(ctx, w.site_tiles);
  release(ctx, w.planes_t); release(ctx, w.planes_h); release(ctx, w.g32); release(ctx, w.yz32); release(ctx, w.psi32);
  release(ctx, w.gamma_chk);
  release(ctx, w.adj_tiles);
  release(ctx, w.gj);
  release(ctx, w.gjb);
  release(ctx, w.oz_planes); release(ctx, w.oz_expo); release(ctx, w.og_planes); release(ctx, w.og_expo);
  release(ctx, w.fft_grid); release(ctx, w.fft_index); release(ctx, w.fft_tw);
  release(ctx, w.induced);
  release(ctx, w.alda_n); release(ctx, w.aug_tab); release(ctx, w.aug_coef);
  w.fft_plan_ok = false;
  release(ctx, w.proj_a); release(ctx, w.proj_b); release(ctx, w.scales); release(ctx, w.proj_scale);
  for (DysonLane& l : ctx->lanes) release_lane_buffers(ctx, l);
}

}  // namespace lrs

using namespace lrs;

extern "C" {

const char* lrs_last_error(void) { return g_last_error.c_str(); }

// The chi0 tensor-core kernel revision lets measurements quote profiler
// counters only for the kernel version they were taken on.
const char* lrs_version(void) { return "lrs 0.6 (sm_103a) chi0-tc r3 dyson-gj r8"; }

int lrs_create(lrs_ctx** out, int device, int precision, void* stream) {
  clear_error();
  if (!out) return set_error(LRS_ERR_ARG, "ctx is NULL");
  *out = nullptr;
  if (precision != LRS_FP64 && precision != LRS_MIXED_BF16X3 && precision != LRS_MIXED_FP16X3)
    return set_error(LRS_ERR_ARG, "unknown precision %d", precision);
  int ndev = 0;
  LRS_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return set_error(LRS_ERR_ARG, "device %d out of range (%d)", device, ndev);
  DeviceGuard g(device);
  if (g.rc) return g.rc;
  cudaDeviceProp prop;
  LRS_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
  if (precision != LRS_FP64 && prop.major * 10 + prop.minor < 100)
    return set_error(LRS_ERR_UNSUPPORTED, "mixed precision needs tcgen05 (sm_100 family), device is sm_%d%d",
                     prop.major, prop.minor);
  lrs_ctx* ctx = new lrs_ctx();
  ctx->device = device;
  ctx->precision = precision;
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->num_sms = prop.multiProcessorCount;
  int rc = ensure(ctx, ctx->ws.status, 64);
  if (rc == LRS_OK) rc = aux_stream_ready(ctx);
  if (rc) {
    const std::string msg = lrs_last_error();
    lrs_destroy(ctx);
    return set_error(rc, "%s", msg.c_str());
  }
  cudaMemsetAsync(ctx->ws.status.ptr, 0, 64 * sizeof(int), ctx->stream);
  *out = ctx;
  return LRS_OK;
}

int lrs_destroy(lrs_ctx* ctx) {
  clear_error();
  if (!ctx) return LRS_OK;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& s : ctx->sites) free_site(ctx, s);
  release(ctx, ctx->coeff);
  release(ctx, ctx->d_gvec);
  release(ctx, ctx->d_kpts);
  release(ctx, ctx->d_t);
  release(ctx, ctx->d_W);
  release(ctx, ctx->e_o); release(ctx, ctx->e_u); release(ctx, ctx->w_o); release(ctx, ctx->w_u);
  release(ctx, ctx->d_col_o); release(ctx, ctx->d_col_u);
  free_workspace(ctx);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  spd_streams_destroy(ctx->spd);
  for (DysonLane& l : ctx->lanes) {
    spd_streams_destroy(l.spd);
    if (l.ev_done) cudaEventDestroy(l.ev_done);
    if (l.s1) cudaStreamDestroy(l.s1);
  }
  if (ctx->ev_lanes) cudaEventDestroy(ctx->ev_lanes);
  for (int s = 0; s < 6; ++s) {
    for (cudaEvent_t e : ctx->ev_begin[s]) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->ev_end[s]) cudaEventDestroy(e);
  }
  delete ctx;
  return LRS_OK;
}

int lrs_set_option(lrs_ctx* ctx, int option, int value) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  switch (option) {
    case LRS_OPT_DYSON_BASIS:
      if (value != LRS_DYSON_AUTO && value != LRS_DYSON_FULL && value != LRS_DYSON_LM)
        return set_error(LRS_ERR_ARG, "unknown Dyson basis %d", value);
      ctx->dyson_basis = value;
      return LRS_OK;
    case LRS_OPT_DYSON_PANEL:
      if (value != 0 && value != 32 && value != SPD_OUTER_BLOCK)
        return set_error(LRS_ERR_ARG, "Dyson pivot-block width %d: 0 (auto), 32 or %d", value, SPD_OUTER_BLOCK);
      ctx->dyson_panel = value;
      return LRS_OK;
    case LRS_OPT_DYSON_LANES:
      if (value < 1 || value > 8) return set_error(LRS_ERR_ARG, "Dyson lanes %d out of [1, 8]", value);
      ctx->dyson_lanes = value;
      return LRS_OK;
    case LRS_OPT_DYSON_UPDATE:
      if (value != LRS_UPDATE_AUTO && value != LRS_UPDATE_FP64 && value != LRS_UPDATE_TC)
        return set_error(LRS_ERR_ARG, "Dyson update mode %d unknown", value);
      ctx->dyson_update = value;
      return LRS_OK;
    case LRS_OPT_REAL_ORBITALS:
      if (value != LRS_REAL_AUTO && value != LRS_REAL_OFF) return set_error(LRS_ERR_ARG, "real-orbital mode %d", value);
      ctx->real_mode = value;
      return LRS_OK;
    case LRS_OPT_GRAPH_PROJECTION:
      if (value != LRS_PROJ_EXACT && value != LRS_PROJ_FFT_LAGRANGE3)
        return set_error(LRS_ERR_ARG, "projection mode %d unknown", value);
      ctx->graph_projection = value;
      return LRS_OK;
    case LRS_OPT_DYSON_SOLVER:
      if (value != LRS_SOLVER_AUTO && value != LRS_SOLVER_LU && value != LRS_SOLVER_SPD)
        return set_error(LRS_ERR_ARG, "Dyson solver %d unknown", value);
      ctx->dyson_solver = value;
      return LRS_OK;
    case LRS_OPT_WORKSPACE_GB:
      if (value < 1 || value > 4096) return set_error(LRS_ERR_ARG, "workspace budget %d GB out of range", value);
      ctx->workspace_budget = 1e9 * value;
      return LRS_OK;
    case LRS_OPT_CHI0_TILE_N:
      if (value != 64 && value != 128) return set_error(LRS_ERR_ARG, "chi0 tile width %d not in {64, 128}", value);
      ctx->chi0_tn = value;
      return LRS_OK;
    case LRS_OPT_CHI0_SEGMENT:
    case LRS_OPT_PROJ_SEGMENT:
      if (value < 1 || value > 1024) return set_error(LRS_ERR_ARG, "segment %d out of [1,1024]", value);
      (option == LRS_OPT_CHI0_SEGMENT ? ctx->seg_chunks : ctx->proj_seg_chunks) = value;
      return LRS_OK;
    default:
      return set_error(LRS_ERR_ARG, "unknown option %d", option);
  }
}

int lrs_set_stream(lrs_ctx* ctx, void* stream) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  ctx->stream = static_cast<cudaStream_t>(stream);
  return LRS_OK;
}

int lrs_load_orbitals(lrs_ctx* ctx, const double* cell, int nk, const double* kpts,
                      const double* kweights, int ng, const int* gvec, int nbands,
                      const int* nocc, const double* coeff, const double* energies) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (!cell || !kpts || !kweights || !gvec || !nocc || !coeff || !energies)
    return set_error(LRS_ERR_ARG, "null input pointer");
  if (nk < 1 || ng < 1 || nbands < 2) return set_error(LRS_ERR_ARG, "nk, ng >= 1 and nbands >= 2 required");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  double det = cell[0] * (cell[4] * cell[8] - cell[5] * cell[7]) -
               cell[1] * (cell[3] * cell[8] - cell[5] * cell[6]) +
               cell[2] * (cell[3] * cell[7] - cell[4] * cell[6]);
  if (!std::isfinite(det) || std::fabs(det) < 1e-12) return set_error(LRS_ERR_ARG, "singular cell");
  if (!finite_all(kpts, 3 * (size_t)nk) || !finite_all(kweights, nk) ||
      !finite_all(energies, (size_t)nk * nbands))
    return set_error(LRS_ERR_ARG, "non-finite k-point, weight or energy");
  int Ko = 0, Ku = 0;
  for (int k = 0; k < nk; ++k) {
    if (nocc[k] < 1 || nocc[k] >= nbands)
      return set_error(LRS_ERR_ARG, "nocc[%d] = %d must be in [1, nbands-1]", k, nocc[k]);
    Ko += nocc[k];
    Ku += nbands - nocc[k];
  }
  // reciprocal rows b_i = 2 pi (cell^-1)^T rows
  double inv[9];
  inv[0] = (cell[4] * cell[8] - cell[5] * cell[7]) / det;
  inv[1] = (cell[2] * cell[7] - cell[1] * cell[8]) / det;
  inv[2] = (cell[1] * cell[5] - cell[2] * cell[4]) / det;
  inv[3] = (cell[5] * cell[6] - cell[3] * cell[8]) / det;
  inv[4] = (cell[0] * cell[8] - cell[2] * cell[6]) / det;
  inv[5] = (cell[2] * cell[3] - cell[0] * cell[5]) / det;
  inv[6] = (cell[3] * cell[7] - cell[4] * cell[6]) / det;
  inv[7] = (cell[1] * cell[6] - cell[0] * cell[7]) / det;
  inv[8] = (cell[0] * cell[4] - cell[1] * cell[3]) / det;
  const double two_pi = 6.283185307179586476925;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) ctx->recip[3 * i + j] = two_pi * inv[3 * j + i];
  std::memcpy(ctx->cell, cell, 9 * sizeof(double));
  ctx->omega = std::fabs(det);
  ctx->nk = nk; ctx->ng = ng; ctx->nb = nbands; ctx->Ko = Ko; ctx->Ku = Ku;
  ctx->nocc.assign(nocc, nocc + nk);
  ctx->kpts.assign(kpts, kpts + 3 * nk);
  ctx->kw.assign(kweights, kweights + nk);
  ctx->energies.assign(energies, energies + (size_t)nk * nbands);
  ctx->energies_on_device_only = false;
  ctx->gvec.assign(gvec, gvec + 3 * (size_t)ng);
  ctx->ws.fft_plan_ok = false;   // the FFT index tables follow the G set
  std::vector<int> partner;
  const bool gamma_candidate = gamma_partners(nk, kpts, ng, gvec, partner);
  ctx->real_orbitals = false;
  for (int i = 0; i < 3; ++i) ctx->gmax_idx[i] = 0;
  for (int gi = 0; gi < ng; ++gi)
    for (int i = 0; i < 3; ++i) ctx->gmax_idx[i] = std::max(ctx->gmax_idx[i], std::abs(gvec[3 * gi + i]));
  // column maps and per-column energies / k-weights
  ctx->col_o.clear(); ctx->col_u.clear();
  std::vector<double> eo, eu, wo, wu;
  for (int k = 0; k < nk; ++k)
    for (int b = 0; b < nbands; ++b) {
      double e = energies[(size_t)k * nbands + b];
      if (b < nocc[k]) { ctx->col_o.push_back(k * nbands + b); eo.push_back(e); wo.push_back(kweights[k]); }
      else { ctx->col_u.push_back(k * nbands + b); eu.push_back(e); wu.push_back(kweights[k]); }
    }
  size_t ncoef = (size_t)nk * ng * nbands;
  LRS_TRY(ensure(ctx, ctx->coeff, ncoef));
  LRS_TRY(ensure(ctx, ctx->d_gvec, 3 * (size_t)ng));
  LRS_TRY(ensure(ctx, ctx->d_kpts, 3 * (size_t)nk));
  LRS_TRY(ensure(ctx, ctx->e_o, Ko)); LRS_TRY(ensure(ctx, ctx->e_u, Ku));
  LRS_TRY(ensure(ctx, ctx->w_o, Ko)); LRS_TRY(ensure(ctx, ctx->w_u, Ku));
  LRS_TRY(ensure(ctx, ctx->d_col_o, Ko)); LRS_TRY(ensure(ctx, ctx->d_col_u, Ku));
  LRS_CUDA_TRY(cudaMemcpyAsync(ctx->coeff.ptr, coeff, ncoef * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
  if (gamma_candidate) {
    // scratch (kept in the workspace: freeing device memory waits for the whole device, which
    // would stall other contexts' work on every load): partner [ng] ints, the max bits, the flag
    const size_t words = (size_t)ng + 6;
    LRS_TRY(ensure(ctx, ctx->ws.gamma_chk, words));
    int* d_partner = ctx->ws.gamma_chk.ptr;
    unsigned long long* d_max = reinterpret_cast<unsigned long long*>(d_partner + ((ng + 1) & ~1));
    int* d_bad = d_partner + ((ng + 1) & ~1) + 2;
    int rc = LRS_OK;
    int bad = 1;
    cudaError_t e = cudaMemcpyAsync(d_partner, partner.data(), ng * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_max, 0, 4 * sizeof(int), ctx->stream);
    if (e == cudaSuccess) {
      coeff_absmax_kernel<<<ctx->num_sms * 4, 256, 0, ctx->stream>>>(ctx->coeff.ptr, ncoef, d_max);
      gamma_real_check_kernel<<<ctx->num_sms * 4, 256, 0, ctx->stream>>>(ctx->coeff.ptr, d_partner, ng, nbands,
                                                                           d_max, d_bad);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) rc = set_error(LRS_ERR_CUDA, "Gamma-point check: %s", cudaGetErrorString(e));
    if (rc != LRS_OK) return rc;
    ctx->real_orbitals = bad == 0;
  }
  LRS_CUDA_TRY(cudaMemcpyAsync(ctx->d_gvec.ptr, gvec, 3 * (size_t)ng * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  LRS_CUDA_TRY(cudaMemcpyAsync(ctx->d_kpts.ptr, kpts, 3 * (size_t)nk * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  LRS_CUDA_TRY(cudaMemcpyAsync(ctx->e_o.ptr, eo.data(), Ko * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  LRS_CUDA_TRY(cudaMemcpyAsync(ctx->e_u.ptr, eu.data(), Ku * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  LRS_CUDA_TRY(cudaMemcpyAsync(ctx->w_o.ptr, wo.data(), Ko * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  LRS_CUDA_TRY(cudaMemcpyAsync(ctx->w_u.ptr, wu.data(), Ku * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  LRS_CUDA_TRY(cudaMemcpyAsync(ctx->d_col_o.ptr, ctx->col_o.data(), Ko * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  LRS_CUDA_TRY(cudaMemcpyAsync(ctx->d_col_u.ptr, ctx->col_u.data(), Ku * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  // the host vectors above go out of scope: wait for the copies
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  ctx->has_orb = true;
  ctx->ws.coeff_planes_valid = false;
  ctx->nf = 0;
  for (auto& s : ctx->sites) s.has_psi = s.has_chi0 = s.has_w = false;
  return LRS_OK;
}

int lrs_set_sites(lrs_ctx* ctx, int nsites, const double* centers, const int* npts,
                  const double* pts, const double* wts, const int* lmax) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (nsites < 1 || !centers || !npts || !pts || !wts || !lmax)
    return set_error(LRS_ERR_ARG, "nsites >= 1 and non-null arrays required");
  size_t off = 0;
  for (int i = 0; i < nsites; ++i) {
    if (npts[i] < 1) return set_error(LRS_ERR_ARG, "npts[%d] = %d", i, npts[i]);
    if (lmax[i] < 0 || lmax[i] > 64) return set_error(LRS_ERR_ARG, "lmax[%d] = %d out of [0,64]", i, lmax[i]);
    for (int p = 0; p < npts[i]; ++p) {
      const double* r = pts + 3 * (off + p);
      double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (!(rr > 0.0) || !std::isfinite(rr) || !std::isfinite(wts[off + p]))
        return set_error(LRS_ERR_ARG, "site %d point %d at the origin or non-finite", i, p);
    }
    off += npts[i];
  }
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  cudaStreamSynchronize(ctx->stream);
  // A recorded build refers to the previous sites.  The device buffers of the sites that remain
  // are kept and regrown only when too small: cudaFree waits for the whole device, which would
  // stall the work other contexts have in flight.
  drop_graph(ctx);
  ctx->w_pending.clear();   // queued solves refer to the previous sites (their status words stay)
  for (size_t i = nsites; i < ctx->sites.size(); ++i) free_site(ctx, ctx->sites[i]);
  ctx->sites.resize(nsites);
  off = 0;
  for (int i = 0; i < nsites; ++i) {
    Site& s = ctx->sites[i];
    s.has_v = s.has_psi = s.has_chi0 = s.has_w = false;
    s.spd = false;
    s.product = false;
    s.fxc_kind = LRS_FXC_NONE;
    s.nrad = s.nang = 0;
    s.npts = npts[i];
    s.lmax = lmax[i];
    std::memcpy(s.center, centers + 3 * i, 3 * sizeof(double));
    LRS_TRY(ensure(ctx, s.pts, 3 * (size_t)s.npts));
    LRS_TRY(ensure(ctx, s.wts, s.npts));
    LRS_TRY(h2d_sync(ctx, s.pts.ptr, pts + 3 * off, 3 * (size_t)s.npts * sizeof(double)));
    LRS_TRY(h2d_sync(ctx, s.wts.ptr, wts + off, (size_t)s.npts * sizeof(double)));
    LRS_TRY(site_detect_product(ctx, s, pts + 3 * off));
    off += npts[i];
  }
  return LRS_OK;
}

int lrs_set_frequency_quadrature(lrs_ctx* ctx, int nf, double mu, double zeta, double* mu_out,
                                 double* zeta_out) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (!ctx->has_orb) return set_error(LRS_ERR_STATE, "load orbitals first");
  if (nf < 1 || nf > 128) return set_error(LRS_ERR_ARG, "nf = %d out of [1,128]", nf);
  {
    DeviceGuard g(ctx->device);
    if (g.rc) return g.rc;
    LRS_TRY(host_energies(ctx));
  }
  if (std::isnan(mu)) {
    double top = -1e300, bottom = 1e300;
    for (int k = 0; k < ctx->nk; ++k)
      for (int b = 0; b < ctx->nb; ++b) {
        double e = ctx->energies[(size_t)k * ctx->nb + b];
        if (b < ctx->nocc[k]) top = std::max(top, e);
        else bottom = std::min(bottom, e);
      }
    mu = 0.5 * (top + bottom);
  }
  if (!std::isfinite(mu)) return set_error(LRS_ERR_ARG, "non-finite mu");
  double dmin = 1e300, dmax = 0.0;
  for (double e : ctx->energies) {
    double d = std::fabs(mu - e);
    dmin = std::min(dmin, d);
    dmax = std::max(dmax, d);
  }
  // every occupied level must lie below mu and every unoccupied one above it
  for (int k = 0; k < ctx->nk; ++k)
    for (int b = 0; b < ctx->nb; ++b) {
      double e = ctx->energies[(size_t)k * ctx->nb + b];
      if ((b < ctx->nocc[k] && !(e < mu)) || (b >= ctx->nocc[k] && !(e > mu)))
        return set_error(LRS_ERR_ARG, "mu = %g does not separate occupied and unoccupied levels", mu);
    }
  if (!(zeta > 0.0)) {
    const double floor_ha = 0.5 / 27.211386245988;  // 0.5 eV added in quadrature
    zeta = std::sqrt(std::sqrt(dmin * dmin + floor_ha * floor_ha) * dmax);
  }
  if (!std::isfinite(zeta)) return set_error(LRS_ERR_ARG, "non-finite zeta");
  std::vector<double> x, w;
  gauss_legendre(nf, x, w);
  ctx->t.resize(nf);
  ctx->W.resize(nf);
  for (int i = 0; i < nf; ++i) {
    double a = 0.5 * (x[i] + 1.0), wa = 0.5 * w[i];
    ctx->t[i] = zeta * a / (1.0 - a);
    ctx->W[i] = zeta * wa / ((1.0 - a) * (1.0 - a));
  }
  LRS_TRY(ensure(ctx, ctx->d_t, nf));
  LRS_TRY(ensure(ctx, ctx->d_W, nf));
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  LRS_TRY(h2d_sync(ctx, ctx->d_t.ptr, ctx->t.data(), nf * sizeof(double)));
  LRS_TRY(h2d_sync(ctx, ctx->d_W.ptr, ctx->W.data(), nf * sizeof(double)));
  ctx->nf = nf;
  ctx->mu = mu;
  ctx->zeta = zeta;
  if (mu_out) *mu_out = mu;
  if (zeta_out) *zeta_out = zeta;
  for (auto& s : ctx->sites) s.has_chi0 = s.has_w = false;
  return LRS_OK;
}

int lrs_get_frequency_quadrature(lrs_ctx* ctx, double* t, double* w) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (ctx->nf == 0) return set_error(LRS_ERR_STATE, "no quadrature set");
  if (t) std::memcpy(t, ctx->t.data(), ctx->nf * sizeof(double));
  if (w) std::memcpy(w, ctx->W.data(), ctx->nf * sizeof(double));
  return LRS_OK;
}

static int alloc_psi(lrs_ctx* ctx, Site& s) {
  LRS_TRY(ensure(ctx, s.psi_o, (size_t)s.npts * ctx->Ko));
  LRS_TRY(ensure(ctx, s.psi_u, (size_t)s.npts * ctx->Ku));
  return LRS_OK;
}

int lrs_project(lrs_ctx* ctx, int nsite, const int* sites, int mode) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (!ctx->has_orb) return set_error(LRS_ERR_STATE, "load orbitals first");
  if (mode != LRS_PROJ_EXACT && mode != LRS_PROJ_FFT_LAGRANGE3)
    return set_error(LRS_ERR_UNSUPPORTED, "projection mode %d not available", mode);
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  std::vector<int> list;
  LRS_TRY(site_list(ctx, nsite, sites, list));
  for (int i : list) LRS_TRY(alloc_psi(ctx, ctx->sites[i]));
  LRS_TRY(stage_begin(ctx, ST_PROJECT));
  if (mode == LRS_PROJ_FFT_LAGRANGE3) {
    LRS_TRY(project_fft(ctx, list));
  } else {
    for (int i : list) {
      Site& s = ctx->sites[i];
      if (ctx->precision == LRS_FP64) LRS_TRY(project_fp64(ctx, s));
      else LRS_TRY(project_mixed(ctx, s));
    }
  }
  for (int i : list) {
    Site& s = ctx->sites[i];
    s.has_psi = true;
    s.has_chi0 = s.has_w = false;
  }
  LRS_TRY(stage_end(ctx, ST_PROJECT));
  return LRS_OK;
}

int lrs_augment(lrs_ctx* ctx, int site, int lmax_aug, int nnu, double r_aug, const double* phi_ae,
                const double* phi_ps) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  LRS_TRY(check_site(ctx, site));
  Site& s = ctx->sites[site];
  if (!s.has_psi) return set_error(LRS_ERR_STATE, "site %d has no orbitals (project first)", site);
  if (!s.product) return set_error(LRS_ERR_UNSUPPORTED, "site %d is not a radial x angular product grid", site);
  if (lmax_aug < 0 || lmax_aug > s.lmax) return set_error(LRS_ERR_ARG, "l_aug %d outside [0, %d]", lmax_aug, s.lmax);
  if (nnu < 1 || nnu > 64) return set_error(LRS_ERR_ARG, "%d partial waves per l outside [1, 64]", nnu);
  if (!(r_aug > 0.0) || !std::isfinite(r_aug)) return set_error(LRS_ERR_ARG, "augmentation radius must be positive");
  const size_t nv = (size_t)(lmax_aug + 1) * nnu * s.nrad;
  if (!phi_ae || !phi_ps) return set_error(LRS_ERR_ARG, "NULL partial waves");
  if (!finite_all(phi_ae, nv) || !finite_all(phi_ps, nv)) return set_error(LRS_ERR_ARG, "non-finite partial wave");
  if (ctx->capturing) return set_error(LRS_ERR_STATE, "augmentation cannot be recorded in a graph");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  LRS_TRY(augment_site(ctx, s, lmax_aug, nnu, r_aug, phi_ae, phi_ps));
  s.has_chi0 = s.has_w = false;
  return LRS_OK;
}

int lrs_set_fxc(lrs_ctx* ctx, int site, int kind, const double* fxc) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  LRS_TRY(check_site(ctx, site));
  if (kind != LRS_FXC_NONE && kind != LRS_FXC_USER && kind != LRS_FXC_ALDA_X)
    return set_error(LRS_ERR_ARG, "f_xc kind %d unknown", kind);
  Site& s = ctx->sites[site];
  if (kind == LRS_FXC_USER) {
    if (!fxc) return set_error(LRS_ERR_ARG, "fxc is NULL");
    if (!finite_all(fxc, (size_t)s.npts)) return set_error(LRS_ERR_ARG, "non-finite f_xc value");
    DeviceGuard g(ctx->device);
    if (g.rc) return g.rc;
    LRS_TRY(ensure(ctx, s.fxc, (size_t)s.npts));
    LRS_CUDA_TRY(cudaMemcpyAsync(s.fxc.ptr, fxc, s.npts * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  }
  s.fxc_kind = kind;
  s.has_w = false;
  return LRS_OK;
}

int lrs_orbitals_are_real(lrs_ctx* ctx, int* is_real) {
  clear_error();
  if (!ctx || !is_real) return set_error(LRS_ERR_ARG, "NULL argument");
  if (!ctx->has_orb) return set_error(LRS_ERR_STATE, "load orbitals first");
  *is_real = ctx->real_orbitals ? 1 : 0;
  return LRS_OK;
}

int lrs_get_density(lrs_ctx* ctx, int site, double* n) {
  clear_error();
  if (!ctx || !n) return set_error(LRS_ERR_ARG, "NULL argument");
  LRS_TRY(check_site(ctx, site));
  Site& s = ctx->sites[site];
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  LRS_TRY(ensure(ctx, ctx->ws.alda_n, (size_t)s.npts));
  LRS_TRY(site_density(ctx, s, ctx->ws.alda_n.ptr));
  LRS_CUDA_TRY(cudaMemcpyAsync(n, ctx->ws.alda_n.ptr, s.npts * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return LRS_OK;
}

int lrs_get_fxc(lrs_ctx* ctx, int site, double* fxc) {
  clear_error();
  if (!ctx || !fxc) return set_error(LRS_ERR_ARG, "NULL argument");
  LRS_TRY(check_site(ctx, site));
  Site& s = ctx->sites[site];
  if (s.fxc_kind == LRS_FXC_NONE) return set_error(LRS_ERR_STATE, "site %d has no f_xc kernel", site);
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  LRS_TRY(site_fxc(ctx, s));
  LRS_CUDA_TRY(cudaMemcpyAsync(fxc, s.fxc.ptr, s.npts * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return LRS_OK;
}

int lrs_site_grid_shape(lrs_ctx* ctx, int site, int* product, int* nrad, int* nang) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (site < 0 || site >= (int)ctx->sites.size()) return set_error(LRS_ERR_ARG, "site %d out of range", site);
  const Site& s = ctx->sites[site];
  if (product) *product = s.product ? 1 : 0;
  if (nrad) *nrad = s.product ? s.nrad : 0;
  if (nang) *nang = s.product ? s.nang : 0;
  return LRS_OK;
}

int lrs_induced_potential(lrs_ctx* ctx, int site, double q, double shell_radius, int lresp, double* rho_lm,
                          double* vind_lm, double* vind_grid) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (site < 0 || site >= (int)ctx->sites.size()) return set_error(LRS_ERR_ARG, "site %d out of range", site);
  Site& s = ctx->sites[site];
  if (!s.has_chi0) return set_error(LRS_ERR_STATE, "site %d has no chi0", site);
  if (!s.product) return set_error(LRS_ERR_UNSUPPORTED, "site %d is not a radial x angular product grid", site);
  if (lresp < 0 || lresp > s.lmax) return set_error(LRS_ERR_ARG, "l_resp %d outside [0, %d]", lresp, s.lmax);
  if (!(shell_radius > 0.0) || !std::isfinite(shell_radius) || !std::isfinite(q))
    return set_error(LRS_ERR_ARG, "shell radius must be positive and finite, q finite");
  if (ctx->capturing) return set_error(LRS_ERR_STATE, "the induced response cannot be recorded in a graph");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  if (s.fxc_kind != LRS_FXC_NONE) LRS_TRY(alda_dress(ctx, s));
  return induced_potential(ctx, s, q, shell_radius, lresp, rho_lm, vind_lm, vind_grid);
}

int lrs_set_fft_grid(lrs_ctx* ctx, int n1, int n2, int n3) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  const int n[3] = {n1, n2, n3};
  const bool automatic = n1 == 0 && n2 == 0 && n3 == 0;
  for (int d = 0; d < 3 && !automatic; ++d)
    if (!fft_length_ok(n[d])) return set_error(LRS_ERR_ARG, "FFT length %d is not 2^a 3^b in [1, %d]", n[d], LRS_FFT_MAX_N);
  for (int d = 0; d < 3; ++d) ctx->fft_n[d] = n[d];
  return LRS_OK;
}

int lrs_get_fft_grid(lrs_ctx* ctx, int* n) {
  clear_error();
  if (!ctx || !n) return set_error(LRS_ERR_ARG, "NULL argument");
  if (!ctx->has_orb) return set_error(LRS_ERR_STATE, "load orbitals first");
  return fft_grid_dims(ctx, n);
}

int lrs_set_energies(lrs_ctx* ctx, const double* energies) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (!ctx->has_orb) return set_error(LRS_ERR_STATE, "load orbitals first");
  if (!energies) return set_error(LRS_ERR_ARG, "energies is NULL");
  const size_t ne = (size_t)ctx->nk * ctx->nb;
  if (!finite_all(energies, ne)) return set_error(LRS_ERR_ARG, "non-finite energy");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  ctx->energies.assign(energies, energies + ne);
  ctx->energies_on_device_only = false;
  std::vector<double> eo(ctx->Ko), eu(ctx->Ku);
  for (int j = 0; j < ctx->Ko; ++j) eo[j] = energies[ctx->col_o[j]];
  for (int j = 0; j < ctx->Ku; ++j) eu[j] = energies[ctx->col_u[j]];
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  LRS_TRY(h2d_sync(ctx, ctx->e_o.ptr, eo.data(), ctx->Ko * sizeof(double)));
  LRS_TRY(h2d_sync(ctx, ctx->e_u.ptr, eu.data(), ctx->Ku * sizeof(double)));
  for (auto& s : ctx->sites) s.has_chi0 = s.has_w = false;
  return LRS_OK;
}

int lrs_set_site_orbitals(lrs_ctx* ctx, int site, const double* psi) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (!ctx->has_orb) return set_error(LRS_ERR_STATE, "load orbitals first");
  LRS_TRY(check_site(ctx, site));
  if (!psi) return set_error(LRS_ERR_ARG, "psi is NULL");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  Site& s = ctx->sites[site];
  LRS_TRY(alloc_psi(ctx, s));
  const size_t ncol = (size_t)ctx->nk * ctx->nb;
  std::vector<double2> o((size_t)s.npts * ctx->Ko), u((size_t)s.npts * ctx->Ku);
  for (int p = 0; p < s.npts; ++p) {
    const double2* row = reinterpret_cast<const double2*>(psi) + p * ncol;
    for (int j = 0; j < ctx->Ko; ++j) o[(size_t)p * ctx->Ko + j] = row[ctx->col_o[j]];
    for (int j = 0; j < ctx->Ku; ++j) u[(size_t)p * ctx->Ku + j] = row[ctx->col_u[j]];
  }
  LRS_CUDA_TRY(cudaMemcpyAsync(s.psi_o.ptr, o.data(), o.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
  LRS_CUDA_TRY(cudaMemcpyAsync(s.psi_u.ptr, u.data(), u.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  s.has_psi = true;
  s.has_chi0 = s.has_w = false;
  return LRS_OK;
}

int lrs_set_energies_dev(lrs_ctx* ctx, const double* energies_dev) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (!ctx->has_orb) return set_error(LRS_ERR_STATE, "load orbitals first");
  if (!energies_dev) return set_error(LRS_ERR_ARG, "energies_dev is NULL");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  const int K = ctx->Ko + ctx->Ku;
  gather_energies_kernel<<<(K + 255) / 256, 256, 0, ctx->stream>>>(energies_dev, ctx->d_col_o.ptr, ctx->d_col_u.ptr,
                                                                   ctx->Ko, ctx->Ku, ctx->e_o.ptr, ctx->e_u.ptr);
  LRS_TRY(after_launch(ctx, "gather_energies_kernel"));
  ctx->energies_on_device_only = true;
  for (auto& s : ctx->sites) s.has_chi0 = s.has_w = false;
  return LRS_OK;
}

int lrs_set_site_orbitals_dev(lrs_ctx* ctx, int site, const double* psi_dev) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (!ctx->has_orb) return set_error(LRS_ERR_STATE, "load orbitals first");
  LRS_TRY(check_site(ctx, site));
  if (!psi_dev) return set_error(LRS_ERR_ARG, "psi_dev is NULL");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  Site& s = ctx->sites[site];
  LRS_TRY(alloc_psi(ctx, s));
  const size_t total = (size_t)s.npts * (ctx->Ko + ctx->Ku);
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 32);
  gather_psi_kernel<<<blocks, 256, 0, ctx->stream>>>(reinterpret_cast<const double2*>(psi_dev), s.npts,
                                                     ctx->nk * ctx->nb, ctx->d_col_o.ptr, ctx->d_col_u.ptr, ctx->Ko,
                                                     ctx->Ku, s.psi_o.ptr, s.psi_u.ptr);
  LRS_TRY(after_launch(ctx, "gather_psi_kernel"));
  s.has_psi = true;
  s.has_chi0 = s.has_w = false;
  return LRS_OK;
}

int lrs_get_site_orbitals(lrs_ctx* ctx, int site, double* psi) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  LRS_TRY(check_site(ctx, site));
  if (!psi) return set_error(LRS_ERR_ARG, "psi is NULL");
  Site& s = ctx->sites[site];
  if (!s.has_psi) return set_error(LRS_ERR_STATE, "site %d has no orbitals", site);
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  const size_t ncol = (size_t)ctx->nk * ctx->nb;
  std::vector<double2> o((size_t)s.npts * ctx->Ko), u((size_t)s.npts * ctx->Ku);
  LRS_CUDA_TRY(cudaMemcpyAsync(o.data(), s.psi_o.ptr, o.size() * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(cudaMemcpyAsync(u.data(), s.psi_u.ptr, u.size() * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  for (int p = 0; p < s.npts; ++p) {
    double2* row = reinterpret_cast<double2*>(psi) + p * ncol;
    for (int j = 0; j < ctx->Ko; ++j) row[ctx->col_o[j]] = o[(size_t)p * ctx->Ko + j];
    for (int j = 0; j < ctx->Ku; ++j) row[ctx->col_u[j]] = u[(size_t)p * ctx->Ku + j];
  }
  return LRS_OK;
}

int lrs_build_chi0(lrs_ctx* ctx, int nsite, const int* sites) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (ctx->nf == 0) return set_error(LRS_ERR_STATE, "set the frequency quadrature first");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  std::vector<int> list;
  LRS_TRY(site_list(ctx, nsite, sites, list));
  for (int i : list)
    if (!ctx->sites[i].has_psi) return set_error(LRS_ERR_STATE, "site %d has no orbitals", i);
  for (int i : list) LRS_TRY(ensure(ctx, ctx->sites[i].chi0, (size_t)ctx->sites[i].npts * ctx->sites[i].npts));
  LRS_TRY(stage_begin(ctx, ST_CHI0));
  LRS_TRY(build_denominators(ctx));
  double flop = 0;
  if (ctx->precision != LRS_FP64) {
    // as many sites per persistent launch as the operand workspace budget allows
    const double kp = 2.0 * (((ctx->Ko + 31) / 32 + (ctx->Ku + 31) / 32) * 32);
    LRS_TRY(ensure(ctx, ctx->ws.site_tiles, list.size()));   // one table slot per site, all groups
    std::vector<int> group;
    double bytes = 0;
    int toff = 0;
    for (size_t i = 0; i < list.size(); ++i) {
      const double np = (double)((ctx->sites[list[i]].npts + 127) / 128 * 128);
      const double b = 2.0 * (ctx->nf + 1) * np * kp * 2.0 + (double)ctx->nf * np * np * 4.0;
      if (!group.empty() && bytes + b > ctx->workspace_budget) {
        LRS_TRY(chi0_mixed(ctx, group, toff));
        toff += (int)group.size();
        group.clear();
        bytes = 0;
      }
      group.push_back(list[i]);
      bytes += b;
    }
    if (!group.empty()) LRS_TRY(chi0_mixed(ctx, group, toff));
  }
  for (int i : list) {
    Site& s = ctx->sites[i];
    if (ctx->precision == LRS_FP64) LRS_TRY(chi0_fp64(ctx, s));
    s.has_chi0 = true;
    s.has_w = false;
    flop += 8.0 * s.npts * (double)s.npts * (ctx->Ko + ctx->Ku) * ctx->nf;
  }
  LRS_TRY(stage_end(ctx, ST_CHI0));
  ctx->stats.flop_chi0 = flop;
  return LRS_OK;
}

// lrs_solve_w up to the device-side status check: queues the solves of the listed sites.
static int solve_w_queue(lrs_ctx* ctx, int nsite, const int* sites, std::vector<int>& list) {
  LRS_TRY(site_list(ctx, nsite, sites, list));
  for (int i : list)
    if (!ctx->sites[i].has_chi0) return set_error(LRS_ERR_STATE, "site %d has no chi0", i);
  LRS_TRY(stage_begin(ctx, ST_W));
  double flop = 0;
  const double fp64_before = ctx->fp64_flops;
  ctx->w_main_flop = 0;
  ctx->w_main_elems = 0;
  ctx->w_main_launches = 0;
  const int nl = std::min<int>(ctx->dyson_lanes, (int)list.size());
  if (nl <= 1) {
    for (int i : list) {
      Site& s = ctx->sites[i];
      if (s.fxc_kind != LRS_FXC_NONE) LRS_TRY(alda_dress(ctx, s));
      LRS_TRY(dyson_solve(ctx, s));
      s.has_w = true;
      flop += 14.0 / 3.0 * (double)s.npts * s.npts * s.npts;
    }
  } else {
    // deal the sites to the lanes by decreasing cost (the lane with the least work so far
    // takes the next), so that each lane sizes its workspace on its first site
    LRS_TRY(lanes_ready(ctx, nl));
    std::vector<int> order(list);
    auto cost = [&](int i) { return std::pow((double)ctx->sites[i].npts, 3.0); };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<std::vector<int>> dealt(nl);
    std::vector<double> load(nl, 0.0);
    for (int i : order) {
      const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      dealt[l].push_back(i);
      load[l] += cost(i);
    }
    LRS_CUDA_TRY(cudaEventRecord(ctx->ev_lanes, ctx->stream));
    for (int l = 0; l < nl; ++l) {
      if (l > 0) {
        lane_swap(ctx, ctx->lanes[l - 1]);
        cudaError_t e = cudaStreamWaitEvent(ctx->stream, ctx->ev_lanes, 0);
        if (e != cudaSuccess) {
          lane_swap(ctx, ctx->lanes[l - 1]);
          return set_error(LRS_ERR_CUDA, "cudaStreamWaitEvent: %s", cudaGetErrorString(e));
        }
      }
      int rc = LRS_OK;
      for (int i : dealt[l]) {
        Site& s = ctx->sites[i];
        if (s.fxc_kind != LRS_FXC_NONE) rc = alda_dress(ctx, s);
        if (rc == LRS_OK) rc = dyson_solve(ctx, s);
        if (rc != LRS_OK) break;
        s.has_w = true;
        flop += 14.0 / 3.0 * (double)s.npts * s.npts * s.npts;
      }
      if (l > 0) {
        cudaError_t e = cudaEventRecord(ctx->lanes[l - 1].ev_done, ctx->stream);
        lane_swap(ctx, ctx->lanes[l - 1]);
        if (rc == LRS_OK && e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->lanes[l - 1].ev_done, 0);
        if (rc == LRS_OK && e != cudaSuccess) rc = set_error(LRS_ERR_CUDA, "lane join: %s", cudaGetErrorString(e));
      }
      if (rc != LRS_OK) return rc;
    }
  }
  LRS_TRY(stage_end(ctx, ST_W));
  ctx->stats.flop_w = flop;
  ctx->stats.flop_w_executed = ctx->fp64_flops - fp64_before;
  ctx->stats.flop_w_main = ctx->w_main_flop;
  ctx->stats.w_main_elements = ctx->w_main_elems;
  ctx->stats.w_main_launches = ctx->w_main_launches;
  return LRS_OK;
}

// The status words of queued solves of `list` (waits for the context stream): a tensor-core
// kernel that gave up a bounded wait, or a zero / non-positive / non-finite pivot (the sites'
// W are then marked missing).
static int solve_w_status(lrs_ctx* ctx, const std::vector<int>& list) {
  if (ctx->capturing) return LRS_OK;   // checked after each replay by lrs_graph_launch's caller
  // zero pivots / non-finite values are reported through the status word
  int status[16] = {0};
  LRS_CUDA_TRY(cudaMemcpyAsync(status, ctx->ws.status.ptr, 16 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  ctx->stats.status_word = status[0] ? status[0] : status[8];
  if (status[8] != 0) {
    cudaMemsetAsync(ctx->ws.status.ptr + 8, 0, sizeof(int), ctx->stream);
    return set_error(LRS_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait (code %d)", status[8]);
  }
  if (status[0] != 0) {
    cudaMemsetAsync(ctx->ws.status.ptr, 0, 4 * sizeof(int), ctx->stream);
    for (int i : list) ctx->sites[i].has_w = false;
    return set_error(LRS_ERR_NUMERIC, "Dyson %s: %s pivot (status %d, column %d)",
                     status[0] == 2 ? "SPD inverse" : "LU", status[0] == 2 ? "non-positive or non-finite"
                     : "zero or non-finite", status[0], status[1]);
  }
  return LRS_OK;
}

int lrs_solve_w(lrs_ctx* ctx, int nsite, const int* sites) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  std::vector<int> list;
  LRS_TRY(solve_w_queue(ctx, nsite, sites, list));
  // solves queued earlier by lrs_solve_w_async share the status words
  list.insert(list.end(), ctx->w_pending.begin(), ctx->w_pending.end());
  ctx->w_pending.clear();
  return solve_w_status(ctx, list);
}

int lrs_solve_w_async(lrs_ctx* ctx, int nsite, const int* sites) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  std::vector<int> list;
  LRS_TRY(solve_w_queue(ctx, nsite, sites, list));
  if (!ctx->capturing) ctx->w_pending.insert(ctx->w_pending.end(), list.begin(), list.end());
  return LRS_OK;
}

static int get_matrix(lrs_ctx* ctx, int site, double* out, int which, bool device_out) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  LRS_TRY(check_site(ctx, site));
  if (!out) return set_error(LRS_ERR_ARG, "out is NULL");
  Site& s = ctx->sites[site];
  const double* src = nullptr;
  if (which == 0) { if (!s.has_chi0) return set_error(LRS_ERR_STATE, "site %d has no chi0", site); src = s.chi0.ptr; }
  if (which == 1) { if (!s.has_w) return set_error(LRS_ERR_STATE, "site %d has no W", site); src = s.w.ptr; }
  if (which == 2) {
    if (!s.has_v) {
      DeviceGuard g0(ctx->device);
      if (g0.rc) return g0.rc;
      LRS_TRY(ensure(ctx, s.v, (size_t)s.npts * s.npts));
      LRS_TRY(coulomb_build(ctx, s, s.v.ptr));
      s.has_v = true;
    }
    src = s.v.ptr;
  }
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  size_t bytes = (size_t)s.npts * s.npts * sizeof(double);
  LRS_CUDA_TRY(cudaMemcpyAsync(out, src, bytes, device_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  if (!device_out) LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return LRS_OK;
}

int lrs_get_chi0(lrs_ctx* ctx, int site, double* out) { return get_matrix(ctx, site, out, 0, false); }
int lrs_get_w(lrs_ctx* ctx, int site, double* out) { return get_matrix(ctx, site, out, 1, false); }
int lrs_get_v(lrs_ctx* ctx, int site, double* out) { return get_matrix(ctx, site, out, 2, false); }
int lrs_get_chi0_dev(lrs_ctx* ctx, int site, double* out) { return get_matrix(ctx, site, out, 0, true); }
int lrs_get_w_dev(lrs_ctx* ctx, int site, double* out) { return get_matrix(ctx, site, out, 1, true); }

int lrs_backward_dev(lrs_ctx* ctx, int site, const double* grad_w_dev, const double* grad_chi0_dev,
                     double* grad_energies_dev, double* grad_psi_dev) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  LRS_TRY(check_site(ctx, site));
  if (!grad_energies_dev || !grad_psi_dev) return set_error(LRS_ERR_ARG, "null output pointer");
  if (!grad_w_dev && !grad_chi0_dev) return set_error(LRS_ERR_ARG, "grad_w and grad_chi0 are both NULL");
  Site& s = ctx->sites[site];
  if (s.fxc_kind != LRS_FXC_NONE)
    return set_error(LRS_ERR_UNSUPPORTED, "the adjoint covers the RPA screening only (site %d has an ALDA kernel)", site);
  if (!s.has_chi0) return set_error(LRS_ERR_STATE, "site %d has no chi0", site);
  if (grad_w_dev && !s.has_w) return set_error(LRS_ERR_STATE, "site %d has no W", site);
  if (ctx->nf == 0) return set_error(LRS_ERR_STATE, "no quadrature");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  LRS_TRY(stage_begin(ctx, ST_BACKWARD));
  LRS_TRY(backward_site(ctx, s, grad_w_dev, grad_chi0_dev, grad_energies_dev,
                        reinterpret_cast<double2*>(grad_psi_dev)));
  LRS_TRY(stage_end(ctx, ST_BACKWARD));
  return LRS_OK;
}

int lrs_backward(lrs_ctx* ctx, int site, const double* grad_w, const double* grad_chi0,
                 double* grad_energies, double* grad_psi) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  LRS_TRY(check_site(ctx, site));
  if (!grad_energies || !grad_psi) return set_error(LRS_ERR_ARG, "null output pointer");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  Site& s = ctx->sites[site];
  size_t nn = (size_t)s.npts * s.npts;
  size_t ne = (size_t)ctx->nk * ctx->nb;
  double *gw = nullptr, *gc = nullptr, *ge = nullptr, *gp = nullptr;
  int rc = LRS_OK;
  if (grad_w) rc = dev_alloc_bytes(ctx, (void**)&gw, nn * sizeof(double));
  if (!rc && grad_chi0) rc = dev_alloc_bytes(ctx, (void**)&gc, nn * sizeof(double));
  if (!rc) rc = dev_alloc_bytes(ctx, (void**)&ge, ne * sizeof(double));
  if (!rc) rc = dev_alloc_bytes(ctx, (void**)&gp, ne * s.npts * sizeof(double2));
  if (!rc && gw && cudaMemcpyAsync(gw, grad_w, nn * sizeof(double), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
    rc = set_error(LRS_ERR_CUDA, "copy of grad_w failed");
  if (!rc && gc && cudaMemcpyAsync(gc, grad_chi0, nn * sizeof(double), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
    rc = set_error(LRS_ERR_CUDA, "copy of grad_chi0 failed");
  if (!rc) rc = lrs_backward_dev(ctx, site, gw, gc, ge, gp);
  if (!rc && cudaMemcpyAsync(grad_energies, ge, ne * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
    rc = set_error(LRS_ERR_CUDA, "copy of grad_energies failed");
  if (!rc && cudaMemcpyAsync(grad_psi, gp, ne * s.npts * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
    rc = set_error(LRS_ERR_CUDA, "copy of grad_psi failed");
  cudaStreamSynchronize(ctx->stream);
  if (gw) dev_free_temp(ctx, gw, nn * sizeof(double));
  if (gc) dev_free_temp(ctx, gc, nn * sizeof(double));
  if (ge) dev_free_temp(ctx, ge, ne * sizeof(double));
  if (gp) dev_free_temp(ctx, gp, ne * s.npts * sizeof(double2));
  return rc;
}

int lrs_graph_capture(lrs_ctx* ctx, int nsite, const int* sites) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (ctx->stream == nullptr)
    return set_error(LRS_ERR_STATE, "graph capture needs a non-default stream (lrs_create/lrs_set_stream)");
  // one eager build allocates every buffer, builds cached operands and checks the status words
  LRS_TRY(lrs_project(ctx, nsite, sites, ctx->graph_projection));
  LRS_TRY(lrs_build_chi0(ctx, nsite, sites));
  LRS_TRY(lrs_solve_w(ctx, nsite, sites));
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (ctx->graph_exec) {
    cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
  }
  LRS_CUDA_TRY(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  ctx->capturing = true;
  int rc = lrs_project(ctx, nsite, sites, ctx->graph_projection);
  if (rc == LRS_OK) rc = lrs_build_chi0(ctx, nsite, sites);
  if (rc == LRS_OK) rc = lrs_solve_w(ctx, nsite, sites);
  ctx->capturing = false;
  std::string err = lrs_last_error();
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
  if (rc != LRS_OK) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return set_error(rc, "while recording the graph: %s", err.c_str());
  }
  if (e != cudaSuccess) return set_error(LRS_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  // per-node priorities (the tensor-core launches carry the highest one)
  e = cudaGraphInstantiate(&ctx->graph_exec, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    ctx->graph_exec = nullptr;
    return set_error(LRS_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  return LRS_OK;
}

int lrs_graph_launch(lrs_ctx* ctx) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (!ctx->graph_exec) return set_error(LRS_ERR_STATE, "no recorded graph (lrs_graph_capture)");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  LRS_CUDA_TRY(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
  return LRS_OK;
}

int lrs_autotune(lrs_ctx* ctx, int nsite, const int* sites, int* tile_n, int* segment, double* ms_best) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  if (ctx->precision == LRS_FP64) return set_error(LRS_ERR_STATE, "autotuning applies to the mixed precisions");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  const int tns[2] = {128, 64};
  const int segs[2] = {4, 2};   // segments of at most 128 K keep the accumulation error below 1e-5
  double best = 1e300;
  int btn = ctx->chi0_tn, bseg = ctx->seg_chunks;
  cudaEvent_t e0, e1;
  LRS_CUDA_TRY(cudaEventCreate(&e0));
  LRS_CUDA_TRY(cudaEventCreate(&e1));
  int rc = LRS_OK;
  for (int tn : tns)
    for (int sg : segs) {
      ctx->chi0_tn = tn;
      ctx->seg_chunks = sg;
      rc = lrs_build_chi0(ctx, nsite, sites);   // warm-up (and allocation)
      if (rc) break;
      cudaEventRecord(e0, ctx->stream);
      for (int r = 0; r < 2 && rc == LRS_OK; ++r) rc = lrs_build_chi0(ctx, nsite, sites);
      cudaEventRecord(e1, ctx->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rc) break;
      if (ms / 2 < best) {
        best = ms / 2;
        btn = tn;
        bseg = sg;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->chi0_tn = btn;
  ctx->seg_chunks = bseg;
  if (rc) return rc;
  if (tile_n) *tile_n = btn;
  if (segment) *segment = bseg;
  if (ms_best) *ms_best = best;
  return LRS_OK;
}

int lrs_synchronize(lrs_ctx* ctx) {
  clear_error();
  if (!ctx) return set_error(LRS_ERR_ARG, "ctx is NULL");
  DeviceGuard g(ctx->device);
  if (g.rc) return g.rc;
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  int tc_status = 0;
  LRS_CUDA_TRY(cudaMemcpyAsync(&tc_status, ctx->ws.status.ptr + 8, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (tc_status != 0) {
    ctx->stats.status_word = tc_status;
    cudaMemsetAsync(ctx->ws.status.ptr + 8, 0, sizeof(int), ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    return set_error(LRS_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait (code %d)", tc_status);
  }
  if (!ctx->w_pending.empty()) {
    const std::vector<int> list = std::move(ctx->w_pending);
    ctx->w_pending.clear();
    LRS_TRY(solve_w_status(ctx, list));
  }
  for (int s = 0; s < 6; ++s)
    if (ctx->ev_pending[s]) {
      double sum = 0.0;
      for (int i = 0; i < ctx->ev_used[s]; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev_begin[s][i], ctx->ev_end[s][i]) == cudaSuccess) sum += ms;
      }
      ctx->ms_acc[s] = sum;
      ctx->ev_pending[s] = false;
    }
  ctx->stats.ms_project = ctx->ms_acc[ST_PROJECT];
  ctx->stats.ms_chi0 = ctx->ms_acc[ST_CHI0];
  ctx->stats.ms_w = ctx->ms_acc[ST_W];
  ctx->stats.ms_backward = ctx->ms_acc[ST_BACKWARD];
  ctx->stats.ms_chi0_main = ctx->ms_acc[ST_CHI0_MAIN];
  ctx->stats.ms_w_main = ctx->ms_acc[ST_W_MAIN];
  return LRS_OK;
}

int lrs_stats(lrs_ctx* ctx, lrs_stats_t* out) {
  LRS_TRY(lrs_synchronize(ctx));
  if (!out) return set_error(LRS_ERR_ARG, "out is NULL");
  *out = ctx->stats;
  return LRS_OK;
}

}  // extern "C"
