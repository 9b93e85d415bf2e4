// Internal declarations of liblrs: context layout, error helpers and the
// kernel launchers implemented in the k_*.cu translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "lrs.h"

namespace lrs {

// ---------------------------------------------------------------- errors
int set_error(int code, const char* fmt, ...);
void clear_error();

#define LRS_CUDA_TRY(call)                                                        \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return ::lrs::set_error(LRS_ERR_CUDA, "%s failed: %s (%s:%d)", #call,        \
                              cudaGetErrorString(e_), __FILE__, __LINE__);        \
  } while (0)

#define LRS_TRY(call)            \
  do {                           \
    int rc_ = (call);            \
    if (rc_ != LRS_OK) return rc_; \
  } while (0)

// Checks the launch that was just issued and counts it.
int after_launch(lrs_ctx* ctx, const char* what, int n = 1);

// ---------------------------------------------------------------- device memory
template <typename T>
struct DevBuf {
  T* ptr = nullptr;
  size_t count = 0;
};

int dev_alloc_bytes(lrs_ctx* ctx, void** p, size_t bytes);
// Frees workspace memory; a recorded graph (which may read it) is dropped.
void dev_free_bytes(lrs_ctx* ctx, void* p, size_t bytes);
// Frees a temporary of one API call (never seen by a recorded graph).
void dev_free_temp(lrs_ctx* ctx, void* p, size_t bytes);
// Drops the recorded multi-site graph, if any.
void drop_graph(lrs_ctx* ctx);

// Launches `kernel` with a launch priority attribute, which (unlike the priority
// of the stream) is kept by the node when the launch is recorded in a CUDA graph.
template <typename... KArgs, typename... Args>
cudaError_t launch_with_priority(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                 int priority, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = priority;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Host-to-device copy on the context stream, complete when the call returns (the host buffer may
// be pageable or short-lived).  Not cudaMemcpy: the legacy default stream would also wait for
// every other blocking stream of the device, e.g. another context's build.
int h2d_sync(lrs_ctx* ctx, void* dst, const void* src, size_t bytes);

template <typename T>
int ensure(lrs_ctx* ctx, DevBuf<T>& b, size_t count) {
  if (b.count >= count && b.ptr) return LRS_OK;
  if (b.ptr) dev_free_bytes(ctx, b.ptr, b.count * sizeof(T));
  b.ptr = nullptr;
  b.count = 0;
  if (count == 0) return LRS_OK;
  void* p = nullptr;
  int rc = dev_alloc_bytes(ctx, &p, count * sizeof(T));
  if (rc != LRS_OK) return rc;
  b.ptr = static_cast<T*>(p);
  b.count = count;
  return LRS_OK;
}

template <typename T>
void release(lrs_ctx* ctx, DevBuf<T>& b) {
  if (b.ptr) dev_free_bytes(ctx, b.ptr, b.count * sizeof(T));
  b.ptr = nullptr;
  b.count = 0;
}

// ---------------------------------------------------------------- state
struct Site {
  int npts = 0, lmax = 0;
  double center[3] = {0, 0, 0};
  DevBuf<double> pts, wts;          // [npts][3], [npts]
  DevBuf<double2> psi_o, psi_u;     // [npts][Ko], [npts][Ku]
  DevBuf<double> chi0, w, v;        // [npts][npts]
  bool has_psi = false, has_chi0 = false, has_w = false, has_v = false;
  // product grid p = j * nang + a (radial shell j, angular point a), if detected
  bool product = false;
  int nrad = 0, nang = 0;
  DevBuf<double> yang;              // [nang][(lmax+1)^2] real spherical harmonics
  DevBuf<double> rl;                // [lmax+1][nrad][nrad] 4pi/(2l+1) r<^l / r>^(l+1)
  DevBuf<double> fl;                // [lmax+1][nrad][nrad] lower Cholesky factor of each rl block
  bool spd = false;                 // fl exists (every rl block is positive definite)
  // ALDA vertex: kernel kind, f(r_p) [npts], dressed polarizability (I - chi0 D)^-1 chi0 [npts][npts]
  int fxc_kind = LRS_FXC_NONE;
  DevBuf<double> fxc, chi_eff;
  // polarizability the Dyson solve and the induced response use
  const double* response_chi() const { return fxc_kind != LRS_FXC_NONE ? chi_eff.ptr : chi0.ptr; }
};

// Split-precision operand planes of one matrix [rows_pad][k_pad] (4 planes:
// re_hi, re_lo, im_hi, im_lo), 16-bit elements.
struct Planes {
  DevBuf<uint16_t> data;
  int rows_pad = 0, k_pad = 0;
  size_t plane_elems() const { return (size_t)rows_pad * k_pad; }
};

// One site of a multi-site tensor-core launch: its work units are
// [unit0, unit0 + m_tiles^2 * batches).
struct SiteTile {
  int unit0;         // first global unit of the site
  int m_tiles;       // np / 128
  int n_tiles;       // np / tile width
  int np;            // padded points (rows of one A batch, leading dimension of the slab)
  int a_row0;        // first row of the site's A planes
  int b_row0;        // first row of the site's B planes
  long long slab0;   // first element of the site's output slab
  int ldc;           // leading dimension of the output (np for chi0 slabs)
  int m_valid;       // rows of the output that exist (stores beyond are skipped)
  int n_valid;       // columns of the output that exist
};

// Unit direction and radius of a grid point.
struct __align__(32) RadialUnit {
  double x, y, z, r;
};

struct Workspace {
  DevBuf<double2> denom_o, denom_u;   // [nf][Ko], [nf][Ku]
  DevBuf<double> dyson_a;             // [n][n]
  DevBuf<int> ipiv;                   // [n]
  DevBuf<double> tinv;                // inverted diagonal blocks of the LU factors
  DevBuf<int> status;                 // device status words
  DevBuf<double2> phase_tab;          // projection phase tables
  DevBuf<double2> kphase;             // [nk][npts]
  DevBuf<RadialUnit> ru;              // [npts] unit vector and radius
  // adjoint
  DevBuf<double> gamma_s;             // [n][n]
  DevBuf<double2> gbuf_o, gbuf_u;     // [n][n] per-frequency Green's functions
  DevBuf<double2> ybuf;               // [n][K]
  DevBuf<double> ge;                  // [K]
  DevBuf<double2> gpsi;               // [n][K]
  DevBuf<double2> gpart;              // [row chunks][K] partial column sums of the energy gradient
  DevBuf<double> tmp_nn;              // [n][n]
  // mixed precision (bf16 hi/lo operand planes)
  DevBuf<uint16_t> planes_a, planes_b;  // chi0: per-frequency A, frequency-independent B
  DevBuf<float> slab;                   // chi0: nf slabs of Np^2 fp32 Re[Go o Gu^T] (layout of slab_index)
  DevBuf<float2> denom32;               // chi0: [nf][Kp] scaled fp32 denominators of the A planes
  DevBuf<float2> phase_tab32;           // projection: fp32 copy of the phase tables
  DevBuf<float> tc_scratch;             // chi0: per-CTA parked occupied sums
  DevBuf<double> slab64;                // FP64 chi0: [nf][n][n] per-frequency W_f Re[Go o Gu^T]
  DevBuf<SiteTile> site_tiles;          // multi-site chi0 unit table
  // tensor-core adjoint
  DevBuf<uint16_t> planes_t;            // transposed orbital planes (B of the Y/Z products)
  DevBuf<uint16_t> planes_h;            // H, H^T planes of one frequency (A of the Y/Z products)
  DevBuf<float2> g32;                   // Go, Gu^T of one frequency
  DevBuf<float2> yz32;                  // Yo, Zo, Yu, Zu of one frequency
  DevBuf<float2> psi32;                 // the site's orbitals in fp32 (mixed adjoint)
  DevBuf<int> gamma_chk;                // Gamma-point check at load: G partners, max bits, flag
  DevBuf<SiteTile> adj_tiles;           // unit table of the adjoint launches
  DevBuf<double> gj;                    // SPD inverse: column block, signed copy, D, pivot inverse
  DevBuf<double> gjb;                   // blocked SPD inverse: C, E, D [n][128] and the pivot block
  DevBuf<uint16_t> oz_planes;           // SPD inverse on tensor cores: slice planes of D, E (two sets)
  DevBuf<int> oz_expo;                  // and their row exponents
  DevBuf<uint16_t> og_planes;           // float64-accurate tensor-core GEMM: slice planes of both operands
  DevBuf<int> og_expo;                  // and their row exponents
  DevBuf<double> induced;               // induced response: T, X, B, right-hand side, outputs
  DevBuf<double> alda_n;                // site density for the exchange-only ALDA kernel
  DevBuf<double> aug_tab;               // augmentation: pseudo waves, corrections, shell mask
  DevBuf<double2> aug_coef;             // augmentation: <phi_ps Y_lm | psi> per orbital column
  // FFT projection: grid [N1][N2][N3][nb] of one k-point (fp32 or fp64 complex), index tables, twiddles
  DevBuf<double2> fft_grid;
  DevBuf<int> fft_index;                // col_xy | col_ptr | ent_g | ent_z | populated x (offsets fft_off)
  DevBuf<double2> fft_tw;               // exp(2 pi i j / N_d), d = 1, 2, 3
  int fft_off[5] = {0, 0, 0, 0, 0};
  int fft_ncol = 0, fft_nx = 0;
  int fft_plan_n[3] = {0, 0, 0};
  bool fft_plan_ok = false;
  DevBuf<uint16_t> proj_a, proj_b;      // projection: phase planes, coefficient planes
  DevBuf<float> scales;                 // chi0: fp16 operand scales per frequency
  DevBuf<float> proj_scale;             // projection: coefficient scale and unscale
  bool coeff_planes_valid = false;
};

// Side streams and events of the SPD inverse (spd_inverse, k_linalg.cu): the
// pivot chain, the write-back of exchanged blocks, the rest of each panel.
enum SpdEvent : int {
  SPD_FORK = 0, SPD_JOIN2, SPD_JOIN3, SPD_JOIN4,
  SPD_PIVOT, SPD_ADIAG = SPD_PIVOT + 2, SPD_GREST = SPD_ADIAG + 2, SPD_AREST = SPD_GREST + 2,
  SPD_BULK = SPD_AREST + 2, SPD_FIX = SPD_BULK + 2, SPD_EVENTS = SPD_FIX + 2   // pairs alternate by block parity
};
struct SpdStreams {
  cudaStream_t s2 = nullptr, s3 = nullptr, s4 = nullptr;
  cudaEvent_t ev[SPD_EVENTS] = {};
};

// Streams, events and Dyson-solve workspace of one lane of lrs_solve_w: the
// sites of one call are spread over lanes whose solves run concurrently
// (lane 0 is the context's own stream and workspace).
struct DysonLane {
  cudaStream_t s1 = nullptr;
  SpdStreams spd;
  cudaEvent_t ev_done = nullptr;
  DevBuf<double> dyson_a, tinv, gj, gjb, alda_n;
  DevBuf<int> ipiv, oz_expo, og_expo;
  DevBuf<uint16_t> oz_planes, og_planes;
  DevBuf<RadialUnit> ru;
};

}  // namespace lrs

struct lrs_ctx {
  int device = 0;
  int precision = LRS_FP64;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int seg_chunks = 4;                  // chi0 tensor-core accumulation segment (K chunks of 32)
  int proj_seg_chunks = 2;             // projection accumulation segment (K chunks of 32)
  int dyson_basis = LRS_DYSON_AUTO;    // full grid or lm basis
  int dyson_solver = LRS_SOLVER_AUTO;  // lm basis: LU of I - C X, or the SPD inverse
  int dyson_update = LRS_UPDATE_AUTO;  // trailing update of the SPD inverse: FP64 pipe or tensor cores
  int chi0_tn = 128;                   // chi0 tensor-core tile width (64 or 128)
  int fft_n[3] = {0, 0, 0};            // FFT grid of the method-2 projection (0: automatic)
  int graph_projection = LRS_PROJ_EXACT;  // projection mode recorded by lrs_graph_capture
  bool real_orbitals = false;          // one k-point at Gamma with C(-G) = conj C(G): orbitals are real
  int real_mode = LRS_REAL_AUTO;       // use the real-orbital contractions when the orbitals are real
  double workspace_budget = 48e9;      // bytes of chi0 operand planes + slabs per launch
  bool capturing = false;              // a CUDA graph is being recorded on the stream
  int dyson_lanes = 4;                 // concurrent Dyson solves of one lrs_solve_w call
  std::vector<int> w_pending;          // sites of queued lrs_solve_w_async calls (status not read yet)
  std::vector<lrs::DysonLane> lanes;   // lanes 1.. (lane 0 is the context itself)
  cudaEvent_t ev_lanes = nullptr;      // fork of the lanes from the context stream

  // orbitals
  bool has_orb = false;
  int nk = 0, ng = 0, nb = 0, Ko = 0, Ku = 0;
  std::vector<int> nocc;
  double cell[9], recip[9], omega = 0;
  std::vector<double> kpts, kw, energies;
  bool energies_on_device_only = false;  // set by lrs_set_energies_dev: host copy read back when needed
  std::vector<int> gvec;
  int gmax_idx[3] = {0, 0, 0};
  lrs::DevBuf<double2> coeff;          // [nk][ng][nb]
  lrs::DevBuf<int> d_gvec;             // [ng][3]
  lrs::DevBuf<double> d_kpts;          // [nk][3]
  lrs::DevBuf<double> e_o, e_u, w_o, w_u;  // per internal column
  std::vector<int> col_o, col_u;       // internal column -> public column (k*nb + b)
  lrs::DevBuf<int> d_col_o, d_col_u;

  // quadrature
  int nf = 0;
  double mu = 0, zeta = 0;
  std::vector<double> t, W;
  lrs::DevBuf<double> d_t, d_W;        // [nf] on the device

  std::vector<lrs::Site> sites;
  lrs::Workspace ws;
  std::vector<lrs::SiteTile> site_tiles_host;
  std::vector<lrs::SiteTile> site_tiles_dev;   // copy of the table last uploaded
  const lrs::SiteTile* site_tiles_dev_ptr = nullptr;
  cudaGraphExec_t graph_exec = nullptr;        // recorded multi-site build
  // side streams of the SPD inverse (higher priority) and their events
  lrs::SpdStreams spd;
  int prio_greatest = 0;               // numerically smallest (highest) stream priority of the device

  lrs_stats_t stats{};
  double fp64_flops = 0;               // running count of FP64 flop issued by the linear algebra
  double w_main_flop = 0;              // algorithmic flop of the SPD-inverse bulk updates of the last solve
  double w_main_elems = 0;             // lower-triangle elements those updates rewrote (summed over launches)
  bool spd_inner = false;              // an spd_inverse inside the blocked one: its updates are not "main"
  int dyson_panel = 0;                 // LRS_OPT_DYSON_PANEL: 0 auto, 32 or SPD_OUTER_BLOCK
  int64_t w_main_launches = 0;
  // stage timing: event pairs of the stage's intervals since its last reset
  // (the main chi0 kernel runs once per workspace group of one build)
  std::vector<cudaEvent_t> ev_begin[6], ev_end[6];
  int ev_used[6] = {};
  bool ev_pending[6] = {};
  double ms_acc[6] = {};
};

namespace lrs {

enum Stage { ST_PROJECT = 0, ST_CHI0 = 1, ST_W = 2, ST_BACKWARD = 3, ST_CHI0_MAIN = 4, ST_W_MAIN = 5 };
int stage_begin(lrs_ctx* ctx, Stage s);
// Creates the side streams of the SPD inverse and their events on first use.
int aux_stream_ready(lrs_ctx* ctx);
int stage_end(lrs_ctx* ctx, Stage s);

// ---------------------------------------------------------------- launchers
// Projection (k_project.cu)
int project_fp64(lrs_ctx* ctx, Site& s);
int project_mixed(lrs_ctx* ctx, Site& s);
// Method 2 (k_fft.cu): FFT to the cell grid + 3rd-degree Lagrange interpolation, all listed sites.
int project_fft(lrs_ctx* ctx, const std::vector<int>& sites);
int fft_grid_dims(lrs_ctx* ctx, int n[3]);
bool fft_length_ok(int n);

// Denominators d[f][col] = w/(mu + i t_f - eps) (k_chi0_fp64.cu)
int build_denominators(lrs_ctx* ctx);

// FP64 chi0 (k_chi0_fp64.cu): S accumulated into s.chi0, then symmetrised.
int chi0_fp64(lrs_ctx* ctx, Site& s);
int symmetrize_chi0(lrs_ctx* ctx, double* chi0, int n);

// Mixed chi0 on tcgen05 (k_chi0_tc.cu)
// One launch for all listed sites; `toff` is the group's offset in the device site table.
int chi0_mixed(lrs_ctx* ctx, const std::vector<int>& sites, int toff);

// Coulomb operator (k_coulomb.cu)
int coulomb_build(lrs_ctx* ctx, Site& s, double* v);

// FP64 linear algebra (k_linalg.cu)
int dgemm(lrs_ctx* ctx, int m, int n, int k, double alpha, const double* a, int lda,
          const double* kscale, const double* b, int ldb, const double* cscale, double beta,
          double* c, int ldc);
int dyson_solve(lrs_ctx* ctx, Site& s);
int dgemm_t(lrs_ctx* ctx, bool ta, bool tb, int m, int n, int k, double alpha, const double* a, int lda,
            const double* ks, const double* b, int ldb, const double* cs, double beta, double* c, int ldc);
int dgemm_batched(lrs_ctx* ctx, bool ta, bool tb, int m, int n, int k, double alpha, const double* a, int lda,
                  long long stride_a, const double* ks, long long stride_ks, const double* b, int ldb,
                  long long stride_b, const double* cs, double beta, double* c, int ldc, long long stride_c,
                  int batch);
// Column blocks j of a symmetric C (C + j n, width n): only tiles on or below
// the diagonal; alpha = 1, beta = 0.
int dgemm_batched_lower(lrs_ctx* ctx, bool ta, bool tb, int m, int n, int k, const double* a, int lda,
                        long long stride_a, const double* ks, long long stride_ks, const double* b, int ldb,
                        double* c, int ldc, int batch);
// Upper triangle of a symmetric matrix from its lower triangle.
int mirror_lower(lrs_ctx* ctx, double* a, int n, int lda);
int lu_factor(lrs_ctx* ctx, double* A, int n, int* ipiv, int* status);
int lu_solve(lrs_ctx* ctx, const double* LU, int n, const int* ipiv, double* B, int nrhs, int ldb);
int lu_solve_inv(lrs_ctx* ctx, const double* LU, int n, const int* ipiv, double* B, int nrhs, int ldb,
                 double* tinv);
// Tensor-core float64-accurate rank-32 update (k_ozaki.cu; the slices come from
// oz_slice_row, oz_slice.cuh): maps over the slice planes; C -= D E^T on the lower
// triangle outside rows and columns [x0, x1).
int oz_make_maps(lrs_ctx* ctx, const uint16_t* dplanes, const uint16_t* eplanes, int rows_pad, CUtensorMap* md,
                 CUtensorMap* me);
int oz_update(lrs_ctx* ctx, const CUtensorMap& md, const CUtensorMap& me, double* C, int n, int ldc,
              const int* ed, const int* ee, int x0, int x1, int rows_pad, cudaStream_t stream);
int oz_rows_pad(int n);
size_t oz_plane_elems(int n);
// Float64-accurate batched GEMM on the tensor cores (k_ozgemm.cu), the
// arguments of dgemm_batched (no column scale); lower_col > 0 computes only
// the tiles of C_b = C + b lower_col that reach the lower triangle of a
// symmetric matrix, as dgemm_batched_lower.
int oz_gemm_batched(lrs_ctx* ctx, bool ta, bool tb, int m, int n, int k, double alpha, const double* a, int lda,
                    long long stride_a, const double* ks, long long stride_ks, const double* b, int ldb,
                    long long stride_b, double beta, double* c, int ldc, long long stride_c, int batch,
                    int lower_col);
// The same GEMM on strided operands: for batch entries b < batch, i < m, j < n,
//   C[b c.sb + i c.rs + j c.cs] = c.alpha sum_kk A(b, i, kk) ks_b[kk] B(b, j, kk) + c.beta C[...]
//                                 + c.dadd [i c.dI + j c.dJ + b c.dB == 0],
// A(b, i, kk) = a.x[b a.sb + i a.si + kk a.sk] and B(b, j, kk) = b.x[b' b.sb + j b.si + kk b.sk]
// with b' = floor(sqrt(b)) when b.sqrt_batch (one radial factor per l serving its 2l + 1 lm
// entries), else b' = b.  A stride of 0 shares one operand between all entries.
struct OzOperand {
  const double* x;
  long long si, sk, sb;
  bool sqrt_batch;
};
struct OzStore {
  double* c = nullptr;
  long long rs = 0, cs = 1, sb = 0;
  double alpha = 1.0, beta = 0.0;
  int dI = 0, dJ = 0, dB = 0;
  double dadd = 0.0;
  bool batch_fastest = false;
  int lower_col = 0;
};
int oz_gemm_strided(lrs_ctx* ctx, int m, int n, int k, int batch, const OzOperand& a, const double* ks,
                    long long stride_ks, const OzOperand& b, const OzStore& c);

// In-place inverse of an SPD matrix; lower triangle in and out.  status[0] = 2
// (status[1] = column) on a pivot that is not positive and finite.
int spd_inverse(lrs_ctx* ctx, double* A, int n, int lda, int* status);
// The same inverse with SPD_OUTER_BLOCK-wide pivot blocks (k_spd_blocked.cu): the 32-wide inverse
// of each pivot block, then D = C P and the trailing update on the float64-accurate tensor-core GEMM.
constexpr int SPD_OUTER_BLOCK = 128;
int spd_inverse_blocked(lrs_ctx* ctx, double* A, int n, int lda, int* status);

// lm-basis Dyson on product grids (k_dyson_lm.cu)
int site_detect_product(lrs_ctx* ctx, Site& s, const double* pts_host);
int dyson_solve_lm(lrs_ctx* ctx, Site& s);

// ALDA (k_alda.cu): density n = 2 sum w |psi_o|^2 into n_dev [npts]; kernel f of the site
// (s.fxc); chi_eff = (I - chi0 diag(f w))^-1 chi0 into s.chi_eff.
int site_density(lrs_ctx* ctx, Site& s, double* n_dev);
int site_fxc(lrs_ctx* ctx, Site& s);
int alda_dress(lrs_ctx* ctx, Site& s);

// Augmentation of the site orbitals in place (k_augment.cu); phi_* host [lmax_aug+1][nnu][nrad].
int augment_site(lrs_ctx* ctx, Site& s, int lmax_aug, int nnu, double r_aug, const double* phi_ae,
                 const double* phi_ps);

// Induced density / potential of a screened short-range spherical potential (k_induced.cu);
// host outputs (rho_lm, vind_lm: [nrad][(lresp+1)^2]; grid: [npts]), each may be NULL.
int induced_potential(lrs_ctx* ctx, Site& s, double q, double rs, int lresp, double* rho_lm, double* vind_lm,
                      double* vind_grid);

// Adjoint (k_adjoint.cu: float64; k_tc.cu: tensor-core version for the mixed precisions)
int backward_site(lrs_ctx* ctx, Site& s, const double* grad_w_dev, const double* grad_chi0_dev,
                  double* grad_e_dev, double2* grad_psi_dev);
int backward_site_mixed(lrs_ctx* ctx, Site& s, const double* grad_w_dev, const double* grad_chi0_dev,
                        double* grad_e_dev, double2* grad_psi_dev);
int gamma_s_build(lrs_ctx* ctx, Site& s, const double* grad_w_dev, const double* grad_chi0_dev);
// ge[b] += Re[e_b d_b^2 / w_b], e_b the sum over `chunks` row chunks of part[chunk][b] (fixed order).
int grad_energy(lrs_ctx* ctx, const double2* part, int chunks, const double2* d, const double* w, int K,
                double* ge);
int scatter_gradients(lrs_ctx* ctx, int n, const double2* gpo, const double2* gpu, const double* ge,
                      double* grad_e, double2* grad_psi);

}  // namespace lrs
