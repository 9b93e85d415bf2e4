/*
 * lrs.h - C-ABI of the GB300 local real-space screening library (liblrs.so).
 *
 * The library computes, for atom-centred site grids, the static RPA
 * polarizability chi0(r, r') and the screened interaction W = v + v chi0 W of
 * Vinson & Shirley, "Fast, efficient, and accurate dielectric screening using
 * a local, real-space approach", and the adjoint of that map.
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: LRS_OK (0) or one of the
 *     LRS_ERR_* codes below.  No function aborts, throws or traps.  After a
 *     failure lrs_last_error() returns a human-readable message for the
 *     calling thread (valid until that thread's next call).
 *   - Host pointers passed in are read during the call only and stay owned by
 *     the caller; the library copies what it needs into device memory that it
 *     allocates and owns until lrs_destroy().  Host output buffers are
 *     written before the call returns.  Device pointers ("_dev" entry points)
 *     are caller-owned, must be on the context's device and are accessed in
 *     stream order on the context's stream.
 *   - Matrices are row-major.  Complex numbers are interleaved (re, im)
 *     float64 pairs.  Site grids index points p = 0 .. npts-1 and, for
 *     product grids, p = radial_shell * nang + angular_point.
 *   - Orbital columns are ordered (k outer, band inner); within each k the
 *     nocc[k] occupied bands come first.
 *   - Units: Hartree atomic units (bohr, Hartree).
 *   - A context is not thread-safe; distinct contexts may be used from
 *     distinct threads.
 */
#ifndef LRS_H
#define LRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LRS_OK            0
#define LRS_ERR_ARG       1   /* invalid argument (null pointer, size, range) */
#define LRS_ERR_OOM       2   /* device allocation failed */
#define LRS_ERR_CUDA      3   /* a CUDA runtime/driver call failed */
#define LRS_ERR_STATE     4   /* call made out of order (e.g. build before load) */
#define LRS_ERR_TIMEOUT   5   /* a bounded device-side wait gave up */
#define LRS_ERR_NUMERIC   6   /* non-finite value or exactly zero pivot */
#define LRS_ERR_UNSUPPORTED 7 /* mode not available on this device/build */

/* arithmetic of the Green's-function contractions (chi0, adjoint, projection) */
#define LRS_FP64          0   /* float64 throughout */
#define LRS_MIXED_BF16X3  1   /* bf16 hi+lo split operands, 3 products, fp32 accumulation */
#define LRS_MIXED_FP16X3  2   /* fp16 hi+lo split operands (power-of-two scaled), fp32 accumulation */

/* projection modes */
#define LRS_PROJ_EXACT    0   /* direct Fourier sum, Sec. VI.B method 1 */
#define LRS_PROJ_FFT_LAGRANGE3 1 /* FFT to the cell grid, 3rd-degree Lagrange interpolation, Sec. VI.B method 2 */
#define LRS_FFT_MAX_N   256   /* largest FFT length per lattice direction */

/* options (lrs_set_option) */
#define LRS_OPT_DYSON_BASIS      1  /* value: LRS_DYSON_AUTO, LRS_DYSON_FULL or LRS_DYSON_LM */
#define LRS_OPT_CHI0_SEGMENT     2  /* value: K chunks of 32 per tensor-core accumulation segment (1..1024) */
#define LRS_OPT_PROJ_SEGMENT     3  /* same for the mixed-precision projection */
#define LRS_OPT_CHI0_TILE_N      4  /* value: 64 or 128 grid points per tensor-core tile column */
#define LRS_OPT_WORKSPACE_GB     5  /* value: GB of chi0 operand planes per launch (sites are grouped; default 48) */
#define LRS_DYSON_AUTO    0   /* lm basis when the site grid is a radial x angular product that it shrinks */
#define LRS_DYSON_FULL    1   /* LU on the full npts x npts grid matrix */
#define LRS_DYSON_LM      2   /* LU in the (radial shell, l, m) basis (product grids only) */
#define LRS_OPT_DYSON_SOLVER     6  /* value: LRS_SOLVER_AUTO, LRS_SOLVER_LU or LRS_SOLVER_SPD (lm basis) */
#define LRS_SOLVER_AUTO   0   /* SPD inverse when every radial Coulomb block has a Cholesky factor, else LU */
#define LRS_SOLVER_LU     1   /* LU with partial pivoting of I - C X, C as right-hand sides */
#define LRS_SOLVER_SPD    2   /* Z = F (I - F^T X F)^-1 F^T with C = F F^T (LRS_ERR_STATE if C has no factor) */
/* exchange-correlation kernel of the ALDA vertex (lrs_set_fxc) */
#define LRS_FXC_NONE      0   /* RPA */
#define LRS_FXC_USER      1   /* f(r_p) = dv_xc/dn at n(r_p), supplied per grid point */
#define LRS_FXC_ALDA_X    2   /* exchange-only ALDA of the site density: f = -(1/3)(3/pi)^(1/3) n^(-2/3) */
#define LRS_OPT_GRAPH_PROJECTION 7  /* value: LRS_PROJ_EXACT (default) or LRS_PROJ_FFT_LAGRANGE3, recorded by lrs_graph_capture */
#define LRS_OPT_REAL_ORBITALS    8  /* value: LRS_REAL_AUTO (default) or LRS_REAL_OFF */
#define LRS_OPT_DYSON_UPDATE     9  /* value: LRS_UPDATE_AUTO (default), LRS_UPDATE_FP64 or LRS_UPDATE_TC */
#define LRS_OPT_DYSON_LANES     10  /* value: 1..8 concurrent Dyson solves in one lrs_solve_w call (default 4) */
#define LRS_OPT_DYSON_PANEL     11  /* value: 0 (auto), 32 or 128: pivot-block width of the lm-basis SPD inverse */
#define LRS_UPDATE_AUTO   0   /* tensor cores in the mixed precisions, the FP64 pipe in LRS_FP64 */
#define LRS_UPDATE_FP64   1   /* lm-basis Dyson products (basis changes, radial blocks, SPD updates) with float64 FMAs */
#define LRS_UPDATE_TC     2   /* the same products float64-accurate from exact bf16 slices on the tensor cores */
#define LRS_REAL_AUTO     0   /* Gamma-point real orbitals (Sec. VI.F) use real-operand tensor-core contractions */
#define LRS_REAL_OFF      1   /* always the complex contractions */

typedef struct lrs_ctx lrs_ctx;

typedef struct lrs_stats_t {
  double ms_project;      /* device time of the last lrs_project call */
  double ms_chi0;         /* device time of the last lrs_build_chi0 call */
  double ms_w;            /* device time of the last lrs_solve_w call */
  double ms_backward;     /* device time of the last lrs_backward call */
  double ms_chi0_main;    /* device time of the main contraction kernel(s) of the last lrs_build_chi0 */
  double flop_chi0;       /* algorithmic flop of the last lrs_build_chi0: sum 8 npts^2 K nfreq */
  double flop_w;          /* algorithmic flop of the last lrs_solve_w: sum 14/3 npts^3 */
  int64_t kernel_launches;/* kernels launched by this context since creation */
  int64_t device_bytes;   /* device memory currently held by the context */
  int64_t device_bytes_peak;
  int status_word;        /* last device-side status (0 = ok) */
  double flop_w_executed; /* float64 flop actually executed by the last lrs_solve_w (GEMM, TRSM, LU) */
  double ms_w_main;       /* device time of the SPD-inverse trailing-update launches of the last lrs_solve_w */
  double flop_w_main;     /* their algorithmic flop: 2 kb x (lower-triangle elements updated), summed */
  int64_t w_main_launches;/* how many such launches */
  double w_main_elements; /* lower-triangle elements they rewrote, summed over the launches */
} lrs_stats_t;

/* Last error message of the calling thread ("" if none). */
const char* lrs_last_error(void);

/* Library version string. */
const char* lrs_version(void);

/*
 * Create a context on CUDA device `device`.  `precision` is LRS_FP64,
 * LRS_MIXED_BF16X3 or LRS_MIXED_FP16X3 and selects the arithmetic of the
 * projection, chi0 and adjoint contractions; energy denominators, frequency
 * accumulation, the Coulomb operator and the Dyson LU are float64 in every
 * mode.  `stream` is a cudaStream_t (NULL = legacy default stream) on which
 * all work of the context is issued.
 * Errors: LRS_ERR_ARG (null ctx, bad precision), LRS_ERR_CUDA.
 */
int lrs_create(lrs_ctx** ctx, int device, int precision, void* stream);

/* Free every device buffer and the context (NULL is accepted). */
int lrs_destroy(lrs_ctx* ctx);

/* Change the stream of an existing context (same device). */
int lrs_set_stream(lrs_ctx* ctx, void* stream);

/*
 * Tuning and algorithm options (LRS_OPT_*).  LRS_OPT_DYSON_BASIS selects how
 * the Dyson equation is solved: on the full grid, or - for product grids
 * p = shell * nang + angular point with the same angular set on every shell -
 * in the basis of radial shells x real spherical harmonics l <= L where the
 * multipole Coulomb operator is block diagonal (Sec. VI.E).  Both give the
 * same W up to rounding.  In the lm basis, with X = Y^T Q chi0 Q Y and the
 * block-diagonal Coulomb matrix C, the Dyson equation reads (I - C X) Z = C.
 * LRS_OPT_DYSON_SOLVER chooses LU with partial pivoting for it, or - since C
 * is positive definite (C = F F^T, F its Cholesky factor per l) and chi0 is
 * negative semidefinite - the symmetric form Z = F (I - F^T X F)^-1 F^T, whose
 * matrix has every eigenvalue >= 1 and is inverted in place by blocked
 * Gauss-Jordan steps without pivoting (n^3 instead of 8/3 n^3 flop).
 * LRS_OPT_DYSON_UPDATE selects the arithmetic of that inverse's rank-32
 * trailing updates: float64 FMAs, or the tensor cores on operands cut into
 * seven exact bf16 slices per row (power-of-two row scales), 28 slice products
 * accumulated per level exactly in fp32 and combined in float64 - an error
 * bound of about 6e-16 of |D|max |E|max per element, as for a float64 dot
 * product of 32 terms.  The same switch moves the basis changes (Y^T Q chi0 Q Y,
 * Y Z Y^T) and the four radial-block products of the SPD form (F^T X F and
 * F M^-1 F^T, one GEMM per lm over the radial index) between the two
 * arithmetics; on the tensor cores they use eight slices per row.
 * LRS_OPT_DYSON_PANEL sets the width of the pivot blocks the SPD inverse
 * exchanges at a time: 32, or 128 - the 128 x 128 pivot block inverted by the
 * 32-wide steps, then D = C P and the rank-128 trailing update float64-accurate
 * on the tensor cores (eight exact bf16 slices per row), so that the trailing
 * matrix is rewritten once per 128 pivots.  Exchanging a block at once equals
 * exchanging its parts in turn.  0 (default) and 32 take the 32-wide exchange,
 * whose trailing updates overlap the serial pivot chain (measured faster on
 * the 3520-point and 64-site workloads).
 * LRS_OPT_DYSON_LANES sets how many sites of one lrs_solve_w call are solved
 * concurrently, each on its own streams and workspace (sites are dealt to the
 * lanes by decreasing cost); a single site's serial pivot chain then overlaps
 * the others' bulk updates.  Each lane holds the workspace of its largest site.
 * Errors: LRS_ERR_ARG (unknown option or value).
 */
int lrs_set_option(lrs_ctx* ctx, int option, int value);

/*
 * Load Bloch coefficients and band energies (Eq. (bloch), Sec. VI.A-B).
 *   cell[9]          lattice vectors a1, a2, a3 as rows (bohr)
 *   nk, kpts[nk*3]   k-points, cartesian (bohr^-1)
 *   kweights[nk]     k-point weights w_k of the Brillouin-zone sum (Sec. VI.D), sum 1
 *   ng, gvec[ng*3]   plane waves as integer multiples of the reciprocal vectors
 *   nbands, nocc[nk] bands per k and how many of them are occupied (0 < nocc < nbands)
 *   coeff            [nk][ng][nbands] complex C_kb(G); psi_kb(r) =
 *                    Omega^-1/2 sum_G C_kb(G) exp(i (k+G).r)
 *   energies         [nk][nbands] band energies (occupied first)
 * Replaces any previous orbitals and invalidates projected site orbitals.
 * Errors: LRS_ERR_ARG, LRS_ERR_OOM, LRS_ERR_CUDA.
 */
int lrs_load_orbitals(lrs_ctx* ctx, const double* cell, int nk, const double* kpts,
                      const double* kweights, int ng, const int* gvec, int nbands,
                      const int* nocc, const double* coeff, const double* energies);

/*
 * Replace the band energies [nk][nbands] (same layout as in lrs_load_orbitals)
 * without touching coefficients or projected orbitals, e.g. for a scissor
 * shift.  The frequency quadrature (mu, t_i, W_i) is kept as it is; chi0 and
 * W of every site become stale.  Errors: LRS_ERR_STATE, LRS_ERR_ARG.
 */
int lrs_set_energies(lrs_ctx* ctx, const double* energies);

/*
 * Define the site grids (Sec. VI.A, App. D.1).
 *   centers[nsites*3]  site centres tau (bohr)
 *   npts[nsites]       points per site
 *   pts                concatenation over sites of [npts][3] offsets r - tau (bohr, nonzero)
 *   wts                concatenation over sites of [npts] integration weights (include r^2,
 *                      angular weights summing to 4 pi)
 *   lmax[nsites]       multipole cutoff L of the Coulomb operator (Sec. VI.E), 0..64
 * Replaces any previous sites.
 * Errors: LRS_ERR_ARG (npts < 1, point at the origin, lmax out of range), LRS_ERR_OOM.
 */
int lrs_set_sites(lrs_ctx* ctx, int nsites, const double* centers, const int* npts,
                  const double* pts, const double* wts, const int* lmax);

/*
 * Imaginary-frequency quadrature of Eq. (chi1) (App. D.1, single-grid map):
 * nf Gauss-Legendre points a_i, weights w_i on [0,1], t_i = zeta a_i/(1-a_i),
 * W_i = zeta w_i/(1-a_i)^2.  mu: chemical potential (NaN = mid-gap over all k).
 * zeta <= 0 selects the rule of App. D.1: geometric mean of the smallest and
 * largest |mu - eps| with 0.5 eV added in quadrature to the smallest.
 * mu_out/zeta_out (may be NULL) receive the values used.  nf in 1..128.
 * Requires orbitals.  Errors: LRS_ERR_ARG, LRS_ERR_STATE.
 */
int lrs_set_frequency_quadrature(lrs_ctx* ctx, int nf, double mu, double zeta,
                                 double* mu_out, double* zeta_out);

/* Read back the quadrature nodes t[nf] and weights W[nf] (host, may be NULL). */
int lrs_get_frequency_quadrature(lrs_ctx* ctx, double* t, double* w);

/*
 * Project the orbitals onto the grids of `nsite` sites (`sites` = NULL means
 * all), psi_kb(tau + r_p), by
 *   LRS_PROJ_EXACT          the direct Fourier sum (Eq. (bloch), Sec. VI.B
 *                           method 1), a complex contraction over G in the
 *                           context's precision;
 *   LRS_PROJ_FFT_LAGRANGE3  Sec. VI.B method 2: u_kb on the grid x_m =
 *                           sum_i (m_i / N_i) a_i by inverse FFT of C_kb(G)
 *                           (fp32 in mixed contexts, float64 in LRS_FP64),
 *                           3rd-degree Lagrange interpolation through the
 *                           nodes floor(s_i) - 1 .. floor(s_i) + 2 of each
 *                           lattice direction (s_i = N_i times the
 *                           fractional coordinate, indices periodic), then
 *                           exp(i k.r) / sqrt(Omega).  An approximation whose
 *                           error falls as N^-4 (lrs_set_fft_grid).  Device
 *                           memory: one grid N1 N2 N3 nbands complex.
 * Errors: LRS_ERR_STATE (no orbitals/sites), LRS_ERR_ARG (grid cannot hold
 * the G set), LRS_ERR_UNSUPPORTED (unknown mode, no FFT length), LRS_ERR_OOM.
 */
int lrs_project(lrs_ctx* ctx, int nsite, const int* sites, int mode);

/*
 * All-electron augmentation of the projected site orbitals (Sec. VI.C,
 * Eq. (eq-aug1) and (eq-aug2)), in place, for every orbital column:
 *   psi <- psi + sum_{l <= lmax_aug, m} sum_{nu,nu'} Y_lm [phi_ae_{nu l} - phi_ps_{nu l}]
 *               (A_l^-1)_{nu nu'} <phi_ps_{nu' l} Y_lm | psi>,
 *   A_{nu nu'; l} = int_0^{r_aug} dr r^2 phi_ps_{nu l} phi_ps_{nu' l},
 * the radial integral taken by the grid's radial quadrature over the shells
 * with r_j <= r_aug and the projection by the point weights on those shells
 * (Y_lm the real harmonics of lrs_induced_potential).  phi_ae, phi_ps: host
 * [lmax_aug + 1][nnu][nrad] radial functions on the site's shells (for
 * example optimal projector functions; an atom at the site centre).
 * Requires projected orbitals and a product grid; invalidates chi0 and W.
 * Errors: LRS_ERR_ARG (lmax_aug > lmax, nnu outside [1, 64], radius, non-finite
 * values), LRS_ERR_STATE (no orbitals, during capture), LRS_ERR_UNSUPPORTED
 * (not a product grid), LRS_ERR_NUMERIC (singular overlap A_l).
 */
int lrs_augment(lrs_ctx* ctx, int site, int lmax_aug, int nnu, double r_aug, const double* phi_ae,
                const double* phi_ps);

/*
 * ALDA vertex correction (Sec. VII "Beyond RPA screening", Eq. (chi-alda)
 * and (kxc_alda)): chi~ = (1 - chi0 (v + f_xc))^-1 chi0 with the contact
 * kernel f_xc(r, r') = delta(r - r') f(r).  Once set for a site, lrs_solve_w
 * returns W~ = v + v chi~ v and lrs_induced_potential screens with chi~; both
 * use the dressed polarizability chi_eff = (I - chi0 diag(f w))^-1 chi0
 * (an FP64 LU with npts right-hand sides) in the RPA Dyson solve of either
 * basis.  lrs_get_chi0 still returns chi0.  kind LRS_FXC_USER takes f
 * (Ha bohr^3, host [npts]) from `fxc`; LRS_FXC_ALDA_X computes the
 * exchange-only kernel from the density of the site orbitals at each solve;
 * LRS_FXC_NONE returns to the RPA.  The correlation parametrisations the
 * paper uses are not built in (pass them through LRS_FXC_USER).  The adjoint
 * (lrs_backward) refuses sites with a kernel (LRS_ERR_UNSUPPORTED).
 * Invalidates the site's W.  Errors: LRS_ERR_ARG.
 */
int lrs_set_fxc(lrs_ctx* ctx, int site, int kind, const double* fxc);

/*
 * Whether the loaded orbitals are real (Sec. VI.F, Gamma point with
 * time-reversal symmetry): one k-point at k = 0, the G set closed under
 * G -> -G and C_b(-G) = conj C_b(G) for every band (to 1e-12 of max |C|).
 * Then psi is real, the B operand of the Green's-function products is real and
 * the mixed-precision chi0 issues half the tensor-core products (unless
 * LRS_OPT_REAL_ORBITALS is LRS_REAL_OFF).  Errors: LRS_ERR_ARG, LRS_ERR_STATE.
 */
int lrs_orbitals_are_real(lrs_ctx* ctx, int* is_real);

/* Electron density n(r_p) = 2 sum_k w_k sum_occ |psi_kv(r_p)|^2 of the site
 * orbitals (host [npts]).  Errors: LRS_ERR_ARG, LRS_ERR_STATE (no orbitals). */
int lrs_get_density(lrs_ctx* ctx, int site, double* n);

/* The kernel f(r_p) a solve would use now (host [npts]).
 * Errors: LRS_ERR_ARG, LRS_ERR_STATE (no kernel set, no orbitals). */
int lrs_get_fxc(lrs_ctx* ctx, int site, double* fxc);

/*
 * Whether site `site` was recognised as a radial x angular product grid
 * (p = shell * nang + a, the same directions on every shell) and its shape;
 * nrad = nang = 0 otherwise.  Any output may be NULL.  Errors: LRS_ERR_ARG.
 */
int lrs_site_grid_shape(lrs_ctx* ctx, int site, int* product, int* nrad, int* nang);

/*
 * Induced density and potential of a screened spherical short-range potential
 * at the site centre (the core-hole response of Sec. VI.E).  The potential is
 * the short-range part of Eq. (eq-partition) for v_ext = q / r:
 *   v1(r) = q (1/r - 1/R_S) for r < R_S (shell_radius), 0 beyond.
 * With chi0 of the site expanded in real spherical harmonics Y_lm, l <= lresp
 * (Y_l^0, sqrt(2) Re Y_l^m for m > 0, sqrt(2) Im Y_l^|m| for m < 0, Y_l^m the
 * complex harmonics with the Condon-Shortley phase; index l^2 + l + m), the
 * paper's S = I - chi0_lm v and chi = S^-1 chi0_lm are formed with every
 * radial integral taken by the grid's radial quadrature, and
 *   rho_lm(r_j)   = int d^3r' chi_(lm;00)(r_j, r') v1(r')      (sqrt(4 pi) Y_00 v1)
 *   v_ind_lm(r_j) = int dr r^2 rho_lm(r) 4 pi/(2l+1) r_<^l / r_>^(l+1)
 * lresp = 0 is the paper's default; lresp = L (the site's lmax) keeps every l
 * and then equals v Q chi Q v1 of the full-grid Dyson equation.
 * Requires chi0 (lrs_build_chi0) and a product grid; FP64 in every precision.
 * Outputs (host, each may be NULL): rho_lm and vind_lm [nrad][(lresp+1)^2],
 * vind_grid [npts] = sum_lm v_ind_lm(r_j) Y_lm(Omega_a).  Synchronous.
 * Errors: LRS_ERR_ARG (site, lresp outside [0, lmax], shell radius),
 * LRS_ERR_STATE (no chi0, during graph capture), LRS_ERR_UNSUPPORTED (not a
 * product grid), LRS_ERR_NUMERIC (singular S).
 */
int lrs_induced_potential(lrs_ctx* ctx, int site, double q, double shell_radius, int lresp, double* rho_lm,
                          double* vind_lm, double* vind_grid);

/*
 * FFT grid of LRS_PROJ_FFT_LAGRANGE3: N_i points along lattice vector a_i,
 * each 2^a 3^b <= LRS_FFT_MAX_N and >= 2 max|n_i| + 1 over the loaded G set
 * (checked at projection).  n1 = n2 = n3 = 0 selects per direction the
 * smallest such length >= 2 (2 max|n_i| + 1) (oversampling 2).
 * lrs_get_fft_grid returns the grid a projection would use now.
 * Errors: LRS_ERR_ARG (not 2^a 3^b, out of range), LRS_ERR_STATE (get
 * without orbitals).
 */
int lrs_set_fft_grid(lrs_ctx* ctx, int n1, int n2, int n3);
int lrs_get_fft_grid(lrs_ctx* ctx, int* n /* [3] */);

/*
 * Set / get the site-grid orbitals directly (bypassing lrs_project).
 * psi: host [npts][nk*nbands] complex in the column order above.
 */
int lrs_set_site_orbitals(lrs_ctx* ctx, int site, const double* psi);
int lrs_get_site_orbitals(lrs_ctx* ctx, int site, double* psi);

/*
 * Device-pointer forms of lrs_set_energies and lrs_set_site_orbitals, for
 * callers whose energies eps_kb (Eq. (eq-green)) and site-grid orbitals
 * psi_kb(tau + r_p) (Eq. (bloch)) already live on the GPU, e.g. tensors of a
 * differentiable program: the values are gathered into the library's column
 * order by a kernel on the context stream, without a host round trip or a
 * stream synchronisation.  The caller's buffer must stay valid until that
 * kernel has run (stream order).  Layouts as in the host forms:
 *   energies_dev  [nk][nbands] float64 (device)
 *   psi_dev       [npts][nk*nbands] complex128 interleaved (device)
 * Values are not inspected on the host: a non-finite energy or orbital shows
 * up later as LRS_ERR_NUMERIC of lrs_solve_w.  After lrs_set_energies_dev the
 * host copy of the energies (needed only when lrs_set_frequency_quadrature
 * derives mu or zeta from them) is read back at that call.  Both invalidate
 * chi0 and W (all sites for the energies, that site for the orbitals).
 * Errors: LRS_ERR_ARG (null pointer, site), LRS_ERR_STATE (no orbitals),
 * LRS_ERR_OOM, LRS_ERR_CUDA.
 */
int lrs_set_energies_dev(lrs_ctx* ctx, const double* energies_dev);
int lrs_set_site_orbitals_dev(lrs_ctx* ctx, int site, const double* psi_dev);

/*
 * Build chi0 on the grids of `nsite` sites (NULL = all), Eq. (chi1) with the
 * Green's functions of Sec. VI.D: per frequency t_i the occupied and
 * unoccupied parts
 *   Go(p,p')  = sum_{kv} conj psi_kv(p) d_kv psi_kv(p'),
 *   Gu^T(p,p')= sum_{kc} psi_kc(p) d_kc conj psi_kc(p'),  d = w_k/(mu + i t - eps),
 * and chi0 = (2/pi)(S + S^T), S = sum_i W_i Re[Go o Gu^T].
 * Requires projected (or set) orbitals and a quadrature.  Asynchronous on the
 * context stream.  Errors: LRS_ERR_STATE, LRS_ERR_ARG, LRS_ERR_OOM.
 */
int lrs_build_chi0(lrs_ctx* ctx, int nsite, const int* sites);

/*
 * Solve the Dyson equation for W (Eq. (eq-reducible), (eq-W), Sec. VI.E) on
 * the site grid: v = sum_{l<=L} r_<^l/r_>^(l+1) P_l(cos gamma),
 * Q = diag(wts), (I - v Q chi0 Q) W = v by float64 LU with partial pivoting.
 * On product grids (see lrs_set_option) the same equation is solved in the
 * (shell, l, m) basis: with v = Y C Y^T and X = Y^T Q chi0 Q Y,
 * W = Y (I - C X)^-1 C Y^T, the LU being of size nrad (L+1)^2.
 * Requires chi0 of those sites.  Errors: LRS_ERR_STATE, LRS_ERR_NUMERIC
 * (zero pivot or non-finite value), LRS_ERR_OOM.
 */
int lrs_solve_w(lrs_ctx* ctx, int nsite, const int* sites);

/*
 * The same solves queued on the context stream without waiting for them
 * (Sec. VI.E, as lrs_solve_w): the call returns once the work is queued, so
 * that one host thread can keep the next build in flight.  W of those sites
 * may be read at once (lrs_get_w copies in stream order, after the solve).
 * Device-side failures (a zero, non-positive or non-finite pivot; a
 * tensor-core kernel that gave up a bounded wait) are reported by the next
 * lrs_synchronize or lrs_solve_w on the context, which then marks W of the
 * queued sites missing; lrs_set_sites forgets the queued sites (call
 * lrs_synchronize first to see their status).
 * Errors (at queueing): LRS_ERR_STATE (no chi0), LRS_ERR_ARG, LRS_ERR_OOM.
 */
int lrs_solve_w_async(lrs_ctx* ctx, int nsite, const int* sites);

/* Copy chi0, W or v of one site ([npts][npts] float64) to host memory. */
int lrs_get_chi0(lrs_ctx* ctx, int site, double* out);
int lrs_get_w(lrs_ctx* ctx, int site, double* out);
int lrs_get_v(lrs_ctx* ctx, int site, double* out);
/* Same into caller-owned device memory, asynchronously on the context stream. */
int lrs_get_chi0_dev(lrs_ctx* ctx, int site, double* out_dev);
int lrs_get_w_dev(lrs_ctx* ctx, int site, double* out_dev);

/*
 * Adjoint of (energies, site orbitals) -> chi0 -> W for one site (the paper
 * has no gradients).  Given dL/dW (grad_w, [npts][npts], may be NULL) and
 * dL/dchi0 (grad_chi0, may be NULL), writes
 *   grad_energies [nk][nbands]            dL/d eps_kb
 *   grad_psi      [npts][nk*nbands] complex dL/dRe psi + i dL/dIm psi
 * at fixed mu and quadrature.  The Green's functions are recomputed per
 * frequency, never stored across frequencies.  Host buffers; the _dev variant
 * takes device pointers.  Requires a prior lrs_solve_w of the site (or
 * lrs_build_chi0 when grad_w is NULL).
 * Errors: LRS_ERR_STATE, LRS_ERR_ARG, LRS_ERR_OOM.
 */
int lrs_backward(lrs_ctx* ctx, int site, const double* grad_w, const double* grad_chi0,
                 double* grad_energies, double* grad_psi);
int lrs_backward_dev(lrs_ctx* ctx, int site, const double* grad_w_dev,
                     const double* grad_chi0_dev, double* grad_energies_dev,
                     double* grad_psi_dev);

/*
 * W for one site without any device allocation (the paper has no counterpart;
 * this is a service to callers that cannot allocate device memory: a plugin
 * inside a program whose caching allocator already holds the GPU's memory, a
 * latency-critical loop that cannot take the device synchronisation of
 * cudaMalloc/cudaFree, or a caller with a memory budget fixed at start-up).
 * Same arithmetic as lrs_solve_w: v of the multipole form, then
 * (I - v Q chi0 Q) W = v by float64 LU with partial pivoting.
 *   npts                1 .. LRS_STATIC_MAX_NPTS (larger sizes: LRS_ERR_ARG, no work done)
 *   lmax                multipole cutoff, 0..64
 *   pts_dev [npts][3]   point offsets from the site centre (device, nonzero)
 *   wts_dev [npts]      integration weights (device)
 *   chi0_dev [npts][npts] chi0 of the site (device, e.g. from lrs_get_chi0_dev)
 *   w_dev [npts][npts]  output W (device, caller-owned)
 *   stream              cudaStream_t of the work (NULL = legacy default stream)
 * Runs on the current device.  Scratch lives in one statically reserved
 * device array of about 2.1 MB (LRS_STATIC_MAX_NPTS^2 doubles plus pivots).
 * The driver reserves it on a GPU when it loads the library's module that
 * holds it: under CUDA's default lazy module loading that is the first call
 * on that device (with CUDA_MODULE_LOADING=EAGER, when the library is loaded);
 * from then on the GPU holds it until the process exits.  A caller whose own
 * allocator reserves the GPU's memory should therefore make one call early,
 * before that reservation.  The first call on a device also looks up that
 * array's device address (cudaGetSymbolAddress) and caches it; make that
 * first call before any stream capture.  Every call shares the array: calls
 * that overlap on the GPU race, so serialise them.  The call waits for its
 * stream to read the pivot status, so a call made while `stream` is being
 * captured is refused (LRS_ERR_STATE) before any work.  No cudaMalloc,
 * cudaFree or allocating library routine is called.
 * Errors: LRS_ERR_ARG, LRS_ERR_STATE, LRS_ERR_CUDA, LRS_ERR_NUMERIC
 * (zero/non-finite pivot).
 */
#define LRS_STATIC_MAX_NPTS 512
int lrs_solve_w_static(int npts, int lmax, const double* pts_dev, const double* wts_dev,
                       const double* chi0_dev, double* w_dev, void* stream);

/*
 * Record the whole build of `nsite` sites (NULL = all) - projection (mode
 * LRS_OPT_GRAPH_PROJECTION), chi0 in
 * one persistent tensor-core launch over every (site, tile, tile, frequency)
 * unit, and the Dyson solves - as a CUDA graph on the context stream, which
 * must not be the legacy default stream.  The call first runs the build once
 * eagerly (allocating every buffer and checking the status words), then
 * records it.  lrs_graph_launch replays it asynchronously on the context
 * stream, recomputing chi0 and W of those sites from the resident orbitals;
 * status words are not read during replays (call lrs_synchronize).  The
 * recording is dropped (lrs_graph_launch then fails with LRS_ERR_STATE) when
 * a later call frees or replaces workspace memory it reads, or changes the
 * multi-site unit table; capture again after such calls.
 * Errors: LRS_ERR_STATE, plus those of the stages.
 */
int lrs_graph_capture(lrs_ctx* ctx, int nsite, const int* sites);
int lrs_graph_launch(lrs_ctx* ctx);

/*
 * Tile shape tuning of the chi0 tensor-core launch for `nsite` sites: times
 * tile widths {128, 64} x accumulation segments {4, 2} chunks of 32 (short
 * segments bound the tensor cores' accumulation error) and keeps the fastest
 * on the context.  Outputs (may be NULL): tile_n, segment, ms_best.
 * Requires mixed precision and orbitals on the sites.
 */
int lrs_autotune(lrs_ctx* ctx, int nsite, const int* sites, int* tile_n, int* segment, double* ms_best);

/* Wait for the context stream; fold device timings into the stats; report the
 * status of solves queued by lrs_solve_w_async (LRS_ERR_NUMERIC,
 * LRS_ERR_TIMEOUT). */
int lrs_synchronize(lrs_ctx* ctx);

/* Statistics of the context (synchronises the stream first). */
int lrs_stats(lrs_ctx* ctx, lrs_stats_t* out);

#ifdef __cplusplus
}
#endif
#endif /* LRS_H */
