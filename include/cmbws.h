/*
 * cmbws -- GB300 (sm_103a) Wiener-filter / constrained-realization solver for
 * multi-resolution CMB component separation with the pseudo-inverse
 * preconditioner of Seljebotn, Baerland, Eriksen, Mardal & Wehus,
 * "Multi-resolution Bayesian CMB component separation through
 * Wiener-filtering with a pseudo-inverse preconditioner" (arXiv:1710.00621).
 *
 * Conventions shared by every call
 * --------------------------------
 * Status: every function returns an int, CMBWS_OK (0) on success or a
 *   negative CMBWS_ERR_* code.  cmbws_last_error() returns a message for the
 *   last failure on the calling host thread.  No C++ exception crosses this
 *   boundary.  When a call fails, the contents of its output buffers are
 *   unspecified.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls that take a stream enqueue their kernels on it and return
 *   without synchronising, except where noted.  A grid or model object owns
 *   workspace that every call on it reuses, so calls on one object must not
 *   overlap in time (serialise them on one stream).
 * Memory: buffers passed as `const double*` / `double*` data arguments are
 *   DEVICE pointers on the current CUDA device, contiguous, FP64, owned by
 *   the caller.  Pointers documented as host pointers are host memory.
 * Harmonic layout (CMBWS_ALM): a field with band-limit L has (L+1)^2 real
 *   coefficients of the real orthonormal basis
 *       Y_l0 = lambda_l0(theta),
 *       Y^c_lm = sqrt(2) lambda_lm(theta) cos(m phi),
 *       Y^s_lm = sqrt(2) lambda_lm(theta) sin(m phi)   (m > 0),
 *   lambda_lm the orthonormal associated Legendre function without the
 *   Condon-Shortley phase; stored m-major: m = 0 (l = 0..L), then for each
 *   m = 1..L the cos block (l = m..L) followed by the sin block (l = m..L).
 *   (L+1)^2 matches the paper's count of columns of U per component (Sec. 3.3).
 * Pixel layout: rings north to south, pixels of a ring in increasing azimuth
 *   phi_j = phi0_r + 2 pi j / nphi_r.
 * Stacked component vectors (x, b, r, z of the solver) hold the components
 *   k = 0..Ncomp-1 one after the other, each in CMBWS_ALM order with its own
 *   band-limit L_k (Sec. 2.2: s_lm = 0 for l > L_k).
 */
#ifndef CMBWS_H
#define CMBWS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CMBWS_OK = 0,
  CMBWS_ERR_ARG = -1,           /* invalid argument or unsupported size */
  CMBWS_ERR_CUDA = -2,          /* a CUDA runtime call failed */
  CMBWS_ERR_NOMEM = -3,         /* device or host allocation failed */
  CMBWS_ERR_SINGULAR = -4,      /* a U block has a column with zero norm */
  CMBWS_ERR_BREAKDOWN = -5,     /* CG: p.Ap <= 0 or a non-finite scalar */
  CMBWS_ERR_NOT_CONVERGED = -6, /* CG: iteration cap reached (x holds the last iterate) */
  CMBWS_ERR_TIMEOUT = -7,       /* wall-clock budget of a solve exhausted, or a bounded
                                   device-side wait ran out (cmbws_device_status) */
  CMBWS_ERR_COMM = -8           /* the all-reduce callback of a sharded solve failed */
};

typedef enum { CMBWS_GRID_GL = 0, CMBWS_GRID_HEALPIX = 1 } cmbws_grid_kind;

/* Arithmetic of the transform stages (Legendre recurrence and contraction,
 * ring FFTs, pixel multiplies).  Vectors at the boundary and CG scalars are
 * always FP64.
 *   CMBWS_FP64:   native FP64 throughout.
 *   CMBWS_FP32:   FP32 throughout (relative error ~1e-6 at L ~ 3000).
 *   CMBWS_FP32X2: FP64-accurate Legendre stage in double-float arithmetic (pairs of FP32
 *                 values, ~48-bit significand, on the FP32 pipe, which GB300 runs 61x
 *                 faster than FP64); ring FFTs and pixel stages in FP64.
 *   CMBWS_TF32:   as CMBWS_FP32, with the Legendre synthesis on the tensor cores (tcgen05,
 *                 TF32 recurrence values and coefficients, FP32 accumulation; relative error
 *                 ~1e-4); the adjoint Legendre stage stays FP32 on the CUDA cores.
 *   CMBWS_3XTF32: as CMBWS_TF32 with split-TF32 products (hi/lo parts, three MMAs per
 *                 step), FP32-level accuracy.
 *   CMBWS_BF16:   as CMBWS_TF32 with BF16 recurrence values and coefficients (tcgen05
 *                 kind::f16, FP32 accumulation; 8 significant bits per factor, relative
 *                 error ~1e-3).
 *   CMBWS_BF16X3: as CMBWS_BF16 with split-BF16 products (hi/lo parts, three MMAs per
 *                 step; about 16 significant bits per factor). */
typedef enum {
  CMBWS_FP64 = 0,
  CMBWS_FP32 = 1,
  CMBWS_FP32X2 = 2,
  CMBWS_TF32 = 3,
  CMBWS_3XTF32 = 4,
  CMBWS_BF16 = 5,
  CMBWS_BF16X3 = 6
} cmbws_prec;

typedef struct cmbws_grid_s* cmbws_grid;    /* opaque, library-owned */
typedef struct cmbws_model_s* cmbws_model;  /* opaque, library-owned */

/* Message for the last failing call on this host thread ("" if none). */
const char* cmbws_last_error(void);
/* Library version string. */
const char* cmbws_version(void);

/*
 * Plan a ring grid and its transform tables on the current CUDA device
 * (Sec. 2.1: Y, Y^T W and Y^T are defined per grid).
 *   kind = CMBWS_GRID_GL:      n = lmax + 1 rings at the Gauss-Legendre nodes,
 *                              2 lmax + 1 pixels per ring, phi0 = 0, weights
 *                              g_r * 2 pi / nphi (Y^T W Y = I exactly, Sec. 2.1).
 *   kind = CMBWS_GRID_HEALPIX: n = Nside; 4 Nside - 1 rings of the HEALPix ring
 *                              scheme, uniform weights 4 pi / Npix (Sec. 3.2,
 *                              App. A.1 accept Y^T W Y ~ I there).
 *   lmax: band-limit of the transforms on this grid (>= 0).
 * Limits: FP64 transforms need every ring length n <= 4096 after padding
 *   (ring FFTs run in shared memory); FP32 n <= 8192.  Larger grids return
 *   CMBWS_ERR_ARG from the transform calls of the precision they exceed.
 * Synchronises the device.  *out is released with cmbws_grid_destroy.
 */
int cmbws_plan_grid(cmbws_grid_kind kind, int n, int lmax, cmbws_grid* out);

/* Host pointers into the grid (valid until destroy): ring colatitudes theta[nring],
 * per-pixel quadrature weight of each ring weight[nring]. */
int cmbws_grid_info(cmbws_grid g, int64_t* npix, int* nring, const double** theta,
                    const double** weight);
/* Host pointers: first-pixel azimuth phi0[nring], pixels per ring nphi[nring],
 * first pixel of each ring offset[nring + 1]; and the band-limit. */
int cmbws_grid_rings(cmbws_grid g, const double** phi0, const int** nphi,
                     const int64_t** offset, int* lmax);
int cmbws_grid_destroy(cmbws_grid g);

/*
 * Spherical harmonic synthesis map = Y alm (Sec. 2.1).
 *   alm: device, nmaps x (lmax+1)^2 FP64, CMBWS_ALM order, map after map.
 *   map: device, nmaps x npix FP64, written.
 */
int cmbws_sht_synth(cmbws_grid g, cmbws_prec prec, const double* alm, double* map, int nmaps,
                    void* stream);
/*
 * weighted = 1: analysis alm = Y^T W map (Sec. 2.1);
 * weighted = 0: adjoint synthesis alm = Y^T map (Sec. 3.2).
 *   map: device, nmaps x npix FP64.  alm: device, nmaps x (lmax+1)^2 FP64, written.
 */
int cmbws_sht_analysis(cmbws_grid g, cmbws_prec prec, const double* map, double* alm, int nmaps,
                       int weighted, void* stream);

/*
 * Same result as cmbws_sht_analysis, with no device allocation.  The paper has no
 * counterpart; this call exists for callers that cannot allocate device memory when
 * they need the transform: runtimes that give the library a fixed memory budget and
 * forbid cudaMalloc after start-up, or loops that must not block on the allocator
 * (cudaMalloc can synchronise the device).  Its workspace is one static device array of
 * 32 MiB (32 << 20 bytes) that every GPU loading the library holds until exit; a call
 * whose workspace (ring spectra nmaps * nring * (lmax+1) complex values, the Legendre
 * adjoint's per-block partial sums and the reduced coefficients) would exceed it returns
 * CMBWS_ERR_ARG with the bytes it needs.  prec must be CMBWS_FP64 or CMBWS_FP32 (the other
 * modes build tables on first use); another precision returns CMBWS_ERR_ARG naming it.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (that device current) and keeps it; make that first call before any
 * stream capture, and do not use the library across a cudaDeviceReset, which makes the
 * kept address stale.  Every call shares the array and overwrites what it reads, so nothing
 * carries over between calls, but calls whose kernels overlap on the GPU race: serialise
 * them.  Keep kernel timing (cmbws_profile_enable) off here, since it creates CUDA events.
 * Other arguments and layouts as for cmbws_sht_analysis; the grid's own tables are
 * allocated once by cmbws_plan_grid.
 */
int cmbws_sht_analysis_noalloc(cmbws_grid g, cmbws_prec prec, const double* map, double* alm,
                               int nmaps, int weighted, void* stream);

/*
 * Model description (Sec. 2.2, Eqs. block-data-model, P, Q; Sec. 2.3, Eq. A).
 * All pointers are host pointers except ninv[nu], which are device pointers.
 * The library copies everything it keeps; the caller may free the inputs
 * after cmbws_model_create returns.
 */
typedef struct {
  int ncomp;                     /* 1 <= Ncomp <= 8 */
  int nobs;                      /* 1 <= Nobs <= 64 */
  const int* lmax_comp;          /* [ncomp] L_k */
  const cmbws_grid* band_grid;   /* [nobs] grid of d_nu; L_nu = that grid's lmax. Bands
                                    sharing a grid handle are transformed together. */
  const double* const* beam;     /* [nobs] host arrays b_{nu,l}, l = 0..L_nu (B_nu) */
  const double* const* cl;       /* [ncomp] host arrays C_{k,l}, l = 0..L_k, or NULL for no
                                    prior; a non-finite or non-positive entry means
                                    C^-1 = 0 at that l (Sec. 3.3) */
  const double* const* ninv;     /* [nobs] device maps tau_nu = diag(N_nu^-1), npix_nu, > 0 */
  const double* mix_scalar;      /* [nobs * ncomp] q_{nu,k}, row nu (spatially constant
                                    mixing, Q~ = q I) */
  /* Spatially variable mixing (Eq. Q), optional: both NULL for scalar mixing everywhere.
   * Entry nu * ncomp + k of each array describes pair (nu, k); a NULL mix_map entry keeps
   * that pair scalar.  For a variable pair, Q~_{nu,k} = Y^T W Q Y on mix_grid[...] (its
   * lmax must be >= max(L_k, L_nu); input zero-padded from L_k, output truncated at L_nu,
   * Sec. 2.2), and mix_map[...] is a device map of q_{nu,k}(n) on that grid, a mask
   * included as zeros.  Pairs sharing a grid handle are transformed together.  The
   * preconditioner uses the scalar of Eq. optimal-q of each variable map. */
  const cmbws_grid* mix_grid;    /* [nobs * ncomp] or NULL */
  const double* const* mix_map;  /* [nobs * ncomp] device pointers or NULL */
} cmbws_model_desc;

/*
 * Build a model: copies tau, computes alpha_nu (Eq. optimal-alpha), the per-l
 * blocks of U (Eqs. U-data, U-prior) and U^+ (Sec. 3.1, pseudo-inverse with a
 * singular-value cut-off of 1e-12 relative), and the pixel factors of A
 * (tau) and of T^+ (alpha^2 w^2 / tau, Sec. 3.3).  `prec` selects the
 * arithmetic of the transform stages of cmbws_apply_A / cmbws_apply_precond.
 * Synchronises `stream`.
 * Errors: CMBWS_ERR_SINGULAR if, at some l <= L_k, component k has neither
 * data nor a prior (a zero column of U).
 */
int cmbws_model_create(const cmbws_model_desc* desc, cmbws_prec prec, void* stream,
                       cmbws_model* out);
int cmbws_model_destroy(cmbws_model m);

/* Length of a stacked component vector, sum_k (L_k+1)^2; SHTs per apply of A and of
 * M_PI as the paper counts them (Sec. 3.3: 2(2 Nmix + Nobs) and 2 Nobs, Nmix = number of
 * variable mixing pairs). */
int cmbws_model_info(cmbws_model m, int64_t* nvec, int* nsht_A, int* nsht_M);

/* y = A x = S^-1 x + P^T N^-1 P x (Eq. A).  x, y: device stacked vectors, distinct. */
int cmbws_apply_A(cmbws_model m, const double* x, double* y, void* stream);

/* z = M_PI r = U^+ T^+ (U^+)^T r (Eq. fullmodel-preconditioner).  r, z distinct. */
int cmbws_apply_precond(cmbws_model m, const double* r, double* z, void* stream);

/*
 * Mask-restricted preconditioner for component `comp` (Sec. 4):
 *   M_mask = Z^T (Z S^-1 Z^T)^-1 Z   (Eq. M_mask),   Z = (pixels in the mask) Y R,
 * R = diag(r_l) the low-pass filter of Eq. rl, r_l = exp(-beta l^2 (l+1)^2) with r^2 = 0.05
 * at L/2.  (Z S^-1 Z^T)^-1 is approximated by one multigrid V-cycle (Sec. 4.4): HEALPix
 * levels with Nside and band-limit halved per level, a coarse pixel kept when its four
 * children are all in the mask, harmonic restriction Y_H R_H Y_h^T W_h, damped constant
 * smoother (omega = 0.2), SVD pseudo-inverse of the dense system at the bottom.  Solves
 * with cmbws_cg_opts.precond = 2 use M_add = M_PI + M_mask (Sec. 4.2).
 *   nside: HEALPix resolution of the mask, normally that of the mixing maps that carry it;
 *     level 0 has band-limit min(3 nside - 1, L_comp).
 *   mask: device map of 12 nside^2 doubles (ring order), nonzero inside the mask (the pixels
 *     whose data the mixing maps exclude).  Copied; the caller may free it.
 *   max_bottom: the coarsest level holds at most this many mask pixels (1..4096; e.g. 400).
 * Several calls add several preconditioners (summed).  Synchronises `stream`.
 * Errors: CMBWS_ERR_ARG (no prior on the component, bad arguments),
 * CMBWS_ERR_SINGULAR (a bottom pixel without coupling).
 */
int cmbws_model_add_mask_precond(cmbws_model m, int comp, int nside, const double* mask,
                                 int max_bottom, void* stream);

/*
 * Observation merging in the preconditioner (App. A.3).  group[nu] (host array of nobs ints)
 * assigns band nu to merged row group[nu] of U; the ids must be 0..G-1 (each used), and the
 * bands of a row must share one grid handle.  Afterwards M_PI (cmbws_apply_precond, and the
 * M_PI part of precond 1 and 2 of the solvers) runs one SHT pair per row instead of per band:
 *   row G of U, per l: the best rank-one fit u_G u_G^T of sum_{nu in G} U_nu^T U_nu (for rows
 *     U_nu = gamma_nu U_1, as for detector splits of one channel, u_G = sqrt(sum gamma^2) U_1,
 *     the exact merge; the paper prints the factor as (gamma + 1)^1/2);
 *   T_G^+ = alpha_G^2 Y^T W N_G W Y with the co-added inverse noise tau_G = sum_{nu in G} tau_nu
 *     and alpha_G of Eq. optimal-alpha (for exact splits T_G^+ equals each band's T^+, and the
 *     merged preconditioner equals M_PI).
 * A is unchanged.  group = NULL restores one row per band.  cmbws_model_info then reports
 * nsht_M = 2 G.  Synchronises `stream`.
 * Errors: CMBWS_ERR_ARG (ids outside 0..nobs-1, an unused id, bands of a row on different
 * grids), CMBWS_ERR_SINGULAR (a component without data or prior at some l).
 */
int cmbws_model_merge_precond(cmbws_model m, const int* group, void* stream);

/*
 * V-cycle of the model's mask preconditioners (Sec. 4.4, Fig. code:mg).
 *   kind 0 (default): the basic V-cycle, 8 SHTs per level.
 *   kind 1: the optimized V-cycle: I_h^H = Y_H R_H Y_h^T W_h and G_h = P Y_h D_h Y_h^T P
 *     inserted so that restriction and interpolation share transforms with G_h, and
 *     J = Y_h^T W_h P Y_h approximated by I as the paper does; 6 SHTs per level, two of them
 *     at the coarser level's band-limit on the finer grid (planned on first use, kept by the
 *     preconditioner).  Still a symmetric operator; not identical to the basic cycle.
 * Errors: CMBWS_ERR_ARG for another kind.
 */
int cmbws_model_set_vcycle(cmbws_model m, int kind);

/* z = M_add r = M_PI r + sum of the model's mask preconditioners (Sec. 4.2).  r, z distinct. */
int cmbws_apply_M_add(cmbws_model m, const double* r, double* z, void* stream);

/*
 * z = M_diag r, the block-diagonal preconditioner the paper compares M_PI with (Sec. 5):
 * M_diag = (U^T diag(T) U)^-1, i.e. for every real coefficient (l, m, cos / sin) the inverse of
 * the Ncomp x Ncomp block C_{k,l}^-1 delta_kk' + sum_nu b_{nu,l}^2 q_{nu,k} q_{nu,k'}
 * diag(Y_nu^T N_nu^-1 Y_nu)_lm, with q the scalars of M_PI (Eq. optimal-q for variable maps)
 * and the diagonal from ring sums of lambda_lm^2 and the ring Fourier sums of tau at even
 * frequencies (FP64 ring sums, FP32 lambda^2 sums, FP64 blocks).  Built on the first call
 * (or the first solve with precond = 3) and kept by the model.  r, z distinct.
 */
int cmbws_apply_M_diag(cmbws_model m, const double* r, double* z, void* stream);

/*
 * b = P^T N^-1 d + P^T N^-1/2 omega1 + S^-1/2 omega2 (Sec. 2.3; the printed S^-1 omega2
 * is read as S^-1/2 omega2, for which Var(b) = A).  b is FP64-accurate for every model:
 * its transforms run in FP64 for FP64 models and in CMBWS_FP32X2 otherwise.
 *   d, omega1: host arrays [nobs] of device maps (npix_nu FP64); omega1 may be NULL.
 *   omega2: device stacked vector or NULL.  b: device stacked vector, written.
 */
int cmbws_rhs(cmbws_model m, const double* const* d, const double* const* omega1,
              const double* omega2, double* b, void* stream);

/*
 * Terms of the gradient of a loss of the solution.  The paper solves A x = b
 * (Eq. A) for fixed parameters; differentiating A x = b gives, for a loss L(x)
 * and the adjoint solution lambda of A lambda = dL/dx (A is symmetric),
 *   dL/dtheta = lambda^T (db/dtheta - (dA/dtheta) x).
 * This call evaluates that form for the scalar mixing entries theta = q_{nu,k}
 * (P_{nu,k} = Y_nu B_nu q_{nu,k}, Eq. P) and for a log-scale theta = t_k of each
 * prior spectrum (C_{k,l} -> exp(t_k) C_{k,l}, at t_k = 0), with b the right-hand
 * side of cmbws_rhs built from the same d, omega1, omega2:
 *   out[nu * ncomp + k] = <B_nu lambda_k, Y^T (N^-1 d + N^-1/2 omega1 - N^-1 P x)>_nu
 *                       - <B_nu x_k, Y^T N^-1 P lambda>_nu
 *   out[nobs * ncomp + k] = lambda_k^T S_k^-1 x_k - 1/2 lambda_k^T S_k^-1/2 omega2_k
 * (dot products over l <= min(L_nu, L_k)).  Spectral indices and amplitudes follow
 * by the chain rule (dq/dbeta = q ln(nu / nu_0) for a power law).
 *   x, lambda: device stacked vectors.  d, omega1: host arrays [nobs] of device maps
 *   (omega1 may be NULL); omega2: device stacked vector or NULL.
 *   out: device array of nobs * ncomp + ncomp doubles, written.
 * For a pair (nu, k) with a spatially variable mixing map (Eq. Q), out[nu * ncomp + k]
 * is the derivative in a uniform offset added to the map: the sum over its pixels of
 * cmbws_grad_mix_maps.
 * The transforms run FP64-accurate (FP64 for FP64 models, CMBWS_FP32X2 otherwise);
 * the sums are reduced in a fixed order.  Uses the model's workspaces: calls on one
 * model must not overlap.
 * Errors: CMBWS_ERR_ARG for NULL arguments or a sharded model.
 */
int cmbws_grad_terms(cmbws_model m, const double* x, const double* lambda,
                     const double* const* d, const double* const* omega1, const double* omega2,
                     double* out, void* stream);

/*
 * Gradient of a loss of the solution with respect to the pixel values of the spatially
 * variable mixing maps (Eq. Q: Q~_{nu,k} = Y_nu^T W diag(q_{nu,k}) Y_k on the pair's
 * mixing grid).  With the same lambda, u_nu = B_nu Y_nu^T (N^-1 d + N^-1/2 omega1 - N^-1 P x)
 * and v_nu = B_nu Y_nu^T N^-1 P lambda as in cmbws_grad_terms,
 *   dL/dq_{nu,k}(p) = w_p [ (Y lambda_k)(p) (Y u_nu)(p) - (Y x_k)(p) (Y v_nu)(p) ],
 * the syntheses on the mixing grid (band-limits L_k and L_nu), w_p its pixel weight.  A
 * spectral-index map beta_k(p) with q = (nu / nu_0)^beta follows by the chain rule.
 *   x, lambda: device stacked vectors.  d, omega1: host arrays [nobs] of device maps
 *   (omega1 may be NULL).
 *   out: host array [nobs * ncomp] of device pointers; entry nu * ncomp + k receives the
 *   gradient map of a variable pair (npix of its mixing grid, in the grid's pixel order);
 *   NULL entries and entries of scalar pairs are not written.
 * FP64-accurate transforms as in cmbws_grad_terms; the model's workspaces are used.
 * Errors: CMBWS_ERR_ARG for NULL arguments, a sharded model or a model without variable
 * mixing.
 */
int cmbws_grad_mix_maps(cmbws_model m, const double* x, const double* lambda,
                        const double* const* d, const double* const* omega1, double* const* out,
                        void* stream);

/*
 * Data-model projection d_nu = P_nu x = Y_nu B_nu sum_k Q~_{nu,k} x_k (Eq. P), e.g. to
 * simulate d = P s + n (Eq. block-data-model).
 *   x: device stacked vector.  d: host array [nobs] of device maps (npix_nu FP64), written.
 * Uses the model's transform precision.
 */
int cmbws_project(cmbws_model m, const double* x, double* const* d, void* stream);

/*
 * Autotuner of the Legendre synthesis tiles (ring pairs per thread and threads per CTA).
 *   mode 0 (default): every launch uses the default tile;
 *   mode 1: a heuristic by the grid's ring-pair count (the smallest CTA holding every pair);
 *   mode 2: on the first synthesis for a (grid, precision, maps) key, each tile variant is
 *     launched and timed with CUDA events on the caller's stream (the first call is then
 *     synchronous), and the fastest is kept for that key for the life of the grid.
 * FP64 results do not depend on the tile; FP32 results can differ in rounding (warps that
 * hold a ring pair near a pole switch to the difference form of the recurrence, and the
 * tile decides which pairs share a warp).  Errors: CMBWS_ERR_ARG for another mode.
 */
int cmbws_set_autotune(int mode);

/* The tuner's decision for synthesis on grid g at precision prec with nmaps maps per
 * launch (1..4): variant index (-1 if none was measured), nvar variants, and their times in
 * ms (ms: array of at least 8 floats, or NULL). */
int cmbws_grid_tuning(cmbws_grid g, int prec, int nmaps, int* variant, float* ms, int* nvar);

/*
 * Kernel timing.  While enabled, the library brackets each of its kernel launches with
 * CUDA events on the launching stream.  Records are kept per slot = stage + 6 * arith,
 * stages 0 Legendre synthesis, 1 Legendre adjoint, 2 adjoint partial-sum reduction,
 * 3 ring FFT, 4 harmonic-space kernels, 5 CG vector kernels; arith 0 = FP32, 1 = FP64,
 * 2 = double-float (CMBWS_FP32X2), 3 = TF32 tensor cores, 4 = split TF32 tensor cores,
 * 5 = BF16 tensor cores, 6 = split BF16 tensor cores.
 * cmbws_profile_read synchronises the recorded events and writes, per slot (host arrays
 * of 42, any may be NULL), since the last reset:
 *   ms: summed milliseconds; launches: launch count;
 *   flops: summed algorithmic flops (Legendre stages: 4 per (l, m, ring pair) for the
 *     recurrence plus 4 per map for the contraction, over the full (l, m) triangle);
 *   elems: summed (l, m, ring pair) elements of the Legendre launches;
 *   map_elems: summed elements x maps per launch (so flops = 4 (elems + map_elems));
 *   bytes: summed algorithmic bytes of the ring FFT launches (ring spectra read and / or
 *     written once, plus the pixel factors or FP64 maps once);
 * 0 where a stage has no such count.  reset = 1 clears the record.
 */
int cmbws_profile_enable(int on);
int cmbws_profile_read(double* ms, int64_t* launches, double* flops, double* elems,
                       double* map_elems, double* bytes, int reset);

typedef struct {
  double tol;         /* stop when ||b - A x||_2 / ||b||_2 <= tol, certified by an FP64 apply */
  int maxiter;        /* cap on CG iterations (all inner iterations counted) */
  int precond;        /* 0 = none, 1 = M_PI, 2 = M_add = M_PI + the model's mask
                         preconditioners (cmbws_model_add_mask_precond), 3 = the block-
                         diagonal M_diag (cmbws_apply_M_diag) */
  double inner_tol;   /* FP32 models: relative reduction per refinement pass (e.g. 1e-3) */
  int max_outer;      /* FP32 models: cap on refinement passes */
  double timeout_s;   /* wall-clock budget, <= 0 for none */
  int cert_prec;      /* arithmetic of the applies that compute the true residual b - A x:
                         CMBWS_FP64 (native) or CMBWS_FP32X2 (double-float); other values
                         mean CMBWS_FP64 */
} cmbws_cg_opts;

typedef struct {
  int status;         /* CMBWS_OK or the error returned */
  int iters;          /* CG iterations (sum over refinement passes) */
  int outer;          /* refinement passes (1 for FP64 models) */
  double rel_res;     /* certified ||b - A x|| / ||b|| with A in FP64 */
  int n_sht;          /* SHTs executed, counted as the paper counts them */
  double ms;          /* wall time of the solve on the host clock */
} cmbws_cg_report;

/*
 * Solve A x = b by preconditioned CG (Sec. 2.3) with M_PI (Sec. 3.3).
 *   b: device stacked vector.  x: device stacked vector; in: initial guess, out: solution.
 * FP64 models run plain PCG in FP64 and certify the final residual with one FP64 apply.
 * FP32 models run iterative refinement: each pass solves A d = r with FP32 transforms
 * (FP64 vectors and scalars) to a relative reduction inner_tol, then x += d and
 * r = b - A x with FP64 transforms, until r certifies tol.
 * Synchronises `stream` (the host reads one scalar per iteration).  `report` may be NULL.
 */
int cmbws_cg_solve(cmbws_model m, const double* b, double* x, const cmbws_cg_opts* opts,
                   cmbws_cg_report* report, void* stream);

/*
 * Arithmetic of the transforms of M_PI inside the solvers (cmbws_cg_solve and the solves
 * built on it): any cmbws_prec, or -1 (default) for the model's own.  The preconditioner only
 * has to approximate A^-1, so its transforms can run in a cheaper precision than those of A,
 * e.g. the BF16 tensor-core synthesis in the FP32 inner solves; cmbws_apply_precond keeps the
 * model's precision.  Errors: CMBWS_ERR_ARG.
 */
int cmbws_model_set_precond_prec(cmbws_model m, int prec);

/*
 * Per-iteration record of the model's last solve (cmbws_cg_solve, cmbws_cg_resume, or one
 * problem of cmbws_cg_solve_batched), the error-tracking method of Sec. 2.3 and Sec. 5:
 *   rel_res[i] = ||r_i|| / ||b||, r_i the recursive residual after CG iteration i (over all
 *     refinement passes; for FP32 models the residual of the correction equation, which
 *     equals b - A x_i up to the FP32 operator's error);
 *   rel_err[i] = ||x_i - x_true|| / ||x_true|| while a reference solution is set with
 *     cmbws_cg_track_error (one extra dot product per iteration), else -1.
 * Host arrays of at least cap entries (either may be NULL); *n receives the number of
 * iterations recorded (entries beyond cap are not written).  Errors: CMBWS_ERR_ARG.
 */
int cmbws_cg_history(cmbws_model m, double* rel_res, double* rel_err, int cap, int* n);

/* Reference solution for the error record of cmbws_cg_history (e.g. x_true with
 * b = A x_true, Sec. 2.3): a device stacked vector, copied (synchronises `stream`); NULL
 * stops the tracking. */
int cmbws_cg_track_error(cmbws_model m, const double* x_true, void* stream);

/*
 * Checkpoint / resume of a PCG solve (models without FP32 transforms: CMBWS_FP64,
 * CMBWS_FP32X2).  With checkpointing on, a solve that stops at its iteration cap
 * (CMBWS_ERR_NOT_CONVERGED) keeps the state of its next iteration: the correction d
 * (the solution is x0 + d), the residual r, the search direction p, and the scalars
 * {iterations done, r.z, r.r}.  cmbws_cg_state_export copies it out (d, r, p: device stacked
 * vectors; scalars: host array of 3), e.g. to storage; cmbws_cg_resume continues from such a
 * state on a model built from the same description, with b and x holding the right-hand
 * side and the initial guess x0 of the interrupted solve (x is overwritten with the
 * solution).  opts.maxiter caps the iterations of both runs together, so an interrupted and
 * resumed solve performs exactly the operations of an uninterrupted one and returns the
 * bitwise same x.  Models with FP32 transforms (iterative refinement) resume by passing the
 * returned x as the initial guess of a new solve instead: CMBWS_ERR_ARG here.
 * Errors: CMBWS_ERR_ARG (no checkpoint, invalid scalars, FP32 models).
 */
int cmbws_cg_checkpointing(cmbws_model m, int on);
int cmbws_cg_state_export(cmbws_model m, double* d, double* r, double* p, double* scalars,
                          void* stream);
int cmbws_cg_resume(cmbws_model m, const double* b, double* x, const double* d, const double* r,
                    const double* p, const double* scalars, const cmbws_cg_opts* opts,
                    cmbws_cg_report* report, void* stream);

/*
 * CUDA graphs for the operator applies inside the solvers (on = 1; default 0).  Each apply of
 * A and of the preconditioner in PCG is tens to hundreds of kernel launches (per grid group:
 * Legendre synthesis, ring FFT, Legendre adjoint; harmonic-space kernels; the multigrid
 * levels of M_add); with graphs on, the second apply for a given operator, precision and
 * pair of buffers is captured into a CUDA graph and later applies replay it with one launch.
 * Results are bitwise those of the eager applies.  Graphs are not used while per-stage
 * profiling is on, and are dropped when the model's preconditioners change
 * (cmbws_model_add_mask_precond, cmbws_model_merge_precond, cmbws_model_set_vcycle) or when
 * graphs are switched off.
 */
int cmbws_model_set_graphs(cmbws_model m, int on);

/*
 * Solve nprob independent systems A_i x_i = b_i (each as cmbws_cg_solve) concurrently.
 *   models: [nprob] distinct models (each owns its workspace); b, x: host arrays [nprob] of
 *   device stacked vectors.  reports: [nprob] or NULL.
 * The problems are distributed over nworkers host threads (<= 0: 8), each driving its own
 * CUDA stream, so the kernels of different problems overlap on the GPU.  Work already
 * queued on `stream` completes before the solves start; the call returns after all solves
 * have finished.  Returns CMBWS_OK if every problem succeeded, else the first failing
 * problem's code (all reports are filled either way).
 */
int cmbws_cg_solve_batched(const cmbws_model* models, int nprob, const double* const* b,
                           double* const* x, const cmbws_cg_opts* opts, cmbws_cg_report* reports,
                           int nworkers, void* stream);

/*
 * Band sharding, for a solve spread over several GPUs (one process and one model per GPU).
 * A is a sum over bands plus the prior (Eq. A), and M_PI = U^+ T^+ (U^+)^T is a sum over the
 * rows of U: one term per band (its T^+_nu) and the prior rows (Sec. 3.3).  With a shard set,
 * this model's cmbws_apply_A, cmbws_apply_precond and cmbws_rhs return only the terms of the
 * bands it owns, plus the prior terms if prior = 1, and run the transforms of those bands
 * only; the sum of the shards' outputs is the full result.  Every shard's model is built from
 * the same full description (U^+ needs every band's alpha, beam and mixing).
 *   owned: host array [nobs] of 0 / 1, or NULL to drop the shard (the full operators again).
 * Other calls that apply or solve (cmbws_cg_solve, batched, resume, M_diag, M_add, mask
 * preconditioners, merging, gradients, CR draws) refuse a sharded model with CMBWS_ERR_ARG.
 * Errors: CMBWS_ERR_ARG (entries other than 0 / 1, merged rows or mask preconditioners set).
 */
int cmbws_model_set_shard(cmbws_model m, const int* owned, int prior);

/*
 * All-reduce callback of a sharded solve: replace the device vector v of n doubles by its sum
 * over all shards, ordered after the work already queued on `stream` (the solve's stream,
 * passed through), and return 0 (nonzero reports CMBWS_ERR_COMM).  Every shard must end up
 * with the bitwise same sum (true of a ring all-reduce, or of a gather-and-add in a fixed order).
 */
typedef int (*cmbws_allreduce_fn)(double* v, int64_t n, void* stream, void* ctx);

/*
 * PCG (precond 0 or 1) over a band-sharded operator: every shard calls this with the same b,
 * initial x and opts on its own model (cmbws_model_set_shard, the shards' bands together
 * covering every band once and one shard owning the prior).  Each apply of A and of M_PI runs
 * the shard's partial terms and one all-reduce of the stacked vector; the CG vectors stay
 * replicated, so the scalars (dot products) are computed identically on every shard and need
 * no collective.  Results as cmbws_cg_solve (up to the summation order of the all-reduce).
 * Errors: as cmbws_cg_solve; CMBWS_ERR_COMM when the callback fails.
 */
int cmbws_cg_solve_sharded(cmbws_model m, const double* b, double* x, const cmbws_cg_opts* opts,
                           cmbws_allreduce_fn allreduce, void* ctx, cmbws_cg_report* report,
                           void* stream);

/*
 * Variates of a counter-based stream, for constrained realizations (Sec. 2.3) drawn on the
 * device.  Generator: Philox4x64-10 (Salmon, Moraes, Dror and Shaw, SC'11).  Variate j of
 * stream `stream_id` is word j % 4 of Philox4x64-10(counter (j / 4, stream_id, 0, 0),
 * key (seed, sample)); a word w gives the uniform u = ((w >> 12) + 1/2) 2^-52 in (0, 1), and
 * the uniform pairs (u0, u1), (u2, u3) of a counter give standard normals by the Box-Muller
 * transform, z = sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b).  So a variate depends only on
 * (seed, sample, stream_id, j), whatever range a call covers.
 *   out[t] = variate offset + t, t = 0 .. n-1 (device, FP64); kind 0 = standard normal,
 *   1 = uniform.  offset, n >= 0; n = 0 does nothing.
 * Errors: CMBWS_ERR_ARG for a negative offset or n, a bad kind, or out NULL with n > 0.
 */
int cmbws_draw(uint64_t seed, uint64_t sample, uint64_t stream_id, int64_t offset, int64_t n,
               int kind, double* out, void* stream);

/*
 * Right-hand side of constrained realization `sample` (Sec. 2.3): omega_2 = stream 0 of
 * cmbws_draw(seed, sample) over the stacked coefficient vector, omega_1 of band nu = stream
 * 1 + nu over its pixels (ring order), both standard normal, drawn on the device into the
 * model's workspace; then b as cmbws_rhs(d, omega_1, omega_2).
 *   d: host array [nobs] of device maps.  b: device stacked vector, written.
 */
int cmbws_cr_rhs(cmbws_model m, const double* const* d, uint64_t seed, uint64_t sample,
                 double* b, void* stream);

/*
 * One constrained realization: b of cmbws_cr_rhs, then A x = b solved as cmbws_cg_solve,
 * starting from the initial guess held in x (e.g. the previous sample of a chain, or the
 * Wiener-filter mean; zero for none).  x: device stacked vector, in/out.  Errors and report
 * as cmbws_cg_solve.
 */
int cmbws_cr_sample(cmbws_model m, const double* const* d, uint64_t seed, uint64_t sample,
                    double* x, const cmbws_cg_opts* opts, cmbws_cg_report* report, void* stream);

/*
 * Mixing map of a power-law SED with a spatially variable spectral index (Eq. Q):
 * q[i] = m[i] (nu / nu_0)^beta[i], m[i] = 0 where mask[i] == 0 and 1 elsewhere (mask NULL:
 * no mask).  beta, mask, q: device arrays of n doubles on a mixing grid, for the mix_map of
 * cmbws_model_desc.  nu_ratio = nu / nu_0 > 0.
 */
int cmbws_powerlaw_mixing(double nu_ratio, const double* beta, const double* mask, int64_t n,
                          double* q, void* stream);

/*
 * Device-side status.  Kernels that wait on an asynchronous event inside the GPU (the
 * tensor-core Legendre synthesis waits on mbarriers for its MMAs) bound every wait; when a
 * wait runs out the kernel stops issuing work, writes NaN into its outputs, records the
 * event in a per-device status word and returns, so the context stays usable.  This call
 * synchronises `stream`, then returns CMBWS_ERR_TIMEOUT if such an event was recorded on the
 * current device since the last call (and clears the record), else CMBWS_OK.  The solvers
 * check the record themselves when a non-finite scalar appears and return CMBWS_ERR_TIMEOUT
 * instead of CMBWS_ERR_BREAKDOWN.
 */
int cmbws_device_status(void* stream);

/*
 * Test support for the bounded waits (no counterpart in the paper).  wait_cycles > 0 makes
 * every CTA of the tensor-core Legendre synthesis (CMBWS_TF32, CMBWS_3XTF32) on the current
 * device first wait at most wait_cycles SM clocks on an mbarrier phase that nothing ever
 * completes: the wait runs out, and the CTA takes the failure path described at
 * cmbws_device_status.  0 (the default) switches it off.  Errors: CMBWS_ERR_ARG outside
 * [0, 2^32].
 */
int cmbws_testing_stall_waits(long long wait_cycles);

#ifdef __cplusplus
}
#endif
#endif /* CMBWS_H */
