/*
 * nd.h -- C-ABI of libnd: the Neuberger-Dirac operator on one GB300 (sm_103a).
 *
 * Walk, Wittig, Dranischnikow, Schomer, "Implementation of the Neuberger-Dirac operator
 * on GPUs" (Lattice 2010).  Section numbers below refer to that paper.
 *
 * Conventions shared by every call
 *   Lattice extents dims = {T, L1, L2, L3}, all even; site x = (x0,x1,x2,x3), mu = 0 is time.
 *   lex(x) = x3 + L3*(x2 + L2*(x1 + L1*x0)); V = T*L1*L2*L3.
 *   Canonical (boundary) layouts, FP64 with interleaved (re, im):
 *     spinor  psi[lex][spin 4][colour 3][2]                 12 complex per site
 *     links   U[mu][lex][row 3][col 3][2]                    U_mu(x), row-major
 *     force   F[mu][lex][a = 1..8]                           coefficient of T^a = lambda^a/2
 *   Gamma matrices: chiral basis, gamma5 = gamma0 gamma1 gamma2 gamma3 = diag(1,1,-1,-1);
 *   in 2x2 blocks gamma0 = [[0,-1],[-1,0]], gamma_k = [[0,-i sigma_k],[i sigma_k,0]].
 *   Boundary conditions periodic; optionally antiperiodic in time.
 *   Internal layouts (opaque to the caller, sized by nd_spinor_bytes): even-odd ordered
 *   structure-of-arrays, eo(x) = p(x)*V/2 + lex(x)/2 with p(x) = (x0+x1+x2+x3) mod 2.
 *
 * Ownership and errors
 *   Every pointer argument named *_dev is device memory owned by the caller; the library
 *   never frees or keeps it beyond the call.  The context owns its own device copies of the
 *   links, its workspaces and its low-mode basis, and frees them in nd_destroy.
 *   All GPU work is ordered on the context's stream.  Calls that return host values
 *   (info structs, host arrays) synchronise that stream before returning.
 *   Every call returns an nd_status; nothing is thrown across the ABI.  On failure the
 *   context keeps a readable message (nd_last_error).  After ND_ERR_CUDA the context is
 *   unusable (ND_ERR_STATE) and must be destroyed.
 *   The library fails loudly (ND_ERR_CUDA) when no CUDA device is present: there is no
 *   CPU fallback.
 */
#ifndef ND_H
#define ND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nd_ctx nd_ctx;

typedef enum {
  ND_OK = 0,
  ND_ERR_INVALID_ARG = -1,   /* bad sizes, odd extents, null pointers, unsupported combination */
  ND_ERR_CUDA = -2,          /* a CUDA call failed; the message names it */
  ND_ERR_OOM = -3,           /* device allocation failed */
  ND_ERR_NOT_CONVERGED = -4, /* iteration limit reached; outputs hold the last iterate, info is filled */
  ND_ERR_BREAKDOWN = -5,     /* (p, A p) <= 0 or a zero pivot in a Krylov recurrence */
  ND_ERR_NAN = -6,           /* a norm became NaN or Inf */
  ND_ERR_STATE = -7          /* call out of order (e.g. no links set) or context poisoned */
} nd_status;

typedef enum {
  ND_FP64 = 0, /* FP64 storage and arithmetic */
  ND_FP32 = 1, /* FP32 storage and arithmetic, FP64 global reductions */
  ND_FP16 = 2  /* FP16 storage with one FP32 scale per site, FP32 arithmetic, FP64 reductions */
} nd_prec;

typedef enum {
  ND_RECON_NONE = 0, /* do not keep links in this precision */
  ND_RECON_8 = 8,    /* 8 reals: a2, a3, b1, arg a1, arg c1 (Sec. 2.1, 8-parameter form) */
  ND_RECON_12 = 12,  /* 12 reals: columns a, b; c = (a x b)^* rebuilt in registers (Sec. 2.1) */
  ND_RECON_18 = 18   /* all 18 reals */
} nd_recon;

/* ---------------------------------------------------------------- lifecycle */

/* Create a context for one lattice.  m is the Wilson bare mass of D_W (Sec. 2.1); s is the
 * overlap parameter of Sec. 2.2 (D_N = (1 + s)(1 + gamma5 sign Q), abar = 1/(1 + s)).
 * stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: ND_ERR_INVALID_ARG for odd or non-positive extents or |s| >= 1; ND_ERR_CUDA when no
 * device is usable. */
nd_status nd_create(nd_ctx** ctx, const int dims[4], int antiperiodic_t, double m, double s, void* stream);
void nd_destroy(nd_ctx* ctx);
/* Every call issues its work on the context's stream.  The mixed-precision refinement of a solve with
 * six or more shifts (nd_solve, nd_apply_sign, nd_apply_DN, nd_propagator) also runs part of its work on
 * a second stream that the context owns: forked from the context's stream with an event and joined back
 * before the call returns, so the caller sees stream order as usual. */
nd_status nd_set_stream(nd_ctx* ctx, void* stream);
const char* nd_status_string(nd_status st);
const char* nd_last_error(const nd_ctx* ctx);
/* Lattice volume and bytes of one internal spinor field of the given precision. */
int64_t nd_volume(const nd_ctx* ctx);
size_t nd_spinor_bytes(const nd_ctx* ctx, nd_prec prec);

/* ---------------------------------------------------------------- fields */

/* Copy the canonical FP64 gauge field U_dev ([4][V][3][3][2], device) into the context and
 * compress it, for each precision p, to recon[p] reals per link (ND_RECON_NONE skips p).
 * The 8-real form is singular when |a1| = 1 (e.g. unit links); such a field returns
 * ND_ERR_INVALID_ARG for recon 8.  Follows Sec. 2.1 (link storage). */
nd_status nd_set_links(nd_ctx* ctx, const double* U_dev, const int recon[3]);

/* Canonical FP64 spinors (nrhs consecutive fields, device) <-> internal layout of precision
 * prec (nrhs consecutive fields of nd_spinor_bytes each, device).  The internal layout is the
 * library's own and may change: the whole lattice, even-odd ordered (parity-0 block first), as a
 * structure of arrays of 16-byte chunks, chunk c of site h of parity p at index (p * NC + c) * V/2 + h;
 * FP64 keeps the canonical component order (NC = 12), FP32 (NC = 6) and FP16 (NC = 3, then one FP32
 * scale per site) hold the components as spin-row pairs (s0, s1) and (s2, s3) of each colour's real
 * and imaginary parts, the operands of packed FP32 arithmetic. */
nd_status nd_pack_spinor(nd_ctx* ctx, void* internal_dev, const double* canon_dev, nd_prec prec, int nrhs);
nd_status nd_unpack_spinor(nd_ctx* ctx, double* canon_dev, const void* internal_dev, nd_prec prec, int nrhs);

/* The same two conversions for canonical fields in single precision ([V][4][3] complex64,
 * interleaved FP32; half the host <-> device bytes of the FP64 form).  Packing to ND_FP64 widens
 * exactly; unpacking from ND_FP64 rounds to nearest. */
nd_status nd_pack_spinor_f32(nd_ctx* ctx, void* internal_dev, const float* canon_dev, nd_prec prec, int nrhs);
nd_status nd_unpack_spinor_f32(nd_ctx* ctx, float* canon_dev, const void* internal_dev, nd_prec prec, int nrhs);

/* Export the GPU's site tables: lex2eo_dev[V] (eo index of each lex site) and
 * nbr_dev[8][V] (eo index of the neighbour of eo site e in direction d = 2*mu + s,
 * s = 0 for x + mu, 1 for x - mu), both int32, device. */
nd_status nd_eo_tables(nd_ctx* ctx, int32_t* lex2eo_dev, int32_t* nbr_dev);

/* ---------------------------------------------------------------- operator Q */

/* out = Q in = gamma5 D_W in (Sec. 2.1) on nrhs internal fields of precision prec, with
 *   D_W phi(x) = (4+m) phi(x) - 1/2 sum_{mu=+-0..+-3} U_mu(x) (1 - gamma_mu) phi(x+mu).
 * out and in must not overlap.  Links must be set in precision prec. */
nd_status nd_apply_Q(nd_ctx* ctx, void* out_dev, const void* in_dev, nd_prec prec, int nrhs);

/* Even-odd block of Q for one output parity (the half pass of an even-odd preconditioned
 * operator): out_p = gamma5 [ diag_coef * in_p - 1/2 sum_mu (hops from in_{1-p}) ].
 * diag_coef = 4+m gives the rows of Q of parity p; diag_coef = 0 gives the pure hopping
 * block (in_p is then not read).  Only the parity-p half of out is written. */
nd_status nd_apply_Q_parity(nd_ctx* ctx, void* out_dev, const void* in_dev, nd_prec prec, int parity,
                            double diag_coef);

/* Q on several lattices of different sizes in one persistent launch: for k < nlat (<= 32),
 * out_dev[k] = Q in_dev[k] on nrhs[k] consecutive internal fields of precision prec of the
 * lattice of ctxs[k] (every context must hold links in prec with the same link form).  Tiles of
 * 64 sites x one RHS are walked lattice by lattice with the RHS fastest, so each lattice's links
 * are read from DRAM once for all its RHS.  Runs on `stream` (a cudaStream_t).  Errors are
 * reported on ctxs[0].  The work list is staged in a device buffer owned by ctxs[0] and filled by a
 * copy from pageable host memory on `stream`: calls that share ctxs[0] must use one stream (a call on
 * another stream could overwrite the list while an earlier launch still reads it), and the call
 * cannot be captured into a CUDA graph. */
nd_status nd_apply_Q_batched(nd_ctx* const* ctxs, int nlat, void* const* out_dev, const void* const* in_dev,
                             const int* nrhs, nd_prec prec, void* stream);

/* Convenience: Q on canonical FP64 device spinors (packs, applies in FP64, unpacks). */
nd_status nd_apply_Q_canonical(nd_ctx* ctx, double* out_dev, const double* in_dev);

/* out = Q in as nd_apply_Q (nrhs = 1), and norms[0] = ||out||^2, norms[1] = ||in||^2 (host,
 * FP64), for callers that may not allocate device memory at call time (a fixed memory budget
 * owned by another allocator, or a loop that promised no allocation after set-up).  The paper
 * has no counterpart; this is a library-service variant of the fused-norm launch.
 * It allocates nothing: the reduction scratch is a static device array of 256 KiB per GPU
 * (kept until exit), which limits the lattice to 4194304 sites (larger: ND_ERR_INVALID_ARG).
 * The first call on a device looks up that array's device address; make it before any
 * stream capture.  That address is kept for the life of the process: after cudaDeviceReset (which
 * also invalidates every nd_ctx of that device) this entry point must not be called again.
 * All calls share the array: calls that overlap on the GPU race on it, and the earlier of two
 * overlapping calls can return the other call's (stale) norms without reporting an error.
 * Synchronises the context's stream. */
nd_status nd_apply_Q_norms_static(nd_ctx* ctx, void* out_dev, const void* in_dev, nd_prec prec, double* norms);

/* ---------------------------------------------------------------- solvers */

typedef struct {
  int iters;             /* Krylov iterations of the (last) multi-shift pass */
  int outer;             /* outer defect-correction steps (mixed precision), else 0 */
  int sloppy_iters;      /* total sloppy-precision iterations including refinement */
  double max_resid;      /* max over shifts of the true FP64 relative residual */
  double time_ms;
} nd_solve_info;

/* Solve (Q^2 + shifts[k]) x_k = b for k < n (multi-shift CG, one Krylov space; each shift
 * stops at relative residual tol).  These are the shifted inverses that the rational approximation
 * of sign(Q) is built from (Sec. 2.2, the approximation of sign(Q); Q as in Sec. 2.1); the paper
 * itself evaluates a polynomial instead and prints no solver.  b_dev and x_dev[k] are canonical FP64 device spinors;
 * x_dev is a host array of n device pointers.  inner = ND_FP64 runs everything in FP64;
 * ND_FP32 / ND_FP16 run the Krylov iterations in that storage precision with FP64
 * reductions and refine every shift in FP64 (defect correction) down to tol.
 * Requires Q^2 + shifts[k] > 0 (shifts >= 0 and Q invertible, or shifts > 0). */
nd_status nd_solve(nd_ctx* ctx, double* const* x_dev, const double* b_dev, const double* shifts, int n,
                   double tol, int maxit, nd_prec inner, nd_solve_info* info);

/* ---------------------------------------------------------------- even-odd preconditioning */

/* out_e = Qhat in_e with the Schur complement of the even sites (Sec. 2.1 even-odd splitting):
 *   Qhat = gamma5 [(4 + m) - D_eo D_oe / (4 + m)],  hermitian like Q.
 * in/out: internal fields of precision prec (nd_spinor_bytes); only their even halves (parity 0,
 * the first half of the field) are read and written, the odd halves are left as they are.
 * out and in must differ.  Two one-parity stencil launches. */
nd_status nd_apply_Qhat(nd_ctx* ctx, void* out_dev, const void* in_dev, nd_prec prec);

/* x = (Q^2)^{-1} b through the Schur complement: Q^2 = D_W^dagger D_W, so
 * (Q^2)^{-1} b = D_W^{-1} gamma5 D_W^{-1} gamma5 b, and each D_W^{-1} is a CG on Qhat^2 over the
 * even sites plus one launch for the odd sites.  An FP64 defect correction on Q^2 wraps the two
 * solves, which run in `inner` (FP64, or FP32 / FP16 storage); stops at ||b - Q^2 x|| <= tol ||b||.
 * b_dev, x_dev: canonical FP64 device spinors (may not overlap).  info->iters counts Qhat^2 CG
 * iterations, info->outer the defect-correction sweeps, info->max_resid the final FP64 residual.
 * ND_ERR_NOT_CONVERGED if a CG hits maxit or the correction stagnates (x holds the last iterate). */
nd_status nd_solve_Q2_eo(nd_ctx* ctx, double* x_dev, const double* b_dev, double tol, int maxit, nd_prec inner,
                         nd_solve_info* info);

/* ---------------------------------------------------------------- low modes (Sec. 2.3) */

typedef struct {
  int l;                  /* number of modes kept */
  int iters;              /* Q^2 applications spent */
  double lambda_max;      /* estimate of the largest eigenvalue of Q^2 */
  double lambda_next;     /* estimate of lambda_{l+1}(Q^2) */
  double kappa_plus;      /* kappa_+ of Sec. 2.3 */
  double kappa_minus;     /* kappa_- of Sec. 2.3 */
  double max_rho;         /* max_k rho_k = ||(Q - nu_k) u_k|| */
  double time_ms;
} nd_lowmode_info;

/* Compute the l lowest modes of Q^2 (Chebyshev-filtered block subspace iteration: filter in FP32
 * until the residuals are small, then FP64; FP64 orthogonalisation and Rayleigh-Ritz of Q^2), then the
 * Rayleigh-Ritz eigenpairs (nu_k, u_k) of Q on their span, the residues rho_k and kappa_+- (Sec. 2.3).
 * The basis stays in the context for nd_apply_DN.  Host outputs (may be NULL):
 * nu[l], rho[l], eval_Q2[l+1] (the Rayleigh-Ritz values of Q^2 from the block, ascending).
 * Converges each of the l+1 lowest Ritz values of Q^2 to relative residual tol. */
nd_status nd_lowmodes(nd_ctx* ctx, int l, double tol, int maxit, double* nu, double* rho, double* eval_Q2,
                      nd_lowmode_info* info);

/* Low modes with l chosen dynamically (Sec. 2.3): in [l_min, l_max] the l with the largest relative
 * gap (sqrt(lambda_{l+1}) - sqrt(lambda_l)) / sqrt(lambda_{l+1}) of the Q^2 Ritz values is taken, so
 * that the kept modes are well separated from the remaining spectrum, and the
 * iteration stops when kappa_+ and kappa_- (as in nd_lowmodes) are both <= kappa_target.  The
 * projector deviation of Sec. 2.3 is then <= kappa (1 + 2 kappa) / (1 - 2 kappa (1 + 2 kappa)).
 * Outputs as nd_lowmodes with l = *l_out modes (host arrays sized for l_max, eval_Q2 for l_max + 1).
 * ND_ERR_NOT_CONVERGED when maxit Q^2 applications do not reach the target. */
nd_status nd_lowmodes_dynamic(nd_ctx* ctx, int l_min, int l_max, double kappa_target, int maxit, int* l_out,
                              double* nu, double* rho, double* eval_Q2, nd_lowmode_info* info);

/* The same choice of l and stopping rule with the paper's own minimiser (Sec. 2.3): l_max + 1
 * vectors, each minimising the Ritz functional (x, Q^2 x) / (x, x) on the complement of the ones
 * before it by nonlinear conjugate gradients (exact minimum on span{x, p} each step), then one
 * Rayleigh-Ritz step of Q^2 on all of them; while kappa_+- > kappa_target the minimisation is
 * repeated with a ten times smaller gradient tolerance (from 1e-4 lambda_max).  FP64 throughout.
 * Converges one vector at a time: slow where the low spectrum is a dense band.  Outputs as
 * nd_lowmodes_dynamic. */
nd_status nd_lowmodes_ritz(nd_ctx* ctx, int l_min, int l_max, double kappa_target, int maxit, int* l_out,
                           double* nu, double* rho, double* eval_Q2, nd_lowmode_info* info);

/* Replace the context's low modes by caller-provided orthonormal vectors (canonical FP64,
 * device, [l][V*12] complex) with their Q eigenvalues nu (host) and an estimate of
 * lambda_{l+1}(Q^2) (host).  rho and kappa are recomputed on the GPU. */
nd_status nd_set_lowmodes(nd_ctx* ctx, int l, const double* evecs_dev, const double* nu, double lambda_next,
                          nd_lowmode_info* info);

/* Copy the context's low modes out: evecs_dev [l][V*12] complex canonical (device), nu[l] (host). */
nd_status nd_get_lowmodes(nd_ctx* ctx, double* evecs_dev, double* nu);

/* The context's low-mode state (host outputs, each may be NULL): the number of modes kept, the
 * estimate of lambda_{l+1}(Q^2) sign(Q) takes eps from, and the lambda_max(Q^2) estimate (0 if
 * none yet).  With nd_get_lowmodes it is what a caller saves to restore the modes later through
 * nd_set_lowmodes (a checkpoint of the expensive part of D_N). */
nd_status nd_lowmode_state(nd_ctx* ctx, int* l, double* lambda_next, double* lambda_max);

/* Estimate lambda_max(Q^2) with iters Lanczos steps (upper Ritz value; not padded). */
nd_status nd_lambda_max(nd_ctx* ctx, int iters, double* lambda_max);

/* ---------------------------------------------------------------- sign(Q) and D_N (Sec. 2.2, 2.3) */

/* Zolotarev coefficients of R(x) = x sum_l b_l / (x^2 + sigma_l) ~ sign(x) on sqrt(eps) <= |x| <= 1
 * (host computation; n poles).  Returns the uniform error delta.  Host arrays sigma[n], b[n]. */
nd_status nd_zolotarev(int n, double eps, double* sigma, double* b, double* delta);

/* Minmax polynomial of Sec. 2.2: P_n(y) = sum_{k=0}^{n} c_k T_k(z), z = (2y - 1 - eps)/(1 - eps),
 * minimising delta = max_{eps <= y <= 1} |1 - sqrt(y) P_n(y)|, so that x P_n(x^2) ~ sign(x) on
 * sqrt(eps) <= |x| <= 1 with uniform error delta (host computation, Remez exchange; tables
 * are cached per (degree, eps)).  c: host array [degree + 1]; 0 <= degree <= 2048.
 * ND_ERR_NOT_CONVERGED if the exchange does not level the error. */
nd_status nd_chebyshev(int degree, double eps, double* c, double* delta);

/* Smallest degree n with delta(n) <= delta_target on [eps, 1] (ND_ERR_INVALID_ARG if above 2048). */
nd_status nd_chebyshev_degree(double eps, double delta_target, int* degree);

/* Approximation of sign(Q) used by nd_apply_sign / nd_apply_DN. */
enum { ND_SIGN_ZOLOTAREV = 0, ND_SIGN_CHEBYSHEV = 1 };

typedef struct {
  int n_poles;         /* Zolotarev poles (shifted systems) */
  double eps;          /* lower end of the X^2 interval; 0 = 0.99 * lambda_next / lambda_max */
  double lambda_max;   /* ||Q||^2 estimate; 0 = 1.01 * Lanczos estimate */
  double tol;          /* error target of the rational part (relative to ||source||) */
  int maxit;           /* Krylov iteration limit per multi-shift pass */
  nd_prec inner_prec;  /* ND_FP64: pure FP64; ND_FP32/ND_FP16: sloppy Krylov + FP64 refinement */
  double m_q;          /* quark mass of D_N^m = (1 - abar m_q / 2) D_N + m_q (0 = massless) */
  int left_only;       /* 1: the paper's literal (1 - P) X R(X^2) eta; 0: (1 - P) X R(X^2) (1 - P) eta */
  int approx;          /* ND_SIGN_ZOLOTAREV (rational, multi-shift CG) or ND_SIGN_CHEBYSHEV (the
                          paper's minmax polynomial X P_n(X^2) by the Clenshaw recurrence) */
  int degree;          /* ND_SIGN_CHEBYSHEV: degree n of P_n; 0 = smallest n with delta <= tol.
                          n_poles and maxit are not used; inner_prec is the precision of the whole
                          recurrence (no refinement: FP32 gives ~1e-6, FP16 ~1e-3 relative) */
} nd_dn_params;

typedef struct {
  int iters;           /* Krylov iterations of the multi-shift pass */
  int sloppy_iters;    /* total sloppy iterations including refinement */
  int outer;           /* FP64 refinement sweeps */
  int n_low;           /* deflated modes used */
  double delta;        /* uniform error of the approximation on [sqrt(eps), 1] */
  double eps;          /* eps used */
  double lambda_max;   /* lambda_max used */
  double max_resid;    /* max over shifts of the FP64 relative residual of the shifted solves */
  double time_ms;
  int degree;          /* ND_SIGN_CHEBYSHEV: degree of P_n used (Clenshaw iterations); else 0 */
  /* work and time of the multi-shift pass (the sloppy pass in mixed precision), for byte counts: */
  double krylov_ms;          /* device time of its iterations (CUDA events on the context's stream) */
  int krylov_live_shifts;    /* sum over its iterations of the shifts whose direction p_l was updated */
  int krylov_active_shifts;  /* sum over its iterations of the shifts whose solution term was updated */
  /* the FP64 defect correction (mixed precision; 0 otherwise): */
  int residuals64;           /* FP64 residuals b - (X^2 + sigma_l) x_l computed */
  int correction_iters;      /* iterations of the correction solves, summed over systems */
  double refine_ms;          /* wall time of the refinement */
} nd_dn_info;

/* out = sign(Q) in with the deflated approximation
 *   sign(Q) ~ P_+ - P_- + (1 - P) X R(X^2) (1 - P),  X = Q / sqrt(lambda_max)   (Sec. 2.3),
 * R the Zolotarev function or the minmax polynomial P_n (p->approx),
 * using the context's low modes (none if nd_lowmodes/nd_set_lowmodes was not called).
 * in_dev/out_dev: canonical FP64 device spinors (may not overlap). */
nd_status nd_apply_sign(nd_ctx* ctx, double* out_dev, const double* in_dev, const nd_dn_params* p, nd_dn_info* info);

/* out = D_N^m in, D_N = (1 + gamma5 sign(Q)) / abar, abar = 1/(1 + s)  (Sec. 2.2, 2.3). */
nd_status nd_apply_DN(nd_ctx* ctx, double* out_dev, const double* in_dev, const nd_dn_params* p, nd_dn_info* info);

/* out = (D_N^m)^dagger in = gamma5 D_N^m gamma5 in (Sec. 2.2: D_N is gamma5-hermitian because sign(Q) is
 * hermitian), computed as (f + m_q) in + f sign(Q) gamma5 in with f = (1 - abar m_q / 2) / abar: one
 * sign(Q) application, the multi-shift solves recomputed.  This is the vector-Jacobian product of
 * in -> D_N^m in.  Exact for the two-sided approximation only: p->left_only = 1 returns
 * ND_ERR_INVALID_ARG.  Arguments, deflation and info as nd_apply_DN. */
nd_status nd_apply_DN_dagger(nd_ctx* ctx, double* out_dev, const double* in_dev, const nd_dn_params* p,
                             nd_dn_info* info);

/* ---------------------------------------------------------------- propagators */

typedef struct {
  int iters;           /* CG iterations on H (one sign(Q) application each), all passes and chiralities */
  int outer;           /* defect-correction passes on D_N^m x = b */
  int sign_iters;      /* Krylov iterations (Zolotarev) or Clenshaw iterations (Chebyshev) of all sign(Q) applications */
  double resid;        /* true relative residual ||b - D_N^m x|| / ||b|| (with the same approximate sign(Q)) */
  double time_ms;
} nd_prop_info;

/* x = (D_N^m)^{-1} b for the massive overlap operator D_N^m = (1 - abar m_q/2) D_N + m_q (Sec. 2.2).
 * D_N^m is normal for a hermitian sign(Q), and H = D_N^m D_N^m^dagger commutes with gamma5; each
 * chirality of b is solved by CG on H (one sign(Q) application per iteration, approximation,
 * deflation and inner precision as in p), and x = gamma5 D_N^m gamma5 y.  An outer defect
 * correction on D_N^m x = b (two more sign(Q) applications per pass) stops at
 * ||b - D_N^m x|| <= tol ||b||, with D_N^m built from the same approximate sign(Q), whose sign^2 = 1
 * holds only to its accuracy.  p->left_only must be 0 (the left-only form is not hermitian).
 * b_dev, x_dev: canonical FP64 device spinors (may not overlap).  ND_ERR_NOT_CONVERGED after
 * maxit iterations of either chirality (x holds the last iterate); m_q > 0 keeps H >= m_q^2. */
nd_status nd_propagator(nd_ctx* ctx, double* x_dev, const double* b_dev, const nd_dn_params* p, double tol,
                        int maxit, nd_prop_info* info);

/* ---------------------------------------------------------------- differentiation */

/* Force of S = phi^dagger (Q^2)^{-1} phi with respect to the links (derived from the definition of
 * Q in Sec. 2.1: dS = -2 Re Y^dagger dQ X with X = (Q^2)^{-1} phi, Y = Q X; the paper has no force
 * passage): F[mu][lex][a] =
 * dS/d omega for U_mu(x) -> exp(i omega T^a) U_mu(x), T^a = lambda^a/2 (F_dev: [4][V][8]
 * FP64, device).  X = (Q^2)^{-1} phi is recomputed by CG (inner precision as nd_solve) to
 * relative residual tol; the force itself is one FP64 pass over the links. */
nd_status nd_force(nd_ctx* ctx, double* F_dev, const double* phi_dev, double tol, int maxit, nd_prec inner,
                   nd_solve_info* info);

/* S = phi^dagger (Q^2)^{-1} phi (host, S may be NULL) and its gradient with respect to the link
 * matrices treated as general complex 3x3 matrices: G_dev [4][V][3][3][2] (device, FP64) is the
 * conjugate Wirtinger derivative dS/dU^*, so dS = 2 Re sum conj(G_mu(x)_ij) dU_mu(x)_ij
 * (torch.autograd's gradient of a real loss is 2 G).  Derived from dS = -2 Re Y^dagger dQ X, Y = Q X (Sec. 2.1 definition of Q);
 * the su(3) projection of the same quantity is nd_force.  X_dev (canonical FP64 spinor, device,
 * may be NULL) receives X = (Q^2)^{-1} phi, which is also dS/dphi^* in the same convention.
 * Solve as nd_force. */
nd_status nd_link_gradient(nd_ctx* ctx, double* G_dev, double* X_dev, double* S, const double* phi_dev, double tol,
                           int maxit, nd_prec inner, nd_solve_info* info);

#ifdef __cplusplus
}
#endif
#endif /* ND_H */
