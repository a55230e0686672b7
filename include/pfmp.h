/*
 * pfmp.h -- C-ABI of the GB300 (sm_103a) library for the data-parallel hot path of
 * polynomial-filtered mass-preconditioned HMC (PF-MP HMC; Haar, Kamleh, Zanotti,
 * Nakamura, "Applying polynomial filtering to mass preconditioned Hybrid Monte Carlo").
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status: PFMP_OK (0) or one of the PFMP_E_* codes;
 *    pfmp_last_error() gives a text for the most recent failure on this host thread.
 *    No C++ exception crosses this boundary.
 *  - All device work is enqueued on the context's CUDA stream.  Functions that return a
 *    host scalar (norms, actions, solver info) synchronise that stream and say so.
 *  - Handles (pfmp_ctx, pfmp_op, pfmp_poly, pfmp_action) are opaque and owned by the
 *    library; each is released by its matching *_destroy.
 *  - Spinor arguments ("void* field") are caller-owned DEVICE buffers of one parity in
 *    the library's device layout: pfmp_spinor_bytes() gives their size; they are
 *    filled with pfmp_spinor_pack() from the canonical layout.  The library never
 *    frees caller buffers.
 *  - Canonical host layout (used for gauge fields, spinors and momenta that cross the
 *    boundary): lexicographic site index s = x + Lx*(y + Ly*(z + Lz*t)); gauge links
 *    [s][mu][row][col] complex double (mu = 0..3 is x, y, z, t); spinors
 *    [s][spin][colour] complex double in the chiral (DeGrand-Rossi) gamma basis;
 *    momenta/forces [s][mu][a] real double, coefficients of P = sum_a p_a T_a with
 *    T_a = lambda_a / 2.  Complex numbers are interleaved (re, im).
 *  - Lattice extents must all be even (even-odd preconditioning) and Lx*Ly*Lz*Lt/2
 *    must fit in an int.
 *
 * Operator (Sec. 2.1 and Table 3.1 of the paper, plus a clover term):
 *    M = A - kappa H,  (H psi)(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu)
 *                                        + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu),
 *    A(x) = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x),
 *    F_{mu nu} = traceless part of (Q_{mu nu} - Q_{mu nu}^dag)/(8i), Q = clover leaves,
 *    M-hat = A_ee - kappa^2 H_eo A_oo^{-1} H_oe (even-odd Schur complement),
 *    K = M-hat^dag M-hat (Sec. 2.1 eq. for S_F), J = the same at kappa' (eq. hasenbusch).
 * Fermion fields in time direction carry the factor bc_t (-1: antiperiodic) across the
 * boundary; gauge links are periodic.
 */
#ifndef PFMP_H
#define PFMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define PFMP_OK 0
#define PFMP_E_INVALID 1         /* bad argument (null pointer, odd extent, bad enum)   */
#define PFMP_E_NOMEM 2           /* device or host allocation failed                     */
#define PFMP_E_CUDA 3            /* a CUDA call failed; see pfmp_last_error()            */
#define PFMP_E_NOT_CONVERGED 4   /* solver hit max_iter before the requested residual    */
#define PFMP_E_TIMEOUT 5         /* a bounded device wait gave up                        */
#define PFMP_E_NAN 6             /* a NaN/Inf appeared in a solver scalar or in dH       */
#define PFMP_E_UNSUPPORTED 7     /* valid but not implemented (e.g. odd polynomial order)*/

/* ---- precisions and locations ---------------------------------------------------- */
#define PFMP_F64 0
#define PFMP_F32 1
/* FP16 storage, FP32 arithmetic (the sloppy precision of PFMP_SOLVER_CG_HALF): an even
 * or odd spinor field is [3][Vh] of 16-byte words (word k holds the complex components
 * 4k .. 4k+3 of the 12, spin-major) followed by one FP32 scale per site (the site's
 * largest |component|; stored values are value / scale), 52 bytes per site; links
 * (24 bytes each) and clover blocks in FP16 without scale (|entries| = O(1)).
 * Accepted by pfmp_dslash, pfmp_mhat, pfmp_kop, pfmp_spinor_pack/unpack, pfmp_convert
 * (to and from PFMP_F32) and pfmp_spinor_bytes.                                      */
#define PFMP_H16 3
#define PFMP_HOST 0
#define PFMP_DEVICE 1

typedef struct pfmp_ctx pfmp_ctx;
typedef struct pfmp_op pfmp_op;

/* Text of a status code (static storage). */
const char* pfmp_strerror(int status);
/* Text of the most recent error on this host thread ("" if none). */
const char* pfmp_last_error(void);
/* Library version, as major*10000 + minor*100 + patch. */
int pfmp_version(void);
/* Number of CUDA kernels this library has launched in this process (all contexts).  */
int64_t pfmp_launch_count(void);

/* ---- context: lattice geometry, stream, gauge field ---------------------------------
 * pfmp_ctx_create: dims = {Lx, Ly, Lz, Lt} (all even, >= 2); bc_t = +1 or -1 is the
 * fermion time boundary factor; stream is a cudaStream_t (NULL: the legacy default
 * stream) borrowed, not owned.  Allocates the gauge field (FP64 master copy, read in full
 * by the FP64 stencil, plus FP32, FP16 and double-float copies, the FP32 and FP16 ones
 * 12-real) and reduction scratch on the current device.
 * Errors: PFMP_E_INVALID (odd or non-positive extent, |bc_t| != 1), PFMP_E_NOMEM.   */
int pfmp_ctx_create(pfmp_ctx** ctx, const int dims[4], int bc_t, void* stream);
int pfmp_ctx_destroy(pfmp_ctx* ctx);
int pfmp_ctx_set_stream(pfmp_ctx* ctx, void* stream);
/* Sites per parity (V/2). */
int64_t pfmp_half_volume(const pfmp_ctx* ctx);
/* Bytes of one single-parity spinor field of precision prec in the device layout. */
int64_t pfmp_spinor_bytes(const pfmp_ctx* ctx, int prec);

/* Gauge field in the canonical layout ([V][4][3][3] complex double), from host or
 * device memory (where = PFMP_HOST / PFMP_DEVICE).  Links must be SU(3): the 12-real
 * FP32 and FP16 copies keep two rows and rebuild the third as conj(row0 x row1).
 * Setting the gauge field invalidates every operator's clover term until
 * pfmp_op_update().                                                                  */
int pfmp_gauge_set(pfmp_ctx* ctx, const double* U, int where);
int pfmp_gauge_get(pfmp_ctx* ctx, double* U, int where);
/* Field initialisation: U_mu(x) = exp(i eps H_mu(x)), H = sum_a h_a T_a with the
 * coefficients h[V][4][8] (canonical order, host or device).  exp by scaling and
 * squaring of the Taylor series, then reunitarised (rows Gram-Schmidt, row2 = cross).*/
int pfmp_gauge_from_algebra(pfmp_ctx* ctx, const double* h, double eps, int where);
/* Mean plaquette <Re tr U_{mu nu}>/3 over all sites and planes (synchronises).       */
int pfmp_plaquette(pfmp_ctx* ctx, double* plaq);

/* ---- spinor layout conversion --------------------------------------------------------
 * pack: take the sites of parity `parity` (0 even, 1 odd) out of a canonical full-lattice
 * spinor ([V][4][3] complex double, host or device) into the device field dst of
 * precision prec.  unpack: write a parity field back into the canonical array; in
 * device memory the other parity's sites are left untouched, in host memory they are
 * written as zero (the whole array is copied back).                                  */
int pfmp_spinor_pack(pfmp_ctx* ctx, void* dst, int prec, const double* src, int where, int parity);
int pfmp_spinor_unpack(pfmp_ctx* ctx, double* dst, int where, const void* src, int prec, int parity);

/* ---- the fermion operator ------------------------------------------------------------
 * pfmp_op_create: an operator at (kappa, c_sw) on the context's gauge field.  Builds the
 * clover blocks A (even sites) and A^{-1} (odd sites) in FP64 and FP32, and
 * sum_{x odd} log det A(x).  A must be positive definite (Cholesky); otherwise
 * PFMP_E_NAN.  pfmp_op_update rebuilds them after the gauge field changed.          */
int pfmp_op_create(pfmp_ctx* ctx, double kappa, double csw, pfmp_op** op);
int pfmp_op_update(pfmp_op* op);
int pfmp_op_destroy(pfmp_op* op);
/* sum over odd sites of log det A(x) (host scalar; synchronises).                    */
int pfmp_op_logdet(pfmp_op* op, double* logdet_oo);
/* Threads per output site of the stencil kernels of this operator for one arithmetic
 * (prec = PFMP_F64, PFMP_F32 or PFMP_DF): 1, 2, 4 or 8.  Splitting a site's 8 hop terms
 * across threads adds parallelism where the kernel is latency- or ALU-bound (small
 * lattices, FP64, double-float).  Results differ only by summation order.  The default
 * comes from pfmp_op_create (a fixed rule on precision and lattice size, so runs are
 * reproducible); pfmp_op_get_split reads it.                                         */
int pfmp_op_set_split(pfmp_op* op, int prec, int nsplit);
int pfmp_op_get_split(pfmp_op* op, int prec, int* nsplit);
/* Threads per block of this operator's stencil kernels (32, 64, 96 or 128; default from
 * pfmp_op_create: the lattice's sites per parity spread over the SMs in whole waves).  */
int pfmp_op_set_block(pfmp_op* op, int threads);

/* Wilson hop restricted to one parity: out (parity out_parity) = H_{out,in} in; with
 * dagger = 1 the adjoint hop H^dag (projectors (1 + g_mu) forward, (1 - g_mu) back).  */
int pfmp_dslash(pfmp_op* op, int prec, void* out, const void* in, int out_parity, int dagger);
/* out = A in (inverse = 0, even parity only) or A^{-1} in (inverse = 1, odd parity only):
 * the blocks the even-odd operator needs.                                            */
int pfmp_clover_apply(pfmp_op* op, int prec, void* out, const void* in, int parity, int inverse);
/* out = M-hat in (dagger = 0) or M-hat^dag in (dagger = 1); even parity fields.      */
int pfmp_mhat(pfmp_op* op, int prec, void* out, const void* in, int dagger);
/* Allocation-free M-hat (no counterpart in the paper: a library convenience).  The same
 * result as pfmp_mhat (same kernels, bit-identical output), for callers that may not
 * allocate or free device memory while they run: a host callback or a latency-bound
 * loop with no room for an allocation (cudaFree also synchronises the device), or a
 * framework whose memory pool owns all device memory.  Its odd-site temporary is a
 * fixed array of PFMP_NOALLOC_SCRATCH_BYTES (64 MiB) inside the library image, held by
 * every GPU that loads the library until exit; a lattice whose temporary
 * (pfmp_spinor_bytes(ctx, prec)) is larger is rejected with PFMP_E_INVALID (FP64: up to
 * 349,525 sites per parity, e.g. 24^3 x 48; FP32: twice that).  prec must be PFMP_F64
 * or PFMP_F32 (PFMP_H16, which pfmp_mhat accepts, is rejected with PFMP_E_INVALID), and
 * the operator's device must be the current device (PFMP_E_INVALID otherwise).  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress).
 * Nothing is allocated or freed.  All calls share the array: calls that overlap on the
 * GPU (different streams or threads at once) race on it; other entry points, which use
 * the operator's own temporaries, do not touch it.                                   */
#define PFMP_NOALLOC_SCRATCH_BYTES (64ll * 1024 * 1024)
int pfmp_mhat_noalloc(pfmp_op* op, int prec, void* out, const void* in, int dagger);
/* out = K in = M-hat^dag M-hat in; if in_K_in is not NULL it receives <in, K in> =
 * ||M-hat in||^2 in FP64 (synchronises).                                             */
int pfmp_kop(pfmp_op* op, int prec, void* out, const void* in, double* in_K_in);

/* True residual r = b - K x of FP64 even fields (x, b, r), K applied in FP64
 * (arith = PFMP_F64) or in double-float, FP32 pairs on the FP32 pipe with ~48-bit
 * significands (arith = PFMP_DF, what the mixed solvers use for their reliable updates).
 * rel (host, may be NULL) receives ||r|| / ||b||.  Synchronises.                     */
#define PFMP_DF 2
int pfmp_true_residual(pfmp_op* op, int arith, void* r, const void* x, const void* b, double* rel);

/* ---- BLAS-1 on single-parity fields (FP64 global sums) ----------------------------- */
int pfmp_norm2(pfmp_ctx* ctx, int prec, const void* x, double* result);  /* synchronises */
int pfmp_cdot(pfmp_ctx* ctx, int prec, const void* x, const void* y, double result[2]);
int pfmp_axpy(pfmp_ctx* ctx, int prec, double a_re, double a_im, const void* x, void* y); /* y += a x */
int pfmp_convert(pfmp_ctx* ctx, void* dst, int dst_prec, const void* src, int src_prec);

/* ---- solvers on K (Sec. 2.1: CG; Sec. 3.1 and App. C: multi-shift CG) ---------------- */
#define PFMP_SOLVER_CG64 0      /* CG in FP64 throughout                                 */
#define PFMP_SOLVER_CG_MIXED 1  /* FP32 CG with FP64 reliable updates (true residual in  */
                                /* FP64, solution accumulated in FP64)                    */
#define PFMP_SOLVER_CG_HALF 2   /* the same with the stencil on FP16 storage (p and Kp    */
                                /* FP16 with per-site scales, x and r FP32, FP32 sums    */
                                /* per thread); delta ~ 1e-2..1e-1 suits FP16            */
typedef struct {
  int method;        /* PFMP_SOLVER_*                                                     */
  double tol;        /* stop when ||b - K x|| / ||b|| < tol, residual recomputed in FP64  */
  int max_iter;      /* iteration cap -> PFMP_E_NOT_CONVERGED                              */
  double delta;      /* mixed: reliable update when the sloppy residual fell by delta      */
  int check_every;   /* iterations per CUDA-graph chunk between host checks (0: default 8) */
  int restart;       /* FGCR: directions kept before a restart (0: default 16)            */
} pfmp_solver_params;

typedef struct {
  int iters;             /* CG iterations                                                 */
  int reliable_updates;  /* FP64 residual recomputations (mixed)                         */
  double true_rel_res;   /* ||b - K x|| / ||b|| recomputed in FP64 at exit                */
  int64_t k_apply;       /* applications of K (either precision)                         */
  int status;            /* PFMP_OK or PFMP_E_NOT_CONVERGED / PFMP_E_NAN                  */
} pfmp_solve_info;

/* x = K^{-1} b with zero initial guess; x, b FP64 even-parity device fields (x may not
 * alias b).  Synchronises; info may be NULL.                                          */
int pfmp_solve(pfmp_op* op, const pfmp_solver_params* params, void* x, const void* b,
               pfmp_solve_info* info);
/* The same call through host memory: b and x are canonical full-lattice spinors in
 * host memory ([V][4][3] complex double; even sites of b are read, x receives the
 * solution on even sites and zero on odd sites).  Copies in, packs, solves, unpacks
 * and copies out inside the call.                                                     */
int pfmp_solve_host(pfmp_op* op, const pfmp_solver_params* params, double* x_host,
                    const double* b_host, pfmp_solve_info* info);

/* ---- multi-shift CG (Sec. 3.1; App. C eq. force_polycorr) ---------------------------
 * x[k] = (K + sigma_k)^{-1} b for nshift complex shifts sigma_k = (sigma_re[k],
 * sigma_im[k]) from one Krylov space of K (the seed system), FP64.  x[k] are FP64 even
 * device fields owned by the caller (nshift <= 1024).  A shift stops being updated once
 * its residual |zeta_k| ||r|| is below tol ||b||; the solve ends when every shift has.  If info is not NULL,
 * info->true_rel_res receives max_k ||b - (K + sigma_k) x_k|| / ||b|| recomputed in
 * FP64 (one extra K per shift).  A shift that is not finite, or real and negative (K is
 * positive definite, so K + sigma can be singular only there), is refused with
 * PFMP_E_INVALID; a right-hand side that is not finite gives PFMP_E_NAN.  Synchronises. */
int pfmp_solve_multishift(pfmp_op* op, int nshift, const double* sigma_re, const double* sigma_im, void* const* x,
                          const void* b, double tol, int max_iter, pfmp_solve_info* info);

/* The same in FP64 (prec = PFMP_F64, as above) or FP32 (PFMP_F32): x[k] and b FP32 even
 * fields, K on the FP32 stencil, FP64 global sums and recurrence scalars; each shift
 * stops once its recursive residual |zeta_k| ||r|| is below tol ||b|| (tol >= ~1e-6 in
 * FP32, where the recursive residual departs from the true one).  This is the solver of
 * the FP32 filter-correction force of the MD.  info->true_rel_res is -1 for FP32.      */
int pfmp_solve_multishift_prec(pfmp_op* op, int prec, int nshift, const double* sigma_re, const double* sigma_im,
                               void* const* x, const void* b, double tol, int max_iter, pfmp_solve_info* info);

/* ---- Chebyshev polynomial filter (App. A) --------------------------------------------
 * P_n(z) = a_n prod_{k=1}^n (z - z_k), z_k = mu (1 - cos t_k) - i sqrt(mu^2 - nu^2) sin t_k,
 * t_k = 2 pi k / (n+1), a_n = 1 / (mu prod_k (mu - z_k)).  pfmp_poly_roots writes the n
 * roots and a_n.  pfmp_poly_apply: out = P_n(K) in (which = 0), R(K) in (which = 1) or
 * R(K)^dag in (which = 2), R = sqrt(a_n) prod_{Im z_k < 0} (K - z_k) so that P = R^dag R;
 * FP64 even fields.  The factors commute; they are applied in bit-reversed order of
 * their index, which keeps every partial product close in size to the final one (in
 * index order the partial products of P_64 grow 1e11-fold and amplify the rounding of
 * each factor).  Even n only (PFMP_E_UNSUPPORTED otherwise), mu >= nu > 0.             */
int pfmp_poly_roots(int n, double mu, double nu, double* z_re, double* z_im, double* a_n);
int pfmp_poly_apply(pfmp_op* op, int n, double mu, double nu, int which, void* out, const void* in);

/* ---- spectral range (App. A) ----------------------------------------------------------
 * The filter approximates K^{-1} only inside its ellipse (0 to 2 mu on the real axis),
 * so (mu, nu) must enclose the spectrum of K.  pfmp_spectrum runs nsteps steps of the
 * Lanczos recurrence on K (FP64, no reorthogonalisation) from the start vector v0 (FP64
 * even device field, non-zero; not modified) and returns the extreme eigenvalues of the
 * Lanczos tridiagonal T_k: lambda_min <= *lmin and *lmax <= lambda_max, converging to
 * them (lmax within a few tens of steps, lmin more slowly, as sqrt of the condition
 * number).  *steps = k, fewer than nsteps when the Krylov space closed.  alpha, beta
 * (host arrays of nsteps, optional): the diagonal and off-diagonal of T_k.
 * PFMP_E_INVALID for a zero start vector or nsteps < 1.  Synchronises.                 */
int pfmp_spectrum(pfmp_op* op, int nsteps, const void* v0, double* lmin, double* lmax, double* alpha, double* beta,
                  int* steps);

/* ---- actions, forces, trajectory (Sec. 2.1-2.5, Sec. 3.6, App. A-C) ----------------
 * An action is a list of terms over hopping parameters kappa[0..nkappa) that share c_sw.
 * kappa[0] is the target operator K = M-hat^dag M-hat; J_a = W_a^dag W_a with
 * W_a = M-hat at kappa[a] (J_0 = K).  Term kinds:
 *   GAUGE       S_G = beta sum_{x,mu<nu} (1 - Re tr U_{mu nu} / 3)        (Table 3.1)
 *   DET         S_det = -2 sum_{x odd} log det A(x) at kappa[a]            (even-odd clover)
 *   FILTER      phi^dag Q(J_a) phi, Q = P_p2 / P_p1 (Sec. 2.3 eq. 2poly; p1 = 0: P_p2;
 *               otherwise (p1 + 1) must divide (p2 + 1), App. A)
 *   FILTERCORR  phi^dag [J_a P_p2(J_a)]^{-1} phi                          (eqs. 1poly, pfmp_action)
 *   RATIO       phi^dag W_a K_b^{-1} W_a^dag phi: the paper's "J_a K_b^{-1}" (Sec. 2.2) in
 *               its Hermitian form, K_b = J_b
 *   INV         phi^dag J_a^{-1} phi                                       (eq. hasenbusch)
 * Every fermion term (FILTER, FILTERCORR, RATIO, INV) owns one pseudofermion; they are
 * numbered in term order.  Heatbath from Gaussian noise xi (density exp(-xi^dag xi)), so
 * that each S_i(phi_i) = xi_i^dag xi_i:  FILTER phi = R_Q(J_a)^{-1} xi with
 * R_Q = sqrt(c) prod_{Im q_k < 0} (J_a - q_k) (Q = c prod (z - q_k));  FILTERCORR
 * phi = R_p2(J_a)^dag W_a^dag xi;  RATIO phi = W_a J_a^{-1} M_b^dag xi;  INV phi = W_a^dag xi.
 * Forces are the algebra coefficients dS/d omega_a for U -> exp(i omega_a T_a) U:
 * FILTER App. C eq. force_poly with the roots of Q (2q - 2 J products), FILTERCORR eq.
 * force_polycorr (one multi-shift solve with z_{p2+1} = 0), RATIO
 * 2 Re chi^dag dW_a^dag phi - chi^dag dK_b chi with chi = K_b^{-1} W_a^dag phi (one CG),
 * INV -chi^dag dJ_a chi with chi = J_a^{-1} phi (one CG).  All FP64.
 * The PF-MP action of Sec. 2.5 (pfmp_action_create) is the term list GAUGE, DET(0),
 * FILTER(1, 0, n), FILTERCORR(1, n), RATIO(1, 0) over kappa = {kappa, kappa_h}.        */
#define PFMP_KIND_GAUGE 0
#define PFMP_KIND_DET 1
#define PFMP_KIND_FILTER 2
#define PFMP_KIND_FILTERCORR 3
#define PFMP_KIND_RATIO 4
#define PFMP_KIND_INV 5
#define PFMP_MAX_TERMS 8
#define PFMP_MAX_KAPPA 4
/* term indices of the PF-MP action */
#define PFMP_TERM_GAUGE 0
#define PFMP_TERM_DET 1
#define PFMP_TERM_POLY 2
#define PFMP_TERM_POLYCORR 3
#define PFMP_TERM_HASEN 4
typedef struct pfmp_action pfmp_action;
typedef struct {
  int kind;        /* PFMP_KIND_*                                                       */
  int a, b;        /* kappa indices: J_a / W_a, and K_b of RATIO                        */
  int p1, p2;      /* filter orders (FILTER: Q = P_p2 / P_p1; FILTERCORR: order p2)     */
} pfmp_term;
typedef struct {
  double beta, csw;
  int nkappa;                         /* 1..PFMP_MAX_KAPPA                             */
  double kappa[PFMP_MAX_KAPPA];       /* kappa[0]: the target operator                 */
  int nterms;                         /* 1..PFMP_MAX_TERMS                             */
  pfmp_term term[PFMP_MAX_TERMS];
  double mu, nu;                      /* Chebyshev ellipse of every filter             */
  double tol;                         /* relative residual of every solve              */
  int max_iter;
  int solver;                         /* CG of the action: PFMP_SOLVER_CG64 (default 0) or
                                         PFMP_SOLVER_CG_MIXED (FP32 iterations, FP64-
                                         accurate true residual); multi-shift stays FP64 */
  int force_prec;                     /* arithmetic of the fermion forces of the MD:
                                         PFMP_F64 (default 0) or PFMP_F32 (spinor products,
                                         filter K chains and the correction term's multi-
                                         shift solve in FP32, CG as `solver`, contractions
                                         summed into the FP64 force; the actions, heatbath
                                         and Hamiltonian stay as before)                  */
  double md_tol;                      /* relative residual of the solves inside the MD
                                         forces (0: tol); with PFMP_F32 forces the FP32
                                         multi-shift solve needs md_tol >= ~1e-6          */
} pfmp_action_def;
typedef struct {
  double beta, kappa, kappa_h, csw;  /* gauge coupling, target and Hasenbusch kappa, c_sw */
  int n;                             /* polynomial order (even)                          */
  double mu, nu;                     /* Chebyshev ellipse                                 */
  double tol;                        /* relative residual of every solve in the action    */
  int max_iter;
} pfmp_action_params;
typedef struct {
  double H0, H1, dH;
  int accepted;
  double S0[PFMP_MAX_TERMS], S1[PFMP_MAX_TERMS];  /* per term at start and end (0 if left out) */
  double plaquette;        /* after the accept/reject decision                             */
  int64_t k_apply;         /* K and J applications (every operator, solves included)       */
  int force_evals;         /* term force evaluations                                        */
  int64_t k_apply_term[PFMP_MAX_TERMS];  /* ... of them spent in each term's forces          */
  int nforce[PFMP_MAX_TERMS];            /* force evaluations of each term                   */
  double fmax[PFMP_MAX_TERMS];  /* max over the trajectory of max_links |F|, |F| = sqrt(sum_a f_a^2) */
  double favg[PFMP_MAX_TERMS];  /* mean over the trajectory of the link average of |F|      */
  double ms_force[PFMP_MAX_TERMS];  /* wall time of each term's force evaluations (ms)       */
  double ms_update;                 /* wall time of the link updates with the rebuild of the
                                       compressed copies and clover terms (ms)              */
  double ms_total;                  /* wall time of the whole call (ms)                     */
} pfmp_traj_info;
/* Schemes compared in Sec. 3 (term lists; kappa[1], kappa[2] are the Hasenbusch kappas):
 *   1PF      GAUGE, DET, FILTER(0; p2), FILTERCORR(0; p2)              (eq. 1poly on K)
 *   2PF      GAUGE, DET, FILTER(0; p1), FILTER(0; p1, p2), FILTERCORR(0; p2)   (eq. 2poly)
 *   1MP      GAUGE, DET, INV(1), RATIO(1, 0)                           (eq. hasenbusch)
 *   2MP      GAUGE, DET, INV(1), RATIO(1, 2), RATIO(2, 0)
 *   PF-MP    GAUGE, DET, FILTER(1; p2), FILTERCORR(1; p2), RATIO(1, 0) (eq. pfmp_action)
 *   2PF-1MP  GAUGE, DET, FILTER(1; p1), FILTER(1; p1, p2), FILTERCORR(1; p2), RATIO(1, 0)
 *   1PF-2MP  GAUGE, DET, FILTER(1; p2), FILTERCORR(1; p2), RATIO(1, 2), RATIO(2, 0)
 * pfmp_action_scheme fills def->nterms and def->term and leaves the other fields.      */
#define PFMP_SCHEME_1PF 0
#define PFMP_SCHEME_2PF 1
#define PFMP_SCHEME_1MP 2
#define PFMP_SCHEME_2MP 3
#define PFMP_SCHEME_PFMP 4
#define PFMP_SCHEME_2PF1MP 5
#define PFMP_SCHEME_1PF2MP 6
int pfmp_action_scheme(int scheme, int p1, int p2, pfmp_action_def* def);
/* PFMP_E_INVALID for out-of-range kinds, kappa indices or counts; PFMP_E_UNSUPPORTED for
 * odd filter orders or orders that do not factorise.                                    */
int pfmp_action_create_def(pfmp_ctx* ctx, const pfmp_action_def* def, pfmp_action** action);
int pfmp_action_create(pfmp_ctx* ctx, const pfmp_action_params* prm, pfmp_action** action);
int pfmp_action_destroy(pfmp_action* action);
/* number of terms and of pseudofermions                                                 */
int pfmp_action_counts(pfmp_action* action, int* nterms, int* npf);
/* rebuild the clover blocks after pfmp_gauge_set                                      */
int pfmp_action_refresh(pfmp_action* action);
/* xi: npf canonical spinors ([npf][V][4][3] complex double; even sites used)           */
int pfmp_action_heatbath(pfmp_action* action, const double* xi, int where);
int pfmp_action_get_phi(pfmp_action* action, int i, double* phi, int where);
int pfmp_action_set_phi(pfmp_action* action, int i, const double* phi, int where);
/* S[nterms] per term at the current gauge field (synchronises)                         */
int pfmp_action_eval(pfmp_action* action, double* S);
/* force of one term, canonical [V][4][8]                                               */
int pfmp_action_force(pfmp_action* action, int term, double* F, int where);
/* 2MN arrays of eq. 2MNSTS chained n times over tau: T and S of length 2n + 1          */
int pfmp_schedule_2mn(int n, double tau, double lambda, double* T, double* S);
/* generalised multi-scale merge (App. B): nschemes schemes, scheme i given by len[i]
 * entries of T and S (concatenated); writes the merged T_out[cap] and
 * S_out[nschemes][cap] and the merged length.                                          */
int pfmp_schedule_merge(int nschemes, const int* len, const double* T, const double* S, int cap, double* T_out,
                        double* S_out, int* len_out);
/* One trajectory: heatbath from xi ([npf] canonical spinors), H0, the merged schedule
 * (T[len], S[nlevels][len]), term t integrated on level term_level[t] (nterms entries;
 * -1: term left out of H and of the MD), H1, Metropolis accept iff u < exp(-dH); a
 * rejected trajectory restores the gauge field.  mom: initial momenta, canonical
 * [V][4][8].  Synchronises.                                                             */
int pfmp_trajectory(pfmp_action* action, int len, const double* T, int nlevels, const double* S,
                    const int* term_level, const double* mom, const double* xi, int where, double u,
                    pfmp_traj_info* info);

/* MD alone (Sec. 2.1, App. B): evolve the gauge field and the momenta mom (canonical
 * [V][4][8], read and overwritten) along the merged schedule with the pseudofermions the
 * action holds (from pfmp_action_heatbath or _set_phi); term_level as for
 * pfmp_trajectory.  No heatbath, no Hamiltonian, no accept/reject.  With mom negated
 * the scheme runs backwards (time reversibility).  Synchronises.                      */
int pfmp_md(pfmp_action* action, int len, const double* T, int nlevels, const double* S, const int* term_level,
            double* mom, int where);

/* ---- step-size balancing and cost (Sec. 2.4 eq. force_tune, Sec. 3.1 eqs. cost_func,
 * error_corrected) ---------------------------------------------------------------------
 * pfmp_balance_steps: step counts over tau for nlev levels from each level's maximal
 * force fmax[l] (e.g. the largest pfmp_traj_info.fmax of the terms on it) so that
 * F_l h_l = constant (h = tau / n): anchored at the level with the smallest force, which
 * keeps n_coarse steps; n[l] = max(1, round(n_coarse fmax[l] / fmax_min)).
 * pfmp_cost: over ntraj trajectories, P_acc = mean(accepted), N_mat = mean(nmat),
 * C = N_mat / P_acc, <exp(-dH)>, each with sigma = sqrt(2 tau_int) sigma_p / sqrt(N)
 * (sigma_p the sample standard deviation); the error of C by linear propagation.
 * PFMP_E_INVALID for ntraj < 2, a non-positive force or n_coarse < 1.  Host only.      */
typedef struct {
  double p_acc, p_acc_err, nmat, nmat_err, cost, cost_err, exp_mdh, exp_mdh_err;
} pfmp_cost_info;
int pfmp_balance_steps(int nlev, const double* fmax, int n_coarse, int* n);
int pfmp_cost(int ntraj, const int* accepted, const double* nmat, const double* dH, double tau_int,
              pfmp_cost_info* info);

/* ---- batched solves ------------------------------------------------------------------
 * Many independent systems K_s x = b (each operator on its own context: lattice, gauge
 * field, kappa; nrhs[s] right-hand sides each, 1..64) solved together in ONE persistent
 * cooperative launch: its blocks take (system, site block, rhs) tiles phase after phase
 * with grid barriers in between, FP32 CG iterations per rhs with reliable updates on the
 * device (x accumulated in FP64, r = b - K x with K in double-float), as in
 * PFMP_SOLVER_CG_MIXED; a rhs whose double-float residual is below tol stops, and the
 * host confirms it with K in FP64 afterwards (relaunching for any it does not confirm).
 * Every barrier wait is bounded (2 s): a wait that runs out ends the launch with
 * PFMP_E_TIMEOUT instead of hanging.  All contexts must live on the current device; the
 * first operator's stream is used for everything during a solve; the operators' clover
 * terms must be current and built in FP64 (pfmp_op_update).  x and b are the sum(nrhs)
 * FP64 even device fields in system order (x overwritten).  check_every is not used.
 * pfmp_batch_tune times one launch of `chunk` iterations for block sizes 64/128/256 and
 * keeps the fastest (call before a solve; it overwrites the batch workspace).  infos
 * (optional) receives one entry per rhs.  Memory: 12 FP32 half-lattice fields per rhs.
 * pfmp_batch_barrier_check runs `rounds` grid barriers of the batch's launch shape with
 * `missing` more blocks expected than launched (no paper counterpart; it tests the
 * bounded wait): missing = 0 returns PFMP_OK, missing > 0 makes every wait run out after
 * limit_s (0 < limit_s <= 10) and returns PFMP_E_TIMEOUT with the context still usable. */
typedef struct pfmp_batch pfmp_batch;
int pfmp_batch_create(int nsys, pfmp_op* const* ops, const int* nrhs, pfmp_batch** batch);
int pfmp_batch_destroy(pfmp_batch* batch);
int pfmp_batch_tune(pfmp_batch* batch, int chunk, int* block, double* ms_per_chunk);
int pfmp_batch_solve(pfmp_batch* batch, const pfmp_solver_params* params, void* const* x, const void* const* b,
                     pfmp_solve_info* infos);
int pfmp_batch_barrier_check(pfmp_batch* batch, int rounds, int missing, double limit_s);

/* ---- learned preconditioner (no counterpart in the paper) ---------------------------
 * A gauge-covariant linear network N used as the preconditioner of FGCR: layer l maps
 * C_l channels to C_{l+1}, y_o(x) = sum_i [W0 a_i(x) + sum_mu (Wf_mu U_mu(x) a_i(x+mu)
 * + Wb_mu U_mu(x-mu)^dag a_i(x-mu))] with complex 4x4 spin matrices W (9 per channel
 * pair) and the fermion boundary factor on time hops; channels[0] = channels[L] = 1;
 * input embedded on even sites, output read on even sites.  prec is the arithmetic of
 * the network kernels (FP32 for use in FGCR, FP64 for gradient checks).  Weights are
 * host arrays of complex doubles (re, im interleaved), layers concatenated, each
 * W[9][c_out][c_in][4][4] with index 0 = site, 1+mu forward hop, 5+mu backward hop.
 * Training: Adam (beta 0.9, 0.999) over (b, x = K^{-1} b) pairs of FP64 even device
 * fields, batch pairs per step, cycling through the pairs, on one of two losses:
 *   PFMP_NN_LOSS_SOLUTION  L = ||N(b) - x||^2 / ||x||^2
 *   PFMP_NN_LOSS_RESIDUAL  L = ||K N(b) - b||^2 / ||b||^2 (needs op; K N close to the
 *                          identity is what a right preconditioner of K needs)        */
#define PFMP_NN_LOSS_SOLUTION 0
#define PFMP_NN_LOSS_RESIDUAL 1
typedef struct pfmp_nn pfmp_nn;
int pfmp_nn_create(pfmp_ctx* ctx, int nlayers, const int* channels, int prec, pfmp_nn** nn);
int pfmp_nn_destroy(pfmp_nn* nn);
int64_t pfmp_nn_num_weights(const pfmp_nn* nn);
int pfmp_nn_set_weights(pfmp_nn* nn, const double* w);
int pfmp_nn_get_weights(pfmp_nn* nn, double* w);
/* out = N(in), even fields of precision prec in the library layout (synchronises)      */
int pfmp_nn_apply(pfmp_nn* nn, int prec, void* out, const void* in);
/* Tensor-core inference (default on for FP32 networks with 1 -> 8, 8 -> 8 or 8 -> 1
 * layers): those layers of pfmp_nn_apply (FP32 io) and of FGCR run as tcgen05 MMAs on
 * FP16 operands
 * (inputs scaled by 1 / rms of the network input, weights packed as [[Re, -Im], [Im,
 * Re]]) with FP32 accumulation; training always uses the FP32 kernels.  on = 0 selects
 * the FP32 kernels everywhere.  PFMP_E_UNSUPPORTED if the network has no such layer;
 * PFMP_E_TIMEOUT from pfmp_nn_apply / pfmp_solve_fgcr if a tensor-core kernel gave up
 * waiting for its MMAs (bounded waits; the context stays usable).                       */
int pfmp_nn_set_tensor_cores(pfmp_nn* nn, int on);
/* loss of one pair and its gradient dL/dRe W + i dL/dIm W (grad: host, may be NULL)     */
int pfmp_nn_loss_grad(pfmp_nn* nn, pfmp_op* op, int kind, const void* b, const void* x, double* loss, double* grad);
int pfmp_nn_train(pfmp_nn* nn, pfmp_op* op, int kind, int npairs, const void* const* b, const void* const* x, int steps,
                  int batch, double lr, double* final_loss);
/* FGCR on K with N as the flexible preconditioner (nn = NULL: GCR), FP32 inner
 * iterations of params->restart directions, stopped when the inner residual fell by
 * params->delta; FP64 outer correction x += e and true residual b - K x; after two
 * outer passes without a 10% gain the rest is solved by the mixed CG (info->
 * reliable_updates then counts those CG iterations).  info->iters counts inner FGCR
 * iterations.  FP64 x, b.                                                              */
int pfmp_solve_fgcr(pfmp_op* op, pfmp_nn* nn, const pfmp_solver_params* params, void* x, const void* b,
                    pfmp_solve_info* info);

/* ---- kernel timing (tracing) ------------------------------------------------------
 * pfmp_profile_begin: from now on every stencil launch of this context is bracketed by
 * CUDA events on the context's stream.  pfmp_profile_end (synchronises) stops recording
 * and reports, for one kernel class, the number of launches, their summed device time
 * in milliseconds, and their summed algorithmic DRAM bytes (per output site: 8 links of
 * 12 reals, one input and one output spinor of 24 reals, plus 72 clover reals and 24
 * local-input reals for the fused even-odd epilogues).                              */
#define PFMP_KERNEL_HOP_F32 0
#define PFMP_KERNEL_HOP_F64 1
#define PFMP_KERNEL_HOP_DF 2   /* double-float (FP32-pair) stencil of the true residual   */
#define PFMP_KERNEL_HOP_H16 3  /* FP16-storage stencil (PFMP_SOLVER_CG_HALF)              */
#define PFMP_KERNEL_CG_F32 4   /* the FP32 CG iteration's four stencil kernels with the CG
                                  vector updates fused in (PFMP_SOLVER_CG_MIXED); bytes count
                                  the CG vectors each reads or writes as well            */
int pfmp_profile_begin(pfmp_ctx* ctx);
int pfmp_profile_end(pfmp_ctx* ctx, int kernel_class, int64_t* launches, double* total_ms, double* total_bytes);
/* Measured FMA throughput of the current GPU on the FP64 (prec = PFMP_F64) or FP32
 * (PFMP_F32) pipe, in TFLOP/s (an FMA counts two flops): a dedicated kernel of
 * independent register FMA chains, 8 blocks of 256 threads per SM, timed by CUDA events
 * on the context's stream after one warm-up launch.  It is the arithmetic roofline of
 * the FP64 stencil and of the double-float stencil (no counterpart in the paper).
 * Synchronises.                                                                      */
int pfmp_fma_rate(pfmp_ctx* ctx, int prec, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* PFMP_H */
