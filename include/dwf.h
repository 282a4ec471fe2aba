/*
 * dwf.h -- C ABI of the GB300 (sm_103a) multisplitting-preconditioned CG solver
 * for the even-odd preconditioned Shamir/Moebius domain-wall-fermion system.
 *
 * Paper: J. Tu, "Solving DWF Dirac Equation Using Multisplitting Preconditioned
 * Conjugate Gradient", LATTICE2018 (arXiv:1811.08488).
 *
 * Operator (paper Sec. 2.2, the even-odd block system and eq. (dirac_equation)):
 *
 *     [ M_5      M^4_eo ] [psi_e]   [phi_e]
 *     [ M^4_oe   M_5    ] [psi_o] = [phi_o],    D_PC = M_5 - M^4_eo M_5^-1 M^4_oe,
 *
 * with M^4 = D^w M_phi (eq. for D^w). The paper defers the entries of M_5 and
 * M_phi to Brower et al. (2014); this library uses the standard Moebius form
 *
 *     Dhop psi(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu)
 *     M^4         = -1/2 Dhop M_phi,      M_phi = b + c C,      M_5 = alpha + beta C,
 *     alpha = b (4 - M5) + 1,   beta = c (4 - M5) - 1,
 *     (C psi)_s   = P_- psi_{s+1} + P_+ psi_{s-1},  psi_{Ls} = -m_f psi_0, psi_{-1} = -m_f psi_{Ls-1},
 *
 * in the chiral gamma basis g_k = [[0,-i s_k],[i s_k,0]], g_4 = [[0,1],[1,0]],
 * g_5 = diag(1,1,-1,-1), P_+- = (1 +- g_5)/2. Shamir is b = 1, c = 0.
 * Boundary conditions: periodic in x, y, z; antiperiodic in t unless disabled.
 * The solve is the normal equation D_PC^+ D_PC psi_e = b (eq. (normal_equation)).
 *
 * ---------------------------------------------------------------------------
 * Layouts
 * ---------------------------------------------------------------------------
 * Sites: lexicographic index idx = ((t*Lz + z)*Ly + y)*Lx + x; parity
 * (x+y+z+t) mod 2 (paper eq. parity); the half index of a site is idx/2, so the
 * sites of one parity are numbered 0 .. V/2-1.
 *
 * Gauge field (input to dwf_gauge_load): complex128 U[t][z][y][x][mu][a][b],
 * mu = 0..3 for x, y, z, t, U_mu(x) the SU(3) matrix on the link x -> x+mu.
 *
 * Canonical half field (import/export and mspcg_solve): complex numbers
 * psi[rhs][s][t][z][y][xh][spin 4][colour 3], with x = 2*xh + ((parity+y+z+t)%2);
 * complex128 (canon_is_fp32 = 0) or complex64 (canon_is_fp32 = 1).
 *
 * Native half field (all operator entry points): one right-hand side after
 * another, each dwf_field_bytes(ctx, prec, 1) bytes (a multiple of 256).
 * Inside one right-hand side, the 24 reals of (site h, s) -- ordered
 * [spin][colour][re,im] -- are cut into 16-byte chunks, and chunk k is stored
 * for all (h, s) before chunk k+1 (chunk-major, s fastest), V = Vh = V4/2:
 *     DWF_FP64: 12 chunks of 2 doubles,  byte offset ((k*V + h)*Ls + s)*16
 *     DWF_FP32:  6 chunks of 4 floats,   byte offset ((k*V + h)*Ls + s)*16
 *     DWF_FP16/BF16: 3 chunks of 8 halves, byte offset ((k*V + h)*Ls + s)*16,
 *         followed (at the next 256-byte boundary) by one float scale per
 *         (h, s) at [h*Ls + s]; the stored value times the scale is the field.
 * Convert with dwf_field_import / dwf_field_export.
 *
 * ---------------------------------------------------------------------------
 * Conventions for every entry point
 * ---------------------------------------------------------------------------
 * - Field pointers are device pointers on the context's device unless stated.
 * - The caller owns every field buffer and the stream; `stream` is a
 *   cudaStream_t (NULL: the legacy default stream). Work is enqueued on it; the
 *   call returns without synchronising unless stated.
 * - `mf` is a HOST array of nrhs quark masses m_f (one per right-hand side).
 * - `nrhs` is 1 .. DWF_MAX_RHS.
 * - The context owns packed links, geometry tables, work buffers and plans; it
 *   allocates them on first need and frees them in dwf_destroy.
 * - A context must not be used from two host threads at once; work on two
 *   streams of one context that shares the context's work buffers races.
 * - The return code is the contract. On an error nothing is written to output
 *   buffers unless stated, and dwf_last_error() describes the failure. Nothing
 *   aborts the process.
 */
#ifndef DWF_H
#define DWF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DWF_MAX_RHS 16
#define DWF_MAX_LS 32
#define DWF_MAX_EIG 64

typedef enum {
  DWF_OK = 0,
  DWF_ERR_INVALID_ARG = 1,   /* bad pointer, size, shape or parameter        */
  DWF_ERR_UNSUPPORTED = 2,   /* valid request the library does not implement */
  DWF_ERR_CUDA = 3,          /* a CUDA call failed; see dwf_last_error        */
  DWF_ERR_NOT_CONVERGED = 4, /* maxiter reached; x and info are still filled  */
  DWF_ERR_TIMEOUT = 5,       /* a bounded device-side wait expired            */
  DWF_ERR_NAN = 6,           /* a NaN/Inf appeared in a solver scalar         */
  DWF_ERR_NO_GAUGE = 7       /* operator called before dwf_gauge_load         */
} dwf_status;

typedef enum { DWF_FP64 = 0, DWF_FP32 = 1, DWF_FP16 = 2, DWF_BF16 = 3 } dwf_prec;

/* The action: lattice and DWF parameters (paper Sec. 2.2). */
typedef struct {
  int dims[4];        /* Lx, Ly, Lz, Lt; all even                            */
  int Ls;             /* fifth-dimension extent, 2 .. DWF_MAX_LS              */
  double b, c;        /* Moebius coefficients (Shamir: b = 1, c = 0)         */
  double M5;          /* domain-wall height                                  */
  int t_antiperiodic; /* 1: antiperiodic in t (default), 0: periodic          */
  int recon12;        /* 1: FP32/FP16 links keep their first two rows and a   
                       * sign; the third row is rebuilt as the conjugate of   
                       * the cross product (SU(3)); 0: all 18 reals (default) */
} dwf_action;

/* Solver parameters. Start from dwf_solver_params_default(). */
typedef struct {
  double tol;         /* stop when |b - A x| / |b| <= tol (recomputed residual) */
  int maxiter;        /* maximum outer iterations                               */
  int inner_iters;    /* k fixed inner CG iterations per block; 0 = plain CG    */
  int block[4];       /* sub-lattice extents (even, dividing dims); all zero:   
                       * the block autotuner's shape (dwf_autotune_block)     */
  dwf_prec outer;     /* DWF_FP64 or DWF_FP32 (FP32: FP64 reliable updates)     */
  dwf_prec inner;     /* DWF_FP32, DWF_FP16 or DWF_BF16 block-solve storage     */
  double delta;       /* reliable update when |r| < delta * max|r| since last   */
  int snake;          /* 1: A_s = P_s A P_s (snake terms), 0: per-hop Dirichlet */
  int use_graph;      /* 1: the outer loop runs on the device as one CUDA graph 
                       * (a while-node over the iteration; after every      
                       * iteration a control kernel decides each rhs's       
                       * reliable update and convergence); the host waits   
                       * once per 256 iterations. 0: the host drives the     
                       * loop with eager launches, checking every            
                       * check_every iterations.                             */
  int io_on_host;     /* mspcg_solve: 1 = x and b are host pointers             */
  int check_every;    /* host-driven loop (use_graph 0): outer iterations      
                       * between host convergence checks, 1 .. 256            */
  int flexible;       /* 1: flexible PCG, beta = <r_new - r, z_new> / <r, z>    
                       * (Polak-Ribiere); 0: Algorithm 1's <r_new, z_new> /   
                       * <r, z> (Fletcher-Reeves)                             */
  int schur;          /* normal equation solved: 0 = D_PC^+ D_PC (the paper's   
                       * Schur complement D_PC = M_5 - M^4_eo M_5^-1 M^4_oe),   
                       * 1 = D_sym^+ D_sym with the symmetric form             
                       * D_sym = 1 - M_5^-1 M^4_eo M_5^-1 M^4_oe = M_5^-1 D_PC; 
                       * both outer operator and block operator follow it     */
  double inner_tol;   /* 0: every block runs inner_iters CG iterations (the     
                       * paper's fixed count); > 0: a block stops as soon as    
                       * its inner residual fell to inner_tol times its start  
                       * (at most inner_iters iterations)                     */
} dwf_solver_params;

/* Parameters of dwf_eig_lowmodes. Start from dwf_eig_params_default(). */
typedef struct {
  int n_ev;           /* wanted low modes, 1 .. m (the Ritz pairs tested for  
                       * convergence; the other m - n_ev guard the subspace) */
  int degree;         /* Chebyshev polynomial degree of one filter pass, >= 1 */
  int max_passes;     /* filter passes at most, >= 0                          */
  double tol;         /* stop once |A v - theta v| <= tol * lambda_max for the
                       * n_ev lowest Ritz pairs; 0: run max_passes passes     */
  double lambda_max;  /* upper bound of A's spectrum; <= 0: estimated as 1.1 x
                       * the Rayleigh quotient after power_steps power
                       * iterations from the first start vector              */
  int power_steps;    /* power iterations of the estimate, >= 1               */
  int schur;          /* the normal operator: 0 = D_PC^+ D_PC, 1 = D_sym^+ D_sym
                       * (as dwf_solver_params.schur)                         */
} dwf_eig_params;

/* Result of dwf_eig_lowmodes. */
typedef struct {
  int passes;         /* filter passes done                                   */
  int converged;      /* 1 when the n_ev lowest pairs met tol                 */
  long long matvecs;  /* applications of A (one per vector)                   */
  double lambda_max;  /* the upper bound used                                 */
  double seconds;     /* wall time of the call                                */
} dwf_eig_info;

/* Per right-hand-side result of mspcg_solve. */
typedef struct {
  int outer_iters;       /* outer (Algorithm 1) iterations                   */
  int inner_iters_total; /* inner CG iterations over the solve, averaged over
                          * the blocks (outer_iters * k without inner_tol)  */
  int reliable_updates;  /* FP64 residual recomputations                     */
  int converged;         /* 1 when true_resid <= tol                         */
  double true_resid;     /* |b - A x| / |b| recomputed in FP64               */
  double seconds;        /* wall time of the whole call (same for all rhs)   */
  double dslash_gbs;     /* compulsory bytes of the outer operator's hop     
                          * launches in params->outer precision during this 
                          * call, over their device time (GB/s; same for all
                          * rhs), from the hop-kernel timer; -1 when the     
                          * timer is off (dwf_profile_enable)               */
  int host_syncs;        /* host waits for the device in the outer loop     */
  int device_loop;       /* 1: convergence and reliable updates were decided
                          * on the device (use_graph), 0: by the host       */
} dwf_solve_info;

/* Device time of one hop-kernel family, from dwf_profile_read. */
typedef struct {
  char name[48];       /* kernel and template arguments, e.g.
                        * "hop2_kernel<F16,1,0,0,1>" (S, DAG, PRE, RECON, EPI) */
  long long launches;  /* launches since profiling was (re)enabled            */
  double seconds;      /* sum over launches of (exit of the last CTA to
                        * finish - entry of CTA 0), from the global timer     */
  double alg_bytes;    /* compulsory bytes summed over the launches: every
                        * output, input, added and dotted element once and
                        * the links of the output and input sites            */
} dwf_kernel_time;

typedef struct dwf_ctx dwf_ctx;

/* Create a context on CUDA device `device` for action `a`.
 * Errors: INVALID_ARG for odd or non-positive extents, Ls out of range;
 * CUDA when the device cannot be used. On error *ctx is NULL. */
dwf_status dwf_create(dwf_ctx **ctx, int device, const dwf_action *a);

/* Free everything the context owns. NULL is accepted. The caller must make
 * sure no work that uses the context is still running. */
void dwf_destroy(dwf_ctx *ctx);

/* Message of the last error on this context ("" if none). The string is owned
 * by the context and valid until the next call on it. NULL ctx: last
 * dwf_create failure. */
const char *dwf_last_error(const dwf_ctx *ctx);

/* Fill *p with the defaults: tol 1e-10, maxiter 100000, inner_iters 6,
 * block = {0,0,0,0} (must be set for MSPCG), outer FP32, inner FP16,
 * delta 0.001, snake 1, use_graph 1, io_on_host 0, check_every 10, flexible 0,
 * schur 0, inner_tol 0. */
void dwf_solver_params_default(dwf_solver_params *p);

/* Load the gauge field U (layout above; host pointer if on_device == 0): the
 * SU(3) links U_mu(x) of the Wilson hop D^w in M^4 = D^w M_phi (paper Sec.
 * 2.2, the definition of D^w). The caller keeps ownership of U; the context
 * copies it. Packs FP64, FP32 and FP16 copies of the links with the antiperiodic time
 * sign folded into the links that cross t = Lt-1 -> 0, and invalidates every
 * cached block plan. Synchronous. Errors: INVALID_ARG (NULL U), CUDA. */
dwf_status dwf_gauge_load(dwf_ctx *ctx, const double *U, int on_device);

/* Bytes of a native half field of precision `prec` with nrhs right-hand sides. */
size_t dwf_field_bytes(const dwf_ctx *ctx, dwf_prec prec, int nrhs);

/* Canonical -> native (import) and native -> canonical (export) conversion of
 * parity half fields (layouts above). Conversion to FP16/BF16 computes the
 * per-(site, s) scale. Errors: INVALID_ARG. */
dwf_status dwf_field_import(dwf_ctx *ctx, void *native_out, dwf_prec prec,
                            const void *canon_in, int canon_is_fp32, int nrhs,
                            void *stream);
dwf_status dwf_field_export(dwf_ctx *ctx, void *canon_out, int canon_is_fp32,
                            const void *native_in, dwf_prec prec, int nrhs,
                            void *stream);

/* Native -> native conversion of nrhs (1 .. DWF_MAX_EIG) half fields from
 * precision in_prec to out_prec (e.g. FP32 low modes to FP16 for
 * mspcg_solve_deflated); FP16/BF16 outputs compute the per-(site, s) scale.
 * The fields must not overlap. Errors: INVALID_ARG, CUDA. */
dwf_status dwf_field_convert(dwf_ctx *ctx, void *native_out, dwf_prec out_prec,
                             const void *native_in, dwf_prec in_prec, int nrhs, void *stream);

/* Hopping block M^4 (paper Sec. 2.2, M^4_{eo/oe} = D^w M_phi):
 *   dagger = 0:  out = -1/2 Dhop (M_phi in)            (M^4_eo or M^4_oe)
 *   dagger = 1:  out = -1/2 M_phi^+ Dhop^+ in          ((M^4)^+)
 * `in` lives on parity 1 - out_parity, `out` on out_parity (0 even, 1 odd).
 * prec: any (native fields; FP16/BF16 use FP16 links and FP32 arithmetic and
 * store the result with a new per-(site, s) scale). out must not alias in. */
dwf_status dwf_dslash_eo(dwf_ctx *ctx, void *out, const void *in, int out_parity,
                         int dagger, dwf_prec prec, int nrhs, const double *mf,
                         void *stream);

/* out = M_5 in, or M_5^+ in (dagger = 1): the 4D-diagonal block of the
 * even-odd system (paper Sec. 2.2). FP64 or FP32 native fields. */
dwf_status dwf_m5(dwf_ctx *ctx, void *out, const void *in, int dagger,
                  dwf_prec prec, int nrhs, const double *mf, void *stream);

/* out = M_5^-1 in, or M_5^-+ in, as used in D_PC and phi_hat (paper eq.
 * (dirac_equation)); computed per chirality by the closed form
 * [alpha (1 + m_f r^Ls)]^-1 sum_{k<Ls} r^k S^k, r = -beta/alpha. */
dwf_status dwf_m5inv(dwf_ctx *ctx, void *out, const void *in, int dagger,
                     dwf_prec prec, int nrhs, const double *mf, void *stream);

/* out = M_5^-1 in (dagger = 0) or M_5^-+ in (dagger = 1), the same operator as
 * dwf_m5inv (paper Sec. 2.2, eq. (dirac_equation)), computed as a dense real
 * GEMM on the tensor cores: per chirality, the Ls x Ls matrix M_5^-1 (built
 * and inverted on the host in FP64 for each right-hand side's m_f) times the
 * Ls-vectors of every (site, spin, colour, re/im), all right-hand sides in
 * one launch. prec: DWF_FP32 (operands split into two FP16 parts, result to
 * about 1e-6 relative), DWF_FP16 or DWF_BF16 (result at the storage's own
 * precision). Any Ls a context takes (<= DWF_MAX_LS = 32: one or two K steps
 * of 16). Fields in the native layout (dwf_field_import);
 * `out` and `in` may not overlap. The call returns after its work on
 * `stream` has finished (it reads the kernel's status word). Uses a small
 * context-owned device buffer, so calls on one context must not overlap.
 * Errors: INVALID_ARG, UNSUPPORTED (FP64 fields), TIMEOUT (a
 * bounded device wait expired), CUDA. */
dwf_status dwf_m5inv_gemm(dwf_ctx *ctx, void *out, const void *in, int dagger,
                          dwf_prec prec, int nrhs, const double *mf, void *stream);

/* out = D_PC in (dagger = 0) or D_PC^+ in (dagger = 1), even parity fields
 * (paper eq. (dirac_equation)). */
dwf_status dwf_mpc(dwf_ctx *ctx, void *out, const void *in, int dagger,
                   dwf_prec prec, int nrhs, const double *mf, void *stream);

/* out = D_PC^+ D_PC in (paper eq. (normal_equation), eq. (DdagD)). */
dwf_status dwf_mdagm(dwf_ctx *ctx, void *out, const void *in, dwf_prec prec,
                     int nrhs, const double *mf, void *stream);

/* Right-hand side of the normal equation for the full system D psi = phi
 * (paper eq. (dirac_equation) and eq. (normal_equation)):
 *   phi_hat_e = phi_e - M^4_eo M_5^-1 phi_o,   b_even = D_PC^+ phi_hat_e.
 * phi_even / phi_odd: the even and odd halves of phi; all three fields native
 * (dwf_field_import) in prec, DWF_FP64 or DWF_FP32; b_even may not alias
 * an input. Uses the context's operator temporaries. Errors: INVALID_ARG,
 * NO_GAUGE, CUDA. */
dwf_status dwf_source_prep(dwf_ctx *ctx, void *b_even, const void *phi_even,
                           const void *phi_odd, dwf_prec prec, int nrhs,
                           const double *mf, void *stream);

/* The symmetric Schur form, a variant of the paper's D_PC (eq.
 * (dirac_equation)) with the diagonal block divided out:
 *   dagger = 0: out = D_sym in = in - M_5^-1 M^4_eo M_5^-1 M^4_oe in (= M_5^-1 D_PC in)
 *   dagger = 1: out = D_sym^+ in = in - (M^4_oe)^+ M_5^-+ (M^4_eo)^+ M_5^-+ in
 * on even native fields (DWF_FP64 or DWF_FP32). D_sym psi_e = M_5^-1 phi_hat_e
 * has the same solution as D_PC psi_e = phi_hat_e. Uses the context's operator
 * temporaries. Errors: INVALID_ARG, NO_GAUGE, CUDA. */
dwf_status dwf_mpc_sym(dwf_ctx *ctx, void *out, const void *in, int dagger, dwf_prec prec,
                       int nrhs, const double *mf, void *stream);

/* out = D_sym^+ D_sym in, the normal operator mspcg_solve iterates on with
 * params->schur = 1 (same arguments and errors as dwf_mdagm). */
dwf_status dwf_mdagm_sym(dwf_ctx *ctx, void *out, const void *in, dwf_prec prec, int nrhs,
                         const double *mf, void *stream);

/* Right-hand side of the symmetric form's normal equation for D psi = phi:
 *   b_even = D_sym^+ M_5^-1 phi_hat_e,  phi_hat_e = phi_e - M^4_eo M_5^-1 phi_o
 * (same arguments and errors as dwf_source_prep; solve with params->schur = 1,
 * then dwf_odd_reconstruct gives the odd half). */
dwf_status dwf_source_prep_sym(dwf_ctx *ctx, void *b_even, const void *phi_even,
                               const void *phi_odd, dwf_prec prec, int nrhs,
                               const double *mf, void *stream);

/* The odd half of the solution of D psi = phi once the even half is known
 * (the second row of the even-odd system, paper eq. (dirac_equation)):
 *   psi_odd = M_5^-1 (phi_odd - M^4_oe psi_even).
 * Native fields in prec (DWF_FP64 or DWF_FP32); psi_odd may not alias an
 * input. Errors: INVALID_ARG, NO_GAUGE, CUDA. */
dwf_status dwf_odd_reconstruct(dwf_ctx *ctx, void *psi_odd, const void *psi_even,
                               const void *phi_odd, dwf_prec prec, int nrhs,
                               const double *mf, void *stream);

/* Size of the library's fixed device scratch array used by dwf_mdagm_noalloc. */
#define DWF_NOALLOC_SCRATCH_BYTES (24u << 20)

/* out = D_PC^+ D_PC in, exactly as dwf_mdagm, but without allocating device
 * memory. The paper has no counterpart: this is an interface for callers that
 * cannot call cudaMalloc -- applications whose own pool allocator already owns
 * the device memory, and host loops that must not take cudaMalloc's implicit
 * device synchronisation. The three half-field temporaries live in one
 * file-scope device array of DWF_NOALLOC_SCRATCH_BYTES bytes that every GPU
 * loading the library holds until exit; the call needs
 * 3 * dwf_field_bytes(ctx, prec, 1) * nrhs bytes of it and returns INVALID_ARG
 * (with a message) when that exceeds the array. The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and should come
 * before any stream capture. All calls share the array and leave their
 * temporaries in it (nothing in it needs to start at zero); calls whose GPU
 * work overlaps race on it, so the caller must serialise them.
 * prec: DWF_FP64 or DWF_FP32. Errors: INVALID_ARG, NO_GAUGE, CUDA. */
dwf_status dwf_mdagm_noalloc(dwf_ctx *ctx, void *out, const void *in, dwf_prec prec,
                             int nrhs, const double *mf, void *stream);

/* Block operator of the multisplitting (paper Sec. 2.3): out = (+)_s A_s in,
 * A_s = P_s D_PC^+ D_PC P_s (snake = 1) or the per-hop Dirichlet operator
 * (snake = 0), on the blocks of params->block, computed in params->inner
 * storage precision. in/out: FP32 native even fields. */
dwf_status dwf_block_apply(dwf_ctx *ctx, void *out, const void *in,
                           const dwf_solver_params *params, int nrhs,
                           const double *mf, void *stream);

/* The multisplitting preconditioner (paper Sec. 2.4): z = M^-1 r with
 * M = (+)_s A_s, each A_s z_s = r_s solved by params->inner_iters CG iterations
 * from a zero guess with block-local scalars. in/out: FP32 native even fields. */
dwf_status dwf_block_precond(dwf_ctx *ctx, void *z, const void *r,
                             const dwf_solver_params *params, int nrhs,
                             const double *mf, void *stream);

/* Block-shape autotuner for the multisplitting preconditioner (the blocks of
 * paper Sec. 2.4). Candidates: b^3 x bt blocks, b in {4, 6, 8, 12, 16}, bt in
 * {4, 6, 8, 12, 16, 24, 32} with b/2 <= bt <= 2b, dividing the lattice, at
 * least two blocks. Each candidate runs one untimed outer iteration and then
 * `trial` (>= 2) timed outer iterations of mspcg_solve on the sources b (as in
 * mspcg_solve: canonical even fields, host pointers when params->io_on_host)
 * with params' other settings; the time to params->tol is predicted from the
 * time per iteration and the rate at which the largest true residual fell.
 * The fastest shape is written to block_out[4], its predicted time to
 * *predicted_seconds (if not null), and remembered in the context, so that
 * mspcg_solve with params->block all zero and the same parameters, masses
 * and nrhs uses it without tuning again (with no remembered shape it tunes
 * first, trial = 20). The other candidates' block plans are released.
 * Synchronous. Errors: INVALID_ARG (inner_iters == 0, trial < 2), NO_GAUGE,
 * UNSUPPORTED (no candidate tiles the lattice), NOT_CONVERGED (no candidate
 * reduced the residual), CUDA. */
dwf_status dwf_autotune_block(dwf_ctx *ctx, const void *b, int nrhs, const double *mf,
                              const dwf_solver_params *params, int trial, int block_out[4],
                              double *predicted_seconds, void *stream);

/* Solve D_PC^+ D_PC x = b for nrhs right-hand sides with Algorithm 1 (MSPCG;
 * plain CG when params->inner_iters == 0). x and b are canonical complex128
 * even half fields (device pointers, or host pointers when params->io_on_host).
 * Outer iterations run in params->outer precision with FP64 reductions; with
 * FP32 outer precision the residual is recomputed in FP64 (reliable update)
 * whenever |r| fell by params->delta, and at convergence. All right-hand
 * sides iterate in the same launches; each stops on its own when its
 * reliable update confirms |b - A x| <= tol |b| (with use_graph the device
 * decides this after every iteration and skips the finished right-hand sides
 * in every later kernel). `info` (host array of nrhs) is filled on success and
 * on NOT_CONVERGED. Synchronous: returns when x is written.
 * Errors: INVALID_ARG, NO_GAUGE, NOT_CONVERGED, NAN, CUDA. */
dwf_status mspcg_solve(dwf_ctx *ctx, void *x, const void *b, int nrhs,
                       const double *mf, const dwf_solver_params *params,
                       dwf_solve_info *info, void *stream);

/* ---------------------------------------------------------------------------
 * Low modes and deflation (paper Sec. 1: for the many solves with one Dirac
 * matrix of the measurement phase, low-lying eigenvectors computed once --
 * EigCG, or Lanczos with a Chebyshev polynomial -- lower the effective
 * condition number of every solve; here they are combined with MSPCG).
 * ------------------------------------------------------------------------- */

void dwf_eig_params_default(dwf_eig_params *p);

/* Low modes of A = D_PC^+ D_PC (or D_sym^+ D_sym, p->schur) at quark mass mf by
 * Chebyshev-filtered subspace iteration: a Rayleigh-Ritz step on the start
 * vectors; then each pass replaces the subspace by T_d(L(A)) V, T_d the
 * Chebyshev polynomial of degree p->degree and L mapping [theta_max,
 * lambda_max] onto [-1, 1] (theta_max the largest current Ritz value), and
 * takes the Ritz pairs of the filtered subspace (Gram matrices in FP64; the
 * small generalised eigenproblem by Cholesky and Jacobi rotations on the
 * device).
 * V: m native FP32 fields (device, dwf_field_bytes(ctx, DWF_FP32, 1) bytes
 *    apart), 1 <= m <= DWF_MAX_EIG, linearly independent start vectors on
 *    entry (e.g. random); the orthonormal Ritz vectors in ascending order of
 *    their Ritz values on return.
 * theta, resid: host arrays of m: Ritz values and |A v - theta v|.
 * info: host, may be NULL. Synchronous. The context allocates 2 m + 48
 * FP32 half fields of work space on first use.
 * Errors: INVALID_ARG, NO_GAUGE, NAN (the filtered subspace lost rank: fewer
 * passes, a lower degree or other start vectors), CUDA. */
dwf_status dwf_eig_lowmodes(dwf_ctx *ctx, void *V, int m, double mf, const dwf_eig_params *p,
                            double *theta, double *resid, dwf_eig_info *info, void *stream);

/* z = (accumulate ? z : 0) + V Lambda^-1 V^+ r for nrhs right-hand sides: the
 * coarse correction of the deflated preconditioner (for exact eigenpairs
 * V Lambda^-1 V^+ = A^-1 on span(V), 0 on its complement).
 * V: n_ev native fields of precision vprec (DWF_FP32, or DWF_FP16 with its
 * per-(site, s) scales, which halves the bytes read; dwf_field_bytes(ctx,
 * vprec, 1) bytes apart), 1 <= n_ev <= DWF_MAX_EIG, orthonormal; lambda: host
 * array of n_ev positive values; z, r: native fields of precision prec
 * (DWF_FP32 or DWF_FP64) that do not alias. FP16 V serves at most 4
 * right-hand sides per call. Synchronous (lambda is copied to the device on
 * `stream` and the call waits for the stream before it returns).
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
dwf_status dwf_deflate(dwf_ctx *ctx, void *z, const void *r, const void *V, dwf_prec vprec,
                       const double *lambda, int n_ev, dwf_prec prec, int nrhs, int accumulate,
                       void *stream);

/* mspcg_solve deflated with n_ev Ritz pairs (V, vprec, lambda as for dwf_deflate) of
 * the solve's normal operator: the outer iteration starts from
 * x_0 = V Lambda^-1 V^+ b (its residual recomputed in FP64), and with
 * coarse = 1 the preconditioner becomes z = M^-1 r + V Lambda^-1 V^+ r (M the
 * multisplitting preconditioner, or 1 for plain CG); with positive lambda the
 * correction is Hermitian positive semi-definite, so Algorithm 1 is unchanged.
 * V should hold eigenvectors of A at the right-hand sides' masses; others only
 * weaken the deflation. Flexible PCG (params->flexible) is not supported with
 * coarse = 1. Otherwise as mspcg_solve.
 * Errors: as mspcg_solve, and UNSUPPORTED. */
dwf_status mspcg_solve_deflated(dwf_ctx *ctx, void *x, const void *b, int nrhs, const double *mf,
                                const dwf_solver_params *params, const void *V, dwf_prec vprec,
                                const double *lambda, int n_ev, int coarse,
                                dwf_solve_info *info, void *stream);

/* Kernel timer for the Dslash (hop) kernels, the operator applications of
 * paper Sec. 2.2 that every solver step is made of (no counterpart in the
 * paper: measurement only). on = 1 turns it on and resets every counter;
 * on = 0 turns it off (counters kept). While on, every hop launch on this
 * context records its span with the GPU's global timer (read by CTA 0 at
 * entry and by the last CTA to finish at exit; one atomic per CTA) into one
 * of 32 slots keyed by (precision, adjoint, M_phi on load, Ls epilogue); the
 * outer-iteration CUDA graphs are re-captured with the timer in them. Hop launches of one context
 * must not overlap in time while it is on (use one stream at a time).
 * Synchronises the device. Errors: INVALID_ARG, CUDA. */
dwf_status dwf_profile_enable(dwf_ctx *ctx, int on);

/* Copy the non-empty timer slots into out[0 .. min(*n, cap) - 1] (host array
 * of cap entries; may be NULL when cap = 0) and set *n to the number of
 * non-empty slots. Synchronises the device. Nothing is recorded unless
 * dwf_profile_enable(ctx, 1) was called. Errors: INVALID_ARG, CUDA. */
dwf_status dwf_profile_read(dwf_ctx *ctx, dwf_kernel_time *out, int cap, int *n);

#ifdef __cplusplus
}
#endif
#endif /* DWF_H */
