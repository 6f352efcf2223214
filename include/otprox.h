/*
 * otprox.h -- C ABI of the GB300 (sm_103a) unbalanced Beckmann-OT proximal
 * library.
 *
 * The library computes the proximal operator of the unbalanced Beckmann
 * optimal-transport regulariser of Lee, Bertrand & Rozell, "Parallel
 * Unbalanced Optimal Transport Regularization for Large-scale Imaging
 * Problems" (arXiv:1909.00149):
 *
 *   prox^mu_{rho V}(p0, p1) = argmin_{x0,x1 >= 0, M, r}
 *        ||M||_{2,1} + mu ||r||_p^p + (1/2 rho) ||[x0;x1] - [p0;p1]||^2
 *        s.t.  D(M) - x0 + x1 = r                           (eq. Prox_UOT)
 *
 * by Algorithm 1 (Sec. III-B), and the RPCA+UOT-DF solver (Algorithm 3,
 * Sec. IV-B) that uses it, for B independent problems at once.
 *
 * Conventions shared by every entry point:
 *  - Images are dense row-major float32 arrays [B][H][W] (row = the paper's
 *    index i, "x"; column = index j, "y").  B independent problems share
 *    H, W and the parameters.
 *  - Array pointers may be HOST or DEVICE memory: the library copies with
 *    cudaMemcpyDefault (unified addressing), so pinned host memory is copied
 *    asynchronously and pageable host memory synchronously.  The caller
 *    keeps ownership of every array it passes; the library never keeps a
 *    caller pointer past the call.  State lives in library-owned device
 *    memory with rows padded to a multiple of 4 floats.
 *  - Work is ordered on the CUDA stream given at create time (NULL = the
 *    legacy default stream).  Calls marked "sync" wait for that stream.
 *  - Every function returns OT_OK (0) or a negative OT_E* code, and sets a
 *    thread-local message readable with ot_last_error().  Invalid arguments
 *    never reach a kernel.
 *  - A handle is not thread-safe: one thread at a time per handle.
 */
#ifndef OTPROX_H
#define OTPROX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define OT_OK          0
#define OT_EINVAL     -1  /* bad argument: shape, pointer, parameter, step rule */
#define OT_ENOMEM     -2  /* device or pinned-host allocation failed            */
#define OT_ECUDA      -3  /* a CUDA runtime call failed (message has the name)  */
#define OT_ENOTCONV   -4  /* max_iter reached before the tolerance; outputs valid */
#define OT_ENONFINITE -5  /* a NaN/Inf appeared in the iterates                 */
#define OT_ETIMEOUT   -6  /* a bounded device wait gave up (the kernel returned
                             early, the context stays usable); the handle's
                             state is then undefined: destroy and recreate it */

/* ------------------------------------------------------------ enumerations */
/* Which arguments of V_mu are variables (Sec. III-B):
 *  PROX        -- x0 and x1 free: eq. (Prox_UOT);
 *  FIXED_FIRST -- x0 frozen at p0 = s, x1 free with prox centre p1: the
 *                 special case eq. (Prox_UOT_specialcase), K = D(M) - s + x - r;
 *  EVAL        -- x0 = p0, x1 = p1 frozen: solves V_mu(p0, p1) itself
 *                 (eq. Unbal_OT_beckman); the objective is the OT cost. */
#define OT_MODE_PROX        0
#define OT_MODE_FIXED_FIRST 1
#define OT_MODE_EVAL        2
/* Flux norm: ISO = ||M||_{2,1} (Sec. III-A); ANISO = sum |Mx| + |My|. */
#define OT_NORM_ISO   0
#define OT_NORM_ANISO 1
/* Kernel choice for Algorithm 1: AUTO picks RESIDENT when one problem's
 * state fits in one CTA's shared memory, TMA otherwise.
 *  TILED    -- one CTA per 16 x 128 tile, loads through the L1 path;
 *  RESIDENT -- one CTA per problem, all iterations of a call in shared memory;
 *  TMA      -- persistent CTAs (one per SM) fed by a multi-stage TMA pipeline;
 *  TEMPORAL -- temporal blocking: tb_depth iterations per pass over the state
 *              (a CTA stages its tile with a halo of tb_depth rounded up to 2
 *              or 4 rows and 4 columns, iterates on it, writes the tile once);
 *              bit-identical to TILED.  Standalone Algorithm 1 only (not the
 *              projection form, the batch, or the inner prox of ot_rpca_* and
 *              ot_uotdf_*); it allocates three more state planes. */
#define OT_KERNEL_AUTO     0
#define OT_KERNEL_TILED    1
#define OT_KERNEL_RESIDENT 2
#define OT_KERNEL_TMA      3
#define OT_KERNEL_TEMPORAL 4
/* Solver of eq. (Prox_UOT):
 *  ALG1       -- Algorithm 1, the paper's primal-dual iteration (Sec. III-B);
 *  PROJECTION -- ADMM with an exact projection onto {K z = k0} through the
 *                DCT-II Neumann solve (K K^T = D D* + n_id I).  Not the
 *                paper's algorithm; the same minimiser.  Its state: M, x, r
 *                are the ADMM iterate z, and a is beta times the last
 *                projection multiplier (the dual of K z = k0 at a fixed point). */
#define OT_ALG_ALG1        0
#define OT_ALG_PROJECTION  1

/* Arithmetic of the dense DCT contractions (the Neumann solve below):
 *  FP32         -- FP32 CUDA-core GEMMs;
 *  SPLIT_BF16   -- tcgen05 tensor-core GEMMs on a 2-piece BF16 split, three
 *                  products (a_hi b_hi + a_hi b_lo + a_lo b_hi), FP32
 *                  accumulation: about 2^-17 relative per product (a solve
 *                  about 1e-5 of its result);
 *  SPLIT_BF16_3 -- the exact 3-piece split (h + m + l = x for every FP32 x)
 *                  and the six products down to 2^-16 (hh, hm, mh, mm, hl,
 *                  lh): FP32-level results at twice the tensor work. */
#define OT_PREC_FP32         0
#define OT_PREC_SPLIT_BF16   1
#define OT_PREC_SPLIT_BF16_3 2

typedef struct ot_prox* ot_prox_t;

typedef struct {
  int32_t B, H, W;        /* problems, rows, columns (all >= 1)                  */
  int32_t mode;           /* OT_MODE_*                                           */
  int32_t norm;           /* OT_NORM_*                                           */
  int32_t balanced;       /* 1: r = 0, the balanced problem (eq. OT_beckman)    */
  int32_t p_exp;          /* 1: mu ||r||_1 (the paper's choice); 2: mu ||r||_2^2 */
  double  mu;             /* growth/decay penalty mu > 0                         */
  double  rho;            /* prox weight: (1/2rho)||x - p||^2, rho > 0           */
  double  tau1, tau2;     /* primal/dual steps; <= 0 selects
                             0.99 / sqrt(lambda_max(D D*) + n_id), which obeys
                             Theorem 1; given steps must satisfy
                             tau1 tau2 (lambda_max + n_id) < 1                   */
  double  tol;            /* stopping tolerance on res_pri and res_fp            */
  int32_t max_iter;       /* iteration cap of ot_prox_solve                      */
  int32_t check_every;    /* iterations between stopping tests (>= 1)            */
  int32_t kernel;         /* OT_KERNEL_*                                         */
  int32_t use_graph;      /* 1: replay each check interval as a CUDA graph       */
  int32_t algorithm;      /* OT_ALG_*                                            */
  int32_t precision;      /* OT_PREC_* of the DCT solves (projection form)       */
  double  beta;           /* ADMM penalty of the projection form (> 0)           */
  int32_t tb_depth;       /* OT_KERNEL_TEMPORAL: iterations per pass, 2..4 (the
                             default 4); a call's n iterations run as
                             ceil(n / tb_depth) passes of near-equal length      */
} ot_prox_params;

typedef struct {
  int32_t iters;          /* iterations run by this call                         */
  int32_t status;         /* OT_OK / OT_ENOTCONV / OT_ENONFINITE                 */
  double  res_pri;        /* ||K(z)|| / ||p||  at the last check                  */
  double  res_fp;         /* ||(z,a)^{k+1}-(z,a)^k|| / ||(z,a)^{k+1}||            */
  double  objective;      /* ||M||_{2,1} + mu ||r||_p^p + (1/2rho)||x - p||^2     */
  double  primal_feasible;/* objective with r' = D(M) + A x (constraint exact)   */
  double  dual_obj;       /* dual objective at the scaled/clipped dual a         */
  double  rel_gap;        /* (primal_feasible - dual_obj) / |primal_feasible|    */
} ot_prox_result;

/* Fill *p with the defaults: mode PROX, iso, unbalanced, p = 1, mu = 3,
 * rho = 0.01, default steps, tol = 1e-5, max_iter = 100000,
 * check_every = 10, kernel AUTO, use_graph = 1, algorithm ALG1,
 * precision FP32, beta = 1.  B, H, W are set to 1. */
void ot_prox_default_params(ot_prox_params* p);

/* lambda_max(D D*) = 4 sin^2(pi (H-1) / 2H) + 4 sin^2(pi (W-1) / 2W): the
 * largest eigenvalue of the Neumann grid Laplacian of Theorem 1. */
double ot_lambda_max(int32_t H, int32_t W);

/* Number of identity blocks n_id of K acting on free variables (x0, x1, r):
 * ||K||^2 = lambda_max + n_id; the full problem of Theorem 1 has n_id = 3. */
int32_t ot_n_identity_blocks(int32_t mode, int32_t balanced);

/* Create a solver for B problems of H x W (Sec. III-B).  Validates every
 * field, applies the default steps, rejects steps that break Theorem 1
 * (tau1 tau2 (lambda_max + n_id) >= 1) with OT_EINVAL, allocates the state
 * (zero) on the current device.  `cuda_stream` is a cudaStream_t or NULL. */
int ot_prox_create(const ot_prox_params* params, void* cuda_stream, ot_prox_t* out);

/* The prox centres [B][H][W]: p0, p1 (PROX), s = p0 and p (FIXED_FIRST),
 * the two arguments of V_mu (EVAL).  Both pointers required.  Async on the
 * handle's stream (synchronous for pageable host memory). */
int ot_prox_set_input(ot_prox_t h, const float* p0, const float* p1);

/* Run n_iter >= 0 iterations of Algorithm 1 from the current (warm) state,
 * with no stopping test: the inexact warm-started use of Sec. III-B that
 * Algorithm 3 line 11 makes.  Async. */
int ot_prox_step(ot_prox_t h, int32_t n_iter);

/* One check interval of ot_prox_solve: n_iter >= 1 iterations, the last one
 * also computing the stopping quantities (res_pri, res_fp, objective; the
 * certificate fields are left 0).  Returns OT_OK or OT_ENONFINITE.  Sync. */
int ot_prox_check_interval(ot_prox_t h, int32_t n_iter, ot_prox_result* res);

/* ot_prox_step bracketed by two CUDA events recorded on the handle's stream;
 * *elapsed_ms receives the device time between them.  Used to time the
 * iteration kernel alone.  Sync. */
int ot_prox_step_timed(ot_prox_t h, int32_t n_iter, double* elapsed_ms);

/* Iterate from the current state until max(res_pri, res_fp) <= tol (tested
 * every check_every iterations) or max_iter iterations; fills *res (may be
 * NULL).  Returns OT_OK, OT_ENOTCONV (outputs still valid) or
 * OT_ENONFINITE.  Sync. */
int ot_prox_solve(ot_prox_t h, ot_prox_result* res);

/* Residuals, objective and duality-gap certificate of the current state,
 * without iterating (res_fp is 0, iters is 0).  Sync. */
int ot_prox_evaluate(ot_prox_t h, ot_prox_result* res);

/* Copy the state out, dense [B][H][W]; any pointer may be NULL to skip it.
 * For a frozen x the copy is its input.  Async (pageable host: sync). */
int ot_prox_get_state(ot_prox_t h, float* Mx, float* My, float* x0, float* x1,
                      float* r, float* a);

/* Copy a warm state in (Algorithm 2 caches the prox state between outer
 * iterations); NULL pointers leave that variable unchanged.  Flux on the
 * outer slots Mx[H-1,:], My[:,W-1] (no edge there) is set to 0; frozen x
 * ignore their pointer.  Async (pageable host: sync). */
int ot_prox_set_state(ot_prox_t h, const float* Mx, const float* My, const float* x0,
                      const float* x1, const float* r, const float* a);

/* Warm start from a predicted state (e.g. ot_unet_forward's output): pred
 * is a DEVICE array [B][4][H][W] float32 of (Mx, My, r, a) per problem.
 * Mx, My, r (unless balanced) and a are copied in, the flux zeroed on the
 * slots without an edge; each free x is set from its step's fixed point
 * given a: x0 = max(p0 + rho a, 0), x1 = max(p1 - rho a, 0) (the inputs
 * must be set).  gate > 0 takes the prediction only at pixels where p0 + p1
 * exceeds gate somewhere in the 5 x 5 neighbourhood; elsewhere the state is
 * written as for a zero prediction (M = r = a = 0, x = p).  gate = 0 takes
 * it everywhere.  Stream-ordered, no sync. */
int ot_prox_warm_start(ot_prox_t h, const float* pred, double gate);

/* Zero the state (Algorithm 2 line 2 initialises the prox state to 0). */
int ot_prox_reset(ot_prox_t h);

/* Resolved parameters (defaults filled in) of a handle. */
int ot_prox_get_params(ot_prox_t h, ot_prox_params* out);

/* Free everything the handle owns; NULL is accepted. */
int ot_prox_destroy(ot_prox_t h);

/* ------------------------------------------------------------------ RPCA */
/* RPCA+UOT-DF (Algorithm 3, Sec. IV-B.1) with Phi_t = I: minimise
 *   1/2 sum_t ||y_t - s_t - l_t||^2 + lambda ||S||_1 + gamma ||L||_*
 *   + kappa sum_{t<T} V_mu(s_t, s_{t+1}),   S, L >= 0           (eq. RPCA_UOTDF)
 * by ADMM with the splitting of Sec. IV-B.1.  Line 10's singular-value
 * thresholding runs through the T x T Gram matrix; line 11 runs n_inner
 * warm-started Algorithm 1 iterations on the T-1 frame pairs (prox weight
 * kappa/rho).  Readings of garbled lines: A += X - S - L (line 12), the
 * x-update keeps rho (line 9), s_t >= 0 (line 7).  Stopping: the ADMM primal
 * and dual residuals (Boyd), each relative to ||Y||, both <= tol. */
typedef struct ot_rpca* ot_rpca_t;
/* Signed foreground (signed_fg = 1; eq. RPCA_UOTDF_PN, Sec. IV-B, the
 * real-video experiment): S = S+ - S- with S+, S- >= 0 and a transport term
 * kappa V_mu(s+-_t, s+-_{t+1}) for each sign.  The paper gives only this
 * objective; the iteration is Algorithm 3's ADMM with its splitting applied
 * to each sign (X = S+ - S- + L, z+-_t = s+-_t, w+-_{t+1} = s+-_{t+1}, duals
 * b+-, c+-), the S+ block updated before the S- block, each by its exact
 * block minimiser (line 7 with S- in S+'s data target, S+ - X + L - A as
 * S-'s), lines 8-10 on S = S+ - S-, line 11 for both signs as one batch of
 * 2 (T - 1) Algorithm 1 problems, lines 12-15 for both signs.  Residuals
 * add both signs' terms.  The SVT runs as its own Gram, eigensolver and
 * apply kernels (not fused with the elementwise passes). */

typedef struct {
  int32_t T, H, W;        /* frames (2..128), rows, columns                      */
  double  lambda;         /* sparsity weight > 0                                  */
  double  gamma;          /* nuclear-norm weight; <= 0: lambda sqrt(max(N, T))    */
  double  kappa;          /* OT weight > 0                                        */
  double  mu;             /* growth/decay penalty of V_mu > 0                     */
  double  rho;            /* ADMM penalty > 0                                     */
  int32_t n_inner;        /* Algorithm 1 iterations per outer iteration (>= 1)    */
  double  tol;            /* tolerance on both relative residuals                 */
  int32_t max_iter;       /* outer-iteration cap of ot_rpca_solve                 */
  int32_t check_every;    /* outer iterations between residual checks (>= 1)     */
  int32_t svt_max_sweeps; /* Jacobi sweeps cap of the T x T eigensolver           */
  int32_t prox_kernel;    /* OT_KERNEL_* of the inner Algorithm 1                 */
  int32_t use_graph;      /* 1: replay warm outer iterations as a CUDA graph     */
  int32_t signed_fg;      /* 1: signed foreground S = S+ - S- (eq. RPCA_UOTDF_PN),
                             see below; 0: S >= 0 (eq. RPCA_UOTDF)                */
} ot_rpca_params;

typedef struct {
  int32_t iters;          /* outer iterations run by this call                   */
  int32_t status;         /* OT_OK / OT_ENOTCONV / OT_ENONFINITE                  */
  double  res_pri;        /* ||(X-S-L, L-T, z-s_t, w-s_{t+1})|| / ||Y||           */
  double  res_dual;       /* rho ||(dX, dT, dz, dw)|| / ||Y||                     */
  int32_t svt_rounds;     /* Jacobi rounds of the last SVT (T_pad - 1 per sweep)  */
  int32_t svt_rank;       /* singular values above gamma/rho in the last SVT     */
} ot_rpca_result;

/* Variables readable with ot_rpca_get; frame variables are [T][H][W], pair
 * variables [T-1][H][W] (pair t couples frames t and t+1). */
#define OT_RPCA_S     0   /* sparse part (frames)                  */
#define OT_RPCA_L     1   /* low-rank part (frames)                */
#define OT_RPCA_X     2   /* data split variable (frames)          */
#define OT_RPCA_T     3   /* nuclear-norm split variable (frames)  */
#define OT_RPCA_A     4   /* scaled dual of X = S + L (frames)     */
#define OT_RPCA_D     5   /* scaled dual of T = L (frames)         */
#define OT_RPCA_B     6   /* scaled dual of z_t = s_t (pairs)      */
#define OT_RPCA_C     7   /* scaled dual of w_{t+1} = s_{t+1} (pairs) */
#define OT_RPCA_Z     8   /* z_t (pairs): first prox output        */
#define OT_RPCA_W     9   /* w_{t+1} (pairs): second prox output   */
#define OT_RPCA_MX   10   /* inner prox flux Mx (pairs)            */
#define OT_RPCA_MY   11   /* inner prox flux My (pairs)            */
#define OT_RPCA_R    12   /* inner prox source r (pairs)           */
#define OT_RPCA_DUAL 13   /* inner prox dual a (pairs)             */
#define OT_RPCA_SP   14   /* signed_fg: S+ (frames)                */
#define OT_RPCA_SM   15   /* signed_fg: S- (frames)                */
/* signed_fg: OT_RPCA_MINUS | (a pair variable, 6..13) reads the S- sign's
 * copy of it; the plain id reads the S+ sign's.  OT_RPCA_S reads S+ - S-. */
#define OT_RPCA_MINUS 0x100

/* Defaults: lambda 0.02, gamma lambda sqrt(max(N,T)), kappa 0.005, mu 3,
 * rho 1, n_inner 1, tol 1e-5, max_iter 5000, check_every 1,
 * svt_max_sweeps 30, prox_kernel AUTO, use_graph 1; T = 2, H = W = 1. */
void ot_rpca_default_params(ot_rpca_params* p);
/* Validate, allocate and zero the state (Algorithm 3 line 2). */
int ot_rpca_create(const ot_rpca_params* params, void* cuda_stream, ot_rpca_t* out);
/* Observations Y [T][H][W] (host or device).  Sync (computes ||Y||). */
int ot_rpca_set_input(ot_rpca_t h, const float* Y);
/* n_outer >= 0 outer iterations, no residual read.  Async. */
int ot_rpca_step(ot_rpca_t h, int32_t n_outer);
/* n_outer >= 1 outer iterations; the residuals of the last one.  Sync.
 * OT_ETIMEOUT if a bounded device wait expired in the prox kernel, a
 * tensor-core kernel or the grid barrier of the pass between iterations. */
int ot_rpca_iterate_checked(ot_rpca_t h, int32_t n_outer, ot_rpca_result* res);
/* Iterate until both residuals <= tol or max_iter.  Returns OT_OK,
 * OT_ENOTCONV (state still valid), OT_ENONFINITE or OT_ETIMEOUT.  Sync. */
int ot_rpca_solve(ot_rpca_t h, ot_rpca_result* res);
/* Two outer iterations (as ot_rpca_step(h, 2)) with CUDA events recorded on
 * the handle's stream between their phases, the eigensolver serialised with
 * the prox; phase_ms[0..7] receives the device time of: 0 lines 4-9 of the
 * first, 1 its Gram matrix, 2 its T x T eigensolver, 3 the second's SVT
 * apply (alone, as for the last outer iteration of every call), 4 the
 * first's n_inner Algorithm 1 iterations, 5 lines 12-15 of the second
 * (alone), 6 the pass between them: lines 12-15 of the first fused with
 * lines 4-9 of the second (for T <= 64 also the first's SVT apply and the
 * second's Gram matrix, its partials reduced in the same launch), 7 the
 * second's Gram where that pass does not produce it (T > 64; about 0
 * otherwise).  With signed_fg: one outer iteration, whose phases are 0 the
 * lines 4-9 pass, 1 the Gram, 2 the eigensolver, 3 the SVT apply, 4 the
 * Algorithm 1 iterations on both signs' pairs, 5 the lines 12-15 pass; 6 and
 * 7 are 0 (no fused pass).  Sync. */
int ot_rpca_step_profiled(ot_rpca_t h, double* phase_ms);

/* Copy one variable (OT_RPCA_*) out, dense.  Sync. */
int ot_rpca_get(ot_rpca_t h, int32_t var, float* out);
/* Zero the state (keeps Y). */
int ot_rpca_reset(ot_rpca_t h);
int ot_rpca_get_params(ot_rpca_t h, ot_rpca_params* out);
int ot_rpca_destroy(ot_rpca_t h);

/* ------------------------------------------------------------------------
 * Batched Algorithm 1 over sequences of uneven size.  Sequence i holds B_i
 * independent H_i x W_i problems of eq. Prox_UOT (e.g. the T_i - 1 frame
 * pairs of a T_i-frame video, Alg. 3 line 11).  One launch per iteration
 * runs every active sequence's tiles (a work list in device memory); each
 * sequence has its own Theorem 1 step sizes, its own residuals (segmented
 * FP64 sums) and leaves the work list when it meets tol.  Iterates are
 * bit-identical to ot_prox_* with kernel OT_KERNEL_TILED on the same inputs
 * (and so to its TMA kernel); OT_ETIMEOUT if a bounded wait expired.
 * `common` supplies mode, norm, balanced, p_exp, mu, rho, tol, max_iter,
 * check_every (even, >= 2) and use_graph; tau1, tau2 must be 0 (chosen per
 * sequence); B, H, W, kernel, algorithm and precision are ignored. */
typedef struct ot_prox_batch* ot_prox_batch_t;

typedef struct {
  int32_t iters;          /* iterations run on this sequence                     */
  int32_t status;         /* OT_OK, OT_ENOTCONV or OT_ENONFINITE                  */
  double  res_pri;        /* ||K(z)|| / ||p|| at the last check                   */
  double  res_fp;         /* relative change of (z, a) at the last check          */
} ot_prox_batch_result;

/* n_seq in [1, 256]; B, H, W: host arrays of n_seq sizes.  State zero. */
int ot_prox_batch_create(int32_t n_seq, const int32_t* B, const int32_t* H, const int32_t* W,
                         const ot_prox_params* common, void* cuda_stream, ot_prox_batch_t* out);
/* Prox centres of sequence seq, [B_i][H_i][W_i] float32, host or device. */
int ot_prox_batch_set_input(ot_prox_batch_t h, int32_t seq, const float* p0, const float* p1);
/* n_iter iterations of every sequence, no stopping test (stream-ordered). */
int ot_prox_batch_step(ot_prox_batch_t h, int32_t n_iter);
/* Iterate every sequence to the stopping rule; res: host array of n_seq.
 * launches (optional): kernel launches made.  Synchronises.  Returns
 * OT_ENOTCONV if some sequence hit max_iter (results still valid). */
int ot_prox_batch_solve(ot_prox_batch_t h, ot_prox_batch_result* res, int32_t* launches);
/* State of sequence seq, [B_i][H_i][W_i] each (NULL to skip); synchronises. */
int ot_prox_batch_get_state(ot_prox_batch_t h, int32_t seq, float* Mx, float* My, float* x0, float* x1, float* r,
                            float* a);
/* Iteration kernel: OT_KERNEL_TMA (the TMA pipeline, one CTA per SM,
 * 16-row tiles; the default) or OT_KERNEL_TILED with tile_rows 8 or 16 and
 * ctas_per_sm persistent CTAs per SM (1..8).  Iterates do not depend on it. */
int ot_prox_batch_set_config(ot_prox_batch_t h, int32_t kernel, int32_t tile_rows, int32_t ctas_per_sm);
/* Time every candidate configuration on the loaded problems (4 plain
 * iterations each, CUDA events) and keep the fastest; outputs optional.  The
 * iterates advance: call ot_prox_batch_reset for a cold start. */
int ot_prox_batch_autotune(ot_prox_batch_t h, int32_t* kernel, int32_t* tile_rows, int32_t* ctas_per_sm,
                           float* ms_per_iter);
/* Zero every sequence's state (keeps the inputs). */
int ot_prox_batch_reset(ot_prox_batch_t h);
int ot_prox_batch_destroy(ot_prox_batch_t h);

/* ------------------------------------------------------------------------
 * UOT-DF / BPDN+UOT-DF (Algorithm 2, Sec. IV-A.1), Phi = I, for B
 * independent frames [B][H][W]:
 *   min_{s >= 0} 1/2 ||y - s||^2 + lambda ||s||_1 + kappa V_mu(s, s0)
 * (eq. UOT-DF for lambda = 0, eq. BPDN+UOT-DF for lambda > 0), s0 the
 * prediction of the current state.  ADMM with the splitting s = x = z of
 * Sec. IV-A.1; line 6 runs n_inner warm-started Algorithm 1 iterations in
 * the fixed-first form (eq. Prox_UOT_specialcase, prox weight kappa/rho).
 * Readings of the printed algorithm: the s-update minimises both augmented
 * terms, s = max((x + a + z + b)/2 - lambda/(2 rho), 0); stopping uses the
 * primal and dual residuals ||(x - s, z - s)|| and rho ||(dx, dz)|| relative
 * to ||y||, both <= tol. */
typedef struct ot_uotdf* ot_uotdf_t;

typedef struct {
  int32_t B, H, W;        /* independent frames, rows, columns                   */
  double  kappa;          /* OT weight > 0                                        */
  double  mu;             /* growth/decay penalty of V_mu > 0                     */
  double  rho;            /* ADMM penalty > 0                                     */
  double  lambda;         /* sparsity weight >= 0 (0: UOT-DF)                     */
  int32_t n_inner;        /* Algorithm 1 iterations per ADMM iteration (>= 1)    */
  int32_t norm;           /* OT_NORM_* of the flux                                */
  int32_t p_exp;          /* 1 or 2: exponent of the source term                  */
  double  tol;            /* tolerance on both relative residuals                 */
  int32_t max_iter;       /* iteration cap of ot_uotdf_solve                      */
  int32_t check_every;    /* iterations between residual checks (>= 1)           */
  int32_t prox_kernel;    /* OT_KERNEL_* of the inner Algorithm 1                 */
} ot_uotdf_params;

typedef struct {
  int32_t iters;          /* ADMM iterations run by this call                     */
  int32_t status;         /* OT_OK / OT_ENOTCONV / OT_ENONFINITE                  */
  double  res_pri;        /* ||(x - s, z - s)|| / ||y||                            */
  double  res_dual;       /* rho ||(dx, dz)|| / ||y||                              */
} ot_uotdf_result;

/* Variables readable with ot_uotdf_get, each [B][H][W]. */
#define OT_UOTDF_S 0
#define OT_UOTDF_X 1
#define OT_UOTDF_Z 2
#define OT_UOTDF_A 3
#define OT_UOTDF_B 4

/* Defaults: kappa 0.5, mu 3, rho 1, lambda 0, n_inner 1, iso, p_exp 1,
 * tol 1e-5, max_iter 20000, check_every 10, prox_kernel AUTO; B = H = W = 1. */
void ot_uotdf_default_params(ot_uotdf_params* p);
/* All state zero (Algorithm 2 line 2).  OT_EINVAL on a bad parameter. */
int ot_uotdf_create(const ot_uotdf_params* params, void* cuda_stream, ot_uotdf_t* out);
/* y: measurements, s0: prediction; [B][H][W] float32, host or device.
 * Synchronises; OT_ENONFINITE if y is not finite. */
int ot_uotdf_set_input(ot_uotdf_t h, const float* y, const float* s0);
/* n ADMM iterations, stream-ordered, no stopping test. */
int ot_uotdf_step(ot_uotdf_t h, int32_t n);
/* n iterations, the last one with the residual sums; synchronises. */
int ot_uotdf_iterate_checked(ot_uotdf_t h, int32_t n, ot_uotdf_result* res);
/* Iterate to the stopping rule (checked every check_every iterations). */
int ot_uotdf_solve(ot_uotdf_t h, ot_uotdf_result* res);
/* Copy variable var (OT_UOTDF_*) to out [B][H][W]; synchronises. */
int ot_uotdf_get(ot_uotdf_t h, int32_t var, float* out);
/* Zero the state (keeps y and s0). */
int ot_uotdf_reset(ot_uotdf_t h);
int ot_uotdf_get_params(ot_uotdf_t h, ot_uotdf_params* out);
int ot_uotdf_destroy(ot_uotdf_t h);

/* ------------------------------------------------------------------------
 * Learned warm start for Algorithm 1.  Sec. III-B caches converged iterates
 * and warm-starts the next solve from them; this network predicts such a
 * state for a new frame pair: a 4-level U-Net (base C channels; 3x3
 * zero-padded convolutions with ReLU, 2x2 average pooling, nearest 2x
 * upsampling, skips concatenated after the upsampled channels, 1x1 head)
 * maps x = (p0, p1) [n][2][H][W] to y = (Mx, My, r, a) [n][4][H][W].
 * Weights are BF16 (FP32 master copy for the optimiser), activations FP32,
 * products accumulated in FP32.  The solver still runs to its stopping rule
 * from the predicted state, so the network only changes the iteration count.
 *
 * Parameters are one flat float32 array: for each convolution in forward
 * order (enc0a, enc0b, enc1a, enc1b, enc2a, enc2b, botta, bottb, dec2a,
 * dec2b, dec1a, dec1b, dec0a, dec0b, head) its weights [co][ci][k][k]
 * followed by its biases [co].  All pointers may be host or device. */
typedef struct ot_unet* ot_unet_t;

/* H, W multiples of 8; max_batch >= 1; base_channels in [1, 256].  All
 * parameters start at zero (set them with ot_unet_set_params). */
int ot_unet_create(int32_t H, int32_t W, int32_t max_batch, int32_t base_channels, void* cuda_stream,
                   ot_unet_t* out);
/* Length of the flat parameter array (OT_EINVAL = -1 for a NULL handle). */
int64_t ot_unet_param_count(ot_unet_t h);
/* Load parameters (resets the optimiser state).  Synchronises. */
int ot_unet_set_params(ot_unet_t h, const float* params);
int ot_unet_get_params(ot_unet_t h, float* params);
/* bias_free = 1: report every bias gradient as 0, so training keeps the
 * biases at their values (zero after ot_unet_set_params with zero biases).
 * A bias-free network maps an all-zero neighbourhood to exactly 0 (every
 * layer is positively homogeneous), which is the converged state there. */
int ot_unet_set_bias_free(ot_unet_t h, int32_t bias_free);
/* y = net(x) for n <= max_batch inputs.  Synchronises. */
int ot_unet_forward(ot_unet_t h, const float* x, float* y, int32_t n);
/* Mean squared error between net(x) and target [n][4][H][W] (loss, optional)
 * and its gradient with respect to the parameters (grads, flat layout,
 * optional).  Synchronises; OT_ENONFINITE on a non-finite loss. */
int ot_unet_gradients(ot_unet_t h, const float* x, const float* target, int32_t n, float* grads, double* loss);
/* ot_unet_gradients followed by one Adam step (beta 0.9, 0.999, eps 1e-8)
 * with learning rate lr on the FP32 master weights. */
int ot_unet_train_step(ot_unet_t h, const float* x, const float* target, int32_t n, float lr, double* loss);
int ot_unet_destroy(ot_unet_t h);

/* Singular-value thresholding shrink*_theta(X) = U max(Sigma - theta, 0) V^T
 * (Sec. IV-B.1, Algorithm 3 line 10) of an N x T matrix stored as T columns of
 * N floats (X + t*N), via the T x T Gram matrix and a Jacobi eigensolver.
 * X, Y: DEVICE pointers, must not alias; 1 <= T <= 128.  Workspace is taken
 * with cudaMallocAsync on the stream and returned before the call ends.
 * Synchronises the stream; OT_ETIMEOUT if a bounded wait in the tensor-core
 * Gram kernel expired. */
int ot_svt(const float* X, float* Y, int64_t N, int32_t T, double theta, void* cuda_stream);

/* ------------------------------------------------------ Neumann solve */
/* Y = (D D* + c I)^{-1} X for B independent H x W images, where D D* is the
 * grid Laplacian with zero-flux (Neumann) boundary of Theorem 1's proof; for
 * c = 0 the pseudo-inverse (the constant mode is dropped).  Solved by the
 * orthonormal DCT-II, which diagonalises D D* (eigenvalues
 * 4 sin^2(pi k / 2H) + 4 sin^2(pi l / 2W)); each transform is one batched
 * GEMM.  X, Y: DEVICE pointers, dense [B][H][W] float32; they may alias.
 * precision: OT_PREC_*.  Allocates its tables per call.  Sync. */
int ot_neumann_solve(const float* X, float* Y, int32_t B, int32_t H, int32_t W, double c, int32_t precision,
                     void* cuda_stream);
/* The same solve on one set of tables, once untimed and then n_rep >= 1
 * times between CUDA events on cuda_stream; *ms_per_solve (host) = the
 * device time of one solve (for split BF16: the operand split and the four
 * tensor-core GEMMs).  X must not alias Y here.  Sync. */
int ot_neumann_solve_timed(const float* X, float* Y, int32_t B, int32_t H, int32_t W, double c, int32_t precision,
                           int32_t n_rep, double* ms_per_solve, void* cuda_stream);

/* ot_prox_evaluate for a state the caller holds, without allocating.
 * The paper has no counterpart: this is a convenience for callers that
 * cannot allocate device memory when they need the answer -- for example
 * code running inside another framework's memory pool that forbids
 * allocations outside it, or a latency-critical loop where cudaMalloc or
 * cudaFree would synchronise the device.  It calls no cudaMalloc, cudaFree
 * or allocating library routine; its scratch is a fixed array of about
 * 114 KB inside the library, present on every GPU that loads it until the
 * process exits.
 *  - params: only B, H, W, mode, norm, balanced, p_exp, mu, rho are read.
 *    B*H*W may be at most 2^31 - 1; larger inputs return OT_EINVAL.
 *  - p0 ... a: DEVICE pointers, dense [B][H][W] float32 (no padding).  x0
 *    may be NULL unless mode is PROX, x1 may be NULL in EVAL mode, r may be
 *    NULL when balanced (frozen x take p0 / p1).
 *  - res: host; filled as by ot_prox_evaluate (res_fp and iters are 0).
 *  - cuda_stream: cudaStream_t or NULL.  Sync: returns after the stream
 *    reaches the end of the evaluation.
 * The first call on a device looks up the scratch array's device address
 * for that device (and looks it up again after a cudaDeviceReset, which
 * ends the context it belongs to); make that first call before any stream
 * capture.  All
 * calls share the one array, so calls that overlap on the GPU (other
 * streams, other threads) race and give wrong results; every call rewrites
 * all the scratch it reads, so nothing needs clearing between calls. */
int ot_prox_evaluate_noalloc(const ot_prox_params* params, const float* p0, const float* p1,
                             const float* Mx, const float* My, const float* x0, const float* x1,
                             const float* r, const float* a, ot_prox_result* res, void* cuda_stream);

/* ----------------------------------------------------------- diagnostics */
/* Runs the grid barrier of the fused Algorithm 3 pass (the one between outer
 * iterations, Alg. 3 lines 12-15 and 4-10) on its own: `ctas` CTAs (1 to
 * the device's SM count) launched cooperatively on a fresh barrier whose
 * arrival count starts at `preset_count` (0 = the state every launch leaves
 * behind).  With 0 every CTA passes and the generation advances by one; with
 * any value from ctas upwards no arrival completes the barrier, every CTA's
 * bounded wait (about a second) gives up and the error flag is set; the
 * context stays usable.  Outputs (host): *err = the device error flag (0 or
 * 1), *generation = the barrier's generation afterwards.  Synchronous on an
 * internal stream.  Returns OT_EINVAL for ctas out of range. */
int ot_debug_grid_barrier(int32_t ctas, uint32_t preset_count, int32_t* err, uint32_t* generation);

/* Message of the last failing call on this thread ("" if none). */
const char* ot_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OTPROX_H */
