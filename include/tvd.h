/*
 * tvd.h -- C ABI of the GB300 TV-deblurring PCG library (libtvd.so).
 *
 * The library implements the inner step of the lagged-diffusivity fixed-point
 * (FP) method for total-variation deblurring of Bai, Donatelli and
 * Serra-Capizzano, "Fast preconditioners for total variation deblurring with
 * anti-reflective boundary conditions": for the FP step at u^k it solves
 *
 *     A x = b,   A = H^T H + alpha L(u^k)                       (eq. (fp))
 *
 * by preconditioned CG (Golub & Van Loan, Alg. 10.3.1, cited in Sec. 1), where
 *   H       is the blur with reflective or anti-reflective boundary conditions
 *           (Sec. 2, eqs. (blurred1d:matrixform), (anti1d) and the 2D corner rules),
 *   L(u)    is the lagged-diffusivity operator -div(psi^-1 grad .),
 *           psi = sqrt(|grad u|^2 + beta^2) (Sec. 1, eq. (el)),
 *   and the preconditioner is one of I, D = I + alpha diag(L) (eq. (D)),
 *   R / M (eqs. (R2), (M), Sec. 3.2) or D_R / D_M = D^1/2 {R|M} D^1/2,
 *   applied with fast trigonometric transforms: the DCT for reflective BCs and
 *   DST-I (hat-S = diag(1, S_{n-2}, 1), eqs. (lambda), (hats)) for
 *   anti-reflective BCs.
 *
 * Conventions shared by every entry point:
 *   - Images are n_rows x n_cols, row-major and contiguous, element (i, j) at
 *     i * n_cols + j. All image pointers are DEVICE pointers owned by the
 *     caller; the library never frees them and never keeps them after a call
 *     returns.
 *   - Element type: the operator calls (ar_blur_apply, tv_operator_apply,
 *     tau_precond_setup, tau_precond_solve) use the plan's operator type:
 *     double for TVD_MODE_FP64 plans, float for TVD_MODE_MIXED plans. The
 *     solver calls (pcg_solve, tv_deblur) always take double buffers: in MIXED
 *     mode the inner CG runs in float with double scalars and the solution is
 *     accumulated in double by iterative refinement.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Operator calls are asynchronous on that stream. Calls that return host
 *     scalars (pcg_solve, tv_deblur, tvd_plan_create) synchronise it.
 *   - The plan owns all workspace, spectra and tables and frees them in
 *     tvd_plan_destroy. A plan must not be used from two host threads at once.
 *   - Every call returns a tvd_status and never aborts or throws; on error,
 *     tvd_last_error() returns a message for the calling thread.
 */
#ifndef TVD_H
#define TVD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tvd_plan_s* tvd_plan;

/* Boundary conditions of the blur, Sec. 2. */
typedef enum {
    TVD_BC_REFLECTIVE = 0,      /* u_{1-j} = u_j, u_{n+j} = u_{n+1-j} */
    TVD_BC_ANTIREFLECTIVE = 1   /* u_{1-j} = 2u_1 - u_{j+1}, u_{n+j} = 2u_n - u_{n-j}, eq. (anti1d) */
} tvd_bc;

/* Preconditioner X of the inner CG (column names of Tables 1-1 and 2-1). */
typedef enum {
    TVD_PC_NONE = 0,   /* I */
    TVD_PC_DIAG = 1,   /* D = I + alpha diag(L(u)), eq. (D) */
    TVD_PC_FAST = 2,   /* R (reflective, eq. (R2)) or M (anti-reflective, Sec. 3.2) */
    TVD_PC_DFAST = 3,  /* D_R = D^1/2 R D^1/2 or D_M = D^1/2 M D^1/2 (default) */
    TVD_PC_FASTD = 4   /* R_D or M_D: H^^* H^ + alpha s_2(D^-1/2 L D^-1/2), H^ = s_2(H) s_2(D^-1/2), the
                          preconditioner of the scaled system eq. (scalesys), applied as D^1/2 M_D D^1/2 */
} tvd_precond;

/* Arithmetic of the plan. */
typedef enum {
    TVD_MODE_FP64 = 0,  /* every kernel in double: the plain method */
    TVD_MODE_MIXED = 1  /* float kernels, double CG scalars, double iterative refinement */
} tvd_mode;

typedef enum {
    TVD_OK = 0,
    TVD_EINVAL = 1,       /* bad argument: size, pointer, parameter */
    TVD_EPSF_ASYM = 2,    /* PSF not quadrantally symmetric (fast preconditioners need it, Sec. 2) */
    TVD_EPSF_SIZE = 3,    /* PSF side even, or half-width m > n - 2 along an axis */
    TVD_ENOMEM = 4,       /* device allocation failed */
    TVD_ECUDA = 5,        /* a CUDA runtime call failed */
    TVD_ENOCONV = 6,      /* CG hit maxit before ||r_k|| / ||r_0|| < tol */
    TVD_EBREAKDOWN = 7,   /* p^T A p <= 0, r^T z <= 0 with r != 0, or a non-finite scalar */
    TVD_ETIMEOUT = 8      /* a bounded device-side wait gave up (a tensor-core transform product waited
                             about a second for operands that never arrived); the solve stops, the
                             plan stays usable */
} tvd_status;

/* Per-call statistics of tv_deblur. inner_iters, g_norm and functional are
 * caller-owned host arrays with room for `cap` entries each; any of them may be
 * NULL (cap = 0 when all are). g_norm and functional cost one double H^T H
 * product (and, for functional, a data-term and a TV-term reduction) per FP
 * step; NULL skips that work. Zero-initialise the structure (fields added at
 * the end keep older callers' layouts valid). */
typedef struct {
    int outer_iters;         /* FP steps taken */
    int* inner_iters;        /* inner CG iterations of each FP step (first min(outer, cap)) */
    int cap;
    int total_inner_iters;   /* sum over all FP steps */
    int refinement_sweeps;   /* MIXED: float CG solves run in total; FP64: equals outer_iters */
    double last_relres;      /* ||r|| / ||r_0|| of the last FP step (double residual) */
    double last_rel_change;  /* ||u^k - u^{k-1}|| / ||u^k|| of the last FP step */
    tvd_status last_status;  /* status of the last inner solve */
    double* g_norm;          /* ||g(u^k)|| of the iterate FP step k starts from, k = 0, 1, ...,
                                g(u) = H^T (H u - v) + alpha L(u) u of eq. (el); on a reblurring plan
                                the residual norm of eq. (fpp), ||H' v - (H' H + alpha L(u^k)) u^k|| */
    double* functional;      /* T(u^k) = 1/2 ||H u^k - v||^2 + alpha sum_pq sqrt(|D u^k|_pq^2 + beta^2),
                                the discretised functional of eq. (mp), for the same iterates */
    double final_g_norm;     /* the same two quantities for the returned iterate (0 when the */
    double final_functional; /* corresponding array is NULL) */
} tvd_stats;

/* Statistics of tv_deblur_newton. */
typedef struct {
    int steps;               /* Newton steps taken */
    int total_cg_iters;      /* CG iterations over all Jacobian solves */
    int halvings;            /* step-length halvings over all steps */
    double last_t;           /* step length of the last step (1 = full Newton step) */
    double last_rel_change;  /* t ||d|| / ||u|| of the last step */
    double last_cg_relres;   /* ||r|| / ||r_0|| of the last Jacobian solve */
    double g_norm_initial;   /* ||g(u)|| of the incoming iterate */
    double g_norm;           /* ||g(u)|| of the returned iterate */
} tvd_newton_stats;

/*
 * tvd_plan_create -- validate the problem and build the plan.
 *   out         receives the plan handle.
 *   n_rows, n_cols  image size, each in [3, 2048] for TVD_MODE_FP64 plans and
 *               in [3, 4096] for TVD_MODE_MIXED plans (each transform line is
 *               held in shared memory). n_rows = 1 makes a 1D signal of n_cols
 *               samples (Sec. 5.1): its PSF has one row, the row axis carries
 *               no boundary condition and no difference of L, and the 2D
 *               transforms reduce to the 1D ones of Sec. 3.1 (the 1-point
 *               transform is the identity). Such plans always use the FFT form.
 *   psf_host    HOST pointer to the (p_rows x p_cols) PSF, row-major doubles,
 *               centred: psf[(m_r + a) * p_cols + (m_c + b)] = h_{a,b}. Copied.
 *               p_rows, p_cols odd. All-zero outer rows/columns are trimmed (this
 *               does not change H). After trimming, m_r <= n_rows - 2 (m_r = 0
 *               when n_rows = 1) and m_c <= n_cols - 2 (else TVD_EPSF_SIZE), and h must be
 *               quadrantally symmetric h_{a,b} = h_{-a,b} = h_{a,-b} to a relative
 *               tolerance of 1e-12 (else TVD_EPSF_ASYM). Normalisation sum h = 1
 *               (Sec. 2) is the caller's choice and is not enforced.
 *   bc, pc, mode  see the enums above.
 *   stream      stream for the set-up copies (synchronised before return).
 */
tvd_status tvd_plan_create(tvd_plan* out, int n_rows, int n_cols,
                           const double* psf_host, int p_rows, int p_cols,
                           tvd_bc bc, tvd_precond pc, tvd_mode mode, void* stream);

/* Free every device and host resource of the plan. NULL is accepted. */
tvd_status tvd_plan_destroy(tvd_plan plan);

/*
 * ar_blur_apply -- y = H x (transpose = 0) or y = H^T x (transpose = 1).
 * H extends x by the plan's BC and convolves with the PSF (Sec. 2,
 * eq. (blurred1d:matrixform)); H^T is its exact transpose (for reflective BCs
 * and a symmetric PSF, H^T = H, Sec. 3.1). x and y: device arrays of the plan's
 * operator type, n_rows x n_cols, not overlapping.
 */
tvd_status ar_blur_apply(tvd_plan plan, int transpose, const void* x, void* y, void* stream);

/*
 * tv_operator_apply -- y = L(u_lag) x with L = D_r^T W D_r + D_c^T W D_c,
 * W = diag((|D u_lag|^2 + beta^2)^{-1/2}), D_r, D_c forward differences that
 * vanish on the last row / column (zero Neumann, Sec. 1, eq. (el)).
 * u_lag, x, y: device arrays of the plan's operator type; y must not overlap
 * u_lag or x. beta > 0.
 */
tvd_status tv_operator_apply(tvd_plan plan, const void* u_lag, double beta,
                             const void* x, void* y, void* stream);

/*
 * tau_precond_setup -- build the preconditioner of the plan for the FP step at
 * u_lag (device array of the plan's operator type): the diffusivity, D = I +
 * alpha diag(L(u_lag)) (eq. (D)) and the eigenvalues Lambda_H^2 + alpha Lambda_L
 * of R / M in the 2D DCT / hat-S basis (Sec. 3.2). alpha >= 0, beta > 0.
 * Returns TVD_EINVAL if some eigenvalue is not positive.
 */
tvd_status tau_precond_setup(tvd_plan plan, const void* u_lag, double alpha, double beta, void* stream);

/*
 * tau_precond_solve -- z = X^{-1} r with the preconditioner last set up
 * (X = D^1/2 U^{-1} diag(Lambda_H^2 + alpha Lambda_L) U D^1/2 for D_R / D_M,
 * U the 2D DCT-II or hat-S transform). r and z: device arrays of the plan's
 * operator type; r == z is allowed. On a MIXED plan in the GEMM transform form
 * (tvd_plan_set_transform) the result carries the products' rounding: about
 * 3e-3 of max |z| element by element with float operands (tf32 products),
 * 6e-3 with bf16 operands. A GEMM-form product whose bounded wait expired is
 * reported as TVD_ETIMEOUT by the next pcg_solve / tv_deblur on the plan.
 */
tvd_status tau_precond_solve(tvd_plan plan, const void* r, void* z, void* stream);

/*
 * Transform form of the fast preconditioners (R, M, D_R, D_M, R_D, M_D) on a
 * TVD_MODE_MIXED plan. The 2D transform U = B_r (x) B_c of Secs. 2-3 (B the
 * orthonormal DST-I hat-S_n = diag(1, S_{n-2}, 1) of eq. (lambda) for AR, the
 * orthonormal DCT-II C_n of Sec. 3.1 for R) is applied either
 *   TVD_TRANSFORM_FFT:  as the paper's fast transforms, O(n^2 log n), by FFT
 *                       line kernels in shared memory (float), or
 *   TVD_TRANSFORM_GEMM: as four dense products with the n x n matrices B_r,
 *                       B_c on the tensor cores by the library's own kernel
 *                       (TMA operand tiles, tcgen05.mma with the accumulator
 *                       in tensor memory, float accumulation; operands in
 *                       float with tf32 products when a side is below 1024,
 *                       in bf16 from 1024 on; TVD_GEMM_STORAGE=f32 / bf16
 *                       overrides), O(n^3) flops but tensor-core rate.
 * Both give the same preconditioner up to rounding; the preconditioner only
 * shapes the CG iteration, so the form changes iteration counts slightly,
 * never the converged solution (the MIXED double residual decides).
 * FP64 plans always use the FFT form.
 */
typedef enum {
    TVD_TRANSFORM_FFT = 0,
    TVD_TRANSFORM_GEMM = 1
} tvd_transform;

/*
 * tvd_plan_set_transform -- choose the transform form of a plan (kind: a
 * tvd_transform value). A new MIXED plan with a fast preconditioner starts
 * with the GEMM form when both image sides are at least 128 (the environment
 * variable TVD_GEMM_MIN_SIDE changes the bound), else with the FFT form; the
 * environment variable TVD_TRANSFORM ("gemm" / "fft") overrides both.
 * Switching to GEMM allocates the transform matrices (B_r, B_c and, for
 * reflective BCs, their transposes; rows padded to a multiple of 8 elements)
 * and two image-sized operand buffers in the operand type, owned by the plan,
 * and encodes their TMA tensor maps (cuTensorMapEncodeTiled, taken from the
 * driver); switching back frees them. Synchronises `stream` (and, when
 * freeing, the device). Errors: TVD_EINVAL for a NULL plan, an unknown kind,
 * or GEMM on an FP64 plan, a 1D plan (n_rows = 1) or with the I / D
 * preconditioners; TVD_ENOMEM,
 * TVD_ECUDA (also when the driver offers no tensor-map encoder).
 */
tvd_status tvd_plan_set_transform(tvd_plan plan, int kind, void* stream);

/* tvd_plan_transform -- the plan's current tvd_transform (FFT for NULL). */
int tvd_plan_transform(tvd_plan plan);

/* tvd_plan_gemm_storage -- operand storage of the plan's GEMM form: 0 none
 * (FFT form or NULL plan), 1 float operands (tf32 products), 2 bf16 operands. */
int tvd_plan_gemm_storage(tvd_plan plan);

/* tvd_plan_gemm_folded -- 1 when the plan's GEMM form runs the folded products
 * (anti-reflective eq. (fp) plans whose sides are multiples of 256: hat-S's
 * symmetry splits each transform into two half-length ones on the sums and
 * differences of mirror-image entries, so each product does n^3 instead of
 * 2 n^3 flops; TVD_GEMM_FOLD=0 at plan set-up keeps the full products), else 0. */
int tvd_plan_gemm_folded(tvd_plan plan);

/* tvd_plan_gemm_tile -- output tile width of the plan's transform products
 * (64 or 128 columns per 128-row tile), 0 in the FFT form or for NULL. */
int tvd_plan_gemm_tile(tvd_plan plan);

/*
 * tvd_plan_tune -- the library's autotuner of the preconditioner's tile
 * shapes. Times every form of the preconditioner solve that a MIXED 2D plan
 * with a fast preconditioner admits -- the FFT-form line passes, the
 * transform products with 128 x 64 and with 128 x 128 output tiles, and the
 * folded products where the plan allows them (tvd_plan_gemm_folded) -- and
 * leaves the plan in the fastest. The preconditioner solve is the only part of
 * a CG or BiCGstab iteration the forms change (the stencils and vector passes
 * are common); each form is set up for u_lag = 0, alpha = 1e-3, beta = 1e-2,
 * TVD_TUNE_SOLVES solves of one seeded residual are captured in one CUDA graph
 * (direct launches while per-kernel profiling is on), and the graph is
 * replayed `reps` times (0: 3) after one warm-up replay, the fastest replay
 * counting. The choice outlasts later tvd_plan_set_method calls; a later
 * tvd_plan_set_transform to GEMM keeps the chosen tile width and fold choice
 * (after the FFT form won, the default rules of the GEMM form apply).
 * Afterwards the plan needs tau_precond_setup again before tau_precond_solve
 * (tv_deblur and the solvers set themselves up). Allocates and frees three
 * image-sized scratch vectors; synchronises `stream` and the device.
 * report (caller-owned, may be NULL) receives every candidate and the index
 * of the chosen one. Errors: TVD_EINVAL (NULL plan, reps < 0, an FP64 or 1D
 * plan, I / D preconditioners), TVD_ENOMEM, TVD_ECUDA, TVD_ETIMEOUT (a
 * product's bounded wait gave up); after an error the plan may be left in
 * the FFT form.
 */
#define TVD_TUNE_MAX 4
#define TVD_TUNE_SOLVES 16
typedef struct {
    int count;                          /* candidates timed */
    int chosen;                         /* index of the form the plan now runs */
    int transform[TVD_TUNE_MAX];        /* tvd_transform of candidate k */
    int tile_n[TVD_TUNE_MAX];           /* product tile width, 0 for the FFT form */
    int folded[TVD_TUNE_MAX];           /* 1 for the folded products */
    double us_per_solve[TVD_TUNE_MAX];  /* fastest replay / TVD_TUNE_SOLVES, microseconds */
} tvd_tune_report;

tvd_status tvd_plan_tune(tvd_plan plan, int reps, tvd_tune_report* report, void* stream);

/*
 * pcg_solve -- solve (H^T H + alpha L(u_lag)) x = b by preconditioned CG from
 * the initial guess in x_inout, stopping when ||r_k||_2 / ||r_0||_2 < tol
 * (Sec. 5) or after maxit iterations. u_lag, b, x_inout: DOUBLE device arrays.
 * *iters receives the CG iterations (products with A) and *relres the final
 * relative residual; both may be NULL. In MIXED mode the residual used for the
 * stopping test is recomputed in double after each float CG sweep.
 * Synchronises `stream`. The iterations run as a captured chunk of four CG
 * iterations inside a CUDA-graph while node whose condition the device sets
 * from the solver state, so the host reads the state once per solve (once
 * per float sweep in MIXED mode); with TVD_CG_DEVICE_LOOP=0 when the chunk is
 * captured, the host instead relaunches the chunk and polls after each one.
 * Returns TVD_ENOCONV if tol was not reached within maxit iterations.
 */
tvd_status pcg_solve(tvd_plan plan, const void* u_lag, double alpha, double beta,
                     const void* b, void* x_inout, double tol, int maxit,
                     int* iters, double* relres, void* stream);

/*
 * tv_deblur -- the FP iteration u^{k+1} = A(u^k)^{-1} H^T v from u^0 = v
 * (Sec. 5), each step solved by pcg_solve warm-started at u^k (on a REBLUR
 * plan: u^{k+1} = A'(u^k)^{-1} H' v, each step solved by pbicgstab_solve). Runs max_outer
 * steps, or stops earlier when ||u^k - u^{k-1}|| / ||u^k|| < outer_tol
 * (outer_tol <= 0: fixed count). v and u_out: DOUBLE device arrays; u_out may
 * equal v. stats may be NULL. Inner non-convergence of a step is recorded in
 * stats->last_status but does not stop the FP loop; the return value is
 * TVD_ENOCONV if any step did not converge.
 */
tvd_status tv_deblur(tvd_plan plan, const void* v, double alpha, double beta,
                     int max_outer, double outer_tol, double inner_tol, int inner_maxit,
                     void* u_out, tvd_stats* stats, void* stream);

/*
 * Reblurring (Sec. 3, eq. (fpp)): each FP step solves
 *     A' u^{k+1} = H' v,   A' = H' H + alpha L(u^k),
 * with H' the blur of the PSF rotated by 180 degrees under the same
 * anti-reflective BCs (H' = H for the quadrantally symmetric PSFs every plan
 * requires), by preconditioned BiCGstab, since A' is not symmetric. On a
 * reblurring plan the fast preconditioner kinds are the reblurring
 * preconditioners of Sec. 3 in their 2D form (Sec. 3.2):
 *   TVD_PC_FAST  = P   = H' H + alpha AR_2(L(u^k)),
 *   TVD_PC_DFAST = D_P = D^1/2 P D^1/2,
 *   TVD_PC_FASTD = P_D = H^' H^ + alpha AR_2(L~), H^ = H AR_2(D^-1/2) (the
 *                  preconditioner of the scaled system eq. (scalereb)),
 *                  applied as D^1/2 P_D D^1/2,
 * all diagonalised by T_n (x) T_n of eq. (Tn), T_n = hat-S (I + U) (the
 * Remark on AR(A)); their eigenvalues are those of the sine projections at
 * interior frequencies, extended to the border ones as AR(.) prescribes.
 * TVD_PC_NONE and TVD_PC_DIAG keep their meaning.
 */
typedef enum {
    TVD_METHOD_FP = 0,         /* eq. (fp), PCG (default) */
    TVD_METHOD_REBLUR = 1,     /* eq. (fpp), PBiCGstab (anti-reflective BCs only) */
    TVD_METHOD_REBLUR_ARL = 2  /* eq. (fpp) with anti-reflective BCs on L as well ("AR+Reblur+AR L"
                                  of Tables 1-1 and 2-1), PBiCGstab (anti-reflective BCs only) */
} tvd_method;

/*
 * L with anti-reflective BCs (TVD_METHOD_REBLUR_ARL; the remark after
 * eq. (scalereb)): L_AR x applies the divergence-form stencil
 *     w_{i-1} (x_i - x_{i-1}) - w_i (x_{i+1} - x_i)   (per axis)
 * to the AR extension of x (eq. (anti1d)), the diffusivity of a ghost pixel
 * taken from its inner neighbour (exact in 1D, where the AR extension of u
 * repeats the first inner difference). On the first and last line of an axis
 * the two differences and weights then coincide, so that axis contributes
 * nothing there; elsewhere L_AR = L. L_AR is not symmetric; for a constant
 * diffusivity it is the AR blur of the 5-point Laplacian. The preconditioners
 * are those of the REBLUR method (AR_2(.) reads only the interior block, where
 * L_AR = L), with D = I + alpha diag(L_AR) (eq. (D) for this L).
 * tv_operator_apply on such a plan applies L_AR.
 */

/*
 * tvd_plan_set_method -- switch the plan between eq. (fp) with PCG and
 * eq. (fpp) with PBiCGstab, with L under zero Neumann or anti-reflective BCs
 * (method: a tvd_method value). REBLUR and REBLUR_ARL need anti-reflective
 * BCs (else TVD_EINVAL); "a REBLUR plan" below means either. Any earlier tau_precond_setup is
 * discarded; a plan in the GEMM transform form rebuilds its matrices (T_n^-1
 * forward, T_n inverse, per side). tau_precond_setup / tau_precond_solve,
 * tv_deblur and pbicgstab_solve follow the method; pcg_solve on a REBLUR plan
 * and pbicgstab_solve on an FP plan return TVD_EINVAL. Synchronises stream.
 */
tvd_status tvd_plan_set_method(tvd_plan plan, int method, void* stream);

/* tvd_plan_method -- the plan's tvd_method (TVD_METHOD_FP for NULL). */
int tvd_plan_method(tvd_plan plan);

/*
 * pbicgstab_solve -- solve (H' H + alpha L(u_lag)) x = b (eq. (fpp); L_AR on a
 * REBLUR_ARL plan) on a REBLUR plan by preconditioned BiCGstab (van der Vorst's method, cited in
 * Sec. 3) from the initial guess in x_inout, stopping when
 * ||r_k||_2 / ||r_0||_2 < tol (Sec. 5), tested on the half-step residual and
 * on r after each iteration, or after maxit iterations (one iteration: two
 * products with A', two preconditioner solves). u_lag, b, x_inout: DOUBLE
 * device arrays. In MIXED mode BiCGstab runs in float with double scalars
 * inside a double iterative refinement: each float solve, from a fresh shadow
 * residual, reduces the double residual b - A' x (recomputed in double after
 * it) by 1e-4 or to the target. *iters receives the BiCGstab iterations (all
 * float solves together), *relres the final double relative residual; both may
 * be NULL. Returns TVD_ENOCONV if tol was not reached within maxit iterations,
 * TVD_EBREAKDOWN on a zero rho, r^T v or t^T t. Synchronises stream.
 */
tvd_status pbicgstab_solve(tvd_plan plan, const void* u_lag, double alpha, double beta, const void* b,
                           void* x_inout, double tol, int maxit, int* iters, double* relres, void* stream);

/*
 * tv_deblur_batched -- tv_deblur of many independent problems at once (the
 * batched solve of a set of images, each with its own size, PSF and
 * parameters; independent problems share nothing, Sec. 5's FP iteration runs
 * per item). Items are taken largest first by `workers` host threads, each
 * owning a CUDA stream, so the kernels of different items overlap on the GPU.
 * Each item runs exactly tv_deblur(plan, v, alpha, beta, max_outer, 0,
 * inner_tol, inner_maxit, u_out, ...) on its worker's stream: results equal
 * those of separate tv_deblur calls.
 *   items       count caller-owned descriptors (host memory); each names a
 *               plan created by tvd_plan_create. Items that name the same plan
 *               run one after another on one worker.
 *   workers     host threads / streams (1..64; 0 selects 8).
 *   stream      the caller's stream: every item starts after the work queued
 *               on it so far. The call returns when every item has finished.
 * Per-item results go to items[i].status and, when non-NULL,
 * items[i].inner_iters (max_outer entries). Returns TVD_EINVAL for invalid
 * arguments (nothing run), else the first non-OK item status in item order
 * (TVD_OK when all items converged), with that item's message.
 */
typedef struct {
    tvd_plan plan;        /* the item's plan (its size, PSF, BC, preconditioner, mode) */
    const void* v;        /* DOUBLE device array, the observation */
    void* u_out;          /* DOUBLE device array, the restored image (may equal v) */
    double alpha, beta;
    int* inner_iters;     /* optional host array of max_outer entries (NULL: not reported) */
    tvd_status status;    /* out: the item's tv_deblur status */
    double outer_tol;     /* the item's FP stopping rule, as tv_deblur's outer_tol (<= 0: max_outer steps) */
    int outer_iters;      /* out: FP steps the item took */
} tvd_batch_item;

tvd_status tv_deblur_batched(tvd_batch_item* items, int count, int max_outer, double inner_tol,
                             int inner_maxit, int workers, void* stream);

/*
 * tv_hessian_apply -- y = nabla^2 J_beta(u) x, the Hessian of the discrete TV
 * term J_beta(u) = sum_pq sqrt(|D u|_pq^2 + beta^2) of the functional whose
 * stationarity is eq. (el): D^T [psi^-1 D x - psi^-3 (D u . D x) D u] per
 * cell, D the forward differences of L (zero on the last row / column).
 * u, x, y: DOUBLE device arrays of the plan's size (any mode); y distinct
 * from u and x. Synchronises the stream (it allocates and frees 2 n doubles).
 */
tvd_status tv_hessian_apply(tvd_plan plan, const void* u, double beta, const void* x, void* y, void* stream);

/*
 * tv_deblur_newton -- finish the fixed point of eq. (fp) by Newton's method on
 * the Euler-Lagrange equation g(u) = H^T (H u - v) + alpha L(u) u = 0 of
 * eq. (el). Not a construction of the paper: the lagged-diffusivity iteration
 * converges linearly, and the adjoint (tv_deblur_adjoint) wants a stationary
 * point to a tolerance that iteration reaches slowly. From the incoming
 * iterate (normally a tv_deblur result), each step solves
 *     J(u) d = -g(u),   J = H^T H + alpha nabla^2 J_beta(u)   (SPD),
 * by PCG from d = 0 to ||r|| / ||r_0|| < cg_tol (at most cg_maxit iterations),
 * preconditioned by the plan's preconditioner of the lagged operator
 * H^T H + alpha L(u) set up at u (MIXED plans: float PCG with double residual
 * replacement, as in tv_deblur_adjoint), and moves to u + t d with t = 1,
 * halved while ||g(u + t d)|| >= ||g(u)|| (at most 10 halvings; a full step
 * with ||d|| / ||u + d|| < tol is taken as it is, since ||g|| is then at its
 * rounding floor). It stops after the first step with t ||d|| / ||u + t d||
 * < tol, or when g(u) = 0.
 *   v            DOUBLE device array, the observation.
 *   u_inout      DOUBLE device array (distinct from v): the starting iterate in,
 *                the finished iterate out.
 *   tol          relative-change stopping rule (> 0); max_steps >= 0 (0: only
 *                ||g(u)|| is evaluated, into stats->g_norm_initial).
 *   stats        may be NULL.
 * Runs in double in both modes; allocates 6 n (MIXED: 7 n) doubles of scratch
 * and synchronises the stream. Returns TVD_OK when the stopping rule was met;
 * TVD_ENOCONV after max_steps steps without it, or when no halving lowered
 * ||g|| (u_inout then holds the last accepted iterate); TVD_EBREAKDOWN,
 * TVD_ETIMEOUT from a Jacobian solve; TVD_EINVAL for invalid arguments or a
 * reblurring plan (its fixed point is not a stationary point of a functional).
 */
tvd_status tv_deblur_newton(tvd_plan plan, const void* v, double alpha, double beta, void* u_inout, double tol,
                            int max_steps, double cg_tol, int cg_maxit, tvd_newton_stats* stats, void* stream);

/*
 * tv_deblur_adjoint -- gradients of a loss l(u*) of the converged fixed point
 * u* of tv_deblur (g(u*) = H^T (H u* - v) + alpha L(u*) u* = 0, eq. (el)) with
 * respect to alpha, beta and the PSF taps, by implicit differentiation: one
 * solve J lambda = dl/du with J = H^T H + alpha nabla^2 J_beta(u*) (SPD) by
 * PCG from lambda = 0, preconditioned by the plan's preconditioner of the
 * lagged operator H^T H + alpha L(u*) (set up here at u*, replacing any
 * earlier tau_precond_setup), then
 *   dl/dalpha = -lambda^T L(u*) u*,
 *   dl/dbeta  = alpha beta (D lambda)^T [psi^-3 D u*],
 *   dl/dh_ab  = -[(E_ab lambda)^T (H u* - v) + (H lambda)^T E_ab u*]
 * (E_ab = dH/dh_ab: the BC extension shifted by the tap offset). Not a
 * construction of the paper: it differentiates the paper's method. Runs in
 * double in both modes.
 *   u_star, v, dl_du   DOUBLE device arrays (u* should satisfy g(u*) ~ 0:
 *                      run tv_deblur, then tv_deblur_newton to a small tol).
 *   lambda_out         DOUBLE device array, receives lambda (distinct from the inputs).
 *   tol, maxit         ||r_k|| / ||r_0|| < tol stopping rule and cap of the adjoint PCG.
 *   dl_dalpha, dl_dbeta  host doubles (may be NULL).
 *   dl_dpsf            host array of p_rows x p_cols doubles as reported by
 *                      tvd_plan_psf_size (the PSF support after trimming zero
 *                      outer rows / columns), row-major like the PSF; may be NULL.
 *   iters, relres      host outputs of the adjoint PCG (may be NULL).
 * Synchronises the stream. Returns TVD_ENOCONV (gradients still written) if
 * the PCG hit maxit, TVD_EBREAKDOWN if it broke down, TVD_EINVAL on a
 * reblurring plan (its linearisation is not symmetric).
 */
tvd_status tv_deblur_adjoint(tvd_plan plan, const void* u_star, const void* v, double alpha, double beta,
                             const void* dl_du, void* lambda_out, double tol, int maxit, double* dl_dalpha,
                             double* dl_dbeta, double* dl_dpsf, int* iters, double* relres, void* stream);

/* Size of the plan's PSF support (after trimming all-zero outer rows / columns). */
tvd_status tvd_plan_psf_size(tvd_plan plan, int* p_rows, int* p_cols);

/* Message of the last failed call on the calling thread ("" if none). */
const char* tvd_last_error(void);

/* Library version string. */
const char* tvd_version(void);

/*
 * tvd_normal_apply_noalloc -- y = H^T H x + alpha L(u_lag) x in double, for
 * callers that cannot allocate device memory. No counterpart in the paper: it
 * is the PCG's normal-equations product (the same kernels as pcg_solve) made
 * callable without a plan, because some callers must not call cudaMalloc:
 * code inside a framework that owns a fixed device-memory pool (a caching
 * allocator, a real-time or embedded memory budget) and callbacks from such
 * a framework, where a cudaMalloc behind the framework's back would break
 * its accounting or synchronise the device at a point it does not expect.
 *   n_rows, n_cols   image size, n_rows * n_cols <= 524288 (e.g. 512 x 1024);
 *                    larger sizes return TVD_EINVAL with a message.
 *   psf_host, p_rows, p_cols, bc   as for tvd_plan_create (HOST PSF, copied).
 *   u_lag, x         DOUBLE device arrays (n_rows x n_cols); beta > 0, alpha >= 0.
 *   y                DOUBLE device array, must not overlap x or u_lag.
 * Scratch: H x, the diffusivity of u_lag and the PSF tables live in fixed
 * device arrays of the library (8 MiB plus about 0.2 MiB), which every GPU
 * that loads the library holds until the process exits. All calls share
 * them and each call overwrites them, so calls that overlap on the GPU (two
 * streams, or two host threads) race: serialise them. The first call on a
 * device looks up the arrays' device addresses (cudaGetSymbolAddress); that
 * first call should come before any stream capture. The call copies the PSF
 * tables from pageable host memory and synchronises `stream` before
 * returning, so it blocks the calling thread until the product is done.
 */
tvd_status tvd_normal_apply_noalloc(int n_rows, int n_cols, const double* psf_host, int p_rows, int p_cols,
                                    tvd_bc bc, const double* u_lag, double alpha, double beta,
                                    const double* x, double* y, void* stream);

/*
 * Diagnostics (no counterpart in the paper).
 * tvd_kernel_launches -- number of CUDA kernels this library has launched in
 *   the process so far (all plans, all streams).
 * tvd_profile_enable -- on != 0: from now on record a CUDA event pair around
 *   the launches of every kernel class (adds host overhead per launch); on = 0
 *   stops. Either call discards earlier records.
 * tvd_profile_read -- summed device time (ms) and launch count of class
 *   `cls` (0 <= cls < tvd_profile_classes()) since profiling was enabled;
 *   waits for the recorded events. tvd_profile_name gives the class name.
 */
unsigned long long tvd_kernel_launches(void);
tvd_status tvd_profile_enable(int on);
int tvd_profile_classes(void);
const char* tvd_profile_name(int cls);
tvd_status tvd_profile_read(int cls, double* total_ms, long long* launches);

#ifdef __cplusplus
}
#endif
#endif /* TVD_H */
