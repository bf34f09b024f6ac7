// Internal declarations shared by the CUDA translation units of libtvd.
//
// Layout in device memory: every image-sized array is n_rows x n_cols,
// row-major, contiguous, in the plan's compute type T (float or double).
// Small per-plan tables (PSF taps, border tail weights, transform twiddles)
// are separate device arrays loaded into shared memory by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/tvd.h"

namespace tvd {

// ---------------------------------------------------------------- errors

void set_error(const std::string& msg);

struct Status {
    tvd_status code = TVD_OK;
    bool ok() const { return code == TVD_OK; }
};

#define TVD_CUDA_TRY(expr)                                                          \
    do {                                                                            \
        cudaError_t _e = (expr);                                                    \
        if (_e != cudaSuccess) {                                                    \
            ::tvd::set_error(std::string("CUDA error: ") + cudaGetErrorString(_e) + \
                             " at " + __FILE__ + ":" + std::to_string(__LINE__));   \
            return TVD_ECUDA;                                                       \
        }                                                                           \
    } while (0)

#define TVD_TRY(expr)                   \
    do {                                \
        tvd_status _s = (expr);         \
        if (_s != TVD_OK) return _s;    \
    } while (0)

// ---------------------------------------------------------------- launch accounting

enum ProfClass {
    PROF_BLUR_FWD = 0, PROF_BLUR_ADJ, PROF_ROW_FWD, PROF_COL_SOLVE, PROF_ROW_INV, PROF_EG_ROW, PROF_EG_COL,
    PROF_CG_INIT, PROF_CG_PUPDATE, PROF_CG_XR, PROF_CG_SIMPLE, PROF_TV, PROF_MISC, PROF_GEMM, PROF_GEMM_EW,
    PROF_NUM_BASE,
    PROF_NUM_CLASSES = 2 * PROF_NUM_BASE     // float launches use the base id, double ones base + PROF_NUM_BASE
};
template <typename T>
constexpr int prof_class(int base) { return base + (sizeof(T) == 8 ? PROF_NUM_BASE : 0); }

void count_launches(int k);
bool profiling_enabled();
// While a CUDA graph is being captured on this thread, launches are not
// counted (the graph's launches are counted when it is replayed).
void set_capturing(bool on);
int captured_kernels();   // kernels launched since set_capturing(true)

// Counts the launches of one launcher call and, when profiling is on, brackets
// them with CUDA events on the launch stream.
class ProfScope {
  public:
    ProfScope(int cls, cudaStream_t s, int nkernels = 1);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

  private:
    int cls_;
    cudaStream_t s_;
    cudaEvent_t start_;
};

// ---------------------------------------------------------------- small types

template <typename T>
struct cplx {
    T re, im;
};

// Radix plan of a length-L complex FFT (Stockham, mixed radix). When L has a
// prime factor above 31, bl = 1 and the transform is Bluestein's: a circular
// convolution of length M2 (a power of two >= 2L - 1) done by M2-point FFTs
// with the radices radix2.
struct FftPlan {
    int L = 0;
    int nstages = 0;
    int radix[24] = {0};
    int bl = 0;
    int M2 = 0;
    int nst2 = 0;
    int radix2[16] = {0};
};

FftPlan make_fft_plan(int L);

// Device-side scalar state of one CG solve. All scalars are double in both
// modes (the CG recurrences and the stopping test stay in FP64).
struct CgState {
    double rho;        // r^T z of the current iteration
    double rho_old;    // r^T z of the previous iteration
    double pq;         // p^T A p
    double rr;         // ||r||^2 after the last update
    double rr0;        // ||r_0||^2
    double alpha;      // step length
    double beta;       // Fletcher-Reeves coefficient
    double tol2;       // tol^2 * rr0, the stopping threshold on rr
    int iter;          // products with A done so far in this solve
    int maxit;
    int done;          // 1 once converged / stopped
    int status;        // tvd_status reached inside the loop
    int fresh;         // 1: the next search direction is p = z (start or restart)
    int pbuf;          // which of the two direction buffers holds the current p
    int pending;       // 1: alpha is known and x += alpha p, r -= alpha q is still to be applied
    int loops;         // chunks run by the device-driven loop since it was armed
    int loop_budget;   // chunks the device-driven loop may run at most
};

// Reduction slots: each reduction writes one double per block, then the last
// block (ticket counter) sums them in a fixed order.
constexpr int kMaxRedBlocks = 1 << 17;

// Per-precision device resources of a plan.
template <typename T>
struct Ops {
    bool allocated = false;
    // PSF (trimmed): dense (2 m_r + 1) x (2 m_c + 1) taps, and for each column
    // offset b the first and last row offset a with a nonzero tap (lo > hi: none)
    T* hdense = nullptr;
    int* arange = nullptr;
    // PSF rows as runs of one value, (a, first b, last b) and the value; the
    // stencil sums runs from row prefix sums when that is cheaper (nruns > 0)
    int nruns = 0;
    int* runs = nullptr;
    T* runv = nullptr;
    // flat PSF (h_{a,b} = flatv on a support symmetric in both axes whose rows
    // and columns are runs centred on 0, half-widths <= 8: the out-of-focus
    // disk): colh[b + m_c] = the half-height g_|b| of column b (-1: empty); the
    // stencil then sums centred vertical box sums along the row (flat != 0;
    // flat == 2: the disk of radius 7, with its column heights fixed at compile time)
    int flat = 0;
    int* colh = nullptr;
    double flatv = 0.0;
    // AR adjoint border tail weights (Sec. 2 folds), sizes in the plan
    T* crow = nullptr;       // (m_r + 1) x (2 m_c + 1)
    T* ccol = nullptr;       // (2 m_r + 1) x (m_c + 1)
    T* ccor = nullptr;       // (m_r + 1) x (m_c + 1)
    // transform tables: twiddles of the row-direction (length L_c) and
    // column-direction (length L_r) complex FFTs, plus per-transform aux tables
    cplx<T>* tw_c = nullptr;
    cplx<T>* tw_r = nullptr;
    cplx<T>* blt_c = nullptr;   // Bluestein tables (plans with bl): chirp (L) | filter spectrum (M2) | M2 twiddles
    cplx<T>* blt_r = nullptr;
    T* aux_c = nullptr;      // see transform.cu: per-length auxiliary factors
    T* aux_r = nullptr;
    // reblurring (AR, eq. (fpp)): per line length the rank-2 correction vectors
    // S p | S J p of T_n = hat-S (I + U) (2 (n - 2) each), and the weights c of
    // the border eigenvalues of AR(.) (n - 2 doubles each)
    T* ucorr_r = nullptr;    // lines along columns (length n_rows)
    T* ucorr_c = nullptr;    // lines along rows (length n_cols)
    double* extc_r = nullptr;
    double* extc_c = nullptr;
    // preconditioner data
    T* lamH2 = nullptr;      // Lambda_H^2
    T* inv_spec = nullptr;   // 1 / (Lambda_H^2 + alpha Lambda_L)
    T* w = nullptr;          // diffusivity psi^-1
    T* dmh = nullptr;        // D^-1/2
    T* dinv = nullptr;       // D^-1
    // CG vectors and scratch
    T* x = nullptr;
    T* r = nullptr;
    T* z = nullptr;
    T* p = nullptr;          // search direction, double-buffered with p2 (CgState.pbuf)
    T* p2 = nullptr;
    T* q = nullptr;
    T* t = nullptr;          // H p, transform intermediate
    T* t2 = nullptr;         // second transform intermediate (spectrum setup)
};

struct Psf {
    int mr = 0, mc = 0;                 // trimmed half-widths
    std::vector<double> h;              // (2 mr + 1) x (2 mc + 1)
    std::vector<int> ta, tb;            // nonzero taps
    std::vector<double> th;
    std::vector<double> crow, ccol, ccor;
};

}  // namespace tvd

struct tvd_plan_s {
    int nr = 0, nc = 0;
    int method = 0;                     // tvd_method: TVD_METHOD_FP (eq. (fp), PCG), TVD_METHOD_REBLUR or
                                        // TVD_METHOD_REBLUR_ARL (eq. (fpp), PBiCGstab; L or L_AR)
    tvd_bc bc = TVD_BC_ANTIREFLECTIVE;
    tvd_precond pc = TVD_PC_DFAST;
    tvd_mode mode = TVD_MODE_FP64;
    tvd::Psf psf;
    tvd::FftPlan fft_r, fft_c;          // lengths of the column-direction / row-direction FFTs
    tvd::Ops<double> d;                 // double resources (always: FP64 residuals)
    tvd::Ops<float> f;                  // float resources (MIXED only)
    // CG bookkeeping (device)
    tvd::CgState* state = nullptr;
    tvd::CgState* hstate = nullptr;     // pinned host copy of *state
    double* red = nullptr;              // kMaxRedBlocks partial sums
    unsigned int* ticket = nullptr;     // last-block counter
    double* scal = nullptr;             // small double scratch on device
    // double-only arrays for MIXED refinement
    double* hx = nullptr;               // H^T H x in double
    const double* hx_for = nullptr;     // the x that hx belongs to (nullptr: none)
    double* res = nullptr;              // double residual
    double* xd = nullptr;               // double iterate
    double* tmp = nullptr;              // double scratch
    // CUDA graph of a chunk of CG iterations, per arithmetic (float / double);
    // valid for one (x, b, alpha) operand set. `loop` is the same chunk inside a
    // while node whose condition a kernel sets after each chunk (the device runs
    // chunks until the CG state is done); nullptr where it could not be built.
    struct CgGraph {
        cudaGraphExec_t exec = nullptr;
        cudaGraphExec_t loop = nullptr;
        const void* x = nullptr;
        const void* b = nullptr;
        double alpha = -1.0;
        int kernels = 0;
        int loop_kernels = 0;   // kernels per chunk of `loop`, with its condition kernel
        void reset() {
            if (exec) cudaGraphExecDestroy(exec);
            if (loop) cudaGraphExecDestroy(loop);
            exec = nullptr;
            loop = nullptr;
        }
    } graph[2];
    cudaStream_t cap_stream = nullptr;  // plan-owned stream used only to capture graphs
    int last_iters[2] = {0, 0};         // iterations of the previous solve (chunking hint)
    bool precond_ready = false;
    double alpha = 0.0, beta = 0.0;     // parameters of the last setup
    // dense-matrix (GEMM) form of the preconditioner transforms, MIXED plans
    // with a fast preconditioner only (gemm_precond.cu); nullptr: FFT form
    void* gemm = nullptr;
    int gemm_bn = 0;                    // tile width chosen by tvd_plan_tune (0: the default rule)
    int gemm_fold = -1;                 // folded products chosen by tvd_plan_tune (-1: the default rule)
    // BiCGstab state and vectors of the reblurring method (reblur.cu)
    void* bicg = nullptr;
    // eq. (fpp), with L or L_AR
    bool reblur() const { return method == TVD_METHOD_REBLUR || method == TVD_METHOD_REBLUR_ARL; }
};

namespace tvd {

// Validate and trim a PSF for an n_rows x n_cols image (host only).
tvd_status build_psf(Psf& out, const double* h, int pr, int pc, int nr, int nc);

// ---------------------------------------------------------------- launchers
// Each launcher is asynchronous on `s` and returns a tvd_status (launch errors).

// y = H x or H^T x. If st is given, the kernel returns at once when st->done.
template <typename T>
tvd_status blur_apply(const tvd_plan_s& p, const Ops<T>& o, bool transpose, const T* x, T* y, cudaStream_t s,
                      CgState* st = nullptr);

// w = psi^-1 of u; then D^-1/2 and D^-1 with D = 1 + alpha diag(L(w)).
template <typename T>
tvd_status diffusivity(const tvd_plan_s& p, const T* u, double beta, T* w, cudaStream_t s);
template <typename T>
tvd_status diag_scale(const tvd_plan_s& p, const T* w, double alpha, T* dmh, T* dinv, cudaStream_t s);

template <typename T>
tvd_status tv_apply(const tvd_plan_s& p, const T* w, const T* x, T* y, cudaStream_t s);
// y -= alpha (L - L_AR) x on the border lines (after a fused product with L)
template <typename T>
tvd_status lar_border(const tvd_plan_s& p, const T* w, const T* x, T* y, double alpha, cudaStream_t s);

// q = H^T t + alpha L(w) p; with st, p is the direction buffer the current
// iteration wrote (p0 / p1 by st->pbuf), and p^T q -> st->pq, alpha = rho / pq;
// without st, p = p0.
template <typename T>
tvd_status normal_finish(const tvd_plan_s& p, const Ops<T>& o, const T* t, const T* p0, const T* p1, double alpha,
                         T* q, CgState* st, cudaStream_t s);

// y = H t + alpha L(w) x (forward blur of t fused with the TV operator of x):
// with t = H x, the product H' H x + alpha L x of eq. (fpp).
template <typename T>
tvd_status forward_fuse(const tvd_plan_s& p, const Ops<T>& o, const T* t, const T* x, double alpha, T* y,
                        cudaStream_t s);

// Reblurring, eq. (fpp) (reblur.cu): the plan's correction and extension
// tables, y = H' H x + alpha L x (hx: scratch), one FP step's PBiCGstab solve
// (FP64, or float BiCGstab inside double refinement for MIXED plans) with the
// preconditioner already set up, and the release of its resources.
tvd_status reblur_tables(tvd_plan_s& p, cudaStream_t s);
template <typename T>
tvd_status reblur_matvec(const tvd_plan_s& p, const Ops<T>& o, const T* x, T* hx, T* y, double alpha,
                         cudaStream_t s);
tvd_status reblur_solve(tvd_plan_s& p, double alpha, const double* b, double* x, double tol, int maxit, int* iters,
                        int* sweeps, double* relres, tvd_status* status, cudaStream_t s);
void reblur_free(tvd_plan_s& p);
void reblur_graphs_reset(tvd_plan_s& p);   // drop captured BiCGstab chunks (the preconditioner form changed)

// Device-driven solver loops (tvd_api.cu). device_loop_enabled: the
// TVD_CG_DEVICE_LOOP switch (default on). build_while_graph: a graph holding
// one while node (condition 1 at each launch) whose body is captured from
// `body(stream, handle)` on p.cap_stream; the body's last kernel must set the
// condition. Returns false, with the CUDA error state cleared, where the
// driver cannot build it; *kernels = kernels captured in the body.
bool device_loop_enabled();
bool build_while_graph(tvd_plan_s& p, const std::function<tvd_status(cudaStream_t, cudaGraphConditionalHandle)>& body,
                       cudaGraphExec_t* out, int* kernels);

// CG direction update fused with the forward blur: p_new = z (fresh) or
// z + beta p_old, with p_old / p_new the two direction buffers chosen by
// st->pbuf; t = H p_new.
template <typename T>
tvd_status blur_pupdate(const tvd_plan_s& p, const Ops<T>& o, const T* z, T* p0, T* p1, T* t, CgState* st,
                        cudaStream_t s);

// Preconditioner spectrum (requires o.w): inv_spec = 1 / (lamH2 + alpha Lambda_L).
template <typename T>
tvd_status spectrum_setup(const tvd_plan_s& p, Ops<T>& o, double alpha, int* bad_flag, cudaStream_t s);

template <typename T>
tvd_status lamH2_setup(const tvd_plan_s& p, Ops<T>& o, cudaStream_t s);

// z = X^{-1} r. If st != nullptr, also reduce r^T z into st->rho (and run the
// CG scalar update that follows it). With x (CG path), the first pass applies
// the pending update x += alpha p, r -= alpha q (r in place, p and q from o)
// and the stopping test before preconditioning r.
// Dense-matrix (GEMM) form of the fast preconditioners' solve on a float plan
// (gemm_precond.cu): create / destroy its matrices, operand buffers and tensor
// maps, and the solve, with the same contract as precond_solve. The products
// run the library's tensor-core kernel; gemm_precond_check reads (and clears)
// its device error flag: TVD_ETIMEOUT if a product's bounded wait expired.
tvd_status gemm_precond_create(tvd_plan_s& p, cudaStream_t s);
void gemm_precond_destroy(tvd_plan_s& p);
int gemm_precond_storage(const tvd_plan_s& p);  // 0: no GEMM form, 1: float operands, 2: bf16 operands
int gemm_precond_folded(const tvd_plan_s& p);   // 1: the folded (half-K) products
int gemm_precond_tile(const tvd_plan_s& p);     // product tile width, 0: no GEMM form
bool gemm_fold_allowed(const tvd_plan_s& p);    // the plan admits the folded products
tvd_status gemm_precond_check(const tvd_plan_s& p, cudaStream_t s);
tvd_status gemm_precond_solve(const tvd_plan_s& p, const Ops<float>& o, const float* r, float* z, CgState* st,
                              cudaStream_t s, float* x);

template <typename T>
tvd_status precond_solve(const tvd_plan_s& p, const Ops<T>& o, const T* r, T* z, CgState* st, cudaStream_t s,
                         T* x = nullptr);

// Adjoint of the converged fixed point (double): per-cell TV Hessian
// coefficients g = D u psi^-3/2 from u and w = psi^-1; y = nabla^2 J_beta(u) x;
// the adjoint CG product q += alpha nabla^2 J_beta p with p^T q (p the
// direction st->pbuf selects); and the gradient reductions: out2[0] =
// lambda^T L(u) u, out2[1] = sum psi^-3 (D lambda . D u), and with taps the
// per-tap values -[(E_ab lambda)^T (H u - v) + (H lambda)^T E_ab u] (uses o.t,
// o.q and scratch_ext of 2 (n_r + 2 m_r)(n_c + 2 m_c) doubles).
tvd_status hess_coef(const tvd_plan_s& p, const double* u, const double* w, double* gr, double* gc, cudaStream_t s);
tvd_status hess_apply(const tvd_plan_s& p, const double* x, double* y, const double* w, const double* gr,
                      const double* gc, cudaStream_t s);
template <typename T>
tvd_status hess_add(const tvd_plan_s& p, T* q, const T* p0, const T* p1, const T* w, const T* gr, const T* gc,
                    double alpha, CgState* st, cudaStream_t s);
// r = b - hq - alpha nabla^2 J_beta x (double), ||r||^2 into *out_norm2
tvd_status adj_residual(const tvd_plan_s& p, const double* b, const double* hq, const double* w, const double* gr,
                        const double* gc, const double* x, double alpha, double* r, double* out_norm2,
                        cudaStream_t s);
tvd_status adjoint_gradients(const tvd_plan_s& p, const Ops<double>& o, const double* lam, const double* u,
                             const double* v, double alpha, double beta, double* scratch_ext, double* taps,
                             double* out2, cudaStream_t s);

// CG kernels
template <typename T>
tvd_status cg_init(const tvd_plan_s& p, const T* b, const T* ax, T* r, CgState* st, double tol, int maxit,
                   cudaStream_t s);
template <typename T>
tvd_status cg_pupdate(const tvd_plan_s& p, const T* z, T* pv, CgState* st, cudaStream_t s);
// x += alpha p, r -= alpha q with p the current iteration's direction buffer;
// the finisher flips st->pbuf.
template <typename T>
tvd_status cg_xrupdate(const tvd_plan_s& p, T* x, T* r, const T* p0, const T* p1, const T* q, CgState* st,
                       cudaStream_t s);
template <typename T>
tvd_status cg_simple_precond(const tvd_plan_s& p, const T* r, const T* dinv, T* z, CgState* st, cudaStream_t s);

// mode 0: fresh start (iteration count and recurrences cleared); 1: resume
// after a residual replacement keeping the search direction; 2: resume with a
// new search direction p = z (iteration count kept).
template <typename T>
tvd_status cg_restart(const tvd_plan_s& p, const T* r, CgState* st, double tol2, int maxit, int mode,
                      cudaStream_t s);
tvd_status residual_lx(const tvd_plan_s& p, const double* b, const double* hx, const double* w, const double* x,
                       double alpha, double* r, double* out_norm2, cudaStream_t s);
// Device-driven CG loop: cg_loop_arm sets the chunk budget and clears the
// chunk count; cg_loop_cond, the last kernel of each chunk inside the while
// node, counts the chunk and keeps the loop going while the state is not done
// and the budget is not spent.
tvd_status cg_loop_arm(CgState* st, int budget, cudaStream_t s);
tvd_status cg_loop_cond(cudaGraphConditionalHandle h, CgState* st, cudaStream_t s);

// elementwise helpers
tvd_status residual_d(const tvd_plan_s& p, const double* b, const double* ax, double* r, double* out_norm2,
                      cudaStream_t s);
tvd_status norm2_d(const tvd_plan_s& p, const double* a, double* out, cudaStream_t s);
tvd_status diffnorm2_d(const tvd_plan_s& p, const double* a, const double* b, double* out, cudaStream_t s);
// b = (float)(a * scale); x += (double)d * scale
tvd_status cast_d2f(const double* a, float* b, size_t n, cudaStream_t s, double scale = 1.0);
// sum_pq sqrt(|D u|_pq^2 + beta^2) into *out (device), the TV term of eq. (mp)
tvd_status tv_sum_d(const tvd_plan_s& p, const double* u, double beta, double* out, cudaStream_t s);
// out = x0 + t d, ||out||^2 into *norm2 (device)
tvd_status axpy_to_d(const tvd_plan_s& p, const double* x0, const double* d, double t, double* out, double* norm2,
                     cudaStream_t s);
tvd_status copy_f(const float* a, float* b, size_t n, cudaStream_t s);
tvd_status axpy_f2d(double* x, const float* d, size_t n, cudaStream_t s, double scale = 1.0);
tvd_status fill_zero_f(float* a, size_t n, cudaStream_t s);

int num_sms();

}  // namespace tvd
