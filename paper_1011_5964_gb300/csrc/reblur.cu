// Reblurring (Sec. 3, eq. (fpp)) with preconditioned BiCGstab.
//
// Each FP step solves A' u^{k+1} = H' v with A' = H' H + alpha L(u^k), H' the
// anti-reflective blur of the PSF rotated by 180 degrees (H' = H: every plan's
// PSF is quadrantally symmetric). A' is not symmetric, so the inner solver is
// BiCGstab (van der Vorst's method, cited in Sec. 3) with the preconditioned
// directions p^ = X^-1 p, s^ = X^-1 s and the shadow residual r^ = r_0; X is
// I, D, or one of the reblurring preconditioners P, D_P, P_D, all of them
// diagonalised by T_n (x) T_n (eq. (Tn)). The preconditioner solve is the
// plan's usual transform solve with T_n = hat-S (I + U) in place of hat-S (the
// rank-2 corrections inside the FFT line passes, or the dense T_n^-1 / T_n in
// the GEMM form) and the AR_2 spectrum (transform.cu).
//
// Iteration (all scalars double, on the device; every kernel returns at once
// once the solve is done, so iterations are enqueued in chunks between host
// checks):
//   rho = r^ . r;  beta = (rho / rho_old)(alpha / omega);  p = r + beta (p - omega v)
//   p^ = X^-1 p;  v = A' p^;  alpha = rho / (r^ . v);  s = r - alpha v
//   ||s|| / ||r_0|| < tol: x += alpha p^, done
//   s^ = X^-1 s;  t = A' s^;  omega = (t . s) / (t . t)
//   x += alpha p^ + omega s^;  r = s - omega t;  ||r|| / ||r_0|| < tol: done
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace tvd {

// ---------------------------------------------------------------- host tables

// S_m[k][j], k, j = 1..m: the orthonormal DST-I of eq. (lambda), argument reduced in integers.
static double sine_entry(int m, int k, int j) {
    const double pi = 3.14159265358979323846;
    const long long a = ((long long)k * j) % (2LL * (m + 1));
    return std::sqrt(2.0 / (m + 1)) * std::sin(pi * (double)a / (m + 1));
}

// (S p | S J p), p_j = 1 - j / (n - 1), j = 1..n-2: the interior of U's border columns.
static void ucorr_vectors(int n, std::vector<double>& out) {
    const int m = n - 2;
    out.assign(2 * (size_t)std::max(m, 0), 0.0);
    for (int k = 1; k <= m; ++k) {
        double a = 0.0, b = 0.0;
        for (int j = 1; j <= m; ++j) {
            const double s = sine_entry(m, k, j);
            a += s * (1.0 - (double)j / (n - 1));
            b += s * ((double)j / (n - 1));
        }
        out[k - 1] = a;
        out[m + k - 1] = b;
    }
}

// c with z_1 + 2 sum_{k >= 2} z_k = c . lam for the tau matrix S diag(lam) S,
// z its Toeplitz generator (first column c_k = z_k - z_{k+2}): the border
// eigenvalue AR(.) assigns from the interior ones.
static void extension_weights(int n, std::vector<double>& c) {
    const int m = n - 2;
    c.assign(std::max(m, 0), 0.0);
    if (m <= 0) return;   // a line of one sample (a 1D signal's row axis) has no border to extend
    std::vector<double> col(m), z(m + 2);
    for (int i = 1; i <= m; ++i) {
        const double s1 = sine_entry(m, i, 1);
        for (int k = 1; k <= m; ++k) col[k - 1] = sine_entry(m, k, i) * s1;
        std::fill(z.begin(), z.end(), 0.0);
        for (int k = m - 1; k >= 0; --k) z[k] = col[k] + z[k + 2];
        double g = z[0];
        for (int k = 1; k < m; ++k) g += 2.0 * z[k];
        c[i - 1] = g;
    }
}

template <typename T>
static tvd_status upload_vec(T** dst, const std::vector<double>& src, cudaStream_t s) {
    if (*dst) return TVD_OK;
    const size_t n = std::max<size_t>(src.size(), 1);
    if (cudaMalloc((void**)dst, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        set_error("cudaMalloc failed for the reblurring tables");
        return TVD_ENOMEM;
    }
    std::vector<T> tmp(src.begin(), src.end());
    if (tmp.empty()) tmp.push_back(T(0));
    TVD_CUDA_TRY(cudaMemcpyAsync(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    TVD_CUDA_TRY(cudaStreamSynchronize(s));
    return TVD_OK;
}

template <typename T>
static tvd_status ops_tables(const tvd_plan_s& p, Ops<T>& o, cudaStream_t s) {
    std::vector<double> v;
    ucorr_vectors(p.nr, v);
    TVD_TRY(upload_vec<T>(&o.ucorr_r, v, s));
    ucorr_vectors(p.nc, v);
    TVD_TRY(upload_vec<T>(&o.ucorr_c, v, s));
    extension_weights(p.nr, v);
    TVD_TRY(upload_vec<double>(&o.extc_r, v, s));
    extension_weights(p.nc, v);
    TVD_TRY(upload_vec<double>(&o.extc_c, v, s));
    return TVD_OK;
}

tvd_status reblur_tables(tvd_plan_s& p, cudaStream_t s) {
    TVD_TRY(ops_tables<double>(p, p.d, s));
    if (p.mode == TVD_MODE_MIXED) TVD_TRY(ops_tables<float>(p, p.f, s));
    return TVD_OK;
}

template <typename T>
static void free_tables(Ops<T>& o) {
    if (o.ucorr_r) cudaFree(o.ucorr_r);
    if (o.ucorr_c) cudaFree(o.ucorr_c);
    if (o.extc_r) cudaFree(o.extc_r);
    if (o.extc_c) cudaFree(o.extc_c);
    o.ucorr_r = o.ucorr_c = nullptr;
    o.extc_r = o.extc_c = nullptr;
}

// ---------------------------------------------------------------- device state and vectors

struct BiState {
    double rho, rho_old, alpha, omega, beta;
    double rv, ss, ts, tt, rr, rr0, tol2;
    int iter, maxit, done, status, half, first;
    int loops, loop_budget;   // device-driven loop: chunks run since armed, and the most it may run
};

template <typename T>
struct BiVecs {
    T *rhat = nullptr, *p = nullptr, *v = nullptr, *phat = nullptr, *s = nullptr, *shat = nullptr, *t = nullptr,
      *hx = nullptr, *b = nullptr;
};

struct BiResources {
    BiState* st = nullptr;
    BiState* hst = nullptr;   // pinned host copy
    BiVecs<float> f;
    BiVecs<double> d;
    bool have_f = false, have_d = false;
    // captured chunk of iterations in a while node, per arithmetic (float / double),
    // valid for one (x, r, alpha)
    struct Loop {
        cudaGraphExec_t exec = nullptr;
        const void* x = nullptr;
        const void* r = nullptr;
        double alpha = -1.0;
        int kernels = 0;
        void reset() {
            if (exec) cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
    } loop[2];
};

template <typename T>
static void free_vecs(BiVecs<T>& v) {
    T* all[] = {v.rhat, v.p, v.v, v.phat, v.s, v.shat, v.t, v.hx, v.b};
    for (T* q : all)
        if (q) cudaFree(q);
    v = BiVecs<T>();
}

void reblur_free(tvd_plan_s& p) {
    free_tables(p.d);
    free_tables(p.f);
    auto* r = static_cast<BiResources*>(p.bicg);
    if (!r) return;
    for (auto& l : r->loop) l.reset();
    if (r->st) cudaFree(r->st);
    if (r->hst) cudaFreeHost(r->hst);
    free_vecs(r->f);
    free_vecs(r->d);
    delete r;
    p.bicg = nullptr;
}

void reblur_graphs_reset(tvd_plan_s& p) {
    auto* r = static_cast<BiResources*>(p.bicg);
    if (r)
        for (auto& l : r->loop) l.reset();
}

template <typename T>
static tvd_status alloc_vecs(BiVecs<T>& v, size_t n) {
    T** all[] = {&v.rhat, &v.p, &v.v, &v.phat, &v.s, &v.shat, &v.t, &v.hx, &v.b};
    for (T** q : all) {
        if (cudaMalloc((void**)q, n * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            *q = nullptr;
            set_error("cudaMalloc failed for the BiCGstab vectors");
            return TVD_ENOMEM;
        }
    }
    return TVD_OK;
}

static tvd_status resources(tvd_plan_s& p, bool need_f, BiResources** out) {
    auto* r = static_cast<BiResources*>(p.bicg);
    if (!r) {
        r = new BiResources();
        p.bicg = r;
        if (cudaMalloc((void**)&r->st, sizeof(BiState)) != cudaSuccess ||
            cudaMallocHost((void**)&r->hst, sizeof(BiState)) != cudaSuccess) {
            cudaGetLastError();
            set_error("allocation of the BiCGstab state failed");
            return TVD_ENOMEM;
        }
    }
    const size_t n = (size_t)p.nr * p.nc;
    if (!r->have_d) {
        TVD_TRY(alloc_vecs(r->d, n));
        r->have_d = true;
    }
    if (need_f && !r->have_f) {
        TVD_TRY(alloc_vecs(r->f, n));
        r->have_f = true;
    }
    *out = r;
    return TVD_OK;
}

// ---------------------------------------------------------------- kernels

// Two block sums in a fixed order, then the last block (ticket) sums the
// per-block partials (red: slots [0, total) and [total, 2 total)).
__device__ __forceinline__ bool block_reduce2_last(double a, double b, double* red, unsigned int* ticket, int total,
                                                   double* oa, double* ob) {
    __shared__ bool s_last;
    const double ba = block_sum(a);
    const double bb = block_sum(b);
    if (threadIdx.x == 0) {
        red[blockIdx.x] = ba;
        red[total + blockIdx.x] = bb;
        __threadfence();
        const unsigned int t = atomicAdd(ticket, 1u);
        s_last = (t == (unsigned int)(total - 1));
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double sa = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        sa += __ldcg(red + i);
        sb += __ldcg(red + total + i);
    }
    sa = block_sum(sa);
    sb = block_sum(sb);
    if (threadIdx.x == 0) {
        *oa = sa;
        *ob = sb;
        *ticket = 0u;
    }
    return true;
}

__device__ __forceinline__ void bi_fail(BiState* st, int status) {
    st->status = status;
    st->done = 1;
}

#define BI_LOOP(i, n) for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

// r = b - A x, r^ = r, ||r_0||^2, the stopping threshold
template <typename T>
__global__ void __launch_bounds__(kThreads)
bi_init_kernel(const T* __restrict__ b, const T* __restrict__ ax, T* __restrict__ r, T* __restrict__ rhat, size_t n,
               double tol2_rel, double tol2_abs, int maxit, BiState* st, double* red, unsigned int* ticket) {
    double part = 0.0;
    BI_LOOP(i, n) {
        const T v = b[i] - ax[i];
        r[i] = v;
        rhat[i] = v;
        part += (double)v * (double)v;
    }
    double sum;
    if (block_reduce_last(part, red, ticket, blockIdx.x, gridDim.x, &sum) && threadIdx.x == 0) {
        st->rr0 = sum;
        st->rr = sum;
        st->tol2 = fmax(tol2_rel * sum, tol2_abs);
        st->iter = 0;
        st->maxit = maxit;
        st->first = 1;
        st->half = 0;
        st->status = TVD_OK;
        st->rho = st->rho_old = st->alpha = st->omega = 1.0;
        st->done = 0;
        if (!isfinite(sum)) bi_fail(st, TVD_EBREAKDOWN);
        else if (sum <= st->tol2) st->done = 1;
        if (maxit <= 0 && !st->done) bi_fail(st, TVD_ENOCONV);
    }
}

// rho = r^ . r and the direction coefficient
template <typename T>
__global__ void __launch_bounds__(kThreads)
bi_rho_kernel(const T* __restrict__ rhat, const T* __restrict__ r, size_t n, BiState* st, double* red,
              unsigned int* ticket) {
    if (st->done) return;
    double part = 0.0;
    BI_LOOP(i, n) part += (double)rhat[i] * (double)r[i];
    double rho;
    if (block_reduce_last(part, red, ticket, blockIdx.x, gridDim.x, &rho) && threadIdx.x == 0) {
        if (st->iter >= st->maxit) bi_fail(st, TVD_ENOCONV);
        else if (!(rho != 0.0) || !isfinite(rho)) bi_fail(st, TVD_EBREAKDOWN);
        else {
            st->beta = st->first ? 0.0 : (rho / st->rho_old) * (st->alpha / st->omega);
            st->rho = rho;
        }
    }
}

// p = r (first iteration) or r + beta (p - omega v)
template <typename T>
__global__ void __launch_bounds__(kThreads)
bi_p_kernel(const T* __restrict__ r, const T* __restrict__ v, T* __restrict__ p, size_t n, const BiState* st) {
    if (st->done) return;
    if (st->first) {
        BI_LOOP(i, n) p[i] = r[i];
        return;
    }
    const T be = T(st->beta), om = T(st->omega);
    BI_LOOP(i, n) p[i] = r[i] + be * (p[i] - om * v[i]);
}

// alpha = rho / (r^ . v)
template <typename T>
__global__ void __launch_bounds__(kThreads)
bi_alpha_kernel(const T* __restrict__ rhat, const T* __restrict__ v, size_t n, BiState* st, double* red,
                unsigned int* ticket) {
    if (st->done) return;
    double part = 0.0;
    BI_LOOP(i, n) part += (double)rhat[i] * (double)v[i];
    double rv;
    if (block_reduce_last(part, red, ticket, blockIdx.x, gridDim.x, &rv) && threadIdx.x == 0) {
        st->rv = rv;
        if (!(rv != 0.0) || !isfinite(rv)) bi_fail(st, TVD_EBREAKDOWN);
        else st->alpha = st->rho / rv;
    }
}

// s = r - alpha v and ||s||^2; below the threshold the iteration ends at this half step
template <typename T>
__global__ void __launch_bounds__(kThreads)
bi_s_kernel(const T* __restrict__ r, const T* __restrict__ v, T* __restrict__ s, size_t n, BiState* st, double* red,
            unsigned int* ticket) {
    if (st->done) return;
    const T al = T(st->alpha);
    double part = 0.0;
    BI_LOOP(i, n) {
        const T w = r[i] - al * v[i];
        s[i] = w;
        part += (double)w * (double)w;
    }
    double ss;
    if (block_reduce_last(part, red, ticket, blockIdx.x, gridDim.x, &ss) && threadIdx.x == 0) {
        st->ss = ss;
        if (!isfinite(ss)) bi_fail(st, TVD_EBREAKDOWN);
        else if (ss < st->tol2) st->half = 1;
    }
}

// half-step exit: x += alpha p^, the iteration counted, done
template <typename T>
__global__ void __launch_bounds__(kThreads)
bi_half_kernel(T* __restrict__ x, const T* __restrict__ phat, size_t n, BiState* st, unsigned int* ticket) {
    if (st->done || !st->half) return;
    const T al = T(st->alpha);
    BI_LOOP(i, n) x[i] += al * phat[i];
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        *ticket = 0u;
        st->rr = st->ss;
        st->iter += 1;
        st->done = 1;
    }
}

// omega = (t . s) / (t . t)
template <typename T>
__global__ void __launch_bounds__(kThreads)
bi_omega_kernel(const T* __restrict__ t, const T* __restrict__ s, size_t n, BiState* st, double* red,
                unsigned int* ticket) {
    if (st->done) return;
    double a = 0.0, b = 0.0;
    BI_LOOP(i, n) {
        a += (double)t[i] * (double)s[i];
        b += (double)t[i] * (double)t[i];
    }
    double ts, tt;
    if (block_reduce2_last(a, b, red, ticket, gridDim.x, &ts, &tt) && threadIdx.x == 0) {
        st->ts = ts;
        st->tt = tt;
        if (!(tt > 0.0) || !isfinite(tt) || !isfinite(ts)) bi_fail(st, TVD_EBREAKDOWN);
        else st->omega = ts / tt;
    }
}

// x += alpha p^ + omega s^, r = s - omega t, ||r||^2 and the stopping test
template <typename T>
__global__ void __launch_bounds__(kThreads)
bi_xr_kernel(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ phat, const T* __restrict__ shat,
             const T* __restrict__ s, const T* __restrict__ t, size_t n, BiState* st, double* red,
             unsigned int* ticket) {
    if (st->done) return;
    const T al = T(st->alpha), om = T(st->omega);
    double part = 0.0;
    BI_LOOP(i, n) {
        x[i] += al * phat[i] + om * shat[i];
        const T w = s[i] - om * t[i];
        r[i] = w;
        part += (double)w * (double)w;
    }
    double rr;
    if (block_reduce_last(part, red, ticket, blockIdx.x, gridDim.x, &rr) && threadIdx.x == 0) {
        st->rr = rr;
        st->iter += 1;
        st->first = 0;
        st->rho_old = st->rho;
        if (!isfinite(rr)) bi_fail(st, TVD_EBREAKDOWN);
        else if (rr < st->tol2) st->done = 1;
        else if (st->omega == 0.0) bi_fail(st, TVD_EBREAKDOWN);
    }
}

// ---------------------------------------------------------------- host drivers

static int bi_blocks(size_t n) {
    size_t b = (n + kThreads - 1) / kThreads;
    const size_t cap = (size_t)num_sms() * 4;
    if (b > cap) b = cap;
    return (int)(b ? b : 1);
}

// y = A' x = H' H x + alpha L(w) x (H' = H: the plan's PSF is symmetric; L_AR on a
// REBLUR_ARL plan, as the fused L product plus its border-line correction); hx: scratch
template <typename T>
tvd_status reblur_matvec(const tvd_plan_s& p, const Ops<T>& o, const T* x, T* hx, T* y, double alpha,
                         cudaStream_t s) {
    TVD_TRY(blur_apply<T>(p, o, false, x, hx, s));
    TVD_TRY(forward_fuse<T>(p, o, hx, x, alpha, y, s));
    if (p.method == TVD_METHOD_REBLUR_ARL) TVD_TRY(lar_border<T>(p, o.w, x, y, alpha, s));
    return TVD_OK;
}

template <typename T>
static tvd_status precond(tvd_plan_s& p, Ops<T>& o, const T* r, T* z, cudaStream_t s) {
    switch (p.pc) {
        case TVD_PC_NONE: return cg_simple_precond<T>(p, r, nullptr, z, nullptr, s);
        case TVD_PC_DIAG: return cg_simple_precond<T>(p, r, o.dinv, z, nullptr, s);
        default: return precond_solve<T>(p, o, r, z, nullptr, s);
    }
}

constexpr int kBiChunk = 4;   // iterations per chunk (between host checks, or per pass of the device loop)

__global__ void bi_loop_arm_kernel(BiState* st, int budget) {
    st->loops = 0;
    st->loop_budget = budget;
}

// Last kernel of a chunk inside the while node (plain stream order: it reads
// the state the chunk's last kernel left): count the chunk, go on while the
// solve is not done and the budget lasts.
__global__ void bi_loop_cond_kernel(cudaGraphConditionalHandle h, BiState* st) {
    const int k = st->loops + 1;
    st->loops = k;
    cudaGraphSetConditional(h, (!st->done && k < st->loop_budget) ? 1u : 0u);
}

// BiCGstab on A' x = b (type T) from the x given; stops when ||r||^2 <=
// max(tol2_rel ||r_0||^2, tol2_abs), or after maxit iterations.
template <typename T>
static tvd_status bicg_run(tvd_plan_s& p, Ops<T>& o, BiVecs<T>& bv, BiResources& res, double alpha, const T* b,
                           T* x, T* r, double tol2_rel, double tol2_abs, int maxit, BiState* out, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    const int blocks = bi_blocks(n);
    BiState* st = res.st;
    double* red = p.red;
    unsigned int* tk = p.ticket + 10;
    TVD_TRY(reblur_matvec<T>(p, o, x, bv.hx, bv.t, alpha, s));
    {
        ProfScope prof(prof_class<T>(PROF_CG_INIT), s);
        bi_init_kernel<T><<<blocks, kThreads, 0, s>>>(b, bv.t, r, bv.rhat, n, tol2_rel, tol2_abs, maxit, st, red, tk);
        TVD_CUDA_TRY(cudaGetLastError());
    }
    // one chunk: kBiChunk iterations on stream q (kernels of a finished solve return at once)
    auto chunk = [&](cudaStream_t q) -> tvd_status {
        for (int it = 0; it < kBiChunk; ++it) {
            {
                ProfScope prof(prof_class<T>(PROF_CG_SIMPLE), q, 2);
                bi_rho_kernel<T><<<blocks, kThreads, 0, q>>>(bv.rhat, r, n, st, red, tk);
                bi_p_kernel<T><<<blocks, kThreads, 0, q>>>(r, bv.v, bv.p, n, st);
                TVD_CUDA_TRY(cudaGetLastError());
            }
            TVD_TRY(precond<T>(p, o, bv.p, bv.phat, q));
            TVD_TRY(reblur_matvec<T>(p, o, bv.phat, bv.hx, bv.v, alpha, q));
            {
                ProfScope prof(prof_class<T>(PROF_CG_SIMPLE), q, 3);
                bi_alpha_kernel<T><<<blocks, kThreads, 0, q>>>(bv.rhat, bv.v, n, st, red, tk);
                bi_s_kernel<T><<<blocks, kThreads, 0, q>>>(r, bv.v, bv.s, n, st, red, tk);
                bi_half_kernel<T><<<blocks, kThreads, 0, q>>>(x, bv.phat, n, st, tk);
                TVD_CUDA_TRY(cudaGetLastError());
            }
            TVD_TRY(precond<T>(p, o, bv.s, bv.shat, q));
            TVD_TRY(reblur_matvec<T>(p, o, bv.shat, bv.hx, bv.t, alpha, q));
            {
                ProfScope prof(prof_class<T>(PROF_CG_XR), q, 2);
                bi_omega_kernel<T><<<blocks, kThreads, 0, q>>>(bv.t, bv.s, n, st, red, tk);
                bi_xr_kernel<T><<<blocks, kThreads, 0, q>>>(x, r, bv.phat, bv.shat, bv.s, bv.t, n, st, red, tk);
                TVD_CUDA_TRY(cudaGetLastError());
            }
        }
        return TVD_OK;
    };
    // device-driven loop: the chunk in a while node, one launch per solve
    auto& L = res.loop[sizeof(T) == 8 ? 1 : 0];
    if (!profiling_enabled() && device_loop_enabled()) {
        if (!(L.exec && L.x == x && L.r == r && L.alpha == alpha)) {
            L.reset();
            const bool built = build_while_graph(
                p,
                [&](cudaStream_t q, cudaGraphConditionalHandle h) -> tvd_status {
                    TVD_TRY(chunk(q));
                    ProfScope prof(PROF_MISC, q);
                    bi_loop_cond_kernel<<<1, 1, 0, q>>>(h, st);
                    TVD_CUDA_TRY(cudaGetLastError());
                    return TVD_OK;
                },
                &L.exec, &L.kernels);
            L.x = x;
            L.r = r;
            L.alpha = built ? alpha : -1.0;
        }
        if (L.exec) {
            {
                ProfScope prof(PROF_MISC, s);
                bi_loop_arm_kernel<<<1, 1, 0, s>>>(st, maxit / kBiChunk + 3);
                TVD_CUDA_TRY(cudaGetLastError());
            }
            TVD_CUDA_TRY(cudaGraphLaunch(L.exec, s));
            TVD_CUDA_TRY(cudaMemcpyAsync(res.hst, st, sizeof(BiState), cudaMemcpyDeviceToHost, s));
            TVD_CUDA_TRY(cudaStreamSynchronize(s));
            count_launches(res.hst->loops * L.kernels);
            if (!res.hst->done) {   // the state stops at maxit, within the chunk budget
                set_error("BiCGstab state did not reach done within its chunk budget");
                return TVD_ECUDA;
            }
            *out = *res.hst;
            return TVD_OK;
        }
    }
    int last_iter = -1;
    for (;;) {
        TVD_TRY(chunk(s));
        TVD_CUDA_TRY(cudaMemcpyAsync(res.hst, st, sizeof(BiState), cudaMemcpyDeviceToHost, s));
        TVD_CUDA_TRY(cudaStreamSynchronize(s));
        if (res.hst->done) break;
        if (res.hst->iter == last_iter) {   // the kernels always advance a running solve
            set_error("BiCGstab made no progress between two checks");
            return TVD_ECUDA;
        }
        last_iter = res.hst->iter;
    }
    *out = *res.hst;
    return TVD_OK;
}

template tvd_status reblur_matvec<float>(const tvd_plan_s&, const Ops<float>&, const float*, float*, float*, double,
                                         cudaStream_t);
template tvd_status reblur_matvec<double>(const tvd_plan_s&, const Ops<double>&, const double*, double*, double*,
                                          double, cudaStream_t);

// eq. (fpp) for one FP step: preconditioner set up by the caller, x updated in place.
tvd_status reblur_solve(tvd_plan_s& p, double alpha, const double* b, double* x, double tol, int maxit, int* iters,
                        int* sweeps, double* relres, tvd_status* status, cudaStream_t s) {
    BiResources* res = nullptr;
    TVD_TRY(resources(p, p.mode == TVD_MODE_MIXED, &res));
    const size_t n = (size_t)p.nr * p.nc;
    *iters = 0;
    *sweeps = 0;
    *relres = 0.0;
    *status = TVD_OK;
    if (p.mode == TVD_MODE_FP64) {
        BiState h;
        TVD_TRY(bicg_run<double>(p, p.d, res->d, *res, alpha, b, x, p.res, tol * tol, 0.0, maxit, &h, s));
        *iters = h.iter;
        *sweeps = 1;
        *relres = h.rr0 > 0.0 ? std::sqrt(h.rr / h.rr0) : 0.0;
        *status = (tvd_status)h.status;
        return TVD_OK;
    }
    // MIXED: float BiCGstab on A' d = r inside a double refinement of x
    BiVecs<double>& vd = res->d;
    BiVecs<float>& vf = res->f;
    auto residual = [&](double* rr) -> tvd_status {
        TVD_TRY(reblur_matvec<double>(p, p.d, x, vd.hx, vd.t, alpha, s));
        TVD_TRY(residual_d(p, b, vd.t, p.res, p.scal, s));
        TVD_CUDA_TRY(cudaMemcpyAsync(rr, p.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
        TVD_CUDA_TRY(cudaStreamSynchronize(s));
        return TVD_OK;
    };
    double rr0 = 0.0;
    TVD_TRY(residual(&rr0));
    if (!std::isfinite(rr0)) {
        *status = TVD_EBREAKDOWN;
        return TVD_OK;
    }
    if (rr0 == 0.0) return TVD_OK;
    const double target = tol * tol * rr0, delta2 = 1e-8;
    *relres = 1.0;
    for (;;) {
        TVD_TRY(cast_d2f(p.res, vf.b, n, s));
        TVD_TRY(fill_zero_f(p.f.x, n, s));
        BiState h;
        // the float solve's own threshold: its residual fell by delta, or below the target
        TVD_TRY(bicg_run<float>(p, p.f, vf, *res, alpha, vf.b, p.f.x, p.f.r, delta2, target,
                                std::max(1, maxit - *iters), &h, s));
        *iters += h.iter;
        *sweeps += 1;
        TVD_TRY(axpy_f2d(x, p.f.x, n, s));
        double rr = 0.0;
        TVD_TRY(residual(&rr));
        if (!std::isfinite(rr) || h.status == TVD_EBREAKDOWN) {
            *status = TVD_EBREAKDOWN;
            break;
        }
        *relres = std::sqrt(rr / rr0);
        if (rr < target) break;
        if (*iters >= maxit || *sweeps > 200) {
            *status = TVD_ENOCONV;
            break;
        }
    }
    return TVD_OK;
}

}  // namespace tvd
