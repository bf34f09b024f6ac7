// Vector kernels of the preconditioned CG of Golub & Van Loan, Alg. 10.3.1
// (cited in Sec. 1 of the paper): residual initialisation, search-direction
// update, iterate/residual update with the stopping test ||r_k|| / ||r_0|| < tol
// (Sec. 5), and the plain preconditioners I and D = I + alpha diag(L) (eq. (D)).
//
// Scalars live in a device CgState (double in every mode); each reduction is a
// fixed-order two-stage sum (per-block partials, then the last block), so
// results are bit-reproducible run to run. Every kernel returns at once when
// the state says the solve is done, so the host may enqueue iterations ahead
// of the convergence test.
#include "common.cuh"

namespace tvd {

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Grid of the vector kernels: about four elements per thread, so that every
// SM has many independent loads in flight (the kernels are latency bound at
// L2-resident sizes otherwise).
static int red_blocks(size_t n) {
    size_t b = (n + 4 * kThreads - 1) / (4 * kThreads);
    size_t cap = (size_t)num_sms() * 32;
    if (cap > (size_t)kMaxRedBlocks) cap = kMaxRedBlocks;
    return (int)(b < cap ? (b ? b : 1) : cap);
}

#define GRID_STRIDE(o, n) for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < (n); o += (size_t)gridDim.x * blockDim.x)

// 16-byte vectors: float4 / double2. The vector kernels process one vector per
// thread (all loads of a thread in flight together) and a scalar tail.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };

template <typename T>
__device__ __forceinline__ typename Vec16<T>::type vload(const T* p, size_t i) {
    return reinterpret_cast<const typename Vec16<T>::type*>(p)[i];
}
template <typename T>
__device__ __forceinline__ void vstore(T* p, size_t i, const typename Vec16<T>::type& v) {
    reinterpret_cast<typename Vec16<T>::type*>(p)[i] = v;
}
template <typename T>
__device__ __forceinline__ T* el(typename Vec16<T>::type& v) { return reinterpret_cast<T*>(&v); }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static int vec_blocks(size_t n, int vec) {
    size_t b = (n / vec + kThreads - 1) / kThreads;
    if (b > (size_t)kMaxRedBlocks) b = kMaxRedBlocks;
    return (int)(b ? b : 1);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
cg_init_kernel(const T* __restrict__ b, const T* __restrict__ ax, T* __restrict__ r, size_t n, CgState* st,
               double* red, unsigned int* ticket, double tol, int maxit) {
    T part = T(0);   // per-thread partial in the kernel's type; block and grid sums in double
    GRID_STRIDE(o, n) {
        const T v = b[o] - ax[o];
        r[o] = v;
        part += v * v;
    }
    double s;
    if (block_reduce_last((double)part, red, ticket, blockIdx.x, gridDim.x, &s) && threadIdx.x == 0) {
        st->rr0 = s;
        st->rr = s;
        st->tol2 = tol * tol * s;
        st->iter = 0;
        st->maxit = maxit;
        st->rho = 0.0;
        st->rho_old = 0.0;
        st->beta = 0.0;
        st->alpha = 0.0;
        st->pq = 0.0;
        st->status = TVD_OK;
        st->done = 0;
        st->fresh = 1;
        st->pending = 0;
        if (!isfinite(s)) {
            st->status = TVD_EBREAKDOWN;
            st->done = 1;
        } else if (s == 0.0 || maxit <= 0) {
            st->done = 1;
            if (s != 0.0) st->status = TVD_ENOCONV;
        }
    }
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(kThreads)
cg_pupdate_kernel(const T* __restrict__ z, T* __restrict__ p, size_t n, const CgState* st) {
    if (st->done) return;
    const bool first = st->fresh != 0;
    const T beta = T(st->beta);
    size_t done = 0;
    if (VEC) {
        constexpr int V = Vec16<T>::N;
        const size_t nv = n / V;
        GRID_STRIDE(i, nv) {
            auto zv = vload(z, i);
            auto pv = vload(p, i);
#pragma unroll
            for (int k = 0; k < V; ++k) el<T>(pv)[k] = first ? el<T>(zv)[k] : el<T>(zv)[k] + beta * el<T>(pv)[k];
            vstore(p, i, pv);
        }
        done = nv * V;
    }
    for (size_t o = done + blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
        p[o] = first ? z[o] : z[o] + beta * p[o];
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(kThreads)
cg_xr_kernel(T* __restrict__ x, T* __restrict__ r, const T* p0, const T* p1, const T* __restrict__ q, size_t n,
             CgState* st, double* red, unsigned int* ticket) {
    if (st->done) return;
    const T* __restrict__ p = st->pbuf ? p0 : p1;   // the direction this iteration wrote
    const T a = T(st->alpha);
    T part = T(0);
    size_t done = 0;
    if (VEC) {
        constexpr int V = Vec16<T>::N;
        const size_t nv = n / V;
        GRID_STRIDE(i, nv) {
            auto xv = vload<T>(x, i);
            auto rv = vload<T>(r, i);
            const auto pv = vload(p, i);
            const auto qv = vload(q, i);
#pragma unroll
            for (int k = 0; k < V; ++k) {
                el<T>(xv)[k] += a * el<T>(const_cast<typename Vec16<T>::type&>(pv))[k];
                const T rn = el<T>(rv)[k] - a * el<T>(const_cast<typename Vec16<T>::type&>(qv))[k];
                el<T>(rv)[k] = rn;
                part += rn * rn;
            }
            vstore(x, i, xv);
            vstore(r, i, rv);
        }
        done = nv * V;
    }
    for (size_t o = done + blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        x[o] += a * p[o];
        const T rv = r[o] - a * q[o];
        r[o] = rv;
        part += rv * rv;
    }
    double s;
    if (block_reduce_last((double)part, red, ticket, blockIdx.x, gridDim.x, &s) && threadIdx.x == 0) {
        st->rr = s;
        st->iter += 1;
        st->fresh = 0;
        st->pbuf ^= 1;
        st->pending = 0;
        if (!isfinite(s)) {
            st->status = TVD_EBREAKDOWN;
            st->done = 1;
        } else if (s < st->tol2) {
            st->done = 1;
        } else if (st->iter >= st->maxit) {
            st->status = TVD_ENOCONV;
            st->done = 1;
        }
    }
}

// (Re)start the CG on the residual already in r (used by the MIXED refinement):
// rr = ||r||^2, stopping threshold tol2 (absolute). A fresh start also clears
// the iteration count and the recurrences; a resume after a residual
// replacement keeps them, so the search direction carries on.
template <typename T>
__global__ void __launch_bounds__(kThreads)
cg_restart_kernel(const T* __restrict__ r, size_t n, CgState* st, double* red, unsigned int* ticket, double tol2,
                  int maxit, int mode) {
    T part = T(0);
    GRID_STRIDE(o, n) part += r[o] * r[o];
    double s;
    if (block_reduce_last((double)part, red, ticket, blockIdx.x, gridDim.x, &s) && threadIdx.x == 0) {
        st->fresh = mode != 1;
        st->pending = 0;
        if (mode == 0) {
            st->iter = 0;
            st->rho = 0.0;
            st->rho_old = 0.0;
            st->beta = 0.0;
            st->alpha = 0.0;
            st->pq = 0.0;
            st->rr0 = s;
        }
        st->maxit = maxit;
        st->rr = s;
        st->tol2 = tol2;
        st->status = TVD_OK;
        st->done = 0;
        if (!isfinite(s)) {
            st->status = TVD_EBREAKDOWN;
            st->done = 1;
        } else if (s < tol2 || st->iter >= maxit) {
            st->done = 1;
        }
    }
}

// r = b - hx - alpha L(w) x (L_AR on a REBLUR_ARL plan) and ||r||^2 (double): the FP-step residual when
// hx = H^T H x is already known.
__global__ void __launch_bounds__(kThreads)
residual_lx_kernel(const double* __restrict__ b, const double* __restrict__ hx, const double* __restrict__ w,
                   const double* __restrict__ x, double alpha, double* __restrict__ r, int nr, int nc, double* out,
                   double* red, unsigned int* ticket, int arl) {
    const size_t n = (size_t)nr * nc;
    double part = 0.0;
    GRID_STRIDE(o, n) {
        const int i = (int)(o / nc), j = (int)(o - (size_t)i * nc);
        const double l = arl ? lap_at_ar(w, x, i, j, nr, nc) : lap_at(w, x, i, j, nr, nc);
        const double v = b[o] - hx[o] - alpha * l;
        r[o] = v;
        part += v * v;
    }
    double s;
    if (block_reduce_last(part, red, ticket, blockIdx.x, gridDim.x, &s) && threadIdx.x == 0) *out = s;
}

// z = r (I) or z = r / D (diagonal preconditioner), with r^T z and the beta update.
template <typename T>
__global__ void __launch_bounds__(kThreads)
cg_simple_precond_kernel(const T* __restrict__ r, const T* __restrict__ dinv, T* __restrict__ z, size_t n,
                         CgState* st, double* red, unsigned int* ticket) {
    if (st && st->done) return;
    T part = T(0);
    GRID_STRIDE(o, n) {
        const T v = dinv ? r[o] * dinv[o] : r[o];
        if (z != r) z[o] = v;
        part += r[o] * v;
    }
    if (!st) return;
    double s;
    if (block_reduce_last((double)part, red, ticket, blockIdx.x, gridDim.x, &s) && threadIdx.x == 0) {
        st->rho_old = st->rho;
        st->rho = s;
        if (!(isfinite(s) && s > 0.0)) {
            st->status = TVD_EBREAKDOWN;
            st->done = 1;
            st->beta = 0.0;
        } else {
            st->beta = st->fresh ? 0.0 : s / st->rho_old;
        }
    }
}

template <typename T>
tvd_status cg_init(const tvd_plan_s& p, const T* b, const T* ax, T* r, CgState* st, double tol, int maxit,
                   cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<T>(PROF_CG_INIT), s);
    cg_init_kernel<T><<<red_blocks(n), kThreads, 0, s>>>(b, ax, r, n, st, p.red, p.ticket + 0, tol, maxit);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

template <typename T>
tvd_status cg_pupdate(const tvd_plan_s& p, const T* z, T* pv, CgState* st, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<T>(PROF_CG_PUPDATE), s);
    if (aligned16(z) && aligned16(pv))
        cg_pupdate_kernel<T, true><<<vec_blocks(n, Vec16<T>::N), kThreads, 0, s>>>(z, pv, n, st);
    else
        cg_pupdate_kernel<T, false><<<red_blocks(n), kThreads, 0, s>>>(z, pv, n, st);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

template <typename T>
tvd_status cg_xrupdate(const tvd_plan_s& p, T* x, T* r, const T* p0, const T* p1, const T* q, CgState* st,
                       cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<T>(PROF_CG_XR), s);
    if (aligned16(x) && aligned16(r) && aligned16(p0) && aligned16(p1) && aligned16(q))
        cg_xr_kernel<T, true><<<vec_blocks(n, Vec16<T>::N), kThreads, 0, s>>>(x, r, p0, p1, q, n, st, p.red, p.ticket + 3);
    else
        cg_xr_kernel<T, false><<<red_blocks(n), kThreads, 0, s>>>(x, r, p0, p1, q, n, st, p.red, p.ticket + 3);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

template <typename T>
tvd_status cg_simple_precond(const tvd_plan_s& p, const T* r, const T* dinv, T* z, CgState* st, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<T>(PROF_CG_SIMPLE), s);
    cg_simple_precond_kernel<T><<<red_blocks(n), kThreads, 0, s>>>(r, dinv, z, n, st, p.red, p.ticket + 4);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

// ---------------------------------------------------------------- double helpers

__global__ void __launch_bounds__(kThreads)
residual_kernel(const double* __restrict__ b, const double* __restrict__ ax, double* __restrict__ r, size_t n,
                double* out, double* red, unsigned int* ticket) {
    double part = 0.0;
    GRID_STRIDE(o, n) {
        const double v = b[o] - ax[o];
        r[o] = v;
        part += v * v;
    }
    double s;
    if (block_reduce_last(part, red, ticket, blockIdx.x, gridDim.x, &s) && threadIdx.x == 0) *out = s;
}

__global__ void __launch_bounds__(kThreads)
diffnorm_kernel(const double* __restrict__ a, const double* __restrict__ b, size_t n, double* out, double* red,
                unsigned int* ticket) {
    double part = 0.0;
    GRID_STRIDE(o, n) {
        const double v = b ? a[o] - b[o] : a[o];
        part += v * v;
    }
    double s;
    if (block_reduce_last(part, red, ticket, blockIdx.x, gridDim.x, &s) && threadIdx.x == 0) *out = s;
}

// sum over pixels of psi = sqrt(|D u|^2 + beta^2) (forward differences, zero
// on the last row / column): the TV term of the functional of eq. (mp).
__global__ void __launch_bounds__(kThreads)
tv_sum_kernel(const double* __restrict__ u, int nr, int nc, double beta2, double* out, double* red,
              unsigned int* ticket) {
    const size_t n = (size_t)nr * nc;
    double part = 0.0;
    GRID_STRIDE(o, n) {
        const int i = (int)(o / nc), j = (int)(o - (size_t)i * nc);
        const double uc = u[o];
        const double dr = i < nr - 1 ? u[o + nc] - uc : 0.0;
        const double dc = j < nc - 1 ? u[o + 1] - uc : 0.0;
        part += sqrt(dr * dr + dc * dc + beta2);
    }
    double s;
    if (block_reduce_last(part, red, ticket, blockIdx.x, gridDim.x, &s) && threadIdx.x == 0) *out = s;
}

// out = x0 + t d and ||out||^2 (double).
__global__ void __launch_bounds__(kThreads)
axpy_to_kernel(const double* __restrict__ x0, const double* __restrict__ d, double t, double* __restrict__ out,
               size_t n, double* norm2, double* red, unsigned int* ticket) {
    double part = 0.0;
    GRID_STRIDE(o, n) {
        const double v = x0[o] + t * d[o];
        out[o] = v;
        part += v * v;
    }
    double s;
    if (block_reduce_last(part, red, ticket, blockIdx.x, gridDim.x, &s) && threadIdx.x == 0) *norm2 = s;
}

__global__ void cast_d2f_kernel(const double* __restrict__ a, float* __restrict__ b, size_t n, double scale) {
    GRID_STRIDE(o, n) b[o] = (float)(a[o] * scale);
}
__global__ void axpy_f2d_kernel(double* __restrict__ x, const float* __restrict__ d, size_t n, double scale) {
    GRID_STRIDE(o, n) x[o] += (double)d[o] * scale;
}
__global__ void copy_f_kernel(const float* __restrict__ a, float* __restrict__ b, size_t n) {
    GRID_STRIDE(o, n) b[o] = a[o];
}
__global__ void fill_zero_f_kernel(float* __restrict__ a, size_t n) {
    GRID_STRIDE(o, n) a[o] = 0.0f;
}

template <typename T>
tvd_status cg_restart(const tvd_plan_s& p, const T* r, CgState* st, double tol2, int maxit, int mode,
                      cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<T>(PROF_CG_INIT), s);
    cg_restart_kernel<T><<<red_blocks(n), kThreads, 0, s>>>(r, n, st, p.red, p.ticket + 6, tol2, maxit, mode);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

__global__ void cg_loop_arm_kernel(CgState* st, int budget) {
    st->loops = 0;
    st->loop_budget = budget;
}

// One thread, launched after the chunk's last kernel has completed (plain
// stream order, no programmatic overlap), so it reads the final state.
__global__ void cg_loop_cond_kernel(cudaGraphConditionalHandle h, CgState* st) {
    const int k = st->loops + 1;
    st->loops = k;
    cudaGraphSetConditional(h, (!st->done && k < st->loop_budget) ? 1u : 0u);
}

tvd_status cg_loop_arm(CgState* st, int budget, cudaStream_t s) {
    ProfScope prof(PROF_MISC, s);
    cg_loop_arm_kernel<<<1, 1, 0, s>>>(st, budget);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

tvd_status cg_loop_cond(cudaGraphConditionalHandle h, CgState* st, cudaStream_t s) {
    ProfScope prof(PROF_MISC, s);
    cg_loop_cond_kernel<<<1, 1, 0, s>>>(h, st);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

tvd_status residual_lx(const tvd_plan_s& p, const double* b, const double* hx, const double* w, const double* x,
                       double alpha, double* r, double* out_norm2, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<double>(PROF_MISC), s);
    residual_lx_kernel<<<red_blocks(n), kThreads, 0, s>>>(b, hx, w, x, alpha, r, p.nr, p.nc, out_norm2, p.red,
                                                          p.ticket + 5, p.method == TVD_METHOD_REBLUR_ARL);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

tvd_status residual_d(const tvd_plan_s& p, const double* b, const double* ax, double* r, double* out_norm2,
                      cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<double>(PROF_MISC), s);
    residual_kernel<<<red_blocks(n), kThreads, 0, s>>>(b, ax, r, n, out_norm2, p.red, p.ticket + 5);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

tvd_status norm2_d(const tvd_plan_s& p, const double* a, double* out, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<double>(PROF_MISC), s);
    diffnorm_kernel<<<red_blocks(n), kThreads, 0, s>>>(a, nullptr, n, out, p.red, p.ticket + 5);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

tvd_status diffnorm2_d(const tvd_plan_s& p, const double* a, const double* b, double* out, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<double>(PROF_MISC), s);
    diffnorm_kernel<<<red_blocks(n), kThreads, 0, s>>>(a, b, n, out, p.red, p.ticket + 5);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

tvd_status tv_sum_d(const tvd_plan_s& p, const double* u, double beta, double* out, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<double>(PROF_MISC), s);
    tv_sum_kernel<<<red_blocks(n), kThreads, 0, s>>>(u, p.nr, p.nc, beta * beta, out, p.red, p.ticket + 5);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

tvd_status axpy_to_d(const tvd_plan_s& p, const double* x0, const double* d, double t, double* out, double* norm2,
                     cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<double>(PROF_MISC), s);
    axpy_to_kernel<<<red_blocks(n), kThreads, 0, s>>>(x0, d, t, out, n, norm2, p.red, p.ticket + 5);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

tvd_status cast_d2f(const double* a, float* b, size_t n, cudaStream_t s, double scale) {
    ProfScope prof(PROF_MISC, s);
    cast_d2f_kernel<<<red_blocks(n), kThreads, 0, s>>>(a, b, n, scale);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

tvd_status axpy_f2d(double* x, const float* d, size_t n, cudaStream_t s, double scale) {
    ProfScope prof(PROF_MISC, s);
    axpy_f2d_kernel<<<red_blocks(n), kThreads, 0, s>>>(x, d, n, scale);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

tvd_status copy_f(const float* a, float* b, size_t n, cudaStream_t s) {
    ProfScope prof(PROF_MISC, s);
    copy_f_kernel<<<red_blocks(n), kThreads, 0, s>>>(a, b, n);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

tvd_status fill_zero_f(float* a, size_t n, cudaStream_t s) {
    ProfScope prof(PROF_MISC, s);
    fill_zero_f_kernel<<<red_blocks(n), kThreads, 0, s>>>(a, n);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

#define INST(T)                                                                                                  \
    template tvd_status cg_init<T>(const tvd_plan_s&, const T*, const T*, T*, CgState*, double, int, cudaStream_t); \
    template tvd_status cg_pupdate<T>(const tvd_plan_s&, const T*, T*, CgState*, cudaStream_t);                  \
    template tvd_status cg_xrupdate<T>(const tvd_plan_s&, T*, T*, const T*, const T*, const T*, CgState*,        \
                                       cudaStream_t);                                                           \
    template tvd_status cg_simple_precond<T>(const tvd_plan_s&, const T*, const T*, T*, CgState*, cudaStream_t); \
    template tvd_status cg_restart<T>(const tvd_plan_s&, const T*, CgState*, double, int, int, cudaStream_t);
INST(float)
INST(double)

}  // namespace tvd
