// Adjoint of the converged fixed point: the TV Hessian operator and the
// gradients of a loss of u* with respect to alpha, beta and the PSF taps.
//
// At the fixed point of the lagged-diffusivity iteration the Euler-Lagrange
// residual F(u, theta) = H^T (H u - v) + alpha grad J_beta(u) of eq. (el)
// vanishes, with J_beta(u) = sum_pq psi_pq, psi = sqrt(|D u|^2 + beta^2) and
// D the forward differences of L (zero on the last row / column). Its
// Jacobian J = H^T H + alpha nabla^2 J_beta(u) is SPD, and for a loss l(u*)
// with J lambda = dl/du:
//   dl/dalpha = -lambda^T L(u) u,
//   dl/dbeta  = alpha beta (D lambda)^T [psi^-3 D u],
//   dl/dh_ab  = -[ (E_ab lambda)^T (H u - v) + (H lambda)^T (E_ab u) ],
// E_ab x being x's BC extension shifted by the tap offset (a, b).
#include "common.cuh"

#include <algorithm>

namespace tvd {

static int adj_blocks(size_t n) {
    size_t b = (n + 4 * kThreads - 1) / (4 * kThreads);
    const size_t cap = (size_t)num_sms() * 32;
    if (b > cap) b = cap;
    return (int)std::max<size_t>(b, 1);
}

// Per cell: g = (d_r u, d_c u) psi^-3/2, with w = psi^-1 (the diffusivity).
__global__ void __launch_bounds__(kThreads)
hess_coef_kernel(const double* __restrict__ u, const double* __restrict__ w, double* __restrict__ gr,
                 double* __restrict__ gc, int nr, int nc) {
    const size_t n = (size_t)nr * nc;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(o / nc), j = (int)(o - (size_t)i * nc);
        const double uo = u[o];
        const double dr = i < nr - 1 ? u[o + nc] - uo : 0.0;
        const double dc = j < nc - 1 ? u[o + 1] - uo : 0.0;
        const double s = w[o] * sqrt(w[o]);
        gr[o] = dr * s;
        gc[o] = dc * s;
    }
}

// a = psi^-1 D x - psi^-3 (D u . D x) D u on the cell (i, j) = w Dx - (g . Dx) g.
template <typename T>
__device__ __forceinline__ void hess_cell(const T* __restrict__ x, const T* __restrict__ w, const T* __restrict__ gr,
                                          const T* __restrict__ gc, int i, int j, int nr, int nc, T& ar, T& ac) {
    const size_t o = (size_t)i * nc + j;
    const T xo = x[o];
    const T xr = i < nr - 1 ? x[o + nc] - xo : T(0);
    const T xc = j < nc - 1 ? x[o + 1] - xo : T(0);
    const T g1 = gr[o], g2 = gc[o], wo = w[o];
    const T s = g1 * xr + g2 * xc;
    ar = wo * xr - s * g1;
    ac = wo * xc - s * g2;
}

// (nabla^2 J_beta x)_ij = (D_r^T a_r + D_c^T a_c)_ij
template <typename T>
__device__ __forceinline__ T hess_at(const T* __restrict__ x, const T* __restrict__ w, const T* __restrict__ gr,
                                     const T* __restrict__ gc, int i, int j, int nr, int nc) {
    T ar, ac, y = T(0);
    hess_cell(x, w, gr, gc, i, j, nr, nc, ar, ac);
    if (i < nr - 1) y -= ar;
    if (j < nc - 1) y -= ac;
    if (i > 0) {
        hess_cell(x, w, gr, gc, i - 1, j, nr, nc, ar, ac);
        y += ar;
    }
    if (j > 0) {
        hess_cell(x, w, gr, gc, i, j - 1, nr, nc, ar, ac);
        y += ac;
    }
    return y;
}

__global__ void __launch_bounds__(kThreads)
hess_apply_kernel(const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ w,
                  const double* __restrict__ gr, const double* __restrict__ gc, int nr, int nc) {
    const size_t n = (size_t)nr * nc;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(o / nc), j = (int)(o - (size_t)i * nc);
        y[o] = hess_at(x, w, gr, gc, i, j, nr, nc);
    }
}

// CG product of the adjoint solve: q (= H^T H p) += alpha nabla^2 J_beta p, then p^T q.
template <typename T>
__global__ void __launch_bounds__(kThreads)
hess_add_kernel(T* __restrict__ q, const T* p0, const T* p1, const T* __restrict__ w, const T* __restrict__ gr,
                const T* __restrict__ gc, double alpha, int nr, int nc, CgState* st, double* red,
                unsigned int* ticket) {
    if (st->done) return;
    const T* __restrict__ pv = st->pbuf ? p0 : p1;   // the direction this iteration wrote
    const size_t n = (size_t)nr * nc;
    const T al = T(alpha);
    T part = T(0);
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(o / nc), j = (int)(o - (size_t)i * nc);
        const T qn = q[o] + al * hess_at(pv, w, gr, gc, i, j, nr, nc);
        q[o] = qn;
        part += pv[o] * qn;
    }
    double sum;
    if (block_reduce_last((double)part, red, ticket, blockIdx.x, gridDim.x, &sum) && threadIdx.x == 0)
        finish_pq(st, sum);
}

// Double residual of the adjoint system: r = b - hq - alpha nabla^2 J_beta x (hq = H^T H x), ||r||^2.
__global__ void __launch_bounds__(kThreads)
adj_residual_kernel(const double* __restrict__ b, const double* __restrict__ hq, const double* __restrict__ w,
                    const double* __restrict__ gr, const double* __restrict__ gc, const double* __restrict__ x,
                    double alpha, double* __restrict__ r, int nr, int nc, double* red, unsigned int* ticket,
                    double* out) {
    const size_t n = (size_t)nr * nc;
    double part = 0.0;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(o / nc), j = (int)(o - (size_t)i * nc);
        const double v = b[o] - hq[o] - alpha * hess_at(x, w, gr, gc, i, j, nr, nc);
        r[o] = v;
        part += v * v;
    }
    double sum;
    if (block_reduce_last(part, red, ticket, blockIdx.x, gridDim.x, &sum) && threadIdx.x == 0) *out = sum;
}

// sum_cells psi^-3 (D lambda . D u), psi^-3 = w^3
__global__ void __launch_bounds__(kThreads)
beta_sum_kernel(const double* __restrict__ lam, const double* __restrict__ u, const double* __restrict__ w, int nr,
                int nc, double* red, unsigned int* ticket, double* out) {
    const size_t n = (size_t)nr * nc;
    double part = 0.0;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(o / nc), j = (int)(o - (size_t)i * nc);
        const double wo = w[o];
        double d = 0.0;
        if (i < nr - 1) d += (lam[o + nc] - lam[o]) * (u[o + nc] - u[o]);
        if (j < nc - 1) d += (lam[o + 1] - lam[o]) * (u[o + 1] - u[o]);
        part += wo * wo * wo * d;
    }
    double sum;
    if (block_reduce_last(part, red, ticket, blockIdx.x, gridDim.x, &sum) && threadIdx.x == 0) *out = sum;
}

__global__ void __launch_bounds__(kThreads)
dot_kernel(const double* __restrict__ a, const double* __restrict__ b, size_t n, double* red, unsigned int* ticket,
           double* out) {
    double part = 0.0;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
        part += a[o] * b[o];
    double sum;
    if (block_reduce_last(part, red, ticket, blockIdx.x, gridDim.x, &sum) && threadIdx.x == 0) *out = sum;
}

__global__ void __launch_bounds__(kThreads)
sub_kernel(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c, size_t n) {
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
        c[o] = a[o] - b[o];
}

// One BC rule per axis: the extended index t of a length-n axis is
// sum_k c_k x[idx_k] (AR: x_{-s} = 2 x_0 - x_s, eq. (anti1d); R: x_{-s} = x_{s-1});
// the 2D extension is the product of the two axes' rules.
__device__ __forceinline__ int ext_rule(int t, int n, bool ar, int* idx, double* c) {
    if (t >= 0 && t < n) {
        idx[0] = t;
        c[0] = 1.0;
        return 1;
    }
    if (ar) {
        idx[0] = t < 0 ? 0 : n - 1;
        c[0] = 2.0;
        idx[1] = t < 0 ? -t : 2 * (n - 1) - t;
        c[1] = -1.0;
        return 2;
    }
    idx[0] = t < 0 ? -t - 1 : 2 * n - 1 - t;
    c[0] = 1.0;
    return 1;
}

// xe[(I + mr) * (nc + 2 mc) + (J + mc)] = extended x at (I, J), |I + ...| within one mirror.
__global__ void __launch_bounds__(kThreads)
extend_kernel(const double* __restrict__ x, double* __restrict__ xe, int nr, int nc, int mr, int mc, int ar) {
    const int We = nc + 2 * mc, He = nr + 2 * mr;
    const size_t n = (size_t)We * He;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int I = (int)(o / We) - mr, J = (int)(o % We) - mc;
        int ri[2], ci[2];
        double rc[2], cc[2];
        const int kr = ext_rule(I, nr, ar != 0, ri, rc), kc = ext_rule(J, nc, ar != 0, ci, cc);
        double v = 0.0;
        for (int s = 0; s < kr; ++s)
            for (int t = 0; t < kc; ++t) v += rc[s] * cc[t] * x[(size_t)ri[s] * nc + ci[t]];
        xe[o] = v;
    }
}

// One block per tap (a, b): out = -sum_ij [ lam~(i-a, j-b) res_ij + u~(i-a, j-b) hlam_ij ].
__global__ void __launch_bounds__(kThreads)
psf_tap_kernel(const double* __restrict__ lame, const double* __restrict__ ue, const double* __restrict__ res,
               const double* __restrict__ hlam, int nr, int nc, int mr, int mc, double* __restrict__ out) {
    const int pc = 2 * mc + 1;
    const int a = (int)blockIdx.x / pc - mr, b = (int)blockIdx.x % pc - mc;
    const int We = nc + 2 * mc;
    const size_t n = (size_t)nr * nc;
    double part = 0.0;
    for (size_t o = threadIdx.x; o < n; o += blockDim.x) {
        const int i = (int)(o / nc), j = (int)(o - (size_t)i * nc);
        const size_t e = (size_t)(i - a + mr) * We + (j - b + mc);
        part += lame[e] * res[o] + ue[e] * hlam[o];
    }
    const double sum = block_sum(part);
    if (threadIdx.x == 0) out[blockIdx.x] = -sum;
}

// ------------------------------------------------------------- launchers

tvd_status hess_coef(const tvd_plan_s& p, const double* u, const double* w, double* gr, double* gc,
                     cudaStream_t s) {
    ProfScope prof(prof_class<double>(PROF_TV), s);
    hess_coef_kernel<<<adj_blocks((size_t)p.nr * p.nc), kThreads, 0, s>>>(u, w, gr, gc, p.nr, p.nc);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

tvd_status hess_apply(const tvd_plan_s& p, const double* x, double* y, const double* w, const double* gr,
                      const double* gc, cudaStream_t s) {
    ProfScope prof(prof_class<double>(PROF_TV), s);
    hess_apply_kernel<<<adj_blocks((size_t)p.nr * p.nc), kThreads, 0, s>>>(x, y, w, gr, gc, p.nr, p.nc);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

template <typename T>
tvd_status hess_add(const tvd_plan_s& p, T* q, const T* p0, const T* p1, const T* w, const T* gr, const T* gc,
                    double alpha, CgState* st, cudaStream_t s) {
    ProfScope prof(prof_class<T>(PROF_BLUR_ADJ), s);
    hess_add_kernel<T><<<adj_blocks((size_t)p.nr * p.nc), kThreads, 0, s>>>(q, p0, p1, w, gr, gc, alpha, p.nr, p.nc,
                                                                            st, p.red, p.ticket + 8);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}
template tvd_status hess_add<float>(const tvd_plan_s&, float*, const float*, const float*, const float*,
                                    const float*, const float*, double, CgState*, cudaStream_t);
template tvd_status hess_add<double>(const tvd_plan_s&, double*, const double*, const double*, const double*,
                                     const double*, const double*, double, CgState*, cudaStream_t);

tvd_status adj_residual(const tvd_plan_s& p, const double* b, const double* hq, const double* w, const double* gr,
                        const double* gc, const double* x, double alpha, double* r, double* out_norm2,
                        cudaStream_t s) {
    ProfScope prof(prof_class<double>(PROF_MISC), s);
    adj_residual_kernel<<<adj_blocks((size_t)p.nr * p.nc), kThreads, 0, s>>>(b, hq, w, gr, gc, x, alpha, r, p.nr,
                                                                             p.nc, p.red, p.ticket + 9, out_norm2);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

tvd_status adjoint_gradients(const tvd_plan_s& p, const Ops<double>& o, const double* lam, const double* u,
                             const double* v, double alpha, double beta, double* scratch_ext, double* taps,
                             double* out2, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    const int nb = adj_blocks(n);
    ProfScope prof(prof_class<double>(PROF_MISC), s, taps ? 6 : 2);
    // dl/dalpha = -lambda^T L(u) u (the negation is applied by the caller)
    TVD_TRY(tv_apply<double>(p, o.w, u, o.t, s));
    dot_kernel<<<nb, kThreads, 0, s>>>(lam, o.t, n, p.red, p.ticket + 9, out2);
    TVD_CUDA_TRY(cudaGetLastError());
    // dl/dbeta = alpha beta sum psi^-3 (D lambda . D u)
    beta_sum_kernel<<<nb, kThreads, 0, s>>>(lam, u, o.w, p.nr, p.nc, p.red, p.ticket + 9, out2 + 1);
    TVD_CUDA_TRY(cudaGetLastError());
    (void)alpha;
    (void)beta;
    if (!taps) return TVD_OK;
    // dl/dh: res = H u - v, H lambda, the extended lambda and u
    const int mr = p.psf.mr, mc = p.psf.mc;
    const size_t ne = (size_t)(p.nr + 2 * mr) * (p.nc + 2 * mc);
    TVD_TRY(blur_apply<double>(p, o, false, u, o.t, s));
    sub_kernel<<<nb, kThreads, 0, s>>>(o.t, v, o.t, n);
    TVD_CUDA_TRY(cudaGetLastError());
    TVD_TRY(blur_apply<double>(p, o, false, lam, o.q, s));
    const int ar = p.bc == TVD_BC_ANTIREFLECTIVE ? 1 : 0;
    extend_kernel<<<adj_blocks(ne), kThreads, 0, s>>>(lam, scratch_ext, p.nr, p.nc, mr, mc, ar);
    extend_kernel<<<adj_blocks(ne), kThreads, 0, s>>>(u, scratch_ext + ne, p.nr, p.nc, mr, mc, ar);
    TVD_CUDA_TRY(cudaGetLastError());
    psf_tap_kernel<<<(2 * mr + 1) * (2 * mc + 1), kThreads, 0, s>>>(scratch_ext, scratch_ext + ne, o.t, o.q, p.nr,
                                                                    p.nc, mr, mc, taps);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

}  // namespace tvd
