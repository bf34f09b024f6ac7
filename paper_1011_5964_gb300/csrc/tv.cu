// Lagged-diffusivity TV operator L(u) (Sec. 1, eq. (el)) and the diagonal
// scaling D = I + alpha diag(L(u)) of eq. (D).
//
// Discretisation: forward differences D_r u = u_{i+1,j} - u_{ij},
// D_c u = u_{i,j+1} - u_{ij}, both zero on the last row / column (zero Neumann),
// diffusivity w_ij = (D_r u^2 + D_c u^2 + beta^2)^{-1/2} per pixel, and
// L = D_r^T W D_r + D_c^T W D_c, a symmetric 5-point stencil.
#include "common.cuh"

namespace tvd {

template <typename T>
__global__ void __launch_bounds__(kThreads)
diffusivity_kernel(const T* __restrict__ u, T* __restrict__ w, int nr, int nc, T beta2) {
    const size_t n = (size_t)nr * nc;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(o / nc), j = (int)(o - (size_t)i * nc);
        const T uc = u[o];
        const T dr = i < nr - 1 ? u[o + nc] - uc : T(0);
        const T dc = j < nc - 1 ? u[o + 1] - uc : T(0);
        w[o] = T(1) / sqrt(dr * dr + dc * dc + beta2);
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
diag_scale_kernel(const T* __restrict__ w, T* __restrict__ dmh, T* __restrict__ dinv, int nr, int nc, T alpha,
                  int arl) {
    const size_t n = (size_t)nr * nc;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(o / nc), j = (int)(o - (size_t)i * nc);
        const T wc = w[o];
        T d = T(0);
        if (arl) {   // diag(L_AR): each axis's pair dropped on its first and last line
            if (i > 0 && i < nr - 1) d += wc + w[o - nc];
            if (j > 0 && j < nc - 1) d += wc + w[o - 1];
        } else {
            if (i < nr - 1) d += wc;
            if (j < nc - 1) d += wc;
            if (i > 0) d += w[o - nc];
            if (j > 0) d += w[o - 1];
        }
        const T D = T(1) + alpha * d;
        dmh[o] = T(1) / sqrt(D);
        dinv[o] = T(1) / D;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
tv_apply_kernel(const T* __restrict__ w, const T* __restrict__ x, T* __restrict__ y, int nr, int nc, int arl) {
    const size_t n = (size_t)nr * nc;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(o / nc), j = (int)(o - (size_t)i * nc);
        y[o] = arl ? lap_at_ar(w, x, i, j, nr, nc) : lap_at(w, x, i, j, nr, nc);
    }
}

// y -= alpha (L - L_AR) x on the border lines (the only pixels where they differ): turns a
// product with L, fused elsewhere, into one with L_AR.
template <typename T>
__global__ void __launch_bounds__(kThreads)
lar_border_kernel(const T* __restrict__ w, const T* __restrict__ x, T* __restrict__ y, int nr, int nc, T alpha) {
    // border pixels in order: row 0, row nr-1 (if nr > 1), then columns 0 and nc-1 of rows 1..nr-2
    const int nrow = nr > 1 ? 2 * nc : nc, ncol = nr > 2 ? 2 * (nr - 2) : 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nrow + ncol; k += gridDim.x * blockDim.x) {
        int i, j;
        if (k < nrow) {
            i = k < nc ? 0 : nr - 1;
            j = k < nc ? k : k - nc;
        } else {
            const int q = k - nrow;
            i = 1 + (q >> 1);
            j = (q & 1) ? nc - 1 : 0;
        }
        const size_t o = (size_t)i * nc + j;
        y[o] -= alpha * (lap_at(w, x, i, j, nr, nc) - lap_at_ar(w, x, i, j, nr, nc));
    }
}

static int ew_blocks(size_t n) {
    size_t b = (n + 4 * kThreads - 1) / (4 * kThreads);
    const size_t cap = (size_t)num_sms() * 32;
    return (int)(b < cap ? (b ? b : 1) : cap);
}

template <typename T>
tvd_status diffusivity(const tvd_plan_s& p, const T* u, double beta, T* w, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<T>(PROF_TV), s);
    diffusivity_kernel<T><<<ew_blocks(n), kThreads, 0, s>>>(u, w, p.nr, p.nc, T(beta * beta));
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

template <typename T>
tvd_status diag_scale(const tvd_plan_s& p, const T* w, double alpha, T* dmh, T* dinv, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<T>(PROF_TV), s);
    diag_scale_kernel<T><<<ew_blocks(n), kThreads, 0, s>>>(w, dmh, dinv, p.nr, p.nc, T(alpha),
                                                           p.method == TVD_METHOD_REBLUR_ARL);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

template <typename T>
tvd_status tv_apply(const tvd_plan_s& p, const T* w, const T* x, T* y, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    ProfScope prof(prof_class<T>(PROF_TV), s);
    tv_apply_kernel<T><<<ew_blocks(n), kThreads, 0, s>>>(w, x, y, p.nr, p.nc, p.method == TVD_METHOD_REBLUR_ARL);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

template <typename T>
tvd_status lar_border(const tvd_plan_s& p, const T* w, const T* x, T* y, double alpha, cudaStream_t s) {
    const int nb = (p.nr > 1 ? 2 * p.nc : p.nc) + (p.nr > 2 ? 2 * (p.nr - 2) : 0);
    ProfScope prof(prof_class<T>(PROF_TV), s);
    lar_border_kernel<T><<<(nb + kThreads - 1) / kThreads, kThreads, 0, s>>>(w, x, y, p.nr, p.nc, T(alpha));
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

template tvd_status diffusivity<float>(const tvd_plan_s&, const float*, double, float*, cudaStream_t);
template tvd_status diffusivity<double>(const tvd_plan_s&, const double*, double, double*, cudaStream_t);
template tvd_status diag_scale<float>(const tvd_plan_s&, const float*, double, float*, float*, cudaStream_t);
template tvd_status diag_scale<double>(const tvd_plan_s&, const double*, double, double*, double*, cudaStream_t);
template tvd_status tv_apply<float>(const tvd_plan_s&, const float*, const float*, float*, cudaStream_t);
template tvd_status tv_apply<double>(const tvd_plan_s&, const double*, const double*, double*, cudaStream_t);
template tvd_status lar_border<float>(const tvd_plan_s&, const float*, const float*, float*, double, cudaStream_t);
template tvd_status lar_border<double>(const tvd_plan_s&, const double*, const double*, double*, double,
                                       cudaStream_t);

}  // namespace tvd
