// Device helpers shared by the kernels: deterministic block reductions with a
// last-block finisher, and the CG scalar finishers.
#pragma once

#include "tvd_internal.cuh"

#include <cstdlib>
#include <mutex>

namespace tvd {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum in a fixed order; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    double s = 0.0;
    if (wid == 0) {
        s = lane < nw ? ws[lane] : 0.0;
        s = warp_sum(s);
    }
    return s;
}

// Writes this block's partial into red[slot]; the last block to arrive (over
// `total` blocks, possibly spread over several kernels that share `ticket`)
// sums red[0..total) in a fixed order and returns true with the sum in *out
// (thread 0 only). The ticket is reset for the next use.
__device__ __forceinline__ bool block_reduce_last(double v, double* red, unsigned int* ticket, int slot,
                                                   int total, double* out) {
    __shared__ bool s_last;
    double b = block_sum(v);
    if (threadIdx.x == 0) {
        red[slot] = b;
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        s_last = (t == (unsigned int)(total - 1));
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    // fixed order: thread t sums slots t, t + blockDim, ... (independent loads
    // that bypass L1), then the block's fixed reduction tree
    double acc = 0.0;
    for (int i = threadIdx.x; i < total; i += blockDim.x) acc += __ldcg(red + i);
    acc = block_sum(acc);
    if (threadIdx.x == 0) {
        *out = acc;
        *ticket = 0u;
    }
    return true;
}

// (L(w) p)_{ij}, 5-point stencil of D_r^T W D_r + D_c^T W D_c (zero Neumann).
template <typename T>
__device__ __forceinline__ T lap_at(const T* __restrict__ w, const T* __restrict__ p, int i, int j, int nr, int nc) {
    const size_t o = (size_t)i * nc + j;
    const T pc = p[o];
    const T wc = w[o];
    T acc = T(0);
    if (i < nr - 1) acc += wc * (pc - p[o + nc]);
    if (j < nc - 1) acc += wc * (pc - p[o + 1]);
    if (i > 0) acc += w[o - nc] * (pc - p[o - nc]);
    if (j > 0) acc += w[o - 1] * (pc - p[o - 1]);
    return acc;
}

// (L_AR p)_ij: the same stencil with anti-reflective BCs (L with AR BCs, the remark
// after eq. (scalereb)): on the first and last line of an axis the AR extension
// makes that axis's two differences and weights equal, so the axis adds nothing there.
template <typename T>
__device__ __forceinline__ T lap_at_ar(const T* __restrict__ w, const T* __restrict__ p, int i, int j, int nr,
                                       int nc) {
    const size_t o = (size_t)i * nc + j;
    const T pc = p[o];
    const T wc = w[o];
    T acc = T(0);
    if (i > 0 && i < nr - 1) acc += wc * (pc - p[o + nc]) + w[o - nc] * (pc - p[o - nc]);
    if (j > 0 && j < nc - 1) acc += wc * (pc - p[o + 1]) + w[o - 1] * (pc - p[o - 1]);
    return acc;
}

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum,
// once per kernel and device (a function attribute is per device), so no
// attribute call repeats while a graph is captured.
constexpr int kMaxDevices = 64;

template <auto Kernel>
inline cudaError_t allow_max_smem() {
    static std::mutex mu;
    static bool done[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, Kernel);
    // the opt-in maximum covers static and dynamic shared memory together
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

// Asynchronous global -> shared copy of one element (cp.async, 4 or 8 bytes);
// many such copies stay in flight per thread until cp_async_wait_all().
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async element size");
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

// Programmatic dependent launch (the CG iteration's kernels): a kernel first
// lets the next kernel in the stream be scheduled (its blocks become resident
// as this kernel's blocks retire), stages what no earlier kernel writes
// (constant tables), and waits for the previous kernel to complete before it
// reads or writes anything that kernel touches. Without a programmatic
// launch both instructions return at once.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with programmatic stream serialisation (see pdl_wait).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    // TVD_PDL=0 launches without the programmatic dependency (tuning / comparison)
    static const bool on = []() {
        const char* v = std::getenv("TVD_PDL");
        return !(v && v[0] == '0');
    }();
    cfg.numAttrs = on ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// End of a CG product q = A p: p^T q, the step alpha = rho / p^T q, and the
// pending x / r update (applied by the next iteration's first pass).
__device__ __forceinline__ void finish_pq(CgState* st, double pq) {
    st->pq = pq;
    if (!finite_pos(pq)) {
        st->status = TVD_EBREAKDOWN;
        st->done = 1;
        st->alpha = 0.0;
    } else {
        st->alpha = st->rho / pq;
        st->pending = 1;
    }
}

// End of a preconditioner solve on the CG path: rho = r^T z and the
// Fletcher-Reeves coefficient beta = rho / rho_old.
__device__ __forceinline__ void finish_rho(CgState* st, double rho) {
    st->rho_old = st->rho;
    st->rho = rho;
    if (!(isfinite(rho) && rho > 0.0)) {
        st->status = TVD_EBREAKDOWN;
        st->done = 1;
        st->beta = 0.0;
        return;
    }
    st->beta = st->fresh ? 0.0 : rho / st->rho_old;
}

// End of a CG iteration (the x / r update applied by the next row pass): the
// residual norm, the iteration count and the stopping test ||r|| / ||r_0|| < tol.
__device__ __forceinline__ void finish_xr(CgState* st, double rr) {
    st->rr = rr;
    st->iter += 1;
    st->fresh = 0;
    st->pbuf ^= 1;
    st->pending = 0;
    if (!isfinite(rr)) {
        st->status = TVD_EBREAKDOWN;
        st->done = 1;
    } else if (rr < st->tol2) {
        st->done = 1;
    } else if (st->iter >= st->maxit) {
        st->status = TVD_ENOCONV;
        st->done = 1;
    }
}

}  // namespace tvd
