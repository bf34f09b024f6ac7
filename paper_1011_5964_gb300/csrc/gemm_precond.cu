// Dense-matrix form of the preconditioner transforms (float plans).
//
// The fast preconditioners of Secs. 2-3 (M, D_M, M_D for AR; R, D_R, R_D for R)
// apply the 2D transform U = B_r (x) B_c, a diagonal, and U^{-1}:
//   z = d o B_r^T [ (B_r (d o r) B_c^T) o (1 / spectrum) ] B_c,   d = D^-1/2 or 1,
// with B = hat-S_n = diag(1, S_{n-2}, 1) (S_m the orthonormal DST-I of
// eq. (lambda), symmetric, an involution) for AR and B = C, the orthonormal
// DCT-II of Sec. 3.1 (B^{-1} = C^T) for R. Here each 1D transform of all
// lines is one matrix product with the n x n matrix B on the tensor cores
// (cuBLASLt; TF32 products of float operands, or, from sides of 1024 on,
// bf16 operands; float accumulation in both), so
// the solve is four GEMMs and three vector kernels instead of the three FFT
// line passes of transform.cu. The preconditioner only shapes the CG
// iteration: its rounding changes the iteration count, not the solution,
// whose accuracy the double residual of the MIXED form decides.
//
// Layout: images are row-major n_r x n_c; cuBLAS is column-major, so the
// row-major X is the column-major X^T and
//   forward  Y^T = B_c X^T B_r^T     (GEMM 1: B_c X^T, GEMM 2: (.) B_r^T)
//   inverse  Z^T = B_c^T Y^T B_r     (GEMM 3: B_c^T Y^T, GEMM 4: (.) B_r)
// with B_r, B_c stored row-major (their column-major views are B^T).
#include "common.cuh"

#include <cublasLt.h>
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace tvd {

// One of the four products with its algorithm, picked at set-up by timing the
// candidates cuBLASLt proposes (the n^3 products of one image fill few SMs at
// n = 1024 with the default tiles; split-K / stream-K variants can fill more).
struct LtGemm {
    cublasLtMatmulDesc_t op = nullptr;
    cublasLtMatrixLayout_t a = nullptr, b = nullptr, c = nullptr;
    cublasLtMatmulAlgo_t algo{};
    bool tuned = false;
    float us = 0.0f;      // measured time of the chosen algorithm
};

struct GemmPrecond {
    cublasHandle_t h = nullptr;
    cublasLtHandle_t lt = nullptr;
    LtGemm g[4];
    cublasComputeType_t ct = CUBLAS_COMPUTE_32F_FAST_TF32;
    // operand storage: float (TF32 products by default), or bf16 (TVD_GEMM_STORAGE=bf16: the matrices
    // and the inputs of each product rounded to bf16, float accumulation, float outputs of the
    // column products)
    bool bf = false;
    void* Br = nullptr;      // n_r x n_r, row-major, operand type
    void* Bc = nullptr;      // n_c x n_c, row-major, operand type (aliases Br for square images)
    void* in = nullptr;      // n_r x n_c, operand type: input of the row products
    void* mid = nullptr;     // n_r x n_c, operand type: row products' output, column products' input
    float* s1 = nullptr;     // n_r x n_c float: column products' output
    void* ws = nullptr;      // cuBLAS workspace (no allocation inside a captured graph)
    size_t ws_bytes = 0;
};

static constexpr size_t kGemmWorkspace = 32u << 20;
static constexpr int kCandidates = 16;   // cuBLASLt heuristic candidates timed per product

// Row-major n x n matrix of the 1D transform: AR hat-S_n, R the DCT-II C_n
// (frequency by space). Arguments are reduced modulo the period in integers.
static void transform_matrix(int n, tvd_bc bc, std::vector<float>& out) {
    out.assign((size_t)n * n, 0.0f);
    const double pi = 3.14159265358979323846;
    if (bc == TVD_BC_ANTIREFLECTIVE) {
        const int M = n - 1;   // S_{n-2}: sqrt(2/M) sin(k l pi / M), k, l = 1..n-2
        const double sc = std::sqrt(2.0 / M);
        out[0] = 1.0f;
        out[(size_t)n * n - 1] = 1.0f;
        for (int k = 1; k <= n - 2; ++k)
            for (int l = 1; l <= n - 2; ++l) {
                const long long a = ((long long)k * l) % (2LL * M);
                out[(size_t)k * n + l] = (float)(sc * std::sin(pi * (double)a / M));
            }
    } else {
        const double c0 = std::sqrt(1.0 / n), c1 = std::sqrt(2.0 / n);
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j) {
                const long long a = ((long long)k * (2 * j + 1)) % (4LL * n);
                out[(size_t)k * n + j] = (float)((k ? c1 : c0) * std::cos(pi * (double)a / (2.0 * n)));
            }
    }
}

static cublasComputeType_t compute_type_from_env() {
    const char* v = std::getenv("TVD_GEMM_COMPUTE");
    if (!v) return CUBLAS_COMPUTE_32F_FAST_TF32;
    if (!std::strcmp(v, "bf16")) return CUBLAS_COMPUTE_32F_FAST_16BF;
    if (!std::strcmp(v, "bf16x9")) return CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
    if (!std::strcmp(v, "fp32")) return CUBLAS_COMPUTE_32F;
    return CUBLAS_COMPUTE_32F_FAST_TF32;
}

static const char* blas_msg(cublasStatus_t e) {
    switch (e) {
        case CUBLAS_STATUS_NOT_INITIALIZED: return "not initialised";
        case CUBLAS_STATUS_ALLOC_FAILED: return "allocation failed";
        case CUBLAS_STATUS_INVALID_VALUE: return "invalid value";
        case CUBLAS_STATUS_ARCH_MISMATCH: return "architecture mismatch";
        case CUBLAS_STATUS_EXECUTION_FAILED: return "execution failed";
        case CUBLAS_STATUS_NOT_SUPPORTED: return "not supported";
        default: return "error";
    }
}

#define TVD_BLAS_TRY(expr)                                                                       \
    do {                                                                                         \
        cublasStatus_t _b = (expr);                                                              \
        if (_b != CUBLAS_STATUS_SUCCESS) {                                                       \
            ::tvd::set_error(std::string("cuBLAS: ") + blas_msg(_b) + " at " + __FILE__ + ":" + \
                             std::to_string(__LINE__));                                         \
            return TVD_ECUDA;                                                                    \
        }                                                                                        \
    } while (0)

void gemm_precond_destroy(tvd_plan_s& p) {
    auto* g = static_cast<GemmPrecond*>(p.gemm);
    if (!g) return;
    for (auto& q : g->g) {
        if (q.op) cublasLtMatmulDescDestroy(q.op);
        if (q.a) cublasLtMatrixLayoutDestroy(q.a);
        if (q.b) cublasLtMatrixLayoutDestroy(q.b);
        if (q.c) cublasLtMatrixLayoutDestroy(q.c);
    }
    if (g->lt) cublasLtDestroy(g->lt);
    if (g->h) cublasDestroy(g->h);
    if (g->Bc && g->Bc != g->Br) cudaFree(g->Bc);
    if (g->Br) cudaFree(g->Br);
    if (g->in && g->in != (void*)g->s1) cudaFree(g->in);
    if (g->mid) cudaFree(g->mid);
    if (g->s1) cudaFree(g->s1);
    if (g->ws) cudaFree(g->ws);
    delete g;
    p.gemm = nullptr;
}

// Shapes of the four products (column-major m x n x k with the operand
// transposes): forward B_c X^T, (.) B_r^T; inverse B_c^T Y^T, (.) B_r.
struct GemmShape {
    cublasOperation_t ta, tb;
    int m, n, k, lda, ldb;
    bool a_is_mat;   // A operand is B_c (else the image scratch)
};
static GemmShape gemm_shape(int i, int nr, int nc) {
    switch (i) {
        case 0: return {CUBLAS_OP_T, CUBLAS_OP_N, nc, nr, nc, nc, nc, true};
        case 1: return {CUBLAS_OP_N, CUBLAS_OP_N, nc, nr, nr, nc, nr, false};
        case 2: return {CUBLAS_OP_N, CUBLAS_OP_N, nc, nr, nc, nc, nc, true};
        default: return {CUBLAS_OP_N, CUBLAS_OP_T, nc, nr, nr, nc, nr, false};
    }
}

// Time the candidate algorithms of each product (up to kCandidates from the
// heuristic, and their split-K variants) on the plan's buffers and keep the
// fastest (3 timed runs after one warm-up each). Products without a usable
// candidate fall back to cublasGemmEx.
static tvd_status tune_lt(tvd_plan_s& p, GemmPrecond& g, cudaStream_t s) {
    if (cublasLtCreate(&g.lt) != CUBLAS_STATUS_SUCCESS) {
        g.lt = nullptr;
        return TVD_OK;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TVD_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        set_error("cudaEventCreate failed");
        return TVD_ECUDA;
    }
    const size_t esz = g.bf ? sizeof(__nv_bfloat16) : sizeof(float);
    TVD_CUDA_TRY(cudaMemsetAsync(g.in, 0, (size_t)p.nr * p.nc * esz, s));
    TVD_CUDA_TRY(cudaMemsetAsync(g.mid, 0, (size_t)p.nr * p.nc * esz, s));
    const float one = 1.0f, zero = 0.0f;
    for (int i = 0; i < 4; ++i) {
        LtGemm& q = g.g[i];
        const GemmShape sh = gemm_shape(i, p.nr, p.nc);
        const cudaDataType_t ot = g.bf ? CUDA_R_16BF : CUDA_R_32F;
        const cudaDataType_t ct = sh.a_is_mat ? ot : CUDA_R_32F;   // row products feed the column products
        if (cublasLtMatmulDescCreate(&q.op, g.bf ? CUBLAS_COMPUTE_32F : g.ct, CUDA_R_32F) != CUBLAS_STATUS_SUCCESS)
            continue;
        cublasLtMatmulDescSetAttribute(q.op, CUBLASLT_MATMUL_DESC_TRANSA, &sh.ta, sizeof(sh.ta));
        cublasLtMatmulDescSetAttribute(q.op, CUBLASLT_MATMUL_DESC_TRANSB, &sh.tb, sizeof(sh.tb));
        const int ar = sh.ta == CUBLAS_OP_N ? sh.m : sh.k, ac = sh.ta == CUBLAS_OP_N ? sh.k : sh.m;
        const int br = sh.tb == CUBLAS_OP_N ? sh.k : sh.n, bc = sh.tb == CUBLAS_OP_N ? sh.n : sh.k;
        if (cublasLtMatrixLayoutCreate(&q.a, ot, ar, ac, sh.lda) != CUBLAS_STATUS_SUCCESS ||
            cublasLtMatrixLayoutCreate(&q.b, ot, br, bc, sh.ldb) != CUBLAS_STATUS_SUCCESS ||
            cublasLtMatrixLayoutCreate(&q.c, ct, sh.m, sh.n, sh.m) != CUBLAS_STATUS_SUCCESS)
            continue;
        cublasLtMatmulPreference_t pref = nullptr;
        if (cublasLtMatmulPreferenceCreate(&pref) != CUBLAS_STATUS_SUCCESS) continue;
        const size_t wsb = g.ws_bytes;
        cublasLtMatmulPreferenceSetAttribute(pref, CUBLASLT_MATMUL_PREF_MAX_WORKSPACE_BYTES, &wsb, sizeof(wsb));
        cublasLtMatmulHeuristicResult_t heur[kCandidates];
        int found = 0;
        cublasStatus_t hs =
            cublasLtMatmulAlgoGetHeuristic(g.lt, q.op, q.a, q.b, q.c, q.c, pref, kCandidates, heur, &found);
        cublasLtMatmulPreferenceDestroy(pref);
        if (hs != CUBLAS_STATUS_SUCCESS) continue;
        // each candidate as proposed, plus split-K variants (2, 4, 8 slices of k, reduced in the
        // compute type through the workspace) where the algorithm supports them
        std::vector<cublasLtMatmulHeuristicResult_t> res;
        for (int c = 0; c < found; ++c) {
            if (heur[c].state != CUBLAS_STATUS_SUCCESS) continue;
            res.push_back(heur[c]);
            int32_t splitk = 0;
            uint32_t schemes = 0;
            size_t wr = 0;
            if (cublasLtMatmulAlgoCapGetAttribute(&heur[c].algo, CUBLASLT_ALGO_CAP_SPLITK_SUPPORT, &splitk,
                                                  sizeof(splitk), &wr) != CUBLAS_STATUS_SUCCESS || !splitk)
                continue;
            if (cublasLtMatmulAlgoCapGetAttribute(&heur[c].algo, CUBLASLT_ALGO_CAP_REDUCTION_SCHEME_MASK, &schemes,
                                                  sizeof(schemes), &wr) != CUBLAS_STATUS_SUCCESS ||
                !(schemes & CUBLASLT_REDUCTION_SCHEME_COMPUTE_TYPE))
                continue;
            for (int32_t parts : {2, 4, 8}) {
                cublasLtMatmulHeuristicResult_t v = heur[c];
                const uint32_t scheme = CUBLASLT_REDUCTION_SCHEME_COMPUTE_TYPE;
                if (cublasLtMatmulAlgoConfigSetAttribute(&v.algo, CUBLASLT_ALGO_CONFIG_SPLITK_NUM, &parts,
                                                         sizeof(parts)) != CUBLAS_STATUS_SUCCESS ||
                    cublasLtMatmulAlgoConfigSetAttribute(&v.algo, CUBLASLT_ALGO_CONFIG_REDUCTION_SCHEME, &scheme,
                                                         sizeof(scheme)) != CUBLAS_STATUS_SUCCESS)
                    continue;
                if (cublasLtMatmulAlgoCheck(g.lt, q.op, q.a, q.b, q.c, q.c, &v.algo, &v) != CUBLAS_STATUS_SUCCESS)
                    continue;
                v.state = CUBLAS_STATUS_SUCCESS;
                res.push_back(v);
            }
        }
        const void* A = sh.a_is_mat ? g.Bc : g.mid;
        const void* B = sh.a_is_mat ? g.in : g.Br;
        void* C = sh.a_is_mat ? g.mid : (void*)g.s1;
        float best = 1e30f;
        for (size_t c = 0; c < res.size(); ++c) {
            if (res[c].state != CUBLAS_STATUS_SUCCESS || res[c].workspaceSize > wsb) continue;
            bool ok = true;
            for (int rep = 0; rep < 4 && ok; ++rep) {
                if (rep == 1) ok = cudaEventRecord(e0, s) == cudaSuccess;
                ok = ok && cublasLtMatmul(g.lt, q.op, &one, A, q.a, B, q.b, &zero, C, q.c, C, q.c, &res[c].algo,
                                          g.ws, wsb, s) == CUBLAS_STATUS_SUCCESS;
            }
            ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0.0f;
            if (!ok || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (ms < best) {
                best = ms;
                q.algo = res[c].algo;
                q.tuned = true;
                q.us = ms * 1000.0f / 3.0f;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // TVD_GEMM_VERBOSE=1: the chosen algorithm of each product on stderr
    const char* vb = std::getenv("TVD_GEMM_VERBOSE");
    if (vb && vb[0] == '1') {
        for (int i = 0; i < 4; ++i) {
            int32_t parts = 1;
            size_t wr = 0;
            if (g.g[i].tuned)
                cublasLtMatmulAlgoConfigGetAttribute(&g.g[i].algo, CUBLASLT_ALGO_CONFIG_SPLITK_NUM, &parts,
                                                     sizeof(parts), &wr);
            std::fprintf(stderr, "tvd gemm %dx%d product %d: tuned %d, split-k %d, %.2f us\n", p.nr, p.nc, i,
                         (int)g.g[i].tuned, parts, g.g[i].us);
        }
    }
    return TVD_OK;
}

int gemm_precond_storage(const tvd_plan_s& p) {
    const auto* g = static_cast<const GemmPrecond*>(p.gemm);
    return g ? (g->bf ? 2 : 1) : 0;
}

tvd_status gemm_precond_create(tvd_plan_s& p, cudaStream_t s) {
    if (p.gemm) return TVD_OK;
    auto* g = new GemmPrecond();
    p.gemm = g;
    g->ct = compute_type_from_env();
    auto fail = [&](tvd_status e) {
        gemm_precond_destroy(p);
        return e;
    };
    const size_t n = (size_t)p.nr * p.nc;
    auto alloc = [&](void** ptr, size_t bytes) -> bool {
        if (cudaMalloc(ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc failed for the GEMM transform buffers");
            return false;
        }
        return true;
    };
    // bf16 operands from sides of 1024 on (measured faster there: 1024^2 10.8 -> 12.0, 2048^2 3.6 ->
    // 4.3 deblurs/s; at 512^2 float operands are 2% faster); TVD_GEMM_STORAGE=bf16 / f32 overrides
    const char* sv = std::getenv("TVD_GEMM_STORAGE");
    if (sv && !std::strcmp(sv, "bf16")) g->bf = true;
    else if (sv && !std::strcmp(sv, "f32")) g->bf = false;
    else g->bf = std::min(p.nr, p.nc) >= 1024;
    const size_t esz = g->bf ? sizeof(__nv_bfloat16) : sizeof(float);
    if (!alloc(&g->Br, (size_t)p.nr * p.nr * esz)) return fail(TVD_ENOMEM);
    if (p.nc == p.nr) g->Bc = g->Br;
    else if (!alloc(&g->Bc, (size_t)p.nc * p.nc * esz)) return fail(TVD_ENOMEM);
    if (!alloc((void**)&g->s1, n * sizeof(float)) || !alloc(&g->mid, n * esz)) return fail(TVD_ENOMEM);
    if (g->bf) {
        if (!alloc(&g->in, n * esz)) return fail(TVD_ENOMEM);
    } else {
        g->in = g->s1;   // float storage: the row products read the column products' output buffer
    }
    if (!alloc(&g->ws, kGemmWorkspace)) return fail(TVD_ENOMEM);
    g->ws_bytes = kGemmWorkspace;
    auto upload = [&](int side, void* dst) -> bool {
        std::vector<float> B;
        transform_matrix(side, p.bc, B);
        cudaError_t e;
        if (g->bf) {
            std::vector<__nv_bfloat16> Bh(B.size());
            for (size_t i = 0; i < B.size(); ++i) Bh[i] = __float2bfloat16_rn(B[i]);
            e = cudaMemcpyAsync(dst, Bh.data(), Bh.size() * esz, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        } else {
            e = cudaMemcpyAsync(dst, B.data(), B.size() * esz, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        if (e != cudaSuccess) set_error("upload of the transform matrix failed");
        return e == cudaSuccess;
    };
    if (!upload(p.nr, g->Br)) return fail(TVD_ECUDA);
    if (g->Bc != g->Br && !upload(p.nc, g->Bc)) return fail(TVD_ECUDA);
    if (cublasCreate(&g->h) != CUBLAS_STATUS_SUCCESS) {
        g->h = nullptr;
        set_error("cublasCreate failed");
        return fail(TVD_ECUDA);
    }
    if (cublasSetWorkspace(g->h, g->ws, g->ws_bytes) != CUBLAS_STATUS_SUCCESS) {
        set_error("cublasSetWorkspace failed");
        return fail(TVD_ECUDA);
    }
    // TVD_GEMM_TUNE=0 keeps cuBLAS's default algorithm for every product
    const char* tv = std::getenv("TVD_GEMM_TUNE");
    if (!(tv && tv[0] == '0')) {
        tvd_status ts = tune_lt(p, *g, s);
        if (ts != TVD_OK) return fail(ts);
    }
    return TVD_OK;
}

// ---------------------------------------------------------------- vector kernels

// Stores of four consecutive values (index i in units of 4) and of one value
// in the operand type of the products.
__device__ __forceinline__ void store4(float* p, size_t i, float4 v) { reinterpret_cast<float4*>(p)[i] = v; }
__device__ __forceinline__ void store4(__nv_bfloat16* p, size_t i, float4 v) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<unsigned int*>(&lo);
    u.y = *reinterpret_cast<unsigned int*>(&hi);
    reinterpret_cast<uint2*>(p)[i] = u;
}
__device__ __forceinline__ void store1(float* p, size_t o, float v) { p[o] = v; }
__device__ __forceinline__ void store1(__nv_bfloat16* p, size_t o, float v) { p[o] = __float2bfloat16_rn(v); }

// First kernel of the solve on the CG path: the previous iteration's pending
// x += alpha p, r -= alpha q with ||r||^2 and the stopping test (as the first
// row pass of the FFT form does), then s = d o r.
template <typename OutT>
__global__ void __launch_bounds__(kThreads)
gemm_pre_kernel(float* __restrict__ r, float* __restrict__ x, const float* __restrict__ q, const float* p0,
                const float* p1, const float* __restrict__ d, OutT* __restrict__ s, size_t n, CgState* st,
                double* red, unsigned int* ticket) {
    pdl_wait();   // everything below reads what earlier kernels in the stream write
    if (st && st->done) return;
    // pending is the same for every block: the last block clears it only
    // after every block has passed its reduction
    const bool upd = x && st && st->pending;
    const float al = upd ? (float)st->alpha : 0.0f;
    const float* __restrict__ pv = (st && st->pbuf) ? p0 : p1;
    float part = 0.0f;
    const size_t nv = n / 4;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nv; i += (size_t)gridDim.x * blockDim.x) {
        float4 rv = reinterpret_cast<const float4*>(r)[i];
        if (upd) {
            const float4 qv = reinterpret_cast<const float4*>(q)[i];
            const float4 pp = reinterpret_cast<const float4*>(pv)[i];
            float4 xv = reinterpret_cast<const float4*>(x)[i];
            rv.x -= al * qv.x; rv.y -= al * qv.y; rv.z -= al * qv.z; rv.w -= al * qv.w;
            xv.x += al * pp.x; xv.y += al * pp.y; xv.z += al * pp.z; xv.w += al * pp.w;
            reinterpret_cast<float4*>(r)[i] = rv;
            reinterpret_cast<float4*>(x)[i] = xv;
            part += rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
        }
        if (d) {
            const float4 dv = reinterpret_cast<const float4*>(d)[i];
            rv.x *= dv.x; rv.y *= dv.y; rv.z *= dv.z; rv.w *= dv.w;
        }
        store4(s, i, rv);
    }
    for (size_t o = nv * 4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        float v = r[o];
        if (upd) {
            v -= al * q[o];
            r[o] = v;
            x[o] += al * pv[o];
            part += v * v;
        }
        store1(s, o, d ? v * d[o] : v);
    }
    if (!upd) return;
    double sum;
    if (block_reduce_last((double)part, red, ticket, blockIdx.x, gridDim.x, &sum) && threadIdx.x == 0)
        finish_xr(st, sum);
}

// out = y o f (the division by the spectrum, f = 1 / spectrum), in the operand
// type of the products (out may be y for float storage).
template <typename OutT>
__global__ void __launch_bounds__(kThreads)
gemm_scale_kernel(const float* y, const float* __restrict__ f, OutT* out, size_t n, const CgState* st) {
    pdl_wait();
    if (st && st->done) return;
    const size_t nv = n / 4;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nv; i += (size_t)gridDim.x * blockDim.x) {
        float4 a = reinterpret_cast<const float4*>(y)[i];
        const float4 b = reinterpret_cast<const float4*>(f)[i];
        a.x *= b.x; a.y *= b.y; a.z *= b.z; a.w *= b.w;
        store4(out, i, a);
    }
    for (size_t o = nv * 4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
        store1(out, o, y[o] * f[o]);
}

// z = d o u, and on the CG path r^T z with the Fletcher-Reeves coefficient.
__global__ void __launch_bounds__(kThreads)
gemm_post_kernel(const float* __restrict__ u, const float* __restrict__ d, const float* __restrict__ r,
                 float* __restrict__ z, size_t n, CgState* st, double* red, unsigned int* ticket) {
    pdl_wait();
    if (st && st->done) return;
    float part = 0.0f;
    const size_t nv = n / 4;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nv; i += (size_t)gridDim.x * blockDim.x) {
        float4 v = reinterpret_cast<const float4*>(u)[i];
        if (d) {
            const float4 dv = reinterpret_cast<const float4*>(d)[i];
            v.x *= dv.x; v.y *= dv.y; v.z *= dv.z; v.w *= dv.w;
        }
        reinterpret_cast<float4*>(z)[i] = v;
        if (st) {
            const float4 rv = reinterpret_cast<const float4*>(r)[i];
            part += rv.x * v.x + rv.y * v.y + rv.z * v.z + rv.w * v.w;
        }
    }
    for (size_t o = nv * 4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const float v = d ? u[o] * d[o] : u[o];
        z[o] = v;
        if (st) part += r[o] * v;
    }
    if (!st) return;
    double sum;
    if (block_reduce_last((double)part, red, ticket, blockIdx.x, gridDim.x, &sum) && threadIdx.x == 0)
        finish_rho(st, sum);
}

// Grid of the vector kernels: at most TVD_EW_BLOCKS_PER_SM (default 2) blocks
// per SM, each thread walking several float4 by the grid-stride loops. With
// one float4 per thread the block reductions dominated (ncu: barrier and
// scoreboard stalls); measured at 1024^2: 16 blocks per SM 11.8, 8 12.0,
// 4 12.8, 2 13.0 deblurs/s.
static int ew_blocks(size_t n) {
    static const int per_sm = []() {
        const char* v = std::getenv("TVD_EW_BLOCKS_PER_SM");
        const int k = v ? std::atoi(v) : 2;
        return k > 0 ? k : 2;
    }();
    size_t b = (n / 4 + kThreads - 1) / kThreads;
    const size_t cap = (size_t)num_sms() * per_sm;
    if (b > cap) b = cap;
    return (int)(b ? b : 1);
}

static bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Product i (gemm_shape) C = op(A) op(B): the tuned cuBLASLt algorithm, else
// cublasGemmEx with cuBLAS's own choice.
static tvd_status gemm(const GemmPrecond& g, int i, int nr, int nc, const void* A, const void* B, void* C,
                       cudaStream_t s) {
    const float one = 1.0f, zero = 0.0f;
    const GemmShape sh = gemm_shape(i, nr, nc);
    ProfScope prof(PROF_GEMM, s, 1, false);
    const LtGemm& q = g.g[i];
    if (q.tuned) {
        TVD_BLAS_TRY(cublasLtMatmul(g.lt, q.op, &one, A, q.a, B, q.b, &zero, C, q.c, C, q.c, &q.algo, g.ws,
                                    g.ws_bytes, s));
        return TVD_OK;
    }
    const cudaDataType_t ot = g.bf ? CUDA_R_16BF : CUDA_R_32F;
    TVD_BLAS_TRY(cublasSetStream(g.h, s));
    TVD_BLAS_TRY(cublasGemmEx(g.h, sh.ta, sh.tb, sh.m, sh.n, sh.k, &one, A, ot, sh.lda, B, ot, sh.ldb, &zero, C,
                              sh.a_is_mat ? ot : CUDA_R_32F, sh.m, g.bf ? CUBLAS_COMPUTE_32F : g.ct,
                              CUBLAS_GEMM_DEFAULT));
    return TVD_OK;
}

tvd_status gemm_precond_solve(const tvd_plan_s& p, const Ops<float>& o, const float* r, float* z, CgState* st,
                              cudaStream_t s, float* x) {
    const auto* g = static_cast<const GemmPrecond*>(p.gemm);
    const bool scaled = (p.pc == TVD_PC_DFAST || p.pc == TVD_PC_FASTD);
    const float* d = scaled ? o.dmh : nullptr;
    const size_t n = (size_t)p.nr * p.nc;
    const int nr = p.nr, nc = p.nc;
    if (!al16(r) || !al16(z) || (x && !al16(x))) {
        set_error("GEMM preconditioner: vectors must be 16-byte aligned");
        return TVD_EINVAL;
    }
    const int blocks = ew_blocks(n);
    using bf16 = __nv_bfloat16;
    {
        ProfScope prof(PROF_GEMM_EW, s);
        if (g->bf)
            TVD_CUDA_TRY(launch_pdl(gemm_pre_kernel<bf16>, dim3(blocks), dim3(kThreads), 0, s, const_cast<float*>(r),
                                    x, o.q, o.p, o.p2, d, (bf16*)g->in, n, st, p.red, p.ticket + 7));
        else
            TVD_CUDA_TRY(launch_pdl(gemm_pre_kernel<float>, dim3(blocks), dim3(kThreads), 0, s, const_cast<float*>(r),
                                    x, o.q, o.p, o.p2, d, (float*)g->in, n, st, p.red, p.ticket + 7));
        TVD_CUDA_TRY(cudaGetLastError());
    }
    // forward: mid = B_c in (row pass), s1 = mid B_r^T (column pass)
    TVD_TRY(gemm(*g, 0, nr, nc, g->Bc, g->in, g->mid, s));
    TVD_TRY(gemm(*g, 1, nr, nc, g->mid, g->Br, g->s1, s));
    {
        ProfScope prof(PROF_GEMM_EW, s);
        if (g->bf)
            TVD_CUDA_TRY(launch_pdl(gemm_scale_kernel<bf16>, dim3(blocks), dim3(kThreads), 0, s, (const float*)g->s1,
                                    (const float*)o.inv_spec, (bf16*)g->in, n, (const CgState*)st));
        else
            TVD_CUDA_TRY(launch_pdl(gemm_scale_kernel<float>, dim3(blocks), dim3(kThreads), 0, s,
                                    (const float*)g->s1, (const float*)o.inv_spec, (float*)g->in, n,
                                    (const CgState*)st));
        TVD_CUDA_TRY(cudaGetLastError());
    }
    // inverse: mid = B_c^T in, s1 = mid B_r
    TVD_TRY(gemm(*g, 2, nr, nc, g->Bc, g->in, g->mid, s));
    TVD_TRY(gemm(*g, 3, nr, nc, g->mid, g->Br, g->s1, s));
    {
        ProfScope prof(PROF_GEMM_EW, s);
        TVD_CUDA_TRY(launch_pdl(gemm_post_kernel, dim3(blocks), dim3(kThreads), 0, s, (const float*)g->s1, d, r, z,
                                n, st, p.red, p.ticket + 2));
        TVD_CUDA_TRY(cudaGetLastError());
    }
    return TVD_OK;
}

}  // namespace tvd
