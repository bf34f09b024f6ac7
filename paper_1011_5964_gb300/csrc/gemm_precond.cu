// Dense-matrix form of the preconditioner transforms (float plans).
//
// The fast preconditioners of Secs. 2-3 (M, D_M, M_D for AR; R, D_R, R_D for R)
// apply the 2D transform U = B_r (x) B_c, a diagonal, and U^{-1}:
//   z = d o B_r^T [ (B_r (d o r) B_c^T) o (1 / spectrum) ] B_c,   d = D^-1/2 or 1,
// with B = hat-S_n = diag(1, S_{n-2}, 1) (S_m the orthonormal DST-I of
// eq. (lambda), symmetric, an involution) for AR and B = C, the orthonormal
// DCT-II of Sec. 3.1 (B^{-1} = C^T) for R. Each 1D transform of all lines is
// one matrix product with the n x n matrix B, run by the library's own
// tensor-core kernel (tc_gemm.cuh: TMA tiles, tcgen05.mma into tensor memory,
// bf16 or tf32 operands, float accumulation). Every product is C = A B^T with
// both operands K-major; the transform matrix is always the A operand, so each
// product writes its output row-major and the next one reads it K-major:
//   1. X1^T = B_c S^T        S = d o r (operand type, rows of n_c)
//   2. Y    = (B_r X1) o f   f = 1 / spectrum (the divide in the epilogue)
//   3. W^T  = B_c^T Y^T      (the inverse along rows)
//   4. z    = d o (B_r^T W)  with r^T z in the epilogue (CG path)
// so the solve is one vector kernel (the pending CG update and S) and four
// products. The preconditioner only shapes the CG iteration: its rounding
// changes the iteration count, not the solution, whose accuracy the double
// residual of the MIXED form decides.
#include "tc_gemm.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace tvd {

using bf16 = __nv_bfloat16;

// Tile widths and pipeline depths of the products (about 192 KB of stages).
constexpr int kStagesBn64 = 8;
constexpr int kStagesBn128 = 6;
// 64-column products whose epilogue stages f (spectral divide) or d and r (last product) in
// shared memory keep fewer stages so that both fit
template <int BN, int EPI>
constexpr int stages_of() {
    return BN == 128 ? kStagesBn128 : (EPI == tc::EPI_POST ? 5 : (EPI == tc::EPI_SCALE ? 7 : kStagesBn64));
}
static_assert(tc::TcSmem<64, stages_of<64, tc::EPI_POST>(), tc::EPI_POST>::kBytes <= 227 * 1024, "smem");
static_assert(tc::TcSmem<64, stages_of<64, tc::EPI_SCALE>(), tc::EPI_SCALE>::kBytes <= 227 * 1024, "smem");
static_assert(tc::TcSmem<64, stages_of<64, tc::EPI_STORE>(), tc::EPI_STORE>::kBytes <= 227 * 1024, "smem");
static_assert(tc::TcSmem<128, stages_of<128, tc::EPI_POST>(), tc::EPI_POST>::kBytes <= 227 * 1024, "smem");

struct GemmPrecond {
    bool bf = false;              // operands: bf16 (kind::f16) or float (kind::tf32)
    int ldr = 0, ldc = 0;         // padded row strides of rows of n_r / n_c elements
    void* Br = nullptr;           // n_r x ldr, transform matrix B_r (row k = basis vector k)
    void* Bc = nullptr;           // n_c x ldc
    void* BrT = nullptr;          // n_r x ldr, B_r^T (aliases Br for AR: hat-S is symmetric)
    void* BcT = nullptr;          // n_c x ldc
    void* bufR = nullptr;         // n_r x ldc: S, then Y
    void* bufC = nullptr;         // n_c x ldr: X1^T, then W^T
    int* err = nullptr;           // device flag: TVD_ETIMEOUT when a product's wait gave up
    int bn = 64;                  // tile width of the products
    CUtensorMap mBr, mBc, mBrT, mBcT, mR, mC;
    // folded products (AR, eq. (fp), sides multiples of 256): n x n/2 matrices of the two
    // half-length transforms, columns indexed by natural (An) or grouped-pair (Ag) slots
    bool fold = false;
    void *An_r = nullptr, *Ag_r = nullptr, *An_c = nullptr, *Ag_c = nullptr;
    CUtensorMap mAn_r, mAg_r, mAn_c, mAg_c, mR32, mC32;
    std::vector<void*> owned;     // distinct device allocations
};

static int pad8(int n) { return (n + 7) / 8 * 8; }

// Position p of the grouped order -> natural index (the host twin of tc::nat_of).
static int nat_host(int p, int n) {
    const int h = n / 2;
    if (p < h) return p == 0 ? 0 : 2 * p - 1;
    const int a = p - h;
    return a == 0 ? n - 1 : n - 2 * a;
}

// n x n/2 matrix of the folded hat-S (n even): row p = output nat_host(p, n); column
// a = input slot a of its half (slot 0: the raw endpoint). grouped_cols: slot a >= 1
// holds the pair (2a - 1, n - 2a) (inputs in grouped order), else (a, n - 1 - a).
static void folded_matrix(int n, bool grouped_cols, std::vector<double>& out) {
    const int h = n / 2, M = n - 1;
    const double pi = 3.14159265358979323846, sc = std::sqrt(2.0 / M);
    out.assign((size_t)n * h, 0.0);
    for (int p = 0; p < n; ++p) {
        const int q = nat_host(p, n);
        if (q == 0 || q == n - 1) {
            out[(size_t)p * h] = 1.0;
            continue;
        }
        for (int a = 1; a < h; ++a) {
            const int l = grouped_cols ? 2 * a - 1 : a;
            const long long t = ((long long)q * l) % (2LL * M);
            out[(size_t)p * h + a] = sc * std::sin(pi * (double)t / M);
        }
    }
}

// Row-major n x n matrix of the 1D transform (row k = basis vector k): AR hat-S_n,
// R the DCT-II C_n (frequency by space); transposed on request. Arguments are
// reduced modulo the period in integers; rows padded to ld.
// For the reblurring method (AR): the forward matrix is T_n^-1 =
// [1 0 0; -S p S -S J p; 0 0 1] and the inverse one T_n = [1 0 0; p S J p; 0 0 1]
// (eq. (Tn) in the block form of Sec. 2, p_i = 1 - i / (n - 1)).
static void transform_matrix(int n, int ld, tvd_bc bc, bool transpose, std::vector<double>& out,
                             bool reblur = false) {
    out.assign((size_t)n * ld, 0.0);
    const double pi = 3.14159265358979323846;
    auto at = [&](int k, int j) -> double& { return transpose ? out[(size_t)j * ld + k] : out[(size_t)k * ld + j]; };
    if (reblur) {
        const int m = n - 2, M = n - 1;
        const double sc = std::sqrt(2.0 / M);
        auto S = [&](int k, int l) { return sc * std::sin(pi * (double)(((long long)k * l) % (2LL * M)) / M); };
        out[0] = 1.0;
        out[(size_t)(n - 1) * ld + n - 1] = 1.0;
        for (int k = 1; k <= m; ++k) {
            double sp = 0.0, sjp = 0.0;
            for (int l = 1; l <= m; ++l) {
                const double skl = S(k, l);
                out[(size_t)k * ld + l] = skl;
                sp += skl * (1.0 - (double)l / M);
                sjp += skl * ((double)l / M);
            }
            if (transpose) {   // T_n
                out[(size_t)k * ld] = 1.0 - (double)k / M;
                out[(size_t)k * ld + n - 1] = (double)k / M;
            } else {           // T_n^-1
                out[(size_t)k * ld] = -sp;
                out[(size_t)k * ld + n - 1] = -sjp;
            }
        }
        return;
    }
    if (bc == TVD_BC_ANTIREFLECTIVE) {
        const int M = n - 1;   // S_{n-2}: sqrt(2/M) sin(k l pi / M), k, l = 1..n-2
        const double sc = std::sqrt(2.0 / M);
        at(0, 0) = 1.0;
        at(n - 1, n - 1) = 1.0;
        for (int k = 1; k <= n - 2; ++k)
            for (int l = 1; l <= n - 2; ++l) {
                const long long a = ((long long)k * l) % (2LL * M);
                at(k, l) = sc * std::sin(pi * (double)a / M);
            }
    } else {
        const double c0 = std::sqrt(1.0 / n), c1 = std::sqrt(2.0 / n);
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j) {
                const long long a = ((long long)k * (2 * j + 1)) % (4LL * n);
                at(k, j) = (k ? c1 : c0) * std::cos(pi * (double)a / (2.0 * n));
            }
    }
}

void gemm_precond_destroy(tvd_plan_s& p) {
    auto* g = static_cast<GemmPrecond*>(p.gemm);
    if (!g) return;
    for (void* q : g->owned) cudaFree(q);
    if (g->err) cudaFree(g->err);
    delete g;
    p.gemm = nullptr;
}

bool gemm_fold_allowed(const tvd_plan_s& p) {
    return p.bc == TVD_BC_ANTIREFLECTIVE && !p.reblur() && p.nr % 256 == 0 && p.nc % 256 == 0;
}

int gemm_precond_folded(const tvd_plan_s& p) {
    const auto* g = static_cast<const GemmPrecond*>(p.gemm);
    return g && g->fold ? 1 : 0;
}

int gemm_precond_tile(const tvd_plan_s& p) {
    const auto* g = static_cast<const GemmPrecond*>(p.gemm);
    return g ? g->bn : 0;
}

int gemm_precond_storage(const tvd_plan_s& p) {
    const auto* g = static_cast<const GemmPrecond*>(p.gemm);
    return g ? (g->bf ? 2 : 1) : 0;
}

template <typename OpT>
static tvd_status prepare_kernels(int bn, bool fold) {
    using namespace tc;
    if (fold) {
        TVD_CUDA_TRY((tc_gemm_prepare<OpT, 64, stages_of<64, EPI_STORE>(), EPI_STORE, 1>()));
        TVD_CUDA_TRY((tc_gemm_prepare<OpT, 64, stages_of<64, EPI_SCALE>(), EPI_SCALE, 2>()));
        TVD_CUDA_TRY((tc_gemm_prepare<OpT, 64, stages_of<64, EPI_STORE>(), EPI_STORE, 3>()));
        TVD_CUDA_TRY((tc_gemm_prepare<OpT, 64, stages_of<64, EPI_POST>(), EPI_POST, 4>()));
        return TVD_OK;
    }
    if (bn == 128) {
        TVD_CUDA_TRY((tc_gemm_prepare<OpT, 128, stages_of<128, EPI_STORE>(), EPI_STORE>()));
        TVD_CUDA_TRY((tc_gemm_prepare<OpT, 128, stages_of<128, EPI_SCALE>(), EPI_SCALE>()));
        TVD_CUDA_TRY((tc_gemm_prepare<OpT, 128, stages_of<128, EPI_POST>(), EPI_POST>()));
    } else {
        TVD_CUDA_TRY((tc_gemm_prepare<OpT, 64, stages_of<64, EPI_STORE>(), EPI_STORE>()));
        TVD_CUDA_TRY((tc_gemm_prepare<OpT, 64, stages_of<64, EPI_SCALE>(), EPI_SCALE>()));
        TVD_CUDA_TRY((tc_gemm_prepare<OpT, 64, stages_of<64, EPI_POST>(), EPI_POST>()));
    }
    return TVD_OK;
}

tvd_status gemm_precond_create(tvd_plan_s& p, cudaStream_t s) {
    if (p.gemm) return TVD_OK;
    auto* g = new GemmPrecond();
    p.gemm = g;
    auto fail = [&](tvd_status e) {
        gemm_precond_destroy(p);
        return e;
    };
    if (!tc::tensor_map_encoder()) {
        set_error("GEMM transforms: cuTensorMapEncodeTiled is not available from the driver");
        return fail(TVD_ECUDA);
    }
    // bf16 operands from sides of 1024 on, float (tf32 products) below; TVD_GEMM_STORAGE=bf16 / f32
    // overrides
    const char* sv = std::getenv("TVD_GEMM_STORAGE");
    if (sv && !std::strcmp(sv, "bf16")) g->bf = true;
    else if (sv && !std::strcmp(sv, "f32")) g->bf = false;
    else g->bf = std::min(p.nr, p.nc) >= 1024;
    const size_t esz = g->bf ? sizeof(bf16) : sizeof(float);
    g->ldr = pad8(p.nr);
    g->ldc = pad8(p.nc);
    // tile width: 128 when the 128 x 128 tiles of a product already cover the SMs, else 64
    const long long tiles128 = (long long)((p.nr + 127) / 128) * ((p.nc + 127) / 128);
    g->bn = tiles128 >= num_sms() ? 128 : 64;
    const char* bv = std::getenv("TVD_GEMM_BN");
    if (bv && (std::atoi(bv) == 64 || std::atoi(bv) == 128)) g->bn = std::atoi(bv);
    // folded products (half the K of each product) for AR plans of eq. (fp) whose sides are
    // multiples of 256; TVD_GEMM_FOLD=0 keeps the full products. The autotuner's choice
    // (tvd_plan_tune) comes before both rules.
    const char* fv = std::getenv("TVD_GEMM_FOLD");
    g->fold = gemm_fold_allowed(p) && (p.gemm_fold >= 0 ? p.gemm_fold == 1 : !(fv && fv[0] == '0'));
    if (p.gemm_bn == 64 || p.gemm_bn == 128) g->bn = p.gemm_bn;
    if (g->fold) g->bn = 64;
    auto alloc = [&](void** ptr, size_t bytes) -> bool {
        if (cudaMalloc(ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc failed for the GEMM transform buffers");
            return false;
        }
        g->owned.push_back(*ptr);
        return true;
    };
    const bool reblur = p.reblur();
    const bool sym = p.bc == TVD_BC_ANTIREFLECTIVE && !reblur;   // hat-S = hat-S^T (T_n is not symmetric)
    if (!alloc(&g->Br, (size_t)p.nr * g->ldr * esz)) return fail(TVD_ENOMEM);
    g->BrT = g->Br;
    if (!sym && !alloc(&g->BrT, (size_t)p.nr * g->ldr * esz)) return fail(TVD_ENOMEM);
    if (p.nc == p.nr) {
        g->Bc = g->Br;
        g->BcT = g->BrT;
    } else {
        if (!alloc(&g->Bc, (size_t)p.nc * g->ldc * esz)) return fail(TVD_ENOMEM);
        g->BcT = g->Bc;
        if (!sym && !alloc(&g->BcT, (size_t)p.nc * g->ldc * esz)) return fail(TVD_ENOMEM);
    }
    if (!alloc(&g->bufR, (size_t)p.nr * g->ldc * esz) || !alloc(&g->bufC, (size_t)p.nc * g->ldr * esz))
        return fail(TVD_ENOMEM);
    if (cudaMalloc(&g->err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        g->err = nullptr;
        set_error("cudaMalloc failed for the GEMM error flag");
        return fail(TVD_ENOMEM);
    }
    // the operand buffers are zeroed once: their row padding is never read (the
    // tensor maps end at the logical sizes) but stays defined
    if (cudaMemsetAsync(g->err, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(g->bufR, 0, (size_t)p.nr * g->ldc * esz, s) != cudaSuccess ||
        cudaMemsetAsync(g->bufC, 0, (size_t)p.nc * g->ldr * esz, s) != cudaSuccess) {
        set_error("clearing the GEMM transform buffers failed");
        return fail(TVD_ECUDA);
    }
    auto upload = [&](int side, int ld, bool transpose, void* dst) -> bool {
        std::vector<double> B;
        transform_matrix(side, ld, p.bc, transpose, B, reblur);
        cudaError_t e;
        if (g->bf) {
            std::vector<bf16> Bh(B.size());
            for (size_t i = 0; i < B.size(); ++i) Bh[i] = __double2bfloat16(B[i]);
            e = cudaMemcpyAsync(dst, Bh.data(), Bh.size() * esz, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        } else {
            std::vector<float> Bf(B.begin(), B.end());
            e = cudaMemcpyAsync(dst, Bf.data(), Bf.size() * esz, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        if (e != cudaSuccess) set_error("upload of the transform matrix failed");
        return e == cudaSuccess;
    };
    if (!upload(p.nr, g->ldr, false, g->Br)) return fail(TVD_ECUDA);
    if (g->BrT != g->Br && !upload(p.nr, g->ldr, true, g->BrT)) return fail(TVD_ECUDA);
    if (g->Bc != g->Br) {
        if (!upload(p.nc, g->ldc, false, g->Bc)) return fail(TVD_ECUDA);
        if (g->BcT != g->Bc && !upload(p.nc, g->ldc, true, g->BcT)) return fail(TVD_ECUDA);
    }
    const int eb = (int)esz;
    const bool maps = tc::make_tc_map(&g->mBr, g->Br, eb, p.nr, p.nr, g->ldr, tc::BM) &&
                      tc::make_tc_map(&g->mBrT, g->BrT, eb, p.nr, p.nr, g->ldr, tc::BM) &&
                      tc::make_tc_map(&g->mBc, g->Bc, eb, p.nc, p.nc, g->ldc, tc::BM) &&
                      tc::make_tc_map(&g->mBcT, g->BcT, eb, p.nc, p.nc, g->ldc, tc::BM) &&
                      tc::make_tc_map(&g->mR, g->bufR, eb, p.nc, p.nr, g->ldc, g->bn) &&
                      tc::make_tc_map(&g->mC, g->bufC, eb, p.nr, p.nc, g->ldr, g->bn);
    if (!maps) {
        set_error("cuTensorMapEncodeTiled failed for the GEMM transform operands");
        return fail(TVD_ECUDA);
    }
    if (g->fold) {
        auto upload_fold = [&](int side, bool grouped, void** dst) -> bool {
            std::vector<double> B;
            folded_matrix(side, grouped, B);
            if (!alloc(dst, B.size() * esz)) return false;
            cudaError_t e;
            if (g->bf) {
                std::vector<bf16> Bh(B.size());
                for (size_t i = 0; i < B.size(); ++i) Bh[i] = __double2bfloat16(B[i]);
                e = cudaMemcpyAsync(*dst, Bh.data(), Bh.size() * esz, cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            } else {
                std::vector<float> Bf(B.begin(), B.end());
                e = cudaMemcpyAsync(*dst, Bf.data(), Bf.size() * esz, cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            }
            if (e != cudaSuccess) set_error("upload of the folded transform matrix failed");
            return e == cudaSuccess;
        };
        if (!upload_fold(p.nr, false, &g->An_r) || !upload_fold(p.nr, true, &g->Ag_r)) return fail(TVD_ECUDA);
        if (p.nc == p.nr) {
            g->An_c = g->An_r;
            g->Ag_c = g->Ag_r;
        } else if (!upload_fold(p.nc, false, &g->An_c) || !upload_fold(p.nc, true, &g->Ag_c)) {
            return fail(TVD_ECUDA);
        }
        const int hr = p.nr / 2, hc = p.nc / 2;
        const bool fmaps = tc::make_tc_map(&g->mAn_r, g->An_r, eb, hr, p.nr, hr, tc::BM) &&
                           tc::make_tc_map(&g->mAg_r, g->Ag_r, eb, hr, p.nr, hr, tc::BM) &&
                           tc::make_tc_map(&g->mAn_c, g->An_c, eb, hc, p.nc, hc, tc::BM) &&
                           tc::make_tc_map(&g->mAg_c, g->Ag_c, eb, hc, p.nc, hc, tc::BM) &&
                           tc::make_tc_map(&g->mR32, g->bufR, eb, p.nc, p.nr, g->ldc, 32) &&
                           tc::make_tc_map(&g->mC32, g->bufC, eb, p.nr, p.nc, g->ldr, 32);
        if (!fmaps) {
            set_error("cuTensorMapEncodeTiled failed for the folded transform operands");
            return fail(TVD_ECUDA);
        }
    }
    // shared-memory opt-in of the product kernels now, outside any stream capture
    const tvd_status ps = g->bf ? prepare_kernels<bf16>(g->bn, g->fold) : prepare_kernels<float>(g->bn, g->fold);
    if (ps != TVD_OK) return fail(ps);
    return TVD_OK;
}

tvd_status gemm_precond_check(const tvd_plan_s& p, cudaStream_t s) {
    const auto* g = static_cast<const GemmPrecond*>(p.gemm);
    if (!g) return TVD_OK;
    int h = 0;
    TVD_CUDA_TRY(cudaMemcpyAsync(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TVD_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) {
        TVD_CUDA_TRY(cudaMemsetAsync(g->err, 0, sizeof(int), s));
        set_error("a tensor-core transform product gave up waiting for its operands (bounded wait expired)");
        return TVD_ETIMEOUT;
    }
    return TVD_OK;
}

// ---------------------------------------------------------------- the vector pass

// Stores of four consecutive values (index i in units of 4) and of one value
// in the operand type of the products.
__device__ __forceinline__ void store4(float* p, size_t i, float4 v) { reinterpret_cast<float4*>(p)[i] = v; }
__device__ __forceinline__ void store4(bf16* p, size_t i, float4 v) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<unsigned int*>(&lo);
    u.y = *reinterpret_cast<unsigned int*>(&hi);
    reinterpret_cast<uint2*>(p)[i] = u;
}
__device__ __forceinline__ void store1(float* p, size_t o, float v) { p[o] = v; }
__device__ __forceinline__ void store1(bf16* p, size_t o, float v) { p[o] = __float2bfloat16_rn(v); }

// First kernel of the solve on the CG path: the previous iteration's pending
// x += alpha p, r -= alpha q with ||r||^2 and the stopping test (as the first
// row pass of the FFT form does), then S = d o r in the operand type, rows
// padded to ld (ld == nc: one contiguous vector walk).
template <typename OutT>
__global__ void __launch_bounds__(kThreads)
gemm_pre_kernel(float* __restrict__ r, float* __restrict__ x, const float* __restrict__ q, const float* p0,
                const float* p1, const float* __restrict__ d, OutT* __restrict__ s, int nr, int nc, int ld,
                CgState* st, double* red, unsigned int* ticket) {
    pdl_wait();   // everything below reads what earlier kernels in the stream write
    if (st && st->done) return;
    // pending is the same for every block: the last block clears it only
    // after every block has passed its reduction
    const bool upd = x && st && st->pending;
    const float al = upd ? (float)st->alpha : 0.0f;
    const float* __restrict__ pv = (st && st->pbuf) ? p0 : p1;
    const size_t n = (size_t)nr * nc;
    float part = 0.0f;
    if (ld == nc) {
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
    }
    const size_t first = ld == nc ? (n / 4) * 4 : 0;
    for (size_t o = first + blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        float v = r[o];
        if (upd) {
            v -= al * q[o];
            r[o] = v;
            x[o] += al * pv[o];
            part += v * v;
        }
        const size_t row = o / (size_t)nc, col = o - row * nc;
        store1(s, row * ld + col, d ? v * d[o] : v);
    }
    if (!upd) return;
    double sum;
    if (block_reduce_last((double)part, red, ticket, blockIdx.x, gridDim.x, &sum) && threadIdx.x == 0)
        finish_xr(st, sum);
}

// The folded form's vector pass: the same pending update and stopping test, then
// S = D^-1/2 r folded along each row for the first folded product: slot a of the
// first half s_a = S_a + S_{nc-1-a}, of the second half S_a - S_{nc-1-a}, a = 1 ..
// nc/2 - 1, slot 0 of each half the raw S_0 and S_{nc-1}. A thread takes a quad of
// columns of the first half and its mirror quad (nc a multiple of 8).
template <typename OutT>
__global__ void __launch_bounds__(kThreads)
gemm_fold_pre_kernel(float* __restrict__ r, float* __restrict__ x, const float* __restrict__ q, const float* p0,
                     const float* p1, const float* __restrict__ d, OutT* __restrict__ s, int nr, int nc,
                     CgState* st, double* red, unsigned int* ticket) {
    pdl_wait();
    if (st && st->done) return;
    const bool upd = x && st && st->pending;
    const float al = upd ? (float)st->alpha : 0.0f;
    const float* __restrict__ pv = (st && st->pbuf) ? p0 : p1;
    const int hq = nc / 8;                     // quads in the first half of a row
    const size_t units = (size_t)nr * hq;
    float part = 0.0f;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
        const size_t row = u / hq;
        const int qd = (int)(u - row * hq);
        const size_t il = (row * nc + 4 * (size_t)qd) / 4;              // float4 index of the low quad
        const size_t ih = (row * nc + (size_t)(nc - 4 - 4 * qd)) / 4;   // and of its mirror quad
        float4 rl = reinterpret_cast<const float4*>(r)[il], rh = reinterpret_cast<const float4*>(r)[ih];
        if (upd) {
            const float4 ql = reinterpret_cast<const float4*>(q)[il], qh = reinterpret_cast<const float4*>(q)[ih];
            const float4 pl = reinterpret_cast<const float4*>(pv)[il], ph = reinterpret_cast<const float4*>(pv)[ih];
            float4 xl = reinterpret_cast<const float4*>(x)[il], xh = reinterpret_cast<const float4*>(x)[ih];
            rl.x -= al * ql.x; rl.y -= al * ql.y; rl.z -= al * ql.z; rl.w -= al * ql.w;
            rh.x -= al * qh.x; rh.y -= al * qh.y; rh.z -= al * qh.z; rh.w -= al * qh.w;
            xl.x += al * pl.x; xl.y += al * pl.y; xl.z += al * pl.z; xl.w += al * pl.w;
            xh.x += al * ph.x; xh.y += al * ph.y; xh.z += al * ph.z; xh.w += al * ph.w;
            reinterpret_cast<float4*>(r)[il] = rl;
            reinterpret_cast<float4*>(r)[ih] = rh;
            reinterpret_cast<float4*>(x)[il] = xl;
            reinterpret_cast<float4*>(x)[ih] = xh;
            part += rl.x * rl.x + rl.y * rl.y + rl.z * rl.z + rl.w * rl.w;
            part += rh.x * rh.x + rh.y * rh.y + rh.z * rh.z + rh.w * rh.w;
        }
        if (d) {
            const float4 dl = reinterpret_cast<const float4*>(d)[il], dh = reinterpret_cast<const float4*>(d)[ih];
            rl.x *= dl.x; rl.y *= dl.y; rl.z *= dl.z; rl.w *= dl.w;
            rh.x *= dh.x; rh.y *= dh.y; rh.z *= dh.z; rh.w *= dh.w;
        }
        // element e of the low quad (column 4 qd + e) pairs with element 3 - e of the mirror quad
        float4 sv = make_float4(rl.x + rh.w, rl.y + rh.z, rl.z + rh.y, rl.w + rh.x);
        float4 dv = make_float4(rl.x - rh.w, rl.y - rh.z, rl.z - rh.y, rl.w - rh.x);
        if (qd == 0) {
            sv.x = rl.x;   // the raw endpoints S_0 and S_{nc-1}
            dv.x = rh.w;
        }
        store4(s, (row * nc + 4 * (size_t)qd) / 4, sv);
        store4(s, (row * nc + nc / 2 + 4 * (size_t)qd) / 4, dv);
    }
    if (!upd) return;
    double sum;
    if (block_reduce_last((double)part, red, ticket, blockIdx.x, gridDim.x, &sum) && threadIdx.x == 0)
        finish_xr(st, sum);
}

// Grid of the vector kernel: at most TVD_EW_BLOCKS_PER_SM (default 2) blocks
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

template <typename OpT>
static tvd_status run_products(const tvd_plan_s& p, const GemmPrecond& g, const Ops<float>& o, const float* d,
                               const float* r, float* z, CgState* st, cudaStream_t s) {
    using namespace tc;
    const int nr = p.nr, nc = p.nc;
    TcEpi e{};
    e.st = st;
    e.err = g.err;
    ProfScope prof(PROF_GEMM, s, 4);
    auto launch = [&](auto kernel_tag, const CUtensorMap& A, const CUtensorMap& B, int M, int N, int K) -> tvd_status {
        constexpr int EPI = decltype(kernel_tag)::value;
        cudaError_t ce;
        if (g.bn == 128) ce = launch_tc_gemm<OpT, 128, stages_of<128, EPI>(), EPI>(A, B, M, N, K, e, s);
        else ce = launch_tc_gemm<OpT, 64, stages_of<64, EPI>(), EPI>(A, B, M, N, K, e, s);
        TVD_CUDA_TRY(ce);
        return TVD_OK;
    };
    using Store = std::integral_constant<int, EPI_STORE>;
    using Scale = std::integral_constant<int, EPI_SCALE>;
    using Post = std::integral_constant<int, EPI_POST>;
    if (g.fold) {
        // folded products (tc_gemm.cuh): each runs K/2 per tile and folds its N direction for the next
        constexpr int S64 = stages_of<64, EPI_STORE>(), C64 = stages_of<64, EPI_SCALE>(),
                      P64 = stages_of<64, EPI_POST>();
        // 1. over the row halves of S (folded by the vector pass): rows k_c grouped, N = image rows
        e.out = g.bufC;
        e.ldo = g.ldr;
        TVD_CUDA_TRY((launch_tc_gemm<OpT, 64, S64, EPI_STORE, 1>(g.mAn_c, g.mR32, nc, nr, nc, e, s)));
        // 2. spectral divide (f gathered at natural indices), rows k_r grouped, N = k_c grouped
        e.out = g.bufR;
        e.ldo = g.ldc;
        e.f = o.inv_spec;
        TVD_CUDA_TRY((launch_tc_gemm<OpT, 64, C64, EPI_SCALE, 2>(g.mAn_r, g.mC32, nr, nc, nr, e, s)));
        // 3. inverse along k_c: rows j (written at their natural index), N = k_r grouped
        e.out = g.bufC;
        e.ldo = g.ldr;
        e.f = nullptr;
        TVD_CUDA_TRY((launch_tc_gemm<OpT, 64, S64, EPI_STORE, 3>(g.mAg_c, g.mR32, nc, nr, nc, e, s)));
        // 4. inverse along k_r: z = d o (.), r^T z, rows i at their natural index, N = j natural
        e.out = z;
        e.ldo = nc;
        e.d = d;
        e.r = r;
        e.red = p.red;
        e.ticket = p.ticket + 2;
        TVD_CUDA_TRY((launch_tc_gemm<OpT, 64, P64, EPI_POST, 4>(g.mAg_r, g.mC, nr, nc, nr, e, s)));
        return TVD_OK;
    }
    // 1. X1^T = B_c S^T  (M = n_c, N = n_r, K = n_c)
    e.out = g.bufC;
    e.ldo = g.ldr;
    TVD_TRY(launch(Store{}, g.mBc, g.mR, nc, nr, nc));
    // 2. Y = (B_r X1) o f  (M = n_r, N = n_c, K = n_r)
    e.out = g.bufR;
    e.ldo = g.ldc;
    e.f = o.inv_spec;
    TVD_TRY(launch(Scale{}, g.mBr, g.mC, nr, nc, nr));
    // 3. W^T = B_c^T Y^T  (M = n_c, N = n_r, K = n_c)
    e.out = g.bufC;
    e.ldo = g.ldr;
    e.f = nullptr;
    TVD_TRY(launch(Store{}, g.mBcT, g.mR, nc, nr, nc));
    // 4. z = d o (B_r^T W), r^T z  (M = n_r, N = n_c, K = n_r)
    e.out = z;
    e.ldo = nc;
    e.d = d;
    e.r = r;
    e.red = p.red;
    e.ticket = p.ticket + 2;
    TVD_TRY(launch(Post{}, g.mBrT, g.mC, nr, nc, nr));
    return TVD_OK;
}

tvd_status gemm_precond_solve(const tvd_plan_s& p, const Ops<float>& o, const float* r, float* z, CgState* st,
                              cudaStream_t s, float* x) {
    const auto* g = static_cast<const GemmPrecond*>(p.gemm);
    const bool scaled = (p.pc == TVD_PC_DFAST || p.pc == TVD_PC_FASTD);
    const float* d = scaled ? o.dmh : nullptr;
    const size_t n = (size_t)p.nr * p.nc;
    if (!al16(r) || !al16(z) || (x && !al16(x))) {
        set_error("GEMM preconditioner: vectors must be 16-byte aligned");
        return TVD_EINVAL;
    }
    if (st && (long long)((p.nr + tc::BM - 1) / tc::BM) * ((p.nc + g->bn - 1) / g->bn) > kMaxRedBlocks) {
        set_error("image too large for the reduction buffer");
        return TVD_EINVAL;
    }
    const int blocks = ew_blocks(n);
    {
        ProfScope prof(PROF_GEMM_EW, s);
        if (g->fold && g->bf)
            TVD_CUDA_TRY(launch_pdl(gemm_fold_pre_kernel<bf16>, dim3(blocks), dim3(kThreads), 0, s,
                                    const_cast<float*>(r), x, o.q, o.p, o.p2, d, (bf16*)g->bufR, p.nr, p.nc, st,
                                    p.red, p.ticket + 7));
        else if (g->fold)
            TVD_CUDA_TRY(launch_pdl(gemm_fold_pre_kernel<float>, dim3(blocks), dim3(kThreads), 0, s,
                                    const_cast<float*>(r), x, o.q, o.p, o.p2, d, (float*)g->bufR, p.nr, p.nc, st,
                                    p.red, p.ticket + 7));
        else if (g->bf)
            TVD_CUDA_TRY(launch_pdl(gemm_pre_kernel<bf16>, dim3(blocks), dim3(kThreads), 0, s, const_cast<float*>(r),
                                    x, o.q, o.p, o.p2, d, (bf16*)g->bufR, p.nr, p.nc, g->ldc, st, p.red,
                                    p.ticket + 7));
        else
            TVD_CUDA_TRY(launch_pdl(gemm_pre_kernel<float>, dim3(blocks), dim3(kThreads), 0, s, const_cast<float*>(r),
                                    x, o.q, o.p, o.p2, d, (float*)g->bufR, p.nr, p.nc, g->ldc, st, p.red,
                                    p.ticket + 7));
        TVD_CUDA_TRY(cudaGetLastError());
    }
    if (g->bf) return run_products<bf16>(p, *g, o, d, r, z, st, s);
    return run_products<float>(p, *g, o, d, r, z, st, s);
}

}  // namespace tvd
