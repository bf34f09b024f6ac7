// Dense transform products on the fifth-generation tensor cores (sm_103a).
//
// C = A B^T with float accumulation, A (M x K) and B (N x K) both row-major
// with K contiguous ("K-major"), C (M x N); operands either bf16 (kind::f16
// products) or float (kind::tf32 products). One CTA computes one 128 x BN tile
// of C:
//   warp 0  (one lane)  streams K-slices of A and B into a ring of shared-
//                       memory stages with TMA (cp.async.bulk.tensor, 128-byte
//                       swizzle), each stage guarded by a "full" mbarrier;
//   warp 1  (one lane)  issues tcgen05.mma (M = 128, N = BN, 32 bytes of K each)
//                       reading both operands from shared memory and
//                       accumulating in tensor memory (TMEM); tcgen05.commit
//                       releases each stage back to the loader ("empty") and
//                       finally signals the finished accumulator;
//   warps 2-5           read the accumulator with tcgen05.ld (warp w owns TMEM
//                       lanes 32 (w % 4) .. + 31, i.e. rows of the tile) and run
//                       the fused epilogue.
// The epilogue variants carry the elementwise passes of the preconditioner
// solve (Sec. 3.2: z = D^-1/2 U^T diag(spectrum)^-1 U D^-1/2 r): a plain
// store in the operand type, a store of C o f (the spectral divide, f =
// 1 / spectrum) and the final z = d o C with the CG inner product r^T z.
// A K-slice of a stage is one 128-byte swizzle row per matrix row: 64 bf16 or
// 32 float elements.
//
// Every wait on an mbarrier is bounded (about one second of SM clock): on
// expiry the kernel records TVD_ETIMEOUT (error flag, and in the CG state when
// one is given, which stops the solve), skips the rest of its work, and still
// releases its tensor memory.
#pragma once

#include "common.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

namespace tvd {
namespace tc {

constexpr int BM = 128;              // tile rows (UMMA M)
constexpr int kRowBytes = 128;       // bytes of K per stage and matrix row (one swizzle row)
constexpr int kTcThreads = 192;      // warp 0 loader, warp 1 MMA issuer, warps 2-5 epilogue
constexpr long long kWaitLimit = 2000000000LL;   // SM clock cycles (~1 s) before a wait gives up

enum { EPI_STORE = 0, EPI_SCALE = 1, EPI_POST = 2 };

struct TcEpi {
    void* out;            // operand type (EPI_STORE, EPI_SCALE) or float (EPI_POST), M x N, row stride ldo
    int ldo;
    const float* f;       // EPI_SCALE: multiplier, M x N, row stride N
    const float* d;       // EPI_POST: diagonal scaling (nullptr: none), M x N, row stride N
    const float* r;       // EPI_POST with st: the residual for r^T z, M x N, row stride N
    CgState* st;          // CG state (nullptr outside the CG): skip when done, r^T z finisher
    double* red;          // per-CTA partial sums (EPI_POST with st)
    unsigned int* ticket;
    int* err;             // set to TVD_ETIMEOUT when a wait gives up (may be nullptr)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with the given parity to complete; false after
// kWaitLimit cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitLimit) return false;
    return true;
}

// 2D tiled TMA load of the box at (c0 = inner coordinate, c1 = row) into
// shared memory, completing `bytes` on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored in the
// 128-byte swizzled layout TMA writes: rows of 128 bytes, groups of 8 rows
// 1024 bytes apart (stride byte offset), descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: float D, A and B K-major of format fmt (1: bf16 for
// kind::f16, 2: tf32 for kind::tf32), M = 128, N.
template <int N, uint32_t fmt>
__host__ __device__ constexpr uint32_t idesc_of() {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// One tcgen05.mma of 32 bytes of K: bf16 operands (K = 16, kind::f16) or float
// operands read as tf32 (K = 8, kind::tf32).
template <typename OpT>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (sizeof(OpT) == 2)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Arrive on `bar` once every tcgen05 operation issued so far by this thread has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Whole warp: allocate ncols TMEM columns, address written to *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Whole warp: 32 consecutive float columns of this warp's 32 TMEM lanes (one row per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
}

// Arrays of float the epilogue needs, staged in shared memory by the epilogue
// warps while the main loop runs (64-column tiles only): EPI_SCALE the
// multiplier f, EPI_POST the scaling d and the residual r. Rows of BN + 1
// floats, so that the 32 threads of a warp (32 rows) reading one column hit 32
// banks.
template <int BN, int EPI>
__host__ __device__ constexpr int pre_arrays() {
    return BN != 64 ? 0 : (EPI == EPI_POST ? 2 : (EPI == EPI_SCALE ? 1 : 0));
}

template <int BN, int STAGES, int EPI = EPI_STORE>
struct TcSmem {
    static constexpr int kABytes = BM * kRowBytes;
    static constexpr int kBBytes = BN * kRowBytes;
    static constexpr int kStageBytes = kABytes + kBBytes;
    static constexpr int kPreStride = BN + 1;                       // floats per staged row
    static constexpr int kPreBytes = pre_arrays<BN, EPI>() * BM * kPreStride * 4;
    static constexpr int kPreOffset = STAGES * kStageBytes;
    static constexpr int kBarOffset = kPreOffset + kPreBytes;
    static constexpr int kBytes = 1024 /* alignment slack */ + kBarOffset + (2 * STAGES + 1) * 8 + 64;
};

template <int BN>
__host__ __device__ constexpr uint32_t tmem_cols() { return BN < 32 ? 32u : (uint32_t)BN; }

// Stores of 32 consecutive values of one row in the operand type (16-byte
// aligned) and of one value.
__device__ __forceinline__ void store_row32(__nv_bfloat16* o, const float (&v)[32]) {
    uint4* o4 = reinterpret_cast<uint4*>(o);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        o4[i] = make_uint4(pack_bf16(v[8 * i], v[8 * i + 1]), pack_bf16(v[8 * i + 2], v[8 * i + 3]),
                           pack_bf16(v[8 * i + 4], v[8 * i + 5]), pack_bf16(v[8 * i + 6], v[8 * i + 7]));
}
__device__ __forceinline__ void store_row32(float* o, const float (&v)[32]) {
    float4* o4 = reinterpret_cast<float4*>(o);
#pragma unroll
    for (int i = 0; i < 8; ++i) o4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
__device__ __forceinline__ void store_one(__nv_bfloat16* o, float v) { *o = __float2bfloat16_rn(v); }
__device__ __forceinline__ void store_one(float* o, float v) { *o = v; }

// 32 consecutive floats of one row (16-byte aligned), read through the L1 cache.
__device__ __forceinline__ void load_row32(const float* p, float (&v)[32]) {
    const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 q = __ldg(p4 + i);
        v[4 * i] = q.x;
        v[4 * i + 1] = q.y;
        v[4 * i + 2] = q.z;
        v[4 * i + 3] = q.w;
    }
}

// Folded products (anti-reflective plans, sides multiples of 256). hat-S is
// symmetric and hat-S[k][n-1-j] = (-1)^(k+1) hat-S[k][j] on the interior, so a
// transform of a line splits into two half-length ones: rows k odd (and the
// endpoint 0) take the sums x_a + x_{n-1-a}, rows k even (and the endpoint
// n-1) the differences, a = 1 .. n/2 - 1 (slot 0 of each half holds the raw
// endpoint value). Outputs are kept in the "grouped" order [0, 1, 3, 5, .. |
// n-1, n-2, n-4, ..] (position p -> index nat_of(p, n)), in which output p of
// the first half and output p of the second half are mirror images. Each
// product then runs K/2 per tile (its rows lie in one half), and its epilogue
// folds its N direction for the next product:
//   FOLD 1: N in natural order; the CTA takes the 32-column tile at a and its
//           mirror tile N - 32 - a (reversed), writes sums / differences;
//   FOLD 2: N grouped; tiles at a and N/2 + a; multiplies by f (gathered at
//           the natural indices), then writes sums / differences;
//   FOLD 3: as 2 without f; rows written to their natural index;
//   FOLD 4: N natural (one 64-column tile); rows written to their natural index
//           (the last product: z = d o C, r^T z).
__device__ __forceinline__ int nat_of(int p, int n) {
    const int h = n >> 1;
    if (p < h) return p == 0 ? 0 : 2 * p - 1;
    const int a = p - h;
    return a == 0 ? n - 1 : n - 2 * a;
}

template <typename OpT, int BN, int STAGES, int EPI, int FOLD = 0>
__global__ void __launch_bounds__(kTcThreads, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
               int K, TcEpi ea) {
    static_assert(BN % 32 == 0 && BN >= 32 && BN <= 256, "BN");
    static_assert(FOLD == 0 || BN == 64, "folded products use 64-column tiles");
    static_assert(FOLD != 4 || EPI == EPI_POST, "FOLD 4 is the last product");
    static_assert(FOLD != 2 || EPI == EPI_SCALE, "FOLD 2 carries the spectral divide");
    static_assert((FOLD != 1 && FOLD != 3) || EPI == EPI_STORE, "FOLD 1 and 3 store");
    constexpr bool kPaired = FOLD >= 1 && FOLD <= 3;
    using L = TcSmem<BN, STAGES, EPI>;
    constexpr int NPRE = pre_arrays<BN, EPI>();
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + L::kBarOffset);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    int* flags = reinterpret_cast<int*>(tmem_slot + 1);        // [0]: skip (solve done), [1]: timeout
    double* wsum = reinterpret_cast<double*>(tmem_slot + 4);   // 4 epilogue warp partials

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int BK = kRowBytes / (int)sizeof(OpT);   // K elements per stage
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
    // folded: half the K range, the second half for tiles in the second half of M
    const int kh = FOLD ? K / 2 : K;
    const int kofs = (FOLD && m0 >= M / 2) ? kh : 0;
    const int nk = (kh + BK - 1) / BK;
    // paired tiles: the 32 B rows at na and the 32 at nb (FOLD 1: mirror, reversed; 2, 3: N/2 + na)
    const int na = kPaired ? blockIdx.x * 32 : n0;
    const int nb = FOLD == 1 ? N - 32 - na : N / 2 + na;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tma_prefetch_map(&mapA);
        tma_prefetch_map(&mapB);
        flags[1] = 0;
    }
    if (warp == 1) tmem_alloc(tmem_slot, tmem_cols<BN>());
    // everything below reads what earlier kernels in the stream write
    pdl_wait();
    if (threadIdx.x == 0) flags[0] = (ea.st && ea.st->done) ? 1 : 0;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const bool skip = flags[0] != 0;

    if (!skip && warp == 0 && lane == 0) {
        // loader
        int issued = 0;
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u)) {
                flags[1] = 1;
                break;
            }
            unsigned char* sa = base + s * L::kStageBytes;
            mbar_expect_tx(&full[s], (uint32_t)L::kStageBytes);
            tma_load_2d(sa, &mapA, &full[s], kb * BK, m0);
            if (kPaired) {   // mapB's box is 32 rows
                tma_load_2d(sa + L::kABytes, &mapB, &full[s], kofs + kb * BK, na);
                tma_load_2d(sa + L::kABytes + 32 * kRowBytes, &mapB, &full[s], kofs + kb * BK, nb);
            } else {
                tma_load_2d(sa + L::kABytes, &mapB, &full[s], kofs + kb * BK, n0);
            }
            issued = kb + 1;
        }
        // no copy may still be landing in shared memory when the CTA exits
        for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
            if (!mbar_wait(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1u)) flags[1] = 1;
    } else if (!skip && warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_of<BN, sizeof(OpT) == 2 ? 1u : 2u>();
        bool ok = true;
        int last = -1;
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
            if (!mbar_wait(&full[s], ph)) {
                flags[1] = 1;
                ok = false;
                break;
            }
            last = kb;
            tc_fence_after();
            const uint32_t sa = smem_u32(base + s * L::kStageBytes);
            const uint64_t da = sw128_desc(sa), db = sw128_desc(sa + L::kABytes);
#pragma unroll
            for (int kk = 0; kk < kRowBytes / 32; ++kk)   // 32 bytes of K = 2 descriptor units per step
                umma<OpT>(tmem, da + 2 * kk, db + 2 * kk, idesc, (kb | kk) != 0 ? 1u : 0u);
            umma_commit(&empty[s]);
        }
        if (ok) umma_commit(done);
        // no MMA may still be running when the tensor memory is released
        if (ok) {
            if (!mbar_wait(done, 0)) flags[1] = 1;
        } else if (last >= 0 && !mbar_wait(&empty[last % STAGES], (uint32_t)(last / STAGES) & 1u)) {
            flags[1] = 1;
        }
    } else if (!skip && warp >= 2) {
        // epilogue: thread = row m0 + 32 q + lane of the tile, q = warp % 4 (its TMEM lane quarter)
        const int q = warp & 3;
        const int m = m0 + 32 * q + lane;
        float* pre = reinterpret_cast<float*>(base + L::kPreOffset);   // NPRE arrays of BM x kPreStride
        if (NPRE > 0) {
            // while the main loop runs: this warp stages its 32 rows of f (SCALE) or d and r
            // (POST), one row at a time with coalesced reads; zeros outside the matrix
            const float* src0 = EPI == EPI_SCALE ? ea.f : ea.d;
            // unrolled so that the loads of several rows are in flight together
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr) {
                const int row = 32 * q + rr;
                // folded products read f, d, r at the natural row and (FOLD 2) natural columns
                const int gm = FOLD ? nat_of(m0 + row, M) : m0 + row;
#pragma unroll
                for (int h = 0; h < BN / 32; ++h) {
                    const int c = lane + 32 * h;
                    const int gn = FOLD == 2 ? nat_of(h == 0 ? na + lane : nb + lane, N) : n0 + c;
                    const bool in = gm < M && gn < N;
                    const size_t off = (size_t)gm * N + gn;
                    pre[row * L::kPreStride + c] = (in && src0) ? __ldg(src0 + off) : (src0 ? 0.0f : 1.0f);
                    if (NPRE > 1)
                        pre[BM * L::kPreStride + row * L::kPreStride + c] = (in && ea.r) ? __ldg(ea.r + off) : 0.0f;
                }
            }
            __syncwarp();
        }
        const bool ok = mbar_wait(done, 0);
        if (!ok) flags[1] = 1;
        tc_fence_after();
        double part = 0.0;
        if (ok && kPaired) {
            // both 32-column halves of the accumulator, then sums / differences of mirror pairs
            float va[32], vb[32];
            tmem_ld32(tmem + ((uint32_t)(32 * q) << 16), va);
            tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 32u, vb);
            if (FOLD == 2) {
                const float* prow = pre + (32 * q + lane) * L::kPreStride;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    va[i] *= prow[i];
                    vb[i] *= prow[32 + i];
                }
            }
            float sv[32], dv[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float b = FOLD == 1 ? vb[31 - i] : vb[i];   // the mirror of column na + i
                sv[i] = va[i] + b;
                dv[i] = va[i] - b;
            }
            if (na == 0) {   // slot 0 of each half: the raw endpoint values
                sv[0] = va[0];
                dv[0] = FOLD == 1 ? vb[31] : vb[0];
            }
            const int row = FOLD == 3 ? nat_of(m, M) : m;
            OpT* o = reinterpret_cast<OpT*>(ea.out) + (size_t)row * ea.ldo;
            store_row32(o + na, sv);
            store_row32(o + N / 2 + na, dv);
        } else if (ok) {
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
                const int n = n0 + c0;
                if (m >= M || n >= N) continue;
                // whole 32-column chunks of rows whose elementwise operands (row stride N)
                // start on 16 bytes move as float4; the rest element by element
                const bool full_cols = n + 32 <= N;
                const bool vec = full_cols && (N % 4) == 0;
                const float* prow = pre + (32 * q + lane) * L::kPreStride + c0;   // staged row (NPRE > 0)
                if (EPI == EPI_STORE || EPI == EPI_SCALE) {
                    OpT* o = reinterpret_cast<OpT*>(ea.out) + (size_t)m * ea.ldo + n;
                    if (EPI == EPI_SCALE && NPRE > 0) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] *= prow[i];
                    } else if (EPI == EPI_SCALE) {
                        const float* f = ea.f + (size_t)m * N + n;
                        if (vec) {
                            float fv[32];
                            load_row32(f, fv);
#pragma unroll
                            for (int i = 0; i < 32; ++i) v[i] *= fv[i];
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                if (full_cols || n + i < N) v[i] *= __ldg(f + i);
                        }
                    }
                    if (full_cols) {
                        store_row32(o, v);
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (n + i < N) store_one(o + i, v[i]);
                    }
                } else {
                    float* o = reinterpret_cast<float*>(ea.out) + (size_t)(FOLD == 4 ? nat_of(m, M) : m) * ea.ldo + n;
                    const float* d = ea.d ? ea.d + (size_t)m * N + n : nullptr;
                    const float* r = ea.r + (size_t)m * N + n;
                    float acc = 0.0f;
                    if (NPRE > 1) {
                        // d (1 where there is none) and r from the staged rows
                        const float* rrow = prow + BM * L::kPreStride;
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] *= prow[i];
                        if (full_cols && (ea.ldo % 4) == 0 && ((uintptr_t)o & 15u) == 0) {
                            store_row32(o, v);
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                if (n + i < N) o[i] = v[i];
                        }
                        if (ea.st) {
#pragma unroll
                            for (int i = 0; i < 32; ++i) acc += rrow[i] * v[i];
                        }
                    } else if (vec && (ea.ldo % 4) == 0) {
                        if (d) {
                            float dv[32];
                            load_row32(d, dv);
#pragma unroll
                            for (int i = 0; i < 32; ++i) v[i] *= dv[i];
                        }
                        store_row32(o, v);
                        if (ea.st) {
                            float rv[32];
                            load_row32(r, rv);
#pragma unroll
                            for (int i = 0; i < 32; ++i) acc += rv[i] * v[i];
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            if (n + i < N) {
                                const float z = d ? v[i] * __ldg(d + i) : v[i];
                                o[i] = z;
                                if (ea.st) acc += __ldg(r + i) * z;
                            }
                        }
                    }
                    part += (double)acc;
                }
            }
        }
        if (EPI == EPI_POST && ea.st) {
            // r^T z: warp sums, then the tile's sum into its slot; the last tile finishes
            part = warp_sum(part);
            if (lane == 0) wsum[q] = part;
            epi_bar();
            if (warp == 2 && lane == 0) {
                const int total = gridDim.x * gridDim.y, slot = blockIdx.y * gridDim.x + blockIdx.x;
                ea.red[slot] = wsum[0] + wsum[1] + wsum[2] + wsum[3];
                __threadfence();
                const unsigned int t = atomicAdd(ea.ticket, 1u);
                flags[2] = (t == (unsigned int)(total - 1)) ? 1 : 0;
            }
            epi_bar();
            if (warp == 2 && flags[2]) {
                __threadfence();
                const int total = gridDim.x * gridDim.y;
                double acc = 0.0;
                for (int i = lane; i < total; i += 32) acc += __ldcg(ea.red + i);
                acc = warp_sum(acc);
                if (lane == 0) {
                    *ea.ticket = 0u;
                    if (!flags[1]) finish_rho(ea.st, acc);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (flags[1] && threadIdx.x == 0) {
        if (ea.err) atomicExch(ea.err, (int)TVD_ETIMEOUT);
        if (ea.st) {
            ea.st->status = TVD_ETIMEOUT;
            ea.st->done = 1;
        }
    }
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols<BN>());
    }
}

// ---------------------------------------------------------------- host side

// cuTensorMapEncodeTiled from the driver (no link against libcuda).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// Tensor map of a row-major matrix of elem_bytes-sized elements (2: bf16, 4:
// float), rows x inner, row stride ld elements (ld * elem_bytes a multiple of
// 16), read in boxes of one 128-byte row of K by box_rows rows with the
// 128-byte swizzle; reads outside the matrix return zeros.
inline bool make_tc_map(CUtensorMap* map, const void* ptr, int elem_bytes, int inner, int rows, int ld,
                        int box_rows) {
    auto enc = tensor_map_encoder();
    if (!enc || ((size_t)ld * elem_bytes) % 16 != 0 || ((uintptr_t)ptr & 15u) != 0) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * elem_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / elem_bytes), (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(map, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
               const_cast<void*>(ptr), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Raise the kernel's dynamic shared-memory limit (once per device; plans call
// this at set-up, before any stream capture), then launch with programmatic
// stream serialisation.
template <typename OpT, int BN, int STAGES, int EPI, int FOLD = 0>
inline cudaError_t tc_gemm_prepare() {
    static std::mutex mu;
    static bool done[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(tc_gemm_kernel<OpT, BN, STAGES, EPI, FOLD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TcSmem<BN, STAGES, EPI>::kBytes);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

template <typename OpT, int BN, int STAGES, int EPI, int FOLD = 0>
inline cudaError_t launch_tc_gemm(const CUtensorMap& mapA, const CUtensorMap& mapB, int M, int N, int K,
                                  const TcEpi& ea, cudaStream_t s) {
    const cudaError_t attr = tc_gemm_prepare<OpT, BN, STAGES, EPI, FOLD>();
    if (attr != cudaSuccess) return attr;
    const dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    return launch_pdl(tc_gemm_kernel<OpT, BN, STAGES, EPI, FOLD>, grid, dim3(kTcThreads),
                      (size_t)TcSmem<BN, STAGES, EPI>::kBytes, s, mapA, mapB, M, N, K, ea);
}

}  // namespace tc
}  // namespace tvd
