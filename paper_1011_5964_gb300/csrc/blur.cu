// Blur operator H under reflective / anti-reflective boundary conditions and
// its exact transpose (Sec. 2 of the paper).
//
//   (H x)_{ij} = sum_{a,b} h_{a,b} x~_{i-a, j-b}, x~ the BC extension of x:
//     AR  (eq. (anti1d), corners of Sec. 2): x~_{-s} = 2 x_0 - x_s,
//         x~_{n-1+s} = 2 x_{n-1} - x_{n-1-s}, separable in 2D;
//     R:  x~_{-s} = x_{s-1}, x~_{n-1+s} = x_{n-s}.
//
// Forward: one CTA computes a 32x32 output tile from a shared-memory tile of
// x~ (tile + PSF halo), built on the fly from x; the extended image is never
// materialised.
//
// Transpose, AR: H = C E (convolution after extension), so H^T = E^T C^T. For a
// quadrantally symmetric h the folds of E^T cancel the boundary lines of y at
// interior outputs, which become a plain convolution of the odd extension
//   y^_{s} = y_s (1 <= s <= n-2), y^_0 = y^_{n-1} = 0,
//   y^_{-s} = -y_s, y^_{n-1+s} = -y_{n-1-s},
// applied separately along rows and columns. The first/last row and column
// of H^T y are tail-weighted sums of y near that border:
//   row 0:   sum_{i=0..m_r} sum_b crow[i][b] yc^_{i, l+b},
//            crow[i][b] = h_{i,b} + 2 sum_{s>i} h_{s,b}
//   corner:  sum_{i,j} ccor[i][j] y_{ij},
//            ccor[i][j] = h_ij + 2 sum_{s>i} h_sj + 2 sum_{t>j} h_it + 4 sum_{s>i,t>j} h_st
// (yc^ = odd extension along the column index only). These weights are built
// on the host from the PSF.
// Transpose, R: H^T = H for a symmetric PSF (Sec. 3.1).
#include "common.cuh"

#include <algorithm>
#include <mutex>

namespace tvd {

enum { EXT_AR = 0, EXT_R = 1, EXT_ODD = 2 };

constexpr int BTW = 32;         // output tile width (one warp across)
constexpr int RB = 8;           // consecutive output rows per thread (register window)
constexpr int BTH = RB * (kThreads / 32);   // output tile height: 64 rows

// Reads the image to be extended: x itself, or the new CG direction
// z + beta p_old (z alone on a fresh start) when the blur is fused with the
// direction update.
template <typename T, bool PUP>
struct Src {
    const T* __restrict__ x;     // x, or z
    const T* __restrict__ pold;
    T beta;
    bool fresh;
    __device__ __forceinline__ T operator[](size_t i) const {
        if (!PUP) return x[i];
        return fresh ? x[i] : x[i] + beta * pold[i];
    }
};

template <typename T, int EXT, typename S>
__device__ __forceinline__ T ext_value(const S& x, int I, int J, int nr, int nc, int mr, int mc) {
    if (I < -mr || I >= nr + mr || J < -mc || J >= nc + mc) return T(0);
    if (EXT == EXT_R) {
        int ri = I < 0 ? -I - 1 : (I >= nr ? 2 * nr - 1 - I : I);
        int ci = J < 0 ? -J - 1 : (J >= nc ? 2 * nc - 1 - J : J);
        return x[(size_t)ri * nc + ci];
    } else if (EXT == EXT_ODD) {
        if (I == 0 || I == nr - 1 || J == 0 || J == nc - 1) return T(0);
        T sg = T(1);
        int ri = I, ci = J;
        if (I < 0) { ri = -I; sg = -sg; } else if (I > nr - 1) { ri = 2 * (nr - 1) - I; sg = -sg; }
        if (J < 0) { ci = -J; sg = -sg; } else if (J > nc - 1) { ci = 2 * (nc - 1) - J; sg = -sg; }
        return sg * x[(size_t)ri * nc + ci];
    } else {
        int ri0, ri1; T cr0, cr1;
        if (I < 0) { ri0 = 0; cr0 = T(2); ri1 = -I; cr1 = T(-1); }
        else if (I >= nr) { ri0 = nr - 1; cr0 = T(2); ri1 = 2 * (nr - 1) - I; cr1 = T(-1); }
        else { ri0 = I; cr0 = T(1); ri1 = I; cr1 = T(0); }
        int ci0, ci1; T cc0, cc1;
        if (J < 0) { ci0 = 0; cc0 = T(2); ci1 = -J; cc1 = T(-1); }
        else if (J >= nc) { ci0 = nc - 1; cc0 = T(2); ci1 = 2 * (nc - 1) - J; cc1 = T(-1); }
        else { ci0 = J; cc0 = T(1); ci1 = J; cc1 = T(0); }
        T v = cr0 * cc0 * x[(size_t)ri0 * nc + ci0];
        if (cc1 != T(0)) v += cr0 * cc1 * x[(size_t)ri0 * nc + ci1];
        if (cr1 != T(0)) {
            v += cr1 * cc0 * x[(size_t)ri1 * nc + ci0];
            if (cc1 != T(0)) v += cr1 * cc1 * x[(size_t)ri1 * nc + ci1];
        }
        return v;
    }
}

struct FuseArgs {
    double alpha;
    CgState* st;          // non-null: return at once when st->done
    double* red;
    unsigned int* ticket;
    int reduce;           // reduce p^T q (FUSE only)
    int total_blocks;     // blocks contributing to the reduction (tile + border)
    int slot0;            // first reduction slot of this kernel
    int finish_here;      // this kernel holds the last contributing blocks
};

// Output tile kernel. EXT selects the extension of the input; for EXT_ODD only
// interior outputs (1..n-2 in both directions) are written. With FUSE, the
// output is q = conv + alpha L(w) pv and p^T q is reduced.
// Each thread computes RB consecutive output rows of one column. For every PSF
// column offset b it walks the rows a of that column's tap range, keeping the
// RB input values it needs in registers and shifting them by one row per tap,
// so one shared-memory load feeds RB multiply-adds.
template <typename T, int EXT, bool FUSE, bool PUP>
__device__ __forceinline__ void tile_body(int bx, int by, int gx, const T* __restrict__ x, T* __restrict__ y, int nr,
                                          int nc, int mr, int mc, const T* __restrict__ hdense,
                                          const int* __restrict__ arange, const int* __restrict__ runs,
                                          const T* __restrict__ runv, int nruns, const T* __restrict__ w, T* p0,
                                          T* p1, const FuseArgs& fa) {
    // FUSE: the direction of this iteration; PUP: old and new direction buffers
    const int pb = fa.st ? fa.st->pbuf : 0;
    const T* pv = fa.st ? (pb ? p0 : p1) : p0;
    const T* pold = pb ? p1 : p0;
    T* pnew = pb ? p0 : p1;
    const Src<T, PUP> src{x, pold, PUP ? T(fa.st->beta) : T(0), PUP ? fa.st->fresh != 0 : true};
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TW = BTW + 2 * mc, TH = BTH + 2 * mr;
    const int PW = 2 * mc + 1, PH = 2 * mr + 1;
    constexpr int LSW = BTW + 2, LSH = BTH + 2;      // w / p tiles with a 1-pixel halo
    T* tile = reinterpret_cast<T*>(smem_raw);
    T* ptile = tile + TW * TH;                       // PUP: p_old tile (inside tiles)
    T* sw = ptile + (PUP ? TW * TH : 0);             // FUSE: w tile
    T* sp = sw + (FUSE ? LSW * LSH : 0);             // FUSE: p tile
    T* sh = sp + (FUSE ? LSW * LSH : 0);             // dense PSF, PH x PW
    T* pre = sh + PH * PW;                           // runs: row prefix sums, TH x (TW + 1)
    T* srv = pre + (nruns ? TH * (TW + 1) : 0);      // runs: values
    int* sr = reinterpret_cast<int*>(srv + nruns);   // per column offset: first and last tap row
    int* srun = sr + 2 * PW;                         // runs: (a, first b, last b)
    const int r0 = by * BTH - mr, c0 = bx * BTW - mc;
    // stage the extended input tile: a plain asynchronous copy where the tile
    // lies inside the image (away from the boundary lines for EXT_ODD), the
    // BC extension computed on the fly elsewhere
    const bool inside = (EXT == EXT_ODD) ? (r0 >= 1 && c0 >= 1 && r0 + TH <= nr - 1 && c0 + TW <= nc - 1)
                                         : (r0 >= 0 && c0 >= 0 && r0 + TH <= nr && c0 + TW <= nc);
    if (inside) {
        for (int idx = threadIdx.x; idx < TW * TH; idx += blockDim.x) {
            const int li = idx / TW, lj = idx - li * TW;
            const size_t o = (size_t)(r0 + li) * nc + (c0 + lj);
            cp_async_elem(tile + idx, x + o);
            if (PUP && !src.fresh) cp_async_elem(ptile + idx, pold + o);
        }
    }
    if (FUSE) {
        const int i0 = by * BTH - 1, j0 = bx * BTW - 1;
        for (int idx = threadIdx.x; idx < LSW * LSH; idx += blockDim.x) {
            const int li = idx / LSW, lj = idx - li * LSW;
            const int i = i0 + li, j = j0 + lj;
            if (i >= 0 && i < nr && j >= 0 && j < nc) {
                cp_async_elem(sw + idx, w + (size_t)i * nc + j);
                cp_async_elem(sp + idx, pv + (size_t)i * nc + j);
            }
        }
    }
    for (int k = threadIdx.x; k < PH * PW; k += blockDim.x) sh[k] = hdense[k];
    for (int k = threadIdx.x; k < 2 * PW; k += blockDim.x) sr[k] = arange[k];
    for (int k = threadIdx.x; k < nruns; k += blockDim.x) {
        srv[k] = runv[k];
        srun[3 * k] = runs[3 * k];
        srun[3 * k + 1] = runs[3 * k + 1];
        srun[3 * k + 2] = runs[3 * k + 2];
    }
    if (!inside) {
#pragma unroll 4
        for (int idx = threadIdx.x; idx < TW * TH; idx += blockDim.x) {
            const int li = idx / TW, lj = idx - li * TW;
            tile[idx] = ext_value<T, EXT>(src, r0 + li, c0 + lj, nr, nc, mr, mc);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (PUP && inside && !src.fresh) {
        for (int idx = threadIdx.x; idx < TW * TH; idx += blockDim.x) tile[idx] += src.beta * ptile[idx];
        __syncthreads();
    }
    if (PUP) {
        // this block's outputs of the new direction (plain values: inside the image)
        for (int idx = threadIdx.x; idx < BTW * BTH; idx += blockDim.x) {
            const int li = idx / BTW, lj = idx - li * BTW;
            const int i = by * BTH + li, j = bx * BTW + lj;
            if (i < nr && j < nc) pnew[(size_t)i * nc + j] = tile[(li + mr) * TW + (lj + mc)];
        }
    }
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    T acc[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) acc[k] = T(0);
    const int row0 = ty * RB + mr;                   // tile row of output row 0 at a = 0
    if (nruns) {
        // PSF rows made of constant runs: sum of a run of x~ along a tile row is a
        // difference of that row's prefix sums, pre[r][c] = sum_{c' < c} tile[r][c']
        const int PS = TW + 1;
        for (int r = threadIdx.x >> 5; r < TH; r += blockDim.x >> 5) {
            T carry = T(0);
            if (tx == 0) pre[r * PS] = T(0);
            for (int c0 = 0; c0 < TW; c0 += 32) {
                const int c = c0 + tx;
                T v = c < TW ? tile[r * TW + c] : T(0);
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const T u = __shfl_up_sync(0xffffffffu, v, o);
                    if (tx >= o) v += u;
                }
                v += carry;
                if (c < TW) pre[r * PS + c + 1] = v;
                carry = __shfl_sync(0xffffffffu, v, 31);
            }
        }
        __syncthreads();
        for (int q = 0; q < nruns; ++q) {
            const int a = srun[3 * q], bs = srun[3 * q + 1], be = srun[3 * q + 2];
            const T hv = srv[q];
            // outputs at tile column tx + mc read x~ columns tx + mc - b, b in [bs, be]
            const T* p = pre + (row0 - a) * PS + tx + mc;
#pragma unroll
            for (int k = 0; k < RB; ++k) acc[k] += hv * (p[k * PS + 1 - bs] - p[k * PS - be]);
        }
    } else
    for (int b = -mc; b <= mc; ++b) {
        const int lo = sr[2 * (b + mc)], hi = sr[2 * (b + mc) + 1];
        if (lo > hi) continue;
        const T* col = tile + (tx + mc - b);
        const T* hb = sh + (b + mc);
        // output k at tap a reads tile row row0 + k - a
        T win[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) win[k] = col[(row0 + k - hi) * TW];
        for (int a = hi;; --a) {
            const T hv = hb[(a + mr) * PW];
#pragma unroll
            for (int k = 0; k < RB; ++k) acc[k] += hv * win[k];
            if (a == lo) break;
#pragma unroll
            for (int k = 0; k < RB - 1; ++k) win[k] = win[k + 1];
            win[RB - 1] = col[(row0 + RB - 1 - (a - 1)) * TW];
        }
    }
    T part = T(0);   // per-thread partial of p^T q in the kernel's type
    const int j = bx * BTW + tx;
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        const int i = by * BTH + ty * RB + k;
        if (i >= nr || j >= nc) continue;
        if (EXT == EXT_ODD && (i == 0 || i == nr - 1 || j == 0 || j == nc - 1)) continue;
        T out = acc[k];
        if (FUSE) {
            // alpha L(w) p from the staged tiles (5-point stencil, zero Neumann)
            const int o = (ty * RB + k + 1) * LSW + (tx + 1);
            const T pc = sp[o], wc = sw[o];
            T l = T(0);
            if (i < nr - 1) l += wc * (pc - sp[o + LSW]);
            if (j < nc - 1) l += wc * (pc - sp[o + 1]);
            if (i > 0) l += sw[o - LSW] * (pc - sp[o - LSW]);
            if (j > 0) l += sw[o - 1] * (pc - sp[o - 1]);
            out += T(fa.alpha) * l;
            part += pc * out;
        }
        y[(size_t)i * nc + j] = out;
    }
    if (FUSE && fa.reduce) {
        const int slot = fa.slot0 + by * gx + bx;
        double s;
        if (block_reduce_last((double)part, fa.red, fa.ticket, slot, fa.total_blocks, &s) && threadIdx.x == 0 &&
            fa.finish_here)
            finish_pq(fa.st, s);
    }
}

// Stencil paths: the general tile stencil (dense taps or row runs), the flat
// PSF on a centred convex support, and the flat disk of radius DR.
enum { PATH_TILE = 0, PATH_FLAT = 1, PATH_DISK = 2 };

// ---------------------------------------------------------------- flat stencil
//
// For a flat PSF, h_{a,b} = v on a support that is symmetric in both axes and
// whose rows and columns are runs centred on 0 (the out-of-focus disk of
// Sec. 5: |b| <= w_|a| exactly when |a| <= g_|b|),
//   y_ij = v sum_{|b| <= m_c} C_{g_|b|}(i, j - b),   C_g(i, c) = sum_{|a| <= g} x~_{i-a, c}.
// Vertical pass: a thread walks one staged column c of the block over 16
// output rows with a register window of the 16 + 2 FMAXM extended values it
// needs and writes the centred vertical sums C_0 .. C_FMAXM of every row to
// shared memory (two adds per level). Horizontal pass: a thread owns one
// output column and FR rows and adds C_{g_|b|}(i, j - b) over the support's
// columns. About 2 (FMAXM + 1) shared-memory accesses per extended pixel and
// 2 (2 m_c + 1) per output, against one load and one multiply-add per tap
// for the direct stencil.
constexpr int FMAXM = 8;                         // largest PSF half-width of the flat path
constexpr int FBW = 64;                          // output columns per block
constexpr int FSEG = 16;                         // output rows per vertical-pass thread
constexpr int FBH = 32;                          // output rows per block
constexpr int FR = FBH * FBW / kThreads;         // output rows per horizontal-pass thread: 8
constexpr int FCS = FBW + 2 * FMAXM;             // shared row stride of the C arrays

template <typename T>
__host__ __device__ constexpr size_t flat_smem_bytes() {
    return (size_t)(FMAXM + 1) * FBH * FCS * sizeof(T) + (2 * FMAXM + 1) * sizeof(int);
}

template <typename T, int EXT, bool FUSE, bool PUP>
__device__ __forceinline__ void flat_body(int bx, int by, int gx, const T* __restrict__ x, T* __restrict__ y, int nr,
                                          int nc, int mr, int mc, const int* __restrict__ colh, T v,
                                          const T* __restrict__ w, T* p0, T* p1, const FuseArgs& fa) {
    const int pb = fa.st ? fa.st->pbuf : 0;
    const T* pv = fa.st ? (pb ? p0 : p1) : p0;
    const T* pold = pb ? p1 : p0;
    T* pnew = pb ? p0 : p1;
    const Src<T, PUP> src{x, pold, PUP ? T(fa.st->beta) : T(0), PUP ? fa.st->fresh != 0 : true};
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* C = reinterpret_cast<T*>(smem_raw);           // [g][row][FCS]: C_g of the block's rows
    int* sh = reinterpret_cast<int*>(C + (FMAXM + 1) * FBH * FCS);   // column heights g_|b|, b = -mc..mc
    const int i0 = by * FBH, j0 = bx * FBW;
    const int TW = FBW + 2 * mc;                     // staged columns j0 - mc .. j0 + FBW + mc - 1
    for (int k = threadIdx.x; k < 2 * mc + 1; k += blockDim.x) sh[k] = colh[k];
    // vertical pass: task = (staged column, 16-row segment)
    const int ntask = TW * (FBH / FSEG);
    if (threadIdx.x < ntask) {
        const int cl = threadIdx.x % TW, seg = threadIdx.x / TW;
        const int J = j0 - mc + cl;
        const int ib = i0 + seg * FSEG;              // first output row of the segment
        const bool inside = (EXT == EXT_ODD)
                                ? (ib - FMAXM >= 1 && ib + FSEG + FMAXM <= nr - 1 && J >= 1 && J <= nc - 2)
                                : (ib - FMAXM >= 0 && ib + FSEG + FMAXM <= nr && J >= 0 && J < nc);
        T win[FSEG + 2 * FMAXM];
        if (inside) {
            const size_t o = (size_t)(ib - FMAXM) * nc + J;
#pragma unroll
            for (int t = 0; t < FSEG + 2 * FMAXM; ++t) win[t] = src[o + (size_t)t * nc];
        } else {
#pragma unroll
            for (int t = 0; t < FSEG + 2 * FMAXM; ++t) win[t] = ext_value<T, EXT>(src, ib - FMAXM + t, J, nr, nc, mr, mc);
        }
        if (PUP && cl >= mc && cl < mc + FBW && J < nc) {
            // this block's outputs of the new direction z + beta p_old (plain values: inside the image)
#pragma unroll
            for (int t = 0; t < FSEG; ++t)
                if (ib + t < nr) pnew[(size_t)(ib + t) * nc + J] = win[t + FMAXM];
        }
        T* cw = C + (size_t)(seg * FSEG) * FCS + cl;
#pragma unroll
        for (int t = 0; t < FSEG; ++t) {
            T acc = win[t + FMAXM];
            cw[t * FCS] = acc;
#pragma unroll
            for (int g = 1; g <= FMAXM; ++g) {
                acc += win[t + FMAXM - g] + win[t + FMAXM + g];
                cw[(size_t)g * FBH * FCS + t * FCS] = acc;
            }
        }
    }
    __syncthreads();
    // horizontal pass: column tx, rows ty * FR .. + FR - 1
    const int tx = threadIdx.x % FBW, ty = threadIdx.x / FBW;
    T acc[FR];
#pragma unroll
    for (int k = 0; k < FR; ++k) acc[k] = T(0);
    for (int b = -mc; b <= mc; ++b) {
        const int g = sh[b + mc];
        if (g < 0) continue;
        const T* cr = C + (size_t)g * FBH * FCS + (size_t)(ty * FR) * FCS + (tx + mc - b);
#pragma unroll
        for (int k = 0; k < FR; ++k) acc[k] += cr[k * FCS];
    }
    T part = T(0);   // per-thread partial of p^T q in the kernel's type
    const int j = j0 + tx;
#pragma unroll
    for (int k = 0; k < FR; ++k) {
        const int i = i0 + ty * FR + k;
        if (i >= nr || j >= nc) continue;
        if (EXT == EXT_ODD && (i == 0 || i == nr - 1 || j == 0 || j == nc - 1)) continue;
        T out = v * acc[k];
        if (FUSE) {
            // alpha L(w) p (5-point stencil, zero Neumann), read through the L1 cache
            out += T(fa.alpha) * lap_at(w, pv, i, j, nr, nc);
            part += __ldg(pv + (size_t)i * nc + j) * out;
        }
        y[(size_t)i * nc + j] = out;
    }
    if (FUSE && fa.reduce) {
        const int slot = fa.slot0 + by * gx + bx;
        double sres;
        if (block_reduce_last((double)part, fa.red, fa.ticket, slot, fa.total_blocks, &sres) && threadIdx.x == 0 &&
            fa.finish_here)
            finish_pq(fa.st, sres);
    }
}

// ---------------------------------------------------------------- disk stencil
//
// The flat disk of radius R (h_{a,b} = v where a^2 + b^2 <= R^2, the
// out-of-focus PSF of Sec. 5) has column heights g_b = floor(sqrt(R^2 - b^2))
// known at compile time, so
//   y_ij = v sum_{|b| <= R} C_{g_b}(i, j - b),   C_g(i, c) = sum_{|a| <= g} x~_{i-a, c}.
// A block is two groups of 128 threads; each thread owns one column of a
// 128-column window (114 outputs and R halo columns on each side) and DROWS
// rows of one group. It keeps its column's DROWS + 2R extended values in
// registers and forms the vertical sums C_g of each row by nested pair
// additions; the sums other columns need (the distinct heights below g_0) go to
// a double-buffered shared row, one barrier per row, and each output thread adds
// its 14 neighbours' terms from there.
constexpr int DR = 7;                            // disk radius of the specialised path
constexpr int DCOLS = 128;                       // window columns of a row group
constexpr int DOUT = DCOLS - 2 * DR;             // output columns per block
constexpr int DROWS = 16;                        // output rows per row group
constexpr int DGROUPS = kThreads / DCOLS;        // row groups per block
constexpr int DBW = DOUT, DBH = DGROUPS * DROWS; // block tile: 114 x 32 outputs
constexpr int DNG = 5;                           // shared heights g_b, b = 1..R: 6 (b <= 3), 5, 4, 3, 0

__host__ __device__ constexpr int disk_height(int b) {
    int g = 0;
    while ((g + 1) * (g + 1) + b * b <= DR * DR) ++g;
    return g;
}

// slot of the shared row that holds C_{g_b} (b = 1..R)
__host__ __device__ constexpr int disk_slot(int b) {
    return b <= 3 ? 0 : b - 3;
}

// x~ at (I, J) near the image border: the extension of Sec. 2 (AR: reflection
// through the boundary value; R: mirror; ODD: the odd extension used by the AR
// transpose), from at most four image values.
template <typename T, int EXT, typename S>
__device__ __forceinline__ T ext_at(const S& x, int I, int J, int nr, int nc) {
    return ext_value<T, EXT>(x, I, J, nr, nc, DR, DR);
}

template <typename T, int EXT, bool FUSE, bool PUP>
__device__ __forceinline__ void disk_body(int bx, int by, int gx, const T* __restrict__ x, T* __restrict__ y, int nr,
                                          int nc, T v, const T* __restrict__ w, T* p0, T* p1, const FuseArgs& fa) {
    static_assert(disk_height(1) == 6 && disk_height(3) == 6 && disk_height(4) == 5 && disk_height(5) == 4 &&
                      disk_height(6) == 3 && disk_height(7) == 0,
                  "the shared-row slots assume the heights of the radius-7 disk");
    __shared__ T crow_buf[2][DGROUPS][DNG][DCOLS];
    const int pb = fa.st ? fa.st->pbuf : 0;
    const T* pv = fa.st ? (pb ? p0 : p1) : p0;
    const T* pold = pb ? p1 : p0;
    T* pnew = pb ? p0 : p1;
    const Src<T, PUP> src{x, pold, PUP ? T(fa.st->beta) : T(0), PUP ? fa.st->fresh != 0 : true};
    const int col = threadIdx.x % DCOLS, grp = threadIdx.x / DCOLS;
    const int jo = bx * DBW;                          // first output column of the block
    const int i0 = by * DBH + grp * DROWS;            // first output row of the group
    const int J = jo - DR + col;                      // this thread's column
    const bool out_col = col >= DR && col < DR + DOUT && J < nc;
    // the window rows i0 - DR .. i0 + DROWS - 1 + DR of column J
    const bool inside = (EXT == EXT_ODD) ? (i0 - DR >= 1 && i0 + DROWS + DR <= nr - 1 && J >= 1 && J <= nc - 2)
                                         : (i0 - DR >= 0 && i0 + DROWS + DR <= nr && J >= 0 && J < nc);
    T win[DROWS + 2 * DR];
    if (inside) {
        const size_t o = (size_t)(i0 - DR) * nc + J;
#pragma unroll
        for (int t = 0; t < DROWS + 2 * DR; ++t) win[t] = src[o + (size_t)t * nc];
    } else {
#pragma unroll
        for (int t = 0; t < DROWS + 2 * DR; ++t) win[t] = ext_at<T, EXT>(src, i0 - DR + t, J, nr, nc);
    }
    T part = T(0);
    const size_t o0 = (size_t)i0 * nc + J;            // (i0, J); row t at o0 + t nc
#pragma unroll
    for (int t = 0; t < DROWS; ++t) {
        const int i = i0 + t;
        const size_t oi = o0 + (size_t)t * nc;
        if (PUP && out_col && i < nr) pnew[oi] = win[t + DR];
        // centred vertical sums of this column at row i
        T c[DR + 1];
        c[0] = win[t + DR];
#pragma unroll
        for (int g = 1; g <= DR; ++g) c[g] = c[g - 1] + (win[t + DR - g] + win[t + DR + g]);
        T(*row)[DCOLS] = crow_buf[t & 1][grp];
        row[0][col] = c[6];
        row[1][col] = c[5];
        row[2][col] = c[4];
        row[3][col] = c[3];
        row[4][col] = c[0];
        // every thread passes every barrier (no early exit before the last row)
        __syncthreads();
        if (!out_col || i >= nr) continue;
        if (EXT == EXT_ODD && (i == 0 || i == nr - 1 || J == 0 || J == nc - 1)) continue;
        T acc = c[disk_height(0)];
#pragma unroll
        for (int b = 1; b <= DR; ++b) acc += row[disk_slot(b)][col - b] + row[disk_slot(b)][col + b];
        T out = v * acc;
        if (FUSE) {
            // alpha L(w) p (5-point stencil, zero Neumann), read through the L1 cache
            out += T(fa.alpha) * lap_at(w, pv, i, J, nr, nc);
            part += __ldg(pv + oi) * out;
        }
        y[oi] = out;
    }
    if (FUSE && fa.reduce) {
        const int slot = fa.slot0 + by * gx + bx;
        double sres;
        if (block_reduce_last((double)part, fa.red, fa.ticket, slot, fa.total_blocks, &sres) && threadIdx.x == 0 &&
            fa.finish_here)
            finish_pq(fa.st, sres);
    }
}

template <typename T, int EXT, bool FUSE, bool PUP>
__global__ void __launch_bounds__(kThreads)
blur_disk_kernel(const T* __restrict__ x, T* __restrict__ y, int nr, int nc, T v, const T* __restrict__ w, T* p0,
                 T* p1, FuseArgs fa) {
    // (the implicit trigger at block exit lets the next kernel launch)
    pdl_wait();
    if (fa.st && fa.st->done) return;
    disk_body<T, EXT, FUSE, PUP>(blockIdx.x, blockIdx.y, gridDim.x, x, y, nr, nc, v, w, p0, p1, fa);
}

template <typename T, int EXT, bool FUSE, bool PUP>
__global__ void __launch_bounds__(kThreads)
blur_flat_kernel(const T* __restrict__ x, T* __restrict__ y, int nr, int nc, int mr, int mc,
                 const int* __restrict__ colh, T v, const T* __restrict__ w, T* p0, T* p1, FuseArgs fa) {
    // (the implicit trigger at block exit lets the next kernel launch)
    pdl_wait();
    if (fa.st && fa.st->done) return;
    flat_body<T, EXT, FUSE, PUP>(blockIdx.x, blockIdx.y, gridDim.x, x, y, nr, nc, mr, mc, colh, v, w, p0, p1, fa);
}

template <typename T, int EXT, bool FUSE, bool PUP>
__global__ void __launch_bounds__(kThreads)
blur_tile_kernel(const T* __restrict__ x, T* __restrict__ y, int nr, int nc, int mr, int mc,
                 const T* __restrict__ hdense, const int* __restrict__ arange,
                 const int* __restrict__ runs, const T* __restrict__ runv, int nruns,
                 const T* __restrict__ w, T* p0, T* p1, FuseArgs fa) {
    // (the implicit trigger at block exit lets the next kernel launch)
    pdl_wait();
    if (fa.st && fa.st->done) return;
    tile_body<T, EXT, FUSE, PUP>(blockIdx.x, blockIdx.y, gridDim.x, x, y, nr, nc, mr, mc, hdense, arange, runs, runv,
                                 nruns, w, p0, p1, fa);
}

// odd extension along one axis: returns the sign (0 on the boundary lines and
// beyond the single mirror image, where no output reads) and the index
__device__ __forceinline__ int odd_map(int I, int n, int* idx) {
    *idx = 0;
    if (I == 0 || I == n - 1) return 0;
    if (I < 0) {
        if (-I > n - 2) return 0;
        *idx = -I;
        return -1;
    }
    if (I > n - 1) {
        if (2 * (n - 1) - I < 1) return 0;
        *idx = 2 * (n - 1) - I;
        return -1;
    }
    *idx = I;
    return 1;
}

// First/last rows and columns of H^T y under AR BCs. Each block computes 32
// consecutive outputs of one border (or the four corners): it stages the
// strip of y the tail-weighted sums read (with the odd extension across the
// other direction) in shared memory, eight thread groups share the strip's
// rows, and a shared-memory reduction combines them.
constexpr int kSeg = 32;

template <typename T, bool FUSE>
__device__ __forceinline__ void border_body(int bid, const T* __restrict__ y, T* __restrict__ out, int nr, int nc,
                                            int mr, int mc, const T* __restrict__ crow, const T* __restrict__ ccol,
                                            const T* __restrict__ ccor, const T* __restrict__ w, const T* p0,
                                            const T* p1, const FuseArgs& fa, T* partial) {
    const int slot = fa.slot0 + bid;
    const T* pv = fa.st ? (fa.st->pbuf ? p0 : p1) : p0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* strip = reinterpret_cast<T*>(smem_raw);
    const int nseg_r = (nc - 2 + kSeg - 1) / kSeg, nseg_c = (nr - 2 + kSeg - 1) / kSeg;
    const int o = threadIdx.x % kSeg, grp = threadIdx.x / kSeg, ngrp = kThreads / kSeg;
    T acc = T(0);
    int oi = -1, oj = -1;
    if (bid < 2 * nseg_r) {
        // top (0) / bottom (nr - 1) row, interior columns l0 .. l0 + 31
        const bool top = bid < nseg_r;
        const int l0 = 1 + (top ? bid : bid - nseg_r) * kSeg;
        const int SW = kSeg + 2 * mc;
        const int cmax = nc - 2 + mc;          // the last column any output of this border reads
        for (int e = threadIdx.x; e < (mr + 1) * SW; e += blockDim.x) {
            const int i = e / SW, cc = e - i * SW;
            const int J = l0 - mc + cc;
            int ci;
            const int sg = J <= cmax ? odd_map(J, nc, &ci) : 0;
            const int ri = top ? i : nr - 1 - i;
            strip[e] = sg ? T(sg) * y[(size_t)ri * nc + ci] : T(0);
        }
        __syncthreads();
        const int l = l0 + o;
        for (int i = grp; i <= mr; i += ngrp) {
            const T* crw = crow + (size_t)i * (2 * mc + 1);
            const T* srow = strip + i * SW + o + mc;
            for (int b = -mc; b <= mc; ++b) acc += __ldg(crw + b + mc) * srow[b];
        }
        // one row (a 1D signal): the top row's sums are complete, the bottom copy writes nothing
        if (l <= nc - 2 && (top || nr > 1)) { oi = top ? 0 : nr - 1; oj = l; }
    } else if (bid < 2 * nseg_r + 2 * nseg_c) {
        // left (0) / right (nc - 1) column, interior rows k0 .. k0 + 31
        bid -= 2 * nseg_r;
        const bool left = bid < nseg_c;
        const int k0 = 1 + (left ? bid : bid - nseg_c) * kSeg;
        const int SH = kSeg + 2 * mr;
        const int rmax = nr - 2 + mr;          // the last row any output of this border reads
        for (int e = threadIdx.x; e < SH * (mc + 1); e += blockDim.x) {
            const int r = e / (mc + 1), j = e - r * (mc + 1);
            const int I = k0 - mr + r;
            int ri;
            const int sg = I <= rmax ? odd_map(I, nr, &ri) : 0;
            const int cj = left ? j : nc - 1 - j;
            strip[e] = sg ? T(sg) * y[(size_t)ri * nc + cj] : T(0);
        }
        __syncthreads();
        const int k = k0 + o;
        for (int j = grp; j <= mc; j += ngrp)
            for (int a = -mr; a <= mr; ++a)
                acc += __ldg(ccol + (size_t)(a + mr) * (mc + 1) + j) * strip[(o + mr + a) * (mc + 1) + j];
        if (k <= nr - 2) { oi = k; oj = left ? 0 : nc - 1; }
    } else {
        // the four corners: output c = o (< 4); groups share the (mr + 1) rows (one row:
        // only the two top corners, which are then the line's two ends)
        if (o < 4 && ((o & 1) == 0 || nr > 1)) {
            const bool top = (o & 1) == 0, left = (o & 2) == 0;
            for (int i = grp; i <= mr; i += ngrp) {
                const int ri = top ? i : nr - 1 - i;
                for (int j = 0; j <= mc; ++j) {
                    const int cj = left ? j : nc - 1 - j;
                    acc += __ldg(ccor + (size_t)i * (mc + 1) + j) * y[(size_t)ri * nc + cj];
                }
            }
            oi = top ? 0 : nr - 1;
            oj = left ? 0 : nc - 1;
        }
    }
    partial[threadIdx.x] = acc;
    __syncthreads();
    T part = T(0);
    if (grp == 0 && oi >= 0) {
        T v = T(0);
        for (int g = 0; g < ngrp; ++g) v += partial[g * kSeg + o];
        if (FUSE) {
            v += T(fa.alpha) * lap_at(w, pv, oi, oj, nr, nc);
            part = pv[(size_t)oi * nc + oj] * v;
        }
        out[(size_t)oi * nc + oj] = v;
    }
    if (FUSE && fa.reduce) {
        double s;
        if (block_reduce_last((double)part, fa.red, fa.ticket, slot, fa.total_blocks, &s) && threadIdx.x == 0 &&
            fa.finish_here)
            finish_pq(fa.st, s);
    }
}

// The AR adjoint in one launch: blocks 0 .. tile_blocks-1 compute the interior
// tiles (gx tiles per row of tiles), the rest the border lines, so the small
// border work runs beside the interior instead of after it. Both parts reduce
// p^T q into one ticket; whichever block arrives last finishes.
template <typename T, bool FUSE, int PATH>
__global__ void __launch_bounds__(kThreads)
ar_adjoint_kernel(const T* __restrict__ x, T* __restrict__ y, int nr, int nc, int mr, int mc,
                  const T* __restrict__ hdense, const int* __restrict__ arange, const int* __restrict__ runs,
                  const T* __restrict__ runv, int nruns, const int* __restrict__ colh, T flatv,
                  const T* __restrict__ crow, const T* __restrict__ ccol, const T* __restrict__ ccor,
                  const T* __restrict__ w, T* p0, T* p1, int tile_blocks, int gx, FuseArgs fa_tile,
                  FuseArgs fa_border) {
    // (the implicit trigger at block exit lets the next kernel launch)
    pdl_wait();
    if (fa_tile.st && fa_tile.st->done) return;
    __shared__ T partial[kThreads];
    const int bid = blockIdx.x;
    if (bid < tile_blocks) {
        if (PATH == PATH_DISK)
            disk_body<T, EXT_ODD, FUSE, false>(bid % gx, bid / gx, gx, x, y, nr, nc, flatv, w, p0, p1, fa_tile);
        else if (PATH == PATH_FLAT)
            flat_body<T, EXT_ODD, FUSE, false>(bid % gx, bid / gx, gx, x, y, nr, nc, mr, mc, colh, flatv, w, p0, p1,
                                               fa_tile);
        else
            tile_body<T, EXT_ODD, FUSE, false>(bid % gx, bid / gx, gx, x, y, nr, nc, mr, mc, hdense, arange, runs,
                                               runv, nruns, w, p0, p1, fa_tile);
    } else
        border_body<T, FUSE>(bid - tile_blocks, x, y, nr, nc, mr, mc, crow, ccol, ccor, w, p0, p1, fa_border,
                             partial);
}

static size_t border_smem(int mr, int mc, size_t elem) {
    const size_t a = (size_t)(mr + 1) * (kSeg + 2 * mc), b = (size_t)(kSeg + 2 * mr) * (mc + 1);
    return (a > b ? a : b) * elem + 16;
}

static size_t tile_smem(int mr, int mc, size_t elem, bool fuse, bool pup, int nruns) {
    const size_t tw = BTW + 2 * mc, th = BTH + 2 * mr;
    const size_t tile = tw * th * elem;
    return tile * (pup ? 2 : 1) + (fuse ? 2 * (BTW + 2) * (BTH + 2) * elem : 0) +
           (size_t)(2 * mr + 1) * (2 * mc + 1) * elem + 2 * (2 * mc + 1) * sizeof(int) +
           (nruns ? th * (tw + 1) * elem + (size_t)nruns * (elem + 3 * sizeof(int)) : 0) + 32;
}

enum BlurMode { BLUR_PLAIN = 0, BLUR_PUP = 1, BLUR_FUSE = 2 };

template <typename T, int EXT, bool FUSE, bool PUP>
static tvd_status launch_tile(dim3 grid, size_t smem, cudaStream_t s, const T* x, T* y, const tvd_plan_s& p,
                              const Ops<T>& o, const T* w, T* p0, T* p1, const FuseArgs& fa) {
    if (o.flat == 2) {
        TVD_CUDA_TRY(launch_pdl(blur_disk_kernel<T, EXT, FUSE, PUP>, grid, dim3(kThreads), smem, s, x, y, p.nr, p.nc,
                                (T)o.flatv, w, p0, p1, fa));
        return TVD_OK;
    }
    if (o.flat) {
        TVD_CUDA_TRY((allow_max_smem<blur_flat_kernel<T, EXT, FUSE, PUP>>()));
        TVD_CUDA_TRY(launch_pdl(blur_flat_kernel<T, EXT, FUSE, PUP>, grid, dim3(kThreads), smem, s, x, y, p.nr, p.nc,
                                p.psf.mr, p.psf.mc, (const int*)o.colh, (T)o.flatv, w, p0, p1, fa));
        return TVD_OK;
    }
    TVD_CUDA_TRY((allow_max_smem<blur_tile_kernel<T, EXT, FUSE, PUP>>()));
    TVD_CUDA_TRY(launch_pdl(blur_tile_kernel<T, EXT, FUSE, PUP>, grid, dim3(kThreads), smem, s, x, y, p.nr, p.nc,
                            p.psf.mr, p.psf.mc, (const T*)o.hdense, (const int*)o.arange, (const int*)o.runs,
                            (const T*)o.runv, o.nruns, w, p0, p1, fa));
    return TVD_OK;
}

template <typename T, bool FUSE, int PATH>
static tvd_status launch_ar_adjoint(int blocks, size_t smem, cudaStream_t s, const T* x, T* y, const tvd_plan_s& p,
                                    const Ops<T>& o, const T* w, T* p0, T* p1, int tile_blocks, int gx,
                                    const FuseArgs& fa, const FuseArgs& fb) {
    TVD_CUDA_TRY((allow_max_smem<ar_adjoint_kernel<T, FUSE, PATH>>()));
    TVD_CUDA_TRY(launch_pdl(ar_adjoint_kernel<T, FUSE, PATH>, dim3(blocks), dim3(kThreads), smem, s, x, y, p.nr,
                            p.nc, p.psf.mr, p.psf.mc, (const T*)o.hdense, (const int*)o.arange, (const int*)o.runs,
                            (const T*)o.runv, o.nruns, (const int*)o.colh, (T)o.flatv, (const T*)o.crow,
                            (const T*)o.ccol, (const T*)o.ccor, w, p0, p1, tile_blocks, gx, fa, fb));
    return TVD_OK;
}

// mode BLUR_PLAIN: y = H x or H^T x. BLUR_PUP: forward blur of the new CG
// direction (x = z). BLUR_FUSE: y = H^T x + alpha L(w) p and p^T q.
template <typename T>
static tvd_status launch_blur(const tvd_plan_s& p, const Ops<T>& o, bool transpose, int mode, const T* x, T* y,
                              const T* w, T* p0, T* p1, double alpha, CgState* st, cudaStream_t s) {
    const int nr = p.nr, nc = p.nc, mr = p.psf.mr, mc = p.psf.mc;
    const int path = o.flat == 2 ? PATH_DISK : (o.flat ? PATH_FLAT : PATH_TILE);
    const int tw = path == PATH_DISK ? DBW : (path == PATH_FLAT ? FBW : BTW);
    const int th = path == PATH_DISK ? DBH : (path == PATH_FLAT ? FBH : BTH);
    const dim3 grid((nc + tw - 1) / tw, (nr + th - 1) / th);
    const bool fuse = mode == BLUR_FUSE, pup = mode == BLUR_PUP;
    const size_t smem = path == PATH_DISK ? 0
                        : path == PATH_FLAT ? flat_smem_bytes<T>()
                                            : tile_smem(mr, mc, sizeof(T), fuse, pup, o.nruns);
    FuseArgs fa{alpha, st, p.red, p.ticket + 1, (fuse && st) ? 1 : 0, 0, 0, 0};
    const int tile_blocks = (int)(grid.x * grid.y);
    const int border_blocks = 2 * ((nc - 2 + kSeg - 1) / kSeg) + 2 * ((nr - 2 + kSeg - 1) / kSeg) + 1;
    const bool ar_adj = transpose && p.bc == TVD_BC_ANTIREFLECTIVE;
    ProfScope prof(prof_class<T>((transpose || fuse) ? PROF_BLUR_ADJ : PROF_BLUR_FWD), s);
    if (fa.reduce) {
        fa.total_blocks = tile_blocks + (ar_adj ? border_blocks : 0);
        if (fa.total_blocks > kMaxRedBlocks) {
            set_error("image too large for the reduction buffer");
            return TVD_EINVAL;
        }
    }
    if (!transpose && fuse) {
        // H t + alpha L(w) p (the reblurring product H' H p + alpha L p with t = H p)
        fa.finish_here = 1;
        if (p.bc == TVD_BC_ANTIREFLECTIVE) TVD_TRY((launch_tile<T, EXT_AR, true, false>(grid, smem, s, x, y, p, o, w, p0, p1, fa)));
        else TVD_TRY((launch_tile<T, EXT_R, true, false>(grid, smem, s, x, y, p, o, w, p0, p1, fa)));
    } else if (!transpose) {
        if (p.bc == TVD_BC_ANTIREFLECTIVE) {
            if (pup) TVD_TRY((launch_tile<T, EXT_AR, false, true>(grid, smem, s, x, y, p, o, w, p0, p1, fa)));
            else TVD_TRY((launch_tile<T, EXT_AR, false, false>(grid, smem, s, x, y, p, o, w, p0, p1, fa)));
        } else {
            if (pup) TVD_TRY((launch_tile<T, EXT_R, false, true>(grid, smem, s, x, y, p, o, w, p0, p1, fa)));
            else TVD_TRY((launch_tile<T, EXT_R, false, false>(grid, smem, s, x, y, p, o, w, p0, p1, fa)));
        }
    } else if (!ar_adj) {
        // H^T = H for reflective BCs
        fa.finish_here = 1;
        if (fuse) TVD_TRY((launch_tile<T, EXT_R, true, false>(grid, smem, s, x, y, p, o, w, p0, p1, fa)));
        else TVD_TRY((launch_tile<T, EXT_R, false, false>(grid, smem, s, x, y, p, o, w, p0, p1, fa)));
    } else {
        // interior tiles and border lines in one launch (1D grid: tiles first)
        FuseArgs fb = fa;
        fa.finish_here = 1;
        fa.slot0 = 0;
        fb.finish_here = 1;
        fb.slot0 = tile_blocks;
        const size_t bsm = border_smem(mr, mc, sizeof(T));
        const size_t msm = smem > bsm ? smem : bsm;
        const int blocks = tile_blocks + border_blocks;
        const int gx = (int)grid.x;
#define TVD_ADJ(F, P) TVD_TRY((launch_ar_adjoint<T, F, P>(blocks, msm, s, x, y, p, o, w, p0, p1, tile_blocks, gx, fa, fb)))
        if (fuse) {
            if (path == PATH_DISK) TVD_ADJ(true, PATH_DISK);
            else if (path == PATH_FLAT) TVD_ADJ(true, PATH_FLAT);
            else TVD_ADJ(true, PATH_TILE);
        } else {
            if (path == PATH_DISK) TVD_ADJ(false, PATH_DISK);
            else if (path == PATH_FLAT) TVD_ADJ(false, PATH_FLAT);
            else TVD_ADJ(false, PATH_TILE);
        }
#undef TVD_ADJ
    }
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

template <typename T>
tvd_status blur_apply(const tvd_plan_s& p, const Ops<T>& o, bool transpose, const T* x, T* y, cudaStream_t s,
                      CgState* st) {
    return launch_blur<T>(p, o, transpose, BLUR_PLAIN, x, y, nullptr, nullptr, nullptr, 0.0, st, s);
}

template <typename T>
tvd_status blur_pupdate(const tvd_plan_s& p, const Ops<T>& o, const T* z, T* p0, T* p1, T* t, CgState* st,
                        cudaStream_t s) {
    return launch_blur<T>(p, o, false, BLUR_PUP, z, t, nullptr, p0, p1, 0.0, st, s);
}

template <typename T>
tvd_status normal_finish(const tvd_plan_s& p, const Ops<T>& o, const T* t, const T* p0, const T* p1, double alpha,
                         T* q, CgState* st, cudaStream_t s) {
    return launch_blur<T>(p, o, true, BLUR_FUSE, t, q, o.w, const_cast<T*>(p0), const_cast<T*>(p1), alpha, st, s);
}

template <typename T>
tvd_status forward_fuse(const tvd_plan_s& p, const Ops<T>& o, const T* t, const T* x, double alpha, T* y,
                        cudaStream_t s) {
    return launch_blur<T>(p, o, false, BLUR_FUSE, t, y, o.w, const_cast<T*>(x), const_cast<T*>(x), alpha, nullptr, s);
}

// ---------------------------------------------------------------- allocation-free normal-equations product
//
// tvd_normal_apply_noalloc computes y = H^T H x + alpha L(u) x without any
// device allocation: the intermediate H x, the diffusivity of u and the PSF
// tables live in the file-scope arrays below, which every GPU that loads the
// library holds until the process exits (8 MiB for the two image arrays plus
// about 0.2 MiB of tables). All calls share them.

constexpr int kNoAllocMaxPixels = 512 * 1024;     // n_rows * n_cols limit
constexpr int kNoAllocMaxHalf = 48;               // PSF half-width limit (as for plans)
constexpr int kNoAllocMaxSide = 2 * kNoAllocMaxHalf + 1;

static __device__ __align__(256) double g_na_hx[kNoAllocMaxPixels];      // H x
static __device__ __align__(256) double g_na_w[kNoAllocMaxPixels];       // diffusivity of u
static __device__ __align__(256) double g_na_h[kNoAllocMaxSide * kNoAllocMaxSide];
static __device__ __align__(256) int g_na_arange[2 * kNoAllocMaxSide];
static __device__ __align__(256) double g_na_crow[(kNoAllocMaxHalf + 1) * kNoAllocMaxSide];
static __device__ __align__(256) double g_na_ccol[kNoAllocMaxSide * (kNoAllocMaxHalf + 1)];
static __device__ __align__(256) double g_na_ccor[(kNoAllocMaxHalf + 1) * (kNoAllocMaxHalf + 1)];

struct NoAllocPtrs {
    bool ready = false;
    double *hx, *w, *h, *crow, *ccol, *ccor;
    int* arange;
};

constexpr int kNoAllocMaxDevices = 64;
static NoAllocPtrs g_na_ptrs[kNoAllocMaxDevices];
static std::mutex g_na_mu;

// Device addresses of the arrays above for the current device, looked up once
// per device (host code cannot use the symbols' own names as device pointers).
static tvd_status noalloc_ptrs(NoAllocPtrs* out) {
    int dev = 0;
    TVD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("tvd_normal_apply_noalloc: device ordinal out of range");
        return TVD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    NoAllocPtrs& p = g_na_ptrs[dev];
    if (!p.ready) {
        TVD_CUDA_TRY(cudaGetSymbolAddress((void**)&p.hx, g_na_hx));
        TVD_CUDA_TRY(cudaGetSymbolAddress((void**)&p.w, g_na_w));
        TVD_CUDA_TRY(cudaGetSymbolAddress((void**)&p.h, g_na_h));
        TVD_CUDA_TRY(cudaGetSymbolAddress((void**)&p.arange, g_na_arange));
        TVD_CUDA_TRY(cudaGetSymbolAddress((void**)&p.crow, g_na_crow));
        TVD_CUDA_TRY(cudaGetSymbolAddress((void**)&p.ccol, g_na_ccol));
        TVD_CUDA_TRY(cudaGetSymbolAddress((void**)&p.ccor, g_na_ccor));
        p.ready = true;
    }
    *out = p;
    return TVD_OK;
}

}  // namespace tvd

extern "C" tvd_status tvd_normal_apply_noalloc(int n_rows, int n_cols, const double* psf_host, int p_rows,
                                               int p_cols, tvd_bc bc, const double* u_lag, double alpha,
                                               double beta, const double* x, double* y, void* stream) {
    using namespace tvd;
    if (!psf_host || !u_lag || !x || !y || y == x || y == u_lag || !(alpha >= 0.0) || !(beta > 0.0) ||
        (bc != TVD_BC_REFLECTIVE && bc != TVD_BC_ANTIREFLECTIVE) || n_rows < 3 || n_cols < 3) {
        set_error("tvd_normal_apply_noalloc: invalid argument");
        return TVD_EINVAL;
    }
    if ((long long)n_rows * n_cols > kNoAllocMaxPixels) {
        set_error("tvd_normal_apply_noalloc: n_rows * n_cols exceeds the fixed scratch of " +
                  std::to_string(kNoAllocMaxPixels) + " pixels");
        return TVD_EINVAL;
    }
    // host-side PSF tables (the plan's validation: odd sides, symmetry, m <= n - 2, m <= 48)
    tvd_plan_s plan;
    plan.nr = n_rows;
    plan.nc = n_cols;
    plan.bc = bc;
    TVD_TRY(build_psf(plan.psf, psf_host, p_rows, p_cols, n_rows, n_cols));
    const int mr = plan.psf.mr, mc = plan.psf.mc, pw = 2 * mc + 1;
    std::vector<int> rng(2 * (size_t)pw);
    for (int b = -mc; b <= mc; ++b) {
        int lo = mr + 1, hi = -mr - 1;
        for (int a = -mr; a <= mr; ++a)
            if (plan.psf.h[(size_t)(a + mr) * pw + (b + mc)] != 0.0) {
                lo = std::min(lo, a);
                hi = std::max(hi, a);
            }
        rng[2 * (b + mc)] = lo;
        rng[2 * (b + mc) + 1] = hi;
    }
    NoAllocPtrs d;
    TVD_TRY(noalloc_ptrs(&d));
    cudaStream_t s = (cudaStream_t)stream;
    // every table entry the kernels read is written here, and the kernels write
    // all of H x and of the diffusivity before reading them: nothing needs clearing
    auto put = [&](void* dst, const void* src, size_t bytes) -> tvd_status {
        TVD_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
        return TVD_OK;
    };
    TVD_TRY(put(d.h, plan.psf.h.data(), plan.psf.h.size() * sizeof(double)));
    TVD_TRY(put(d.arange, rng.data(), rng.size() * sizeof(int)));
    TVD_TRY(put(d.crow, plan.psf.crow.data(), plan.psf.crow.size() * sizeof(double)));
    TVD_TRY(put(d.ccol, plan.psf.ccol.data(), plan.psf.ccol.size() * sizeof(double)));
    TVD_TRY(put(d.ccor, plan.psf.ccor.data(), plan.psf.ccor.size() * sizeof(double)));
    Ops<double> o;
    o.hdense = d.h;
    o.arange = d.arange;
    o.crow = d.crow;
    o.ccol = d.ccol;
    o.ccor = d.ccor;
    o.w = d.w;
    TVD_TRY(diffusivity<double>(plan, u_lag, beta, d.w, s));
    TVD_TRY(blur_apply<double>(plan, o, false, x, d.hx, s));
    TVD_TRY(normal_finish<double>(plan, o, d.hx, x, x, alpha, y, nullptr, s));
    // the host tables above are copied from pageable memory; wait so they may be freed
    TVD_CUDA_TRY(cudaStreamSynchronize(s));
    return TVD_OK;
}

namespace tvd {

#define INST(T)                                                                                                  \
    template tvd_status blur_apply<T>(const tvd_plan_s&, const Ops<T>&, bool, const T*, T*, cudaStream_t, CgState*); \
    template tvd_status blur_pupdate<T>(const tvd_plan_s&, const Ops<T>&, const T*, T*, T*, T*, CgState*,       \
                                        cudaStream_t);                                                           \
    template tvd_status normal_finish<T>(const tvd_plan_s&, const Ops<T>&, const T*, const T*, const T*, double, \
                                         T*, CgState*, cudaStream_t);                                            \
    template tvd_status forward_fuse<T>(const tvd_plan_s&, const Ops<T>&, const T*, const T*, double, T*,       \
                                        cudaStream_t);
INST(float)
INST(double)

}  // namespace tvd
