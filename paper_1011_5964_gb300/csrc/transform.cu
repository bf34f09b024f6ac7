// Fast trigonometric transforms of the preconditioners (Secs. 2-3 of the paper)
// and the preconditioner spectrum.
//
// The 2D transform U = B_r (x) B_c acts on an n_r x n_c image as a pass over
// rows (B_c on each row) and a pass over columns (B_r on each column):
//   AR: B = hat-S_n = diag(1, S_{n-2}, 1), S_m the orthonormal DST-I of eq. (lambda);
//   R:  B = C, the orthonormal DCT-II of Sec. 3.1; B^{-1} = C^T (DCT-III).
// The preconditioner solve (D_R / D_M, Sec. 3.2) is
//   z = D^{-1/2} U^{-1} [ (U D^{-1/2} r) / (Lambda_H^2 + alpha Lambda_L) ],
// done in three kernels: row pass (scale, forward), column pass (forward,
// divide by the spectrum, inverse, all in shared memory), row pass (inverse,
// scale, r^T z).
//
// Every line transform is computed from one complex FFT of a pair of real
// lines packed as re + i im, in shared memory (Stockham autosort, mixed radix;
// radices up to 31 in registers, larger prime factors by direct sums):
//   DST-I, length N = n-2, M = N+1: with y_j = sin(j pi/M)(x_j + x_{M-j})
//     + (x_j - x_{M-j})/2 (x_0 = x_M = 0) and Y = DFT_M(y):
//     F_{2k} = -Im Y_k, F_{2k+1} = F_{2k-1} + Re Y_k, F_1 = Re Y_0 / 2;
//     S_N x = sqrt(2/M) F. (The auxiliary-array method for the sine
//     transform via a real FFT of length M.)
//   DCT-II, length n: Makhoul's even/odd reordering v, V = DFT_n(v),
//     X_k = c_k Re(exp(-i pi k/(2n)) V_k); DCT-III inverts these steps.
// Preconditioner spectrum: Lambda_L[i,j] = (b_i (x) b_j)^T L (b_i (x) b_j)
// = sum_pq w_pq [G_r(i,p) E_c(j,q) + E_r(i,p) G_c(j,q)] with E = b_k(p)^2,
// G = ((D_1 b_k)_p)^2. For the sine and cosine bases every row of E and G is
// a constant plus a cosine series, so E f and G f for a line f come from one
// real DFT of f; a row pass gives E_c w and G_c w, a column pass combines them.
#include "common.cuh"

#include <cmath>
#include <cstdlib>

namespace tvd {

enum { OP_ROW_FWD = 0, OP_COL_SOLVE = 1, OP_ROW_INV = 2, OP_ROW_EG = 3, OP_COL_EG = 4, OP_ROW_X = 5, OP_COL_X = 6 };
enum { BCK_AR = 0, BCK_R = 1 };

// Auxiliary tables per transform length, 8 slots of 2n values of T each:
//  AR: slot0 sin(j pi / M)              (real, j < M)
//      slot1 exp(i pi k / M)            (complex)
//      slot2 (4/M) sin^2(k pi / (2M))   (real)
//  R:  slot0 c_k                        (real)
//      slot1 (cos, sin)(pi k / (2n))    (complex)
//      slot2 exp(i pi k / n)            (complex)
//      slot3 c_k^2 / 2                  (real)
//      slot4 2 c_k^2 sin^2(pi k / (2n)) (real)
//      slot5 1 / (n c_k)                (real)


template <typename T>
struct LineArgs {
    const T* in0;        // input lines (x / t / w / A)
    const T* in1;        // second input (B for OP_COL_EG)
    T* out0;             // output lines
    T* out1;             // second output (B for OP_ROW_EG)
    const T* scale;      // D^{-1/2} (optional), applied on load (ROW_FWD) or store (ROW_INV)
    const T* spec;       // inv_spec (COL_SOLVE) / lamH2 (COL_EG)
    T* inv_out;          // COL_EG: inv_spec output
    T* lam_out;          // COL_EG: when set, Lambda_L itself instead of inv_out
    // reblurring (AR): the rank-2 corrections of T_n = hat-S (I + U), T_n^-1 =
    // (I - U) hat-S along each line: ucorr[k - 1] = (S p)_k, ucorr[n - 2 + k - 1]
    // = (S J p)_k for the interior k = 1..n-2 (nullptr: hat-S alone)
    const T* ucorr;
    const T* rvec;       // ROW_INV: r for r^T z
    const cplx<T>* tw;   // twiddles, length L
    const cplx<T>* blt;  // Bluestein tables (fp.bl): chirp exp(-i pi j^2 / L) (L) | filter spectrum / M2 (M2) | M2 twiddles
    const T* aux;        // auxiliary tables, kAuxSlots * 2n
    int n;               // line length
    int ns;              // stride of the lines in shared memory (odd: no bank conflicts across lines)
    int nlines;          // number of lines (image lines)
    int nr, nc;          // image shape
    int P;               // line pairs per block
    int L;               // complex FFT length
    FftPlan fp;
    double alpha;
    CgState* st;
    double* red;
    unsigned int* ticket;
    int* bad;            // COL_EG: set if a spectrum entry is not positive
    int xa, xb;          // ROW_X / COL_X: contraction of line a (in0) / b (in1): 0 = E, 1 = F
    // ROW_FWD on the CG path: the pending x += alpha p, r -= alpha q of the
    // previous iteration (in0 is r, updated in place) and the stopping test
    T* xvec;
    const T* qvec;
    const T* p0;
    const T* p1;
    unsigned int* ticket2;
};

template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// ------------------------------------------------------------- FFT stages

// R-point DFT of v (already multiplied by the stage twiddles), written to
// dst[t * Ns], t = 0..R-1. Radix constants exp(-+2 pi i t / R) come from the
// shared twiddle table (tw[t * LR], conjugated for the inverse transform).
template <typename T, int R>
__device__ __forceinline__ void dft_store(cplx<T> (&v)[R], cplx<T>* __restrict__ dst, int Ns,
                                          const cplx<T>* __restrict__ tw, int LR, bool inv, int g, int G) {
    if constexpr (R == 2) {
        dst[0] = {v[0].re + v[1].re, v[0].im + v[1].im};
        dst[Ns] = {v[0].re - v[1].re, v[0].im - v[1].im};
    } else if constexpr (R == 4) {
        const T sg = inv ? T(1) : T(-1);      // exp(-+ i pi / 2) = -+ i
        const cplx<T> s02 = {v[0].re + v[2].re, v[0].im + v[2].im};
        const cplx<T> d02 = {v[0].re - v[2].re, v[0].im - v[2].im};
        const cplx<T> s13 = {v[1].re + v[3].re, v[1].im + v[3].im};
        const cplx<T> d13 = {v[1].re - v[3].re, v[1].im - v[3].im};
        const cplx<T> jd = {-sg * d13.im, sg * d13.re};
        dst[0] = {s02.re + s13.re, s02.im + s13.im};
        dst[2 * Ns] = {s02.re - s13.re, s02.im - s13.im};
        dst[Ns] = {d02.re + jd.re, d02.im + jd.im};
        dst[3 * Ns] = {d02.re - jd.re, d02.im - jd.im};
    } else {
        // out[k] = v0 + sum_{j=1}^{H} (s_j cos_jk + i d_j sin_jk) [+ v_{R/2} (-1)^k],
        // s_j = v_j + v_{R-j}, d_j = v_j - v_{R-j}; out[R-k] takes the opposite sign of i.
        constexpr int H = (R - 1) / 2;
        constexpr bool even = (R % 2) == 0;
        const cplx<T> v0 = v[0];
        cplx<T> vh = {T(0), T(0)};
        if constexpr (even) vh = v[R / 2];
#pragma unroll
        for (int j = 1; j <= H; ++j) {
            const cplx<T> a = v[j], b = v[R - j];
            v[j] = {a.re + b.re, a.im + b.im};
            v[R - j] = {a.re - b.re, a.im - b.im};
        }
        if (g == 0) {
            cplx<T> o0 = v0;
#pragma unroll
            for (int j = 1; j <= H; ++j) { o0.re += v[j].re; o0.im += v[j].im; }
            if constexpr (even) { o0.re += vh.re; o0.im += vh.im; }
            dst[0] = o0;
        }
        // the inputs stay in registers; the output loop is rolled for large
        // radices to keep the register count (and so the occupancy) moderate,
        // and its output pairs are shared among G threads (this one takes g, g + G, ...)
#pragma unroll (R <= 8 ? H : 1)
        for (int k = 1 + g; k <= H; k += G) {
            cplx<T> a = v0, b = {T(0), T(0)};
#pragma unroll
            for (int j = 1; j <= H; ++j) {
                const cplx<T> wk = tw[((j * k) % R) * LR];
                const T sn = inv ? -wk.im : wk.im;
                a.re += v[j].re * wk.re; a.im += v[j].im * wk.re;
                b.re += v[R - j].re * sn; b.im += v[R - j].im * sn;
            }
            if constexpr (even) {
                const T sg = (k & 1) ? T(-1) : T(1);
                a.re += sg * vh.re; a.im += sg * vh.im;
            }
            dst[k * Ns] = {a.re - b.im, a.im + b.re};
            dst[(R - k) * Ns] = {a.re + b.im, a.im - b.re};
        }
        if (even && g == 0) {
            cplx<T> m = v0;
#pragma unroll
            for (int j = 1; j <= H; ++j) {
                const T sg = (j & 1) ? T(-1) : T(1);
                m.re += sg * v[j].re; m.im += sg * v[j].im;
            }
            const T sh = ((R / 2) & 1) ? T(-1) : T(1);
            m.re += sh * vh.re; m.im += sh * vh.im;
            dst[(R / 2) * Ns] = m;
        }
    }
}

// Walks e = threadIdx.x, threadIdx.x + kThreads, ... over P blocks of m
// entries as (hi, lo) = (e / m, e % m) without a division per step.
struct Walk {
    int hi, lo;
    __device__ __forceinline__ explicit Walk(int m) : hi((int)threadIdx.x / m), lo((int)threadIdx.x - hi * m) {}
    __device__ __forceinline__ void next(int m) {
        lo += kThreads;
        while (lo >= m) {
            lo -= m;
            ++hi;
        }
    }
};

// One Stockham stage of radix R over P complex lines of length L, run by the
// block's kThreads threads. Large radices: G threads share a butterfly's output
// pairs. Thread t takes share g = t % G of butterflies j = t / G, t / G + S, ...
// (S = kThreads / G) running over the P lines back to back; j = q Ns + k, and
// since L / R = ts Ns, stepping to the next line keeps k and lowers q by ts, so
// the loop divides only once per stage.
template <typename T, int R>
__device__ void fft_stage(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int P, int L, int Ns,
                          const cplx<T>* __restrict__ tw, bool inv) {
    const int LR = L / R;
    const int ts = L / (Ns * R);
    constexpr int H = (R - 1) / 2;
    int G = 1;
    if constexpr (R > 8) {
        // G minimises rounds x per-item cost (per item: the R inputs, then H / G pairs)
        int best = 1 << 30;
#pragma unroll
        for (int g = 1; g <= H; ++g) {
            const int rounds = (P * LR + kThreads / g - 1) / (kThreads / g);
            const int cost = rounds * (5 * R + 4 * R * ((H + g - 1) / g));
            if (cost < best) { best = cost; G = g; }
        }
    }
    const int S = kThreads / G;
    const int t = threadIdx.x;
    if (t >= S * G) return;
    const int g = t - (t / G) * G;
    int j = t / G, pp = 0;
    while (j >= LR && pp < P) {
        j -= LR;
        ++pp;
    }
    int q = j / Ns, k = j - (j / Ns) * Ns;
    const int dq = S / Ns, dk = S - dq * Ns;
    while (pp < P) {
        const cplx<T>* src = in + (size_t)pp * L;
        cplx<T> v[R];
        v[0] = src[j];
#pragma unroll
        for (int r = 1; r < R; ++r) {
            cplx<T> w = tw[k * r * ts];
            if (inv) w.im = -w.im;
            v[r] = cmul(src[j + r * LR], w);
        }
        dft_store<T, R>(v, out + (size_t)pp * L + q * Ns * R + k, Ns, tw, LR, inv, g, G);
        j += S;
        q += dq;
        k += dk;
        if (k >= Ns) {
            k -= Ns;
            ++q;
        }
        while (j >= LR) {
            j -= LR;
            q -= ts;
            ++pp;
        }
    }
}

// Radix without a register kernel: one thread per output, direct sum over R inputs.
template <typename T>
__device__ void fft_stage_generic(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int P, int L, int Ns,
                                  int R, const cplx<T>* __restrict__ tw, bool inv) {
    const int LR = L / R;
    const int ts = L / (Ns * R);
    for (int e = threadIdx.x; e < P * L; e += kThreads) {
        const int pp = e / L, q = e - pp * L;
        const int t = q / LR, j = q - t * LR;
        const int k = j % Ns;
        const cplx<T>* src = in + (size_t)pp * L;
        cplx<T> acc = {T(0), T(0)};
        for (int r = 0; r < R; ++r) {
            cplx<T> w1 = tw[k * r * ts];
            cplx<T> w2 = tw[((r * t) % R) * LR];
            if (inv) { w1.im = -w1.im; w2.im = -w2.im; }
            const cplx<T> x = cmul(cmul(src[j + r * LR], w1), w2);
            acc.re += x.re;
            acc.im += x.im;
        }
        out[(size_t)pp * L + (j / Ns) * Ns * R + k + t * Ns] = acc;
    }
}

// Runs all stages of a length-L plan, __syncthreads between them; returns the
// buffer holding the result.
template <typename T>
__device__ cplx<T>* fft_run(cplx<T>* a, cplx<T>* b, int P, int L, int nstages, const int* radix, const cplx<T>* tw,
                            bool inv) {
    int Ns = 1;
    for (int s = 0; s < nstages; ++s) {
        const int R = radix[s];
        switch (R) {
            case 2: fft_stage<T, 2>(a, b, P, L, Ns, tw, inv); break;
            case 3: fft_stage<T, 3>(a, b, P, L, Ns, tw, inv); break;
            case 4: fft_stage<T, 4>(a, b, P, L, Ns, tw, inv); break;
            case 5: fft_stage<T, 5>(a, b, P, L, Ns, tw, inv); break;
            case 7: fft_stage<T, 7>(a, b, P, L, Ns, tw, inv); break;
            case 8: fft_stage<T, 8>(a, b, P, L, Ns, tw, inv); break;
            case 9: fft_stage<T, 9>(a, b, P, L, Ns, tw, inv); break;
            case 11: fft_stage<T, 11>(a, b, P, L, Ns, tw, inv); break;
            case 13: fft_stage<T, 13>(a, b, P, L, Ns, tw, inv); break;
            case 17: fft_stage<T, 17>(a, b, P, L, Ns, tw, inv); break;
            case 19: fft_stage<T, 19>(a, b, P, L, Ns, tw, inv); break;
            case 23: fft_stage<T, 23>(a, b, P, L, Ns, tw, inv); break;
            case 29: fft_stage<T, 29>(a, b, P, L, Ns, tw, inv); break;
            case 31: fft_stage<T, 31>(a, b, P, L, Ns, tw, inv); break;
            default: fft_stage_generic<T>(a, b, P, L, Ns, R, tw, inv); break;
        }
        __syncthreads();
        cplx<T>* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// P complex lines of length L (stride L in a) -> their DFTs (inverse: conjugate
// twiddles, unnormalised). Plans with bl use Bluestein's identity
// jk = (j^2 + k^2 - (k - j)^2) / 2: X_k = c_k sum_j (x_j c_j) conj(c_{k-j}),
// c_j = exp(-i pi j^2 / L), the sum a circular convolution of length M2 done
// as IFFT(FFT(x c) FFT(b)) with the filter spectrum FFT(b) / M2 precomputed;
// the inverse transform is conj(DFT(conj x)). a and b then hold P * M2
// entries and tw the M2 twiddles. The result is returned at stride L.
template <typename T>
__device__ cplx<T>* fft_pairs(cplx<T>* a, cplx<T>* b, int P, const FftPlan& fp, const cplx<T>* tw, bool inv,
                              const cplx<T>* __restrict__ blt) {
    if (!fp.bl) return fft_run<T>(a, b, P, fp.L, fp.nstages, fp.radix, tw, inv);
    const int L = fp.L, M2 = fp.M2;
    const cplx<T>* __restrict__ chirp = blt;
    const cplx<T>* __restrict__ filt = blt + L;
    const T sg = inv ? T(-1) : T(1);
    for (Walk w(M2); w.hi < P; w.next(M2)) {
        const int pp = w.hi, m = w.lo;
        cplx<T> v = {T(0), T(0)};
        if (m < L) {
            const cplx<T> x = a[(size_t)pp * L + m];
            v = cmul(cplx<T>{x.re, sg * x.im}, chirp[m]);
        }
        b[(size_t)pp * M2 + m] = v;
    }
    __syncthreads();
    cplx<T>* Z = fft_run<T>(b, a, P, M2, fp.nst2, fp.radix2, tw, false);
    for (Walk w(M2); w.hi < P; w.next(M2)) {
        const cplx<T> y = cmul(Z[(size_t)w.hi * M2 + w.lo], filt[w.lo]);
        Z[(size_t)w.hi * M2 + w.lo] = {y.re, -y.im};   // conj: the inverse FFT by a forward one
    }
    __syncthreads();
    Z = fft_run<T>(Z, Z == a ? b : a, P, M2, fp.nst2, fp.radix2, tw, false);
    cplx<T>* out = Z == a ? b : a;
    for (Walk w(L); w.hi < P; w.next(L)) {
        const int pp = w.hi, k = w.lo;
        const cplx<T> z = Z[(size_t)pp * M2 + k];
        const cplx<T> y = cmul(cplx<T>{z.re, -z.im}, chirp[k]);
        out[(size_t)pp * L + k] = {y.re, sg * y.im};
    }
    __syncthreads();
    return out;
}

// ------------------------------------------------------------- line transforms in shared memory
// raw[l * ns + idx]: 2P real lines of length n at the odd stride ns. bufA, bufB: P complex lines of length L.

template <typename T>
__device__ __forceinline__ void split_pair(const cplx<T>* Z, int k, int L, cplx<T>& Fa, cplx<T>& Fb) {
    const cplx<T> z = Z[k];
    const cplx<T> zm = Z[k == 0 ? 0 : L - k];
    Fa = {T(0.5) * (z.re + zm.re), T(0.5) * (z.im - zm.im)};
    Fb = {T(0.5) * (z.im + zm.im), T(-0.5) * (z.re - zm.re)};
}

// DST-I on positions 1..n-2 of each raw line (AR); positions 0, n-1 untouched.
template <typename T>
__device__ void dst1_lines(T* raw, cplx<T>* bufA, cplx<T>* bufB, const LineArgs<T>& a, const cplx<T>* tw) {
    const int n = a.n, ns = a.ns, M = n - 1, N = n - 2, P = a.P;
    const T* sinh = a.aux;                    // slot0
    for (Walk w(M); w.hi < P; w.next(M)) {
        const int pp = w.hi, j = w.lo;
        const T* xa = raw + (size_t)(2 * pp) * ns;
        const T* xb = xa + ns;
        const T a0 = j >= 1 ? xa[j] : T(0), a1 = j >= 1 ? xa[M - j] : T(0);
        const T b0 = j >= 1 ? xb[j] : T(0), b1 = j >= 1 ? xb[M - j] : T(0);
        const T sj = __ldg(sinh + j);
        bufA[(size_t)pp * M + j] = {sj * (a0 + a1) + T(0.5) * (a0 - a1), sj * (b0 + b1) + T(0.5) * (b0 - b1)};
    }
    __syncthreads();
    const cplx<T>* Z = fft_pairs<T>(bufA, bufB, P, a.fp, a.fp.bl ? a.blt + a.fp.L + a.fp.M2 : tw, false, a.blt);
    // the FFT buffer not holding the result keeps the recurrence terms (2P * K <= 2P * L values)
    T* scan = reinterpret_cast<T*>(Z == bufA ? bufB : bufA);
    const T sc = sqrt(T(2) / T(M));
    const int nodd = (N + 1) / 2;             // F_1, F_3, ...
    const int neven = N / 2;                  // F_2, F_4, ...
    // even outputs and the R_k terms of the odd recurrence (into scan[line][k])
    const int K = nodd > neven + 1 ? nodd : neven + 1;
    for (Walk w(K); w.hi < P; w.next(K)) {
        const int pp = w.hi, k = w.lo;
        cplx<T> Fa, Fb;
        split_pair(Z + (size_t)pp * M, k, M, Fa, Fb);
        if (k >= 1 && k <= neven) {
            raw[(size_t)(2 * pp) * ns + 2 * k] = -sc * Fa.im;
            raw[(size_t)(2 * pp + 1) * ns + 2 * k] = -sc * Fb.im;
        }
        if (k < nodd) {
            scan[(size_t)(2 * pp) * K + k] = k == 0 ? T(0.5) * Fa.re : Fa.re;
            scan[(size_t)(2 * pp + 1) * K + k] = k == 0 ? T(0.5) * Fb.re : Fb.re;
        }
    }
    __syncthreads();
    // inclusive prefix sums of scan, one warp per line
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = kThreads >> 5;
    for (int l = wid; l < 2 * P; l += nw) {
        T carry = T(0);
        for (int c0 = 0; c0 < nodd; c0 += 32) {
            const int k = c0 + lane;
            T v = k < nodd ? scan[(size_t)l * K + k] : T(0);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const T u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            v += carry;
            if (k < nodd) raw[(size_t)l * ns + 2 * k + 1] = sc * v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
}

// Orthonormal DCT-II (inv = false) or DCT-III (inv = true) of each raw line (R).
template <typename T>
__device__ void dct_lines(T* raw, cplx<T>* bufA, cplx<T>* bufB, const LineArgs<T>& a, const cplx<T>* tw, bool inv) {
    const int n = a.n, ns = a.ns, P = a.P, h = (n + 1) / 2;
    const T* ck = a.aux;                                              // slot0
    const cplx<T>* th = reinterpret_cast<const cplx<T>*>(a.aux + 2 * n);  // slot1 (cos, sin)(pi k / 2n)
    const T* icn = a.aux + 10 * n;                                    // slot5 1/(n c_k)
    if (!inv) {
        for (Walk w(n); w.hi < P; w.next(n)) {
            const int pp = w.hi, p = w.lo;
            const int src = p < h ? 2 * p : 2 * (n - 1 - p) + 1;
            bufA[(size_t)pp * n + p] = {raw[(size_t)(2 * pp) * ns + src], raw[(size_t)(2 * pp + 1) * ns + src]};
        }
        __syncthreads();
        const cplx<T>* Z = fft_pairs<T>(bufA, bufB, P, a.fp, a.fp.bl ? a.blt + a.fp.L + a.fp.M2 : tw, false, a.blt);
        for (Walk w(n); w.hi < P; w.next(n)) {
            const int pp = w.hi, k = w.lo;
            cplx<T> Va, Vb;
            split_pair(Z + (size_t)pp * n, k, n, Va, Vb);
            const cplx<T> cs = th[k];
            const T c = __ldg(ck + k);
            raw[(size_t)(2 * pp) * ns + k] = c * (cs.re * Va.re + cs.im * Va.im);
            raw[(size_t)(2 * pp + 1) * ns + k] = c * (cs.re * Vb.re + cs.im * Vb.im);
        }
        __syncthreads();
    } else {
        for (Walk w(n); w.hi < P; w.next(n)) {
            const int pp = w.hi, k = w.lo;
            const T* xa = raw + (size_t)(2 * pp) * ns;
            const T* xb = xa + ns;
            const T s0 = __ldg(icn + k);
            const T ya = xa[k] * s0, yb = xb[k] * s0;
            T yra = T(0), yrb = T(0);
            if (k > 0) {
                const T s1 = __ldg(icn + n - k);
                yra = xa[n - k] * s1;
                yrb = xb[n - k] * s1;
            }
            const cplx<T> cs = th[k];
            const cplx<T> Va = {cs.re * ya + cs.im * yra, cs.im * ya - cs.re * yra};
            const cplx<T> Vb = {cs.re * yb + cs.im * yrb, cs.im * yb - cs.re * yrb};
            bufA[(size_t)pp * n + k] = {Va.re - Vb.im, Va.im + Vb.re};
        }
        __syncthreads();
        const cplx<T>* Z = fft_pairs<T>(bufA, bufB, P, a.fp, a.fp.bl ? a.blt + a.fp.L + a.fp.M2 : tw, true, a.blt);
        for (Walk w(n); w.hi < P; w.next(n)) {
            const int pp = w.hi, p = w.lo;
            const int dst = p < h ? 2 * p : 2 * (n - 1 - p) + 1;
            const cplx<T> z = Z[(size_t)pp * n + p];
            raw[(size_t)(2 * pp) * ns + dst] = z.re;
            raw[(size_t)(2 * pp + 1) * ns + dst] = z.im;
        }
        __syncthreads();
    }
}

// E f and G f for each raw line pair member; writes E into eo[l*n+k], G into go.
template <typename T, int BC>
__device__ void eg_lines(const T* raw, cplx<T>* bufA, cplx<T>* bufB, T* eo, T* go, const LineArgs<T>& a,
                         const cplx<T>* tw, bool second_f = false) {
    const int n = a.n, ns = a.ns, P = a.P, L = a.L;
    for (Walk w(L); w.hi < P; w.next(L)) {
        const int pp = w.hi, j = w.lo;
        bufA[(size_t)pp * L + j] = {raw[(size_t)(2 * pp) * ns + j], raw[(size_t)(2 * pp + 1) * ns + j]};
    }
    __syncthreads();
    const cplx<T>* Z = fft_pairs<T>(bufA, bufB, P, a.fp, a.fp.bl ? a.blt + a.fp.L + a.fp.M2 : tw, false, a.blt);
    for (Walk w(n); w.hi < P; w.next(n)) {
        const int pp = w.hi, k = w.lo;
        const cplx<T>* Zp = Z + (size_t)pp * L;
        const T* fa = raw + (size_t)(2 * pp) * ns;
        const T* fb = fa + ns;
        T ea, ga, eb, gb;
        if (BC == BCK_AR) {
            const int M = L;
            if (k == 0) {
                ea = ga = fa[0];
                eb = gb = fb[0];
                if (second_f) ga = gb = T(0);   // e_0: no neighbour product
            } else if (k == n - 1) {
                ea = fa[n - 1]; ga = fa[n - 2];
                eb = fb[n - 1]; gb = fb[n - 2];
                if (second_f) ga = gb = T(0);   // e_{n-1}: no forward neighbour
            } else {
                cplx<T> F0a, F0b, Fa, Fb;
                split_pair(Zp, 0, M, F0a, F0b);
                split_pair(Zp, k, M, Fa, Fb);
                const cplx<T> eh = reinterpret_cast<const cplx<T>*>(a.aux + 2 * n)[k];   // exp(i pi k/M)
                const T g = a.aux[4 * n + k];
                const T invM = T(1) / T(M);
                ea = (F0a.re - Fa.re) * invM;
                eb = (F0b.re - Fb.re) * invM;
                if (second_f) {
                    // F[k,p] = b_k(p) b_k(p+1) = (cos(k pi/M) - cos(k (2p+1) pi/M)) / M
                    ga = (eh.re * F0a.re - (eh.re * Fa.re + eh.im * Fa.im)) * invM;
                    gb = (eh.re * F0b.re - (eh.re * Fb.re + eh.im * Fb.im)) * invM;
                } else {
                    ga = g * (F0a.re + eh.re * Fa.re + eh.im * Fa.im);
                    gb = g * (F0b.re + eh.re * Fb.re + eh.im * Fb.im);
                }
            }
        } else {
            cplx<T> F0a, F0b, Fa, Fb;
            split_pair(Zp, 0, L, F0a, F0b);
            split_pair(Zp, k, L, Fa, Fb);
            const cplx<T> eh = reinterpret_cast<const cplx<T>*>(a.aux + 4 * n)[k];       // exp(i pi k/n)
            const cplx<T> w = a.tw[k];                                                   // exp(-2 pi i k/n)
            const T ce = a.aux[6 * n + k], cg = a.aux[8 * n + k];
            ea = ce * (F0a.re + eh.re * Fa.re + eh.im * Fa.im);
            eb = ce * (F0b.re + eh.re * Fb.re + eh.im * Fb.im);
            if (second_f) {
                // F[k,p] = c_k^2 / 2 (cos(pi k/n) + cos(2 pi k (p+1)/n)) for p < n-1, 0 at p = n-1
                ga = ce * (eh.re * F0a.re + (w.re * Fa.re - w.im * Fa.im) - (eh.re + T(1)) * fa[n - 1]);
                gb = ce * (eh.re * F0b.re + (w.re * Fb.re - w.im * Fb.im) - (eh.re + T(1)) * fb[n - 1]);
            } else {
                ga = cg * (F0a.re - (w.re * Fa.re - w.im * Fa.im));
                gb = cg * (F0b.re - (w.re * Fb.re - w.im * Fb.im));
            }
        }
        eo[(size_t)(2 * pp) * ns + k] = ea;
        eo[(size_t)(2 * pp + 1) * ns + k] = eb;
        go[(size_t)(2 * pp) * ns + k] = ga;
        go[(size_t)(2 * pp + 1) * ns + k] = gb;
    }
    __syncthreads();
}

// ------------------------------------------------------------- the line kernel


// Extra shared memory (elements of T) each operation stages next to the lines:
// ROW_FWD: D^-1/2; COL_SOLVE: 1/spectrum; ROW_INV: D^-1/2 and r; ROW_EG: the
// E and G outputs; COL_EG: E, G outputs and Lambda_H^2.
__host__ __device__ constexpr size_t line_extra(int op, size_t lines, size_t n, size_t P) {
    return op == OP_ROW_FWD ? lines * n
         : op == OP_COL_SOLVE ? lines * n
         : op == OP_ROW_INV ? 2 * lines * n
         : (op == OP_ROW_EG || op == OP_ROW_X || op == OP_COL_X) ? 2 * lines * n
         : 2 * lines * n + P * n;
}


// Resident blocks per SM the float kernels' register allocation aims for (tuning: more blocks
// hide more latency, at the price of spilled large-radix butterflies).
#ifndef TVD_LINE_MINB
#define TVD_LINE_MINB 2
#endif

template <typename T, int BC, int OP>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? TVD_LINE_MINB : 1) line_kernel(LineArgs<T> a) {
    // (the implicit trigger at block exit lets the next kernel launch)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n, ns = a.ns, P = a.P, L = a.L;
    const int lines = 2 * P;       // a power of two
    const int lsh = __ffs(lines) - 1;
    const int ln = lines * n;      // line elements of the block
    const int lns = lines * ns;    // shared-memory size of one set of lines
    // FFT twiddles: L of them in shared memory; a Bluestein plan reads its M2
    // twiddles from the (L1-cached) table instead, leaving the shared memory to
    // its FFT buffers of M2 entries per line pair
    const int ntw = a.fp.bl ? 0 : L, Lb = a.fp.bl ? a.fp.M2 : L;
    const cplx<T>* twsrc = a.tw;
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* bufA = tw + ntw;
    cplx<T>* bufB = bufA + (size_t)P * Lb;
    T* raw = reinterpret_cast<T*>(bufB + (size_t)P * Lb);
    T* ex = raw + lns;
    constexpr bool cols = (OP == OP_COL_SOLVE || OP == OP_COL_EG || OP == OP_COL_X);
    // line pairs from two arrays (line a of pair pp from in0, line b from in1)
    constexpr bool two_in = (OP == OP_COL_EG || OP == OP_ROW_X || OP == OP_COL_X);
    // global line index of local line l, or -1
    auto gline = [&](int l) -> int {
        int g;
        if (two_in) g = blockIdx.x * P + (l >> 1);
        else g = blockIdx.x * lines + l;
        return g < a.nlines ? g : -1;
    };

    // ---- stage the lines and their per-pixel factors: asynchronous copies,
    // all of them in flight before the first wait
    for (int i = threadIdx.x; i < ntw; i += kThreads)
        cp_async_elem(&tw[i].re, &twsrc[i].re), cp_async_elem(&tw[i].im, &twsrc[i].im);
    // everything below reads or writes what earlier kernels in the stream touch
    pdl_wait();
    if (a.st && a.st->done) {
        cp_async_wait_all();
        return;
    }
    if (!cols) {
        for (Walk w(n); w.hi < lines; w.next(n)) {
            const int l = w.hi, idx = w.lo;
            const int si = l * ns + idx;
            const int g = gline(l);
            if (g < 0) {
                raw[si] = T(0);
                continue;
            }
            const size_t o = (size_t)g * a.nc + idx;
            cp_async_elem(raw + si, ((two_in && (l & 1)) ? a.in1 : a.in0) + o);
            if ((OP == OP_ROW_FWD || OP == OP_ROW_INV) && a.scale) cp_async_elem(ex + si, a.scale + o);
            if (OP == OP_ROW_INV && a.st) cp_async_elem(ex + lns + si, a.rvec + o);
        }
    } else {
        for (int e = threadIdx.x; e < ln; e += kThreads) {
            const int idx = e >> lsh, l = e & (lines - 1);
            const int g = gline(l);
            const int si = l * ns + idx;
            if (g < 0) {
                raw[si] = T(0);
                continue;
            }
            const size_t o = (size_t)idx * a.nc + g;
            cp_async_elem(raw + si, ((two_in && (l & 1)) ? a.in1 : a.in0) + o);
            if (OP == OP_COL_SOLVE) cp_async_elem(ex + si, a.spec + o);
            if (OP == OP_COL_EG && !(l & 1)) cp_async_elem(ex + 2 * lns + (l >> 1) * ns + idx, a.spec + o);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    // CG path: apply the previous iteration's x += alpha p, r -= alpha q first
    // (this pass preconditions the updated r), then the stopping test
    // (pending is the same for every block: the last block clears it only
    // after all blocks have passed their reduction)
    if (OP == OP_ROW_FWD && a.xvec && a.st->pending) {
        const T al = T(a.st->alpha);
        const T* pv = a.st->pbuf ? a.p0 : a.p1;
        T* rg = const_cast<T*>(a.in0);
        T part = T(0);
        for (Walk w(n); w.hi < lines; w.next(n)) {
            const int l = w.hi, idx = w.lo;
            const int g = gline(l);
            if (g < 0) continue;
            const size_t o = (size_t)g * a.nc + idx;
            const int si = l * ns + idx;
            const T v = raw[si] - al * __ldg(a.qvec + o);
            raw[si] = v;
            rg[o] = v;
            a.xvec[o] += al * __ldg(pv + o);
            part += v * v;
        }
        double sum;
        if (block_reduce_last((double)part, a.red, a.ticket2, blockIdx.x, gridDim.x, &sum) && threadIdx.x == 0)
            finish_xr(a.st, sum);
        __syncthreads();
    }
    if (OP == OP_ROW_FWD && a.scale) {
        for (Walk w(n); w.hi < lines; w.next(n)) {
            const int l = w.hi, si = l * ns + w.lo;
            if (gline(l) >= 0) raw[si] *= ex[si];
        }
        __syncthreads();
    }

    // ---- transform(s)
    if (OP == OP_ROW_X || OP == OP_COL_X) {
        // line a -> out0 = (xa ? F : E) a, line b -> out1 = (xb ? F : E) b, both in the input layout
        T* eo = ex;
        T* fo = ex + lns;
        eg_lines<T, BC>(raw, bufA, bufB, eo, fo, a, tw, true);
        for (Walk w(n); w.hi < lines; w.next(n)) {
            const int l = w.hi, idx = w.lo;
            const int g = gline(l);
            if (g < 0) continue;
            const bool second = (l & 1) ? a.xb != 0 : a.xa != 0;
            const T v = second ? fo[l * ns + idx] : eo[l * ns + idx];
            T* out = (l & 1) ? a.out1 : a.out0;
            out[cols ? (size_t)idx * a.nc + g : (size_t)g * a.nc + idx] = v;
        }
        return;
    }
    if (OP == OP_ROW_EG || OP == OP_COL_EG) {
        T* eo = ex;
        T* go = ex + lns;
        eg_lines<T, BC>(raw, bufA, bufB, eo, go, a, tw);
        if (OP == OP_ROW_EG) {
            for (Walk w(n); w.hi < lines; w.next(n)) {
                const int l = w.hi, idx = w.lo;
                const int g = gline(l);
                if (g < 0) continue;
                const size_t o = (size_t)g * a.nc + idx;
                a.out0[o] = eo[l * ns + idx];
                a.out1[o] = go[l * ns + idx];
            }
        } else {
            // Lambda_L column = G(A col) + E(B col); spec = lamH2 + alpha Lambda_L
            const T* lam = ex + 2 * lns;
            for (int e = threadIdx.x; e < P * n; e += kThreads) {
                const int idx = e >> (lsh - 1), pp = e & (P - 1);
                const int g = gline(2 * pp);
                if (g < 0) continue;
                const T lamL = go[(size_t)(2 * pp) * ns + idx] + eo[(size_t)(2 * pp + 1) * ns + idx];
                if (a.lam_out) {
                    a.lam_out[(size_t)idx * a.nc + g] = lamL;
                    continue;
                }
                const double sp = (double)lam[pp * ns + idx] + a.alpha * (double)lamL;
                if (!(sp > 1e-300) || !isfinite(sp)) atomicOr(a.bad, 1);
                a.inv_out[(size_t)idx * a.nc + g] = T(1.0 / sp);
            }
        }
        return;
    }

    // reblurring: y -/+= y_0 (S p) + y_{n-1} (S J p) on every line's interior (the
    // endpoints, which hat-S passes through, are read but not written)
    auto ucorrect = [&](T sign) {
        __syncthreads();
        for (Walk w(n); w.hi < lines; w.next(n)) {
            const int l = w.hi, idx = w.lo;
            if (idx == 0 || idx == n - 1 || gline(l) < 0) continue;
            const int b0 = l * ns;
            raw[b0 + idx] += sign * (raw[b0] * a.ucorr[idx - 1] + raw[b0 + n - 1] * a.ucorr[n - 2 + idx - 1]);
        }
        __syncthreads();
    };
    if (BC == BCK_AR && OP == OP_ROW_INV && a.ucorr) ucorrect(T(1));    // T_n = hat-S (I + U): (I + U) first
    if (BC == BCK_AR) dst1_lines<T>(raw, bufA, bufB, a, tw);
    else dct_lines<T>(raw, bufA, bufB, a, tw, OP == OP_ROW_INV);
    if (BC == BCK_AR && (OP == OP_ROW_FWD || OP == OP_COL_SOLVE) && a.ucorr) ucorrect(T(-1));   // T_n^-1 = (I - U) hat-S

    if (OP == OP_COL_SOLVE) {
        for (Walk w(n); w.hi < lines; w.next(n)) {
            const int l = w.hi, si = l * ns + w.lo;
            if (gline(l) >= 0) raw[si] *= ex[si];
        }
        __syncthreads();
        if (BC == BCK_AR && a.ucorr) ucorrect(T(1));
        if (BC == BCK_AR) dst1_lines<T>(raw, bufA, bufB, a, tw);
        else dct_lines<T>(raw, bufA, bufB, a, tw, true);
        for (int e = threadIdx.x; e < ln; e += kThreads) {
            const int idx = e >> lsh, l = e & (lines - 1);
            const int g = gline(l);
            if (g >= 0) a.out0[(size_t)idx * a.nc + g] = raw[(size_t)l * ns + idx];
        }
        return;
    }
    // ---- row store (ROW_FWD / ROW_INV)
    T part = T(0);
    for (Walk w(n); w.hi < lines; w.next(n)) {
        const int l = w.hi, idx = w.lo;
        const int g = gline(l);
        if (g < 0) continue;
        const size_t o = (size_t)g * a.nc + idx;
        const int si = l * ns + idx;
        T v = raw[si];
        if (OP == OP_ROW_INV && a.scale) v *= ex[si];
        a.out0[o] = v;
        if (OP == OP_ROW_INV && a.st) part += ex[lns + si] * v;
    }
    if (OP == OP_ROW_INV && a.st) {
        double s;
        if (block_reduce_last((double)part, a.red, a.ticket, blockIdx.x, gridDim.x, &s) && threadIdx.x == 0)
            finish_rho(a.st, s);
    }
}

// ------------------------------------------------------------- host side

FftPlan make_fft_plan(int L) {
    FftPlan fp;
    fp.L = L;
    int m = L;
    auto push = [&](int r) { fp.radix[fp.nstages++] = r; m /= r; };
    while (m % 4 == 0) push(4);
    while (m % 2 == 0) push(2);
    while (m % 9 == 0) push(9);
    static const int odd[] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31};
    for (int r : odd)
        while (m % r == 0) push(r);
    for (int r = 37; m > 1; r += 2)
        while (m % r == 0) push(r);
    // Bluestein from the smallest prime factor that the register butterflies do
    // not take (32); TVD_BLUESTEIN_MIN_PRIME lowers the threshold (tuning)
    static const int min_prime = []() {
        const char* v = std::getenv("TVD_BLUESTEIN_MIN_PRIME");
        const int q = v ? std::atoi(v) : 0;
        return q >= 3 && q <= 32 ? q : 32;
    }();
    for (int s = 0; s < fp.nstages; ++s)
        if (fp.radix[s] >= min_prime) fp.bl = 1;
    if (fp.bl) {
        int M2 = 1;
        while (M2 < 2 * L - 1) M2 *= 2;
        fp.M2 = M2;
        int q = M2;
        while (q % 4 == 0) fp.radix2[fp.nst2++] = 4, q /= 4;
        while (q % 2 == 0) fp.radix2[fp.nst2++] = 2, q /= 2;
    }
    return fp;
}

template <typename T>
static size_t line_smem(const LineArgs<T>& a, int op) {
    const size_t lines = 2 * (size_t)a.P;
    // tw + bufA + bufB + raw + the operation's staged factors / outputs
    const size_t Lb = a.fp.bl ? (size_t)a.fp.M2 : (size_t)a.L;
    return sizeof(cplx<T>) * ((a.fp.bl ? 0 : (size_t)a.L) + 2 * (size_t)a.P * Lb) +
           sizeof(T) * (lines * a.ns + line_extra(op, lines, a.ns, a.P)) + 64;
}

// Tuning override of the line pairs per block (TVD_LINE_PAIRS_ROW / _COL,
// 1..8); 0 = the built-in choice.
static int env_pairs(const char* name) {
    const char* v = std::getenv(name);
    const int P = v ? std::atoi(v) : 0;
    return P >= 1 && P <= 8 ? P : 0;
}

template <typename T>
static void pick_pairs(LineArgs<T>& a, bool cols, int op) {
    // columns: 2 pairs (4 contiguous elements of each row); rows: about 4096
    // (float) / 2048 (double) line elements per block (measured best of the
    // 1-4 pair choices at 1024 x 1024)
    static const int row_env = env_pairs("TVD_LINE_PAIRS_ROW"), col_env = env_pairs("TVD_LINE_PAIRS_COL");
    int P;
    if (cols) {
        P = col_env ? col_env : 2;
    } else {
        P = (int)((sizeof(T) == 4 ? 2048 : 1024) / a.n);
        P = P < 1 ? 1 : (P > 8 ? 8 : P);
        if (row_env) P = row_env;
    }
    while (P & (P - 1)) P &= P - 1;   // a power of two (column index maps use shifts)
    const size_t cap = 160 * 1024;
    for (;;) {
        a.P = P;
        if (cols) {
            // column passes stage element idx of line l at l * ns + idx, a warp
            // covering 32 / 2P indices of all 2P lines: ns = K / 2P (mod K), K the
            // shared-memory words of T in 128 bytes, spreads them over distinct banks
            const int K = 128 / (int)sizeof(T), r = K / (2 * P);
            a.ns = a.n + ((r - a.n % K) % K + K) % K;
        }
        if (P == 1 || line_smem<T>(a, op) <= cap) break;
        P = P / 2;
    }
}

// A column pass over lines of one sample (a 1D signal stored as one row): the
// 1-point transform is the identity, its E weights are 1 and its G (difference)
// and F (neighbour) weights 0, so each operation reduces to an elementwise one.
template <typename T, int OP>
__global__ void __launch_bounds__(kThreads) col1_kernel(LineArgs<T> a) {
    pdl_wait();
    if (a.st && a.st->done) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.nc; j += gridDim.x * blockDim.x) {
        if (OP == OP_COL_SOLVE) {
            a.out0[j] = a.in0[j] * a.spec[j];
        } else if (OP == OP_COL_EG) {
            // Lambda_L = G_col (E_row w) + E_col (G_row w) = G_row w
            const T lamL = a.in1[j];
            if (a.lam_out) {
                a.lam_out[j] = lamL;
                continue;
            }
            const double sp = (double)a.spec[j] + a.alpha * (double)lamL;
            if (!(sp > 1e-300) || !isfinite(sp)) atomicOr(a.bad, 1);
            a.inv_out[j] = T(1.0 / sp);
        } else {   // OP_COL_X: out = (x ? F : E) in
            a.out0[j] = a.xa ? T(0) : a.in0[j];
            a.out1[j] = a.xb ? T(0) : a.in1[j];
        }
    }
}

template <typename T, int BC, int OP>
static tvd_status launch_line(LineArgs<T> a, cudaStream_t s) {
    const bool cols = (OP == OP_COL_SOLVE || OP == OP_COL_EG || OP == OP_COL_X);
    if constexpr (OP == OP_COL_SOLVE || OP == OP_COL_EG || OP == OP_COL_X) {
        if (a.n == 1) {
            ProfScope prof(prof_class<T>(OP == OP_COL_SOLVE ? PROF_COL_SOLVE : PROF_EG_COL), s);
            TVD_CUDA_TRY(launch_pdl(col1_kernel<T, OP>, dim3((a.nc + kThreads - 1) / kThreads), dim3(kThreads), 0,
                                    s, a));
            TVD_CUDA_TRY(cudaGetLastError());
            return TVD_OK;
        }
    }
    pick_pairs<T>(a, cols, OP);
    if (a.fp.bl && line_smem<T>(a, OP) > 227 * 1024) {
        a.fp.bl = 0;   // the M2-point buffers do not fit: direct sums for the large prime factors
        pick_pairs<T>(a, cols, OP);
    }
    const int per_block = (OP == OP_COL_EG || OP == OP_ROW_X || OP == OP_COL_X) ? a.P : 2 * a.P;
    const int blocks = (a.nlines + per_block - 1) / per_block;
    const size_t smem = line_smem<T>(a, OP);
    if (smem > 227 * 1024) {
        set_error("transform line too long for shared memory");
        return TVD_EINVAL;
    }
    if (OP == OP_ROW_INV && a.st && blocks > kMaxRedBlocks) {
        set_error("image too large for the reduction buffer");
        return TVD_EINVAL;
    }
    TVD_CUDA_TRY((allow_max_smem<line_kernel<T, BC, OP>>()));
    constexpr int cls = OP == OP_ROW_FWD ? PROF_ROW_FWD : OP == OP_COL_SOLVE ? PROF_COL_SOLVE
                      : OP == OP_ROW_INV ? PROF_ROW_INV : (OP == OP_ROW_EG || OP == OP_ROW_X) ? PROF_EG_ROW
                      : PROF_EG_COL;
    ProfScope prof(prof_class<T>(cls), s);
    TVD_CUDA_TRY(launch_pdl(line_kernel<T, BC, OP>, dim3(blocks), dim3(kThreads), smem, s, a));
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

template <typename T>
static LineArgs<T> base_args(const tvd_plan_s& p, const Ops<T>& o, bool cols) {
    LineArgs<T> a{};
    a.nr = p.nr;
    a.nc = p.nc;
    a.n = cols ? p.nr : p.nc;
    a.ns = a.n | 1;
    a.nlines = cols ? p.nc : p.nr;
    a.fp = cols ? p.fft_r : p.fft_c;
    a.L = a.fp.L;
    a.tw = cols ? o.tw_r : o.tw_c;
    a.blt = cols ? o.blt_r : o.blt_c;
    a.aux = cols ? o.aux_r : o.aux_c;
    a.red = p.red;
    a.ticket = p.ticket + 2;
    a.ucorr = p.reblur() ? (cols ? o.ucorr_r : o.ucorr_c) : nullptr;
    return a;
}

template <typename T>
tvd_status precond_solve(const tvd_plan_s& p, const Ops<T>& o, const T* r, T* z, CgState* st, cudaStream_t s,
                         T* x) {
    if constexpr (sizeof(T) == 4) {
        if (p.gemm) return gemm_precond_solve(p, o, r, z, st, s, x);
    }
    const bool scaled = (p.pc == TVD_PC_DFAST || p.pc == TVD_PC_FASTD);
    LineArgs<T> a = base_args<T>(p, o, false);
    a.in0 = r;
    a.out0 = o.t;
    a.scale = scaled ? o.dmh : nullptr;
    a.st = st;                   // with x also: the CG iteration's pending x / r update and stopping test
    a.xvec = x;
    a.qvec = o.q;
    a.p0 = o.p;
    a.p1 = o.p2;
    a.ticket2 = p.ticket + 7;
    LineArgs<T> c = base_args<T>(p, o, true);
    c.in0 = o.t;
    c.out0 = o.t;
    c.spec = o.inv_spec;
    c.st = st;
    LineArgs<T> b = base_args<T>(p, o, false);
    b.in0 = o.t;
    b.out0 = z;
    b.scale = scaled ? o.dmh : nullptr;
    b.rvec = r;
    b.st = st;
    if (p.bc == TVD_BC_ANTIREFLECTIVE) {
        TVD_TRY((launch_line<T, BCK_AR, OP_ROW_FWD>(a, s)));
        TVD_TRY((launch_line<T, BCK_AR, OP_COL_SOLVE>(c, s)));
        TVD_TRY((launch_line<T, BCK_AR, OP_ROW_INV>(b, s)));
    } else {
        TVD_TRY((launch_line<T, BCK_R, OP_ROW_FWD>(a, s)));
        TVD_TRY((launch_line<T, BCK_R, OP_COL_SOLVE>(c, s)));
        TVD_TRY((launch_line<T, BCK_R, OP_ROW_INV>(b, s)));
    }
    return TVD_OK;
}

// Weights of the scaled-system spectrum (R_D / M_D), d = D^-1/2: S = d^2 diag(L(w))
// (the stencil diagonal with d^2 at the pixel), gamma = w d_{i+1,j} d_ij (rows),
// delta = w d_{i,j+1} d_ij (columns), zero where the forward difference is.
template <typename T>
__global__ void __launch_bounds__(kThreads)
scaled_weights_kernel(const T* __restrict__ w, const T* __restrict__ d, T* __restrict__ S, T* __restrict__ gam,
                      T* __restrict__ dlt, T* __restrict__ dout, int nr, int nc) {
    const size_t n = (size_t)nr * nc;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(o / nc), j = (int)(o - (size_t)i * nc);
        const T di = d[o];
        T diag = T(0);
        if (i < nr - 1) diag += w[o];
        if (i > 0) diag += w[o - nc];
        if (j < nc - 1) diag += w[o];
        if (j > 0) diag += w[o - 1];
        S[o] = di * di * diag;
        gam[o] = i < nr - 1 ? w[o] * d[o + nc] * di : T(0);
        dlt[o] = j < nc - 1 ? w[o] * d[o + 1] * di : T(0);
        dout[o] = di;
    }
}

// 1 / (Lambda_H^2 Lambda_D^2 + alpha Lambda_L~) with Lambda_L~ = U1 - 2 U2 - 2 U3, Lambda_D = U4.
template <typename T>
__global__ void __launch_bounds__(kThreads)
scaled_spec_kernel(const T* __restrict__ lamH2, const T* __restrict__ U1, const T* __restrict__ U2,
                   const T* __restrict__ U3, const T* __restrict__ U4, double alpha, T* __restrict__ inv_out,
                   int* bad, size_t n) {
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const double ld = (double)U4[o];
        const double lt = (double)U1[o] - 2.0 * (double)U2[o] - 2.0 * (double)U3[o];
        const double sp = (double)lamH2[o] * ld * ld + alpha * lt;
        if (!(sp > 1e-300) || !isfinite(sp)) atomicOr(bad, 1);
        inv_out[o] = T(1.0 / sp);
    }
}

// The R_D / M_D spectrum: Lambda_D = E_r d E_c^T and
// Lambda_L~ = E_r S E_c^T - 2 F_r gamma E_c^T - 2 E_r delta F_c^T as two row passes
// (E_c S, E_c gamma | F_c delta, E_c d), two column passes and an elementwise finish.
// Uses o.z, o.p, o.p2, o.q, o.r, o.x, o.t, o.t2 as scratch (free between solves).
template <typename T>
static tvd_status scaled_spectrum_setup(const tvd_plan_s& p, Ops<T>& o, double alpha, int* bad_flag,
                                        cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    const int blocks = num_sms() * 4;
    {
        ProfScope prof(prof_class<T>(PROF_TV), s);
        scaled_weights_kernel<T><<<blocks, kThreads, 0, s>>>(o.w, o.dmh, o.z, o.p, o.p2, o.q, p.nr, p.nc);
        TVD_CUDA_TRY(cudaGetLastError());
    }
    auto pass = [&](bool cols, const T* in0, const T* in1, T* out0, T* out1, int xa, int xb) -> tvd_status {
        LineArgs<T> a = base_args<T>(p, o, cols);
        a.in0 = in0;
        a.in1 = in1;
        a.out0 = out0;
        a.out1 = out1;
        a.xa = xa;
        a.xb = xb;
        if (p.bc == TVD_BC_ANTIREFLECTIVE)
            return cols ? launch_line<T, BCK_AR, OP_COL_X>(a, s) : launch_line<T, BCK_AR, OP_ROW_X>(a, s);
        return cols ? launch_line<T, BCK_R, OP_COL_X>(a, s) : launch_line<T, BCK_R, OP_ROW_X>(a, s);
    };
    TVD_TRY(pass(false, o.z, o.p, o.t, o.t2, 0, 0));    // E_c S, E_c gamma
    TVD_TRY(pass(false, o.p2, o.q, o.r, o.x, 1, 0));    // F_c delta, E_c d
    TVD_TRY(pass(true, o.t, o.t2, o.z, o.p, 0, 1));     // E_r (E_c S), F_r (E_c gamma)
    TVD_TRY(pass(true, o.r, o.x, o.p2, o.q, 0, 0));     // E_r (F_c delta), E_r (E_c d)
    ProfScope prof(prof_class<T>(PROF_EG_COL), s);
    scaled_spec_kernel<T><<<blocks, kThreads, 0, s>>>(o.lamH2, o.z, o.p, o.p2, o.q, alpha, o.inv_spec, bad_flag, n);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

// ---------------------------------------------------------------- reblurring spectrum
//
// Eigenvalues of the level-2 projection AR_2(X) (Sec. 3.2) from the interior
// ones, which equal those of the sine projection of X's interior block: along
// each dimension the two border eigenvalues are the symbol at 0 of the tau
// matrix with those interior eigenvalues, a fixed linear functional c of them
// (c from the host). Border columns first (interior rows), then border rows
// over all columns (so the corners get both functionals).
template <typename T>
__global__ void __launch_bounds__(kThreads)
ar_ext_cols_kernel(T* __restrict__ X, int nr, int nc, const double* __restrict__ cc) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    // interior rows; a single row (a 1D signal) has no border row, so it is extended itself
    const int i0 = nr == 1 ? 0 : 1, i1 = nr == 1 ? 0 : nr - 2;
    for (int i = i0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); i <= i1; i += warps) {
        const T* row = X + (size_t)i * nc;
        double acc = 0.0;
        for (int j = 1 + lane; j <= nc - 2; j += 32) acc += cc[j - 1] * (double)row[j];
        acc = warp_sum(acc);
        if (lane == 0) X[(size_t)i * nc] = X[(size_t)i * nc + nc - 1] = T(acc);
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
ar_ext_rows_kernel(T* __restrict__ X, int nr, int nc, const double* __restrict__ cr) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nc; j += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int i = 1; i <= nr - 2; ++i) acc += cr[i - 1] * (double)X[(size_t)i * nc + j];
        X[j] = X[(size_t)(nr - 1) * nc + j] = T(acc);
    }
}

// lamLt = U1 - 2 U2 - 2 U3 (the scaled-system Lambda_L~ before the extension)
template <typename T>
__global__ void __launch_bounds__(kThreads)
combine_lt_kernel(const T* __restrict__ U1, const T* __restrict__ U2, const T* __restrict__ U3, T* __restrict__ out,
                  size_t n) {
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
        out[o] = T((double)U1[o] - 2.0 * (double)U2[o] - 2.0 * (double)U3[o]);
}

// 1 / (Lambda_H^2 [Lambda_D^2] + alpha Lambda_L)
template <typename T>
__global__ void __launch_bounds__(kThreads)
reblur_spec_kernel(const T* __restrict__ lamH2, const T* __restrict__ lamL, const T* __restrict__ lamD,
                   double alpha, T* __restrict__ inv_out, int* bad, size_t n) {
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        double h2 = (double)lamH2[o];
        if (lamD) h2 *= (double)lamD[o] * (double)lamD[o];
        const double sp = h2 + alpha * (double)lamL[o];
        if (!(sp > 1e-300) || !isfinite(sp)) atomicOr(bad, 1);
        inv_out[o] = T(1.0 / sp);
    }
}

template <typename T>
static tvd_status ar_extend(const tvd_plan_s& p, const Ops<T>& o, T* X, cudaStream_t s) {
    const int blocks = num_sms() * 4;
    ar_ext_cols_kernel<T><<<blocks, kThreads, 0, s>>>(X, p.nr, p.nc, o.extc_c);
    TVD_CUDA_TRY(cudaGetLastError());
    if (p.nr == 1) return TVD_OK;
    ar_ext_rows_kernel<T><<<(p.nc + kThreads - 1) / kThreads, kThreads, 0, s>>>(X, p.nr, p.nc, o.extc_r);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

// P / D_P: Lambda_H^2 + alpha Lambda_AR2(L); P_D: Lambda_H^2 Lambda_D^2 + alpha Lambda_L~ with both
// projections extended (uses o.z, o.p, o.p2, o.q, o.r, o.x, o.t, o.t2 as scratch).
template <typename T>
static tvd_status reblur_spectrum_setup(const tvd_plan_s& p, Ops<T>& o, double alpha, int* bad_flag,
                                        cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    const int blocks = num_sms() * 4;
    if (p.pc == TVD_PC_FASTD) {
        {
            ProfScope prof(prof_class<T>(PROF_TV), s);
            scaled_weights_kernel<T><<<blocks, kThreads, 0, s>>>(o.w, o.dmh, o.z, o.p, o.p2, o.q, p.nr, p.nc);
            TVD_CUDA_TRY(cudaGetLastError());
        }
        auto pass = [&](bool cols, const T* in0, const T* in1, T* out0, T* out1, int xa, int xb) -> tvd_status {
            LineArgs<T> a = base_args<T>(p, o, cols);
            a.in0 = in0;
            a.in1 = in1;
            a.out0 = out0;
            a.out1 = out1;
            a.xa = xa;
            a.xb = xb;
            return cols ? launch_line<T, BCK_AR, OP_COL_X>(a, s) : launch_line<T, BCK_AR, OP_ROW_X>(a, s);
        };
        TVD_TRY(pass(false, o.z, o.p, o.t, o.t2, 0, 0));
        TVD_TRY(pass(false, o.p2, o.q, o.r, o.x, 1, 0));
        TVD_TRY(pass(true, o.t, o.t2, o.z, o.p, 0, 1));
        TVD_TRY(pass(true, o.r, o.x, o.p2, o.q, 0, 0));
        ProfScope prof(prof_class<T>(PROF_EG_COL), s, 4);
        combine_lt_kernel<T><<<blocks, kThreads, 0, s>>>(o.z, o.p, o.p2, o.t, n);
        TVD_CUDA_TRY(cudaGetLastError());
        TVD_TRY(ar_extend<T>(p, o, o.t, s));     // Lambda_L~
        TVD_TRY(ar_extend<T>(p, o, o.q, s));     // Lambda_D
        reblur_spec_kernel<T><<<blocks, kThreads, 0, s>>>(o.lamH2, o.t, o.q, alpha, o.inv_spec, bad_flag, n);
        TVD_CUDA_TRY(cudaGetLastError());
        return TVD_OK;
    }
    LineArgs<T> a = base_args<T>(p, o, false);
    a.in0 = o.w;
    a.out0 = o.t;
    a.out1 = o.t2;
    LineArgs<T> c = base_args<T>(p, o, true);
    c.in0 = o.t;
    c.in1 = o.t2;
    c.spec = o.lamH2;
    c.lam_out = o.z;
    c.alpha = alpha;
    c.bad = bad_flag;
    TVD_TRY((launch_line<T, BCK_AR, OP_ROW_EG>(a, s)));
    TVD_TRY((launch_line<T, BCK_AR, OP_COL_EG>(c, s)));
    ProfScope prof(prof_class<T>(PROF_EG_COL), s, 3);
    TVD_TRY(ar_extend<T>(p, o, o.z, s));
    reblur_spec_kernel<T><<<blocks, kThreads, 0, s>>>(o.lamH2, o.z, (const T*)nullptr, alpha, o.inv_spec, bad_flag,
                                                       n);
    TVD_CUDA_TRY(cudaGetLastError());
    return TVD_OK;
}

template <typename T>
tvd_status spectrum_setup(const tvd_plan_s& p, Ops<T>& o, double alpha, int* bad_flag, cudaStream_t s) {
    if (p.reblur()) return reblur_spectrum_setup<T>(p, o, alpha, bad_flag, s);
    if (p.pc == TVD_PC_FASTD) return scaled_spectrum_setup<T>(p, o, alpha, bad_flag, s);
    LineArgs<T> a = base_args<T>(p, o, false);
    a.in0 = o.w;
    a.out0 = o.t;
    a.out1 = o.t2;
    LineArgs<T> c = base_args<T>(p, o, true);
    c.in0 = o.t;
    c.in1 = o.t2;
    c.spec = o.lamH2;
    c.inv_out = o.inv_spec;
    c.alpha = alpha;
    c.bad = bad_flag;
    if (p.bc == TVD_BC_ANTIREFLECTIVE) {
        TVD_TRY((launch_line<T, BCK_AR, OP_ROW_EG>(a, s)));
        TVD_TRY((launch_line<T, BCK_AR, OP_COL_EG>(c, s)));
    } else {
        TVD_TRY((launch_line<T, BCK_R, OP_ROW_EG>(a, s)));
        TVD_TRY((launch_line<T, BCK_R, OP_COL_EG>(c, s)));
    }
    return TVD_OK;
}

// Lambda_H^2[i,j] = (sum_a cos(a y_i) G[a][j])^2, G[a][j] = sum_b h_ab cos(b y_j) (eq. (symb)
// at the grid of eq. (gridy) for AR, y_k = k pi / n for R). cr: n_r x (2 m_r + 1) table of cos(a y_i).
template <typename T>
__global__ void lamH2_kernel(const double* __restrict__ cr, const double* __restrict__ G, T* __restrict__ out,
                             int nr, int nc, int pr) {
    const size_t n = (size_t)nr * nc;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(o / nc), j = (int)(o - (size_t)i * nc);
        double acc = 0.0;
        for (int a = 0; a < pr; ++a) acc += cr[(size_t)i * pr + a] * G[(size_t)a * nc + j];
        out[o] = T(acc * acc);
    }
}

static std::vector<double> symbol_grid(int n, tvd_bc bc) {
    if (n == 1) return std::vector<double>(1, 0.0);   // one sample: the constant, y = 0
    std::vector<double> y(n);
    for (int k = 0; k < n; ++k) y[k] = (bc == TVD_BC_ANTIREFLECTIVE) ? k * M_PI / (n - 1) : k * M_PI / n;
    if (bc == TVD_BC_ANTIREFLECTIVE) {
        y[0] = 0.0;
        y[n - 1] = 0.0;
    }
    return y;
}

template <typename T>
tvd_status lamH2_setup(const tvd_plan_s& p, Ops<T>& o, cudaStream_t s) {
    const int mr = p.psf.mr, mc = p.psf.mc, pr = 2 * mr + 1, pc = 2 * mc + 1;
    const std::vector<double> yr = symbol_grid(p.nr, p.bc), yc = symbol_grid(p.nc, p.bc);
    std::vector<double> cr((size_t)p.nr * pr), G((size_t)pr * p.nc, 0.0);
    for (int i = 0; i < p.nr; ++i)
        for (int a = -mr; a <= mr; ++a) cr[(size_t)i * pr + a + mr] = std::cos(a * yr[i]);
    for (int a = 0; a < pr; ++a)
        for (int j = 0; j < p.nc; ++j) {
            double acc = 0.0;
            for (int b = -mc; b <= mc; ++b) acc += p.psf.h[(size_t)a * pc + b + mc] * std::cos(b * yc[j]);
            G[(size_t)a * p.nc + j] = acc;
        }
    double *dcr = nullptr, *dG = nullptr;
    TVD_CUDA_TRY(cudaMalloc(&dcr, cr.size() * sizeof(double)));
    if (cudaMalloc(&dG, G.size() * sizeof(double)) != cudaSuccess) {
        cudaFree(dcr);
        set_error("cudaMalloc failed");
        return TVD_ENOMEM;
    }
    cudaMemcpyAsync(dcr, cr.data(), cr.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dG, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    count_launches(1);
    lamH2_kernel<T><<<num_sms() * 4, kThreads, 0, s>>>(dcr, dG, o.lamH2, p.nr, p.nc, pr);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(dcr);
    cudaFree(dG);
    if (e != cudaSuccess) {
        set_error(std::string("CUDA error: ") + cudaGetErrorString(e));
        return TVD_ECUDA;
    }
    return TVD_OK;
}

template tvd_status precond_solve<float>(const tvd_plan_s&, const Ops<float>&, const float*, float*, CgState*,
                                         cudaStream_t, float*);
template tvd_status precond_solve<double>(const tvd_plan_s&, const Ops<double>&, const double*, double*, CgState*,
                                          cudaStream_t, double*);
template tvd_status spectrum_setup<float>(const tvd_plan_s&, Ops<float>&, double, int*, cudaStream_t);
template tvd_status spectrum_setup<double>(const tvd_plan_s&, Ops<double>&, double, int*, cudaStream_t);
template tvd_status lamH2_setup<float>(const tvd_plan_s&, Ops<float>&, cudaStream_t);
template tvd_status lamH2_setup<double>(const tvd_plan_s&, Ops<double>&, cudaStream_t);

}  // namespace tvd
