// C ABI of libtvd: plan construction and validation, the operator entry
// points, the PCG driver (Golub & Van Loan Alg. 10.3.1, as cited in Sec. 1),
// mixed-precision iterative refinement and the lagged-diffusivity FP loop of
// eq. (fp) with u^0 = v and warm starts u^k (Sec. 5).
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>

namespace tvd {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

template <typename T>
static tvd_status dalloc(T** p, size_t n) {
    if (n == 0) n = 1;
    if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed");
        return TVD_ENOMEM;
    }
    return TVD_OK;
}

template <typename T>
static void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

template <typename T>
static tvd_status upload(T** dst, const std::vector<double>& src, cudaStream_t s) {
    TVD_TRY(dalloc(dst, src.size()));
    std::vector<T> tmp(src.begin(), src.end());
    TVD_CUDA_TRY(cudaMemcpyAsync(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    TVD_CUDA_TRY(cudaStreamSynchronize(s));
    return TVD_OK;
}

// Twiddles exp(-2 pi i k / L) and the auxiliary tables of transform.cu for a
// line of length n (slot layout documented there).
static void transform_tables(int n, tvd_bc bc, std::vector<double>& tw, std::vector<double>& aux) {
    const int L = (bc == TVD_BC_ANTIREFLECTIVE) ? n - 1 : n;
    tw.assign(2 * (size_t)L, 0.0);
    for (int k = 0; k < L; ++k) {
        const double a = 2.0 * M_PI * k / L;
        tw[2 * k] = std::cos(a);
        tw[2 * k + 1] = -std::sin(a);
    }
    aux.assign(16 * (size_t)n, 0.0);
    double* s0 = aux.data();
    double* s1 = aux.data() + 2 * n;
    double* s2 = aux.data() + 4 * n;
    double* s3 = aux.data() + 6 * n;
    double* s4 = aux.data() + 8 * n;
    double* s5 = aux.data() + 10 * n;
    if (bc == TVD_BC_ANTIREFLECTIVE) {
        const int M = n - 1;
        for (int j = 0; j < M; ++j) s0[j] = std::sin(j * M_PI / M);
        for (int k = 0; k < n; ++k) {
            s1[2 * k] = std::cos(M_PI * k / M);
            s1[2 * k + 1] = std::sin(M_PI * k / M);
            const double sh = std::sin(k * M_PI / (2.0 * M));
            s2[k] = 4.0 / M * sh * sh;
        }
    } else {
        for (int k = 0; k < n; ++k) {
            const double c = k == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
            s0[k] = c;
            s1[2 * k] = std::cos(M_PI * k / (2.0 * n));
            s1[2 * k + 1] = std::sin(M_PI * k / (2.0 * n));
            s2[2 * k] = std::cos(M_PI * k / n);
            s2[2 * k + 1] = std::sin(M_PI * k / n);
            s3[k] = c * c / 2.0;
            const double sh = std::sin(M_PI * k / (2.0 * n));
            s4[k] = 2.0 * c * c * sh * sh;
            s5[k] = 1.0 / (n * c);
        }
    }
}

// Bluestein tables of a plan with fp.bl, as interleaved (re, im) doubles:
// chirp c_j = exp(-i pi j^2 / L) (j < L); the spectrum of the filter
// b_m = conj(c_|m|) (m = -(L-1) .. L-1, circular in M2) divided by M2; the M2
// twiddles exp(-2 pi i k / M2). The filter spectrum comes from a radix-2 FFT
// on the host in double.
static void bluestein_tables(const FftPlan& fp, std::vector<double>& out) {
    const int L = fp.L, M2 = fp.M2;
    std::vector<std::complex<double>> c(L), b(M2, 0.0);
    for (int j = 0; j < L; ++j) {
        const long long q = ((long long)j * j) % (2LL * L);   // exact j^2 mod 2L keeps the angle small
        c[j] = std::polar(1.0, -M_PI * (double)q / L);
    }
    b[0] = std::conj(c[0]);
    for (int m = 1; m < L; ++m) b[m] = b[M2 - m] = std::conj(c[m]);
    // iterative radix-2 DFT of b (bit reversal, then butterflies)
    for (int i = 1, j = 0; i < M2; ++i) {
        int bit = M2 >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(b[i], b[j]);
    }
    for (int len = 2; len <= M2; len <<= 1)
        for (int i = 0; i < M2; i += len)
            for (int k = 0; k < len / 2; ++k) {
                const std::complex<double> w = std::polar(1.0, -2.0 * M_PI * k / len);
                const std::complex<double> u = b[i + k], v = b[i + k + len / 2] * w;
                b[i + k] = u + v;
                b[i + k + len / 2] = u - v;
            }
    out.assign(2 * ((size_t)L + 2 * (size_t)M2), 0.0);
    for (int j = 0; j < L; ++j) {
        out[2 * j] = c[j].real();
        out[2 * j + 1] = c[j].imag();
    }
    for (int m = 0; m < M2; ++m) {
        out[2 * ((size_t)L + m)] = b[m].real() / M2;
        out[2 * ((size_t)L + m) + 1] = b[m].imag() / M2;
        const std::complex<double> w = std::polar(1.0, -2.0 * M_PI * m / M2);
        out[2 * ((size_t)L + M2 + m)] = w.real();
        out[2 * ((size_t)L + M2 + m) + 1] = w.imag();
    }
}

template <typename T>
static tvd_status ops_alloc(tvd_plan_s& p, Ops<T>& o, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    T** arrays[] = {&o.lamH2, &o.inv_spec, &o.w, &o.dmh, &o.dinv, &o.x, &o.r, &o.z, &o.p, &o.p2, &o.q, &o.t, &o.t2};
    for (T** a : arrays) TVD_TRY(dalloc(a, n));
    o.allocated = true;
    // PSF taps: dense, plus per-column tap-row ranges
    const int mr = p.psf.mr, mc = p.psf.mc, pw = 2 * mc + 1;
    std::vector<double> rng(2 * (size_t)pw);
    for (int b = -mc; b <= mc; ++b) {
        int lo = mr + 1, hi = -mr - 1;
        for (int a = -mr; a <= mr; ++a)
            if (p.psf.h[(size_t)(a + mr) * pw + (b + mc)] != 0.0) {
                lo = std::min(lo, a);
                hi = std::max(hi, a);
            }
        rng[2 * (b + mc)] = lo;
        rng[2 * (b + mc) + 1] = hi;
    }
    TVD_TRY(upload<int>(&o.arange, rng, s));
    TVD_TRY(upload<T>(&o.hdense, p.psf.h, s));
    // constant runs along each PSF row; used when 2 prefix loads + 1 FMA per run
    // beat the register-window stencil (~2.4 instructions per nonzero tap)
    std::vector<double> run_ab, run_v;
    int nz = 0;
    for (int a = -mr; a <= mr; ++a) {
        int b = -mc;
        while (b <= mc) {
            const double v = p.psf.h[(size_t)(a + mr) * pw + (b + mc)];
            int e = b;
            while (e + 1 <= mc && p.psf.h[(size_t)(a + mr) * pw + (e + 1 + mc)] == v) ++e;
            if (v != 0.0) {
                run_ab.push_back(a);
                run_ab.push_back(b);
                run_ab.push_back(e);
                run_v.push_back(v);
                nz += e - b + 1;
            }
            b = e + 1;
        }
    }
    const int nr_runs = (int)run_v.size();
    if (nr_runs > 0 && 4.0 * nr_runs + 4.0 < 2.4 * nz) {
        TVD_TRY(upload<int>(&o.runs, run_ab, s));
        TVD_TRY(upload<T>(&o.runv, run_v, s));
        o.nruns = nr_runs;
    }
    // flat PSF on a centred, symmetric support whose rows and columns are runs (the disk)
    {
        double fv = 0.0;
        bool flat = mr <= 8 && mc <= 8;
        for (size_t k = 0; k < p.psf.h.size() && flat; ++k) {
            const double hv = p.psf.h[k];
            if (hv == 0.0) continue;
            if (fv == 0.0) fv = hv;
            else if (hv != fv) flat = false;
        }
        flat = flat && fv != 0.0;
        auto nz = [&](int a, int b) { return p.psf.h[(size_t)(a + mr) * pw + (b + mc)] != 0.0; };
        std::vector<double> colh(pw, -1.0);
        for (int b = -mc; b <= mc && flat; ++b) {
            int g = -1;
            while (g + 1 <= mr && nz(g + 1, b)) ++g;    // column b: rows -g .. g, nothing beyond
            for (int a = g + 1; a <= mr && flat; ++a) flat = !nz(a, b) && !nz(-a, b);
            colh[b + mc] = g;
        }
        for (int a = -mr; a <= mr && flat; ++a) {      // rows: runs centred on 0
            int w = -1;
            while (w + 1 <= mc && nz(a, w + 1)) ++w;
            for (int b = w + 1; b <= mc && flat; ++b) flat = !nz(a, b) && !nz(a, -b);
        }
        if (flat) {
            TVD_TRY(upload<int>(&o.colh, colh, s));
            o.flatv = fv;
            o.flat = 1;
            // the disk of radius 7 exactly (a^2 + b^2 <= 49) has its own stencil
            bool disk = mr == 7 && mc == 7;
            for (int a = -mr; a <= mr && disk; ++a)
                for (int b = -mc; b <= mc && disk; ++b) disk = nz(a, b) == (a * a + b * b <= 49);
            if (disk) o.flat = 2;
        }
    }
    TVD_TRY(upload<T>(&o.crow, p.psf.crow, s));
    TVD_TRY(upload<T>(&o.ccol, p.psf.ccol, s));
    TVD_TRY(upload<T>(&o.ccor, p.psf.ccor, s));
    std::vector<double> tw, aux;
    transform_tables(p.nc, p.bc, tw, aux);
    TVD_TRY(upload<T>((T**)&o.tw_c, tw, s));
    TVD_TRY(upload<T>(&o.aux_c, aux, s));
    if (p.nr > 1) {
        transform_tables(p.nr, p.bc, tw, aux);
    } else {
        tw.assign(2, 0.0);
        aux.assign(16, 0.0);
    }
    TVD_TRY(upload<T>((T**)&o.tw_r, tw, s));
    TVD_TRY(upload<T>(&o.aux_r, aux, s));
    if (p.fft_c.bl) {
        bluestein_tables(p.fft_c, tw);
        TVD_TRY(upload<T>((T**)&o.blt_c, tw, s));
    }
    if (p.fft_r.bl) {
        bluestein_tables(p.fft_r, tw);
        TVD_TRY(upload<T>((T**)&o.blt_r, tw, s));
    }
    TVD_TRY(lamH2_setup<T>(p, o, s));
    return TVD_OK;
}

template <typename T>
static void ops_free(Ops<T>& o) {
    dfree(o.hdense); dfree(o.arange); dfree(o.runs); dfree(o.runv); o.nruns = 0; dfree(o.colh); o.flat = 0; dfree(o.crow); dfree(o.ccol); dfree(o.ccor);
    dfree(o.tw_c); dfree(o.tw_r); dfree(o.aux_c); dfree(o.aux_r); dfree(o.blt_c); dfree(o.blt_r);
    dfree(o.lamH2); dfree(o.inv_spec); dfree(o.w); dfree(o.dmh); dfree(o.dinv);
    dfree(o.x); dfree(o.r); dfree(o.z); dfree(o.p); dfree(o.p2); dfree(o.q); dfree(o.t); dfree(o.t2);
    o.allocated = false;
}

// Drop every captured solver chunk: they hold the current preconditioner form's launches.
static void reset_graphs(tvd_plan_s& p) {
    for (auto& g : p.graph) g.reset();
    reblur_graphs_reset(p);
}

static void plan_free(tvd_plan_s* p) {
    for (auto& g : p->graph) g.reset();
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    p->cap_stream = nullptr;
    gemm_precond_destroy(*p);
    reblur_free(*p);
    ops_free(p->d);
    ops_free(p->f);
    dfree(p->state); dfree(p->red); dfree(p->ticket); dfree(p->scal);
    dfree(p->hx); dfree(p->res); dfree(p->xd); dfree(p->tmp);
    if (p->hstate) cudaFreeHost(p->hstate);
    p->hstate = nullptr;
}

// Validate and trim the PSF; build the nonzero tap list and the AR border tail weights.
tvd_status build_psf(Psf& out, const double* h, int pr, int pc, int nr, int nc) {
    if (!h || pr < 1 || pc < 1 || pr % 2 == 0 || pc % 2 == 0) {
        set_error("PSF sides must be odd and positive");
        return TVD_EPSF_SIZE;
    }
    int mr = pr / 2, mc = pc / 2;
    double hmax = 0.0;
    for (int i = 0; i < pr * pc; ++i) {
        if (!std::isfinite(h[i])) {
            set_error("PSF has a non-finite entry");
            return TVD_EINVAL;
        }
        hmax = std::max(hmax, std::fabs(h[i]));
    }
    if (hmax == 0.0) {
        set_error("PSF is zero");
        return TVD_EINVAL;
    }
    auto H = [&](int a, int b) { return h[(size_t)(a + pr / 2) * pc + (b + pc / 2)]; };
    const double tol = 1e-12 * hmax;
    for (int a = -pr / 2; a <= pr / 2; ++a)
        for (int b = -pc / 2; b <= pc / 2; ++b)
            if (std::fabs(H(a, b) - H(-a, b)) > tol || std::fabs(H(a, b) - H(a, -b)) > tol) {
                set_error("PSF is not quadrantally symmetric (h_{a,b} = h_{-a,b} = h_{a,-b} is required)");
                return TVD_EPSF_ASYM;
            }
    // trim all-zero outer rows / columns (H does not change)
    auto row_zero = [&](int a) {
        for (int b = -mc; b <= mc; ++b) if (H(a, b) != 0.0) return false;
        return true;
    };
    auto col_zero = [&](int b) {
        for (int a = -mr; a <= mr; ++a) if (H(a, b) != 0.0) return false;
        return true;
    };
    while (mr > 0 && row_zero(mr) && row_zero(-mr)) --mr;
    while (mc > 0 && col_zero(mc) && col_zero(-mc)) --mc;
    if ((nr == 1 ? mr > 0 : mr > nr - 2) || mc > nc - 2) {
        set_error(nr == 1 ? "a 1D signal (n_rows = 1) needs a PSF of one row"
                          : "PSF half-width exceeds n - 2 along an axis");
        return TVD_EPSF_SIZE;
    }
    if (mr > 48 || mc > 48) {
        set_error("PSF half-width above 48 is not supported");
        return TVD_EPSF_SIZE;
    }
    out.mr = mr;
    out.mc = mc;
    const int qr = 2 * mr + 1, qc = 2 * mc + 1;
    out.h.assign((size_t)qr * qc, 0.0);
    out.ta.clear(); out.tb.clear(); out.th.clear();
    for (int a = -mr; a <= mr; ++a)
        for (int b = -mc; b <= mc; ++b) {
            const double v = H(a, b);
            out.h[(size_t)(a + mr) * qc + (b + mc)] = v;
            if (v != 0.0) {
                out.ta.push_back(a);
                out.tb.push_back(b);
                out.th.push_back(v);
            }
        }
    auto Hs = [&](int a, int b) { return out.h[(size_t)(a + mr) * qc + (b + mc)]; };
    out.crow.assign((size_t)(mr + 1) * qc, 0.0);
    for (int i = 0; i <= mr; ++i)
        for (int b = -mc; b <= mc; ++b) {
            double v = Hs(i, b);
            for (int s = i + 1; s <= mr; ++s) v += 2.0 * Hs(s, b);
            out.crow[(size_t)i * qc + b + mc] = v;
        }
    out.ccol.assign((size_t)qr * (mc + 1), 0.0);
    for (int a = -mr; a <= mr; ++a)
        for (int j = 0; j <= mc; ++j) {
            double v = Hs(a, j);
            for (int t = j + 1; t <= mc; ++t) v += 2.0 * Hs(a, t);
            out.ccol[(size_t)(a + mr) * (mc + 1) + j] = v;
        }
    out.ccor.assign((size_t)(mr + 1) * (mc + 1), 0.0);
    for (int i = 0; i <= mr; ++i)
        for (int j = 0; j <= mc; ++j) {
            double v = Hs(i, j);
            for (int s = i + 1; s <= mr; ++s) v += 2.0 * Hs(s, j);
            for (int t = j + 1; t <= mc; ++t) v += 2.0 * Hs(i, t);
            for (int s = i + 1; s <= mr; ++s)
                for (int t = j + 1; t <= mc; ++t) v += 4.0 * Hs(s, t);
            out.ccor[(size_t)i * (mc + 1) + j] = v;
        }
    return TVD_OK;
}

// ---------------------------------------------------------------- transform form

static bool fast_pc(tvd_precond pc) { return pc == TVD_PC_FAST || pc == TVD_PC_DFAST || pc == TVD_PC_FASTD; }

// Transform form a new MIXED plan with a fast preconditioner starts with: the
// GEMM form when both sides are at least TVD_GEMM_MIN_SIDE (default 128;
// measured faster than the FFT line kernels from 128 to 2048, and the batch of
// 128-512 images 74 -> 87 deblurs/s against a bound of 256), else the FFT form.
// TVD_TRANSFORM=gemm / fft overrides the rule.
static tvd_transform default_transform(const tvd_plan_s& p) {
    if (p.mode != TVD_MODE_MIXED || !fast_pc(p.pc) || p.nr == 1) return TVD_TRANSFORM_FFT;
    const char* v = std::getenv("TVD_TRANSFORM");
    if (v && !std::strcmp(v, "gemm")) return TVD_TRANSFORM_GEMM;
    if (v && !std::strcmp(v, "fft")) return TVD_TRANSFORM_FFT;
    const char* m = std::getenv("TVD_GEMM_MIN_SIDE");
    const int min_side = m ? std::atoi(m) : 128;
    return std::min(p.nr, p.nc) >= min_side ? TVD_TRANSFORM_GEMM : TVD_TRANSFORM_FFT;
}

// ---------------------------------------------------------------- CG driver

template <typename T>
static tvd_status read_state(tvd_plan_s& p, cudaStream_t s) {
    TVD_CUDA_TRY(cudaMemcpyAsync(p.hstate, p.state, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    TVD_CUDA_TRY(cudaStreamSynchronize(s));
    return TVD_OK;
}

// One CG iteration (GV96 Alg. 10.3.1): z = M^-1 r, rho, beta; p = z + beta p
// with t = H p; q = A p, alpha; x += alpha p, r -= alpha q, stopping test.
// With the transform preconditioners the x / r update and the test are
// applied by the next iteration's first row pass (CgState.pending), which
// reads r anyway; with I and D they are a kernel of their own.
template <typename T>
static tvd_status enqueue_iteration(tvd_plan_s& p, Ops<T>& o, double alpha, T* x, CgState* st, cudaStream_t s) {
    const bool fused_xr = (p.pc == TVD_PC_FAST || p.pc == TVD_PC_DFAST || p.pc == TVD_PC_FASTD);
    switch (p.pc) {
        case TVD_PC_NONE: TVD_TRY(cg_simple_precond<T>(p, o.r, nullptr, o.z, st, s)); break;
        case TVD_PC_DIAG: TVD_TRY(cg_simple_precond<T>(p, o.r, o.dinv, o.z, st, s)); break;
        default: TVD_TRY(precond_solve<T>(p, o, o.r, o.z, st, s, x)); break;
    }
    TVD_TRY(blur_pupdate<T>(p, o, o.z, o.p, o.p2, o.t, st, s));
    TVD_TRY(normal_finish<T>(p, o, o.t, o.p, o.p2, alpha, o.q, st, s));
    if (!fused_xr) TVD_TRY(cg_xrupdate<T>(p, x, o.r, o.p, o.p2, o.q, st, s));
    return TVD_OK;
}

constexpr int kChunk = 4;   // CG iterations per graph replay

// Capture kChunk iterations into a CUDA graph for this (x, b, alpha). The
// capture runs on a plan-owned stream; the graph is replayed on the caller's.
// The device-driven loop (a while node around the chunk; TVD_CG_DEVICE_LOOP=0
// at graph capture turns it off): one launch runs chunks until the solver state
// is done, so the host neither polls after each chunk nor launches chunks past
// convergence.
bool device_loop_enabled() {
    const char* v = std::getenv("TVD_CG_DEVICE_LOOP");
    return !(v && v[0] == '0');
}

bool build_while_graph(tvd_plan_s& p, const std::function<tvd_status(cudaStream_t, cudaGraphConditionalHandle)>& body,
                       cudaGraphExec_t* out, int* kernels) {
    *out = nullptr;
    if (!p.cap_stream && cudaStreamCreateWithFlags(&p.cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaGraph_t graph = nullptr;
    cudaGraphConditionalHandle h;
    bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess &&
              cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    cudaGraph_t bg = nullptr;
    if (ok) {
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        ok = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) == cudaSuccess;
        if (ok) bg = np.conditional.phGraph_out[0];
    }
    if (ok) ok = cudaStreamBeginCaptureToGraph(p.cap_stream, bg, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        set_capturing(true);
        const tvd_status st = body(p.cap_stream, h);
        *kernels = captured_kernels();
        set_capturing(false);
        cudaGraph_t captured = nullptr;
        const cudaError_t e = cudaStreamEndCapture(p.cap_stream, &captured);
        ok = st == TVD_OK && e == cudaSuccess;
    }
    if (ok) ok = cudaGraphInstantiate(out, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        *out = nullptr;
        cudaGetLastError();
    }
    return ok;
}

// g.loop: kChunk CG iterations and the condition kernel in a while node.
template <typename T>
static bool build_loop_graph(tvd_plan_s& p, Ops<T>& o, double alpha, T* x, tvd_plan_s::CgGraph& g) {
    return build_while_graph(
        p,
        [&](cudaStream_t q, cudaGraphConditionalHandle h) -> tvd_status {
            for (int c = 0; c < kChunk; ++c) TVD_TRY(enqueue_iteration<T>(p, o, alpha, x, p.state, q));
            return cg_loop_cond(h, p.state, q);
        },
        &g.loop, &g.loop_kernels);
}

template <typename T>
static tvd_status ensure_graph(tvd_plan_s& p, Ops<T>& o, double alpha, const T* b, T* x) {
    auto& g = p.graph[sizeof(T) == 8 ? 1 : 0];
    if (g.exec && g.x == x && g.b == b && g.alpha == alpha) return TVD_OK;
    g.reset();
    if (!p.cap_stream) TVD_CUDA_TRY(cudaStreamCreateWithFlags(&p.cap_stream, cudaStreamNonBlocking));
    TVD_CUDA_TRY(cudaStreamBeginCapture(p.cap_stream, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    tvd_status st = TVD_OK;
    for (int c = 0; c < kChunk && st == TVD_OK; ++c) st = enqueue_iteration<T>(p, o, alpha, x, p.state, p.cap_stream);
    const int kernels = captured_kernels();
    set_capturing(false);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(p.cap_stream, &graph);
    if (st != TVD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    TVD_CUDA_TRY(e);
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    TVD_CUDA_TRY(e);
    g.x = x;
    g.b = b;
    g.alpha = alpha;
    g.kernels = kernels;
    if (device_loop_enabled()) build_loop_graph<T>(p, o, alpha, x, g);
    return TVD_OK;
}

// Run the device-driven loop: arm it with a budget of chunks, launch it once,
// read the state. The budget (enough chunks for maxit iterations from the
// start, plus slack) ends the loop even if the state never reported done.
static tvd_status run_device_loop(tvd_plan_s& p, const tvd_plan_s::CgGraph& g, int maxit, cudaStream_t s) {
    TVD_TRY(cg_loop_arm(p.state, maxit / kChunk + 3, s));
    TVD_CUDA_TRY(cudaGraphLaunch(g.loop, s));
    TVD_CUDA_TRY(cudaMemcpyAsync(p.hstate, p.state, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    TVD_CUDA_TRY(cudaStreamSynchronize(s));
    count_launches(p.hstate->loops * g.loop_kernels);
    return TVD_OK;
}

// PCG on A x = b with A = H^T H + alpha L(o.w); x is updated in place.
// The preconditioner must be set up in `o`. Iterations are enqueued in chunks
// (replays of a captured CUDA graph unless per-kernel profiling is on); the
// kernels of iterations past convergence return at once. The first batch of
// chunks covers the previous solve's iteration count, then the host checks
// the device state after every chunk.
template <typename T>
static tvd_status cg_run(tvd_plan_s& p, Ops<T>& o, double alpha, const T* b, T* x, double tol, int maxit,
                         CgState* out, cudaStream_t s) {
    CgState* st = p.state;
    TVD_TRY(blur_apply<T>(p, o, false, x, o.t, s));
    TVD_TRY(normal_finish<T>(p, o, o.t, x, x, alpha, o.q, nullptr, s));
    TVD_TRY(cg_init<T>(p, b, o.q, o.r, st, tol, maxit, s));
    const bool use_graph = !profiling_enabled();
    if (use_graph) TVD_TRY(ensure_graph<T>(p, o, alpha, b, x));
    auto& g = p.graph[sizeof(T) == 8 ? 1 : 0];
    int& hint = p.last_iters[sizeof(T) == 8 ? 1 : 0];
    int first = std::max(1, (std::min(hint, maxit) - 2) / kChunk);
    int done_iters = 0;
    if (use_graph && g.loop) {
        TVD_TRY(run_device_loop(p, g, maxit, s));
        if (!p.hstate->done) {
            set_error("CG state did not reach done after maxit iterations");
            return TVD_ECUDA;
        }
    }
    while (!(use_graph && g.loop)) {
        for (int c = 0; c < first; ++c) {
            if (use_graph) {
                TVD_CUDA_TRY(cudaGraphLaunch(g.exec, s));
                count_launches(g.kernels);
            } else {
                for (int i = 0; i < kChunk; ++i) TVD_TRY(enqueue_iteration<T>(p, o, alpha, x, st, s));
            }
        }
        done_iters += first * kChunk;
        first = 1;
        TVD_TRY(read_state<T>(p, s));
        if (p.hstate->done) break;
        if (done_iters > maxit + 2 * kChunk) {   // the kernels always advance a running solve
            set_error("CG state did not reach done after maxit iterations");
            return TVD_ECUDA;
        }
    }
    *out = *p.hstate;
    hint = out->iter;
    return TVD_OK;
}

// Preconditioner set-up for the FP step at u_lag (type T).
template <typename T>
static tvd_status setup_precond(tvd_plan_s& p, Ops<T>& o, const T* u_lag, double alpha, double beta,
                                cudaStream_t s) {
    TVD_TRY(diffusivity<T>(p, u_lag, beta, o.w, s));
    TVD_TRY(diag_scale<T>(p, o.w, alpha, o.dmh, o.dinv, s));
    if (p.pc == TVD_PC_FAST || p.pc == TVD_PC_DFAST || p.pc == TVD_PC_FASTD) {
        int* bad = reinterpret_cast<int*>(p.scal + 8);
        TVD_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
        TVD_TRY(spectrum_setup<T>(p, o, alpha, bad, s));
        int hb = 0;
        TVD_CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        TVD_CUDA_TRY(cudaStreamSynchronize(s));
        if (hb) {
            set_error("preconditioner eigenvalue Lambda_H^2 + alpha Lambda_L is not positive");
            return TVD_EINVAL;
        }
    }
    p.precond_ready = true;
    p.alpha = alpha;
    p.beta = beta;
    return TVD_OK;
}

// MIXED-mode preconditioner: diffusivity and scaling from the double iterate,
// cast to float, spectrum in float.
static tvd_status setup_mixed(tvd_plan_s& p, const double* u_lag, double alpha, double beta, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    TVD_TRY(diffusivity<double>(p, u_lag, beta, p.d.w, s));
    TVD_TRY(diag_scale<double>(p, p.d.w, alpha, p.d.dmh, p.d.dinv, s));
    TVD_TRY(cast_d2f(p.d.w, p.f.w, n, s));
    TVD_TRY(cast_d2f(p.d.dmh, p.f.dmh, n, s));
    TVD_TRY(cast_d2f(p.d.dinv, p.f.dinv, n, s));
    if (p.pc == TVD_PC_FAST || p.pc == TVD_PC_DFAST || p.pc == TVD_PC_FASTD) {
        int* bad = reinterpret_cast<int*>(p.scal + 8);
        TVD_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
        TVD_TRY(spectrum_setup<float>(p, p.f, alpha, bad, s));
        int hb = 0;
        TVD_CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        TVD_CUDA_TRY(cudaStreamSynchronize(s));
        if (hb) {
            set_error("preconditioner eigenvalue Lambda_H^2 + alpha Lambda_L is not positive");
            return TVD_EINVAL;
        }
    }
    p.precond_ready = true;
    p.alpha = alpha;
    p.beta = beta;
    return TVD_OK;
}

static tvd_status read_scalars(tvd_plan_s& p, double* h, int count, cudaStream_t s) {
    TVD_CUDA_TRY(cudaMemcpyAsync(h, p.scal, count * sizeof(double), cudaMemcpyDeviceToHost, s));
    TVD_CUDA_TRY(cudaStreamSynchronize(s));
    return TVD_OK;
}

// A tensor-core transform product's bounded wait expired (TVD_ETIMEOUT in the
// CG state): the products after it skipped their work and left the reduction
// tickets mid-count, so those are cleared (and the plan's flag read back)
// before the error is returned; the plan stays usable.
static tvd_status timeout_exit(tvd_plan_s& p, cudaStream_t s) {
    cudaMemsetAsync(p.ticket, 0, 16 * sizeof(unsigned int), s);
    gemm_precond_check(p, s);
    cudaStreamSynchronize(s);
    set_error("a tensor-core transform product gave up waiting for its operands (bounded wait expired); "
              "the solve was stopped");
    return TVD_ETIMEOUT;
}

struct SolveResult {
    int iters = 0;
    int sweeps = 0;
    double relres = 0.0;
    tvd_status status = TVD_OK;
};

// MIXED: float PCG with residual replacement ("reliable updates"). The float
// CG runs on A d = r from d = 0; whenever its recursive residual has fallen by
// a factor 1e-4 since the last replacement, or claims convergence, the host
// folds d into the double iterate x, recomputes the residual b - A x in double
// (H^T H x with the double kernels, cached in p.hx), and the CG resumes from
// that residual with its search direction kept. The stopping test is on the
// double residual: ||b - A x|| / ||b - A x_0|| < tol. With cached_hx, p.hx
// already holds H^T H x for the incoming x (the previous FP step's last check).
static tvd_status solve_mixed(tvd_plan_s& p, double alpha, const double* b, double* x, double tol, int maxit,
                              bool cached_hx, SolveResult* res, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    double h1 = 0.0;
    auto true_residual = [&](bool recompute, double* rr) -> tvd_status {
        if (recompute) {
            TVD_TRY(blur_apply<double>(p, p.d, false, x, p.d.t, s));
            TVD_TRY(blur_apply<double>(p, p.d, true, p.d.t, p.hx, s));
        }
        TVD_TRY(residual_lx(p, b, p.hx, p.d.w, x, alpha, p.res, p.scal, s));
        TVD_TRY(read_scalars(p, &h1, 1, s));
        *rr = h1;
        return TVD_OK;
    };
    p.hx_for = nullptr;
    double rr0 = 0.0;
    TVD_TRY(true_residual(!cached_hx, &rr0));
    p.hx_for = x;
    res->iters = 0;
    res->sweeps = 0;
    res->relres = 0.0;
    res->status = TVD_OK;
    if (!std::isfinite(rr0)) {
        res->status = TVD_EBREAKDOWN;
        return TVD_OK;
    }
    if (rr0 == 0.0) return TVD_OK;
    const double target = tol * tol * rr0;
    // replace once the float residual fell by 1e-4 (TVD_MIXED_DELTA2 overrides, tuning)
    static const double delta2 = []() {
        const char* v = std::getenv("TVD_MIXED_DELTA2");
        const double d = v ? std::atof(v) : 0.0;
        return d > 0.0 && d < 1.0 ? d : 1e-8;
    }();
    double rr_ref = rr0;
    res->relres = 1.0;
    // each float CG segment stops on the device once its residual fell by delta2
    // (or below the target): the replacement point is then an iteration count,
    // independent of how often the host polls
    TVD_TRY(cast_d2f(p.res, p.f.r, n, s));
    TVD_TRY(fill_zero_f(p.f.x, n, s));
    TVD_TRY(cg_restart<float>(p, p.f.r, p.state, std::max(target, delta2 * rr_ref), maxit, 0, s));
    const bool use_graph = !profiling_enabled();
    if (use_graph) TVD_TRY(ensure_graph<float>(p, p.f, alpha, nullptr, p.f.x));
    auto& g = p.graph[0];
    int& hint = p.last_iters[0];
    int batch = std::max(1, (std::min(hint, maxit) - 2) / kChunk);
    int last_iter = -1;
    for (;;) {
        if (use_graph && g.loop) {
            TVD_TRY(run_device_loop(p, g, maxit, s));
        } else {
            for (int c = 0; c < batch; ++c) {
                if (use_graph) {
                    TVD_CUDA_TRY(cudaGraphLaunch(g.exec, s));
                    count_launches(g.kernels);
                } else {
                    for (int i = 0; i < kChunk; ++i)
                        TVD_TRY(enqueue_iteration<float>(p, p.f, alpha, p.f.x, p.state, s));
                }
            }
            batch = 1;
            TVD_TRY(read_state<float>(p, s));
        }
        const CgState h = *p.hstate;
        res->iters = h.iter;
        if (h.status == TVD_ETIMEOUT) return timeout_exit(p, s);
        if (!h.done) {
            if (h.iter == last_iter) {   // the kernels always advance a running solve
                set_error("CG made no progress between two checks");
                return TVD_ECUDA;
            }
            last_iter = h.iter;
            continue;
        }
        last_iter = -1;
        // fold the float correction into x and check the residual in double
        TVD_TRY(axpy_f2d(x, p.f.x, n, s));
        TVD_TRY(fill_zero_f(p.f.x, n, s));
        double rr = 0.0;
        TVD_TRY(true_residual(true, &rr));
        res->sweeps += 1;
        if (!std::isfinite(rr) || h.status == TVD_EBREAKDOWN) {
            res->status = TVD_EBREAKDOWN;
            break;
        }
        res->relres = std::sqrt(rr / rr0);
        if (rr < target) break;
        if (h.iter >= maxit || res->sweeps > 200) {
            res->status = TVD_ENOCONV;
            break;
        }
        // keep the search direction only while the float recursion still tracks
        // the true residual; a larger gap (float operator error) restarts it
        const int mode = (rr < 4.0 * h.rr) ? 1 : 2;
        rr_ref = rr;
        TVD_TRY(cast_d2f(p.res, p.f.r, n, s));
        TVD_TRY(cg_restart<float>(p, p.f.r, p.state, std::max(target, delta2 * rr_ref), maxit, mode, s));
    }
    hint = res->iters;
    return gemm_precond_check(p, s);
}

static tvd_status solve(tvd_plan_s& p, const double* u_lag, double alpha, double beta, const double* b, double* x,
                        double tol, int maxit, SolveResult* res, cudaStream_t s, bool cached_hx = false) {
    if (p.reblur()) {
        // eq. (fpp): the preconditioner of the reblurring method, then PBiCGstab
        if (p.mode == TVD_MODE_FP64) TVD_TRY(setup_precond<double>(p, p.d, u_lag, alpha, beta, s));
        else TVD_TRY(setup_mixed(p, u_lag, alpha, beta, s));
        TVD_TRY(reblur_solve(p, alpha, b, x, tol, maxit, &res->iters, &res->sweeps, &res->relres, &res->status, s));
        return p.mode == TVD_MODE_MIXED ? gemm_precond_check(p, s) : TVD_OK;
    }
    if (p.mode == TVD_MODE_FP64) {
        TVD_TRY(setup_precond<double>(p, p.d, u_lag, alpha, beta, s));
        CgState cs;
        TVD_TRY(cg_run<double>(p, p.d, alpha, b, x, tol, maxit, &cs, s));
        res->iters = cs.iter;
        res->sweeps = 1;
        res->relres = cs.rr0 > 0.0 ? std::sqrt(cs.rr / cs.rr0) : 0.0;
        res->status = (tvd_status)cs.status;
        return TVD_OK;
    }
    TVD_TRY(setup_mixed(p, u_lag, alpha, beta, s));
    return solve_mixed(p, alpha, b, x, tol, maxit, cached_hx && p.hx_for == x, res, s);
}

}  // namespace tvd

using namespace tvd;

// ---------------------------------------------------------------- C ABI

extern "C" {

const char* tvd_last_error(void) { return g_err.c_str(); }

tvd_status tvd_plan_set_transform(tvd_plan plan, int kind, void* stream) {
    if (!plan || (kind != TVD_TRANSFORM_FFT && kind != TVD_TRANSFORM_GEMM)) {
        set_error("tvd_plan_set_transform: NULL plan or unknown transform kind");
        return TVD_EINVAL;
    }
    if (kind == TVD_TRANSFORM_GEMM && (plan->mode != TVD_MODE_MIXED || !fast_pc(plan->pc) || plan->nr == 1)) {
        set_error("tvd_plan_set_transform: the GEMM form needs a MIXED 2D plan with a fast preconditioner");
        return TVD_EINVAL;
    }
    if ((kind == TVD_TRANSFORM_GEMM) == (plan->gemm != nullptr)) return TVD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("stream synchronisation failed");
        return TVD_ECUDA;
    }
    // the captured float CG iterations hold the previous form's launches
    reset_graphs(*plan);
    if (kind == TVD_TRANSFORM_FFT) {
        cudaDeviceSynchronize();
        gemm_precond_destroy(*plan);
        return TVD_OK;
    }
    return gemm_precond_create(*plan, s);
}

int tvd_plan_transform(tvd_plan plan) { return plan && plan->gemm ? TVD_TRANSFORM_GEMM : TVD_TRANSFORM_FFT; }

int tvd_plan_gemm_storage(tvd_plan plan) { return plan ? gemm_precond_storage(*plan) : 0; }

int tvd_plan_gemm_folded(tvd_plan plan) { return plan ? gemm_precond_folded(*plan) : 0; }

int tvd_plan_gemm_tile(tvd_plan plan) { return plan ? gemm_precond_tile(*plan) : 0; }

}  // extern "C"

namespace tvd {

// Put the plan in one preconditioner form: FFT, or the products with tile width
// bn (64 / 128) and the folded products on or off.
static tvd_status tune_apply(tvd_plan_s& p, int transform, int bn, int fold, cudaStream_t s) {
    TVD_CUDA_TRY(cudaStreamSynchronize(s));
    reset_graphs(p);
    TVD_CUDA_TRY(cudaDeviceSynchronize());
    gemm_precond_destroy(p);
    p.gemm_bn = bn;
    p.gemm_fold = fold;
    return transform == TVD_TRANSFORM_GEMM ? gemm_precond_create(p, s) : TVD_OK;
}

// Average time of one preconditioner solve r -> z in the plan's current form:
// TVD_TUNE_SOLVES solves per graph replay, the fastest of `reps` replays after
// one warm-up.
static tvd_status tune_time(tvd_plan_s& p, const float* r, float* z, int reps, double* us, cudaStream_t s) {
    const bool use_graph = !profiling_enabled();
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
    if (use_graph) {
        if (!p.cap_stream) TVD_CUDA_TRY(cudaStreamCreateWithFlags(&p.cap_stream, cudaStreamNonBlocking));
        TVD_CUDA_TRY(cudaStreamBeginCapture(p.cap_stream, cudaStreamCaptureModeThreadLocal));
        set_capturing(true);
        tvd_status st = TVD_OK;
        for (int k = 0; k < TVD_TUNE_SOLVES && st == TVD_OK; ++k)
            st = precond_solve<float>(p, p.f, r, z, nullptr, p.cap_stream);
        kernels = captured_kernels();
        set_capturing(false);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(p.cap_stream, &graph);
        if (st != TVD_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        TVD_CUDA_TRY(e);
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        TVD_CUDA_TRY(ei);
    }
    auto run = [&]() -> tvd_status {
        if (use_graph) {
            TVD_CUDA_TRY(cudaGraphLaunch(exec, s));
            count_launches(kernels);
            return TVD_OK;
        }
        for (int k = 0; k < TVD_TUNE_SOLVES; ++k) TVD_TRY(precond_solve<float>(p, p.f, r, z, nullptr, s));
        return TVD_OK;
    };
    cudaEvent_t ev[2] = {nullptr, nullptr};
    tvd_status st = TVD_OK;
    double best = 1e300;
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
        set_error("cudaEventCreate failed");
        st = TVD_ECUDA;
    }
    for (int k = 0; k <= reps && st == TVD_OK; ++k) {   // k = 0: warm-up
        if (cudaEventRecord(ev[0], s) != cudaSuccess) st = TVD_ECUDA;
        if (st == TVD_OK) st = run();
        if (st == TVD_OK && (cudaEventRecord(ev[1], s) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess))
            st = TVD_ECUDA;
        float ms = 0.0f;
        if (st == TVD_OK && cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) st = TVD_ECUDA;
        if (st == TVD_OK && k > 0) best = std::min(best, 1e3 * (double)ms / TVD_TUNE_SOLVES);
    }
    if (st == TVD_ECUDA) set_error("timing a preconditioner form failed");
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    if (exec) cudaGraphExecDestroy(exec);
    if (st == TVD_OK && p.gemm) st = gemm_precond_check(p, s);
    *us = best;
    return st;
}

}  // namespace tvd

extern "C" {

tvd_status tvd_plan_tune(tvd_plan plan, int reps, tvd_tune_report* report, void* stream) {
    if (!plan || reps < 0) {
        set_error("tvd_plan_tune: NULL plan or reps < 0");
        return TVD_EINVAL;
    }
    if (plan->mode != TVD_MODE_MIXED || !fast_pc(plan->pc) || plan->nr == 1) {
        set_error("tvd_plan_tune: only MIXED 2D plans with a fast preconditioner have forms to choose from");
        return TVD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (reps == 0) reps = 3;
    tvd_tune_report rep{};
    // {transform, tile width, fold}; the FFT form leaves the product rules at their defaults
    const int cand[TVD_TUNE_MAX][3] = {{TVD_TRANSFORM_FFT, 0, -1},
                                       {TVD_TRANSFORM_GEMM, 64, 0},
                                       {TVD_TRANSFORM_GEMM, 128, 0},
                                       {TVD_TRANSFORM_GEMM, 64, 1}};
    const int count = gemm_fold_allowed(*plan) ? 4 : 3;
    const size_t n = (size_t)plan->nr * plan->nc;
    // scratch: u_lag = 0 (double), a seeded residual r in [-1, 1) and z (float)
    double* u0 = nullptr;
    float *r = nullptr, *z = nullptr;
    tvd_status st = dalloc(&u0, n);
    if (st == TVD_OK) st = dalloc(&r, n);
    if (st == TVD_OK) st = dalloc(&z, n);
    if (st == TVD_OK) {
        std::vector<float> hr(n);
        unsigned long long x = 0x9E3779B97F4A7C15ull;   // splitmix64 stream
        for (size_t i = 0; i < n; ++i) {
            x += 0x9E3779B97F4A7C15ull;
            unsigned long long y = x;
            y = (y ^ (y >> 30)) * 0xBF58476D1CE4E5B9ull;
            y = (y ^ (y >> 27)) * 0x94D049BB133111EBull;
            y ^= y >> 31;
            hr[i] = (float)((double)(y >> 11) * 0x1.0p-52 - 1.0);
        }
        if (cudaMemsetAsync(u0, 0, n * sizeof(double), s) != cudaSuccess ||
            cudaMemcpyAsync(r, hr.data(), n * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            set_error("tvd_plan_tune: scratch set-up failed");
            st = TVD_ECUDA;
        }
    }
    for (int k = 0; k < count && st == TVD_OK; ++k) {
        st = tune_apply(*plan, cand[k][0], cand[k][1], cand[k][2], s);
        if (st == TVD_OK) st = setup_mixed(*plan, u0, 1e-3, 1e-2, s);
        double us = 0.0;
        if (st == TVD_OK) st = tune_time(*plan, r, z, reps, &us, s);
        rep.transform[k] = cand[k][0];
        rep.tile_n[k] = cand[k][1];
        rep.folded[k] = cand[k][2] == 1 ? 1 : 0;
        rep.us_per_solve[k] = us;
        rep.count = k + 1;
        if (st == TVD_OK && us < rep.us_per_solve[rep.chosen]) rep.chosen = k;
    }
    if (st == TVD_OK) {
        const int c = rep.chosen;
        st = tune_apply(*plan, cand[c][0], cand[c][1], cand[c][2], s);
    }
    plan->precond_ready = false;
    cudaStreamSynchronize(s);
    dfree(u0);
    dfree(r);
    dfree(z);
    if (report) *report = rep;
    return st;
}

const char* tvd_version(void) { return "tvd-gb300 0.1"; }

tvd_status tvd_plan_create(tvd_plan* out, int n_rows, int n_cols, const double* psf_host, int p_rows, int p_cols,
                           tvd_bc bc, tvd_precond pc, tvd_mode mode, void* stream) {
    g_err.clear();
    if (!out) {
        set_error("out is NULL");
        return TVD_EINVAL;
    }
    *out = nullptr;
    // line transforms keep two lines (float: up to 4096) or one line pair in shared memory;
    // n_rows = 1 is a 1D signal of n_cols samples (Sec. 5.1)
    const int max_side = (mode == TVD_MODE_FP64) ? 2048 : 4096;
    if ((n_rows < 3 && n_rows != 1) || n_cols < 3 || n_rows > max_side || n_cols > max_side) {
        set_error("image sides must be in [3, 2048] (FP64 plans) or [3, 4096] (MIXED plans); n_rows may be 1 "
                  "(a 1D signal)");
        return TVD_EINVAL;
    }
    if ((bc != TVD_BC_REFLECTIVE && bc != TVD_BC_ANTIREFLECTIVE) || pc < TVD_PC_NONE || pc > TVD_PC_FASTD ||
        (mode != TVD_MODE_FP64 && mode != TVD_MODE_MIXED)) {
        set_error("invalid bc / preconditioner / mode");
        return TVD_EINVAL;
    }
    tvd_plan_s* p = new tvd_plan_s();
    p->nr = n_rows;
    p->nc = n_cols;
    p->bc = bc;
    p->pc = pc;
    p->mode = mode;
    cudaStream_t s = (cudaStream_t)stream;
    tvd_status st = build_psf(p->psf, psf_host, p_rows, p_cols, n_rows, n_cols);
    if (st != TVD_OK) {
        delete p;
        return st;
    }
    const int Lr = bc == TVD_BC_ANTIREFLECTIVE ? n_rows - 1 : n_rows;
    const int Lc = bc == TVD_BC_ANTIREFLECTIVE ? n_cols - 1 : n_cols;
    // one row: the column passes are elementwise (the 1-point transform is the identity)
    if (n_rows > 1) p->fft_r = make_fft_plan(Lr);
    p->fft_c = make_fft_plan(Lc);
    const size_t n = (size_t)n_rows * n_cols;
    auto fail = [&](tvd_status e) {
        plan_free(p);
        delete p;
        return e;
    };
    if ((st = dalloc(&p->state, 1)) != TVD_OK) return fail(st);
    if ((st = dalloc(&p->red, kMaxRedBlocks)) != TVD_OK) return fail(st);
    if ((st = dalloc(&p->ticket, 16)) != TVD_OK) return fail(st);
    if ((st = dalloc(&p->scal, 16)) != TVD_OK) return fail(st);
    if ((st = dalloc(&p->hx, n)) != TVD_OK) return fail(st);
    if ((st = dalloc(&p->res, n)) != TVD_OK) return fail(st);
    if ((st = dalloc(&p->xd, n)) != TVD_OK) return fail(st);
    if ((st = dalloc(&p->tmp, n)) != TVD_OK) return fail(st);
    if (cudaMallocHost((void**)&p->hstate, sizeof(CgState)) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMallocHost failed");
        return fail(TVD_ENOMEM);
    }
    if (cudaMemsetAsync(p->ticket, 0, 16 * sizeof(unsigned int), s) != cudaSuccess ||
        cudaMemsetAsync(p->state, 0, sizeof(CgState), s) != cudaSuccess) {
        set_error("cudaMemset failed");
        return fail(TVD_ECUDA);
    }
    if ((st = ops_alloc<double>(*p, p->d, s)) != TVD_OK) return fail(st);
    if (mode == TVD_MODE_MIXED && (st = ops_alloc<float>(*p, p->f, s)) != TVD_OK) return fail(st);
    if (mode == TVD_MODE_MIXED && default_transform(*p) == TVD_TRANSFORM_GEMM &&
        (st = gemm_precond_create(*p, s)) != TVD_OK)
        return fail(st);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("stream synchronisation failed");
        return fail(TVD_ECUDA);
    }
    *out = p;
    return TVD_OK;
}

tvd_status tvd_plan_destroy(tvd_plan plan) {
    if (!plan) return TVD_OK;
    cudaDeviceSynchronize();
    plan_free(plan);
    delete plan;
    return TVD_OK;
}

tvd_status ar_blur_apply(tvd_plan plan, int transpose, const void* x, void* y, void* stream) {
    if (!plan || !x || !y || x == y) {
        set_error("ar_blur_apply: NULL plan / pointer, or x == y");
        return TVD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->mode == TVD_MODE_FP64)
        return blur_apply<double>(*plan, plan->d, transpose != 0, (const double*)x, (double*)y, s);
    return blur_apply<float>(*plan, plan->f, transpose != 0, (const float*)x, (float*)y, s);
}

tvd_status tv_operator_apply(tvd_plan plan, const void* u_lag, double beta, const void* x, void* y, void* stream) {
    if (!plan || !u_lag || !x || !y || y == x || y == u_lag || !(beta > 0.0)) {
        set_error("tv_operator_apply: invalid argument");
        return TVD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->mode == TVD_MODE_FP64) {
        TVD_TRY(diffusivity<double>(*plan, (const double*)u_lag, beta, plan->d.t2, s));
        return tv_apply<double>(*plan, plan->d.t2, (const double*)x, (double*)y, s);
    }
    TVD_TRY(diffusivity<float>(*plan, (const float*)u_lag, beta, plan->f.t2, s));
    return tv_apply<float>(*plan, plan->f.t2, (const float*)x, (float*)y, s);
}

tvd_status tv_hessian_apply(tvd_plan plan, const void* u, double beta, const void* x, void* y, void* stream) {
    if (!plan || !u || !x || !y || y == x || y == u || !(beta > 0.0)) {
        set_error("tv_hessian_apply: invalid argument");
        return TVD_EINVAL;
    }
    tvd_plan_s& p = *plan;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)p.nr * p.nc;
    double* g = nullptr;
    TVD_TRY(dalloc(&g, 2 * n));
    tvd_status st = diffusivity<double>(p, (const double*)u, beta, p.d.t2, s);
    if (st == TVD_OK) st = hess_coef(p, (const double*)u, p.d.t2, g, g + n, s);
    if (st == TVD_OK) st = hess_apply(p, (const double*)x, (double*)y, p.d.t2, g, g + n, s);
    if (st == TVD_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("tv_hessian_apply: CUDA error");
        st = TVD_ECUDA;
    }
    dfree(g);
    return st;
}

}  // extern "C"

// MIXED adjoint solve J lambda = b, J = H^T H + alpha nabla^2 J_beta(u*), lambda from 0 (double):
// float CG segments with the plan's float preconditioner, each stopping on the device once its
// recursive residual fell by 1e-4 (or below the target); the float correction is folded into
// lambda and the residual recomputed in double, which decides convergence (as solve_mixed does
// for the FP step). gr, gc: double Hessian coefficients; grf, gcf: their float copies.
static tvd_status adjoint_mixed(tvd_plan_s& p, const double* b, double* lam, const double* gr, const double* gc,
                                const float* grf, const float* gcf, double alpha, double tol, int maxit,
                                int* iters_out, double* relres_out, cudaStream_t s) {
    const size_t n = (size_t)p.nr * p.nc;
    Ops<float>& f = p.f;
    CgState* st = p.state;
    TVD_CUDA_TRY(cudaMemsetAsync(lam, 0, n * sizeof(double), s));
    TVD_TRY(norm2_d(p, b, p.scal + 10, s));
    double rr0 = 0.0;
    TVD_CUDA_TRY(cudaMemcpyAsync(&rr0, p.scal + 10, sizeof(double), cudaMemcpyDeviceToHost, s));
    TVD_CUDA_TRY(cudaStreamSynchronize(s));
    *iters_out = 0;
    *relres_out = 0.0;
    if (!std::isfinite(rr0)) {
        set_error("Jacobian solve: non-finite right-hand side");
        return TVD_EBREAKDOWN;
    }
    if (rr0 == 0.0) return TVD_OK;
    const double target = tol * tol * rr0, delta2 = 1e-8;
    const bool transform_pc = (p.pc == TVD_PC_FAST || p.pc == TVD_PC_DFAST || p.pc == TVD_PC_FASTD);
    double rr_ref = rr0;
    int sweeps = 0, last_iter = -1, stalled = 0;
    // The float CG runs on the residual times sc, a power of two that brings its norm
    // to [1, 2) (exact in float): a tiny right-hand side, as in the last Newton steps,
    // would otherwise reach the float denormal range, where products flush to zero.
    // sc is renewed (with a fresh search direction) once the scaled residual fell below 2^-40.
    auto pow2_scale = [](double rr) { return std::ldexp(1.0, -std::ilogb(std::sqrt(rr))); };
    double sc = pow2_scale(rr0);
    TVD_TRY(cast_d2f(b, f.r, n, s, sc));
    TVD_TRY(fill_zero_f(f.x, n, s));
    TVD_TRY(cg_restart<float>(p, f.r, st, std::max(target, delta2 * rr_ref) * sc * sc, maxit, 0, s));
    // one chunk: 2 kChunk iterations of the Jacobian CG on stream q
    auto chunk = [&](cudaStream_t q) -> tvd_status {
        for (int k = 0; k < 2 * kChunk; ++k) {
            switch (p.pc) {
                case TVD_PC_NONE: TVD_TRY(cg_simple_precond<float>(p, f.r, nullptr, f.z, st, q)); break;
                case TVD_PC_DIAG: TVD_TRY(cg_simple_precond<float>(p, f.r, f.dinv, f.z, st, q)); break;
                default: TVD_TRY(precond_solve<float>(p, f, f.r, f.z, st, q, f.x)); break;
            }
            TVD_TRY(blur_pupdate<float>(p, f, f.z, f.p, f.p2, f.t, st, q));
            TVD_TRY(blur_apply<float>(p, f, true, f.t, f.q, q, st));
            TVD_TRY(hess_add<float>(p, f.q, f.p, f.p2, f.w, grf, gcf, alpha, st, q));
            if (!transform_pc) TVD_TRY(cg_xrupdate<float>(p, f.x, f.r, f.p, f.p2, f.q, st, q));
        }
        return TVD_OK;
    };
    // the device-driven loop, as for the FP step's CG: the chunk in a while node, built for
    // this solve (its operands grf, gcf and alpha belong to the call) and released on return
    struct LoopGraph {
        cudaGraphExec_t exec = nullptr;
        int kernels = 0;
        ~LoopGraph() {
            if (exec) cudaGraphExecDestroy(exec);
        }
    } loop;
    if (!profiling_enabled() && device_loop_enabled())
        build_while_graph(
            p,
            [&](cudaStream_t q, cudaGraphConditionalHandle hc) -> tvd_status {
                TVD_TRY(chunk(q));
                return cg_loop_cond(hc, st, q);
            },
            &loop.exec, &loop.kernels);
    for (;;) {
        if (loop.exec) {
            TVD_TRY(cg_loop_arm(st, maxit / (2 * kChunk) + 3, s));
            TVD_CUDA_TRY(cudaGraphLaunch(loop.exec, s));
            TVD_TRY(read_state<float>(p, s));
            count_launches(p.hstate->loops * loop.kernels);
        } else {
            TVD_TRY(chunk(s));
            TVD_TRY(read_state<float>(p, s));
        }
        const CgState h = *p.hstate;
        *iters_out = h.iter;
        if (h.status == TVD_ETIMEOUT) return timeout_exit(p, s);
        if (!h.done) {
            if (h.iter == last_iter) {   // the kernels always advance a running solve
                set_error("Jacobian CG made no progress between two checks");
                return TVD_ECUDA;
            }
            last_iter = h.iter;
            continue;
        }
        last_iter = -1;
        TVD_TRY(axpy_f2d(lam, f.x, n, s, 1.0 / sc));
        TVD_TRY(fill_zero_f(f.x, n, s));
        TVD_TRY(blur_apply<double>(p, p.d, false, lam, p.d.t, s));
        TVD_TRY(blur_apply<double>(p, p.d, true, p.d.t, p.d.q, s));
        TVD_TRY(adj_residual(p, b, p.d.q, p.d.w, gr, gc, lam, alpha, p.res, p.scal + 10, s));
        double rr = 0.0;
        TVD_CUDA_TRY(cudaMemcpyAsync(&rr, p.scal + 10, sizeof(double), cudaMemcpyDeviceToHost, s));
        TVD_CUDA_TRY(cudaStreamSynchronize(s));
        ++sweeps;
        if (!std::isfinite(rr) || h.status == TVD_EBREAKDOWN) {
            set_error("Jacobian solve: the CG broke down");
            return TVD_EBREAKDOWN;
        }
        *relres_out = std::sqrt(rr / rr0);
        if (rr < target) return gemm_precond_check(p, s);
        // each float sweep lowers the residual by about 1e4; three sweeps in a row that
        // do not halve the double residual mean it sits at its rounding floor
        stalled = rr > 0.25 * rr_ref ? stalled + 1 : 0;
        if (h.iter >= maxit || sweeps > 200 || stalled >= 3) {
            set_error(stalled >= 3 ? "Jacobian solve: the double residual stagnated above the tolerance"
                                   : "Jacobian solve: the CG did not reach its tolerance");
            return TVD_ENOCONV;
        }
        int mode = (rr * sc * sc < 4.0 * h.rr) ? 1 : 2;
        if (rr * sc * sc < 0x1p-80) {
            sc = pow2_scale(rr);
            mode = 2;
        }
        rr_ref = rr;
        TVD_TRY(cast_d2f(p.res, f.r, n, s, sc));
        TVD_TRY(cg_restart<float>(p, f.r, st, std::max(target, delta2 * rr_ref) * sc * sc, maxit, mode, s));
    }
}

// lam = J(u)^-1 b from lam = 0, J = H^T H + alpha nabla^2 J_beta(u) (SPD), by PCG
// preconditioned with the plan's preconditioner of the lagged operator at u,
// which the caller has set up (setup_precond / setup_mixed at u: o.w holds
// w(u)), with the Hessian coefficients gr, gc of hess_coef at u (and their
// float copies grf, gcf on MIXED plans). FP64 plans run one double PCG; MIXED
// plans the float PCG with double residual replacement of adjoint_mixed.
// Returns TVD_OK, TVD_ENOCONV (lam holds the last iterate), TVD_EBREAKDOWN,
// TVD_ETIMEOUT or a CUDA error, with *iters and *relres.
static tvd_status jacobian_solve(tvd_plan_s& p, const double* b, double* lam, const double* gr, const double* gc,
                                 const float* grf, const float* gcf, double alpha, double tol, int maxit, int* iters,
                                 double* relres, cudaStream_t s) {
    *iters = 0;
    *relres = 0.0;
    if (p.mode == TVD_MODE_MIXED) return adjoint_mixed(p, b, lam, gr, gc, grf, gcf, alpha, tol, maxit, iters, relres, s);
    const size_t n = (size_t)p.nr * p.nc;
    Ops<double>& o = p.d;
    TVD_CUDA_TRY(cudaMemsetAsync(lam, 0, n * sizeof(double), s));
    TVD_CUDA_TRY(cudaMemsetAsync(o.q, 0, n * sizeof(double), s));
    CgState* st = p.state;
    TVD_TRY(cg_init<double>(p, b, o.q, o.r, st, tol, maxit, s));
    const bool fused_xr = (p.pc == TVD_PC_FAST || p.pc == TVD_PC_DFAST || p.pc == TVD_PC_FASTD);
    int done_iters = 0;
    for (;;) {
        for (int k = 0; k < 2 * kChunk; ++k) {
            switch (p.pc) {
                case TVD_PC_NONE: TVD_TRY(cg_simple_precond<double>(p, o.r, nullptr, o.z, st, s)); break;
                case TVD_PC_DIAG: TVD_TRY(cg_simple_precond<double>(p, o.r, o.dinv, o.z, st, s)); break;
                default: TVD_TRY(precond_solve<double>(p, o, o.r, o.z, st, s, lam)); break;
            }
            TVD_TRY(blur_pupdate<double>(p, o, o.z, o.p, o.p2, o.t, st, s));
            TVD_TRY(blur_apply<double>(p, o, true, o.t, o.q, s, st));
            TVD_TRY(hess_add(p, o.q, o.p, o.p2, o.w, gr, gc, alpha, st, s));
            if (!fused_xr) TVD_TRY(cg_xrupdate<double>(p, lam, o.r, o.p, o.p2, o.q, st, s));
        }
        done_iters += 2 * kChunk;
        TVD_TRY(read_state<double>(p, s));
        if (p.hstate->done) break;
        if (done_iters > maxit + 4 * kChunk) {
            set_error("Jacobian CG state did not reach done after maxit iterations");
            return TVD_ECUDA;
        }
    }
    const CgState h = *p.hstate;
    *iters = h.iter;
    *relres = h.rr0 > 0.0 ? std::sqrt(h.rr / h.rr0) : 0.0;
    if (h.status == TVD_EBREAKDOWN) {
        set_error("Jacobian solve: the CG broke down");
        return TVD_EBREAKDOWN;
    }
    if (h.status == TVD_ENOCONV) {
        set_error("Jacobian solve: the CG did not reach its tolerance");
        return TVD_ENOCONV;
    }
    return TVD_OK;
}

// g(x) = H^T (H x - v) + alpha L(x) x of eq. (el), returned as r = -g(x) = b - H^T H x - alpha L(w(x)) x
// with b = H^T v (double, any mode), and ||g||^2 on the host. w(x) goes to p.d.w, H x to p.d.t,
// H^T H x to p.hx (for x, recorded in p.hx_for). On a reblurring plan, with b = H' v, the same call
// gives the residual of eq. (fpp), b - H' H x - alpha L(w(x)) x (H' = H for the plans' PSFs).
// With data_out non-NULL, also ||H x - v||^2 and sum psi(x) (the two terms of the functional).
static tvd_status el_residual(tvd_plan_s& p, const double* x, const double* v, const double* b, double alpha,
                              double beta, double* r, double* g2, double* data_out, cudaStream_t s) {
    TVD_TRY(diffusivity<double>(p, x, beta, p.d.w, s));
    TVD_TRY(blur_apply<double>(p, p.d, false, x, p.d.t, s));
    if (data_out) {
        TVD_TRY(diffnorm2_d(p, p.d.t, v, p.scal + 13, s));
        TVD_TRY(tv_sum_d(p, x, beta, p.scal + 14, s));
    }
    TVD_TRY(blur_apply<double>(p, p.d, !p.reblur(), p.d.t, p.hx, s));
    TVD_TRY(residual_lx(p, b, p.hx, p.d.w, x, alpha, r, p.scal + 12, s));
    p.hx_for = x;
    double h3[3] = {0.0, 0.0, 0.0};
    TVD_CUDA_TRY(cudaMemcpyAsync(h3, p.scal + 12, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    TVD_CUDA_TRY(cudaStreamSynchronize(s));
    *g2 = h3[0];
    if (data_out) {
        data_out[0] = h3[1];
        data_out[1] = h3[2];
    }
    return TVD_OK;
}

extern "C" {

tvd_status tv_deblur_adjoint(tvd_plan plan, const void* u_star, const void* v, double alpha, double beta,
                             const void* dl_du, void* lambda_out, double tol, int maxit, double* dl_dalpha,
                             double* dl_dbeta, double* dl_dpsf, int* iters, double* relres, void* stream) {
    if (!plan || !u_star || !v || !dl_du || !lambda_out || lambda_out == dl_du || lambda_out == u_star ||
        lambda_out == v || !(alpha >= 0.0) || !(beta > 0.0) || !(tol > 0.0) || maxit < 0) {
        set_error("tv_deblur_adjoint: invalid argument");
        return TVD_EINVAL;
    }
    if (plan->reblur()) {
        set_error("tv_deblur_adjoint: differentiates the fixed point of eq. (fp); a reblurring plan's "
                  "linearisation is not symmetric");
        return TVD_EINVAL;
    }
    tvd_plan_s& p = *plan;
    Ops<double>& o = p.d;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)p.nr * p.nc;
    const int mr = p.psf.mr, mc = p.psf.mc;
    const size_t ne = (size_t)(p.nr + 2 * mr) * (p.nc + 2 * mc);
    const size_t ntap = (size_t)(2 * mr + 1) * (2 * mc + 1);
    const double* u = (const double*)u_star;
    double* lam = (double*)lambda_out;
    p.hx_for = nullptr;
    // the lagged operator's preconditioner at u* (w = psi^-1 of u*, D, the spectrum): in
    // double for FP64 plans, in float (from the double coefficients) for MIXED plans
    const bool mixed = p.mode == TVD_MODE_MIXED;
    if (mixed) TVD_TRY(setup_mixed(p, u, alpha, beta, s));
    else TVD_TRY(setup_precond<double>(p, o, u, alpha, beta, s));
    double* scratch = nullptr;
    TVD_TRY(dalloc(&scratch, 2 * n + 2 * ne + ntap + 2 + (mixed ? n : 0)));
    double *gr = scratch, *gc = scratch + n, *ext = scratch + 2 * n, *taps = ext + 2 * ne, *out2 = taps + ntap;
    float* gf = mixed ? reinterpret_cast<float*>(out2 + 2) : nullptr;   // float g_r, g_c (n each)
    auto run = [&]() -> tvd_status {
        TVD_TRY(hess_coef(p, u, o.w, gr, gc, s));
        if (mixed) {
            TVD_TRY(cast_d2f(gr, gf, n, s));
            TVD_TRY(cast_d2f(gc, gf + n, n, s));
        }
        int it = 0;
        double rel = 0.0;
        const tvd_status cg = jacobian_solve(p, (const double*)dl_du, lam, gr, gc, gf, mixed ? gf + n : nullptr, alpha,
                                             tol, maxit, &it, &rel, s);
        if (iters) *iters = it;
        if (relres) *relres = rel;
        if (cg != TVD_OK && cg != TVD_ENOCONV) return cg;   // gradients still written after ENOCONV
        TVD_TRY(adjoint_gradients(p, o, lam, u, (const double*)v, alpha, beta, ext, dl_dpsf ? taps : nullptr, out2,
                                  s));
        double h2[2] = {0.0, 0.0};
        TVD_CUDA_TRY(cudaMemcpyAsync(h2, out2, sizeof(h2), cudaMemcpyDeviceToHost, s));
        if (dl_dpsf) TVD_CUDA_TRY(cudaMemcpyAsync(dl_dpsf, taps, ntap * sizeof(double), cudaMemcpyDeviceToHost, s));
        TVD_CUDA_TRY(cudaStreamSynchronize(s));
        if (dl_dalpha) *dl_dalpha = -h2[0];
        if (dl_dbeta) *dl_dbeta = alpha * beta * h2[1];
        if (cg == TVD_ENOCONV) set_error("tv_deblur_adjoint: the adjoint CG did not reach its tolerance");
        return cg;
    };
    const tvd_status st = run();
    cudaStreamSynchronize(s);
    dfree(scratch);
    return st;
}

tvd_status tvd_plan_psf_size(tvd_plan plan, int* p_rows, int* p_cols) {
    if (!plan || !p_rows || !p_cols) {
        set_error("tvd_plan_psf_size: invalid argument");
        return TVD_EINVAL;
    }
    *p_rows = 2 * plan->psf.mr + 1;
    *p_cols = 2 * plan->psf.mc + 1;
    return TVD_OK;
}

tvd_status tau_precond_setup(tvd_plan plan, const void* u_lag, double alpha, double beta, void* stream) {
    if (!plan || !u_lag || !(alpha >= 0.0) || !(beta > 0.0)) {
        set_error("tau_precond_setup: invalid argument");
        return TVD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    plan->precond_ready = false;
    if (plan->mode == TVD_MODE_FP64) return setup_precond<double>(*plan, plan->d, (const double*)u_lag, alpha, beta, s);
    return setup_precond<float>(*plan, plan->f, (const float*)u_lag, alpha, beta, s);
}

tvd_status tau_precond_solve(tvd_plan plan, const void* r, void* z, void* stream) {
    if (!plan || !r || !z) {
        set_error("tau_precond_solve: invalid argument");
        return TVD_EINVAL;
    }
    if (!plan->precond_ready) {
        set_error("tau_precond_solve: call tau_precond_setup first");
        return TVD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->mode == TVD_MODE_FP64) {
        auto& o = plan->d;
        if (plan->pc == TVD_PC_NONE || plan->pc == TVD_PC_DIAG)
            return cg_simple_precond<double>(*plan, (const double*)r, plan->pc == TVD_PC_DIAG ? o.dinv : nullptr,
                                             (double*)z, nullptr, s);
        return precond_solve<double>(*plan, o, (const double*)r, (double*)z, nullptr, s);
    }
    auto& o = plan->f;
    if (plan->pc == TVD_PC_NONE || plan->pc == TVD_PC_DIAG)
        return cg_simple_precond<float>(*plan, (const float*)r, plan->pc == TVD_PC_DIAG ? o.dinv : nullptr,
                                        (float*)z, nullptr, s);
    return precond_solve<float>(*plan, o, (const float*)r, (float*)z, nullptr, s);
}

tvd_status tvd_plan_set_method(tvd_plan plan, int method, void* stream) {
    if (!plan || (method != TVD_METHOD_FP && method != TVD_METHOD_REBLUR && method != TVD_METHOD_REBLUR_ARL)) {
        set_error("tvd_plan_set_method: invalid argument");
        return TVD_EINVAL;
    }
    if (method != TVD_METHOD_FP && plan->bc != TVD_BC_ANTIREFLECTIVE) {
        set_error("tvd_plan_set_method: the reblurring method needs anti-reflective BCs (Sec. 3)");
        return TVD_EINVAL;
    }
    if (plan->method == method) return TVD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    TVD_CUDA_TRY(cudaStreamSynchronize(s));
    if (method != TVD_METHOD_FP) TVD_TRY(reblur_tables(*plan, s));
    const bool same_transforms = (method != TVD_METHOD_FP) == plan->reblur();
    plan->method = method;
    plan->precond_ready = false;
    reset_graphs(*plan);   // captured chunks hold the previous method's operator
    if (plan->gemm && !same_transforms) {
        // the transform matrices follow the method: rebuild them
        TVD_CUDA_TRY(cudaDeviceSynchronize());
        gemm_precond_destroy(*plan);
        TVD_TRY(gemm_precond_create(*plan, s));
    }
    return TVD_OK;
}

int tvd_plan_method(tvd_plan plan) { return plan ? plan->method : TVD_METHOD_FP; }

tvd_status pbicgstab_solve(tvd_plan plan, const void* u_lag, double alpha, double beta, const void* b,
                           void* x_inout, double tol, int maxit, int* iters, double* relres, void* stream) {
    if (!plan || !u_lag || !b || !x_inout || !(alpha >= 0.0) || !(beta > 0.0) || !(tol > 0.0) || maxit < 0) {
        set_error("pbicgstab_solve: invalid argument");
        return TVD_EINVAL;
    }
    if (!plan->reblur()) {
        set_error("pbicgstab_solve: the plan solves eq. (fp); call tvd_plan_set_method(plan, TVD_METHOD_REBLUR)");
        return TVD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    SolveResult r;
    TVD_TRY(solve(*plan, (const double*)u_lag, alpha, beta, (const double*)b, (double*)x_inout, tol, maxit, &r, s));
    if (iters) *iters = r.iters;
    if (relres) *relres = r.relres;
    if (r.status != TVD_OK)
        set_error(r.status == TVD_ENOCONV ? "pbicgstab_solve: tolerance not reached within maxit"
                                          : "pbicgstab_solve: BiCGstab breakdown (zero rho, r^T v or t^T t)");
    return r.status;
}

tvd_status pcg_solve(tvd_plan plan, const void* u_lag, double alpha, double beta, const void* b, void* x_inout,
                     double tol, int maxit, int* iters, double* relres, void* stream) {
    if (!plan || !u_lag || !b || !x_inout || !(alpha >= 0.0) || !(beta > 0.0) || !(tol > 0.0) || maxit < 0) {
        set_error("pcg_solve: invalid argument");
        return TVD_EINVAL;
    }
    if (plan->reblur()) {
        set_error("pcg_solve: the plan solves eq. (fpp) (not symmetric); use pbicgstab_solve");
        return TVD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    SolveResult r;
    TVD_TRY(solve(*plan, (const double*)u_lag, alpha, beta, (const double*)b, (double*)x_inout, tol, maxit, &r, s));
    if (iters) *iters = r.iters;
    if (relres) *relres = r.relres;
    if (r.status != TVD_OK) {
        set_error(r.status == TVD_ENOCONV ? "pcg_solve: tolerance not reached within maxit"
                                          : "pcg_solve: CG breakdown (non-positive curvature or non-finite value)");
    }
    return r.status;
}

tvd_status tv_deblur(tvd_plan plan, const void* v, double alpha, double beta, int max_outer, double outer_tol,
                     double inner_tol, int inner_maxit, void* u_out, tvd_stats* stats, void* stream) {
    if (!plan || !v || !u_out || !(alpha >= 0.0) || !(beta > 0.0) || max_outer < 0 || !(inner_tol > 0.0) ||
        inner_maxit < 0) {
        set_error("tv_deblur: invalid argument");
        return TVD_EINVAL;
    }
    tvd_plan_s& p = *plan;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)p.nr * p.nc;
    double* u = (double*)u_out;
    p.hx_for = nullptr;
    // b = H^T v (eq. (fp)) or H' v = H v (eq. (fpp), symmetric PSF) into p.xd; u^0 = v
    const bool reblur = p.reblur();
    TVD_TRY(blur_apply<double>(p, p.d, !reblur, (const double*)v, p.xd, s));
    if (u != (const double*)v) TVD_CUDA_TRY(cudaMemcpyAsync(u, v, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (stats) {
        stats->outer_iters = 0;
        stats->total_inner_iters = 0;
        stats->refinement_sweeps = 0;
        stats->last_relres = 0.0;
        stats->last_rel_change = 0.0;
        stats->last_status = TVD_OK;
        stats->final_g_norm = 0.0;
        stats->final_functional = 0.0;
    }
    tvd_status overall = TVD_OK;
    const bool track_g = stats && stats->g_norm, track_f = stats && stats->functional;
    // ||g(x)|| and T(x) of an iterate x (eq. (el), eq. (mp)), on request; w(x) and H^T H x land
    // in p.d.w / p.hx, where the next FP step's set-up and first residual take them anyway
    auto track = [&](const double* x, double* gn, double* fn) -> tvd_status {
        double g2 = 0.0, parts[2] = {0.0, 0.0};
        TVD_TRY(el_residual(p, x, (const double*)v, p.xd, alpha, beta, p.res, &g2, track_f ? parts : nullptr, s));
        if (track_g) *gn = std::sqrt(g2);
        if (track_f) *fn = 0.5 * parts[0] + alpha * parts[1];
        return TVD_OK;
    };
    for (int k = 0; k < max_outer; ++k) {
        if ((track_g || track_f) && k < stats->cap) {
            double gn = 0.0, fn = 0.0;
            TVD_TRY(track(u, &gn, &fn));
            if (track_g) stats->g_norm[k] = gn;
            if (track_f) stats->functional[k] = fn;
        }
        TVD_CUDA_TRY(cudaMemcpyAsync(p.tmp, u, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        SolveResult r;
        // u_lag = u^k (kept in p.tmp), x starts at u^k and becomes u^{k+1} in place
        // from the second step on, H^T H u^k is known from the previous step's last residual check
        TVD_TRY(solve(p, p.tmp, alpha, beta, p.xd, u, inner_tol, inner_maxit, &r, s, k > 0 && !reblur));
        double h2[2];
        TVD_TRY(diffnorm2_d(p, u, p.tmp, p.scal + 2, s));
        TVD_TRY(norm2_d(p, u, p.scal + 3, s));
        TVD_CUDA_TRY(cudaMemcpyAsync(h2, p.scal + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        TVD_CUDA_TRY(cudaStreamSynchronize(s));
        const double change = std::sqrt(h2[0]) / std::max(std::sqrt(h2[1]), 1e-300);
        if (r.status != TVD_OK) overall = (overall == TVD_OK) ? r.status : overall;
        if (stats) {
            if (k < stats->cap && stats->inner_iters) stats->inner_iters[k] = r.iters;
            stats->outer_iters = k + 1;
            stats->total_inner_iters += r.iters;
            stats->refinement_sweeps += r.sweeps;
            stats->last_relres = r.relres;
            stats->last_rel_change = change;
            stats->last_status = r.status;
        }
        if (r.status == TVD_EBREAKDOWN) break;
        if (outer_tol > 0.0 && change < outer_tol) break;
    }
    if (track_g || track_f) {
        double gn = 0.0, fn = 0.0;
        TVD_TRY(track(u, &gn, &fn));
        stats->final_g_norm = gn;
        stats->final_functional = fn;
    }
    if (overall != TVD_OK)
        set_error(overall == TVD_ENOCONV ? "tv_deblur: an inner solve did not reach its tolerance"
                                         : "tv_deblur: an inner solve broke down");
    return overall;
}

tvd_status tv_deblur_newton(tvd_plan plan, const void* v, double alpha, double beta, void* u_inout, double tol,
                            int max_steps, double cg_tol, int cg_maxit, tvd_newton_stats* stats, void* stream) {
    if (!plan || !v || !u_inout || u_inout == v || !(alpha >= 0.0) || !(beta > 0.0) || !(tol > 0.0) ||
        max_steps < 0 || !(cg_tol > 0.0) || cg_maxit < 0) {
        set_error("tv_deblur_newton: invalid argument");
        return TVD_EINVAL;
    }
    if (plan->reblur()) {
        set_error("tv_deblur_newton: finishes the fixed point of eq. (fp) (a stationary point of the functional); "
                  "a reblurring plan has no such functional");
        return TVD_EINVAL;
    }
    tvd_plan_s& p = *plan;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)p.nr * p.nc;
    const bool mixed = p.mode == TVD_MODE_MIXED;
    double* u = (double*)u_inout;
    tvd_newton_stats local{};
    tvd_newton_stats& ns = stats ? *stats : local;
    ns = tvd_newton_stats{};
    p.hx_for = nullptr;
    double* scratch = nullptr;
    // b = H^T v, r = -g, d (the step), u0 (the iterate the step starts from), g_r, g_c, float g_r, g_c
    TVD_TRY(dalloc(&scratch, 6 * n + (mixed ? n : 0)));
    double *b = scratch, *r = b + n, *d = r + n, *u0 = d + n, *gr = u0 + n, *gc = gr + n;
    float* gf = mixed ? reinterpret_cast<float*>(gc + n) : nullptr;
    auto run = [&]() -> tvd_status {
        TVD_TRY(blur_apply<double>(p, p.d, true, (const double*)v, b, s));
        double g2 = 0.0;
        TVD_TRY(el_residual(p, u, (const double*)v, b, alpha, beta, r, &g2, nullptr, s));
        ns.g_norm_initial = std::sqrt(g2);
        ns.g_norm = ns.g_norm_initial;
        for (int k = 0; k < max_steps; ++k) {
            if (g2 == 0.0) return TVD_OK;
            if (!std::isfinite(g2)) {
                set_error("tv_deblur_newton: non-finite gradient");
                return TVD_EBREAKDOWN;
            }
            // J(u) d = -g(u) with the FP step's preconditioner at u
            if (mixed) TVD_TRY(setup_mixed(p, u, alpha, beta, s));
            else TVD_TRY(setup_precond<double>(p, p.d, u, alpha, beta, s));
            TVD_TRY(hess_coef(p, u, p.d.w, gr, gc, s));
            if (mixed) {
                TVD_TRY(cast_d2f(gr, gf, n, s));
                TVD_TRY(cast_d2f(gc, gf + n, n, s));
            }
            int it = 0;
            double rel = 0.0;
            const tvd_status cg = jacobian_solve(p, r, d, gr, gc, gf, mixed ? gf + n : nullptr, alpha, cg_tol,
                                                 cg_maxit, &it, &rel, s);
            ns.total_cg_iters += it;
            if (cg != TVD_OK && cg != TVD_ENOCONV) return cg;   // an inexact direction is still taken
            TVD_TRY(norm2_d(p, d, p.scal + 11, s));
            double d2 = 0.0;
            TVD_CUDA_TRY(cudaMemcpyAsync(&d2, p.scal + 11, sizeof(double), cudaMemcpyDeviceToHost, s));
            TVD_CUDA_TRY(cudaMemcpyAsync(u0, u, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            // u = u0 + t d, t = 1 halved while ||g|| does not fall (at most 10 halvings); a full
            // step whose relative change is already below tol is taken as it is (near the
            // solution ||g|| is at its rounding floor and need not fall)
            double t = 1.0, g2_new = 0.0, u2 = 0.0;
            bool accepted = false;
            for (int h = 0; h <= 10; ++h) {
                TVD_TRY(axpy_to_d(p, u0, d, t, u, p.scal + 11, s));
                TVD_TRY(el_residual(p, u, (const double*)v, b, alpha, beta, r, &g2_new, nullptr, s));
                TVD_CUDA_TRY(cudaMemcpyAsync(&u2, p.scal + 11, sizeof(double), cudaMemcpyDeviceToHost, s));
                TVD_CUDA_TRY(cudaStreamSynchronize(s));
                const bool tiny = h == 0 && std::sqrt(d2) < tol * std::sqrt(u2);
                if (g2_new < g2 || tiny) {
                    accepted = true;
                    break;
                }
                t *= 0.5;
                ++ns.halvings;
            }
            if (!accepted) {
                TVD_CUDA_TRY(cudaMemcpyAsync(u, u0, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
                TVD_CUDA_TRY(cudaStreamSynchronize(s));
                p.hx_for = nullptr;
                set_error("tv_deblur_newton: no step along the Newton direction lowered ||g||");
                return TVD_ENOCONV;
            }
            g2 = g2_new;
            ns.steps = k + 1;
            ns.last_t = t;
            ns.last_cg_relres = rel;
            ns.last_rel_change = t * std::sqrt(d2) / std::max(std::sqrt(u2), 1e-300);
            ns.g_norm = std::sqrt(g2);
            if (ns.last_rel_change < tol) return TVD_OK;
        }
        if (max_steps == 0 || g2 == 0.0) return TVD_OK;
        set_error("tv_deblur_newton: max_steps reached before the relative change fell below tol");
        return TVD_ENOCONV;
    };
    const tvd_status st = run();
    cudaStreamSynchronize(s);
    p.hx_for = nullptr;
    dfree(scratch);
    return st;
}

}  // extern "C"
