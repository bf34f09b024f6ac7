// Launch accounting and optional CUDA-event timing per kernel class.
//
// Every launcher counts the kernels it enqueues. When profiling is enabled,
// it also records a CUDA event pair around its launches on the launching
// stream; tvd_profile_read synchronises on those events and returns the summed
// device time and launch count of a class.
#include "common.cuh"

#include <atomic>
#include <mutex>

namespace tvd {

static std::atomic<unsigned long long> g_launches{0};
thread_local int capture_kernels_ = 0;
static std::atomic<int> g_profile{0};

struct ClassRecord {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    long long launches = 0;
};
static std::mutex g_mu;
static ClassRecord g_rec[PROF_NUM_CLASSES];

static const char* kNames[PROF_NUM_BASE] = {
    "blur_forward", "blur_adjoint_L", "precond_row_forward", "precond_column_solve", "precond_row_inverse",
    "spectrum_row", "spectrum_column", "cg_init", "cg_p_update", "cg_xr_update", "cg_simple_precond",
    "tv_coefficients", "vector_misc", "precond_gemm_tc", "precond_gemm_vector"};

static thread_local bool t_capturing = false;

void set_capturing(bool on) {
    t_capturing = on;
    if (on) capture_kernels_ = 0;
}
int captured_kernels() { return capture_kernels_; }
bool profiling_enabled() { return g_profile.load(std::memory_order_relaxed) != 0; }

void count_launches(int k) {
    if (!t_capturing) g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed);
}

ProfScope::ProfScope(int cls, cudaStream_t s, int nkernels) : cls_(cls), s_(s), start_(nullptr) {
    count_launches(nkernels);
    if (t_capturing) capture_kernels_ += nkernels;
    if (g_profile.load(std::memory_order_relaxed) && !t_capturing) {
        if (cudaEventCreate(&start_) == cudaSuccess) cudaEventRecord(start_, s_);
        else start_ = nullptr;
        std::lock_guard<std::mutex> lk(g_mu);
        g_rec[cls_].launches += nkernels;
    }
}

ProfScope::~ProfScope() {
    if (!start_) return;
    cudaEvent_t stop;
    if (cudaEventCreate(&stop) != cudaSuccess) {
        cudaEventDestroy(start_);
        return;
    }
    cudaEventRecord(stop, s_);
    std::lock_guard<std::mutex> lk(g_mu);
    g_rec[cls_].ev.emplace_back(start_, stop);
}

static void clear_records() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : g_rec) {
        for (auto& e : r.ev) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
        r.ev.clear();
        r.launches = 0;
    }
}

}  // namespace tvd

extern "C" {

unsigned long long tvd_kernel_launches(void) { return tvd::g_launches.load(); }

tvd_status tvd_profile_enable(int on) {
    tvd::clear_records();
    tvd::g_profile.store(on ? 1 : 0);
    return TVD_OK;
}

int tvd_profile_classes(void) { return tvd::PROF_NUM_CLASSES; }

const char* tvd_profile_name(int cls) {
    static thread_local std::string name;
    if (cls < 0 || cls >= tvd::PROF_NUM_CLASSES) return "";
    name = std::string(tvd::kNames[cls % tvd::PROF_NUM_BASE]) + (cls >= tvd::PROF_NUM_BASE ? ".f64" : ".f32");
    return name.c_str();
}

tvd_status tvd_profile_read(int cls, double* total_ms, long long* launches) {
    if (cls < 0 || cls >= tvd::PROF_NUM_CLASSES || !total_ms || !launches) {
        tvd::set_error("tvd_profile_read: invalid argument");
        return TVD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(tvd::g_mu);
    double acc = 0.0;
    for (auto& e : tvd::g_rec[cls].ev) {
        if (cudaEventSynchronize(e.second) != cudaSuccess) {
            tvd::set_error("tvd_profile_read: event synchronisation failed");
            return TVD_ECUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e.first, e.second);
        acc += ms;
    }
    *total_ms = acc;
    *launches = tvd::g_rec[cls].launches;
    return TVD_OK;
}

}  // extern "C"
