// Batched FP solves of independent problems: a pool of host worker threads,
// each owning a CUDA stream, takes items largest first (whole groups of items
// that share a plan, so a plan is never used by two streams at once). The
// items' kernels overlap on the GPU; no item depends on another, so there is
// no exchange between them.
#include "common.cuh"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <numeric>
#include <thread>
#include <unordered_map>
#include <vector>

extern "C" tvd_status tv_deblur_batched(tvd_batch_item* items, int count, int max_outer, double inner_tol,
                                        int inner_maxit, int workers, void* stream) {
    using tvd::set_error;
    if (count < 0 || (count > 0 && !items) || max_outer < 0 || !(inner_tol > 0.0) || inner_maxit < 0 ||
        workers < 0 || workers > 64) {
        set_error("tv_deblur_batched: invalid argument");
        return TVD_EINVAL;
    }
    for (int i = 0; i < count; ++i)
        if (!items[i].plan || !items[i].v || !items[i].u_out || !(items[i].alpha >= 0.0) || !(items[i].beta > 0.0)) {
            set_error("tv_deblur_batched: item " + std::to_string(i) + " has a null plan / buffer or a bad alpha, beta");
            return TVD_EINVAL;
        }
    if (count == 0) return TVD_OK;
    if (workers == 0) workers = 8;

    // groups of items sharing a plan, largest plan first
    std::unordered_map<tvd_plan, int> gid;
    std::vector<std::vector<int>> groups;
    for (int i = 0; i < count; ++i) {
        auto it = gid.find(items[i].plan);
        if (it == gid.end()) {
            gid.emplace(items[i].plan, (int)groups.size());
            groups.push_back({i});
        } else {
            groups[it->second].push_back(i);
        }
    }
    std::stable_sort(groups.begin(), groups.end(), [&](const std::vector<int>& a, const std::vector<int>& b) {
        const tvd_plan pa = items[a[0]].plan, pb = items[b[0]].plan;
        return (size_t)pa->nr * pa->nc * a.size() > (size_t)pb->nr * pb->nc * b.size();
    });
    workers = std::min<int>(workers, (int)groups.size());

    // the items start after the work already queued on the caller's stream
    cudaStream_t caller = (cudaStream_t)stream;
    cudaEvent_t ready = nullptr;
    TVD_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    if (cudaEventRecord(ready, caller) != cudaSuccess) {
        cudaEventDestroy(ready);
        set_error("tv_deblur_batched: cudaEventRecord failed");
        return TVD_ECUDA;
    }

    std::atomic<int> next{0};
    std::vector<std::string> msgs(count);
    auto work = [&]() {
        cudaStream_t s = nullptr;
        const bool ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
                        cudaStreamWaitEvent(s, ready, 0) == cudaSuccess;
        for (;;) {
            const int g = next.fetch_add(1);
            if (g >= (int)groups.size()) break;
            for (int i : groups[g]) {
                tvd_batch_item& it = items[i];
                if (!ok) {
                    it.status = TVD_ECUDA;
                    msgs[i] = "tv_deblur_batched: could not create a worker stream";
                    continue;
                }
                tvd_stats stats{};
                stats.inner_iters = it.inner_iters;
                stats.cap = it.inner_iters ? max_outer : 0;
                it.status = tv_deblur(it.plan, it.v, it.alpha, it.beta, max_outer, it.outer_tol, inner_tol,
                                      inner_maxit, it.u_out, &stats, s);
                it.outer_iters = stats.outer_iters;
                if (it.status != TVD_OK) msgs[i] = tvd_last_error();
            }
        }
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    };
    std::vector<std::thread> pool;
    pool.reserve(workers);
    for (int t = 0; t < workers; ++t) pool.emplace_back(work);
    for (auto& t : pool) t.join();
    cudaEventDestroy(ready);
    for (int i = 0; i < count; ++i)
        if (items[i].status != TVD_OK) {
            set_error("item " + std::to_string(i) + ": " + msgs[i]);
            return items[i].status;
        }
    return TVD_OK;
}
