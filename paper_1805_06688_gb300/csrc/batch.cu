// The batched form: independent problem instances solved concurrently on one GPU.
//
// A single MGRIT solve is latency-bound on its coarse levels (few slices per launch, long chains of
// dependent steps), so one instance leaves most of the GPU idle there.  Independent instances have
// no data dependence at all: each one runs its own solve (inner V-cycles replayed as its own CUDA
// graph) on its own stream, driven by a pool of host threads, and the hardware interleaves their
// launches.  A context created on the legacy default stream gets a private non-blocking stream for
// the duration of the call.
//
// The batch ends with its slowest instance, so instances start in order of decreasing work per
// step sweep, N_t P_x P_y (P_x + P_y), and the quarter with the most work gets the highest stream
// priority: the long solves run at full speed from the start and the short ones fill in around
// them (longest-processing-time-first scheduling).
#include <algorithm>
#include <atomic>
#include <thread>
#include <unordered_set>
#include <vector>

#include "sfde_internal.cuh"

static sfde_status batch_solve_impl(int n, sfde_ctx* const* ctxs, const mgrit_opts* opts, double* const* U_T,
                                    mgrit_stats* stats, sfde_status* status) {
    if (n < 1 || !ctxs) return SFDE_EINVAL;
    std::unordered_set<const sfde_ctx*> seen;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i] || !seen.insert(ctxs[i]).second) return SFDE_EINVAL;   // distinct contexts only
    int dev = 0;
    SFDE_CUDA(cudaGetDevice(&dev));
    std::vector<int> order(n);
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) {
        order[i] = i;
        const sfde_ctx* c = ctxs[i];
        cost[i] = (double)c->nt * c->x.P * c->y.P * (double)(c->x.P + c->y.P);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    int prio_low = 0, prio_high = 0;
    SFDE_CUDA(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    std::vector<cudaStream_t> own(n, nullptr);
    sfde_status first = SFDE_OK;
    for (int r = 0; r < n && first == SFDE_OK; ++r) {
        const int i = order[r];
        if (!ctxs[i]->stream) {
            const int prio = r < (n + 3) / 4 ? prio_high : prio_low;
            if (cudaStreamCreateWithPriority(&own[i], cudaStreamNonBlocking, prio) != cudaSuccess) first = SFDE_ECUDA;
            else ctxs[i]->stream = own[i];
        }
    }
    std::vector<sfde_status> st(n, SFDE_OK);
    if (first == SFDE_OK) {
        std::atomic<int> next{0};
        auto work = [&]() {
            cudaSetDevice(dev);   // a new host thread starts on device 0
            for (int r; (r = next.fetch_add(1)) < n;) {
                const int i = order[r];
                st[i] = mgrit_solve(ctxs[i], opts, nullptr, U_T ? U_T[i] : nullptr, stats ? &stats[i] : nullptr);
                if (st[i] == SFDE_OK || st[i] == SFDE_ENOCONV) {
                    const cudaError_t e = cudaStreamSynchronize(ctxs[i]->stream);
                    if (e != cudaSuccess) { sfde_set_last_cuda_error(e, "batch solve", __FILE__, __LINE__); st[i] = SFDE_ECUDA; }
                }
            }
        };
        const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        const int nth = std::max(1, std::min({n, 16, hw}));
        std::vector<std::thread> pool;
        pool.reserve(nth);
        for (int t = 1; t < nth; ++t) {
            try {
                pool.emplace_back(work);
            } catch (...) {   // no more threads: those running (and this one) take the remaining instances
                break;
            }
        }
        work();
        for (auto& t : pool) t.join();
        for (int i = 0; i < n; ++i)
            if (st[i] != SFDE_OK && first == SFDE_OK) first = st[i];
    }
    for (int i = 0; i < n; ++i)
        if (own[i]) {
            cudaStreamSynchronize(own[i]);
            ctxs[i]->stream = nullptr;
            cudaStreamDestroy(own[i]);
        }
    if (status) std::copy(st.begin(), st.end(), status);
    return first;
}

extern "C" sfde_status sfde_batch_solve(int n, sfde_ctx* const* ctxs, const mgrit_opts* opts, double* const* U_T,
                                       mgrit_stats* stats, sfde_status* status) {
    return sfde_no_throw([&] { return batch_solve_impl(n, ctxs, opts, U_T, stats, status); });
}
