// Per-kernel timing with CUDA events and a launch counter.
//
// When enabled, every kernel launch of this library is bracketed by two
// events recorded on the launch stream; tc_profile_collect synchronises them
// and reports launch counts and summed device milliseconds per kernel.  Used
// by the benchmark to measure each kernel's average duration inside the
// timed region (roofline).  Disabled by default: launches then pay nothing
// but a counter increment.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "profile.cuh"

namespace {

const char *kNames[TCK_COUNT] = {
    "k_fwd_col", "k_fwd_row", "k_fwd_det", "k_adj_det", "k_adj_row", "k_adj_col",
    "k_prior", "k_dots_gzx_gg", "k_update", "k_reduce_finalize", "k_solver_scalar",
    "k_dot", "k_scale_inv_sqrt", "k_fill_scalars", "k_nrm_col_fwd", "k_nrm_row", "k_nrm_col_adj",
    "k_prior_next", "k_restart_fixup"};

struct Rec {
    int id;
    cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
std::atomic<long long> g_launches{0};

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

}  // namespace

int prof_begin(int id, cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_on) return -1;
    std::lock_guard<std::mutex> lk(g_mu);
    Rec r{id, get_event(), get_event()};
    if (!r.a || !r.b) return -1;
    cudaEventRecord(r.a, s);
    g_recs.push_back(r);
    return (int)g_recs.size() - 1;
}

void prof_end(int h, cudaStream_t s) {
    if (h < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (h < (int)g_recs.size()) cudaEventRecord(g_recs[h].b, s);
}

extern "C" {

int tc_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    for (Rec &r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    return TC_OK;
}

int tc_profile_collect(int max_kernels, long long *counts, double *ms) {
    if (max_kernels < 0 || (max_kernels > 0 && (!counts || !ms))) return TC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    for (int i = 0; i < max_kernels; ++i) {
        counts[i] = 0;
        ms[i] = 0.0;
    }
    for (Rec &r : g_recs) {
        TC_CUDA(cudaEventSynchronize(r.b));
        float t = 0.f;
        TC_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        if (r.id < max_kernels) {
            counts[r.id] += 1;
            ms[r.id] += t;
        }
    }
    return TCK_COUNT;
}

const char *tc_profile_kernel_name(int id) {
    return (id >= 0 && id < TCK_COUNT) ? kNames[id] : "";
}

long long tc_launch_count(void) { return g_launches.load(); }

}  // extern "C"
