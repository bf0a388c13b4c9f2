// Diagnostics: a process-wide kernel launch counter and opt-in per-kernel
// device timing with CUDA events recorded on the stream each kernel runs on.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "rs_common.cuh"
#include "rs_diag.cuh"

namespace rs {
namespace {

std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_timing_on{0};

struct Pending {
    cudaEvent_t a, b;
    int device;
};

struct KernelStat {
    double ms = 0.0;
    unsigned long long launches = 0;
    double work = 0.0;  // algorithmic flops or bytes the launch site reported
    std::vector<Pending> pending;
};

std::mutex g_mu;
std::map<std::string, KernelStat>& stats() {
    static std::map<std::string, KernelStat> m;
    return m;
}

void resolve(KernelStat& s) {
    for (Pending& p : s.pending) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != p.device) cudaSetDevice(p.device);
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
            s.ms += ms;
        cudaGetLastError();
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
        if (cur != p.device) cudaSetDevice(cur);
    }
    s.pending.clear();
}

}  // namespace

void note_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int timing_mode() { return g_timing_on.load(std::memory_order_relaxed); }

KernelTimer::KernelTimer(const char* name, cudaStream_t st, double work, bool major,
                         bool allow_events)
    : name_(name), st_(st), work_(work) {
    note_launch(1);
    int mode = g_timing_on.load(std::memory_order_relaxed);
    if (!allow_events || mode == 0 || (mode == 1 && !major)) return;
    if (cudaEventCreate(&a_) != cudaSuccess || cudaEventCreate(&b_) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(a_, st_);
    active_ = true;
}

KernelTimer::~KernelTimer() {
    if (!active_) return;
    cudaEventRecord(b_, st_);
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    KernelStat& s = stats()[name_];
    s.pending.push_back({a_, b_, dev});
    s.launches += 1;
    s.work += work_;
}

}  // namespace rs

extern "C" {

unsigned long long rs_stats_kernel_launches(void) {
    return rs::g_launches.load(std::memory_order_relaxed);
}

rs_status rs_timing_enable(int mode) {
    if (mode < 0 || mode > 2) {
        rs::set_error("rs_timing_enable: mode %d not in {0, 1, 2}", mode);
        return RS_ERR_INVALID;
    }
    rs::g_timing_on.store(mode);
    return RS_OK;
}

rs_status rs_timing_reset(void) {
    std::lock_guard<std::mutex> lk(rs::g_mu);
    for (auto& kv : rs::stats()) rs::resolve(kv.second);
    rs::stats().clear();
    return RS_OK;
}

int rs_timing_count(void) {
    std::lock_guard<std::mutex> lk(rs::g_mu);
    return (int)rs::stats().size();
}

rs_status rs_timing_get(int index, char* name, size_t name_len, double* total_ms,
                        unsigned long long* launches, double* work) {
    rs::clear_error();
    std::lock_guard<std::mutex> lk(rs::g_mu);
    if (index < 0 || index >= (int)rs::stats().size() || !name || name_len == 0) {
        rs::set_error("rs_timing_get: bad index or buffer");
        return RS_ERR_INVALID;
    }
    auto it = rs::stats().begin();
    std::advance(it, index);
    rs::resolve(it->second);
    strncpy(name, it->first.c_str(), name_len - 1);
    name[name_len - 1] = 0;
    if (total_ms) *total_ms = it->second.ms;
    if (launches) *launches = it->second.launches;
    if (work) *work = it->second.work;
    return RS_OK;
}

}  // extern "C"
