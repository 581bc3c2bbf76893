// Per-kernel device timing of the library's own launches (tracing).  When enabled,
// every launch made through DD_PROFILED brackets the kernel with two CUDA events on
// the launching stream; dd_profile_read waits for the recorded events and returns,
// per kernel name, the launch count and the summed device time.
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "dd_internal.h"

namespace {

struct Pending {
    std::string name;
    cudaEvent_t a, b;
};
struct Totals {
    int64_t launches = 0;
    double ms = 0.0;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Pending> g_pending;
std::map<std::string, Totals> g_totals;

}  // namespace

namespace dd {

bool profile_on() {
    std::lock_guard<std::mutex> lock(g_mu);
    return g_on;
}

ProfScope::ProfScope(const char *name, cudaStream_t stream) : name_(name), stream_(stream) {
    if (!profile_on()) return;
    if (cudaEventCreate(&a_) != cudaSuccess || cudaEventCreate(&b_) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(a_, stream_);
    active_ = true;
}

ProfScope::~ProfScope() {
    if (!active_) return;
    cudaEventRecord(b_, stream_);
    std::lock_guard<std::mutex> lock(g_mu);
    g_pending.push_back({name_, a_, b_});
}

}  // namespace dd

extern "C" {

dd_status dd_profile_enable(int32_t on) {
    dd::clear_error();
    std::lock_guard<std::mutex> lock(g_mu);
    g_on = on != 0;
    return DD_OK;
}

dd_status dd_profile_reset(void) {
    dd::clear_error();
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto &p : g_pending) {
        cudaEventSynchronize(p.b);
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pending.clear();
    g_totals.clear();
    return DD_OK;
}

dd_status dd_profile_read(char *names, int64_t *launches, double *total_ms, int32_t max_entries,
                          int32_t *n_entries) {
    dd::clear_error();
    if (!n_entries || max_entries < 0 || (max_entries > 0 && (!names || !launches || !total_ms)))
        return dd::fail(DD_EINVAL, "dd_profile_read: bad arguments");
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto &p : g_pending) {
        cudaError_t err = cudaEventSynchronize(p.b);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, p.a, p.b);
        if (err != cudaSuccess) return dd::fail_cuda(err, "dd_profile_read: event");
        Totals &t = g_totals[p.name];
        t.launches += 1;
        t.ms += ms;
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pending.clear();
    int32_t k = 0;
    for (auto &kv : g_totals) {
        if (k >= max_entries) break;
        std::strncpy(names + 64 * k, kv.first.c_str(), 63);
        names[64 * k + 63] = 0;
        launches[k] = kv.second.launches;
        total_ms[k] = kv.second.ms;
        ++k;
    }
    *n_entries = (int32_t)g_totals.size();
    return DD_OK;
}

}  // extern "C"
