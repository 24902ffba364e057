// Kernel tracing: CUDA event pairs around launches, summed per kernel name.
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "internal.cuh"

namespace argcsr {
namespace {

struct Record { const char *name; cudaEvent_t start, stop; };
struct Summary { const char *name; int64_t launches; double ms; };

constexpr size_t kTracePool = 4096;   // events made ahead by argcsr_trace_begin

std::mutex g_mu;
bool g_on = false;
char g_only[64] = "";                // non-empty: trace only the kernel of this name
std::vector<cudaEvent_t> g_free;     // reusable events
std::vector<Record> g_records;
std::vector<Summary> g_summary;

cudaEvent_t take_event() {
    if (!g_free.empty()) { cudaEvent_t e = g_free.back(); g_free.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

}  // namespace

int trace_start(const char *name, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_on) return -1;
    if (g_only[0] && strcmp(name, g_only) != 0) return -1;
    Record r{name, take_event(), take_event()};
    if (!r.start || !r.stop) return -1;
    cudaEventRecord(r.start, s);
    g_records.push_back(r);
    return (int)g_records.size() - 1;
}

bool trace_active() {
    std::lock_guard<std::mutex> lock(g_mu);
    return g_on;
}

void trace_stop(int token, cudaStream_t s) {
    if (token < 0) return;
    std::lock_guard<std::mutex> lock(g_mu);
    if (token < (int)g_records.size()) cudaEventRecord(g_records[token].stop, s);
}

}  // namespace argcsr

using namespace argcsr;

extern "C" {

static argcsr_status trace_begin(const char *only) {
    std::lock_guard<std::mutex> lock(g_mu);
    snprintf(g_only, sizeof g_only, "%s", only ? only : "");
    for (auto &r : g_records) { g_free.push_back(r.start); g_free.push_back(r.stop); }
    g_records.clear();
    g_summary.clear();
    // events for the first kTracePool / 2 launches are made here, so that a
    // traced region does not pay for cudaEventCreate on its launch path
    while (g_free.size() < kTracePool) {
        cudaEvent_t e = nullptr;
        const cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return record_cuda(err, "argcsr_trace_begin");
        g_free.push_back(e);
    }
    g_records.reserve(kTracePool / 2);
    g_on = true;
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_trace_begin(void) { return trace_begin(nullptr); }

ARGCSR_API argcsr_status argcsr_trace_begin_kernel(const char *name) {
    if (name && strlen(name) >= sizeof g_only) return ARGCSR_EINVAL;
    return trace_begin(name);
}

ARGCSR_API argcsr_status argcsr_trace_end(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_on = false;
    g_summary.clear();
    for (auto &r : g_records) {
        cudaError_t e = cudaEventSynchronize(r.stop);
        if (e != cudaSuccess) return record_cuda(e, "argcsr_trace_end");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, r.start, r.stop);
        if (e != cudaSuccess) return record_cuda(e, "argcsr_trace_end");
        Summary *sum = nullptr;
        for (auto &x : g_summary) if (strcmp(x.name, r.name) == 0) sum = &x;
        if (!sum) { g_summary.push_back({r.name, 0, 0.0}); sum = &g_summary.back(); }
        sum->launches += 1;
        sum->ms += ms;
    }
    return ARGCSR_OK;
}

ARGCSR_API int32_t argcsr_trace_kernel_count(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    return (int32_t)g_summary.size();
}

ARGCSR_API argcsr_status argcsr_trace_kernel(int32_t index, const char **name, int64_t *launches,
                                             double *total_ms) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (index < 0 || index >= (int32_t)g_summary.size()) return ARGCSR_EINVAL;
    if (name) *name = g_summary[index].name;
    if (launches) *launches = g_summary[index].launches;
    if (total_ms) *total_ms = g_summary[index].ms;
    return ARGCSR_OK;
}

}  // extern "C"
