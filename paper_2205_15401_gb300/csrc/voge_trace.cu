// voge_trace.cu -- optional per-kernel timing with CUDA events.
//
// When enabled, every kernel launch of the library is bracketed by two CUDA
// events recorded on the launch stream.  voge_trace_read() waits for the
// recorded events, sums the device time per kernel name and recycles the
// events.  Not for use while a stream is being captured into a CUDA graph.
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/voge.h"
#include "voge_trace.cuh"

namespace voge {
namespace {

struct Rec {
    int name;
    cudaEvent_t a, b;
};

struct Tracer {
    std::mutex mu;
    bool on = false;
    std::vector<std::string> names;
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    std::vector<int64_t> launches;
    std::vector<double> total_ms;

    int name_id(const char* n) {
        for (size_t q = 0; q < names.size(); ++q)
            if (names[q] == n) return (int)q;
        names.emplace_back(n);
        launches.push_back(0);
        total_ms.push_back(0.0);
        return (int)names.size() - 1;
    }
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
};

Tracer& tracer() {
    static Tracer* t = new Tracer();  // never destroyed: events may outlive static teardown
    return *t;
}

}  // namespace

TraceScope::TraceScope(const char* name, cudaStream_t s) : stream_(s), rec_(-1), a_(nullptr), b_(nullptr) {
    Tracer& t = tracer();
    std::lock_guard<std::mutex> g(t.mu);
    if (!t.on) return;
    a_ = t.get();
    b_ = t.get();
    if (!a_ || !b_) return;
    rec_ = t.name_id(name);
    cudaEventRecord(a_, s);
}

TraceScope::~TraceScope() {
    if (rec_ < 0) return;
    Tracer& t = tracer();
    std::lock_guard<std::mutex> g(t.mu);
    cudaEventRecord(b_, stream_);
    t.recs.push_back({rec_, a_, b_});
    t.launches[rec_] += 1;
}

}  // namespace voge

using voge::tracer;

extern "C" {

int voge_trace_enable(int on) {
    auto& t = voge::tracer();
    std::lock_guard<std::mutex> g(t.mu);
    const int prev = t.on ? 1 : 0;
    t.on = on != 0;
    return prev;
}

int voge_trace_read(voge_trace_entry* out, int max_entries) {
    auto& t = voge::tracer();
    std::lock_guard<std::mutex> g(t.mu);
    for (auto& r : t.recs) {
        float ms = 0.0f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess)
            t.total_ms[r.name] += ms;
        t.pool.push_back(r.a);
        t.pool.push_back(r.b);
    }
    t.recs.clear();
    const int n = (int)t.names.size();
    for (int q = 0; q < n && q < max_entries && out; ++q) {
        memset(&out[q], 0, sizeof(out[q]));
        strncpy(out[q].name, t.names[q].c_str(), sizeof(out[q].name) - 1);
        out[q].launches = t.launches[q];
        out[q].total_ms = t.total_ms[q];
    }
    return n;
}

void voge_trace_reset(void) {
    auto& t = voge::tracer();
    std::lock_guard<std::mutex> g(t.mu);
    for (auto& r : t.recs) {
        cudaEventSynchronize(r.b);
        t.pool.push_back(r.a);
        t.pool.push_back(r.b);
    }
    t.recs.clear();
    for (auto& x : t.launches) x = 0;
    for (auto& x : t.total_ms) x = 0.0;
}

}  // extern "C"
