// voge_trace.cuh -- RAII bracket of one kernel launch for voge_trace_* timing.
#pragma once

#include <cuda_runtime.h>

namespace voge {

class TraceScope {
   public:
    TraceScope(const char* name, cudaStream_t s);
    ~TraceScope();
    TraceScope(const TraceScope&) = delete;
    TraceScope& operator=(const TraceScope&) = delete;

   private:
    cudaStream_t stream_;
    int rec_;
    cudaEvent_t a_, b_;
};

}  // namespace voge
