// Kernel profiler of libmsbicg: when enabled, every kernel launch of the
// library is bracketed by CUDA events on the stream it is launched on and
// attributed to a kernel class together with its algorithmic bytes and
// floating-point operations (the minimum the method must move / compute per
// launch, fixed by the problem sizes).  Results are read with
// msb_profile_read().  While enabled, the solver launches kernels directly
// instead of replaying CUDA graphs so that every launch can be timed.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

namespace msb {

bool prof_on();

// Records an event before the launch (constructor) and after it (done()).
struct ProfScope {
    int id = -1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    double bytes = 0, flops = 0;
    ProfScope(const char* name, cudaStream_t s, double alg_bytes, double alg_flops);
    void done();
    ~ProfScope() { done(); }
};

// Replace the work figures of the most recently recorded launch of `name`.
void prof_patch_last(const char* name, double alg_bytes, double alg_flops);

// Resolve the recorded events of completed work into the totals (call after a sync).
void prof_collect();

}  // namespace msb
