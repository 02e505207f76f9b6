// The context object behind the opaque tc_ctx handle.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <utility>
#include <vector>

#include "../../include/tc.h"

namespace tc {
struct Server;
tc_opts plan_for(tc_ctx* ctx, size_t s);
}  // namespace tc

struct tc_ctx {
    int device = 0;
    size_t budget = 0;
    void* arena = nullptr;      // level scratch (grown on demand, never above budget)
    size_t arena_bytes = 0;
    void* aux = nullptr;        // staging buffers of the host-pointer entry point
    size_t aux_bytes = 0;
    std::vector<std::pair<size_t, tc_opts>> table;  // autotuned plans: (max limbs, plan)
    tc::Server* server = nullptr;
    // phase timing (tc_profile_enable)
    bool profile = false;
    struct Rec { int kind, level; cudaEvent_t a, b; double bytes, lp; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> event_pool;
};

tc_status tc_fail_cuda(cudaError_t e);
