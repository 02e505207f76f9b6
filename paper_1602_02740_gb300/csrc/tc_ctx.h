// The context object behind the opaque tc_ctx handle.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <utility>
#include <vector>

#include "../../include/tc.h"

#include "tc_internal.h"

namespace tc {
struct Server;
tc_opts plan_for(tc_ctx* ctx, size_t s);
bool plan_valid(const tc_opts& o, size_t s);

// Scratch layout of a uniform batch (byte offsets into one scratch block).
struct BatchLayout {
    std::vector<LevelGeom> g;
    std::vector<long> P;          // products at each level (P[0] = count)
    std::vector<size_t> evalU, evalV, sgnU, sgnV, prod, work, evwork;
    int base = TC_BASE_SCHOOLBOOK;
    size_t ntt = 0;               // transform scratch of the base products (TC_BASE_NTT)
    size_t total = 0;
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

BatchLayout layout_for(size_t count, size_t s, const tc_opts& o, bool square);

// Run a uniform batch of `count` s x s products (operand rows A/Bm, result rows
// OUT) with scratch `base` laid out by L.  ctx may be null (no phase timing).
// Segment-parallel levels OR their bounded-wait error words into *sticky
// (device memory; nullptr = not reported), by kernels on `st`: nothing waits.
tc_status run_uniform(const BatchLayout& L, char* base, size_t count, size_t s, const uint32_t* A,
                      long lda, const uint32_t* Bm, long ldb, uint32_t* OUT, long ldo, bool square,
                      cudaStream_t st, tc_ctx* ctx, int* sticky);

// Bits of a sticky device error word.
constexpr int TC_STICKY_TIMEOUT = 1;  // a bounded wait gave up
constexpr int TC_STICKY_INVALID = 2;  // a device-side table entry was out of range

// *sticky |= TC_STICKY_TIMEOUT if *word is set, on `st` (one thread).
cudaError_t launch_or_error(int* sticky, const int* word, cudaStream_t st);

// Padded balanced length class of an operand length (at most 50% padding).
size_t size_class(size_t L);

// Independent work on several streams: fork() makes every stream of the fan wait
// for the work enqueued so far on `st`, join() makes `st` wait for every stream
// of the fan.  Events only, so a fork/join inside a stream capture becomes
// parallel branches of the graph.
struct StreamFan {
    static constexpr int K = 8;
    cudaStream_t s[K] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[K] = {};
    bool ready = false;
    cudaError_t init();
    void destroy();
    cudaError_t fork(cudaStream_t st);
    cudaError_t join(cudaStream_t st);
};
}  // namespace tc

struct tc_ctx {
    int device = 0;
    size_t budget = 0;
    void* arena = nullptr;      // level scratch (grown on demand, never above budget)
    size_t arena_bytes = 0;
    void* aux = nullptr;        // staging buffers of the host-pointer entry point
    size_t aux_bytes = 0;
    std::vector<std::pair<size_t, tc_opts>> table;  // autotuned plans: (max limbs, plan)
    int* err_dev = nullptr;     // sticky bounded-wait error word of this context's calls (tc_check)
    // pinned staging of tc_mul_batch's index tables: two buffers used in turn, each
    // reused only after the copy that last read it has completed (pin_ev)
    void* pin[2] = {nullptr, nullptr};
    size_t pin_bytes[2] = {0, 0};
    cudaEvent_t pin_ev[2] = {nullptr, nullptr};
    int pin_turn = 0;
    tc::StreamFan fan;          // size classes of tc_mul_batch run concurrently on these
    tc::Server* server = nullptr;
    // phase timing (tc_profile_enable)
    bool profile = false;
    struct Rec { int kind, level; cudaEvent_t a, b; double bytes, lp; const char* kernel; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> event_pool;
};

tc_status tc_fail_cuda(cudaError_t e);
