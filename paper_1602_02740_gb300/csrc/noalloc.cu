// tc_toom_interpolate_noalloc: the interpolation step with built-in scratch.
//
// Some callers must not allocate device memory once they are running: for
// example a service that reserved all of the GPU's memory for its own pool at
// start-up, or a latency-critical loop where cudaMalloc/cudaFree (which can
// synchronise the device) is not acceptable.  This entry point computes
// exactly what tc_toom_interpolate computes, but the scratch that call takes
// from the caller lives here in a fixed device array, so nothing is
// allocated per call.
//
// The array below is TC_NOALLOC_SCRATCH_BYTES long and is part of the
// library's device image: every GPU that loads the library holds it until the
// process exits.  In host code its name is only a host-side stand-in, not a
// device address, so the host asks the runtime for the device address once
// per device (with that device current) and passes that pointer to the
// kernels.
#include <mutex>

#include "../../include/tc.h"
#include "tc_ctx.h"
#include "tc_internal.h"

namespace {

__device__ __align__(256) unsigned char noalloc_scratch[TC_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu[MAX_DEVICES];
void* g_addr[MAX_DEVICES];

// Device address of noalloc_scratch on the current device.  A successful
// lookup is cached for the device; a failed one is returned and not cached, so
// the next call tries again.
cudaError_t scratch_address(int device, void** out) {
    std::lock_guard<std::mutex> lk(g_mu[device]);
    if (!g_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();  // clear it: the next call starts clean
            *out = nullptr;
            return e;
        }
        g_addr[device] = p;
    }
    *out = g_addr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" tc_status tc_toom_interpolate_noalloc(size_t count, size_t limbs, int B,
                                                 const uint32_t* Y, size_t ystride,
                                                 const uint8_t* SGN_U, const uint8_t* SGN_V,
                                                 uint32_t* OUT, size_t ldo, void* stream) {
    if (count == 0) return TC_OK;
    if (!Y || !OUT || B < 2 || B > 32 || limbs == 0 || limbs > (1u << 30)) return TC_EINVAL;
    tc::LevelGeom g = tc::make_level((int)limbs, B);
    if (ystride < (size_t)(2 * g.e) || ystride % 4) return TC_EINVAL;
    if (reinterpret_cast<uintptr_t>(Y) & 15u) return TC_EINVAL;
    if (count > 1 && ldo < 2 * limbs) return TC_EINVAL;
    g.ystride = (int)ystride;
    const size_t need = count * tc::interp_work_bytes(g, (long)count);
    if (need > (size_t)TC_NOALLOC_SCRATCH_BYTES) return TC_ENOMEM;  // beyond the fixed array
    uint32_t* work = nullptr;
    if (need) {
        int device = 0;
        cudaError_t e = cudaGetDevice(&device);
        if (e != cudaSuccess) return tc_fail_cuda(e);
        if (device < 0 || device >= MAX_DEVICES) return TC_EINVAL;
        void* p = nullptr;
        e = scratch_address(device, &p);
        if (e != cudaSuccess || !p) return tc_fail_cuda(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        work = static_cast<uint32_t*>(p);
    }
    cudaError_t e = tc::launch_interp(g, Y, SGN_U, SGN_V, OUT, (long)ldo, 2 * g.s, work,
                                      (long)count, (cudaStream_t)stream);
    return e == cudaSuccess ? TC_OK : tc_fail_cuda(e);
}
