// Measured ceiling of the base case's inner step on this GPU.
//
// The schoolbook base case spends its time in one operation: a 32 x 32 ->
// 64-bit limb product added into a 96-bit column sum (mad.lo.cc, madc.hi.cc,
// addc: two integer multiplies and one add with the carry flag).  This kernel
// runs only that operation, on registers, with eight rows times eight columns
// of independent products per iteration (15 column sums, consecutive products
// on different columns), so the number it gives is what the integer pipes
// sustain for the base case's instruction mix with no loads, no stores and no
// carry resolution: the roofline of the base case.
#include "../../include/tc.h"
#include "tc_ctx.h"

namespace {

__device__ __forceinline__ void madc3(uint32_t& lo, uint32_t& mid, uint32_t& hi, uint32_t a,
                                      uint32_t b) {
    asm volatile(
        "mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(lo), "+r"(mid), "+r"(hi)
        : "r"(a), "r"(b));
}

constexpr int PEAK_THREADS = 256;

__global__ void __launch_bounds__(PEAK_THREADS)
peak_madc_kernel(int iters, uint32_t* sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[8], b[8], c0[15], c1[15], c2[15];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        a[i] = t * 2654435761u + 97u * i + 1u;
        b[i] = t * 40503u + 131u * i + 7u;
    }
#pragma unroll
    for (int c = 0; c < 15; ++c) c0[c] = c1[c] = c2[c] = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int i = 0; i < 8; ++i) madc3(c0[i + j], c1[i + j], c2[i + j], a[i], b[j]);
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] += c0[i];  // the next iteration's operands depend on this one
    }
    uint32_t x = 0;
#pragma unroll
    for (int c = 0; c < 15; ++c) x ^= c0[c] + c1[c] + c2[c];
    sink[t] = x;
}

}  // namespace

extern "C" tc_status tc_peak_madc(int blocks, int iters, uint32_t* sink, void* stream,
                                  double* limb_products) {
    if (blocks <= 0 || iters <= 0 || !sink || !limb_products) return TC_EINVAL;
    peak_madc_kernel<<<blocks, PEAK_THREADS, 0, (cudaStream_t)stream>>>(iters, sink);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tc_fail_cuda(e);
    *limb_products = (double)blocks * PEAK_THREADS * (double)iters * 64.0;
    return TC_OK;
}
