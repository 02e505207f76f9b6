// Internal host-side interface between the C-ABI layer and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace tc {

// Name of the kernel (or kernel sequence) the last launch_* call on this thread
// chose; the phase timer records it beside each launch's time.
extern thread_local const char* g_kernel_name;
inline void note_kernel(const char* name) { g_kernel_name = name; }

// Geometry of one Toom level for operands of s limbs split into B blocks.
struct LevelGeom {
    int B, n;      // blocks, degree n = B - 1
    int s;         // operand length (limbs)
    int b;         // block size = ceil(s / B)
    int e;         // evaluation length = b + ceil((n(n-1)+1)/32)
    int estride;   // evaluation row stride: roundup(e, 4)
    int ystride;   // pointwise-product row stride: roundup(2e, 4)
    int K;         // limbs per lane in interpolation passes (4 or 8)
    int Y;         // interpolation value length: roundup(2e + 2, 32 K)
};

LevelGeom make_level(int s, int B);

// Exact-division constants of the Newton loops, passed by value to kernels.
struct DivTable;

// Largest operand length the base-case kernel accepts.
constexpr int LEAF_MAX = 1024;

cudaError_t launch_leaf(const uint32_t* A, long lda, const uint32_t* Bm, long ldb,
                        uint32_t* OUT, long ldo, int s, long P, cudaStream_t st);
// Limb products launch_leaf performs for P products of s limbs (s^2 each, or
// 2k^2 + (s - k)^2 with the in-kernel Karatsuba level).
double leaf_limb_products(int s, long P);

// Plain schoolbook of any operand length (column sums in `cols`, see below).
size_t schoolbook_big_bytes(int s, long P);
cudaError_t launch_schoolbook_big(const uint32_t* A, long lda, const uint32_t* Bm, long ldb,
                                  uint32_t* OUT, long ldo, int s, long P, uint32_t* cols,
                                  cudaStream_t st);

// `work`: wide_eval_work_bytes(g, P) bytes when use_wide_eval(g, P), else unused.
// Both operands of P products (rows in / in2); one launch when P is small.
cudaError_t launch_eval2(const uint32_t* in, long in_stride, uint32_t* out, uint8_t* sgn,
                         const uint32_t* in2, long in2_stride, uint32_t* out2, uint8_t* sgn2,
                         const LevelGeom& g, long P, void* work, cudaStream_t st);
cudaError_t launch_eval(const uint32_t* in, long in_stride, const LevelGeom& g,
                        uint32_t* out, uint8_t* sgn, long P, void* work, cudaStream_t st);
bool use_wide_eval(const LevelGeom& g, long P);
size_t wide_eval_work_bytes(const LevelGeom& g, long P);
int* wide_eval_error_word(void* work, const LevelGeom& g, long P);
cudaError_t launch_wide_eval(const uint32_t* in, long in_stride, const LevelGeom& g, uint32_t* out,
                             uint8_t* sgn, long P, void* work, cudaStream_t st);

// Per-product bytes of global work the interpolation of P products needs (0 = shared memory).
size_t interp_work_bytes(const LevelGeom& g, long P);

cudaError_t launch_interp(const LevelGeom& g, const uint32_t* y, const uint8_t* su,
                          const uint8_t* sv, uint32_t* out, long out_stride, int out_len,
                          uint32_t* work, long P, cudaStream_t st);

// Levels with few, huge products: segment-parallel interpolation (wide.cu).
bool use_wide(const LevelGeom& g, long P);
size_t wide_work_bytes(const LevelGeom& g, long P);
int* wide_error_word(void* work, const LevelGeom& g, long P);
cudaError_t launch_wide_interp(const LevelGeom& g, const uint32_t* y, const uint8_t* su,
                               const uint8_t* sv, uint32_t* out, long out_stride, int out_len,
                               void* work, long P, cudaStream_t st);

// out[0 .. out_len) = sum_k w_k 2^(32 off k), w_k = rows[k*row_stride .. + row_len),
// for `count` terms; one output (single CTA).  Used to add sliced partial products.
cudaError_t launch_overlap_add(const uint32_t* rows, long row_stride, int row_len, long count,
                               long off, uint32_t* out, long out_len, cudaStream_t st);

cudaError_t launch_zero(uint32_t* p, size_t n, cudaStream_t st);

// Base product by number-theoretic transform (ntt.cu): P products of s x s limbs.
constexpr int NTT_MAX_LIMBS = 1 << 24;
int ntt_log2(int s);
size_t ntt_work_bytes(int s, long P, bool square);
cudaError_t launch_ntt_mul(const uint32_t* A, long lda, const uint32_t* Bm, long ldb, uint32_t* OUT,
                           long ldo, int s, long P, bool square, void* work, cudaStream_t st);

}  // namespace tc
