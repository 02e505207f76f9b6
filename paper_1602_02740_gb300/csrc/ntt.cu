// Exact products by a number-theoretic transform: the base product for
// Toom-Cook over a fast multiply (Section 5: Toom-Cook as the parallel
// wrapper around an FFT multiplication, with the 2B-1 pointwise products of
// the top level computed by the FFT product).
//
// Arithmetic is modulo the prime p = 2^64 - 2^32 + 1, whose multiplicative
// group has order 2^32 (2^32 - 1): it holds roots of unity of every order 2^n,
// n <= 32, and reduces a 128-bit product with shifts, adds and subtractions
// (2^64 = 2^32 - 1 and 2^96 = -1 modulo p).
//
// Product of two s-limb operands: each operand is read as 2s digits of 16 bits,
// zero-padded to N = 2^n >= 4s points; the cyclic convolution of length N of
// the digit vectors is the exact digit-wise product, because every coefficient
// is below N (2^16 - 1)^2 < 2^(n + 32) < p for n <= 31.  The transform is a
// four-step decomposition over fields of the point index (at most 8 bits,
// 256 points, per pass): each pass runs, for every column of a block, an
// in-place radix-2 transform of one field in shared memory and multiplies the
// results by the four-step twiddles.  Forward passes go from the top field
// down and leave the spectrum in a fixed permuted order; the inverse passes
// undo them in reverse order, so no reordering pass is needed.  The
// coefficients c_k are then placed at bit 16k and carried into 2s limbs.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/tc.h"
#include "tc_ctx.h"
#include "tc_device.cuh"
#include "tc_internal.h"

namespace tc {

constexpr u64 GL_P = 0xFFFFFFFF00000001ull;
constexpr int NTT_TILE = 4096;       // transform elements per CTA and pass
constexpr int NTT_KMAX = 8;          // largest field (256-point sub-transforms)
constexpr int NTT_THREADS = 256;
constexpr int CARRY_SEG = 32 * CH;   // output limbs per carry segment (one warp)

// ---------------------------------------------------------------- arithmetic mod p
// Operands and results in [0, p).

__device__ __forceinline__ u64 gl_add(u64 a, u64 b) {
    const u64 s = a + b;
    if (s < a) return s + 0xFFFFFFFFull;  // a + b = s + 2^64 = s + 2^32 - 1 (mod p), below p
    return s >= GL_P ? s - GL_P : s;
}

__device__ __forceinline__ u64 gl_sub(u64 a, u64 b) {
    const u64 d = a - b;
    return a < b ? d + GL_P : d;          // wraps to a - b + p
}

__device__ __forceinline__ u64 gl_mul(u64 a, u64 b) {
    const u64 lo = a * b, hi = __umul64hi(a, b);
    const u64 hh = hi >> 32, hl = hi & 0xFFFFFFFFull;
    u64 t = lo - hh;                      // lo - hh 2^96 with 2^96 = -1
    if (lo < hh) t -= 0xFFFFFFFFull;      // borrow: + p
    const u64 u = (hl << 32) - hl;        // hl 2^64 with 2^64 = 2^32 - 1
    u64 r = t + u;
    if (r < u) r += 0xFFFFFFFFull;        // carry: + 2^64 = + (2^32 - 1)
    return r >= GL_P ? r - GL_P : r;
}

// ---------------------------------------------------------------- host side

static u64 h_mul(u64 a, u64 b) {
    return (u64)(((unsigned __int128)a * b) % GL_P);
}

static u64 h_pow(u64 a, u64 e) {
    u64 r = 1;
    while (e) {
        if (e & 1) r = h_mul(r, a);
        a = h_mul(a, a);
        e >>= 1;
    }
    return r;
}

// A primitive 2^n-th root of unity: g^((p-1) / 2^n) for the generator g = 7
// of the multiplicative group modulo p.
static u64 h_root(int n) { return h_pow(7, (GL_P - 1) >> n); }

// Twiddle tables of one transform length N = 2^n, on one device:
// w^x = hi[x >> h] lo[x & (2^h - 1)] with w = root(n) (fwd) or its inverse.
struct NttTables {
    u64* fwd_lo = nullptr;
    u64* fwd_hi = nullptr;
    u64* inv_lo = nullptr;
    u64* inv_hi = nullptr;
    int h = 0;
    u64 ninv = 0;   // N^-1 mod p
};

static std::mutex g_tab_mu;
static std::map<std::pair<int, int>, NttTables> g_tabs;  // (device, n)

static cudaError_t ntt_tables(int n, NttTables* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_tab_mu);
    auto it = g_tabs.find({dev, n});
    if (it != g_tabs.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    NttTables t;
    t.h = (n + 1) / 2;
    const size_t nlo = (size_t)1 << t.h, nhi = (size_t)1 << (n - t.h);
    const u64 w = h_root(n), wi = h_pow(w, GL_P - 2);
    std::vector<u64> buf(2 * (nlo + nhi));
    for (int dir = 0; dir < 2; ++dir) {
        const u64 base = dir ? wi : w;
        u64* lo = buf.data() + dir * (nlo + nhi);
        u64* hi = lo + nlo;
        u64 x = 1;
        for (size_t i = 0; i < nlo; ++i) { lo[i] = x; x = h_mul(x, base); }
        const u64 step = x;  // base^(2^h)
        x = 1;
        for (size_t i = 0; i < nhi; ++i) { hi[i] = x; x = h_mul(x, step); }
    }
    u64* d = nullptr;
    e = cudaMalloc(&d, buf.size() * 8);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(d, buf.data(), buf.size() * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return e;
    }
    t.fwd_lo = d;
    t.fwd_hi = d + nlo;
    t.inv_lo = d + nlo + nhi;
    t.inv_hi = t.inv_lo + nlo;
    t.ninv = h_pow((u64)1 << n, GL_P - 2);
    g_tabs[{dev, n}] = t;
    *out = t;
    return cudaSuccess;
}

// ---------------------------------------------------------------- kernels

struct NttPassArgs {
    u64* X;          // the whole batch: P transforms of N points, back to back
    long cols;       // columns of the pass over the batch: P N / R
    int n, m, k;     // N = 2^n; blocks of M = 2^m points; R = 2^k-point sub-transforms
    const u64* tlo;  // two-level table of w^x (w = the N-th root, or its inverse)
    const u64* thi;
    int h;
};

__device__ __forceinline__ u64 root_pow(const NttPassArgs& a, unsigned x) {
    return gl_mul(a.thi[x >> a.h], a.tlo[x & ((1u << a.h) - 1)]);
}

// One pass: for each column (block Bg, column sigma) the R points
// Bg M + r S + sigma (S = M / R) are transformed along r.  Forward: radix-2
// decimation in frequency (result for frequency kappa at r = bitrev(kappa)),
// then the point at (r, sigma) is multiplied by w_M^(sigma kappa).  Inverse:
// multiplied by w_M^(-sigma kappa) first, then radix-2 decimation in time back
// to natural order (the sub-transform's factor R is removed by N^-1 later).
template <bool INV>
__global__ void __launch_bounds__(NTT_THREADS)
ntt_pass_kernel(NttPassArgs a) {
    extern __shared__ u64 sm[];
    const int R = 1 << a.k, C = NTT_TILE >> a.k, pitch = C + 1;
    const int ms = a.m - a.k;                     // log2 S
    const long S = 1L << ms;
    u64* wr = sm;                                 // w_R^t, t < R / 2 (forward or inverse)
    u64* sx = sm + (R / 2 > 0 ? R / 2 : 1);       // [R][pitch]
    const long gc0 = (long)blockIdx.x * C;
    const int tid = threadIdx.x;
    const unsigned rstep = 1u << (a.n - a.k);     // w_R = w^(N/R)
    for (int t = tid; t < R / 2; t += NTT_THREADS) wr[t] = root_pow(a, (unsigned)t * rstep);
    // load the tile, coalesced: C consecutive columns of one block (S >= C), or
    // C / S whole consecutive blocks (S < C)
    for (int idx = tid; idx < NTT_TILE; idx += NTT_THREADS) {
        int r, c;
        if (S >= C) {
            r = idx / C;
            c = idx - r * C;
        } else {
            const int blk = idx >> a.m, rem = idx & ((1 << a.m) - 1);
            r = rem >> ms;
            c = blk * (int)S + (rem & (int)(S - 1));
        }
        const long gc = gc0 + c;
        u64 v = 0;
        if (gc < a.cols) {
            const long pos = ((gc >> ms) << a.m) + ((long)r << ms) + (gc & (S - 1));
            v = a.X[pos];
        }
        sx[r * pitch + c] = v;
    }
    __syncthreads();
    auto twiddle = [&](bool inv) {
        if (S == 1) return;                        // sigma = 0: every factor is 1
        const unsigned sh = (unsigned)(a.n - a.m);  // w_M = w^(N/M)
        for (int idx = tid; idx < NTT_TILE; idx += NTT_THREADS) {
            const int r = idx / C, c = idx - r * C;
            const long sigma = (gc0 + c) & (S - 1);
            const unsigned kappa = __brev((unsigned)r) >> (32 - a.k);
            const unsigned x = (unsigned)((sigma * kappa) << sh);  // < N
            if (x) {
                const u64 w = root_pow(a, x);
                sx[r * pitch + c] = gl_mul(sx[r * pitch + c], w);
            }
        }
        (void)inv;
        __syncthreads();
    };
    const int nbf = (R / 2) * C;
    if (!INV) {
        for (int s = a.k - 1; s >= 0; --s) {
            const int hs = 1 << s;
            for (int bf = tid; bf < nbf; bf += NTT_THREADS) {
                const int q = bf / C, c = bf - q * C;
                const int j = q & (hs - 1);
                const int r0 = ((q >> s) << (s + 1)) + j, r1 = r0 + hs;
                const u64 x = sx[r0 * pitch + c], y = sx[r1 * pitch + c];
                sx[r0 * pitch + c] = gl_add(x, y);
                sx[r1 * pitch + c] = gl_mul(gl_sub(x, y), wr[j << (a.k - 1 - s)]);
            }
            __syncthreads();
        }
        twiddle(false);
    } else {
        twiddle(true);
        for (int s = 0; s < a.k; ++s) {
            const int hs = 1 << s;
            for (int bf = tid; bf < nbf; bf += NTT_THREADS) {
                const int q = bf / C, c = bf - q * C;
                const int j = q & (hs - 1);
                const int r0 = ((q >> s) << (s + 1)) + j, r1 = r0 + hs;
                const u64 x = sx[r0 * pitch + c];
                const u64 y = gl_mul(sx[r1 * pitch + c], wr[j << (a.k - 1 - s)]);
                sx[r0 * pitch + c] = gl_add(x, y);
                sx[r1 * pitch + c] = gl_sub(x, y);
            }
            __syncthreads();
        }
    }
    for (int idx = tid; idx < NTT_TILE; idx += NTT_THREADS) {
        int r, c;
        if (S >= C) {
            r = idx / C;
            c = idx - r * C;
        } else {
            const int blk = idx >> a.m, rem = idx & ((1 << a.m) - 1);
            r = rem >> ms;
            c = blk * (int)S + (rem & (int)(S - 1));
        }
        const long gc = gc0 + c;
        if (gc < a.cols) {
            const long pos = ((gc >> ms) << a.m) + ((long)r << ms) + (gc & (S - 1));
            a.X[pos] = sx[r * pitch + c];
        }
    }
}

// Digit vectors: point i of product p is digit i (16 bits) of row p, zero from 2s on.
__global__ void ntt_digits_kernel(const u32* A, long lda, int s, u64* X, int n, long P) {
    const long N = 1L << n;
    const long total = P * N;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
         i += (long)gridDim.x * blockDim.x) {
        const long p = i >> n;
        const long d = i & (N - 1);
        u64 v = 0;
        if (d < 2L * s) {
            const u32 limb = A[p * lda + (d >> 1)];
            v = (d & 1) ? (limb >> 16) : (limb & 0xFFFFu);
        }
        X[i] = v;
    }
}

// Z = X Y N^-1 pointwise (Y == X: squares).
__global__ void ntt_pointwise_kernel(u64* X, const u64* Y, long total, u64 ninv) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
         i += (long)gridDim.x * blockDim.x)
        X[i] = gl_mul(gl_mul(X[i], Y[i]), ninv);
}

// Column sum of output limb j (coefficient c_k at bit 16 k, c_k < 2^56).
__device__ __forceinline__ u64 ntt_column(const u64* Z, long j, long ncoef) {
    auto c = [&](long k) -> u64 { return (k >= 0 && k < ncoef) ? Z[k] : 0ull; };
    const long e = 2 * j;
    return (c(e) & 0xFFFFFFFFull) + (c(e - 2) >> 32) + ((c(e + 1) & 0xFFFFull) << 16) +
           ((c(e - 1) >> 16) & 0xFFFFFFFFull) + (c(e - 3) >> 48);
}

// Carry, pass 1: one warp per segment of CARRY_SEG output limbs, normalised
// with carry-in 0; flags[seg] = generate | propagate << 1 (propagate: every
// limb of the segment is 2^32 - 1, so a carry-in passes through).
__global__ void ntt_carry_kernel(const u64* Zall, int n, u32* OUT, long ldo, int out_len,
                                 int nseg, long P, uint8_t* flags) {
    const long w = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    if (w >= P * nseg) return;
    const long p = w / nseg;
    const int seg = (int)(w - p * nseg);
    const u64* Z = Zall + (p << n);
    const long ncoef = 1L << n;
    u32* out = OUT + p * ldo;
    const int lane = lane_id();
    const int start = seg * CARRY_SEG, end = min(start + CARRY_SEG, out_len);
    UnsignedNorm st{start > 0 ? (ntt_column(Z, start - 1, ncoef) >> 32) : 0ull, 0u};
    bool ones = true;
    for (int base = start; base < end; base += CH) {
        const int l0 = base + 4 * lane;
        u64 cols[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) cols[j] = l0 + j < end ? ntt_column(Z, l0 + j, ncoef) : 0ull;
        u32 d[4];
        warp_norm_unsigned(cols, st, d);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (l0 + j < end) {
                out[l0 + j] = d[j];
                ones = ones && d[j] == 0xFFFFFFFFu;
            }
    }
    ones = __all_sync(FULL, ones);
    if (lane == 0) flags[w] = (uint8_t)((st.carry ? 1 : 0) | (ones ? 2 : 0));
}

// Carry, pass 2: the carry into each segment from the flags of the segments
// below it (the nearest one that generates or does not propagate decides),
// added by a ripple from the segment's first limb.
__global__ void ntt_carry_fix_kernel(u32* OUT, long ldo, int out_len, int nseg, long P,
                                     const uint8_t* flags) {
    const long w = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    if (w >= P * nseg) return;
    const long p = w / nseg;
    const int seg = (int)(w - p * nseg);
    if (seg == 0) return;
    const int lane = lane_id();
    const uint8_t* f = flags + p * nseg;
    u32 cin = 0;
    for (int hi = seg - 1; hi >= 0; hi -= 32) {
        const int i = hi - lane;
        const uint8_t v = i >= 0 ? f[i] : (uint8_t)1;  // below segment 0: no carry (decides 0)
        const bool decides = i < 0 || (v & 1) || !(v & 2);
        const unsigned m = __ballot_sync(FULL, decides);
        if (m) {
            const int first = __ffs(m) - 1;           // nearest deciding segment
            const int src = hi - first;
            cin = (src >= 0) ? (f[src] & 1) : 0u;
            break;
        }
    }
    if (!cin) return;
    u32* out = OUT + p * ldo;
    const int start = seg * CARRY_SEG, end = min(start + CARRY_SEG, out_len);
    for (int base = start; base < end; base += CH) {
        const int l0 = base + 4 * lane;
        u32 d[4];
        bool ones = true;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            d[j] = l0 + j < end ? out[l0 + j] : 0u;
            ones = ones && (l0 + j >= end || d[j] == 0xFFFFFFFFu);
        }
        // lanes below the first limb that is not 2^32 - 1 wrap to 0; that limb gets + 1
        const unsigned notall = __ballot_sync(FULL, !ones);
        const int stop = notall ? __ffs(notall) - 1 : 32;
        if (lane < stop) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (l0 + j < end) out[l0 + j] = 0u;
        } else if (lane == stop) {
            u32 c = 1;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (l0 + j < end && c) {
                    out[l0 + j] = d[j] + 1;
                    c = d[j] == 0xFFFFFFFFu ? 1u : 0u;
                }
            }
        }
        if (notall) break;
    }
}

// ---------------------------------------------------------------- launch

int ntt_log2(int s) {
    int n = 1;
    while ((1L << n) < 4L * s) ++n;
    return n;
}

static std::vector<int> ntt_fields(int n) {
    const int r = (n + NTT_KMAX - 1) / NTT_KMAX;
    std::vector<int> k(r, n / r);
    for (int i = 0; i < n % r; ++i) ++k[i];
    return k;
}

size_t ntt_work_bytes(int s, long P, bool square) {
    const int n = ntt_log2(s);
    const size_t pts = (size_t)P << n;
    const int nseg = (2 * s + CARRY_SEG - 1) / CARRY_SEG;
    return (square ? 1 : 2) * pts * 8 + (((size_t)P * nseg + 255) / 256) * 256;
}

static cudaError_t run_passes(u64* X, long P, int n, const NttTables& t, bool inv, cudaStream_t st) {
    const std::vector<int> ks = ntt_fields(n);
    std::vector<int> ms(ks.size());
    int m = n;
    for (size_t j = 0; j < ks.size(); ++j) {
        ms[j] = m;
        m -= ks[j];
    }
    static std::once_flag attr;
    std::call_once(attr, [] {
        const int smem = (NTT_TILE / 2 + 1) * 8 + (NTT_TILE + (1 << NTT_KMAX)) * 8;
        cudaFuncSetAttribute(ntt_pass_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(ntt_pass_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    for (size_t q = 0; q < ks.size(); ++q) {
        const size_t j = inv ? ks.size() - 1 - q : q;
        NttPassArgs a;
        a.X = X;
        a.n = n;
        a.m = ms[j];
        a.k = ks[j];
        a.cols = (P << n) >> ks[j];
        a.tlo = inv ? t.inv_lo : t.fwd_lo;
        a.thi = inv ? t.inv_hi : t.fwd_hi;
        a.h = t.h;
        const int R = 1 << a.k, C = NTT_TILE / R;
        const size_t smem = (size_t)(R / 2 > 0 ? R / 2 : 1) * 8 + (size_t)R * (C + 1) * 8;
        const unsigned grid = (unsigned)((a.cols + C - 1) / C);
        if (inv) ntt_pass_kernel<true><<<grid, NTT_THREADS, smem, st>>>(a);
        else ntt_pass_kernel<false><<<grid, NTT_THREADS, smem, st>>>(a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static unsigned flat_grid(long items, int threads) {
    const long b = (items + threads - 1) / threads;
    return (unsigned)std::max<long>(1, std::min<long>(b, 152L * 64));
}

// P products of s x s limbs (rows of A and Bm), 2s-limb results at OUT + p ldo.
cudaError_t launch_ntt_mul(const u32* A, long lda, const u32* Bm, long ldb, u32* OUT, long ldo,
                           int s, long P, bool square, void* work, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    note_kernel("ntt passes");
    const int n = ntt_log2(s);
    NttTables t;
    cudaError_t e = ntt_tables(n, &t);
    if (e != cudaSuccess) return e;
    const long total = P << n;
    u64* X = static_cast<u64*>(work);
    u64* Y = square ? X : X + total;
    uint8_t* flags = reinterpret_cast<uint8_t*>(X + (square ? 1 : 2) * total);
    ntt_digits_kernel<<<flat_grid(total, 256), 256, 0, st>>>(A, lda, s, X, n, P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = run_passes(X, P, n, t, false, st)) != cudaSuccess) return e;
    if (!square) {
        ntt_digits_kernel<<<flat_grid(total, 256), 256, 0, st>>>(Bm, ldb, s, Y, n, P);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = run_passes(Y, P, n, t, false, st)) != cudaSuccess) return e;
    }
    ntt_pointwise_kernel<<<flat_grid(total, 256), 256, 0, st>>>(X, Y, total, t.ninv);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = run_passes(X, P, n, t, true, st)) != cudaSuccess) return e;
    const int out_len = 2 * s;
    const int nseg = (out_len + CARRY_SEG - 1) / CARRY_SEG;
    const long warps = P * nseg;
    const unsigned grid = (unsigned)((warps * 32 + 255) / 256);
    ntt_carry_kernel<<<grid, 256, 0, st>>>(X, n, OUT, ldo, out_len, nseg, P, flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (nseg > 1) {
        ntt_carry_fix_kernel<<<grid, 256, 0, st>>>(OUT, ldo, out_len, nseg, P, flags);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace tc

using namespace tc;

extern "C" size_t tc_ntt_work_bytes(size_t count, size_t limbs) {
    if (limbs == 0 || limbs > ((size_t)1 << 24)) return 0;
    return ntt_work_bytes((int)limbs, (long)count, false);
}

extern "C" tc_status tc_ntt_mul(size_t count, size_t limbs, const uint32_t* A, size_t lda,
                                const uint32_t* Bv, size_t ldb, uint32_t* OUT, size_t ldo,
                                void* work, void* stream) {
    if (count == 0) return TC_OK;
    if (!A || !Bv || !OUT || !work || limbs == 0 || limbs > ((size_t)1 << 24)) return TC_EINVAL;
    if (count > 1 && (lda < limbs || ldb < limbs || ldo < 2 * limbs)) return TC_EINVAL;
    if (reinterpret_cast<uintptr_t>(work) & 15u) return TC_EINVAL;
    const bool square = A == Bv && lda == ldb;
    const cudaError_t e = launch_ntt_mul(A, (long)lda, Bv, (long)ldb, OUT, (long)ldo, (int)limbs,
                                         (long)count, square, work, (cudaStream_t)stream);
    return e == cudaSuccess ? TC_OK : tc_fail_cuda(e);
}

extern "C" tc_status tc_ntt_root(int log2n, uint64_t* root) {
    if (log2n < 0 || log2n > 32 || !root) return TC_EINVAL;
    *root = h_root(log2n);
    return TC_OK;
}
