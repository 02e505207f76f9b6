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
// four-step decomposition over fields of the point index (at most 6 bits,
// 64 points, per pass): each pass runs, for every column of a block, a
// radix-2 transform of one field (staged in shared memory, its stages in
// registers) and multiplies the results by the four-step twiddles.  The
// transform's root is chosen so that the roots of order <= 64 are powers of 2
// (see h_root): the sub-transforms multiply by shifts only.  Forward
// passes go from the top field down and leave the spectrum in a fixed permuted
// order; the inverse passes undo them in reverse order, so no reordering pass
// is needed.  The first forward pass reads the digits straight from the limbs
// and the second operand's last forward pass multiplies by the first
// operand's spectrum (the pointwise product).  The coefficients c_k are then
// placed at bit 16k and carried into 2s limbs.
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
constexpr int NTT_KMAX = 6;          // largest field (64-point sub-transforms: shifts only)
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

// (hi 2^64 + lo) mod p, any hi and lo.
__device__ __forceinline__ u64 gl_reduce(u64 lo, u64 hi) {
    const u64 hh = hi >> 32, hl = hi & 0xFFFFFFFFull;
    u64 t = lo - hh;                      // lo - hh 2^96 with 2^96 = -1
    if (lo < hh) t -= 0xFFFFFFFFull;      // borrow: + p
    const u64 u = (hl << 32) - hl;        // hl 2^64 with 2^64 = 2^32 - 1
    u64 r = t + u;
    if (r < u) r += 0xFFFFFFFFull;        // carry: + 2^64 = + (2^32 - 1)
    return r >= GL_P ? r - GL_P : r;
}

// a 2^e mod p for 0 <= e < 96, by shifts: 2^e for e >= 64 is 2^(e-64) 2^64 =
// 2^(e-32) - 2^(e-64) (mod p).
__device__ __forceinline__ u64 gl_shl(u64 a, unsigned e) {  // e < 64
    return e ? gl_reduce(a << e, a >> (64 - e)) : a;
}
__device__ __forceinline__ u64 gl_mul_pow2(u64 a, unsigned e) {
    if (e < 64) return gl_shl(a, e);
    const u64 x = gl_shl(a, e - 32), y = gl_shl(a, e - 64);
    return x >= y ? x - y : x - y + GL_P;
}
// a 2^-e mod p for 0 <= e < 96: 2^-e = 2^(192 - e) = -2^(96 - e).
__device__ __forceinline__ u64 gl_mul_pow2_inv(u64 a, unsigned e) {
    if (!e) return a;
    const u64 x = gl_mul_pow2(a, 96 - e);
    return x ? GL_P - x : 0;
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

// The primitive 2^n-th root of unity the transform uses.  8 = 2^3 has order
// 64 modulo p (2^96 = -1), so the root is chosen with w^(2^n / 64) = 8: then
// every root of unity of order <= 64 is a power of 2 and the sub-transforms of
// at most 64 points multiply by shifts only.  For n >= 6 it is the power of
// w0 = g^((p-1) / 2^n) (g = 7 generates the multiplicative group) whose
// (2^n / 64)-th power is 8; for n < 6 it is 8^(64 / 2^n).
static u64 h_root(int n) {
    if (n < 6) return h_pow(8, (u64)64 >> n);
    const u64 w0 = h_pow(7, (GL_P - 1) >> n);
    const u64 t = h_pow(w0, (u64)1 << (n - 6));  // a primitive 64th root: 8^j for one odd j
    u64 pw = 8;
    int j = 1;
    while (pw != t && j < 64) {
        pw = h_mul(pw, 64);  // 8^(j + 2)
        j += 2;
    }
    // w0^(j^-1 mod 2^n): its (2^n / 64)-th power is t^(j^-1) = 8
    u64 inv = 1;  // j^-1 mod 2^n by Newton's iteration (j odd)
    for (int i = 0; i < 6; ++i) inv *= 2 - (u64)j * inv;
    inv &= n >= 64 ? ~0ull : (((u64)1 << n) - 1);
    return h_pow(w0, inv);
}

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
    int n, m;        // N = 2^n; blocks of M = 2^m points
    const u64* tlo;  // two-level table of w^x (w = the N-th root, or its inverse)
    const u64* thi;
    int h;
    // optional fusions
    const u32* limbs;  // first forward pass: points are the 16-bit digits of these rows
    long lda;
    int s;             // limbs per row (digits 2s, zero beyond)
    const u64* mulby;  // last forward pass: outputs multiplied by mulby[pos] and by ninv
    int square;        // last forward pass: outputs squared and multiplied by ninv
    u64 ninv;
};

__device__ __forceinline__ u64 root_pow(const NttPassArgs& a, unsigned x) {
    return gl_mul(a.thi[x >> a.h], a.tlo[x & ((1u << a.h) - 1)]);
}

// One pass: for each column (block Bg, column sigma) the R = 2^K points
// Bg M + r S + sigma (S = M / R) are transformed along r.  Forward: radix-2
// decimation in frequency (the result for frequency kappa at r = bitrev(kappa)),
// then the point at (r, sigma) is multiplied by w_M^(sigma kappa).  Inverse:
// multiplied by w_M^(-sigma kappa) first, then radix-2 decimation in time back
// to natural order (the factor R is removed by N^-1 at the pointwise product).
// The tile (4096 points: R rows x C columns) is staged in shared memory; each
// thread runs the stages of one half of the index bits in registers: round 1
// the high stages on groups of 2^K1 points strided by 2^K2, round 2 the low
// stages on groups of 2^K2 consecutive points (K = K1 + K2).
template <bool INV, int K>
__global__ void __launch_bounds__(NTT_THREADS)
ntt_pass_kernel(NttPassArgs a) {
    constexpr int R = 1 << K, C = NTT_TILE >> K, PITCH = C + 1;
    constexpr int K1 = (K + 1) / 2, K2 = K / 2;
    constexpr int G1 = 1 << K1, G2 = 1 << K2;
    constexpr int NG1 = NTT_TILE / G1 / NTT_THREADS, NG2 = NTT_TILE / G2 / NTT_THREADS;
    static_assert(K <= 6, "sub-transform roots are powers of 2 up to 64 points");
    extern __shared__ u64 sx[];                  // [R][PITCH]
    const int ms = a.m - K;                      // log2 S
    const long S = 1L << ms;
    const long gc0 = (long)blockIdx.x * C;
    const int tid = threadIdx.x;
    const long N = 1L << a.n;
    // coalesced tile order: C consecutive columns of one block (S >= C), or C / S
    // whole consecutive blocks (S < C)
    auto tile_rc = [&](int idx, int& r, int& c) {
        if (S >= C) {
            r = idx / C;
            c = idx - r * C;
        } else {
            const int blk = idx >> a.m, rem = idx & ((1 << a.m) - 1);
            r = rem >> ms;
            c = blk * (int)S + (rem & (int)(S - 1));
        }
    };
    // every load of the tile in flight before the first store to shared memory
    constexpr int PER = NTT_TILE / NTT_THREADS;
    u64 lv[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        int r, c;
        tile_rc(tid + NTT_THREADS * q, r, c);
        const long gc = gc0 + c;
        u64 v = 0;
        if (gc < a.cols) {
            const long pos = ((gc >> ms) << a.m) + ((long)r << ms) + (gc & (S - 1));
            if (a.limbs) {
                const long pr = pos >> a.n, d = pos & (N - 1);
                if (d < 2L * a.s) {
                    const u32 limb = a.limbs[pr * a.lda + (d >> 1)];
                    v = (d & 1) ? (limb >> 16) : (limb & 0xFFFFu);
                }
            } else {
                v = a.X[pos];
            }
        }
        lv[q] = v;
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        int r, c;
        tile_rc(tid + NTT_THREADS * q, r, c);
        sx[r * PITCH + c] = lv[q];
    }
    __syncthreads();
    // four-step twiddle of the points (r, c) of a round-2 group
    auto twiddle = [&](u64 v[G2], int hi, int c) {
        if (S == 1) return;                      // sigma = 0: every factor is 1
        const long sigma = (gc0 + c) & (S - 1);
        const unsigned sh = (unsigned)(a.n - a.m);  // w_M = w^(N/M)
#pragma unroll
        for (int i = 0; i < G2; ++i) {
            const unsigned kappa = __brev((unsigned)(G2 * hi + i)) >> (32 - K);
            const unsigned x = (unsigned)((sigma * kappa) << sh);  // < N
            if (x) v[i] = gl_mul(v[i], root_pow(a, x));
        }
    };
    auto round1 = [&]() {  // stages K-1 .. K2 on groups of G1 points strided by G2
#pragma unroll
        for (int q = 0; q < NG1; ++q) {
            const int gid = tid + NTT_THREADS * q;
            const int c = gid % C, lo = gid / C;
            u64 v[G1];
#pragma unroll
            for (int i = 0; i < G1; ++i) v[i] = sx[(lo + G2 * i) * PITCH + c];
            if (!INV) {
#pragma unroll
                for (int s = K - 1; s >= K2; --s) {
                    const int di = 1 << (s - K2);
#pragma unroll
                    for (int i0 = 0; i0 < G1; ++i0) {
                        if (i0 & di) continue;
                        const int j = lo + G2 * (i0 & (di - 1));
                        const u64 x = v[i0], y = v[i0 + di];
                        v[i0] = gl_add(x, y);
                        v[i0 + di] = gl_mul_pow2(gl_sub(x, y), (unsigned)(3 * j) << (5 - s));
                    }
                }
            } else {
#pragma unroll
                for (int s = K2; s <= K - 1; ++s) {
                    const int di = 1 << (s - K2);
#pragma unroll
                    for (int i0 = 0; i0 < G1; ++i0) {
                        if (i0 & di) continue;
                        const int j = lo + G2 * (i0 & (di - 1));
                        const u64 x = v[i0], y = gl_mul_pow2_inv(v[i0 + di], (unsigned)(3 * j) << (5 - s));
                        v[i0] = gl_add(x, y);
                        v[i0 + di] = gl_sub(x, y);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < G1; ++i) sx[(lo + G2 * i) * PITCH + c] = v[i];
        }
    };
    auto round2 = [&]() {  // stages K2-1 .. 0 on groups of G2 consecutive points
#pragma unroll
        for (int q = 0; q < NG2; ++q) {
            const int gid = tid + NTT_THREADS * q;
            const int c = gid % C, hi = gid / C;
            u64 v[G2];
#pragma unroll
            for (int i = 0; i < G2; ++i) v[i] = sx[(G2 * hi + i) * PITCH + c];
            if (!INV) {
#pragma unroll
                for (int s = K2 - 1; s >= 0; --s) {
                    const int di = 1 << s;
#pragma unroll
                    for (int i0 = 0; i0 < G2; ++i0) {
                        if (i0 & di) continue;
                        const int j = i0 & (di - 1);
                        const u64 x = v[i0], y = v[i0 + di];
                        v[i0] = gl_add(x, y);
                        v[i0 + di] = gl_mul_pow2(gl_sub(x, y), (unsigned)(3 * j) << (5 - s));
                    }
                }
                twiddle(v, hi, c);
            } else {
                twiddle(v, hi, c);
#pragma unroll
                for (int s = 0; s < K2; ++s) {
                    const int di = 1 << s;
#pragma unroll
                    for (int i0 = 0; i0 < G2; ++i0) {
                        if (i0 & di) continue;
                        const int j = i0 & (di - 1);
                        const u64 x = v[i0], y = gl_mul_pow2_inv(v[i0 + di], (unsigned)(3 * j) << (5 - s));
                        v[i0] = gl_add(x, y);
                        v[i0 + di] = gl_sub(x, y);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < G2; ++i) sx[(G2 * hi + i) * PITCH + c] = v[i];
        }
    };
    if (!INV) {
        round1();
        __syncthreads();
        round2();
    } else {
        round2();
        __syncthreads();
        round1();
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        int r, c;
        tile_rc(tid + NTT_THREADS * q, r, c);
        const long gc = gc0 + c;
        if (gc < a.cols) {
            const long pos = ((gc >> ms) << a.m) + ((long)r << ms) + (gc & (S - 1));
            u64 v = sx[r * PITCH + c];
            if (a.mulby) v = gl_mul(gl_mul(v, a.mulby[pos]), a.ninv);
            else if (a.square) v = gl_mul(gl_mul(v, v), a.ninv);
            a.X[pos] = v;
        }
    }
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

template <bool INV>
static cudaError_t launch_pass(const NttPassArgs& a, int k, cudaStream_t st) {
    const int R = 1 << k, C = NTT_TILE / R;
    const size_t smem = (size_t)R * (C + 1) * 8;
    const unsigned grid = (unsigned)((a.cols + C - 1) / C);
    switch (k) {
#define TC_NTT_PASS(KK)                                                           \
    case KK:                                                                      \
        ntt_pass_kernel<INV, KK><<<grid, NTT_THREADS, smem, st>>>(a);             \
        break;
        TC_NTT_PASS(1) TC_NTT_PASS(2) TC_NTT_PASS(3) TC_NTT_PASS(4)
        TC_NTT_PASS(5) TC_NTT_PASS(6)
#undef TC_NTT_PASS
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The passes of one forward (top field first) or inverse (bottom field first)
// transform of P x 2^n points.  `limbs`: the first forward pass reads the
// digits of these rows; `mulby`: the last forward pass multiplies its outputs
// by mulby and N^-1 (the pointwise product); `square`: by themselves and N^-1.
static cudaError_t run_passes(u64* X, long P, int n, const NttTables& t, bool inv, const u32* limbs,
                              long lda, int s, const u64* mulby, bool square, cudaStream_t st) {
    const std::vector<int> ks = ntt_fields(n);
    std::vector<int> ms(ks.size());
    int m = n;
    for (size_t j = 0; j < ks.size(); ++j) {
        ms[j] = m;
        m -= ks[j];
    }
    for (size_t q = 0; q < ks.size(); ++q) {
        const size_t j = inv ? ks.size() - 1 - q : q;
        NttPassArgs a;
        a.X = X;
        a.n = n;
        a.m = ms[j];
        a.cols = (P << n) >> ks[j];
        a.tlo = inv ? t.inv_lo : t.fwd_lo;
        a.thi = inv ? t.inv_hi : t.fwd_hi;
        a.h = t.h;
        a.limbs = (!inv && q == 0) ? limbs : nullptr;
        a.lda = lda;
        a.s = s;
        const bool last_fwd = !inv && q + 1 == ks.size();
        a.mulby = last_fwd ? mulby : nullptr;
        a.square = last_fwd && square ? 1 : 0;
        a.ninv = t.ninv;
        const cudaError_t e = inv ? launch_pass<true>(a, ks[j], st) : launch_pass<false>(a, ks[j], st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
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
    // X = transform of a's digits; Y = transform of b's digits, multiplied by X and
    // N^-1 in its last pass (squares: X times itself); then the inverse of Y
    u64* Z = square ? X : Y;
    if ((e = run_passes(X, P, n, t, false, A, lda, s, nullptr, square, st)) != cudaSuccess) return e;
    if (!square && (e = run_passes(Y, P, n, t, false, Bm, ldb, s, X, false, st)) != cudaSuccess)
        return e;
    if ((e = run_passes(Z, P, n, t, true, nullptr, 0, s, nullptr, false, st)) != cudaSuccess) return e;
    const int out_len = 2 * s;
    const int nseg = (out_len + CARRY_SEG - 1) / CARRY_SEG;
    const long warps = P * nseg;
    const unsigned grid = (unsigned)((warps * 32 + 255) / 256);
    ntt_carry_kernel<<<grid, 256, 0, st>>>(Z, n, OUT, ldo, out_len, nseg, P, flags);
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
