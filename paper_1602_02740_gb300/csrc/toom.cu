// One Toom-Cook level on the GPU: evaluation, interpolation, recomposition.
//
// Level geometry (all lengths in 32-bit limbs): operands of s limbs are cut
// into B blocks of b = ceil(s/B) limbs (Section 1, eq. 1.1-1.3; the top block
// is zero-padded).  Evaluation values have e = b + ceil((n(n-1)+1)/32) limbs,
// pointwise products 2e limbs, and interpolation values Y >= 2e + 2 limbs.
//
// Points (Section 6): x = 0 and x = +-2^j, j = 0..n-1, stored in the order
// 0, +1, -1, +2, -2, ...; signed values are sign-magnitude.
#include <cstring>
#include <mutex>
#include <vector>

#include "tc_device.cuh"
#include "tc_internal.h"

namespace tc {

thread_local const char* g_kernel_name = "";

LevelGeom make_level(int s, int B) {
    LevelGeom g;
    g.B = B;
    g.n = B - 1;
    g.s = s;
    g.b = (s + B - 1) / B;
    g.e = g.b + (g.n * (g.n - 1) + 1 + 31) / 32;
    g.estride = (g.e + 3) / 4 * 4;
    g.ystride = (2 * g.e + 3) / 4 * 4;
    const int need = 2 * g.e + 2;
    g.K = need > 1536 ? 8 : 4;  // limbs per lane in interpolation passes
    g.Y = (need + 32 * g.K - 1) / (32 * g.K) * (32 * g.K);
    return g;
}

// ===========================================================================
// Evaluation (Section 4, eq. 4.1-4.2).
//
// For x = 2^j the even part E = sum_{i even} u_i 2^(j i) and the odd part
// O = sum_{i odd} u_i 2^(j i) are formed column by column (each block shifted
// by j i bits), then U(x) = E + O and |U(-x)| = |E - O|.  The sign of E - O
// is decided first by a scan from the top limb down (it almost always
// settles on the first limb), so the magnitude is produced in one bottom-up
// pass with no negation afterwards.  Warp j handles x = 2^j.
// ===========================================================================

__device__ __forceinline__ u32 blk(const u32* row, int s, int b, int i, int x) {
    const int g = i * b + x;
    return (x >= 0 && x < b && g < s) ? __ldg(row + g) : 0u;
}

// Column sums of E and O at output limb l for x = 2^j.
__device__ __forceinline__ void eval_cols(const u32* row, int s, int B, int b, int j, int l,
                                          i64& E, i64& O) {
    u64 e = 0, o = 0;
    for (int i = 0; i < B; ++i) {
        const int sh = j * i;
        const int qa = sh >> 5, r = sh & 31;
        const u32 hi = blk(row, s, b, i, l - qa);
        const u32 lo = blk(row, s, b, i, l - qa - 1);
        const u32 t = fshl(lo, hi, (u32)r);
        if (i & 1) o += t; else e += t;
    }
    E = (i64)e;
    O = (i64)o;
}

struct EvalCarry {
    u32 minus;  // borrow of |E - O| into this chunk
    u32 dtop;   // top limb of O in the previous chunk (the bit that 2 O shifts in)
};

// Column sums e, o (non-negative) of one chunk -> digits of U(x) = E + O and of
// |U(-x)| = sign (E - O).  E + O is normalised directly; |E - O| is
// (E + O) - 2 O (sign > 0) or 2 O - (E + O) (sign < 0), so only O is normalised
// besides, and one borrow scan finishes.
__device__ __forceinline__ void eval_finish(const u64 e[4], const u64 o[4], int sign,
                                            UnsignedNorm& np, UnsignedNorm& no, EvalCarry& c,
                                            u32 dp[4], u32 dm[4]) {
    u64 s[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = e[j] + o[j];
    warp_norm_unsigned(s, np, dp);
    u32 O[4];
    warp_norm_unsigned(o, no, O);
    const u32 up = __shfl_up_sync(FULL, O[3], 1);
    const u32 below = lane_id() == 0 ? c.dtop : up;
    u32 O2[4];
    O2[0] = fshl(below, O[0], 1);
#pragma unroll
    for (int j = 1; j < 4; ++j) O2[j] = fshl(O[j - 1], O[j], 1);
    c.dtop = __shfl_sync(FULL, O[3], 31);
    if (sign > 0) warp_sub_seg<4>(dp, O2, c.minus, dm);
    else warp_sub_seg<4>(O2, dp, c.minus, dm);
}

// Padded shared-memory index: one spare word per 32 makes the lane pattern
// 4t + c conflict-free.
__host__ __device__ __forceinline__ int pad32(int x) { return x + (x >> 5); }

// Blocks P .. 2P - 1 (when in2 is given) evaluate the second operand's rows into
// out2 / sgn2, so both operands of few products take one launch.
template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
eval_kernel(const u32* __restrict__ in, long in_stride, LevelGeom g, u32* __restrict__ out,
            uint8_t* __restrict__ sgn, long P, const u32* __restrict__ in2, long in2_stride,
            u32* __restrict__ out2, uint8_t* __restrict__ sgn2) {
    extern __shared__ __align__(16) u32 win[];  // [2][B][pad32(CH + W) + 1]
    long k = blockIdx.x;
    if (k >= P) {
        if (!in2 || k >= 2 * P) return;
        k -= P;
        in = in2;
        in_stride = in2_stride;
        out = out2;
        sgn = sgn2;
    }
    const u32* row = in + k * in_stride;
    const int npts = 2 * g.B - 1;
    u32* orow0 = out + (k * npts) * (long)g.estride;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) sgn[k * npts] = 0;

    const int warp = tid >> 5, lane = tid & 31;
    const int j = warp;             // this warp evaluates x = 2^j (blockDim = 32 max(n, 1))
    const bool has_point = j < g.n;
    // Chunks of CH output limbs are staged in shared memory by asynchronous copies,
    // double-buffered: chunk c+1 is in flight while chunk c is summed.
    const int W = ((g.n - 1) * g.n >> 5) + 1;  // halo: largest limb shift + 1
    const int wlen = pad32(CH + W) + 1;
    const int bufw = g.B * wlen;
    // staging map, fixed for the kernel: thread -> window offsets xo (one when the
    // block has a window's width of threads) and blocks i0, i0 + istep, ...
    const int span = CH + W;
    const bool wide_blk = nt >= span;
    const int istep = wide_blk ? nt / span : 1;
    const int xo0 = wide_blk ? tid % span : tid, xstep = wide_blk ? span : nt;
    const int i0 = wide_blk ? tid / span : 0;
    auto stage = [&](int base, u32* buf) {
        if (i0 < istep) {
            for (int xo = xo0; xo < span; xo += xstep) {
                const int x = base - W + xo;  // limb index within each block
                const bool inb = x >= 0 && x < g.b;
                int gi = i0 * g.b + x;
                u32* d = buf + i0 * wlen + pad32(xo);
                for (int i = i0; i < g.B; i += istep, gi += istep * g.b, d += istep * wlen) {
                    if (inb && gi < g.s) cp_async4(d, row + gi);
                    else *d = 0u;
                }
            }
        }
        cp_async_commit();
    };
    stage(0, win);
    // ---- sign of E - O, top-down (global reads; almost always one window) ----
    int sign = 1;
    if (has_point) {
        i64 T = 0;
        sign = 0;
        for (int top = g.e - 1; top >= 0 && sign == 0; top -= 32) {
            const int l = top - lane;
            i64 d = 0;
            if (l >= 0) {
                i64 E, O;
                eval_cols(row, g.s, g.B, g.b, j, l, E, O);
                d = E - O;
            }
            const unsigned nz = __ballot_sync(FULL, d != 0);
            if (T == 0 && nz == 0) continue;
            for (int t = 0; t < 32; ++t) {
                const i64 dt = __shfl_sync(FULL, d, t);
                if (top - t < 0) break;
                T = T * 4294967296LL + dt;
                if (T >= 17) { sign = 1; break; }
                if (T <= -17) { sign = -1; break; }
            }
        }
        if (sign == 0) sign = T < 0 ? -1 : 1;
    }

    // ---- bottom-up pass over the staged chunks ----
    u32* rp = out + (k * npts + 2 * j + 1) * (long)g.estride;
    u32* rm = out + (k * npts + 2 * j + 2) * (long)g.estride;
    UnsignedNorm ne{0, 0}, no{0, 0};
    EvalCarry cpm{0, 0};
    int c = 0;
    for (int base = 0; base < g.estride; base += CH, ++c) {
        const u32* cur = win + (c & 1) * bufw;
        if (base + CH < g.estride) stage(base + CH, win + ((c + 1) & 1) * bufw);
        else cp_async_commit();  // one group per chunk: the wait below is for chunk c
        cp_async_wait_prev();
        __syncthreads();
        // point 0: U(0) = u_0, block 0 of the staged chunk (zero past b and s)
        for (int x = tid; x < CH && base + x < g.estride; x += nt) orow0[base + x] = cur[pad32(W + x)];
        if (has_point) {
            u64 e[4] = {0, 0, 0, 0}, o[4] = {0, 0, 0, 0};
            // block i shifted left by j i bits: limbs x = 4 lane + jj - qa - 1 .. + 0 of
            // block i (window offset W), added into E (i even) or O (i odd)
            auto add_block = [&](int i, u64 acc[4]) {
                const int sh = j * i;
                const int qa = sh >> 5;
                const u32 r = (u32)(sh & 31);
                const u32* w = cur + i * wlen;
                const int x0 = 4 * lane + W - qa - 1;
                u32 v[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) v[q] = w[pad32(x0 + q)];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[jj] += fshl(v[jj], v[jj + 1], r);
            };
            for (int i = 0; i < g.B; i += 2) {
                add_block(i, e);
                if (i + 1 < g.B) add_block(i + 1, o);
            }
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                if (base + 4 * lane + jj >= g.e) { e[jj] = 0; o[jj] = 0; }
            u32 dp[4], dm[4];
            eval_finish(e, o, sign, ne, no, cpm, dp, dm);
            const int pos = base + 4 * lane;
            if (pos < g.estride) {  // estride is a multiple of 4
                st4(rp + pos, dp);
                st4(rm + pos, dm);
            }
        }
        __syncthreads();  // this buffer is staged again two chunks on
    }
    if (has_point && lane == 0) {
        sgn[k * npts + 2 * j + 1] = 0;
        sgn[k * npts + 2 * j + 2] = sign < 0 ? 1 : 0;
    }
}

// Staged block of eval_pts_kernel: limbs x in [-PTS_LO, roundup(estride, CH) + 4)
// (the bottom-up pass reads x in [l0 - 2, l0 + 4) for every lane's l0 below
// roundup(estride, CH); the sign scan x >= -2; shifts j i < 64 bits reach one
// limb further down).
constexpr int PTS_LO = 4;
__host__ __device__ inline int pts_block_words(const LevelGeom& g) {
    return PTS_LO + (g.estride + CH - 1) / CH * CH + 4;
}

// Short rows: one warp per row, every point of the row, the row staged in
// shared memory (padded layout), several rows per block, no block barriers.
// Warp per row for small B (B <= 8, every shift j i < 64 bits): the same staging
// as eval_warp_kernel, but each 128-limb chunk's block limbs are read once and
// serve all points x = 2^j (column sums for every j from the same registers),
// and the top-down sign scans of all points share their loads.
template <int BB>
__global__ void __launch_bounds__(256, BB <= 4 ? 4 : 1)
eval_pts_kernel(const u32* __restrict__ in, long in_stride, LevelGeom g, u32* __restrict__ out,
                uint8_t* __restrict__ sgn, long P, int rowlen) {
    constexpr int N = BB - 1;
    extern __shared__ __align__(16) u32 rows_sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long k = (long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (k >= P) return;  // warp-uniform
    u32* rs = rows_sm + (long)warp * rowlen;
    const u32* row = in + k * in_stride;
    const int npts = 2 * BB - 1;
    // block i is staged as limbs x in [-PTS_LO, bw - PTS_LO), zeros outside [0, b),
    // wide enough for every read below, so reads need no bounds checks
    const int bw = pts_block_words(g);
    // all blocks' limbs of a round are loaded before any is stored, so the global
    // loads of a row are in flight together
    for (int r0 = 0; r0 < bw; r0 += 128) {
        u32 v[BB][4];
#pragma unroll
        for (int i = 0; i < BB; ++i)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int xo = r0 + lane + 32 * u, xi = xo - PTS_LO, gi = i * g.b + xi;
                v[i][u] = (xo < bw && xi >= 0 && xi < g.b && gi < g.s) ? __ldg(row + gi) : 0u;
            }
#pragma unroll
        for (int i = 0; i < BB; ++i)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int xo = r0 + lane + 32 * u;
                if (xo < bw) rs[i * bw + xo] = v[i][u];
            }
    }
    __syncwarp();
    // Unpadded: the scalar reads below are consecutive across lanes, and the
    // bottom-up pass reads each lane's four limbs as one 16-byte vector
    // (bw and PTS_LO are multiples of 4) and the two below from the lane below.
    auto U = [&](int i, int x) -> u32 {  // limb x of block i, -PTS_LO <= x < bw - PTS_LO
        return rs[i * bw + PTS_LO + x];
    };
    auto U4 = [&](int i, int x, u32 v[4]) {  // limbs x .. x + 3 of block i, x a multiple of 4
        const uint4 q = *reinterpret_cast<const uint4*>(rs + i * bw + PTS_LO + x);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    };
    u32* orow0 = out + (k * npts) * (long)g.estride;
    for (int pos = 4 * lane; pos < g.estride; pos += CH) {
        u32 v[4];
        U4(0, pos, v);  // zero past b
        st4(orow0 + pos, v);
    }
    // ---- signs of E - O at every x = 2^j, top-down, loads shared ----
    i64 T[N];
    int sign[N];
#pragma unroll
    for (int j = 0; j < N; ++j) { T[j] = 0; sign[j] = 0; }
    for (int top = g.e - 1; top >= 0; top -= 32) {
        bool open = false;
#pragma unroll
        for (int j = 0; j < N; ++j) open |= sign[j] == 0;
        if (!open) break;
        const int l = top - lane;
        u32 w[BB][3];  // limbs l-2, l-1, l of each block
#pragma unroll
        for (int i = 0; i < BB; ++i) {
            w[i][0] = l >= 0 ? U(i, l - 2) : 0u;
            w[i][1] = l >= 0 ? U(i, l - 1) : 0u;
            w[i][2] = l >= 0 ? U(i, l) : 0u;
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (sign[j] != 0) continue;
            i64 d = 0;
            if (l >= 0) {
                u64 e = 0, o = 0;
#pragma unroll
                for (int i = 0; i < BB; ++i) {
                    const int sh = j * i, qa = sh >> 5, r = sh & 31;
                    const u32 tv = fshl(w[i][1 - qa], w[i][2 - qa], (u32)r);
                    if (i & 1) o += tv; else e += tv;
                }
                d = (i64)e - (i64)o;
            }
            const unsigned nz = __ballot_sync(FULL, d != 0);
            if (T[j] == 0 && nz == 0) continue;
            for (int tt = 0; tt < 32; ++tt) {
                const i64 dt = __shfl_sync(FULL, d, tt);
                if (top - tt < 0) break;
                T[j] = T[j] * 4294967296LL + dt;
                if (T[j] >= 17) { sign[j] = 1; break; }
                if (T[j] <= -17) { sign[j] = -1; break; }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < N; ++j)
        if (sign[j] == 0) sign[j] = T[j] < 0 ? -1 : 1;
    // ---- bottom-up: every point of a chunk from one read of the block limbs ----
    UnsignedNorm ne[N], no[N];
    EvalCarry cpm[N];
#pragma unroll
    for (int j = 0; j < N; ++j) { ne[j] = {0, 0}; no[j] = {0, 0}; cpm[j] = {0, 0}; }
    for (int base = 0; base < g.estride; base += CH) {
        const int l0 = base + 4 * lane;
        u32 v[BB][6];  // limbs l0-2 .. l0+3 of each block
#pragma unroll
        for (int i = 0; i < BB; ++i) {
            U4(i, l0, v[i] + 2);
            const u32 b2 = __shfl_up_sync(FULL, v[i][4], 1), b3 = __shfl_up_sync(FULL, v[i][5], 1);
            v[i][0] = lane == 0 ? U(i, l0 - 2) : b2;
            v[i][1] = lane == 0 ? U(i, l0 - 1) : b3;
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            u64 e[4] = {0, 0, 0, 0}, o[4] = {0, 0, 0, 0};
#pragma unroll
            for (int i = 0; i < BB; ++i) {
                const int sh = j * i, qa = sh >> 5, r = sh & 31;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const u32 tv = fshl(v[i][jj - qa + 1], v[i][jj - qa + 2], (u32)r);
                    if (i & 1) o[jj] += tv; else e[jj] += tv;
                }
            }
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                if (l0 + jj >= g.e) { e[jj] = 0; o[jj] = 0; }
            u32 dp[4], dm[4];
            eval_finish(e, o, sign[j], ne[j], no[j], cpm[j], dp, dm);
            if (l0 < g.estride) {
                st4(out + (k * npts + 2 * j + 1) * (long)g.estride + l0, dp);
                st4(out + (k * npts + 2 * j + 2) * (long)g.estride + l0, dm);
            }
        }
    }
    if (lane == 0) {
        sgn[k * npts] = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            sgn[k * npts + 2 * j + 1] = 0;
            sgn[k * npts + 2 * j + 2] = sign[j] < 0 ? 1 : 0;
        }
    }
}

__global__ void __launch_bounds__(256)
eval_warp_kernel(const u32* __restrict__ in, long in_stride, LevelGeom g, u32* __restrict__ out,
                 uint8_t* __restrict__ sgn, long P, int rowlen) {
    extern __shared__ __align__(16) u32 rows_sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long k = (long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (k >= P) return;  // warp-uniform
    u32* rs = rows_sm + (long)warp * rowlen;
    const u32* row = in + k * in_stride;
    const int npts = 2 * g.B - 1;
    const int W = ((g.n - 1) * g.n >> 5) + 1;
    // staged layout: block i occupies padded slots [i (b + W), i (b + W) + b + W), first W zero
    const int bw = g.b + W;
    for (int i = 0; i < g.B; ++i)
        for (int xo = lane; xo < bw; xo += 32) {
            const int xi = xo - W, gi = i * g.b + xi;
            rs[pad32(i * bw + xo)] = (xi >= 0 && gi < g.s) ? __ldg(row + gi) : 0u;
        }
    __syncwarp();
    auto U = [&](int i, int x) -> u32 {  // limb x of block i (zero outside [0, b))
        return (x < g.b) ? rs[pad32(i * bw + W + x)] : 0u;
    };
    u32* orow0 = out + (k * npts) * (long)g.estride;
    for (int pos = 4 * lane; pos < g.estride; pos += CH) {
        u32 v[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) v[jj] = (pos + jj < g.b && pos + jj < g.s) ? U(0, pos + jj) : 0u;
        st4(orow0 + pos, v);
    }
    if (lane == 0) sgn[k * npts] = 0;
    for (int j = 0; j < g.n; ++j) {
        // sign of E - O, top-down
        i64 T = 0;
        int sign = 0;
        for (int top = g.e - 1; top >= 0 && sign == 0; top -= 32) {
            const int l = top - lane;
            i64 d = 0;
            if (l >= 0) {
                u64 e = 0, o = 0;
                for (int i = 0; i < g.B; ++i) {
                    const int sh = j * i, qa = sh >> 5, r = sh & 31;
                    const u32 hi = (l - qa >= 0) ? U(i, l - qa) : 0u;
                    const u32 lo = (l - qa - 1 >= 0) ? U(i, l - qa - 1) : 0u;
                    const u32 t = fshl(lo, hi, (u32)r);
                    if (i & 1) o += t; else e += t;
                }
                d = (i64)e - (i64)o;
            }
            const unsigned nz = __ballot_sync(FULL, d != 0);
            if (T == 0 && nz == 0) continue;
            for (int t = 0; t < 32; ++t) {
                const i64 dt = __shfl_sync(FULL, d, t);
                if (top - t < 0) break;
                T = T * 4294967296LL + dt;
                if (T >= 17) { sign = 1; break; }
                if (T <= -17) { sign = -1; break; }
            }
        }
        if (sign == 0) sign = T < 0 ? -1 : 1;
        u32* rp = out + (k * npts + 2 * j + 1) * (long)g.estride;
        u32* rm = out + (k * npts + 2 * j + 2) * (long)g.estride;
        UnsignedNorm ne{0, 0}, no{0, 0};
        EvalCarry cpm{0, 0};
        for (int base = 0; base < g.estride; base += CH) {
            u64 e[4] = {0, 0, 0, 0}, o[4] = {0, 0, 0, 0};
            const int l0 = base + 4 * lane;
            if (l0 < g.e) {
                for (int i = 0; i < g.B; ++i) {
                    const int sh = j * i, qa = sh >> 5, r = sh & 31;
                    const int x0 = l0 - qa - 1;  // >= -W: the zero halo covers it
                    u32 v[5];
#pragma unroll
                    for (int q = 0; q < 5; ++q)
                        v[q] = (x0 + q < g.b) ? rs[pad32(i * bw + W + x0 + q)] : 0u;
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const u32 t = fshl(v[jj], v[jj + 1], (u32)r);
                        if (i & 1) o[jj] += t; else e[jj] += t;
                    }
                }
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (l0 + jj >= g.e) { e[jj] = 0; o[jj] = 0; }
            }
            u32 dp[4], dm[4];
            eval_finish(e, o, sign, ne, no, cpm, dp, dm);
            if (l0 < g.estride) {
                st4(rp + l0, dp);
                st4(rm + l0, dm);
            }
        }
        if (lane == 0) {
            sgn[k * npts + 2 * j + 1] = 0;
            sgn[k * npts + 2 * j + 2] = sign < 0 ? 1 : 0;
        }
    }
}

cudaError_t launch_eval2(const u32* in, long in_stride, u32* out, uint8_t* sgn, const u32* in2,
                         long in2_stride, u32* out2, uint8_t* sgn2, const LevelGeom& g, long P,
                         void* work, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    const int Wh = ((g.n - 1) * g.n >> 5) + 1;
    const bool warp_rows = P >= 1024 && (pad32(g.B * (g.b + Wh)) + 4) * 4 <= 12 * 1024;
    if (!(use_wide_eval(g, P) && work) && !warp_rows) {
        // the block-per-row kernel (few rows, or long ones): both operands in one
        // launch, which also halves the partly filled last waves
        const int warps = g.n < 1 ? 1 : g.n;
        const int W = ((g.n - 1) * g.n >> 5) + 1;
        const size_t smem = (size_t)2 * g.B * ((CH + W) + ((CH + W) >> 5) + 1) * 4;
        if (warps * 32 <= 384) {
            note_kernel("eval_kernel<384,3>");
            eval_kernel<384, 3><<<(unsigned)(2 * P), warps * 32, smem, st>>>(in, in_stride, g, out, sgn, P,
                                                                          in2, in2_stride, out2, sgn2);
        } else {
            note_kernel("eval_kernel<1024,1>");
            eval_kernel<1024, 1><<<(unsigned)(2 * P), warps * 32, smem, st>>>(in, in_stride, g, out, sgn, P,
                                                                           in2, in2_stride, out2, sgn2);
        }
        return cudaGetLastError();
    }
    cudaError_t e = launch_eval(in, in_stride, g, out, sgn, P, work, st);
    if (e == cudaSuccess) e = launch_eval(in2, in2_stride, g, out2, sgn2, P, work, st);
    return e;
}

cudaError_t launch_eval(const u32* in, long in_stride, const LevelGeom& g, u32* out,
                        uint8_t* sgn, long P, void* work, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    // few huge rows with scratch available: segment-parallel evaluation
    if (use_wide_eval(g, P) && work) return launch_wide_eval(in, in_stride, g, out, sgn, P, work, st);
    {
        const int W = ((g.n - 1) * g.n >> 5) + 1;
        const int staged = g.B * (g.b + W);
        int rowlen = pad32(staged) + 4;
        if (P >= 1024 && rowlen * 4 <= 12 * 1024) {
            if (g.B <= 8) rowlen = g.B * pts_block_words(g) + 4;  // unpadded, 16-byte rows
            static std::once_flag attr_once;
            std::call_once(attr_once, [] {
                cudaFuncSetAttribute(eval_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     100 * 1024);
            });
            int wpb = (int)((48 * 1024) / ((size_t)rowlen * 4));
            if (wpb > 8) wpb = 8;
            if (wpb < 1) wpb = 1;
            const long grid = (P + wpb - 1) / wpb;
            const size_t smem = (size_t)wpb * rowlen * 4;
            switch (g.B) {
#define TC_EVAL_PTS(BB) \
    case BB: note_kernel("eval_pts_kernel<" #BB ">"); eval_pts_kernel<BB><<<(unsigned)grid, wpb * 32, smem, st>>>(in, in_stride, g, out, sgn, P, rowlen); \
        return cudaGetLastError();
                TC_EVAL_PTS(2) TC_EVAL_PTS(3) TC_EVAL_PTS(4) TC_EVAL_PTS(5)
                TC_EVAL_PTS(6) TC_EVAL_PTS(7) TC_EVAL_PTS(8)
#undef TC_EVAL_PTS
                default: break;
            }
            note_kernel("eval_warp_kernel");
            eval_warp_kernel<<<(unsigned)grid, wpb * 32, (size_t)wpb * rowlen * 4, st>>>(
                in, in_stride, g, out, sgn, P, rowlen);
            return cudaGetLastError();
        }
    }
    const int warps = g.n < 1 ? 1 : g.n;  // n <= 31: one warp per point pair
    const int W = ((g.n - 1) * g.n >> 5) + 1;
    const size_t smem = (size_t)2 * g.B * ((CH + W) + ((CH + W) >> 5) + 1) * 4;  // two chunk buffers
    if (warps * 32 <= 384) {  // up to B = 13: three blocks per SM (at most 56 registers)
        note_kernel("eval_kernel<384,3>");
        eval_kernel<384, 3><<<(unsigned)P, warps * 32, smem, st>>>(in, in_stride, g, out, sgn, P,
                                                                    nullptr, 0, nullptr, nullptr);
    } else {
        note_kernel("eval_kernel<1024,1>");
        eval_kernel<1024, 1><<<(unsigned)P, warps * 32, smem, st>>>(in, in_stride, g, out, sgn, P,
                                                                     nullptr, 0, nullptr, nullptr);
    }
    return cudaGetLastError();
}

// ===========================================================================
// Interpolation (Sections 3 and 4).
//
// Values of W_e and X W_o at the nodes X = 0, 1, 4, ..., 4^(n-1) are formed
// by the even-odd combine, then both polynomials go through the two Newton
// double loops.  Within one stage of a loop every update reads only values of
// the previous stage, so a stage is a set of independent "chains", each a
// pass over Y limbs run by one warp; stages are separated by __syncthreads.
// Each value has two slots (ping-pong) so a stage never overwrites a value
// another chain of the same stage still reads.
//
//   loop 1, stage k (Theorem 3.2): c[m] = (c[m] - c[m-1]) / (X[m] - X[m-k]),
//     m = k..n.  For m = k the divisor is 4^(m-1) (a shift); otherwise it is
//     4^(m-k-1) (4^k - 1): a right shift, then exact division by the odd
//     4^k - 1 (two 32-bit divisions 2^k - 1 and 2^k + 1 when k >= 16).
//   loop 2, stage m (Theorem 3.3): c[k] -= X[m] c[k+1], k = m..n-1, i.e.
//     a subtraction of c[k+1] shifted left by 2(m-1).  Stage m = 0 is empty
//     because X[0] = 0.
//
// Right shifts need the limbs above, so those chains emit chunk c-1 while
// loading chunk c (a one-chunk lag); stores stay 16-byte aligned.
// ===========================================================================

struct DivTable {
    DivConst d[2][32];  // [first/second divisor][k]; d == 1 means none
};

static u32 inv32(u32 d) {
    u32 x = d;  // correct to 3 bits for odd d
    for (int i = 0; i < 5; ++i) x *= 2u - d * x;
    return x;
}

static u32 powmod_host(u64 base, u64 e, u32 m) {
    u64 r = 1 % m;
    base %= m;
    while (e) {
        if (e & 1) r = r * base % m;
        base = base * base % m;
        e >>= 1;
    }
    return (u32)r;
}

// Constants for exact division by odd d with KL limbs per lane.
static DivConst make_div(u32 d, int KL) {
    DivConst c;
    c.d = d;
    c.inv = inv32(d);
    c.ninv = 0u - c.inv;
    for (int i = 0; i < 5; ++i) c.rkm[i] = 0;
    c.unit = (d > 1 && d < (1u << 26) && powmod_host(2, 32ull * KL, d) == 1) ? 1u : 0u;
    c.recip = d > 1 ? 0xffffffffu / d : 0u;
    if (d > 1) {
        // rk = rho^KL = 2^(-32 KL) mod d: the inverse of 2^(32 KL) mod d by extended Euclid.
        const u32 t = powmod_host(2, 32ull * KL, d);
        i64 a = t, m = d, x0 = 1, x1 = 0;
        while (m) {
            i64 q = a / m, r = a - q * m;
            a = m; m = r;
            r = x0 - q * x1; x0 = x1; x1 = r;
        }
        u64 rk = (u64)((x0 % (i64)d + d) % d);
        for (int i = 0; i < 5; ++i) {
            c.rkm[i] = (u32)((rk << 32) % d);
            rk = rk * rk % d;
        }
    }
    return c;
}

// The same constants for other translation units (the matrix interpolation).
DivConst make_div_const(u32 d, int KL) { return make_div(d, KL); }

static DivTable make_div_table(int KL) {
    DivTable t;
    for (int k = 0; k < 32; ++k) {
        u32 d1 = 1, d2 = 1;
        if (k >= 1 && k < 16) d1 = (u32)((1ull << (2 * k)) - 1);
        if (k >= 16) {
            d1 = (u32)((1ull << k) - 1);
            d2 = (u32)((1ull << k) + 1);
        }
        t.d[0][k] = make_div(d1, KL);
        t.d[1][k] = make_div(d2, KL);
    }
    return t;
}

// Shifted emission: w = this lane's KL limbs; below = the limb under w[0];
// a0, a1 = the two limbs above w[KL-1].  sh < 0 shifts right by -sh (< 64),
// sh >= 0 shifts left by sh (< 32).
template <int KL>
__device__ __forceinline__ void shift_window(const u32 w[KL], u32 below, u32 a0, u32 a1, int sh,
                                             u32 out[KL]) {
    u32 x[KL + 3];  // x[i + 1] = limb i
    x[0] = below;
#pragma unroll
    for (int j = 0; j < KL; ++j) x[j + 1] = w[j];
    x[KL + 1] = a0;
    x[KL + 2] = a1;
    if (sh < 0) {
        const int R = -sh, qa = R >> 5, r = R & 31;
#pragma unroll
        for (int j = 0; j < KL; ++j) {
            const u32 lo = qa ? x[j + 2] : x[j + 1];
            const u32 hi = qa ? x[j + 3] : x[j + 2];
            out[j] = fshr(lo, hi, (u32)r);
        }
    } else {
#pragma unroll
        for (int j = 0; j < KL; ++j) out[j] = fshl(x[j], x[j + 1], (u32)sh);
    }
}

// Two chains at once (the even and the odd polynomial share every shift and
// divisor): O_p = ((X_p - Z_p) >> R) / d1 / d2 for p = 0, 1.  R < 64; a
// divisor of 1 means no division.  The two chains are independent, so their
// scans and multiply chains interleave.
template <int KL>
__device__ void chain2_sub_shr_div(const u32* X0, const u32* Z0, u32* O0, const u32* X1,
                                   const u32* Z1, u32* O1, int Y, int R, const DivConst& d1,
                                   const DivConst& d2) {
    constexpr int C = 32 * KL;
    const int lane = lane_id();
    const int nch = Y / C;
    const u32* X[2] = {X0, X1};
    const u32* Z[2] = {Z0, Z1};
    u32* O[2] = {O0, O1};
    u32 bw[2] = {0, 0}, B1[2] = {0, 0}, B2[2] = {0, 0};
    u32 prev[2][KL];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int j = 0; j < KL; ++j) prev[p][j] = 0;
    for (int c = 0; c <= nch; ++c) {
        u32 cur[2][KL];
        if (c < nch) {
            u32 x[2][KL], z[2][KL];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                ld_seg<KL>(X[p] + c * C + KL * lane, x[p]);
                ld_seg<KL>(Z[p] + c * C + KL * lane, z[p]);
            }
#pragma unroll
            for (int p = 0; p < 2; ++p) warp_sub_seg<KL>(x[p], z[p], bw[p], cur[p]);
        } else {
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int j = 0; j < KL; ++j) cur[p][j] = 0;
        }
        if (c > 0) {
            u32 v[2][KL];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                u32 a0 = __shfl_down_sync(FULL, prev[p][0], 1), a1 = __shfl_down_sync(FULL, prev[p][1], 1);
                const u32 c0 = __shfl_sync(FULL, cur[p][0], 0), c1 = __shfl_sync(FULL, cur[p][1], 0);
                if (lane == 31) { a0 = c0; a1 = c1; }
                shift_window<KL>(prev[p], 0u, a0, a1, -R, v[p]);
            }
            if (d1.d > 1) {
#pragma unroll
                for (int p = 0; p < 2; ++p) warp_exact_div_seg<KL>(v[p], d1, B1[p]);
            }
            if (d2.d > 1) {
#pragma unroll
                for (int p = 0; p < 2; ++p) warp_exact_div_seg<KL>(v[p], d2, B2[p]);
            }
#pragma unroll
            for (int p = 0; p < 2; ++p) st_seg<KL>(O[p] + (c - 1) * C + KL * lane, v[p]);
        }
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int j = 0; j < KL; ++j) prev[p][j] = cur[p][j];
    }
}

// Two chains at once: O_p = X_p - (Z_p << S), p = 0, 1 (S < 64).
template <int KL>
__device__ void chain2_sub_shl(const u32* X0, const u32* Z0, u32* O0, const u32* X1,
                               const u32* Z1, u32* O1, int Y, int S) {
    constexpr int C = 32 * KL;
    const int lane = lane_id();
    const int nch = Y / C;
    const int qa = S >> 5, s = S & 31;
    const u32* X[2] = {X0, X1};
    const u32* Z[2] = {Z0, Z1};
    u32* O[2] = {O0, O1};
    u32 bw[2] = {0, 0}, t2[2] = {0, 0}, t3[2] = {0, 0};
    for (int c = 0; c < nch; ++c) {
        u32 x[2][KL], z[2][KL];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            ld_seg<KL>(X[p] + c * C + KL * lane, x[p]);
            ld_seg<KL>(Z[p] + c * C + KL * lane, z[p]);
        }
        u32 r[2][KL];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            u32 m1 = __shfl_up_sync(FULL, z[p][KL - 1], 1), m2 = __shfl_up_sync(FULL, z[p][KL - 2], 1);
            if (lane == 0) { m1 = t3[p]; m2 = t2[p]; }
            u32 zw[KL + 2];  // zw[i + 2] = limb i
            zw[0] = m2;
            zw[1] = m1;
#pragma unroll
            for (int j = 0; j < KL; ++j) zw[j + 2] = z[p][j];
            u32 sz[KL];
#pragma unroll
            for (int j = 0; j < KL; ++j) {
                const u32 hi = qa ? zw[j + 1] : zw[j + 2];
                const u32 lo = qa ? zw[j] : zw[j + 1];
                sz[j] = fshl(lo, hi, (u32)s);
            }
            warp_sub_seg<KL>(x[p], sz, bw[p], r[p]);
        }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            st_seg<KL>(O[p] + c * C + KL * lane, r[p]);
            t3[p] = __shfl_sync(FULL, z[p][KL - 1], 31);
            t2[p] = __shfl_sync(FULL, z[p][KL - 2], 31);
        }
    }
}

// Even-odd combine for node m >= 1 (eq. 4.5-4.6):
//   A = W(x) + |W(-x)|, D = W(x) - |W(-x)|  (W(x) >= |W(-x)|)
//   ye_m = (neg ? D : A) / 2,   yo_m = x (neg ? A : D) / 2,  x = 2^(m-1)
template <int KL>
__device__ void chain_even_odd(const u32* Pp, const u32* Mm, int len, bool neg, int m,
                               u32* CE, u32* CO, int Y) {
    constexpr int C = 32 * KL;
    const int lane = lane_id();
    const int nch = Y / C;
    u32 cA = 0, bD = 0;
    u32 pA[KL], pD[KL];
#pragma unroll
    for (int j = 0; j < KL; ++j) { pA[j] = 0; pD[j] = 0; }
    u32 tA = 0, tD = 0;  // last limb of chunk c-2
    const int sh_o = m == 1 ? -1 : m - 2;
    for (int c = 0; c <= nch; ++c) {
        u32 A[KL], D[KL];
        if (c < nch) {
            u32 p[KL], q[KL];
            ld_seg_masked<KL>(Pp, c * C + KL * lane, len, p);
            ld_seg_masked<KL>(Mm, c * C + KL * lane, len, q);
            warp_add_seg<KL>(p, q, cA, A);
            warp_sub_seg<KL>(p, q, bD, D);
        } else {
#pragma unroll
            for (int j = 0; j < KL; ++j) { A[j] = 0; D[j] = 0; }
        }
        if (c > 0) {
            u32 bA = __shfl_up_sync(FULL, pA[KL - 1], 1), bDv = __shfl_up_sync(FULL, pD[KL - 1], 1);
            if (lane == 0) { bA = tA; bDv = tD; }
            u32 aA0 = __shfl_down_sync(FULL, pA[0], 1), aA1 = __shfl_down_sync(FULL, pA[1], 1);
            u32 aD0 = __shfl_down_sync(FULL, pD[0], 1), aD1 = __shfl_down_sync(FULL, pD[1], 1);
            const u32 nA0 = __shfl_sync(FULL, A[0], 0), nA1 = __shfl_sync(FULL, A[1], 0);
            const u32 nD0 = __shfl_sync(FULL, D[0], 0), nD1 = __shfl_sync(FULL, D[1], 0);
            if (lane == 31) { aA0 = nA0; aA1 = nA1; aD0 = nD0; aD1 = nD1; }
            u32 e_out[KL], o_out[KL];
            if (neg) {
                shift_window<KL>(pD, bDv, aD0, aD1, -1, e_out);
                shift_window<KL>(pA, bA, aA0, aA1, sh_o, o_out);
            } else {
                shift_window<KL>(pA, bA, aA0, aA1, -1, e_out);
                shift_window<KL>(pD, bDv, aD0, aD1, sh_o, o_out);
            }
            st_seg<KL>(CE + (c - 1) * C + KL * lane, e_out);
            st_seg<KL>(CO + (c - 1) * C + KL * lane, o_out);
        }
        tA = __shfl_sync(FULL, pA[KL - 1], 31);
        tD = __shfl_sync(FULL, pD[KL - 1], 31);
#pragma unroll
        for (int j = 0; j < KL; ++j) { pA[j] = A[j]; pD[j] = D[j]; }
    }
}

// Copy a row of `len` limbs into a value of Y limbs (zero-extended); zero if src == null.
template <int KL>
__device__ void chain_copy(const u32* src, int len, u32* dst, int Y) {
    constexpr int C = 32 * KL;
    const int lane = lane_id();
    for (int c = 0; c < Y; c += C) {
        u32 v[KL];
#pragma unroll
        for (int j = 0; j < KL; ++j) v[j] = 0;
        if (src) ld_seg_masked<KL>(src, c + KL * lane, len, v);
        st_seg<KL>(dst + c + KL * lane, v);
    }
}

// out[0..out_len) = sum over terms t < nterms of term_t shifted by t * bstep limbs,
// where term t has Y limbs and get(t, x) returns its limb x (0 <= x < Y).
template <class Get>
__device__ void block_recompose(Get get, long nterms, long Y, long bstep, u32* out, long out_len,
                                u32* sh) {
    BlockNormState st{0, 0};
    const int tid = threadIdx.x;
    const long chunk = 4L * blockDim.x;
    const bool aligned = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
    for (long base = 0; base < out_len; base += chunk) {
        u64 cols[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long l = base + 4L * tid + j;
            u64 S = 0;
            if (l < out_len) {
                // terms t with 0 <= l - t*bstep < Y, scanned down from the last one reaching l
                long t = l / bstep;
                if (t > nterms - 1) t = nterms - 1;
                for (; t >= 0; --t) {
                    const long x = l - t * bstep;
                    if (x >= Y) break;
                    S += get(t, x);
                }
            }
            cols[j] = S;
        }
        u32 d[4];
        block_norm_unsigned(cols, st, d, sh);
        const long pos = base + 4L * tid;
        if (aligned && pos + 4 <= out_len) {
            st4(out + pos, d);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (pos + j < out_len) out[pos + j] = d[j];
        }
    }
}

struct InterpArgs {
    LevelGeom g;
    const u32* y;
    const uint8_t* su;
    const uint8_t* sv;
    u32* out;
    long out_stride;
    int out_len;
    u32* work;        // global work base (per product 4 (n+1) Y limbs), null = shared
    int use_smem;
};

template <int KL>
__global__ void __launch_bounds__(512)
interp_kernel(InterpArgs a, DivTable dt, long P) {
    extern __shared__ __align__(16) u32 sm[];
    const long k = blockIdx.x;
    if (k >= P) return;
    const LevelGeom& g = a.g;
    const int n = g.n, Y = g.Y;
    const int npts = 2 * g.B - 1;
    const int tid = threadIdx.x, warp = tid >> 5, nw = blockDim.x >> 5;

    __shared__ int slot[2][33];
    __shared__ __align__(16) u32 shscan[2 * 1024 + 80];
    __shared__ const u32* terms[65];
    u32* base = a.use_smem ? sm : a.work + k * (long)(4 * (n + 1)) * Y;
    auto val = [&](int sl, int poly, int m) -> u32* {
        return base + ((long)((sl * 2 + poly) * (n + 1) + m)) * Y;
    };
    const u32* yk = a.y + k * npts * (long)g.ystride;
    auto sgn = [&](int p) -> bool {
        bool s = false;
        if (a.su) s ^= a.su[k * npts + p] != 0;
        if (a.sv) s ^= a.sv[k * npts + p] != 0;
        return s;
    };
    if (tid < 66) slot[tid / 33][tid % 33] = 0;
    __syncthreads();

    // ---- even-odd combine (chain 0: node 0) ----
    for (int c = warp; c <= n; c += nw) {
        if (c == 0) {
            chain_copy<KL>(yk, 2 * g.e, val(0, 0, 0), Y);
            chain_copy<KL>(nullptr, 0, val(0, 1, 0), Y);
        } else {
            const u32* Pp = yk + (2 * c - 1) * (long)g.ystride;
            const u32* Mm = yk + (2 * c) * (long)g.ystride;
            chain_even_odd<KL>(Pp, Mm, 2 * g.e, sgn(2 * c), c, val(0, 0, c), val(0, 1, c), Y);
        }
    }
    __syncthreads();

    // ---- Newton loop 1 (Theorem 3.2); both polynomials in one warp ----
    // (the two polynomials' slots move together, so slot[0][.] serves both)
    for (int kk = 1; kk <= n; ++kk) {
        const int cnt = n - kk + 1;
        for (int c = warp; c < cnt; c += nw) {
            const int m = kk + c;
            const int sx = slot[0][m], sz = slot[0][m - 1];
            const int R = m == kk ? 2 * (m - 1) : 2 * (m - kk - 1);
            const bool div = m > kk;
            chain2_sub_shr_div<KL>(val(sx, 0, m), val(sz, 0, m - 1), val(1 - sx, 0, m),
                                   val(sx, 1, m), val(sz, 1, m - 1), val(1 - sx, 1, m), Y, R,
                                   div ? dt.d[0][kk] : dt.d[0][0], div ? dt.d[1][kk] : dt.d[1][0]);
        }
        __syncthreads();
        if (tid < cnt) slot[0][kk + tid] ^= 1;
        __syncthreads();
    }

    // ---- Newton loop 2 (Theorem 3.3) ----
    for (int m = n - 1; m >= 1; --m) {
        const int cnt = n - m;
        for (int c = warp; c < cnt; c += nw) {
            const int kx = m + c;
            const int sx = slot[0][kx], sz = slot[0][kx + 1];
            chain2_sub_shl<KL>(val(sx, 0, kx), val(sz, 0, kx + 1), val(1 - sx, 0, kx),
                               val(sx, 1, kx), val(sz, 1, kx + 1), val(1 - sx, 1, kx), Y,
                               2 * (m - 1));
        }
        __syncthreads();
        if (tid < cnt) slot[0][m + tid] ^= 1;
        __syncthreads();
    }

    // ---- re-interleave and recompose: w_2i = ce_i, w_2i+1 = co_(i+1) ----
    if (tid <= 2 * n) {
        const int poly = tid & 1, m = (tid + 1) >> 1;
        terms[tid] = val(slot[0][m], poly, m);
    }
    __syncthreads();
    block_recompose([&](long t, long x) -> u32 { return terms[t][x]; }, 2 * n + 1, Y, g.b,
                    a.out + k * a.out_stride, a.out_len, shscan);
}

// ---------------------------------------------------------------------------
// Warp-per-product interpolation for small values (many products per level).
// One warp runs every chain of one product in sequence, so the paper's in-place
// orders apply directly: loop 1 visits m from n down to k (each update reads the
// old c[m-1]); loop 2 visits k upward (each update reads the old c[k+1]).  One
// value slot per (polynomial, node); no block barriers.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
interp_warp_kernel(InterpArgs a, DivTable dt, long P) {
    extern __shared__ __align__(16) u32 sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const long k = (long)blockIdx.x * wpb + warp;
    if (k >= P) return;  // warp-uniform
    const LevelGeom& g = a.g;
    const int n = g.n, Y = g.Y;
    const int npts = 2 * g.B - 1;
    // values: shared memory when they fit, else this product's slice of the work buffer
    u32* base = a.use_smem ? sm + (long)warp * 2 * (n + 1) * Y : a.work + k * (long)(2 * (n + 1)) * Y;
    auto val = [&](int poly, int m) -> u32* { return base + (long)(poly * (n + 1) + m) * Y; };
    const u32* yk = a.y + k * npts * (long)g.ystride;
    auto sgn = [&](int p) -> bool {
        bool s = false;
        if (a.su) s ^= a.su[k * npts + p] != 0;
        if (a.sv) s ^= a.sv[k * npts + p] != 0;
        return s;
    };
    chain_copy<4>(yk, 2 * g.e, val(0, 0), Y);
    chain_copy<4>(nullptr, 0, val(1, 0), Y);
    for (int m = 1; m <= n; ++m) {
        const u32* Pp = yk + (2 * m - 1) * (long)g.ystride;
        const u32* Mm = yk + (2 * m) * (long)g.ystride;
        chain_even_odd<4>(Pp, Mm, 2 * g.e, sgn(2 * m), m, val(0, m), val(1, m), Y);
    }
    __syncwarp();
    for (int kk = 1; kk <= n; ++kk)
        for (int m = n; m >= kk; --m) {
            const int R = m == kk ? 2 * (m - 1) : 2 * (m - kk - 1);
            const bool div = m > kk;
            chain2_sub_shr_div<4>(val(0, m), val(0, m - 1), val(0, m), val(1, m), val(1, m - 1),
                                  val(1, m), Y, R, div ? dt.d[0][kk] : dt.d[0][0],
                                  div ? dt.d[1][kk] : dt.d[1][0]);
            __syncwarp();
        }
    for (int m = n - 1; m >= 1; --m)
        for (int kx = m; kx <= n - 1; ++kx) {
            chain2_sub_shl<4>(val(0, kx), val(0, kx + 1), val(0, kx), val(1, kx), val(1, kx + 1),
                              val(1, kx), Y, 2 * (m - 1));
            __syncwarp();
        }
    // recompose: out[l] = sum_t w_t[l - t b], w_2i = ce_i, w_2i+1 = co_(i+1)
    u32* out = a.out + k * a.out_stride;
    const bool aligned = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
    UnsignedNorm st{0, 0};
    const int nterms = 2 * n + 1;
    for (int base_l = 0; base_l < a.out_len; base_l += CH) {
        u64 cols[4];
        const int l0 = base_l + 4 * lane;
        int t0 = l0 / g.b;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int l = l0 + j;
            u64 S = 0;
            if (l < a.out_len) {
                int t = t0;
                while ((t + 1) * g.b <= l) ++t;  // t = floor(l / b)
                if (t > nterms - 1) t = nterms - 1;
                for (; t >= 0; --t) {
                    const int x = l - t * g.b;
                    if (x >= Y) break;
                    S += val(t & 1, (t + 1) >> 1)[x];
                }
            }
            cols[j] = S;
        }
        u32 d[4];
        warp_norm_unsigned(cols, st, d);
        if (aligned && l0 + 4 <= a.out_len) {
            st4(out + l0, d);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (l0 + j < a.out_len) out[l0 + j] = d[j];
        }
    }
}

// ---------------------------------------------------------------------------
// Streaming warp-per-product interpolation for values too long for shared
// memory (many products, long values).
//
// Every chain of the even-odd combine and of both Newton loops reads its
// operands from low limbs to high, carrying a borrow, a remainder or a few
// limbs of look-behind, so one warp can push a 32 KL-limb window through all
// of them before moving on: the values live in shared memory one window at a
// time and the work buffer is touched a fixed number of times instead of
// once per chain.
//
// Pass A (even-odd combine, Section 4, and Theorem 3.2): a right shift by R
// needs the limbs above its output, so each right-shifting stage emits the
// window two limbs lower than its input (offset 2 after the combine, 2kk + 2
// after stage kk).  Every chain of stage kk reads values written by stage
// kk - 1, so offsets agree within a stage; c_m is final after stage m, at
// offset 2(m + 1), and is written to the work buffer at its true position.
//
// The odd divisors of Theorem 3.2 are deferred: stage kk keeps
// c'_m = c_m d_1 ... d_kk for m > kk (no division), and the one chain that
// meets operands of different scale, m = kk, multiplies c'_(kk-1) by
// d_(kk-1) first.  So c'_m = c_m d_1 ... d_(m-1) when c_m is final, and it is
// divided then, by products of consecutive d_j grouped below 2^31: n(n-1)/2
// divisions become a few per node (21 instead of 55 for n = 11).  Every
// shift stays exact (the scale factors are odd) and every intermediate stays
// non-negative; the scaled values are up to n(n-1) bits longer, which the
// step count covers.
//
// Pass B (Theorem 3.3) re-reads the final Newton coefficients with aligned
// windows; its left shifts only look behind.  Pass C recomposes.
// ---------------------------------------------------------------------------

// e[t] = limb (KL lane - NB + t) of the chunk, t < KL + NB; lane 0 takes the
// NB limbs below the chunk from h (h[NB - 1] the highest).
template <int KL, int NB>
__device__ __forceinline__ void look_behind(const u32 x[KL], const u32 h[NB], u32 e[KL + NB]) {
    const int lane = lane_id();
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        const u32 v = __shfl_up_sync(FULL, x[KL - NB + t], 1);
        e[t] = lane == 0 ? h[t] : v;
    }
#pragma unroll
    for (int j = 0; j < KL; ++j) e[NB + j] = x[j];
}

// y = x f for a streamed value x and f < 2^31: limb j of y is lo(x_j f) +
// hi(x_(j-1) f) + carry, with the carry 0 or 1.  hi_in: hi(f x) of the limb
// below the chunk; carry: into the chunk (both updated, warp-uniform).
template <int KL>
__device__ __forceinline__ void warp_mul_small(const u32 x[KL], u32 f, u32& hi_in, u32& carry,
                                               u32 y[KL]) {
    u32 lo[KL], hi[KL], sh[KL];
#pragma unroll
    for (int j = 0; j < KL; ++j) {
        lo[j] = x[j] * f;
        hi[j] = __umulhi(x[j], f);
    }
    const u32 hp = __shfl_up_sync(FULL, hi[KL - 1], 1);
    sh[0] = lane_id() == 0 ? hi_in : hp;
#pragma unroll
    for (int j = 1; j < KL; ++j) sh[j] = hi[j - 1];
    warp_add_seg<KL>(lo, sh, carry, y);
    hi_in = __shfl_sync(FULL, hi[KL - 1], 31);
}

// Grouped divisors of the deferred division: the odd factors of d_1, d_2, ...
// in order, packed greedily into products below 2^31 ("full" groups).  Node m
// divides by the full groups inside the factors of d_1 .. d_(m-1), then by the
// product of the factors left over ("part").
struct FinTable {
    DivConst full[48];
    DivConst part[32];
    unsigned char nfull[32];
    unsigned char haspart[32];
    short off[33];  // first remainder slot of node m (both polynomials: 2 words per slot)
};

// Per-warp shared memory: value windows c_1..c_n of both polynomials plus
// ce_0 (co_0 = 0 is not stored), then chain states: even-odd (8 words per
// node), Newton loop 1 (6 words per chain: 3 per polynomial), the scale
// multiplications (8 words per node), the deferred divisions (2 words per
// divisor).  Loop 2 reuses the loop-1 space (6 words per chain).
struct StreamLayout {
    int vals, st0, st1, stm, stf, words;
};

__host__ __device__ inline StreamLayout stream_layout(int n, int C, int fin_slots) {
    StreamLayout L;
    L.vals = (2 * n + 1) * C;
    L.st0 = 8 * (n + 1);
    L.st1 = (3 * n * (n + 1) + 3) / 4 * 4;  // every region a multiple of 4 words: the value
                                           // windows of the next warp stay 16-byte aligned
    L.stm = 8 * (n + 1);
    L.stf = (2 * fin_slots + 3) / 4 * 4;
    L.words = L.vals + L.st0 + L.st1 + L.stm + L.stf;
    return L;
}

// Write this lane's KL limbs of a window starting at absolute limb `start`
// (even) into a row of Y limbs (even), dropping limbs outside [0, Y).
template <int KL>
__device__ __forceinline__ void st_window(u32* row, int start, int Y, const u32 v[KL]) {
    const int p0 = start + KL * lane_id();
#pragma unroll
    for (int j = 0; j < KL; j += 2) {
        const int p = p0 + j;
        if (p >= 0 && p + 2 <= Y) *reinterpret_cast<uint2*>(row + p) = make_uint2(v[j], v[j + 1]);
    }
}

__global__ void __launch_bounds__(256)
interp_stream_kernel(InterpArgs a, DivTable dt, FinTable ft, long P) {
    constexpr int KL = 4, C = 32 * KL;
    extern __shared__ __align__(16) u32 sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const long k = (long)blockIdx.x * wpb + warp;
    if (k >= P) return;  // warp-uniform
    const LevelGeom& g = a.g;
    const int n = g.n, Y = g.Y, len = 2 * g.e;
    const int npts = 2 * g.B - 1;
    const StreamLayout L = stream_layout(n, C, ft.off[n + 1]);
    u32* vals = sm + (long)warp * L.words;
    u32* st0 = vals + L.vals;
    u32* st1 = st0 + L.st0;
    u32* stm = st1 + L.st1;
    u32* stf = stm + L.stm;
    u32* W = a.work + k * (long)(2 * (n + 1)) * Y;
    // this lane's limbs of the window of c_m (m >= 1) or ce_0 (p = 0, m = 0)
    auto V = [&](int p, int m) -> u32* {
        return vals + (m == 0 ? 2 * n : p * n + m - 1) * C + KL * lane;
    };
    auto Wrow = [&](int p, int m) -> u32* { return W + (long)(p * (n + 1) + m) * Y; };
    const u32* yk = a.y + k * npts * (long)g.ystride;
    auto sgn = [&](int p) -> bool {
        bool s = false;
        if (a.su) s ^= a.su[k * npts + p] != 0;
        if (a.sv) s ^= a.sv[k * npts + p] != 0;
        return s;
    };
    auto ldv = [&](const u32* p, u32 v[KL]) {
        const uint4 q = *reinterpret_cast<const uint4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    };
    u32 negmask = 0;  // bit m: |W(-2^(m-1))| was negated
    for (int m = 1; m <= n; ++m) negmask |= sgn(2 * m) ? 1u << m : 0u;
    for (int i = lane; i < L.st0 + L.st1 + L.stm + L.stf; i += 32) st0[i] = 0;
    __syncwarp();

    // ---- pass A: even-odd combine and Newton loop 1 ----
    const int grow = (n * (n - 1) + 31) / 32 + 1;  // limbs of the deferred scale factors
    // every combine output and Newton coefficient fits in 2e limbs, so the windows
    // stop once positions 2e + 2 and up (all zero) are reached; the tail of the
    // work rows they would have written is zeroed after the pass
    const int ext = 2 * g.e + 2 < Y ? 2 * g.e + 2 : Y;
    const int stepsA = (ext + 2 * n + 2 + grow + C - 1) / C;
    for (int step = 0; step < stepsA; ++step) {
        const int base = C * step;  // absolute limb of an offset-0 window
        __syncwarp();
        {   // node 0: ce_0 = y_0, co_0 = 0 (delayed by two limbs to offset 2)
            u32 y0[KL], h[2] = {st0[0], st0[1]}, e[KL + 2], o[KL];
            ld_seg_masked<KL>(yk, base + KL * lane, len, y0);
            look_behind<KL, 2>(y0, h, e);
#pragma unroll
            for (int j = 0; j < KL; ++j) o[j] = e[j];
            st_seg<KL>(V(0, 0), o);
            __syncwarp();
            if (lane == 31) { st0[0] = y0[KL - 2]; st0[1] = y0[KL - 1]; }
            st_window<KL>(Wrow(0, 0), base - 2, Y, o);
        }
        // the rows of node m+1 are loaded while node m is combined
        u32 pn[KL], qn[KL];
        ld_seg_masked<KL>(yk + (long)g.ystride, base + KL * lane, len, pn);
        ld_seg_masked<KL>(yk + 2 * (long)g.ystride, base + KL * lane, len, qn);
        for (int m = 1; m <= n; ++m) {
            // eq. 4.5-4.6: A = W(x) + |W(-x)|, D = W(x) - |W(-x)|, x = 2^(m-1);
            // ce_m = (neg ? D : A) / 2, co_m = x (neg ? A : D) / 2
            u32* s = st0 + 8 * m;
            const bool neg = (negmask >> m) & 1u;
            u32 pv[KL], qv[KL], A[KL], D[KL];
#pragma unroll
            for (int j = 0; j < KL; ++j) { pv[j] = pn[j]; qv[j] = qn[j]; }
            if (m < n) {
                ld_seg_masked<KL>(yk + (2 * m + 1) * (long)g.ystride, base + KL * lane, len, pn);
                ld_seg_masked<KL>(yk + (2 * m + 2) * (long)g.ystride, base + KL * lane, len, qn);
            }
            u32 cA = s[0], bD = s[1];
            const u32 hS[3] = {s[2], s[3], s[4]}, hT[3] = {s[5], s[6], s[7]};
            warp_add_seg<KL>(pv, qv, cA, A);
            warp_sub_seg<KL>(pv, qv, bD, D);
            u32 S[KL], T[KL];
#pragma unroll
            for (int j = 0; j < KL; ++j) { S[j] = neg ? D[j] : A[j]; T[j] = neg ? A[j] : D[j]; }
            u32 eS[KL + 3], eT[KL + 3], ce[KL], co[KL];
            look_behind<KL, 3>(S, hS, eS);
            look_behind<KL, 3>(T, hT, eT);
            const u32 sh = m >= 2 ? (u32)(m - 2) : 0u;
#pragma unroll
            for (int j = 0; j < KL; ++j) {
                ce[j] = fshr(eS[j + 1], eS[j + 2], 1);
                co[j] = m == 1 ? fshr(eT[j + 1], eT[j + 2], 1) : fshl(eT[j], eT[j + 1], sh);
            }
            st_seg<KL>(V(0, m), ce);
            st_seg<KL>(V(1, m), co);
            __syncwarp();
            if (lane == 0) { s[0] = cA; s[1] = bD; }
            if (lane == 31) {
                s[2] = S[KL - 3]; s[3] = S[KL - 2]; s[4] = S[KL - 1];
                s[5] = T[KL - 3]; s[6] = T[KL - 2]; s[7] = T[KL - 1];
            }
        }
        // Theorem 3.2 on the scaled values, in place with m descending (each
        // update reads the old c'_(m-1))
        int t1 = 0;  // index of chain (kk, kk)
        for (int kk = 1; kk <= n; ++kk) {
            for (int m = n; m >= kk; --m) {
                const int R = m == kk ? 2 * (m - 1) : 2 * (m - kk - 1);
                const int q = R >> 5;
                const u32 r = (u32)(R & 31);
                // scale of c'_(kk-1) to meet c'_kk: d_(kk-1) = f1 f2 (f2 = 1 below k = 16)
                const u32 f1 = m == kk && kk >= 2 ? dt.d[0][kk - 1].d : 1u;
                const u32 f2 = m == kk && kk >= 2 ? dt.d[1][kk - 1].d : 1u;
                u32* s = st1 + 6 * (t1 + m - kk);  // per polynomial: 2 limbs, borrow
                u32* sm8 = stm + 8 * kk;           // per polynomial: (hi, carry) per factor
                u32 out[2][KL], dtop[2][2], bw[2] = {s[2], s[5]}, mst[2][4];
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    u32 x[KL], z[KL] = {0, 0, 0, 0}, dv[KL], e[KL + 2];
                    ldv(V(p, m), x);
                    if (m > 1 || p == 0) ldv(V(p, m - 1), z);
                    if (f1 > 1) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) mst[p][i] = sm8[4 * p + i];
                        u32 zz[KL];
                        warp_mul_small<KL>(z, f1, mst[p][0], mst[p][1], zz);
#pragma unroll
                        for (int j = 0; j < KL; ++j) z[j] = zz[j];
                    }
                    if (f2 > 1) {
                        u32 zz[KL];
                        warp_mul_small<KL>(z, f2, mst[p][2], mst[p][3], zz);
#pragma unroll
                        for (int j = 0; j < KL; ++j) z[j] = zz[j];
                    }
                    const u32 h[2] = {s[3 * p], s[3 * p + 1]};
                    warp_sub_seg<KL>(x, z, bw[p], dv);
                    look_behind<KL, 2>(dv, h, e);
#pragma unroll
                    for (int j = 0; j < KL; ++j)
                        out[p][j] = q ? fshr(e[j + 1], e[j + 2], r) : fshr(e[j], e[j + 1], r);
                    dtop[p][0] = dv[KL - 2];
                    dtop[p][1] = dv[KL - 1];
                }
#pragma unroll
                for (int p = 0; p < 2; ++p) st_seg<KL>(V(p, m), out[p]);
                __syncwarp();
                if (lane == 0) {
                    s[2] = bw[0]; s[5] = bw[1];
                    if (f1 > 1) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) { sm8[i] = mst[0][i]; sm8[4 + i] = mst[1][i]; }
                    }
                }
                if (lane == 31) {
                    s[0] = dtop[0][0]; s[1] = dtop[0][1];
                    s[3] = dtop[1][0]; s[4] = dtop[1][1];
                }
            }
            t1 += n - kk + 1;
            // c'_kk is final, at offset 2 kk + 2: divide by d_1 ... d_(kk-1) and store
            u32 v[2][KL];
            ldv(V(0, kk), v[0]);
            ldv(V(1, kk), v[1]);
            u32* sf = stf + 2 * ft.off[kk];
            const int nf = ft.nfull[kk] + ft.haspart[kk];
            for (int i = 0; i < nf; ++i) {
                const DivConst& dc = i < ft.nfull[kk] ? ft.full[i] : ft.part[kk];
                u32 B[2] = {sf[2 * i], sf[2 * i + 1]};
                warp_exact_div_seg<KL>(v[0], dc, B[0]);
                warp_exact_div_seg<KL>(v[1], dc, B[1]);
                __syncwarp();
                if (lane == 0) { sf[2 * i] = B[0]; sf[2 * i + 1] = B[1]; }
            }
            st_window<KL>(Wrow(0, kk), base - 2 * kk - 2, Y, v[0]);
            st_window<KL>(Wrow(1, kk), base - 2 * kk - 2, Y, v[1]);
        }
    }
    // positions the windows did not reach (all at or above 2e + 2: zero)
    for (int z = C * stepsA - 2 * n - 2 + lane; z < Y; z += 32)
        for (int m = 0; m <= n; ++m) {
            Wrow(0, m)[z] = 0u;
            if (m >= 1) Wrow(1, m)[z] = 0u;
        }
    __syncwarp();
    for (int i = lane; i < L.st1; i += 32) st1[i] = 0;
    __syncwarp();

    // ---- pass B: Newton to monomial basis (Theorem 3.3), aligned windows ----
    for (int base = 0; base < Y; base += C) {
        __syncwarp();
        // the window of every value, all copies in flight together
        for (int p = 0; p < 2; ++p)
            for (int m = 1; m <= n; ++m) cp_async16(V(p, m), Wrow(p, m) + base + KL * lane);
        cp_async_wait_all();
        __syncwarp();
        // in place with kx ascending (each update reads the old c_(kx+1))
        int t2 = 0;  // index of chain (m, m)
        for (int m = n - 1; m >= 1; --m) {
            const int S = 2 * (m - 1);
            const int q = S >> 5;
            const u32 sh = (u32)(S & 31);
            for (int kx = m; kx <= n - 1; ++kx) {
                u32* s = st1 + 6 * (t2 + kx - m);
                u32 ztop[2][2];
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    u32 x[KL], z[KL], e[KL + 2], sz[KL], r[KL];
                    ldv(V(p, kx), x);
                    ldv(V(p, kx + 1), z);
                    u32 bw = s[3 * p];
                    const u32 h[2] = {s[3 * p + 1], s[3 * p + 2]};
                    look_behind<KL, 2>(z, h, e);
#pragma unroll
                    for (int j = 0; j < KL; ++j)
                        sz[j] = q ? fshl(e[j], e[j + 1], sh) : fshl(e[j + 1], e[j + 2], sh);
                    warp_sub_seg<KL>(x, sz, bw, r);
                    st_seg<KL>(V(p, kx), r);
                    ztop[p][0] = z[KL - 2];
                    ztop[p][1] = z[KL - 1];
                    __syncwarp();
                    if (lane == 0) s[3 * p] = bw;
                    if (lane == 31) { s[3 * p + 1] = ztop[p][0]; s[3 * p + 2] = ztop[p][1]; }
                }
            }
            t2 += n - m;
        }
        for (int p = 0; p < 2; ++p)
            for (int m = 1; m <= n - 1; ++m) {
                u32 v[KL];
                ldv(V(p, m), v);
                st_seg<KL>(Wrow(p, m) + base + KL * lane, v);
            }
    }
    __syncwarp();

    // ---- pass C: recompose out[l] = sum_t w_t[l - t b], w_2i = ce_i, w_2i+1 = co_(i+1) ----
    u32* out = a.out + k * a.out_stride;
    const bool aligned = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
    UnsignedNorm nst{0, 0};
    const int nterms = 2 * n + 1;
    // Terms t with 0 <= l - t b < Y for some l in [l0, l0 + 4), highest first.  The
    // first four of a chunk are loaded before any is added, and those of chunk c+1
    // while chunk c is normalised (software pipelined); more terms (short b) follow
    // in a plain loop.
    auto load_term = [&](int l0, int tt, u32 q[4]) {
        const int x = l0 - tt * g.b;
        const u32* w = Wrow(tt & 1, (tt + 1) >> 1);
        if (x >= 0 && x + 4 <= Y && ((x & 3) == 0)) {
            const uint4 v = ld4(w + x);
            q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) q[j] = x + j >= 0 && x + j < Y ? w[x + j] : 0u;
        }
    };
    auto issue = [&](int l0, u32 q[4][4], int& trest) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) q[i][j] = 0;
        trest = -1;
        if (l0 >= a.out_len) return;
        int t = (l0 + 3) / g.b;
        if (t > nterms - 1) t = nterms - 1;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (t - i >= 0 && l0 - (t - i) * g.b < Y) load_term(l0, t - i, q[i]);
        trest = t - 4;
    };
    u32 qn[4][4];
    int tn;
    issue(4 * lane, qn, tn);
    for (int base_l = 0; base_l < a.out_len; base_l += CH) {
        u64 cols[4] = {0, 0, 0, 0};
        const int l0 = base_l + 4 * lane;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) cols[j] += qn[i][j];
        for (int t = tn; t >= 0 && l0 - t * g.b < Y; --t) {
            u32 r[4];
            load_term(l0, t, r);
#pragma unroll
            for (int j = 0; j < 4; ++j) cols[j] += r[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (l0 + j >= a.out_len) cols[j] = 0;
        issue(l0 + CH, qn, tn);
        u32 d[4];
        warp_norm_unsigned(cols, nst, d);
        if (aligned && l0 + 4 <= a.out_len) {
            st4(out + l0, d);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (l0 + j < a.out_len) out[l0 + j] = d[j];
        }
    }
}

// Grouping of the deferred divisors for degree n (see the streaming kernel).
static FinTable make_fin_table(int n, int KL) {
    FinTable f;
    memset(&f, 0, sizeof(f));
    // odd factors of d_1 .. d_(n-1), with the node after whose d_j each ends
    std::vector<u32> fac;
    std::vector<int> upto;  // fac[i] belongs to d_(upto[i])
    for (int j = 1; j <= n - 1; ++j) {
        if (j < 16) {
            fac.push_back((u32)((1ull << (2 * j)) - 1));
            upto.push_back(j);
        } else {
            fac.push_back((u32)((1ull << j) - 1));
            upto.push_back(j);
            fac.push_back((u32)((1ull << j) + 1));
            upto.push_back(j);
        }
    }
    // greedy groups below 2^31
    std::vector<int> gstart;
    std::vector<u64> gprod;
    for (size_t i = 0; i < fac.size(); ++i) {
        if (gprod.empty() || gprod.back() * fac[i] >= (1ull << 31)) {
            gstart.push_back((int)i);
            gprod.push_back(fac[i]);
        } else {
            gprod.back() *= fac[i];
        }
    }
    for (size_t i = 0; i < gprod.size() && i < 48; ++i) f.full[i] = make_div((u32)gprod[i], KL);
    int slot = 0;
    for (int m = 0; m <= n; ++m) {
        f.off[m] = (short)slot;
        // factors of d_1 .. d_(m-1)
        size_t cnt = 0;
        while (cnt < fac.size() && upto[cnt] <= m - 1) ++cnt;
        int full = 0;
        while (full < (int)gstart.size() &&
               (full + 1 < (int)gstart.size() ? (size_t)gstart[full + 1] : fac.size()) <= cnt)
            ++full;
        u64 part = 1;
        for (size_t i = full < (int)gstart.size() ? (size_t)gstart[full] : cnt; i < cnt; ++i) part *= fac[i];
        f.nfull[m] = (unsigned char)full;
        f.haspart[m] = part > 1 ? 1 : 0;
        if (part > 1) f.part[m] = make_div((u32)part, KL);
        slot += full + f.haspart[m];
    }
    f.off[n + 1] = (short)slot;
    return f;
}

// ---------------------------------------------------------------------------
// Streaming interpolation with the two polynomials on two warps.
//
// After the even-odd combine (Section 4) the even polynomial (values ce) and
// the odd one (co) go through Theorems 3.2 and 3.3 independently, so each
// product gets a pair of warps: warp 2q+0 streams ce, warp 2q+1 streams co.
// Both read the pointwise products and form their own half of the combine
// (the even warp S = W(x) +- |W(-x)|, the odd warp T = W(x) -+ |W(-x)|).  A
// warp keeps one polynomial's n + 1 value windows, so its shared memory is
// about half of the one-warp design and twice as many products are resident.
//
// The same windows as interp_stream_kernel, with these differences: every
// stage emits its window one limb lower (a right shift by R < 32 bits reads
// the limb above, so one limb of look-behind per chain suffices), hence c_m is
// final at offset m + 1; chain borrows are packed one bit per chain; the
// deferred divisions are the same (FinTable, one word per slot).  After the
// Theorem 3.3 pass both warps of a block meet at a barrier and the even warp
// recomposes the product from the work buffer.
// ---------------------------------------------------------------------------
struct SplitLayout {
    int vals, st0, st1, stb, stm, stf, words;
};

__host__ __device__ inline SplitLayout split_layout(int n, int C, int fin_slots) {
    SplitLayout L;
    const int chains = n * (n + 1) / 2;
    L.vals = (n + 1) * C;
    L.st0 = 3 * (n + 1);          // combine: carry or borrow, up to two look-behind limbs
    L.st1 = chains;               // one look-behind limb per chain (loop 1; loop 2 reuses it)
    L.stb = (chains + 31) / 32;   // chain borrows, one bit per chain
    L.stm = 4 * (n + 1);          // deferred multiplications: (hi, carry) per factor
    L.stf = fin_slots;            // deferred divisions: one borrow per divisor
    const int w = L.vals + L.st0 + L.st1 + L.stb + L.stm + L.stf;
    L.words = (w + 3) / 4 * 4;    // the next warp's windows stay 16-byte aligned
    return L;
}

// Store this lane's KL limbs of a window starting at absolute limb `start`
// (any parity) into a row of Y limbs, dropping limbs outside [0, Y).
template <int KL>
__device__ __forceinline__ void st_window_any(u32* row, int start, int Y, const u32 v[KL]) {
    const int p0 = start + KL * lane_id();
    if ((start & 1) == 0) {
#pragma unroll
        for (int j = 0; j < KL; j += 2) {
            const int q = p0 + j;
            if (q >= 0 && q + 2 <= Y) *reinterpret_cast<uint2*>(row + q) = make_uint2(v[j], v[j + 1]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < KL; ++j) {
            const int q = p0 + j;
            if (q >= 0 && q < Y) row[q] = v[j];
        }
    }
}

__device__ __forceinline__ u32 get_bit(const u32* words, int t) { return (words[t >> 5] >> (t & 31)) & 1u; }

template <int KL, int MINB>
__global__ void __launch_bounds__(256, MINB)
interp_split_kernel(InterpArgs a, DivTable dt, FinTable ft, long P) {
    constexpr int C = 32 * KL;
    extern __shared__ __align__(16) u32 sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = warp & 1;  // 0: even polynomial, 1: odd polynomial
    const long k = (long)blockIdx.x * (blockDim.x >> 6) + (warp >> 1);
    const bool active = k < P;  // every warp reaches the block barrier below
    const LevelGeom& g = a.g;
    const int n = g.n, Y = g.Y, len = 2 * g.e;
    const int npts = 2 * g.B - 1;
    const SplitLayout L = split_layout(n, C, ft.off[n + 1]);
    u32* vals = sm + (long)warp * L.words;
    u32* st0 = vals + L.vals;
    u32* st1 = st0 + L.st0;
    u32* stb = st1 + L.st1;
    u32* stm = stb + L.stb;
    u32* stf = stm + L.stm;
    u32* W = a.work + (active ? k : 0) * (long)(2 * (n + 1)) * Y;
    auto V = [&](int m) -> u32* { return vals + m * C + KL * lane; };
    auto Wrow = [&](int pp, int m) -> u32* { return W + (long)(pp * (n + 1) + m) * Y; };
    auto ldv = [&](const u32* q, u32 v[KL]) { ld_seg<KL>(q, v); };
    auto set_bit = [&](u32* words, int t, u32 b) {  // lane 0 only
        const u32 m = 1u << (t & 31);
        words[t >> 5] = b ? (words[t >> 5] | m) : (words[t >> 5] & ~m);
    };
    if (active) {
        const u32* yk = a.y + k * npts * (long)g.ystride;
        u32 negmask = 0;  // bit m: |W(-2^(m-1))| was negated
        for (int m = 1; m <= n; ++m) {
            bool sg = false;
            if (a.su) sg ^= a.su[k * npts + 2 * m] != 0;
            if (a.sv) sg ^= a.sv[k * npts + 2 * m] != 0;
            negmask |= sg ? 1u << m : 0u;
        }
        for (int i = lane; i < L.st0 + L.st1 + L.stb + L.stm + L.stf; i += 32) st0[i] = 0;
        __syncwarp();

        // ---- pass A: even-odd combine and Newton loop 1 ----
        const int grow = (n * (n - 1) + 31) / 32 + 1;  // limbs of the deferred scale factors
        // windows up to the values' real length 2e + 2, as in the one-warp kernel
        const int ext = 2 * g.e + 2 < Y ? 2 * g.e + 2 : Y;
        const int stepsA = (ext + 2 * n + 2 + grow + C - 1) / C;
        for (int step = 0; step < stepsA; ++step) {
            const int base = C * step;
            __syncwarp();
            if (p == 0) {  // node 0: ce_0 = y_0, one limb lower
                u32 y0[KL], e[KL + 1], o[KL];
                const u32 h[1] = {st0[1]};
                ld_seg_masked<KL>(yk, base + KL * lane, len, y0);
                look_behind<KL, 1>(y0, h, e);
#pragma unroll
                for (int j = 0; j < KL; ++j) o[j] = e[j];
                st_seg<KL>(V(0), o);
                __syncwarp();
                if (lane == 31) st0[1] = y0[KL - 1];
                st_window_any<KL>(Wrow(0, 0), base - 1, Y, o);
            }
            // eq. 4.5-4.6, x = 2^(m-1): the even warp forms S = neg ? D : A and
            // ce_m = S / 2; the odd warp T = neg ? A : D and co_m = x T / 2, where
            // A = W(x) + |W(-x)|, D = W(x) - |W(-x)|; the next node's rows load
            // while this node is combined
            u32 pn[KL], qn[KL];
            ld_seg_masked<KL>(yk + (long)g.ystride, base + KL * lane, len, pn);
            ld_seg_masked<KL>(yk + 2 * (long)g.ystride, base + KL * lane, len, qn);
            for (int m = 1; m <= n; ++m) {
                u32* s = st0 + 3 * m;
                const bool neg = (negmask >> m) & 1u;
                u32 pv[KL], qv[KL], r[KL], out[KL];
#pragma unroll
                for (int j = 0; j < KL; ++j) { pv[j] = pn[j]; qv[j] = qn[j]; }
                if (m < n) {
                    ld_seg_masked<KL>(yk + (2 * m + 1) * (long)g.ystride, base + KL * lane, len, pn);
                    ld_seg_masked<KL>(yk + (2 * m + 2) * (long)g.ystride, base + KL * lane, len, qn);
                }
                u32 cb = s[0];
                if ((p == 0) != neg) warp_add_seg_scan<KL>(pv, qv, cb, r);
                else warp_sub_seg_scan<KL>(pv, qv, cb, r);
                const bool right = p == 0 || m == 1;  // / 2 (else a left shift by m - 2)
                if (right) {
                    u32 e[KL + 1];
                    const u32 h[1] = {s[2]};
                    look_behind<KL, 1>(r, h, e);
#pragma unroll
                    for (int j = 0; j < KL; ++j) out[j] = fshr(e[j], e[j + 1], 1);
                } else {
                    u32 e[KL + 2];
                    const u32 h[2] = {s[1], s[2]};
                    look_behind<KL, 2>(r, h, e);
#pragma unroll
                    for (int j = 0; j < KL; ++j) out[j] = fshl(e[j], e[j + 1], (u32)(m - 2));
                }
                st_seg<KL>(V(m), out);
                __syncwarp();
                if (lane == 0) s[0] = cb;
                if (lane == 31) { s[1] = r[KL - 2]; s[2] = r[KL - 1]; }
            }
            // Theorem 3.2 on the scaled values, in place with m descending (each
            // update reads the old c'_(m-1)); the odd polynomial's c_0 is 0.  The
            // chains of a stage are independent, so they run in pairs (m, m - 1).
            int t1 = 0;  // chain index of (kk, kk)
            for (int kk = 1; kk <= n; ++kk) {
                for (int m = n; m >= kk; m -= 2) {
                    const bool two = m - 1 >= kk;          // warp-uniform
                    const int mb = m - 1;
                    const int ta = t1 + m - kk, tb = ta - 1;
                    const u32 Ra = (u32)(m == kk ? 2 * (m - 1) : 2 * (m - kk - 1));
                    const u32 Rb = (u32)(mb == kk ? 2 * (mb - 1) : 2 * (mb - kk - 1));
                    // the chain (kk, kk) scales c'_(kk-1) by d_(kk-1) = f1 f2 first
                    const bool scale = (two ? mb : m) == kk && kk >= 2;
                    const u32 f1 = scale ? dt.d[0][kk - 1].d : 1u;
                    const u32 f2 = scale ? dt.d[1][kk - 1].d : 1u;
                    u32* sm4 = stm + 4 * kk;
                    u32 xa[KL], za[KL], zb[KL], ms[4];
#pragma unroll
                    for (int j = 0; j < KL; ++j) { za[j] = 0; zb[j] = 0; }
                    ldv(V(m), xa);
                    if (m > 1 || p == 0) ldv(V(m - 1), za);   // also chain b's x
                    if (two && (mb > 1 || p == 0)) ldv(V(mb - 1), zb);
                    if (f1 > 1) {
                        u32* zs = two ? zb : za;
#pragma unroll
                        for (int i = 0; i < 4; ++i) ms[i] = sm4[i];
                        u32 zz[KL];
                        warp_mul_small<KL>(zs, f1, ms[0], ms[1], zz);
#pragma unroll
                        for (int j = 0; j < KL; ++j) zs[j] = zz[j];
                        if (f2 > 1) {
                            warp_mul_small<KL>(zs, f2, ms[2], ms[3], zz);
#pragma unroll
                            for (int j = 0; j < KL; ++j) zs[j] = zz[j];
                        }
                    }
                    u32 bwa = get_bit(stb, ta), bwb = two ? get_bit(stb, tb) : 0u;
                    u32 dva[KL], dvb[KL], ea[KL + 1], eb[KL + 1], oa[KL], ob[KL];
                    const u32 ha[1] = {st1[ta]};
                    if (two) {
                        const u32 hb[1] = {st1[tb]};
                        // chain b: x = old c'_(m-1) = za (before any scaling of chain a: none)
                        u32 xb[KL];
#pragma unroll
                        for (int j = 0; j < KL; ++j) xb[j] = za[j];
                        warp_sub_seg2<KL>(xa, za, bwa, dva, xb, zb, bwb, dvb);
                        look_behind<KL, 1>(dva, ha, ea);
                        look_behind<KL, 1>(dvb, hb, eb);
#pragma unroll
                        for (int j = 0; j < KL; ++j) {
                            oa[j] = fshr(ea[j], ea[j + 1], Ra);
                            ob[j] = fshr(eb[j], eb[j + 1], Rb);
                        }
                        st_seg<KL>(V(m), oa);
                        st_seg<KL>(V(mb), ob);
                    } else {
                        warp_sub_seg_scan<KL>(xa, za, bwa, dva);
                        look_behind<KL, 1>(dva, ha, ea);
#pragma unroll
                        for (int j = 0; j < KL; ++j) oa[j] = fshr(ea[j], ea[j + 1], Ra);
                        st_seg<KL>(V(m), oa);
                    }
                    __syncwarp();
                    if (lane == 0) {
                        set_bit(stb, ta, bwa);
                        if (two) set_bit(stb, tb, bwb);
                        if (f1 > 1) {
#pragma unroll
                            for (int i = 0; i < 4; ++i) sm4[i] = ms[i];
                        }
                    }
                    if (lane == 31) {
                        st1[ta] = dva[KL - 1];
                        if (two) st1[tb] = dvb[KL - 1];
                    }
                    __syncwarp();
                }
                t1 += n - kk + 1;
                // c'_kk is final, at offset kk + 1: divide by d_1 ... d_(kk-1) and store
                u32 v[KL];
                ldv(V(kk), v);
                u32* sf = stf + ft.off[kk];
                const int nf = ft.nfull[kk] + ft.haspart[kk];
                for (int i = 0; i < nf; ++i) {
                    const DivConst& dc = i < ft.nfull[kk] ? ft.full[i] : ft.part[kk];
                    u32 B = sf[i];
                    warp_exact_div_seg<KL>(v, dc, B);
                    __syncwarp();
                    if (lane == 0) sf[i] = B;
                }
                st_window_any<KL>(Wrow(p, kk), base - kk - 1, Y, v);
            }
        }
        // positions the windows did not reach (all at or above 2e + 2: zero)
        for (int z = C * stepsA - 2 * n - 2 + lane; z < Y; z += 32)
            for (int m = p == 0 ? 0 : 1; m <= n; ++m) Wrow(p, m)[z] = 0u;
        __syncwarp();
        for (int i = lane; i < L.st1 + L.stb; i += 32) st1[i] = 0;
        __syncwarp();

        // ---- pass B: Newton to monomial basis (Theorem 3.3), aligned windows ----
        for (int base = 0; base < Y; base += C) {
            __syncwarp();
            for (int m = 1; m <= n; ++m)
#pragma unroll
                for (int j = 0; j < KL; j += 4) cp_async16(V(m) + j, Wrow(p, m) + base + KL * lane + j);
            cp_async_wait_all();
            __syncwarp();
            int t2 = 0;  // chain index of (m, m)
            for (int m = n - 1; m >= 1; --m) {
                const u32 S = (u32)(2 * (m - 1));
                // in place, kx ascending: each chain reads the old c_(kx+1); the chains
                // of a stage are independent and run in pairs (kx, kx + 1)
                for (int kx = m; kx <= n - 1; kx += 2) {
                    const bool two = kx + 1 <= n - 1;  // warp-uniform
                    const int ta = t2 + kx - m, tb = ta + 1;
                    u32 xa[KL], za[KL], zb[KL], ea[KL + 1], eb[KL + 1], sa[KL], sb[KL], ra[KL], rb[KL];
                    ldv(V(kx), xa);
                    ldv(V(kx + 1), za);                // also chain b's x
                    u32 bwa = get_bit(stb, ta), bwb = two ? get_bit(stb, tb) : 0u;
                    const u32 ha[1] = {st1[ta]};
                    look_behind<KL, 1>(za, ha, ea);
#pragma unroll
                    for (int j = 0; j < KL; ++j) sa[j] = fshl(ea[j], ea[j + 1], S);
                    if (two) {
                        ldv(V(kx + 2), zb);
                        const u32 hb[1] = {st1[tb]};
                        look_behind<KL, 1>(zb, hb, eb);
#pragma unroll
                        for (int j = 0; j < KL; ++j) sb[j] = fshl(eb[j], eb[j + 1], S);
                        warp_sub_seg2<KL>(xa, sa, bwa, ra, za, sb, bwb, rb);
                        st_seg<KL>(V(kx), ra);
                        st_seg<KL>(V(kx + 1), rb);
                    } else {
                        warp_sub_seg_scan<KL>(xa, sa, bwa, ra);
                        st_seg<KL>(V(kx), ra);
                    }
                    __syncwarp();
                    if (lane == 0) {
                        set_bit(stb, ta, bwa);
                        if (two) set_bit(stb, tb, bwb);
                    }
                    if (lane == 31) {
                        st1[ta] = za[KL - 1];
                        if (two) st1[tb] = zb[KL - 1];
                    }
                    __syncwarp();
                }
                t2 += n - m;
            }
            for (int m = 1; m <= n - 1; ++m) {
                u32 v[KL];
                ldv(V(m), v);
                st_seg<KL>(Wrow(p, m) + base + KL * lane, v);
            }
        }
    }
    __syncthreads();  // both polynomials of every product of the block are in the work buffer
    if (!active || p != 0) return;

    // ---- pass C: recompose out[l] = sum_t w_t[l - t b], w_2i = ce_i, w_2i+1 = co_(i+1) ----
    u32* out = a.out + k * a.out_stride;
    const bool aligned = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
    UnsignedNorm nst{0, 0};
    const int nterms = 2 * n + 1;
    auto load_term = [&](int l0, int tt, u32 q[4]) {
        const int x = l0 - tt * g.b;
        const u32* w = Wrow(tt & 1, (tt + 1) >> 1);
        if (x >= 0 && x + 4 <= Y && ((x & 3) == 0)) {
            const uint4 v = ld4(w + x);
            q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) q[j] = x + j >= 0 && x + j < Y ? w[x + j] : 0u;
        }
    };
    auto issue = [&](int l0, u32 q[4][4], int& trest) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) q[i][j] = 0;
        trest = -1;
        if (l0 >= a.out_len) return;
        int t = (l0 + 3) / g.b;
        if (t > nterms - 1) t = nterms - 1;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (t - i >= 0 && l0 - (t - i) * g.b < Y) load_term(l0, t - i, q[i]);
        trest = t - 4;
    };
    u32 qn[4][4];
    int tn;
    issue(4 * lane, qn, tn);
    for (int base_l = 0; base_l < a.out_len; base_l += CH) {
        u64 cols[4] = {0, 0, 0, 0};
        const int l0 = base_l + 4 * lane;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) cols[j] += qn[i][j];
        for (int t = tn; t >= 0 && l0 - t * g.b < Y; --t) {
            u32 r[4];
            load_term(l0, t, r);
#pragma unroll
            for (int j = 0; j < 4; ++j) cols[j] += r[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (l0 + j >= a.out_len) cols[j] = 0;
        issue(l0 + CH, qn, tn);
        u32 d[4];
        warp_norm_unsigned(cols, nst, d);
        if (aligned && l0 + 4 <= a.out_len) {
            st4(out + l0, d);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (l0 + j < a.out_len) out[l0 + j] = d[j];
        }
    }
}

// ---------------------------------------------------------------------------
// Register-resident warp-per-product interpolation for short values
// (Y <= 32 KL, degree n small): each lane holds KL limbs of every value, so a
// whole value is one warp chunk and every chain of Section 4 / Theorems 3.2
// and 3.3 is a single warp operation with no carried state; shifts take the
// neighbouring lane's limbs by shuffle (right shifts look one lane up, left
// shifts one lane down).  The values go to shared memory only for the
// recomposition.
// ---------------------------------------------------------------------------
template <int KL>
__device__ __forceinline__ void shr_chunk(const u32 x[KL], u32 r, u32 out[KL]) {
    // out = x >> r (r < 32) over the whole warp chunk; the top lane's limb above is 0
    const u32 up = __shfl_down_sync(FULL, x[0], 1);
    const u32 above = lane_id() == 31 ? 0u : up;
#pragma unroll
    for (int j = 0; j < KL; ++j) out[j] = fshr(x[j], j + 1 < KL ? x[j + 1] : above, r);
}

template <int KL>
__device__ __forceinline__ void shl_chunk(const u32 x[KL], u32 s, u32 out[KL]) {
    // out = x << s (s < 32), truncated to the chunk; the bottom lane's limb below is 0
    const u32 dn = __shfl_up_sync(FULL, x[KL - 1], 1);
    const u32 below = lane_id() == 0 ? 0u : dn;
#pragma unroll
    for (int j = 0; j < KL; ++j) out[j] = fshl(j > 0 ? x[j - 1] : below, x[j], s);
}

template <int KL, int N>
__global__ void __launch_bounds__(256)
interp_reg_kernel(InterpArgs a, DivTable dt, long P) {
    extern __shared__ __align__(16) u32 sm[];
    constexpr int C = 32 * KL;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const long k = (long)blockIdx.x * wpb + warp;
    if (k >= P) return;  // warp-uniform
    const LevelGeom& g = a.g;
    const int npts = 2 * N + 1, len = 2 * g.e;
    const u32* yk = a.y + k * npts * (long)g.ystride;
    auto sgn = [&](int p) -> bool {
        bool s = false;
        if (a.su) s ^= a.su[k * npts + p] != 0;
        if (a.sv) s ^= a.sv[k * npts + p] != 0;
        return s;
    };
    // Shared memory: 2N+1 slots of C + 4 words; first the input rows (all copies in
    // flight together, zero past the 2e valid limbs), at the end the recomposed terms.
    constexpr int SLOT = C + 4;
    u32* sw = sm + (long)warp * (2 * N + 1) * SLOT;
#pragma unroll
    for (int r = 0; r <= 2 * N; ++r) {
        const u32* row = yk + r * (long)g.ystride;
#pragma unroll
        for (int jj = 0; jj < KL; jj += 4) {
            const int pos = KL * lane + jj;
            const int left = len - pos;
            const unsigned bytes = left >= 4 ? 16u : left > 0 ? 4u * left : 0u;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                         :: "r"((unsigned)__cvta_generic_to_shared(sw + r * SLOT + pos)),
                            "l"(bytes ? row + pos : row), "r"(bytes) : "memory");
        }
    }
    cp_async_wait_all();
    __syncwarp();
    u32 c[2][N + 1][KL];
    // ---- even-odd combine (eq. 4.5-4.6) ----
    ld_seg<KL>(sw + KL * lane, c[0][0]);
#pragma unroll
    for (int j = 0; j < KL; ++j) c[1][0][j] = 0;
#pragma unroll
    for (int m = 1; m <= N; ++m) {
        u32 pv[KL], qv[KL], A[KL], D[KL];
        ld_seg<KL>(sw + (2 * m - 1) * SLOT + KL * lane, pv);
        ld_seg<KL>(sw + (2 * m) * SLOT + KL * lane, qv);
        u32 z = 0;
        warp_add_seg<KL>(pv, qv, z, A);
        z = 0;
        warp_sub_seg<KL>(pv, qv, z, D);
        const bool ng = sgn(2 * m);
        u32 S[KL], T[KL];
#pragma unroll
        for (int j = 0; j < KL; ++j) { S[j] = ng ? D[j] : A[j]; T[j] = ng ? A[j] : D[j]; }
        shr_chunk<KL>(S, 1, c[0][m]);
        if (m == 1) shr_chunk<KL>(T, 1, c[1][m]);
        else shl_chunk<KL>(T, (u32)(m - 2), c[1][m]);
    }
    // ---- Theorem 3.2, in place with m descending ----
#pragma unroll
    for (int kk = 1; kk <= N; ++kk) {
#pragma unroll
        for (int m = N; m >= kk; --m) {
            const u32 R = (u32)(m == kk ? 2 * (m - 1) : 2 * (m - kk - 1));
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                u32 dv[KL], z = 0;
                warp_sub_seg<KL>(c[p][m], c[p][m - 1], z, dv);
                shr_chunk<KL>(dv, R, c[p][m]);
            }
            if (m > kk) {
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    u32 B = 0;
                    warp_exact_div_seg<KL>(c[p][m], dt.d[0][kk], B);
                    if (dt.d[1][kk].d > 1) {
                        B = 0;
                        warp_exact_div_seg<KL>(c[p][m], dt.d[1][kk], B);
                    }
                }
            }
        }
    }
    // ---- Theorem 3.3, in place with kx ascending ----
#pragma unroll
    for (int mm = N - 1; mm >= 1; --mm) {
#pragma unroll
        for (int kx = mm; kx <= N - 1; ++kx) {
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                u32 sz[KL], z = 0;
                shl_chunk<KL>(c[p][kx + 1], (u32)(2 * (mm - 1)), sz);
                warp_sub_seg<KL>(c[p][kx], sz, z, c[p][kx]);
            }
        }
    }
    // ---- recompose out[l] = sum_t w_t[l - t b] from shared memory ----
    // Term t (w_2i = ce_i, w_2i+1 = co_(i+1)) is stored shifted by d_t = (t b) mod 4
    // words inside a slot of C + 4 words, so limb l - t b of it sits at a 16-byte
    // aligned index whenever l is a multiple of 4: one vector load per term per lane.
    __syncwarp();  // every lane has read its input rows
    const int b = g.b;
#pragma unroll
    for (int t = 0; t <= 2 * N; ++t) {
        const u32* w = c[t & 1][(t + 1) >> 1];
        u32* slot = sw + t * SLOT;
        const int dt = (t * b) & 3;
        if (lane == 0) { slot[0] = slot[1] = slot[2] = slot[3] = 0u; }
        if (lane == 31) { slot[C] = slot[C + 1] = slot[C + 2] = slot[C + 3] = 0u; }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < KL; ++j) slot[dt + KL * lane + j] = w[j];
    }
    __syncwarp();
    u32* out = a.out + k * a.out_stride;
    const bool aligned = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
    UnsignedNorm nst{0, 0};
    for (int base_l = 0; base_l < a.out_len; base_l += CH) {
        u64 cols[4] = {0, 0, 0, 0};
        const int l0 = base_l + 4 * lane;
#pragma unroll
        for (int t = 0; t <= 2 * N; ++t) {
            if (base_l + CH <= t * b || base_l >= t * b + C) continue;  // warp-uniform
            const int dt = (t * b) & 3;
            const int x = l0 - t * b;  // x + dt is a multiple of 4
            if (x < -dt || x > C - dt) continue;
            const uint4 q = *reinterpret_cast<const uint4*>(sw + t * SLOT + dt + x);
            cols[0] += q.x; cols[1] += q.y; cols[2] += q.z; cols[3] += q.w;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (l0 + j >= a.out_len) cols[j] = 0;
        u32 d[4];
        warp_norm_unsigned(cols, nst, d);
        if (aligned && l0 + 4 <= a.out_len) {
            st4(out + l0, d);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (l0 + j < a.out_len) out[l0 + j] = d[j];
        }
    }
}

// Limbs per lane of the register-resident kernel for a level, 0 if none applies.
static int reg_interp_kl(const LevelGeom& g) {
    const int n = g.n;
    if (n <= 2 && g.Y <= 32 * 16 && g.Y > 32 * 12) return 16;
    if (n <= 3 && g.Y <= 32 * 12 && g.Y > 32 * 8) return 12;
    if (n <= 5 && g.Y <= 32 * 8) return 8;
    return 0;
}

template <int KL, int N>
static cudaError_t launch_reg_interp(const InterpArgs& a, long P, cudaStream_t st) {
    static const DivTable dtk = make_div_table(KL);
    const size_t per_warp = (size_t)(2 * N + 1) * (32 * KL + 4) * 4;
    int wpb = (int)((96 * 1024) / per_warp);
    if (wpb > 8) wpb = 8;
    if (wpb < 1) wpb = 1;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(interp_reg_kernel<KL, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
    });
    const long grid = (P + wpb - 1) / wpb;
    note_kernel(KL == 8 ? "interp_reg_kernel<8>" : KL == 12 ? "interp_reg_kernel<12>" : "interp_reg_kernel<16>");
    interp_reg_kernel<KL, N><<<(unsigned)grid, wpb * 32, wpb * per_warp, st>>>(a, dtk, P);
    return cudaGetLastError();
}

static cudaError_t launch_reg_interp_kl(int kl, const InterpArgs& a, long P, cudaStream_t st) {
    const int n = a.g.n;
    if (kl == 16) return n == 1 ? launch_reg_interp<16, 1>(a, P, st) : launch_reg_interp<16, 2>(a, P, st);
    if (kl == 12) {
        if (n == 1) return launch_reg_interp<12, 1>(a, P, st);
        if (n == 2) return launch_reg_interp<12, 2>(a, P, st);
        return launch_reg_interp<12, 3>(a, P, st);
    }
    switch (n) {
        case 1: return launch_reg_interp<8, 1>(a, P, st);
        case 2: return launch_reg_interp<8, 2>(a, P, st);
        case 3: return launch_reg_interp<8, 3>(a, P, st);
        case 4: return launch_reg_interp<8, 4>(a, P, st);
        default: return launch_reg_interp<8, 5>(a, P, st);
    }
}

// Kernel choice for a level: many products -> one warp per product (values in
// shared memory when they fit, else in the work buffer); few products -> one
// block per product.
static bool use_warp_kernel(const LevelGeom& g, long P) { return P >= 2048; }
static size_t warp_values_bytes(const LevelGeom& g) { return (size_t)2 * (g.n + 1) * g.Y * 4; }
static size_t block_values_bytes(const LevelGeom& g) { return (size_t)4 * (g.n + 1) * g.Y * 4; }
constexpr size_t WARP_SMEM_MAX = 24 * 1024;
constexpr int STREAM_SMEM_MAX = 227 * 1024;  // per block
constexpr int SM_SMEM_BYTES = 228 * 1024;    // per SM
constexpr size_t BLOCK_SMEM_MAX = 160 * 1024;

size_t interp_work_bytes(const LevelGeom& g, long P) {
    if (use_wide(g, P)) return (wide_work_bytes(g, P) + P - 1) / P;  // per product, rounded up
    if (use_warp_kernel(g, P) && reg_interp_kl(g)) return 0;
    if (use_warp_kernel(g, P)) return warp_values_bytes(g) <= WARP_SMEM_MAX ? 0 : warp_values_bytes(g);
    return block_values_bytes(g) <= BLOCK_SMEM_MAX ? 0 : block_values_bytes(g);
}

cudaError_t launch_interp(const LevelGeom& g, const u32* y, const uint8_t* su, const uint8_t* sv,
                          u32* out, long out_stride, int out_len, u32* work, long P,
                          cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (use_wide(g, P)) {
        if (!work) return cudaErrorInvalidValue;
        return launch_wide_interp(g, y, su, sv, out, out_stride, out_len, work, P, st);
    }
    static const DivTable dt4 = make_div_table(4), dt8 = make_div_table(8);
    const DivTable& dt = dt4;
    // many products: one warp per product
    if (use_warp_kernel(g, P) && reg_interp_kl(g)) {
        InterpArgs a;
        a.g = g; a.y = y; a.su = su; a.sv = sv; a.out = out; a.out_stride = out_stride;
        a.out_len = out_len; a.work = nullptr; a.use_smem = 1;
        return launch_reg_interp_kl(reg_interp_kl(g), a, P, st);
    }
    if (use_warp_kernel(g, P)) {
        const size_t warp_smem = warp_values_bytes(g);
        InterpArgs a;
        a.g = g; a.y = y; a.su = su; a.sv = sv; a.out = out; a.out_stride = out_stride;
        a.out_len = out_len; a.work = work; a.use_smem = warp_smem <= WARP_SMEM_MAX;
        if (!a.use_smem && !work) return cudaErrorInvalidValue;
        if (!a.use_smem) {
            // long values: stream windows through shared memory; pick the warps per
            // block that keep the most warps resident (1 KB reserved per block)
            static FinTable fins[32];
            static std::once_flag fin_once;
            std::call_once(fin_once, [] {
                for (int nn = 1; nn < 32; ++nn) fins[nn] = make_fin_table(nn, 4);
            });
            const FinTable& ft = fins[g.n];
            if (g.n >= 8 && g.n <= 15 && g.Y % 256 == 0) {
                // two warps per product (one per polynomial), four products per block,
                // windows of 256 limbs (8 per lane; Y is a multiple of 256).  Only for
                // high degree: there the one-warp kernel's windows of both polynomials
                // limit it to 16 resident warps per SM; at low degree it already holds 32
                // and the split kernel's duplicated combine makes it slower
                static FinTable fins8[32];
                static std::once_flag fin8_once;
                std::call_once(fin8_once, [] {
                    for (int nn = 1; nn < 32; ++nn) fins8[nn] = make_fin_table(nn, 8);
                });
                const FinTable& ft8 = fins8[g.n];
                const int split_warp = split_layout(g.n, 256, ft8.off[g.n + 1]).words * 4;
                const size_t smem = (size_t)8 * split_warp;
                if (smem <= (size_t)STREAM_SMEM_MAX) {
                    static std::once_flag split_once;
                    std::call_once(split_once, [] {
                        cudaFuncSetAttribute(interp_split_kernel<8, 2>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, STREAM_SMEM_MAX);
                    });
                    note_kernel("interp_split_kernel<8>");
                    interp_split_kernel<8, 2><<<(unsigned)((P + 3) / 4), 256, smem, st>>>(a, dt8, ft8, P);
                    return cudaGetLastError();
                }
            }
            const int per_warp = stream_layout(g.n, 128, ft.off[g.n + 1]).words * 4;
            // registers per warp as allocated (per thread rounded up to 8)
            static int regs_per_warp = 0;
            static std::once_flag regs_once;
            std::call_once(regs_once, [] {
                cudaFuncAttributes fa;
                regs_per_warp = cudaFuncGetAttributes(&fa, interp_stream_kernel) == cudaSuccess
                                    ? (fa.numRegs + 7) / 8 * 8 * 32 : 64 * 32;
            });
            int best_w = 1, best_res = 0;
            for (int w = 1; w <= 8; ++w) {
                if (w * per_warp > STREAM_SMEM_MAX) break;
                int blocks = SM_SMEM_BYTES / (w * per_warp + 1024);
                const int reg_blocks = 65536 / (w * regs_per_warp);
                if (blocks > reg_blocks) blocks = reg_blocks;
                if (blocks > 32) blocks = 32;
                int res = blocks * w;
                if (res > 64) res = 64;
                if (res >= best_res) { best_res = res; best_w = w; }
            }
            if (best_res == 0) return cudaErrorInvalidConfiguration;
            static std::once_flag stream_once;
            std::call_once(stream_once, [] {
                cudaFuncSetAttribute(interp_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     STREAM_SMEM_MAX);
            });
            const long grid = (P + best_w - 1) / best_w;
            note_kernel("interp_stream_kernel");
            interp_stream_kernel<<<(unsigned)grid, best_w * 32, (size_t)best_w * per_warp, st>>>(a, dt, ft, P);
            return cudaGetLastError();
        }
        int wpb = a.use_smem ? (int)((96 * 1024) / warp_smem) : 4;
        if (wpb > 8) wpb = 8;
        if (wpb < 1) wpb = 1;
        static std::once_flag attr_once;
        std::call_once(attr_once, [] {
            cudaFuncSetAttribute(interp_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
        });
        const long grid = (P + wpb - 1) / wpb;
        note_kernel("interp_warp_kernel");
        interp_warp_kernel<<<(unsigned)grid, wpb * 32, a.use_smem ? wpb * warp_smem : 0, st>>>(a, dt, P);
        return cudaGetLastError();
    }
    InterpArgs a;
    a.g = g;
    a.y = y;
    a.su = su;
    a.sv = sv;
    a.out = out;
    a.out_stride = out_stride;
    a.out_len = out_len;
    const size_t wb = interp_work_bytes(g, P);
    a.use_smem = wb == 0;
    a.work = work;
    if (!a.use_smem && !work) return cudaErrorInvalidValue;
    const size_t smem = a.use_smem ? (size_t)4 * (g.n + 1) * g.Y * 4 : 0;
    int warps = g.n + 1;  // a warp per node pair in the widest stage (even-odd: n + 1)
    if (warps < 4) warps = 4;
    if (warps > 16) warps = 16;
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        cudaFuncSetAttribute(interp_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        cudaFuncSetAttribute(interp_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    });
    // 8 limbs per lane whenever the values are whole 256-limb windows: half the
    // windows per chain, and a lone product's interpolation is a chain of windows
    if (g.K == 8 || g.Y % 256 == 0) {
        note_kernel("interp_kernel<8>");
        interp_kernel<8><<<(unsigned)P, warps * 32, smem, st>>>(a, dt8, P);
    } else {
        note_kernel("interp_kernel<4>");
        interp_kernel<4><<<(unsigned)P, warps * 32, smem, st>>>(a, dt4, P);
    }
    return cudaGetLastError();
}

// ===========================================================================
// Overlap-add of equally spaced rows (sliced unbalanced products).
// ===========================================================================
__global__ void __launch_bounds__(1024)
overlap_add_kernel(const u32* rows, long row_stride, int row_len, long count, long off, u32* out,
                   long out_len) {
    __shared__ __align__(16) u32 shscan[2 * 1024 + 80];
    block_recompose([&](long t, long x) -> u32 { return rows[t * row_stride + x]; }, count,
                    row_len, off, out, out_len, shscan);
}

cudaError_t launch_overlap_add(const u32* rows, long row_stride, int row_len, long count, long off,
                               u32* out, long out_len, cudaStream_t st) {
    if (count <= 0) return cudaErrorInvalidValue;
    overlap_add_kernel<<<1, 1024, 0, st>>>(rows, row_stride, row_len, count, off, out, out_len);
    return cudaGetLastError();
}

__global__ void zero_kernel(u32* p, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        p[i] = 0;
}

cudaError_t launch_zero(u32* p, size_t n, cudaStream_t st) {
    if (!n) return cudaSuccess;
    size_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    zero_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, n);
    return cudaGetLastError();
}

}  // namespace tc
