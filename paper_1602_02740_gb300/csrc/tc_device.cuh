// Device-side limb primitives shared by the Toom-Cook kernels.
//
// Limbs are little-endian uint32.  Every multi-limb pass here works on
// chunks of 128 limbs per warp: lane t holds limbs [4t, 4t+4) of the chunk,
// so a warp-wide uint4 load or store moves 512 contiguous bytes.  Carries,
// borrows and exact-division borrows cross lanes through warp scans and cross
// chunks through a small per-warp state carried in registers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tc {

typedef uint32_t u32;
typedef uint64_t u64;
typedef int64_t i64;

constexpr unsigned FULL = 0xffffffffu;
constexpr int K = 4;          // limbs per lane per chunk
constexpr int CH = 32 * K;    // limbs per warp chunk

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Low 32 bits of (hi:lo) >> r, r in [0, 32).
__device__ __forceinline__ u32 fshr(u32 lo, u32 hi, u32 r) { return __funnelshift_r(lo, hi, r); }
// Low 32 bits of ((hi:lo) << s) >> 32, i.e. (hi << s) | (lo >> (32 - s)), s in [0, 32).
__device__ __forceinline__ u32 fshl(u32 lo, u32 hi, u32 s) { return __funnelshift_l(lo, hi, s); }

__device__ __forceinline__ uint4 ld4(const u32* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ void st4(u32* p, const u32 v[4]) {
    *reinterpret_cast<uint4*>(p) = make_uint4(v[0], v[1], v[2], v[3]);
}

// Load 4 limbs starting at index `pos` of a row of `len` valid limbs (zeros
// beyond).  `pos` is a multiple of 4 and the row base is 16-byte aligned.
__device__ __forceinline__ void ld4_masked(const u32* row, int pos, int len, u32 v[4]) {
    if (pos + 4 <= len) {
        uint4 q = ld4(row + pos);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = (pos + j < len) ? row[pos + j] : 0u;
    }
}

// ---------------------------------------------------------------------------
// Binary carry-lookahead across a warp.
// g: this lane's segment produces a carry out with carry-in 0.
// p: this lane's segment passes a carry-in straight through (disjoint from g).
// cin: carry into lane 0 (warp-uniform, 0 or 1).
// Returns the carry into this lane; *cout receives the warp's carry out.
// The adder G + (G|P) + cin has, at bit i, exactly the carry into lane i.
// ---------------------------------------------------------------------------
__device__ __forceinline__ u32 warp_carry_scan(bool g, bool p, u32 cin, u32* cout) {
    u32 G = __ballot_sync(FULL, g);
    u32 P = __ballot_sync(FULL, p);
    u64 S = (u64)G + (u64)(G | P) + (u64)cin;
    u32 C = (u32)S ^ P;
    *cout = (u32)(S >> 32);
    return (C >> lane_id()) & 1u;
}

// ---------------------------------------------------------------------------
// 4-limb add/sub with carry, as plain 64-bit arithmetic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ u32 add4(const u32 a[4], const u32 b[4], u32 cin, u32 r[4]) {
    u64 c = cin;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        u64 t = (u64)a[j] + b[j] + c;
        r[j] = (u32)t;
        c = t >> 32;
    }
    return (u32)c;
}

__device__ __forceinline__ u32 sub4(const u32 a[4], const u32 b[4], u32 bin, u32 r[4]) {
    u64 bw = bin;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        u64 t = (u64)a[j] - b[j] - bw;
        r[j] = (u32)t;
        bw = (t >> 32) & 1u;
    }
    return (u32)bw;
}

__device__ __forceinline__ bool all_zero4(const u32 r[4]) { return (r[0] | r[1] | r[2] | r[3]) == 0u; }
__device__ __forceinline__ bool all_ones4(const u32 r[4]) { return (r[0] & r[1] & r[2] & r[3]) == FULL; }

// Warp-wide a + b + cin over one chunk; cin/cout are warp-uniform carries.
__device__ __forceinline__ void warp_add_chunk(const u32 a[4], const u32 b[4], u32& carry, u32 r[4]) {
    u32 g = add4(a, b, 0u, r);
    bool p = !g && all_ones4(r);
    u32 cout;
    u32 cin = warp_carry_scan(g != 0u, p, carry, &cout);
    add4(a, b, cin, r);
    carry = cout;
}

// Warp-wide a - b - bin over one chunk.
__device__ __forceinline__ void warp_sub_chunk(const u32 a[4], const u32 b[4], u32& borrow, u32 r[4]) {
    u32 g = sub4(a, b, 0u, r);
    bool p = !g && all_zero4(r);
    u32 bout;
    u32 bin = warp_carry_scan(g != 0u, p, borrow, &bout);
    sub4(a, b, bin, r);
    borrow = bout;
}

// ---------------------------------------------------------------------------
// Normalisation of signed column sums.
//
// A value given as sum_l col[l] 2^(32 l) with |col| < 2^62 is turned into
// digits.  Each column splits into a digit and a carry; the carry is added to
// the next column's digit, which leaves every limb within one unit of the
// digit range, so the remaining carries are in {-1, 0, +1}.  Those are
// resolved by composing, across the warp, the per-limb maps
// x -> floor((y + x) / 2^32) on {-1, 0, 1}.
// A map is stored in 6 bits: bits [2c, 2c+2) hold f(c - 1) + 1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int map3_apply(u32 f, int x) { return (int)((f >> (2 * (x + 1))) & 3u) - 1; }

__device__ __forceinline__ u32 map3_compose(u32 g, u32 f) {  // g after f
    u32 r = 0;
#pragma unroll
    for (int x = -1; x <= 1; ++x) r |= (u32)(map3_apply(g, map3_apply(f, x)) + 1) << (2 * (x + 1));
    return r;
}

__device__ __forceinline__ u32 map3_of(i64 y) {
    u32 r = 0;
#pragma unroll
    for (int x = -1; x <= 1; ++x) {
        i64 c = (y + x) >> 32;  // arithmetic: floor
        r |= (u32)(c + 1) << (2 * (x + 1));
    }
    return r;
}

struct SignedNorm {
    i64 col_carry;  // carry of the previous chunk's last column (added to this chunk's first limb)
    int unit;       // resolved {-1,0,1} carry into this chunk
};

// cols: this lane's 4 column sums; out: digits.  State is warp-uniform.
__device__ __forceinline__ void warp_norm_signed(const i64 cols[4], SignedNorm& st, u32 out[4]) {
    const int lane = lane_id();
    i64 c[4];
    u32 d[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        d[j] = (u32)cols[j];
        c[j] = cols[j] >> 32;
    }
    i64 prev_c = __shfl_up_sync(FULL, c[3], 1);
    if (lane == 0) prev_c = st.col_carry;
    i64 y[4];
    y[0] = (i64)d[0] + prev_c;
#pragma unroll
    for (int j = 1; j < 4; ++j) y[j] = (i64)d[j] + c[j - 1];
    u32 f = map3_of(y[0]);
#pragma unroll
    for (int j = 1; j < 4; ++j) f = map3_compose(map3_of(y[j]), f);
    // inclusive scan of maps across lanes (lower lanes applied first)
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        u32 o = __shfl_up_sync(FULL, f, s);
        if (lane >= s) f = map3_compose(f, o);
    }
    int out_unit = map3_apply(f, st.unit);
    int x = __shfl_up_sync(FULL, out_unit, 1);
    if (lane == 0) x = st.unit;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        i64 v = y[j] + x;
        out[j] = (u32)v;
        x = (int)(v >> 32);
    }
    st.unit = __shfl_sync(FULL, out_unit, 31);
    st.col_carry = __shfl_sync(FULL, c[3], 31);
}

// ---------------------------------------------------------------------------
// Exact division by an odd constant d < 2^32 (multiply by d^-1 mod 2^32,
// Jebelean / Granlund-Montgomery style), chunk-parallel.
//
// Serial step on limb a with borrow B: x = a - B (mod 2^32), q = x d^-1,
// B' = hi32(q d) + [a < B].  For an exact quotient the borrow entering limb
// position p is B_p = (-(a mod 2^(32p)) 2^(-32p)) mod d, so across a lane of
// four limbs B_out = (B_out(0) + B_in rho^4) mod d with rho = 2^-32 mod d.
// That affine recurrence is scanned across the warp; then each lane reruns
// its four serial steps from its true borrow.
// ---------------------------------------------------------------------------
struct DivConst {
    u32 d;       // odd divisor (1 = no division)
    u32 inv;     // d^-1 mod 2^32
    u64 magic;   // floor(2^64 / d) for Barrett reduction
    u32 rk[5];   // (rho^4)^(2^i) mod d, i = 0..4
};

__device__ __forceinline__ u32 mod_reduce(u64 x, u32 d, u64 magic) {
    u64 q = __umul64hi(x, magic);
    u64 r = x - q * (u64)d;
    return (u32)(r >= d ? r - d : r);
}

__device__ __forceinline__ u32 mod_mul(u32 a, u32 b, u32 d, u64 magic) {
    return mod_reduce((u64)a * b, d, magic);
}

__device__ __forceinline__ u32 div_step(u32 a, u32 B, u32 d, u32 inv, u32& q) {
    u32 x = a - B;
    q = x * inv;
    return __umulhi(q, d) + (a < B ? 1u : 0u);
}

// In-place exact division of this warp's chunk v (4 limbs per lane).
// `borrow` is the warp-uniform borrow entering the chunk; updated on return.
__device__ __forceinline__ void warp_exact_div_chunk(u32 v[4], const DivConst& dc, u32& borrow) {
    const int lane = lane_id();
    u32 q;
    u32 b0 = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) b0 = div_step(v[j], b0, dc.d, dc.inv, q);
    u32 t = b0;
    if (lane == 0) {
        u32 x = mod_mul(borrow, dc.rk[0], dc.d, dc.magic) + t;
        t = x >= dc.d ? x - dc.d : x;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        int s = 1 << i;
        u32 o = __shfl_up_sync(FULL, t, s);
        if (lane >= s) {
            u32 x = mod_mul(o, dc.rk[i], dc.d, dc.magic) + t;
            t = x >= dc.d ? x - dc.d : x;
        }
    }
    u32 bin = __shfl_up_sync(FULL, t, 1);
    if (lane == 0) bin = borrow;
    u32 B = bin;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        B = div_step(v[j], B, dc.d, dc.inv, q);
        v[j] = q;
    }
    borrow = __shfl_sync(FULL, t, 31);
}

}  // namespace tc
