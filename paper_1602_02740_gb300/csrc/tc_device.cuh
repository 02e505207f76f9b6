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

// Asynchronous 4-byte copy global -> shared (no registers held while in flight);
// cp_async_wait_all() waits for this thread's copies, a barrier then publishes them.
__device__ __forceinline__ void cp_async4(u32* dst, const u32* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                 :: "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
// Asynchronous 16-byte copy global -> shared (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(u32* dst, const u32* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// all but the most recently committed group complete
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

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

// Normalisation of NON-NEGATIVE column sums (< 2^62): after adding each
// column's carry to the next digit every limb is below 2^32 + 2^30, so one
// binary carry-lookahead (generate: y >= 2^32, propagate: y = 2^32 - 1)
// finishes the job.
struct UnsignedNorm {
    u64 col_carry;  // carry of the previous chunk's last column
    u32 carry;      // 0/1 carry into this chunk
};

__device__ __forceinline__ u32 inc4(u32* r, u32 c);  // r += c over 4 limbs, the carry out

__device__ __forceinline__ void warp_norm_unsigned(const u64 cols[4], UnsignedNorm& st, u32 out[4]) {
    const int lane = lane_id();
    u64 c[4];
    u32 d[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        d[j] = (u32)cols[j];
        c[j] = cols[j] >> 32;
    }
    u64 prev_c = __shfl_up_sync(FULL, c[3], 1);
    if (lane == 0) prev_c = st.col_carry;
    u64 y[4];
    y[0] = (u64)d[0] + prev_c;
#pragma unroll
    for (int j = 1; j < 4; ++j) y[j] = (u64)d[j] + c[j - 1];
    // the lane's digits with carry-in 0 (y < 2^33 - 1, so every carry is 0 or 1);
    // then the carry out of the lane below, passed on only by an all-ones lane
    // (a lane that carried out itself is at most 2^128 - 2 after it), whose
    // chains a lookahead resolves when a vote finds any, as in warp_add_seg
    u32 x = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const u64 v = y[j] + x;
        out[j] = (u32)v;
        x = (u32)(v >> 32);
    }
    u32 cin = __shfl_up_sync(FULL, x, 1);
    if (lane == 0) cin = st.carry;
    const u32 o = inc4(out, cin);
    u32 cw = __shfl_sync(FULL, x | o, 31);
    if (__any_sync(FULL, o)) {
        u32 cout;
        const bool ones = (out[0] & out[1] & out[2] & out[3]) == FULL;
        const u32 e = warp_carry_scan(o != 0u, ones, 0u, &cout);
        inc4(out, e);
        cw |= cout;
    }
    st.carry = cw;
    st.col_carry = __shfl_sync(FULL, c[3], 31);
}

// ---------------------------------------------------------------------------
// Exact division by an odd constant d < 2^31 (multiply by d^-1 mod 2^32, the
// Jebelean / Granlund-Montgomery exact division), chunk-parallel.
//
// Serial step on limb a with borrow B: x = a - B (mod 2^32), q = x d^-1,
// B' = hi32(q d) + [a < B].  For an exact quotient the borrow entering limb
// position p is B_p = (-(a mod 2^(32p)) 2^(-32p)) mod d, so across a lane of
// KL limbs B_out = (B_out(0) + B_in rho^KL) mod d with rho = 2^-32 mod d.
// That affine recurrence, with the same multiplier in every lane, is scanned
// across the warp (Kogge-Stone, multiplier rho^(KL 2^i) at step i); then each
// lane reruns its serial steps from its true borrow.  The modular products
// of the scan use Montgomery reduction with R = 2^32.
// ---------------------------------------------------------------------------
struct DivConst {
    u32 d;       // odd divisor (1 = no division), d < 2^31
    u32 inv;     // d^-1 mod 2^32
    u32 ninv;    // -d^-1 mod 2^32
    u32 rkm[5];  // (rho^KL)^(2^i) 2^32 mod d: Montgomery form of the scan multipliers
    u32 unit;    // 1 when rho^KL = 1 (mod d) and d < 2^26: the scan is a plain sum
    u32 recip;   // floor((2^32 - 1) / d), for reductions of small sums mod d
};

// Montgomery product a b 2^-32 mod d for a, b < d < 2^31.
__device__ __forceinline__ u32 mont_mul(u32 a, u32 b, u32 d, u32 ninv) {
    const u64 t = (u64)a * b;
    const u32 m = (u32)t * ninv;
    const u64 u = ((u64)m * d + t) >> 32;  // t + m d < 2^64 since d < 2^31
    const u32 r = (u32)u;
    return r >= d ? r - d : r;
}

__device__ __forceinline__ u32 div_step(u32 a, u32 B, u32 d, u32 inv, u32& q) {
    const u32 x = a - B;
    q = x * inv;
    return __umulhi(q, d) + (a < B ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// The same primitives for KL limbs per lane (chunks of 32 KL limbs).
// ---------------------------------------------------------------------------
template <int KL>
__device__ __forceinline__ void ld_seg(const u32* p, u32 v[KL]) {
#pragma unroll
    for (int j = 0; j < KL; j += 4) {
        const uint4 q = ld4(p + j);
        v[j] = q.x; v[j + 1] = q.y; v[j + 2] = q.z; v[j + 3] = q.w;
    }
}

template <int KL>
__device__ __forceinline__ void st_seg(u32* p, const u32 v[KL]) {
#pragma unroll
    for (int j = 0; j < KL; j += 4) st4(p + j, v + j);
}

// KL limbs at `pos` of a row with `len` valid limbs (zeros beyond); row 16-byte aligned.
template <int KL>
__device__ __forceinline__ void ld_seg_masked(const u32* row, int pos, int len, u32 v[KL]) {
#pragma unroll
    for (int j = 0; j < KL; j += 4) ld4_masked(row, pos + j, len, v + j);
}

// Four-limb carry chains in PTX: r = a + b + cin (cin 0 or 1) returning the
// carry out, r = a - b - bin returning the borrow out, and r += c / r -= c for
// c in {0, 1}.  The incoming carry enters the flag through cin + (2^32 - 1).
__device__ __forceinline__ u32 add4c(const u32* a, const u32* b, u32 cin, u32* r) {
    u32 c;
    asm("{\n\t.reg .u32 t;\n\t"
        "add.cc.u32 t, %5, -1;\n\t"
        "addc.cc.u32 %0, %6, %10;\n\t"
        "addc.cc.u32 %1, %7, %11;\n\t"
        "addc.cc.u32 %2, %8, %12;\n\t"
        "addc.cc.u32 %3, %9, %13;\n\t"
        "addc.u32 %4, 0, 0;\n\t}"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(c)
        : "r"(cin), "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]),
          "r"(b[3]));
    return c;
}

__device__ __forceinline__ u32 sub4b(const u32* a, const u32* b, u32 bin, u32* r) {
    u32 c;
    asm("{\n\t.reg .u32 t;\n\t"
        "sub.cc.u32 t, 0, %5;\n\t"
        "subc.cc.u32 %0, %6, %10;\n\t"
        "subc.cc.u32 %1, %7, %11;\n\t"
        "subc.cc.u32 %2, %8, %12;\n\t"
        "subc.cc.u32 %3, %9, %13;\n\t"
        "subc.u32 %4, 0, 0;\n\t}"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(c)
        : "r"(bin), "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]),
          "r"(b[3]));
    return c & 1u;
}

__device__ __forceinline__ u32 inc4(u32* r, u32 c) {
    u32 o;
    asm("add.cc.u32 %0, %0, %5;\n\t"
        "addc.cc.u32 %1, %1, 0;\n\t"
        "addc.cc.u32 %2, %2, 0;\n\t"
        "addc.cc.u32 %3, %3, 0;\n\t"
        "addc.u32 %4, 0, 0;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "=r"(o)
        : "r"(c));
    return o;
}

__device__ __forceinline__ u32 dec4(u32* r, u32 c) {
    u32 o;
    asm("sub.cc.u32 %0, %0, %5;\n\t"
        "subc.cc.u32 %1, %1, 0;\n\t"
        "subc.cc.u32 %2, %2, 0;\n\t"
        "subc.cc.u32 %3, %3, 0;\n\t"
        "subc.u32 %4, 0, 0;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "=r"(o)
        : "r"(c));
    return o & 1u;
}

// r = a + b + cin over KL limbs (KL a multiple of 4); returns the carry out.
template <int KL>
__device__ __forceinline__ u32 add_seg(const u32 a[KL], const u32 b[KL], u32 cin, u32 r[KL]) {
    u32 c = cin;
#pragma unroll
    for (int j = 0; j < KL; j += 4) c = add4c(a + j, b + j, c, r + j);
    return c;
}

// r = a - b - bin over KL limbs; returns the borrow out.
template <int KL>
__device__ __forceinline__ u32 sub_seg(const u32 a[KL], const u32 b[KL], u32 bin, u32 r[KL]) {
    u32 c = bin;
#pragma unroll
    for (int j = 0; j < KL; j += 4) c = sub4b(a + j, b + j, c, r + j);
    return c;
}

template <int KL>
__device__ __forceinline__ void inc_seg(u32 r[KL], u32 c) {
#pragma unroll
    for (int j = 0; j < KL; j += 4) c = inc4(r + j, c);
}

template <int KL>
__device__ __forceinline__ void dec_seg(u32 r[KL], u32 c) {
#pragma unroll
    for (int j = 0; j < KL; j += 4) c = dec4(r + j, c);
}

template <int KL>
__device__ __forceinline__ bool zero_seg(const u32 r[KL]) {
    u32 x = 0;
#pragma unroll
    for (int j = 0; j < KL; ++j) x |= r[j];
    return x == 0u;
}

template <int KL>
__device__ __forceinline__ bool ones_seg(const u32 r[KL]) {
    u32 x = FULL;
#pragma unroll
    for (int j = 0; j < KL; ++j) x &= r[j];
    return x == FULL;
}

// r += c (c in {0, 1}) / r -= c over KL limbs, returning the carry / borrow out.
template <int KL>
__device__ __forceinline__ u32 inc_seg_out(u32 r[KL], u32 c) {
#pragma unroll
    for (int j = 0; j < KL; j += 4) c = inc4(r + j, c);
    return c;
}

template <int KL>
__device__ __forceinline__ u32 dec_seg_out(u32 r[KL], u32 c) {
#pragma unroll
    for (int j = 0; j < KL; j += 4) c = dec4(r + j, c);
    return c;
}

// Warp-wide add of two chunks of 32 KL limbs.  Each lane adds its KL limbs with
// carry-in 0 and then adds the carry out of the lane below (lane 0: the chunk's
// carry-in).  That is the whole carry unless a lane's sum was all ones and
// received a carry, which passes it on; when a vote finds such lanes (never on
// uniform data, common in structured values such as all-ones operands) one
// ballot lookahead finishes every chain.  A lane gives out at most one carry
// in total: one that produced a carry itself is not all ones after its
// carry-in.
template <int KL>
__device__ __forceinline__ void warp_add_seg(const u32 a[KL], const u32 b[KL], u32& carry, u32 r[KL]) {
    const int lane = lane_id();
    const u32 g = add_seg<KL>(a, b, 0u, r);
    u32 cin = __shfl_up_sync(FULL, g, 1);
    if (lane == 0) cin = carry;
    const u32 o = inc_seg_out<KL>(r, cin);
    u32 c = __shfl_sync(FULL, g | o, 31);
    if (__any_sync(FULL, o)) {
        // the rest of the chain in one lookahead: lanes that passed a carry on
        // generate, lanes now all ones propagate; each lane adds its extra carry
        u32 cout;
        const u32 x = warp_carry_scan(o != 0u, ones_seg<KL>(r), 0u, &cout);
        inc_seg<KL>(r, x);
        c |= cout;
    }
    carry = c;
}

// The same for r = a - b with borrows (a propagating lane: difference 0).
template <int KL>
__device__ __forceinline__ void warp_sub_seg(const u32 a[KL], const u32 b[KL], u32& borrow, u32 r[KL]) {
    const int lane = lane_id();
    const u32 g = sub_seg<KL>(a, b, 0u, r);
    u32 bin = __shfl_up_sync(FULL, g, 1);
    if (lane == 0) bin = borrow;
    const u32 o = dec_seg_out<KL>(r, bin);
    u32 c = __shfl_sync(FULL, g | o, 31);
    if (__any_sync(FULL, o)) {
        u32 bout;
        const u32 x = warp_carry_scan(o != 0u, zero_seg<KL>(r), 0u, &bout);
        dec_seg<KL>(r, x);
        c |= bout;
    }
    borrow = c;
}

// The same add and subtract with every lane's carry resolved by the lookahead
// scan in one step (no data-dependent rounds).
template <int KL>
__device__ __forceinline__ void warp_add_seg_scan(const u32 a[KL], const u32 b[KL], u32& carry, u32 r[KL]) {
    const u32 g = add_seg<KL>(a, b, 0u, r);
    const bool p = !g && ones_seg<KL>(r);
    u32 cout;
    const u32 cin = warp_carry_scan(g != 0u, p, carry, &cout);
    inc_seg<KL>(r, cin);
    carry = cout;
}

template <int KL>
__device__ __forceinline__ void warp_sub_seg_scan(const u32 a[KL], const u32 b[KL], u32& borrow, u32 r[KL]) {
    const u32 g = sub_seg<KL>(a, b, 0u, r);
    const bool p = !g && zero_seg<KL>(r);
    u32 bout;
    const u32 bin = warp_carry_scan(g != 0u, p, borrow, &bout);
    dec_seg<KL>(r, bin);
    borrow = bout;
}

// Two independent warp subtractions with the lookahead scan, interleaved step by
// step (the ballots of one between the instructions of the other).  The
// latency-bound two-warp interpolation uses the scan forms throughout: there
// they measured faster than the lane-by-lane rounds.
template <int KL>
__device__ __forceinline__ void warp_sub_seg2(const u32 a0[KL], const u32 b0[KL], u32& bor0, u32 r0[KL],
                                              const u32 a1[KL], const u32 b1[KL], u32& bor1, u32 r1[KL]) {
    const u32 g0 = sub_seg<KL>(a0, b0, 0u, r0);
    const u32 g1 = sub_seg<KL>(a1, b1, 0u, r1);
    const bool p0 = !g0 && zero_seg<KL>(r0);
    const bool p1 = !g1 && zero_seg<KL>(r1);
    u32 o0, o1;
    const u32 c0 = warp_carry_scan(g0 != 0u, p0, bor0, &o0);
    const u32 c1 = warp_carry_scan(g1 != 0u, p1, bor1, &o1);
    dec_seg<KL>(r0, c0);
    dec_seg<KL>(r1, c1);
    bor0 = o0;
    bor1 = o1;
}

// Exact division of a warp chunk of 32 KL limbs by dc.d (constants built for this KL).
// x mod d for x < 2^32, d odd (q below is floor(x / d) or at most two less).
__device__ __forceinline__ u32 mod_small(u32 x, u32 d, u32 recip) {
    const u32 q = __umulhi(x, recip);
    u32 r = x - q * d;
    r = r >= d ? r - d : r;
    return r >= d ? r - d : r;
}

template <int KL>
__device__ __forceinline__ void warp_exact_div_seg(u32 v[KL], const DivConst& dc, u32& borrow) {
    const int lane = lane_id();
    u32 q;
    u32 b0 = 0;
#pragma unroll
    for (int j = 0; j < KL; ++j) b0 = div_step(v[j], b0, dc.d, dc.inv, q);
    if (dc.unit) {
        // rho^KL = 1 (e.g. d = 2^m - 1 with m | 32 KL): a lane's borrow out is its own
        // b0 plus its borrow in, mod d, so the borrows are prefix sums (each b0 <= d,
        // so 32 of them plus the chunk's borrow stay below 2^32 for d < 2^26)
        u32 s = b0 + (lane == 0 ? borrow : 0u);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const int w = 1 << i;
            const u32 o = __shfl_up_sync(FULL, s, w);
            if (lane >= w) s += o;
        }
        s = mod_small(s, dc.d, dc.recip);
        u32 bin = __shfl_up_sync(FULL, s, 1);
        if (lane == 0) bin = borrow;
        u32 B = bin;
#pragma unroll
        for (int j = 0; j < KL; ++j) {
            B = div_step(v[j], B, dc.d, dc.inv, q);
            v[j] = q;
        }
        borrow = __shfl_sync(FULL, s, 31);
        return;
    }
    u32 t = b0;
    if (lane == 0) {
        const u32 x = mont_mul(borrow, dc.rkm[0], dc.d, dc.ninv) + t;
        t = x >= dc.d ? x - dc.d : x;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int s = 1 << i;
        const u32 o = __shfl_up_sync(FULL, t, s);
        if (lane >= s) {
            const u32 x = mont_mul(o, dc.rkm[i], dc.d, dc.ninv) + t;
            t = x >= dc.d ? x - dc.d : x;
        }
    }
    u32 bin = __shfl_up_sync(FULL, t, 1);
    if (lane == 0) bin = borrow;
    u32 B = bin;
#pragma unroll
    for (int j = 0; j < KL; ++j) {
        B = div_step(v[j], B, dc.d, dc.inv, q);
        v[j] = q;
    }
    borrow = __shfl_sync(FULL, t, 31);
}

// ---------------------------------------------------------------------------
// Block-wide normalisation of non-negative column sums (recomposition).
// ---------------------------------------------------------------------------
struct BlockNormState {
    u64 col_carry;  // carry of the previous chunk's last column
    u32 carry;      // resolved 0/1 carry into this chunk
};

// cols: this thread's 4 column sums (each < 2^62).  sh: >= 2*warps+... words of shared scratch.
static __device__ void block_norm_unsigned(const u64 cols[4], BlockNormState& st, u32 out[4], u32* sh) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    u64* sh_c = reinterpret_cast<u64*>(sh);           // [blockDim] last-column carries
    u32* sh_gp = sh + 2 * blockDim.x;                 // [nw] warp g/p bits, then [nw] warp carries
    u32 d[4];
    u64 c[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) { d[j] = (u32)cols[j]; c[j] = cols[j] >> 32; }
    sh_c[tid] = c[3];
    __syncthreads();
    const u64 prev_c = tid == 0 ? st.col_carry : sh_c[tid - 1];
    u64 y[4];
    y[0] = (u64)d[0] + prev_c;
#pragma unroll
    for (int j = 1; j < 4; ++j) y[j] = (u64)d[j] + c[j - 1];
    // per-limb generate (y >= 2^32) / propagate (y == 2^32 - 1), composed low to high
    bool g = false, p = true;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool gj = y[j] >> 32, pj = y[j] == 0xffffffffull;
        g = gj || (pj && g);
        p = pj && p;
    }
    u32 wout;
    warp_carry_scan(g, p, 0u, &wout);                 // warp aggregate with carry-in 0
    const bool wp = __ballot_sync(FULL, p) == FULL;
    if (lane == 0) sh_gp[warp] = (wout ? 1u : 0u) | (wp ? 2u : 0u);
    const u64 last_c = sh_c[blockDim.x - 1];
    __syncthreads();
    if (warp == 0) {
        // lanes past the last warp pass the carry through so lane 31 reports the block's carry
        const u32 v = lane < nw ? sh_gp[lane] : 2u;
        u32 bout;
        const u32 cin = warp_carry_scan((v & 1u) != 0, (v & 2u) != 0, st.carry, &bout);
        if (lane < nw) sh_gp[nw + lane] = cin;
        if (lane == 0) sh_gp[2 * nw] = bout;
    }
    __syncthreads();
    const u32 wcin = sh_gp[nw + warp];
    u32 dummy;
    u32 x = warp_carry_scan(g, p, wcin, &dummy);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const u64 v = y[j] + x;
        out[j] = (u32)v;
        x = (u32)(v >> 32);
    }
    const u32 new_carry = sh_gp[2 * nw];
    __syncthreads();
    st.carry = new_carry;
    st.col_carry = last_c;
}

}  // namespace tc
