// Interpolation of levels with few, huge products, spread over the whole GPU.
//
// The Newton stages are the same as in toom.cu (even-odd combine, Theorem 3.2
// divided differences with exact division, Theorem 3.3 conversion,
// recomposition), but each stage is a pass over every (product, chain,
// segment) task of the level: one warp per task, segments of WSEG limbs.
// Carries, borrows and exact-division borrows cross segments through a
// decoupled look-back: a task publishes its segment's aggregate (computed
// with a zero carry-in), walks back over earlier segments of its chain until
// it can form its carry-in, publishes its inclusive carry-out, then recomputes
// its segment and writes it.  Tasks take tickets in segment-major order, so a
// task only ever waits on tasks that hold earlier tickets (already running or
// done).  Every wait is bounded; a wait that runs out sets an error word that
// the host checks, and the kernel moves on instead of hanging.
//
// All shifts read neighbouring limbs of fully written values, so no state
// other than the carries crosses a segment boundary.
#include <algorithm>
#include <vector>

#include "../../include/tc.h"
#include "tc_ctx.h"
#include "tc_device.cuh"
#include "tc_internal.h"

namespace tc {

constexpr int WSEG_CH = 16;            // warp chunks per segment
constexpr int WSEG = WSEG_CH * CH;     // limbs per segment
constexpr int WMAXCH = 64;             // chains per pass
constexpr u64 F_AGG = 1ull << 62, F_INCL = 2ull << 62, F_MASK = 3ull << 62;
constexpr int SPIN_LIMIT = 1 << 22;    // x >= 64 ns sleeps: about a quarter second

struct WideChain {
    const u32* X;  // product-0 base of the first operand
    const u32* Z;  // product-0 base of the second operand (add/sub only)
    u32* O;        // product-0 base of the output
    long sX, sZ, sO;  // per-product strides
    int lenX, lenZ;   // valid limbs (zero beyond)
    int op;           // add/sub: 0 add, 1 subtract; div: divisor index k (0 = none)
    int shift;        // add/sub: left shift of Z (< 64); div: right shift of X (< 64)
    int lenO;         // limbs written (multiple of 4); 0 = the pass's Y
    const uint8_t* swap;  // add/sub: per-product flag (stride sSwap): exchange X and Z
    long sSwap;
};

struct WidePass {
    int nch, nseg, Y;  // chains, segments per chain, limbs written per chain
    long P;            // products
    WideChain ch[WMAXCH];
};

struct WideDiv {
    u32 d, inv, ninv;
    u32 rkm[5];   // lane-scan multipliers (Montgomery form), as DivConst
    u32 segm;     // (2^-32)^WSEG * 2^32 mod d: one segment's multiplier, Montgomery form
    u32 onem;     // 2^32 mod d: Montgomery form of 1
};

struct WideDivTable {
    WideDiv d[2][32];
};

__device__ __forceinline__ u64 ld_acq(const u64* p) {
    u64 v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_rel(u64* p, u64 v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Failure-detection test settings of this device (tc_test_bounded_waits):
// g_wait_polls > 0 replaces SPIN_LIMIT; g_withhold != 0 makes the first segment
// of every add/subtract chain skip its publishes, so the waits behind it run out.
__device__ int g_wait_polls = 0;
__device__ int g_withhold = 0;

// Wait (bounded) until status word *p is published; returns it.
__device__ __forceinline__ u64 wait_status(const u64* p, int* err) {
    u64 v;
    int it = 0;
    const int limit = g_wait_polls > 0 ? g_wait_polls : SPIN_LIMIT;
    while (((v = ld_acq(p)) & F_MASK) == 0) {
        if (++it > limit) {
            atomicExch(err, 1);
            return F_INCL;  // give up: carry-in 0, result flagged invalid
        }
        __nanosleep(64);
    }
    return v;
}

__device__ __forceinline__ int next_ticket(int* counter) {
    int t = 0;
    if (lane_id() == 0) t = atomicAdd(counter, 1);
    return __shfl_sync(FULL, t, 0);
}

__device__ __forceinline__ u32 ldm(const u32* p, long x, int len) {
    return (x >= 0 && x < len) ? p[x] : 0u;
}

// ---------------------------------------------------------------------------
// add / subtract: O = X +- (Z << shift)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void addsub_chunk(const WideChain& C, const u32* X, const u32* Z, int pos,
                                             u32& carry, u32 r[4], bool& same) {
    const int lane = lane_id();
    const int l0 = pos + 4 * lane;
    u32 x[4], z[4];
    ld4_masked(X, l0, C.lenX, x);
    const int qa = C.shift >> 5, s = C.shift & 31;
    u32 w[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) w[q] = ldm(Z, (long)l0 - qa - 1 + q, C.lenZ);
#pragma unroll
    for (int j = 0; j < 4; ++j) z[j] = fshl(w[j], w[j + 1], (u32)s);
    if (C.op == 0) {
        warp_add_seg<4>(x, z, carry, r);
        same = same && (__ballot_sync(FULL, !ones_seg<4>(r)) == 0);
    } else {
        warp_sub_seg<4>(x, z, carry, r);
        same = same && (__ballot_sync(FULL, !zero_seg<4>(r)) == 0);
    }
}

__global__ void __launch_bounds__(128)
wide_addsub_kernel(WidePass wp, u64* status, int* counter, int* err) {
    const long total = wp.P * wp.nch * (long)wp.nseg;
    for (;;) {
        const long t = next_ticket(counter);
        if (t >= total) return;
        const int seg = (int)(t / (wp.P * wp.nch));
        const long rem = t - (long)seg * wp.P * wp.nch;
        const long p = rem / wp.nch;
        const int c = (int)(rem - p * wp.nch);
        WideChain C = wp.ch[c];
        if (C.swap && C.swap[p * C.sSwap]) {  // operands exchanged for this product
            const u32* tX = C.X; C.X = C.Z; C.Z = tX;
            const long ts = C.sX; C.sX = C.sZ; C.sZ = ts;
            const int tl = C.lenX; C.lenX = C.lenZ; C.lenZ = tl;
        }
        const u32* X = C.X + p * C.sX;
        const u32* Z = C.Z + p * C.sZ;
        u32* O = C.O + p * C.sO;
        const int lenO = C.lenO ? C.lenO : wp.Y;
        u64* st = status + (p * wp.nch + c) * wp.nseg;
        const int start = seg * WSEG;
        const int end = min(start + WSEG, wp.Y);
        // phase 1: aggregate with carry-in 0
        u32 carry = 0;
        bool same = true;
        u32 r[4];
        for (int pos = start; pos < end; pos += CH) addsub_chunk(C, X, Z, pos, carry, r, same);
        const u32 g = carry, pr = (!g && same) ? 1u : 0u;
        const bool publish = !(seg == 0 && g_withhold);
        if (lane_id() == 0 && publish) st_rel(st + seg, F_AGG | g | (pr << 1));
        // look back
        u32 cin = 0;
        if (lane_id() == 0) {
            for (int j = seg - 1; j >= 0; --j) {
                const u64 v = wait_status(st + j, err);
                if ((v & F_MASK) == F_INCL) { cin = (u32)(v & 1u); break; }
                if (v & 1u) { cin = 1; break; }          // generates
                if (!(v & 2u)) { cin = 0; break; }       // kills
            }
            if (publish) st_rel(st + seg, F_INCL | (g | (pr & cin)));
        }
        cin = __shfl_sync(FULL, cin, 0);
        // phase 2: with the true carry-in
        carry = cin;
        for (int pos = start; pos < end; pos += CH) {
            addsub_chunk(C, X, Z, pos, carry, r, same);
            const int l0 = pos + 4 * lane_id();
            if (l0 < lenO) st4(O + l0, r);
        }
    }
}

// ---------------------------------------------------------------------------
// shift right and divide: O = (X >> shift) / d_k (k = 0: shift only)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void shr_chunk(const WideChain& C, const u32* X, int pos, u32 v[4]) {
    const int l0 = pos + 4 * lane_id();
    const int qa = C.shift >> 5, r = C.shift & 31;
    u32 w[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) w[q] = ldm(X, (long)l0 + qa + q, C.lenX);
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = fshr(w[j], w[j + 1], (u32)r);
}

// Look-back for an exact-division borrow; returns this segment's borrow-in.
__device__ u32 div_lookback(u64* st, int seg, u32 bo0, const WideDiv& D, int* err) {
    u32 bin = 0;
    if (lane_id() == 0) {
        st_rel(st + seg, F_AGG | bo0);
        u32 acc = 0, mult = D.onem;
        for (int j = seg - 1; j >= 0; --j) {
            const u64 v = wait_status(st + j, err);
            const u32 x = (u32)v;
            const u32 add = mont_mul(mult, x, D.d, D.ninv);
            const u32 s = acc + add;
            acc = s >= D.d ? s - D.d : s;
            if ((v & F_MASK) == F_INCL) break;
            mult = mont_mul(mult, D.segm, D.d, D.ninv);
        }
        bin = acc;  // no inclusive predecessor: the chain's borrow-in is 0
        const u32 s = bo0 + mont_mul(D.segm, bin, D.d, D.ninv);
        st_rel(st + seg, F_INCL | (s >= D.d ? s - D.d : s));
    }
    return __shfl_sync(FULL, bin, 0);
}

__global__ void __launch_bounds__(128)
wide_shrdiv_kernel(WidePass wp, WideDivTable dt, u64* status1, u64* status2, int* counter, int* err) {
    const long total = wp.P * wp.nch * (long)wp.nseg;
    const int lane = lane_id();
    for (;;) {
        const long t = next_ticket(counter);
        if (t >= total) return;
        const int seg = (int)(t / (wp.P * wp.nch));
        const long rem = t - (long)seg * wp.P * wp.nch;
        const long p = rem / wp.nch;
        const int c = (int)(rem - p * wp.nch);
        const WideChain& C = wp.ch[c];
        const u32* X = C.X + p * C.sX;
        u32* O = C.O + p * C.sO;
        const int start = seg * WSEG;
        const int end = min(start + WSEG, wp.Y);
        const int k = C.op;
        const WideDiv& D1 = dt.d[0][k];
        const WideDiv& D2 = dt.d[1][k];
        const long sidx = (p * wp.nch + c) * wp.nseg;
        u32 v[4];
        if (D1.d <= 1) {  // plain shift
            for (int pos = start; pos < end; pos += CH) {
                shr_chunk(C, X, pos, v);
                st4(O + pos + 4 * lane, v);
            }
            continue;
        }
        DivConst dc1{D1.d, D1.inv, D1.ninv, {D1.rkm[0], D1.rkm[1], D1.rkm[2], D1.rkm[3], D1.rkm[4]}};
        u32 b = 0;
        for (int pos = start; pos < end; pos += CH) {
            shr_chunk(C, X, pos, v);
            warp_exact_div_seg<4>(v, dc1, b);
        }
        b = div_lookback(status1 + sidx, seg, b, D1, err);
        for (int pos = start; pos < end; pos += CH) {
            shr_chunk(C, X, pos, v);
            warp_exact_div_seg<4>(v, dc1, b);
            st4(O + pos + 4 * lane, v);
        }
        if (D2.d > 1) {
            __syncwarp();
            DivConst dc2{D2.d, D2.inv, D2.ninv, {D2.rkm[0], D2.rkm[1], D2.rkm[2], D2.rkm[3], D2.rkm[4]}};
            b = 0;
            for (int pos = start; pos < end; pos += CH) {
                const uint4 q = ld4(O + pos + 4 * lane);
                u32 w[4] = {q.x, q.y, q.z, q.w};
                warp_exact_div_seg<4>(w, dc2, b);
            }
            b = div_lookback(status2 + sidx, seg, b, D2, err);
            for (int pos = start; pos < end; pos += CH) {
                const uint4 q = ld4(O + pos + 4 * lane);
                u32 w[4] = {q.x, q.y, q.z, q.w};
                warp_exact_div_seg<4>(w, dc2, b);
                st4(O + pos + 4 * lane, w);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// even-odd combine, second half: ce_m = (neg ? D : A) >> 1,
// co_m = x_m (neg ? A : D) / 2 (x_m = 2^(m-1)); node 0: ce_0 = W(0), co_0 = 0.
// Limb-local given A and D.
// ---------------------------------------------------------------------------
struct EoArgs {
    const u32* y;          // child products, product-0 base
    long ystride;          // limbs between child products
    int npts, len;         // 2B - 1, 2e
    const uint8_t* su;
    const uint8_t* sv;
    const u32* AD;         // [2n][P][Y]: A_m at 2(m-1), D_m at 2(m-1) + 1
    u32* ce[33];           // product-0 bases
    u32* co[33];
    int n, Y;
    long P;
};

__global__ void __launch_bounds__(256) wide_eo_shift_kernel(EoArgs a) {
    const long per = (long)(a.n + 1) * (a.Y / 4);  // quads per product
    const long total = a.P * per;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const long p = q / per;
        const long r = q - p * per;
        const int m = (int)(r / (a.Y / 4));
        const int l0 = (int)(r - (long)m * (a.Y / 4)) * 4;
        u32* CE = a.ce[m] + p * a.Y;
        u32* CO = a.co[m] + p * a.Y;
        u32 e[4], o[4];
        if (m == 0) {
            const u32* y0 = a.y + p * a.npts * a.ystride;
#pragma unroll
            for (int j = 0; j < 4; ++j) { e[j] = ldm(y0, l0 + j, a.len); o[j] = 0; }
        } else {
            bool neg = false;
            const long si = p * a.npts + 2 * m;
            if (a.su) neg ^= a.su[si] != 0;
            if (a.sv) neg ^= a.sv[si] != 0;
            const u32* A = a.AD + ((long)(2 * (m - 1)) * a.P + p) * a.Y;
            const u32* D = a.AD + ((long)(2 * (m - 1) + 1) * a.P + p) * a.Y;
            const u32* E = neg ? D : A;
            const u32* Od = neg ? A : D;
            u32 w[5];
#pragma unroll
            for (int q2 = 0; q2 < 5; ++q2) w[q2] = ldm(E, l0 + q2, a.Y);
#pragma unroll
            for (int j = 0; j < 4; ++j) e[j] = fshr(w[j], w[j + 1], 1u);
            if (m == 1) {
#pragma unroll
                for (int q2 = 0; q2 < 5; ++q2) w[q2] = ldm(Od, l0 + q2, a.Y);
#pragma unroll
                for (int j = 0; j < 4; ++j) o[j] = fshr(w[j], w[j + 1], 1u);
            } else {
                const int sh = m - 2;
#pragma unroll
                for (int q2 = 0; q2 < 5; ++q2) w[q2] = ldm(Od, l0 - 1 + q2, a.Y);
#pragma unroll
                for (int j = 0; j < 4; ++j) o[j] = fshl(w[j], w[j + 1], (u32)sh);
            }
        }
        st4(CE + l0, e);
        st4(CO + l0, o);
    }
}

// ---------------------------------------------------------------------------
// recomposition: out = sum_t w_t 2^(32 b t) with a small-integer carry look-back.
// A segment's carry-out as a function of its carry-in C (0 <= C <= 63) is
// q + [C >= T]: T = 2^32 - (first digit) when every later digit is all ones,
// else never (T = 64).  Such maps compose in closed form.
// ---------------------------------------------------------------------------
struct RecArgs {
    const u32* w[65];  // product-0 bases of the 2n+1 coefficients
    int nterms, Y, b;
    long P;
    u32* out;
    long ostride;
    int out_len, nseg;
};

__device__ __forceinline__ void rec_compose(u32& q, u32& T, u32 q1, u32 T1) {
    // (q, T) := (q, T) after (q1, T1): apply (q1, T1) first
    const u32 nq = q + (q1 >= T ? 1u : 0u);
    const u32 nT = (q1 < T && q1 + 1 >= T) ? T1 : 64u;
    q = nq;
    T = nT;
}

// One segment-parallel column-normalisation task: out = digits of
// sum_l col(l) 2^(32 l) over [start, end), with the small-integer carry map
// look-back.  col(l) returns the (non-negative) column sum at limb l.
template <class ColFn>
__device__ void colnorm_task(ColFn col, u64* st, int seg, int start, int end, int out_len,
                             u32* out, int* err) {
    const int lane = lane_id();
    UnsignedNorm ns{0, 0};
    u32 d[4];
    u32 d0 = 0;
    bool rest_ones = true;
    for (int pos = start; pos < end; pos += CH) {
        u64 cols[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) cols[j] = col(pos + 4 * lane + j);
        warp_norm_unsigned(cols, ns, d);
        const int l0 = pos + 4 * lane;
        bool ok = true;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int l = l0 + j;
            if (l == start) d0 = d[j];
            else if (l < out_len && d[j] != FULL) ok = false;
        }
        rest_ones = rest_ones && (__ballot_sync(FULL, !ok) == 0);
    }
    d0 = __shfl_sync(FULL, d0, 0);
    const u32 q0 = (u32)ns.col_carry + ns.carry;
    const u32 T0 = rest_ones ? (d0 >= FULL - 62 ? (u32)(0x100000000ull - d0) : 64u) : 64u;
    u32 cin = 0;
    if (lane == 0) {
        st_rel(st + seg, F_AGG | ((u64)T0 << 32) | q0);
        u32 q = 0, T = 64;
        bool have = false;
        u32 base = 0;
        for (int j = seg - 1; j >= -1; --j) {
            u64 v;
            if (j < 0) v = F_INCL;  // carry into the first segment is 0
            else v = wait_status(st + j, err);
            const u32 qj = (u32)(v & 0xffffffffu), Tj = (u32)((v >> 32) & 0x3fffffffu);
            if ((v & F_MASK) == F_INCL) { base = (j < 0) ? 0u : qj; break; }
            if (!have) { q = qj; T = Tj; have = true; }
            else rec_compose(q, T, qj, Tj);  // older map applied first
        }
        cin = have ? q + (base >= T ? 1u : 0u) : base;
        st_rel(st + seg, F_INCL | (u64)(q0 + (cin >= T0 ? 1u : 0u)));
    }
    cin = __shfl_sync(FULL, cin, 0);
    ns.col_carry = cin;
    ns.carry = 0;
    const bool aligned = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
    for (int pos = start; pos < end; pos += CH) {
        u64 cols[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) cols[j] = col(pos + 4 * lane + j);
        warp_norm_unsigned(cols, ns, d);
        const int l0 = pos + 4 * lane;
        if (aligned && l0 + 4 <= out_len) {
            st4(out + l0, d);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (l0 + j < out_len) out[l0 + j] = d[j];
        }
    }
}

__global__ void __launch_bounds__(128) wide_recompose_kernel(RecArgs a, u64* status, int* counter, int* err) {
    const long total = a.P * (long)a.nseg;
    for (;;) {
        const long t = next_ticket(counter);
        if (t >= total) return;
        const int seg = (int)(t / a.P);
        const long p = t - (long)seg * a.P;
        const int start = seg * WSEG;
        const int end = min(start + WSEG, (a.out_len + CH - 1) / CH * CH);
        auto col = [&](int l) -> u64 {
            u64 S = 0;
            if (l < a.out_len) {
                int tt = l / a.b;
                if (tt > a.nterms - 1) tt = a.nterms - 1;
                for (; tt >= 0; --tt) {
                    const int x = l - tt * a.b;
                    if (x >= a.Y) break;
                    S += a.w[tt][p * a.Y + x];
                }
            }
            return S;
        };
        colnorm_task(col, status + p * a.nseg, seg, start, end, a.out_len, a.out + p * a.ostride, err);
    }
}

// ---------------------------------------------------------------------------
// Evaluation of few, huge operand rows: E_j and O_j (even and odd parts at
// x = 2^j, Section 4 eq. 4.1) normalised segment-parallel, the sign of E - O
// from the top differing limb, then U(x) = E + O and |U(-x)| by the add/sub
// pass, and U(0) = u_0 copied.
// ---------------------------------------------------------------------------
struct EvalNormArgs {
    const u32* in;
    long in_stride;
    int s, B, b, n, e;
    u32* EO;      // [2n][P][Ew]: E_j at 2j, O_j at 2j + 1
    int Ew;
    long P;
    int nseg;
};

__global__ void __launch_bounds__(128) wide_evalnorm_kernel(EvalNormArgs a, u64* status, int* counter, int* err) {
    const int nch = 2 * a.n;
    const long total = a.P * nch * (long)a.nseg;
    for (;;) {
        const long t = next_ticket(counter);
        if (t >= total) return;
        const int seg = (int)(t / (a.P * nch));
        const long rem = t - (long)seg * a.P * nch;
        const long p = rem / nch;
        const int c = (int)(rem - p * nch);
        const int j = c >> 1, parity = c & 1;
        const u32* row = a.in + p * a.in_stride;
        const int start = seg * WSEG;
        const int end = min(start + WSEG, a.Ew);
        auto col = [&](int l) -> u64 {
            u64 S = 0;
            if (l < a.e) {
                for (int i = parity; i < a.B; i += 2) {
                    const int sh = j * i, qa = sh >> 5, r = sh & 31;
                    const int xh = l - qa, xl = l - qa - 1;
                    const u32 hi = (xh >= 0 && xh < a.b && i * a.b + xh < a.s) ? __ldg(row + i * a.b + xh) : 0u;
                    const u32 lo = (xl >= 0 && xl < a.b && i * a.b + xl < a.s) ? __ldg(row + i * a.b + xl) : 0u;
                    S += fshl(lo, hi, (u32)r);
                }
            }
            return S;
        };
        colnorm_task(col, status + (p * nch + c) * a.nseg, seg, start, end, a.Ew,
                     a.EO + ((long)c * a.P + p) * a.Ew, err);
    }
}

// sign of E_j - O_j per (row, j): one block per pair, top differing limb
__global__ void __launch_bounds__(256) wide_evalsign_kernel(const u32* EO, int Ew, long P, int n,
                                                            uint8_t* swap, uint8_t* sgn, int npts) {
    const long pj = blockIdx.x;
    const long p = pj / n;
    const int j = (int)(pj - p * n);
    const u32* E = EO + ((long)(2 * j) * P + p) * Ew;
    const u32* O = EO + ((long)(2 * j + 1) * P + p) * Ew;
    __shared__ int best[8];
    int top = -1;
    for (int l = threadIdx.x; l < Ew; l += blockDim.x)
        if (E[l] != O[l]) top = l;
    for (int o = 16; o; o >>= 1) top = max(top, __shfl_xor_sync(FULL, top, o));
    if ((threadIdx.x & 31) == 0) best[threadIdx.x >> 5] = top;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = -1;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = max(t, best[w]);
        const bool neg = t >= 0 && O[t] > E[t];
        swap[p * n + j] = neg ? 1 : 0;
        sgn[p * npts + 2 * j + 1] = 0;
        sgn[p * npts + 2 * j + 2] = neg ? 1 : 0;
        if (j == 0) sgn[p * npts] = 0;
    }
}

// U(0) = u_0 into row 0 of each product's evaluations
__global__ void wide_evalzero_kernel(const u32* in, long in_stride, int s, int b, u32* out, int estride,
                                     int npts, long P) {
    const long total = P * (long)estride;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const long p = q / estride;
        const int l = (int)(q - p * estride);
        out[p * npts * (long)estride + l] = (l < b && l < s) ? in[p * in_stride + l] : 0u;
    }
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
static WideDivTable make_wide_div_table() {
    WideDivTable t;
    auto inv32 = [](u32 d) {
        u32 x = d;
        for (int i = 0; i < 5; ++i) x *= 2u - d * x;
        return x;
    };
    auto powmod = [](u64 b, u64 e, u64 m) {
        u64 r = 1 % m;
        b %= m;
        while (e) {
            if (e & 1) r = r * b % m;
            b = b * b % m;
            e >>= 1;
        }
        return r;
    };
    auto invmod = [](u64 a, u64 m) {
        long long r0 = (long long)m, r1 = (long long)(a % m), s0 = 0, s1 = 1;
        while (r1) {
            long long q = r0 / r1, x = r0 - q * r1;
            r0 = r1; r1 = x;
            x = s0 - q * s1; s0 = s1; s1 = x;
        }
        return (u64)((s0 % (long long)m + (long long)m) % (long long)m);
    };
    for (int k = 0; k < 32; ++k)
        for (int which = 0; which < 2; ++which) {
            u32 d = 1;
            if (which == 0 && k >= 1 && k < 16) d = (u32)((1ull << (2 * k)) - 1);
            if (k >= 16) d = which == 0 ? (u32)((1ull << k) - 1) : (u32)((1ull << k) + 1);
            WideDiv& w = t.d[which][k];
            w.d = d;
            w.inv = inv32(d);
            w.ninv = 0u - w.inv;
            for (int i = 0; i < 5; ++i) w.rkm[i] = 0;
            w.segm = w.onem = 0;
            if (d > 1) {
                u64 rk = invmod(powmod(2, 32ull * 4, d), d);  // rho^4 for 4 limbs per lane
                for (int i = 0; i < 5; ++i) {
                    w.rkm[i] = (u32)((rk << 32) % d);
                    rk = rk * rk % d;
                }
                const u64 seg = invmod(powmod(2, 32ull * WSEG, d), d);  // rho^WSEG
                w.segm = (u32)((seg << 32) % d);
                w.onem = (u32)((1ull << 32) % d);
            }
        }
    return t;
}

bool use_wide(const LevelGeom& g, long P) {
    return P * (long)(g.n + 1) < 152L * 4 && g.Y >= 8192;
}

// scratch: values 2(n+1) P Y limbs, temporaries 2n P Y limbs, status words,
// counters and an error word
size_t wide_work_bytes(const LevelGeom& g, long P) {
    const int Yw = (g.Y + WSEG - 1) / WSEG * WSEG;
    const long nseg_v = Yw / WSEG;
    const size_t vals = (size_t)(4 * g.n + 2) * P * Yw * 4;
    const int passes = 2 + 2 * g.n + (g.n - 1) + 1 + 4;
    const size_t stat = (size_t)passes * 2 * P * WMAXCH * (nseg_v + 8) * 8;
    return vals + stat + 4096;
}

// Error word of a wide level (set if a bounded wait gave up); inside `work`.
int* wide_error_word(void* work, const LevelGeom& g, long P) {
    const int Yw = (g.Y + WSEG - 1) / WSEG * WSEG;
    const long nseg_v = Yw / WSEG;
    const size_t vals = (size_t)(4 * g.n + 2) * P * Yw * 4;
    const int passes = 2 + 2 * g.n + (g.n - 1) + 1 + 4;
    const size_t stat = (size_t)passes * 2 * P * WMAXCH * (nseg_v + 8) * 8;
    return (int*)((char*)work + vals + stat + 2048);
}

bool use_wide_eval(const LevelGeom& g, long P) { return P * (long)g.n < 152L * 4 && g.e >= 4096; }

static size_t wide_eval_parts(const LevelGeom& g, long P, size_t* stat_off, size_t* swap_off,
                              size_t* cnt_off) {
    const int Ew = (g.e + WSEG - 1) / WSEG * WSEG;
    const long nseg = Ew / WSEG;
    size_t off = (size_t)2 * g.n * P * Ew * 4;
    *stat_off = off;
    off += (size_t)2 * P * 2 * g.n * nseg * 8;
    *swap_off = off;
    off += ((size_t)P * g.n + 255) / 256 * 256;
    *cnt_off = off;
    return off + 4096;
}

size_t wide_eval_work_bytes(const LevelGeom& g, long P) {
    size_t a, b, c;
    return wide_eval_parts(g, P, &a, &b, &c);
}

int* wide_eval_error_word(void* work, const LevelGeom& g, long P) {
    size_t a, b, c;
    wide_eval_parts(g, P, &a, &b, &c);
    return (int*)((char*)work + c + 2048);
}

cudaError_t launch_wide_eval(const u32* in, long in_stride, const LevelGeom& g, u32* out, uint8_t* sgn,
                             long P, void* work, cudaStream_t st) {
    note_kernel("wide_eval passes");
    size_t stat_off, swap_off, cnt_off;
    wide_eval_parts(g, P, &stat_off, &swap_off, &cnt_off);
    char* base = (char*)work;
    const int Ew = (g.e + WSEG - 1) / WSEG * WSEG;
    const int nseg = Ew / WSEG;
    const int n = g.n, npts = 2 * g.B - 1;
    u32* EO = (u32*)base;
    u64* stat = (u64*)(base + stat_off);
    const size_t stat_pass = (size_t)P * 2 * n * nseg;
    uint8_t* swap = (uint8_t*)(base + swap_off);
    int* cnt = (int*)(base + cnt_off);
    int* err = (int*)(base + cnt_off + 2048);
    cudaError_t e = cudaMemsetAsync(base + stat_off, 0, cnt_off - stat_off + 4096, st);
    if (e != cudaSuccess) return e;
    auto grid_for = [&](long tasks) {
        long b = (tasks + 3) / 4;
        return (unsigned)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
    };
    EvalNormArgs ea;
    ea.in = in; ea.in_stride = in_stride; ea.s = g.s; ea.B = g.B; ea.b = g.b; ea.n = n; ea.e = g.e;
    ea.EO = EO; ea.Ew = Ew; ea.P = P; ea.nseg = nseg;
    wide_evalnorm_kernel<<<grid_for(P * 2 * n * (long)nseg), 128, 0, st>>>(ea, stat, cnt, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    wide_evalsign_kernel<<<(unsigned)(P * n), 256, 0, st>>>(EO, Ew, P, n, swap, sgn, npts);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    WidePass wp;
    wp.nch = 2 * n; wp.nseg = nseg; wp.Y = Ew; wp.P = P;
    for (int j = 0; j < n; ++j)
        for (int pm = 0; pm < 2; ++pm) {
            WideChain& C = wp.ch[2 * j + pm];
            C.X = EO + (long)(2 * j) * P * Ew; C.sX = Ew; C.lenX = Ew;
            C.Z = EO + (long)(2 * j + 1) * P * Ew; C.sZ = Ew; C.lenZ = Ew;
            C.O = out + (long)(2 * j + 1 + pm) * g.estride; C.sO = (long)npts * g.estride;
            C.lenO = g.estride;
            C.op = pm;          // U(x) = E + O; |U(-x)| = E - O, operands exchanged when negative
            C.shift = 0;
            C.swap = pm ? swap + j : nullptr;
            C.sSwap = n;
        }
    wide_addsub_kernel<<<grid_for(P * 2 * n * (long)nseg), 128, 0, st>>>(wp, stat + stat_pass, cnt + 1, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long tot = P * (long)g.estride;
    wide_evalzero_kernel<<<(unsigned)std::min<long>((tot + 255) / 256, 152 * 32), 256, 0, st>>>(
        in, in_stride, g.s, g.b, out, g.estride, npts, P);
    return cudaGetLastError();
}

cudaError_t launch_wide_interp(const LevelGeom& g, const u32* y, const uint8_t* su, const uint8_t* sv,
                               u32* out, long out_stride, int out_len, void* work, long P,
                               cudaStream_t st) {
    note_kernel("wide_interp passes");
    int* err_dev = wide_error_word(work, g, P);
    static const WideDivTable dt = make_wide_div_table();
    const int n = g.n;
    const int Yw = (g.Y + WSEG - 1) / WSEG * WSEG;   // value length, whole segments
    const int nseg = Yw / WSEG;
    char* base = (char*)work;
    auto value = [&](int idx) { return (u32*)(base + (size_t)idx * P * Yw * 4); };
    // values 0 .. 2n+1: ce[0..n] then co[0..n]; temporaries from 2n+2
    u32* ce[33];
    u32* co[33];
    for (int m = 0; m <= n; ++m) { ce[m] = value(m); co[m] = value(n + 1 + m); }
    u32* tmp[64];
    for (int i = 0; i < 2 * n; ++i) tmp[i] = value(2 * n + 2 + i);
    char* sbase = base + (size_t)(4 * n + 2) * P * Yw * 4;
    const int passes = 2 + 2 * n + (n - 1) + 1 + 4;
    const size_t stat_per_pass = (size_t)2 * P * WMAXCH * (nseg + 8);
    u64* status = (u64*)sbase;
    int* counters = (int*)(sbase + passes * stat_per_pass * 8);
    cudaError_t e = cudaMemsetAsync(sbase, 0, passes * stat_per_pass * 8 + 4096, st);
    if (e != cudaSuccess) return e;
    int pass = 0;
    auto grid_for = [&](long tasks) {
        long b = (tasks + 3) / 4;
        return (unsigned)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
    };
    auto run_addsub = [&](WidePass& wp) -> cudaError_t {
        u64* s1 = status + (size_t)pass * stat_per_pass;
        int* cnt = counters + pass;
        ++pass;
        wide_addsub_kernel<<<grid_for(wp.P * wp.nch * (long)wp.nseg), 128, 0, st>>>(wp, s1, cnt, err_dev);
        return cudaGetLastError();
    };
    auto run_shrdiv = [&](WidePass& wp) -> cudaError_t {
        u64* s1 = status + (size_t)pass * stat_per_pass;
        u64* s2 = s1 + stat_per_pass / 2;
        int* cnt = counters + pass;
        ++pass;
        wide_shrdiv_kernel<<<grid_for(wp.P * wp.nch * (long)wp.nseg), 128, 0, st>>>(wp, dt, s1, s2, cnt, err_dev);
        return cudaGetLastError();
    };
    const long ys = (long)(2 * g.B - 1) * g.ystride;  // child products per parent product
    // ---- even-odd: A_m = W(x) + |W(-x)|, D_m = W(x) - |W(-x)| ----
    {
        WidePass wp;
        wp.nch = 2 * n; wp.nseg = nseg; wp.Y = Yw; wp.P = P;
        for (int m = 1; m <= n; ++m)
            for (int s2 = 0; s2 < 2; ++s2) {
                WideChain& C = wp.ch[2 * (m - 1) + s2];
                C.X = y + (long)(2 * m - 1) * g.ystride; C.sX = ys; C.lenX = 2 * g.e;
                C.Z = y + (long)(2 * m) * g.ystride; C.sZ = ys; C.lenZ = 2 * g.e;
                C.O = tmp[0] + (long)(2 * (m - 1) + s2) * P * Yw; C.sO = Yw;
                C.op = s2; C.shift = 0; C.lenO = 0; C.swap = nullptr; C.sSwap = 0;
            }
        // A/D occupy tmp[0 .. 2n) as one [2n][P][Yw] array
        if ((e = run_addsub(wp)) != cudaSuccess) return e;
        EoArgs ea;
        ea.y = y; ea.ystride = g.ystride; ea.npts = 2 * g.B - 1; ea.len = 2 * g.e;
        ea.su = su; ea.sv = sv; ea.AD = tmp[0]; ea.n = n; ea.Y = Yw; ea.P = P;
        for (int m = 0; m <= n; ++m) { ea.ce[m] = ce[m]; ea.co[m] = co[m]; }
        const long quads = P * (long)(n + 1) * (Yw / 4);
        wide_eo_shift_kernel<<<(unsigned)std::min<long>((quads + 255) / 256, 152 * 32), 256, 0, st>>>(ea);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // ---- Newton loop 1 (Theorem 3.2) ----
    for (int k = 1; k <= n; ++k) {
        const int cnt = n - k + 1;
        WidePass ws, wd;
        ws.nch = wd.nch = 2 * cnt; ws.nseg = wd.nseg = nseg; ws.Y = wd.Y = Yw; ws.P = wd.P = P;
        for (int i = 0; i < cnt; ++i) {
            const int m = k + i;
            for (int poly = 0; poly < 2; ++poly) {
                u32** c = poly ? co : ce;
                WideChain& S = ws.ch[2 * i + poly];
                S.X = c[m]; S.sX = Yw; S.lenX = Yw;
                S.Z = c[m - 1]; S.sZ = Yw; S.lenZ = Yw;
                S.O = tmp[2 * i + poly]; S.sO = Yw; S.op = 1; S.shift = 0;
                S.lenO = 0; S.swap = nullptr; S.sSwap = 0;
                WideChain& Dv = wd.ch[2 * i + poly];
                Dv.lenO = 0; Dv.swap = nullptr; Dv.sSwap = 0;
                Dv.X = tmp[2 * i + poly]; Dv.sX = Yw; Dv.lenX = Yw;
                Dv.Z = nullptr; Dv.sZ = 0; Dv.lenZ = 0;
                Dv.O = c[m]; Dv.sO = Yw;
                Dv.shift = m == k ? 2 * (m - 1) : 2 * (m - k - 1);
                Dv.op = m == k ? 0 : k;
            }
        }
        if ((e = run_addsub(ws)) != cudaSuccess) return e;
        if ((e = run_shrdiv(wd)) != cudaSuccess) return e;
    }
    // ---- Newton loop 2 (Theorem 3.3): c[k] -= 4^(m-1) c[k+1], into temporaries, then swap ----
    for (int m = n - 1; m >= 1; --m) {
        const int cnt = n - m;
        WidePass ws;
        ws.nch = 2 * cnt; ws.nseg = nseg; ws.Y = Yw; ws.P = P;
        for (int i = 0; i < cnt; ++i) {
            const int kx = m + i;
            for (int poly = 0; poly < 2; ++poly) {
                u32** c = poly ? co : ce;
                WideChain& S = ws.ch[2 * i + poly];
                S.X = c[kx]; S.sX = Yw; S.lenX = Yw;
                S.Z = c[kx + 1]; S.sZ = Yw; S.lenZ = Yw;
                S.O = tmp[2 * i + poly]; S.sO = Yw; S.op = 1; S.shift = 2 * (m - 1);
                S.lenO = 0; S.swap = nullptr; S.sSwap = 0;
            }
        }
        if ((e = run_addsub(ws)) != cudaSuccess) return e;
        for (int i = 0; i < cnt; ++i) {
            const int kx = m + i;
            std::swap(ce[kx], tmp[2 * i]);
            std::swap(co[kx], tmp[2 * i + 1]);
        }
    }
    // ---- recomposition ----
    {
        RecArgs ra;
        ra.nterms = 2 * n + 1; ra.Y = Yw; ra.b = g.b; ra.P = P; ra.out = out; ra.ostride = out_stride;
        ra.out_len = out_len;
        ra.nseg = ((out_len + CH - 1) / CH * CH + WSEG - 1) / WSEG;
        for (int t = 0; t <= 2 * n; ++t) ra.w[t] = (t & 1) ? co[(t + 1) >> 1] : ce[t >> 1];
        u64* s1 = status + (size_t)pass * stat_per_pass;
        int* cnt = counters + pass;
        ++pass;
        wide_recompose_kernel<<<grid_for(P * (long)ra.nseg), 128, 0, st>>>(ra, s1, cnt, err_dev);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace tc

extern "C" tc_status tc_test_bounded_waits(int polls, int withhold) {
    if (polls < 0) return TC_EINVAL;
    const int w = withhold ? 1 : 0;
    cudaError_t e = cudaMemcpyToSymbol(tc::g_wait_polls, &polls, sizeof polls);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(tc::g_withhold, &w, sizeof w);
    return e == cudaSuccess ? TC_OK : tc_fail_cuda(e);
}
