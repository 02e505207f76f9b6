// Interpolation by the inverse Vandermonde matrix, specialised per degree.
//
// Section 3 ends with the direct alternative to the Newton loops: the
// coefficients w = (w_0, .., w_2n) of W satisfy V w = y with V[p][i] = x_p^i
// for the 2n+1 points x_p (0, +1, -1, +2, -2, .., +-2^(n-1); Section 6), so
// w = V^-1 y.  Row i of V^-1 over its common denominator D_i = 2^s_i d_i
// (d_i odd) is a fixed integer vector M_i, and
//
//     w_i = (sum_p M_ip W(x_p)) / (2^s_i d_i),
//
// one fused pass per coefficient: signed small-multiple sums of the point
// values, one exact division by d_i (multiplication by d_i^-1 with the lanes'
// borrows scanned), one right shift.  No combine step and no chain of
// dependent stages; more multiply-adds than the even-odd Newton route.
//
// Rows of V^-1 come from the Lagrange basis: column p of V^-1 holds the
// coefficients of prod_(q != p) (X - x_q) divided by prod_(q != p) (x_p - x_q),
// all in exact integer arithmetic on the host.  For n <= 5 every |M_ip| < 2^29,
// sum_p |M_ip| < 2^31 (so the 64-bit column sums of the 2n+1 terms cannot
// overflow), every d_i < 2^20 and every s_i <= 21; the kernel takes n <= 5 and
// values of at most 1024 limbs.
#include <cstring>
#include <mutex>

#include "../../include/tc.h"
#include "tc_ctx.h"
#include "tc_device.cuh"
#include "tc_internal.h"

namespace tc {

DivConst make_div_const(u32 d, int KL);

constexpr int MAT_MAXN = 5;
constexpr int MAT_MAXP = 2 * MAT_MAXN + 1;

struct MatTable {
    int np;                     // 2n + 1 points and coefficients
    int M[MAT_MAXP][MAT_MAXP];  // [coefficient i][point p]
    int shift[MAT_MAXP];        // s_i
    u32 odd[MAT_MAXP];          // d_i
    DivConst div[MAT_MAXP];     // constants for d_i at 4 limbs per lane
};

namespace {

typedef __int128 i128;

i128 iabs(i128 x) { return x < 0 ? -x : x; }
i128 gcd128(i128 a, i128 b) {
    a = iabs(a);
    b = iabs(b);
    while (b) {
        i128 r = a % b;
        a = b;
        b = r;
    }
    return a;
}

// Integer form of V^-1 for degree n (1 <= n <= MAT_MAXN); false if a bound fails.
bool build_mat(int n, MatTable& t) {
    std::memset(&t, 0, sizeof(t));
    const int np = 2 * n + 1;
    t.np = np;
    long long x[MAT_MAXP];
    x[0] = 0;
    for (int j = 0; j < n; ++j) {
        x[2 * j + 1] = 1ll << j;
        x[2 * j + 2] = -(1ll << j);
    }
    i128 num[MAT_MAXP][MAT_MAXP], den[MAT_MAXP];
    for (int p = 0; p < np; ++p) {
        i128 c[MAT_MAXP + 1] = {1};
        int deg = 0;
        i128 d = 1;
        for (int q = 0; q < np; ++q) {
            if (q == p) continue;
            // c(X) <- c(X) (X - x_q)
            for (int k = deg + 1; k >= 1; --k) c[k] = c[k - 1] - (i128)x[q] * c[k];
            c[0] = -(i128)x[q] * c[0];
            ++deg;
            d *= (i128)(x[p] - x[q]);
        }
        for (int i = 0; i < np; ++i) num[p][i] = c[i];
        den[p] = d;
    }
    for (int i = 0; i < np; ++i) {
        i128 D = 1;
        for (int p = 0; p < np; ++p) {
            if (num[p][i] == 0) continue;
            const i128 r = iabs(den[p]) / gcd128(num[p][i], den[p]);
            D = D / gcd128(D, r) * r;
        }
        for (int p = 0; p < np; ++p) {
            // M = num / den * D, exactly: den / gcd divides D
            const i128 g = num[p][i] ? gcd128(num[p][i], den[p]) : 1;
            const i128 m = (num[p][i] / g) * (D / (den[p] / g));
            if (iabs(m) >= ((i128)1 << 31)) return false;
            t.M[i][p] = (int)m;
        }
        int s = 0;
        while (!(D & 1)) {
            D >>= 1;
            ++s;
        }
        if (s >= 32 || D >= ((i128)1 << 31)) return false;
        t.shift[i] = s;
        t.odd[i] = (u32)D;
        t.div[i] = make_div_const((u32)D, 4);
    }
    return true;
}

const MatTable* mat_table(int n) {
    static MatTable tabs[MAT_MAXN + 1];
    static bool ok[MAT_MAXN + 1];
    static std::once_flag once;
    std::call_once(once, [] {
        for (int k = 1; k <= MAT_MAXN; ++k) ok[k] = build_mat(k, tabs[k]);
    });
    return (n >= 1 && n <= MAT_MAXN && ok[n]) ? &tabs[n] : nullptr;
}

}  // namespace

// One warp per product, streaming the values in 128-limb chunks.  Shared
// memory per warp: the current chunk of each of the 2N+1 point values, then
// 2N+1 slots of YM + 4 words for the coefficients, each stored shifted by
// (i b) mod 4 words so that the recomposition reads limb l - i b of it with
// one aligned 16-byte load.  For every chunk and every coefficient i the warp
// forms the positive and negative column sums of M_ip W(x_p), normalises both,
// subtracts, and divides exactly by d_i; the normalisation, subtraction and
// division states of every coefficient are carried from chunk to chunk in
// registers.  The right shifts by s_i (they read the limb above) run on the
// slots once all chunks are done.
template <int N, int NC>
__global__ void __launch_bounds__(128)
interp_matrix_kernel(const u32* __restrict__ y, long ystride, int len, const uint8_t* __restrict__ su,
                     const uint8_t* __restrict__ sv, u32* __restrict__ out, long out_stride,
                     int out_len, int b, MatTable mt, long P) {
    constexpr int NP = 2 * N + 1, C = 128, YM = NC * C, SLOT = YM + 4;
    extern __shared__ __align__(16) u32 msm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long k = (long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (k >= P) return;  // warp-uniform
    u32* stage = msm + (long)warp * NP * (C + SLOT);
    u32* slots = stage + NP * C;
    const u32* yk = y + k * NP * ystride;
    u32 negm = 0;  // bit p: W(x_p) < 0
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        bool sg = false;
        if (su) sg ^= su[k * NP + p] != 0;
        if (sv) sg ^= sv[k * NP + p] != 0;
        negm |= sg ? 1u << p : 0u;
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        u32* slot = slots + i * SLOT;
        if (lane < 4) slot[lane] = 0u;
        if (lane >= 28) slot[YM + lane - 28] = 0u;
    }
    UnsignedNorm npos[NP], nneg[NP];
    u32 bw[NP], dB[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        npos[i] = UnsignedNorm{0, 0};
        nneg[i] = UnsignedNorm{0, 0};
        bw[i] = 0;
        dB[i] = 0;
    }
    for (int c = 0; c < NC; ++c) {
        // this chunk of every point value, all copies in flight together
        __syncwarp();
#pragma unroll
        for (int r = 0; r < NP; ++r) {
            const u32* row = yk + r * ystride;
            const int pos = c * C + 4 * lane;
            const int left = len - pos;
            const unsigned bytes = left >= 4 ? 16u : left > 0 ? 4u * left : 0u;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                         :: "r"((unsigned)__cvta_generic_to_shared(stage + r * C + 4 * lane)),
                            "l"(bytes ? row + pos : row), "r"(bytes) : "memory");
        }
        cp_async_wait_all();
        __syncwarp();
        // D_i w_i = sum_p M_ip W(x_p), chunk c, then exact division by d_i
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            u64 pos[4] = {0, 0, 0, 0}, neg[4] = {0, 0, 0, 0};
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int m = mt.M[i][p];
                if (m == 0) continue;
                const u32 am = (u32)(m < 0 ? -m : m);
                const uint4 v = ld4(stage + p * C + 4 * lane);
                if ((m < 0) != (((negm >> p) & 1u) != 0)) {
                    neg[0] += (u64)v.x * am; neg[1] += (u64)v.y * am;
                    neg[2] += (u64)v.z * am; neg[3] += (u64)v.w * am;
                } else {
                    pos[0] += (u64)v.x * am; pos[1] += (u64)v.y * am;
                    pos[2] += (u64)v.z * am; pos[3] += (u64)v.w * am;
                }
            }
            u32 dp[4], dn[4], r[4];
            warp_norm_unsigned(pos, npos[i], dp);
            warp_norm_unsigned(neg, nneg[i], dn);
            warp_sub_seg<4>(dp, dn, bw[i], r);  // D_i w_i >= 0
            if (mt.odd[i] > 1) warp_exact_div_seg<4>(r, mt.div[i], dB[i]);
            u32* slot = slots + i * SLOT + ((i * b) & 3) + c * C + 4 * lane;
#pragma unroll
            for (int j = 0; j < 4; ++j) slot[j] = r[j];
        }
    }
    __syncwarp();
    // w_i = (D_i w_i / d_i) >> s_i, in place, chunks low to high
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const u32 sh = (u32)mt.shift[i];
        if (!sh) continue;
        u32* w = slots + i * SLOT + ((i * b) & 3);
        for (int c = 0; c < NC; ++c) {
            u32 v[5];
#pragma unroll
            for (int j = 0; j < 5; ++j) v[j] = w[c * C + 4 * lane + j];  // the limb above included
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 4; ++j) w[c * C + 4 * lane + j] = fshr(v[j], v[j + 1], sh);
            __syncwarp();
        }
    }
    __syncwarp();
    // ---- recompose out[l] = sum_i w_i[l - i b] ----
    u32* o = out + k * out_stride;
    const bool aligned = ((reinterpret_cast<uintptr_t>(o) & 15u) == 0);
    UnsignedNorm nst{0, 0};
    for (int base_l = 0; base_l < out_len; base_l += C) {
        u64 cols[4] = {0, 0, 0, 0};
        const int l0 = base_l + 4 * lane;
#pragma unroll
        for (int t = 0; t < NP; ++t) {
            if (base_l + C <= t * b || base_l >= t * b + YM) continue;  // warp-uniform
            const int dt = (t * b) & 3;
            const int x = l0 - t * b;  // x + dt is a multiple of 4
            if (x < -dt || x > YM - dt) continue;
            const uint4 q = ld4(slots + t * SLOT + dt + x);
            cols[0] += q.x; cols[1] += q.y; cols[2] += q.z; cols[3] += q.w;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (l0 + j >= out_len) cols[j] = 0;
        u32 d[4];
        warp_norm_unsigned(cols, nst, d);
        if (aligned && l0 + 4 <= out_len) {
            st4(o + l0, d);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (l0 + j < out_len) o[l0 + j] = d[j];
        }
    }
}

namespace {

template <int N, int NC>
cudaError_t launch_matrix(const LevelGeom& g, const u32* y, const uint8_t* su, const uint8_t* sv,
                          u32* out, long ldo, int out_len, long P, cudaStream_t st) {
    const MatTable* mt = mat_table(N);
    if (!mt) return cudaErrorInvalidValue;
    constexpr int NP = 2 * N + 1, YM = NC * 128;
    const size_t per_warp = (size_t)NP * (128 + YM + 4) * 4;
    static int regs_per_warp = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(interp_matrix_kernel<N, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
        cudaFuncAttributes fa;
        regs_per_warp = cudaFuncGetAttributes(&fa, interp_matrix_kernel<N, NC>) == cudaSuccess
                            ? (fa.numRegs + 7) / 8 * 8 * 32 : 128 * 32;
    });
    int wpb = 1, best = 0;
    for (int w = 1; w <= 4; ++w) {
        if (w * per_warp > 200 * 1024) break;
        int blocks = (int)((228 * 1024) / (w * per_warp + 1024));
        const int reg_blocks = 65536 / (w * regs_per_warp);
        if (blocks > reg_blocks) blocks = reg_blocks;
        if (blocks > 32) blocks = 32;
        if (blocks * w >= best) { best = blocks * w; wpb = w; }
    }
    if (best == 0) return cudaErrorInvalidConfiguration;
    const long grid = (P + wpb - 1) / wpb;
    interp_matrix_kernel<N, NC><<<(unsigned)grid, wpb * 32, wpb * per_warp, st>>>(
        y, (long)g.ystride, 2 * g.e, su, sv, out, ldo, out_len, g.b, *mt, P);
    return cudaGetLastError();
}

}  // namespace

// Values of 2e + 2 limbs (with room for the denominators' growth) in 128-limb
// chunks, rounded up to 1, 2, 4 or 8 chunks.
static int matrix_chunks(const LevelGeom& g) {
    const int c = (2 * g.e + 2 + 127) / 128;
    return c <= 1 ? 1 : c <= 2 ? 2 : c <= 4 ? 4 : c <= 8 ? 8 : 0;
}

bool matrix_interp_supported(const LevelGeom& g) {
    return g.n >= 1 && g.n <= MAT_MAXN && matrix_chunks(g) >= 1;
}

cudaError_t launch_interp_matrix(const LevelGeom& g, const u32* y, const uint8_t* su,
                                 const uint8_t* sv, u32* out, long ldo, int out_len, long P,
                                 cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (!matrix_interp_supported(g)) return cudaErrorInvalidValue;
    const int nc = matrix_chunks(g);
    const int ci = nc == 1 ? 0 : nc == 2 ? 1 : nc == 4 ? 2 : 3;
    switch (g.n * 4 + ci) {
#define TC_MATRIX_CASE(NN, CI, NCC) \
    case NN * 4 + CI: return launch_matrix<NN, NCC>(g, y, su, sv, out, ldo, out_len, P, st);
#define TC_MATRIX_N(NN) TC_MATRIX_CASE(NN, 0, 1) TC_MATRIX_CASE(NN, 1, 2) TC_MATRIX_CASE(NN, 2, 4) \
    TC_MATRIX_CASE(NN, 3, 8)
        TC_MATRIX_N(1) TC_MATRIX_N(2) TC_MATRIX_N(3) TC_MATRIX_N(4) TC_MATRIX_N(5)
#undef TC_MATRIX_N
#undef TC_MATRIX_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tc

extern "C" tc_status tc_interp_matrix_table(int B, int64_t* M, int* shift, uint32_t* odd) {
    if (B < 2 || B > tc::MAT_MAXN + 1 || !M || !shift || !odd) return TC_EINVAL;
    const tc::MatTable* t = tc::mat_table(B - 1);
    if (!t) return TC_EINVAL;
    const int np = t->np;
    for (int i = 0; i < np; ++i) {
        for (int p = 0; p < np; ++p) M[i * np + p] = t->M[i][p];
        shift[i] = t->shift[i];
        odd[i] = t->odd[i];
    }
    return TC_OK;
}

extern "C" tc_status tc_toom_interpolate_matrix(size_t count, size_t limbs, int B, const uint32_t* Y,
                                                size_t ystride, const uint8_t* SGN_U,
                                                const uint8_t* SGN_V, uint32_t* OUT, size_t ldo,
                                                void* stream) {
    if (count == 0) return TC_OK;
    if (!Y || !OUT || B < 2 || B > 32 || limbs == 0 || limbs > (1u << 30)) return TC_EINVAL;
    tc::LevelGeom g = tc::make_level((int)limbs, B);
    if (!tc::matrix_interp_supported(g)) return TC_EINVAL;
    if (ystride < (size_t)(2 * g.e) || ystride % 4) return TC_EINVAL;
    if (reinterpret_cast<uintptr_t>(Y) & 15u) return TC_EINVAL;
    if (count > 1 && ldo < 2 * limbs) return TC_EINVAL;
    g.ystride = (int)ystride;
    const cudaError_t e = tc::launch_interp_matrix(g, Y, SGN_U, SGN_V, OUT, (long)ldo, 2 * g.s,
                                                   (long)count, (cudaStream_t)stream);
    return e == cudaSuccess ? TC_OK : tc_fail_cuda(e);
}
