// Base-case product: batched schoolbook on CUDA cores.
//
// Below the last Toom level the pointwise products are formed directly (the
// paper uses a plain multiply below its Toom threshold, Section 6).  Each CTA
// handles one or more products of s x s limbs held in shared memory.
//
// Work split.  The partial products a_i b_j live on the parallelogram
// 0 <= i < s, i <= c = i + j < i + s.  Rows are cut into blocks of H rows and
// each block's columns into tiles of 4, so a thread computes H x 4 products
// that all land in 4 known columns: every thread does the same work (no
// triangle imbalance) and the only waste is the zero-padded corners of each
// row block.  Per column a thread keeps a 96-bit Comba accumulator updated by
// mad.lo.cc / madc.hi.cc / addc (two 32-bit multiplies per limb product).
// Four rows of a (one 16-byte load, shared by the tiles of a row block) and
// eight limbs of b (two 16-byte loads) feed 16 limb products.
//
// Reduction.  Tiles write their column accumulators to shared memory, one
// window of columns per row block; then every warp takes 128-column chunks of
// the products, sums the row blocks per output limb and normalises the chunk,
// one lane per product adds each chunk's carry into the next, and the block
// writes the limbs out.
#include <mutex>

#include "../../include/tc.h"
#include "tc_device.cuh"
#include "tc_internal.h"

namespace tc {

__device__ __forceinline__ void mac96(u32& lo, u32& mid, u32& hi, u32 a, u32 b) {
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(lo), "+r"(mid), "+r"(hi)
        : "r"(a), "r"(b));
}

struct LeafGeom {
    int s, H;
    int s_pad;   // roundup(s, H)
    int RB;      // row blocks
    int CT;      // column tiles per row block
    int NW;      // column window per row block = 4 * CT
    int sa_len, sb_len, sb_off;
    int words;   // shared words per product
};

static LeafGeom leaf_geom(int s) {
    LeafGeom g;
    g.s = s;
    g.H = s <= 48 ? 8 : s <= 256 ? 16 : s <= 512 ? 32 : 64;
    g.s_pad = (s + g.H - 1) / g.H * g.H;
    g.RB = g.s_pad / g.H;
    g.CT = (g.H + s - 1 + 3) / 4;
    g.NW = 4 * g.CT;
    g.sa_len = g.s_pad;
    g.sb_off = g.H;
    g.sb_len = g.H + g.NW + 4;
    g.words = g.sa_len + g.sb_len + 3 * g.RB * g.NW;
    return g;
}

__global__ void __launch_bounds__(256)
leaf_kernel(const u32* __restrict__ A, long lda, const u32* __restrict__ Bm, long ldb,
            u32* __restrict__ OUT, long ldo, LeafGeom g, long P, int ppc) {
    extern __shared__ __align__(16) u32 sm[];
    const int tid = threadIdx.x, nt = blockDim.x;
    const long p0 = (long)blockIdx.x * ppc;
    const int np = (int)min((long)ppc, P - p0);

    for (int k = 0; k < np; ++k) {
        u32* sa = sm + k * g.words;
        u32* sb = sa + g.sa_len;
        u32* part = sb + g.sb_len;
        const u32* a = A + (p0 + k) * lda;
        const u32* b = Bm + (p0 + k) * ldb;
        for (int i = tid; i < g.sa_len; i += nt) sa[i] = i < g.s ? a[i] : 0u;
        for (int i = tid; i < g.sb_len; i += nt) {
            int j = i - g.sb_off;
            sb[i] = (j >= 0 && j < g.s) ? b[j] : 0u;
        }
        for (int i = tid; i < 3 * g.RB * g.NW; i += nt) part[i] = 0u;
    }
    __syncthreads();

    const int tiles = g.RB * g.CT;
    for (int T = tid; T < np * tiles; T += nt) {
        const int k = T / tiles;
        const int rem = T - k * tiles;
        const int r = rem / g.CT;
        const int q = rem - r * g.CT;
        const u32* sa = sm + k * g.words;
        const u32* sb = sa + g.sa_len;
        u32* part = const_cast<u32*>(sb) + g.sb_len;
        u32 lo[4] = {0, 0, 0, 0}, mid[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0};
        for (int grp = 0; grp < g.H / 4; ++grp) {
            const int i0 = r * g.H + 4 * grp;
            uint4 av = *reinterpret_cast<const uint4*>(sa + i0);
            const int jb = g.sb_off + 4 * q - 4 * grp - 4;
            uint4 b0 = *reinterpret_cast<const uint4*>(sb + jb);
            uint4 b1 = *reinterpret_cast<const uint4*>(sb + jb + 4);
            const u32 a4[4] = {av.x, av.y, av.z, av.w};
            const u32 b8[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int rho = 0; rho < 4; ++rho)
#pragma unroll
                for (int w = 0; w < 4; ++w) mac96(lo[w], mid[w], hi[w], a4[rho], b8[4 + w - rho]);
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int cw = 4 * q + w;  // column offset within the row block's window
            part[(0 * g.RB + r) * g.NW + cw] = lo[w];
            part[(1 * g.RB + r) * g.NW + cw] = mid[w];
            part[(2 * g.RB + r) * g.NW + cw] = hi[w];
        }
    }
    __syncthreads();

    // Reduction, chunk-parallel: every warp takes (product, 128-column chunk) items,
    // sums the row blocks' columns and normalises the chunk with carry-in 0 into the
    // product's staging rows (dead after the tile pass; they hold 2s + 2H + 3 words);
    // then one lane per product adds each chunk's carry out into the next chunk (it
    // rarely ripples past a limb or two), and the block copies the limbs out.
    const int warp = tid >> 5, nwarps = nt >> 5, lane = tid & 31;
    const int out_len = 2 * g.s;
    const int nch = (out_len + CH - 1) / CH;
    for (int item = warp; item < np * nch; item += nwarps) {
        const int k = item / nch, ch = item - k * nch;
        const u32* part = sm + k * g.words + g.sa_len + g.sb_len;
        u32* dig = sm + k * g.words;          // 2s digits, then the chunks' carries
        u64 cols[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int c = ch * CH + 4 * lane + jj;
            u64 S = 0;
            for (int r = 0; r < g.RB; ++r) {
                const int x = c - r * g.H;
                if (x >= 0 && x < g.NW) S += part[(0 * g.RB + r) * g.NW + x];
                if (x - 1 >= 0 && x - 1 < g.NW) S += part[(1 * g.RB + r) * g.NW + x - 1];
                if (x - 2 >= 0 && x - 2 < g.NW) S += part[(2 * g.RB + r) * g.NW + x - 2];
            }
            cols[jj] = c < out_len ? S : 0;
        }
        UnsignedNorm st{0, 0};
        u32 d[4];
        warp_norm_unsigned(cols, st, d);
        const int pos = ch * CH + 4 * lane;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
            if (pos + jj < out_len) dig[pos + jj] = d[jj];
        if (lane == 0) {  // carry out of the chunk: the last column's high part plus the carry bit
            const u64 E = st.col_carry + st.carry;
            dig[out_len + 2 * ch] = (u32)E;
            dig[out_len + 2 * ch + 1] = (u32)(E >> 32);
        }
    }
    __syncthreads();
    for (int k = tid >> 5; k < np && lane == 0; k += nwarps) {
        u32* dig = sm + k * g.words;
        u64 E = 0;
        for (int ch = 0; ch + 1 < nch; ++ch) {
            E += (u64)dig[out_len + 2 * ch] | ((u64)dig[out_len + 2 * ch + 1] << 32);
            for (int i = (ch + 1) * CH; E != 0 && i < out_len; ++i) {
                if (i == (ch + 2) * CH) break;  // ran off this chunk: joins the next carry
                const u64 v = (u64)dig[i] + E;
                dig[i] = (u32)v;
                E = v >> 32;
            }
        }
    }
    __syncthreads();
    for (int k = 0; k < np; ++k) {
        const u32* dig = sm + k * g.words;
        u32* out = OUT + (p0 + k) * ldo;
        for (int i = tid; i < out_len; i += nt) out[i] = dig[i];
    }
}

// ---------------------------------------------------------------------------
// Lane-per-product schoolbook for large batches.
//
// A warp holds 32 independent products, one per lane, so all lanes follow the
// same schedule.  A lane walks the 8x8 tiles (I, J) of its product one
// anti-diagonal D = I + J at a time; tile products land in columns
// 8D .. 8D+14, kept as fifteen 96-bit Comba accumulators in registers.  Once
// anti-diagonal D is done, columns 8D .. 8D+7 are final: the lane folds them
// into a running 64-bit carry, writes eight result limbs and slides the
// window by eight columns.  Operand slices come straight from global memory
// as 32-byte vectors (L1-resident: a warp touches 32 x 2s limbs).
//
// Squaring (a == b) accumulates only the products a_i a_j with i < j and
// doubles them at emission, adding the squares a_i^2 on the even columns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load8(const u32* row, int pos, int s, bool vec, u32 v[8]) {
    if (vec && pos + 8 <= s) {
        const uint4 x = *reinterpret_cast<const uint4*>(row + pos);
        const uint4 y = *reinterpret_cast<const uint4*>(row + pos + 4);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
        v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = (pos + k < s) ? row[pos + k] : 0u;
    }
}

template <bool SQ>
__global__ void __launch_bounds__(128)
leaf_lane_kernel(const u32* __restrict__ A, long lda, const u32* __restrict__ Bm, long ldb,
                 u32* __restrict__ OUT, long ldo, int s, long P, int vec) {
    const long p0 = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = p0 < P;
    const long p = active ? p0 : P - 1;
    const u32* a = A + p * lda;
    const u32* b = SQ ? a : Bm + p * ldb;
    u32* out = OUT + p * ldo;
    const int T = (s + 7) / 8;
    const int out_len = 2 * s;
    u32 lo[15], mid[15], hi[15];
#pragma unroll
    for (int k = 0; k < 15; ++k) { lo[k] = 0; mid[k] = 0; hi[k] = 0; }
    u64 carry = 0;
    for (int D = 0; D <= 2 * T - 2; ++D) {
        const int Ilo = D - T + 1 > 0 ? D - T + 1 : 0;
        const int Ihi = D < T - 1 ? D : T - 1;
        for (int I = Ilo; I <= Ihi; ++I) {
            const int J = D - I;
            if (SQ && I > J) break;
            u32 a8[8], b8[8];
            load8(a, 8 * I, s, vec, a8);
            load8(b, 8 * J, s, vec, b8);
            if (SQ && I == J) {
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int c = r + 1; c < 8; ++c) mac96(lo[r + c], mid[r + c], hi[r + c], a8[r], b8[c]);
            } else {
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) mac96(lo[r + c], mid[r + c], hi[r + c], a8[r], b8[c]);
            }
        }
        // columns 8D .. 8D+7 are complete (8D .. 8D+14 when D is the last)
        const bool last = D == 2 * T - 2;
        u32 sq8[8];
        if (SQ) load8(a, 4 * D, s, false, sq8);  // a_(4D + k/2) for the even columns
#pragma unroll
        for (int k = 0; k < 15; ++k) {
            if (k >= 8 && !last) break;
            u64 vlo = lo[k], vmid = mid[k], vhi = hi[k];
            if (SQ) {
                // 2 (lo + mid 2^32 + hi 2^64) + a_(c/2)^2 on even columns c = 8D + k
                vhi = (vhi << 1) | (vmid >> 31);
                vmid = ((vmid << 1) & 0xffffffffull) | (vlo >> 31);
                vlo = (vlo << 1) & 0xffffffffull;
                if ((k & 1) == 0) {
                    const int i = 4 * D + k / 2;
                    u32 x = 0;
                    if (k < 8) x = sq8[k / 2];
                    else if (i < s) x = a[i];
                    const u64 sqv = (u64)x * x;
                    vlo += sqv & 0xffffffffull;
                    vmid += sqv >> 32;
                }
            }
            const u64 t = vlo + (carry & 0xffffffffull);
            const int c = 8 * D + k;
            if (active && c < out_len) out[c] = (u32)t;
            carry = (carry >> 32) + (t >> 32) + vmid + (vhi << 32);
        }
        if (last) {
            const int c = 8 * D + 15;
            if (active && c < out_len) out[c] = (u32)carry;
        }
#pragma unroll
        for (int k = 0; k < 15; ++k) {
            lo[k] = k + 8 < 15 ? lo[k + 8] : 0u;
            mid[k] = k + 8 < 15 ? mid[k + 8] : 0u;
            hi[k] = k + 8 < 15 ? hi[k + 8] : 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// Plain schoolbook for operands of any length (the comparison path).
//
// A block owns 1024 consecutive output columns of one product and walks every
// row that reaches them, 256 rows at a time: the 256 limbs of a and the
// matching 1284-limb window of b are staged in shared memory and each thread
// accumulates its 4 columns with the same 4 x 4 Comba step as the tile kernel.
// The 96-bit column sums go to a column buffer; one block per product then
// folds them into limbs with a block-wide carry scan.
// ---------------------------------------------------------------------------
constexpr int BIG_COLS = 1024, BIG_ROWS = 256;

__global__ void __launch_bounds__(256)
bigmul_columns_kernel(const u32* __restrict__ A, long lda, const u32* __restrict__ Bm, long ldb,
                      u32* __restrict__ cols, int s, int ctiles) {
    __shared__ __align__(16) u32 sa[BIG_ROWS];
    __shared__ __align__(16) u32 sb[BIG_COLS + BIG_ROWS + 8];
    const long p = blockIdx.x / ctiles;
    const int ct = blockIdx.x - (int)(p * ctiles);
    const int c0 = ct * BIG_COLS;
    const u32* a = A + p * lda;
    const u32* b = Bm + p * ldb;
    const int t = threadIdx.x;
    int ilo = c0 - s + 1;
    if (ilo < 0) ilo = 0;
    ilo = ilo / BIG_ROWS * BIG_ROWS;
    const int ihi = c0 + BIG_COLS < s ? c0 + BIG_COLS : s;
    u32 lo[4] = {0, 0, 0, 0}, mid[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0};
    for (int i0 = ilo; i0 < ihi; i0 += BIG_ROWS) {
        __syncthreads();
        const int jb = c0 - i0 - BIG_ROWS;  // sb[x] = b[jb + x]
        for (int x = t; x < BIG_ROWS; x += blockDim.x) sa[x] = i0 + x < s ? a[i0 + x] : 0u;
        for (int x = t; x < BIG_COLS + BIG_ROWS + 8; x += blockDim.x) {
            const int j = jb + x;
            sb[x] = (j >= 0 && j < s) ? b[j] : 0u;
        }
        __syncthreads();
#pragma unroll 4
        for (int grp = 0; grp < BIG_ROWS / 4; ++grp) {
            const uint4 av = *reinterpret_cast<const uint4*>(sa + 4 * grp);
            const int xb = BIG_ROWS + 4 * t - 4 * grp - 4;
            const uint4 b0 = *reinterpret_cast<const uint4*>(sb + xb);
            const uint4 b1 = *reinterpret_cast<const uint4*>(sb + xb + 4);
            const u32 a4[4] = {av.x, av.y, av.z, av.w};
            const u32 b8[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int rho = 0; rho < 4; ++rho)
#pragma unroll
                for (int w = 0; w < 4; ++w) mac96(lo[w], mid[w], hi[w], a4[rho], b8[4 + w - rho]);
        }
    }
    const long ncol = 2L * s;
    u32* cl = cols + p * 3 * ncol;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const long c = c0 + 4 * t + w;
        if (c < ncol) {
            cl[c] = lo[w];
            cl[ncol + c] = mid[w];
            cl[2 * ncol + c] = hi[w];
        }
    }
}

__global__ void __launch_bounds__(1024)
bigmul_normalise_kernel(const u32* __restrict__ cols, u32* __restrict__ OUT, long ldo, int s) {
    __shared__ __align__(16) u32 shscan[2 * 1024 + 80];
    const long p = blockIdx.x;
    const long ncol = 2L * s;
    const u32* lo = cols + p * 3 * ncol;
    const u32* mid = lo + ncol;
    const u32* hi = mid + ncol;
    u32* out = OUT + p * ldo;
    const bool aligned = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
    BlockNormState st{0, 0};
    const long chunk = 4L * blockDim.x;
    for (long base = 0; base < ncol; base += chunk) {
        u64 cs[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long c = base + 4L * threadIdx.x + j;
            u64 v = 0;
            if (c < ncol) {
                v = lo[c];
                if (c >= 1) v += mid[c - 1];
                if (c >= 2) v += hi[c - 2];
            }
            cs[j] = v;
        }
        u32 d[4];
        block_norm_unsigned(cs, st, d, shscan);
        const long pos = base + 4L * threadIdx.x;
        if (aligned && pos + 4 <= ncol) {
            st4(out + pos, d);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (pos + j < ncol) out[pos + j] = d[j];
        }
    }
}

size_t schoolbook_big_bytes(int s, long P) { return (size_t)P * 3 * 2 * (size_t)s * 4; }

cudaError_t launch_schoolbook_big(const u32* A, long lda, const u32* Bm, long ldb, u32* OUT,
                                  long ldo, int s, long P, u32* cols, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    const int ctiles = (2 * s + BIG_COLS - 1) / BIG_COLS;
    note_kernel("bigmul_columns_kernel+bigmul_normalise_kernel");
    bigmul_columns_kernel<<<(unsigned)(P * ctiles), BIG_COLS / 4, 0, st>>>(A, lda, Bm, ldb, cols, s, ctiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bigmul_normalise_kernel<<<(unsigned)P, 1024, 0, st>>>(cols, OUT, ldo, s);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pair-per-product schoolbook for large batches, operands staged in shared
// memory.
//
// A warp takes 16 products; lanes 2q and 2q+1 share product q.  Both walk the
// same 8x8 tiles (I, J) by anti-diagonal D = I + J, lane 2q+h multiplying
// rows 8I+4h .. 8I+4h+3 of a by the eight limbs 8J .. 8J+7 of b, so its
// products land in columns 8D+4h .. 8D+4h+10: twelve 96-bit Comba
// accumulators, slot k holding column 8D+4h+k.  After diagonal D the odd lane
// hands its slots 0..7 (columns 8D+4 .. 8D+11, which it will not touch again)
// to the even lane, which then holds columns 8D .. 8D+7 complete and emits
// them by two carry chains over the eight 96-bit column sums (the overflow
// past column 8D+7 becomes the next window's column 0); both lanes slide
// their windows by eight columns.  A final diagonal with no tiles flushes the
// top columns.
//
// Every operand limb is read from global memory once (coalesced, into
// shared memory).  Rows are staged with a stride of 8 or 24 (mod 32) words,
// so the 16-byte slice loads of the lane pairs of four products (a quarter
// warp) fall in distinct bank groups, and both lanes of a pair read the same
// b slice (a broadcast).
//
// Squaring accumulates a_i a_j for i < j only (tiles I <= J; inside a
// diagonal tile the even/odd rows keep columns c > row) and doubles at
// emission, adding a_i^2 on the even columns.
// ---------------------------------------------------------------------------
//
// One Karatsuba level inside the kernel (rows of at least g_kara_min_limbs
// limbs, 384 by default: measured on GB300 it is 4 % faster at 456 limbs and
// 10 % at 792, but slower at 234 and below, where the three sweeps' extra
// diagonals cost more than the 23 % of tiles they save).  With a = a0 + a1 X, b = b0 + b1 X, X = 2^(32k), k = 8 ceil(T/2):
//   P0 = a0 b0, P2 = a1 b1, P1 = |a0 - a1| |b0 - b1|,
//   a b = P0 + (P0 + P2 - s P1) X + P2 X^2,  s = sign((a0 - a1)(b0 - b1)),
// three sub-products of ceil(T/2)^2, floor(T/2)^2 and ceil(T/2)^2 tiles instead
// of T^2 (177 instead of 225 at 15 tiles).  The lane pair runs the same
// diagonal sweep three times: P0 into columns [0, 2k) and P2 into [2k, 2s) of
// the output row (disjoint, plain stores); then the differences overwrite a0
// and b0 in shared memory (one lane each), and with H0 = P0 div X and
// L2 = P2 mod X the even lane forms T = H0 + L2 and stores it over both.
// Splitting P0 = L0 + H0 X, P2 = L2 + H2 X, P1 = L1 + H1 X, the product is
//   L0 + (T + L0 - s L1) X + (T + H2 - s H1) X^2 + H2 X^3,
// so the third sweep, over the windows of P1, adds T (already in place) plus
// L0 or H2 (untouched rows of the output) and subtracts or adds its own window,
// with a signed carry from window to window; the last carry ripples into H2's
// columns.  Every window of the combine is read and written once.
// ---------------------------------------------------------------------------
constexpr int PAIR_WARPS = 2;
constexpr int PAIR_KARA_MIN_LIMBS = 49;  // from 7 tiles on, 2s >= 3k holds

__host__ __device__ inline int pair_stride(int s) {
    int sp = (s + 7) / 8 * 8;  // a multiple of 8 words: 8 or 24 (mod 32) wanted
    if (sp % 32 == 0 || sp % 32 == 16) sp += 8;
    return sp;
}

__device__ __forceinline__ void add96(u32& lo, u32& mid, u32& hi, u32 a, u32 b, u32 c) {
    asm("add.cc.u32 %0, %0, %3;\n\t"
        "addc.cc.u32 %1, %1, %4;\n\t"
        "addc.u32 %2, %2, %5;"
        : "+r"(lo), "+r"(mid), "+r"(hi)
        : "r"(a), "r"(b), "r"(c));
}

// R[0..10] = sum_(k<8) (lo_k + mid_k 2^32 + hi_k 2^64) 2^(32k): lo plus mid one limb
// up, then plus hi two limbs up, each one carry chain.
__device__ __forceinline__ void add8_shifted(const u32* lo, const u32* mid, const u32* hi, u32* R) {
    R[0] = lo[0];
    asm("add.cc.u32 %0, %9, %16;\n\t"
        "addc.cc.u32 %1, %10, %17;\n\t"
        "addc.cc.u32 %2, %11, %18;\n\t"
        "addc.cc.u32 %3, %12, %19;\n\t"
        "addc.cc.u32 %4, %13, %20;\n\t"
        "addc.cc.u32 %5, %14, %21;\n\t"
        "addc.cc.u32 %6, %15, %22;\n\t"
        "addc.cc.u32 %7, %23, 0;\n\t"
        "addc.u32 %8, 0, 0;"
        : "=r"(R[1]), "=r"(R[2]), "=r"(R[3]), "=r"(R[4]), "=r"(R[5]), "=r"(R[6]), "=r"(R[7]),
          "=r"(R[8]), "=r"(R[9])
        : "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(lo[5]), "r"(lo[6]), "r"(lo[7]),
          "r"(mid[0]), "r"(mid[1]), "r"(mid[2]), "r"(mid[3]), "r"(mid[4]), "r"(mid[5]), "r"(mid[6]),
          "r"(mid[7]));
    asm("add.cc.u32 %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, %10;\n\t"
        "addc.cc.u32 %2, %2, %11;\n\t"
        "addc.cc.u32 %3, %3, %12;\n\t"
        "addc.cc.u32 %4, %4, %13;\n\t"
        "addc.cc.u32 %5, %5, %14;\n\t"
        "addc.cc.u32 %6, %6, %15;\n\t"
        "addc.cc.u32 %7, %7, %16;\n\t"
        "addc.u32 %8, 0, 0;"
        : "+r"(R[2]), "+r"(R[3]), "+r"(R[4]), "+r"(R[5]), "+r"(R[6]), "+r"(R[7]), "+r"(R[8]),
          "+r"(R[9]), "=r"(R[10])
        : "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]), "r"(hi[5]), "r"(hi[6]),
          "r"(hi[7]));
}

// R[0..10] += (x0 + x1 2^32 + x2 2^64) at limb 0 (squaring path: the carry kept apart).
__device__ __forceinline__ void add3_into11(u32* R, u32 x0, u32 x1, u32 x2) {
    asm("add.cc.u32 %0, %0, %11;\n\t"
        "addc.cc.u32 %1, %1, %12;\n\t"
        "addc.cc.u32 %2, %2, %13;\n\t"
        "addc.cc.u32 %3, %3, 0;\n\t"
        "addc.cc.u32 %4, %4, 0;\n\t"
        "addc.cc.u32 %5, %5, 0;\n\t"
        "addc.cc.u32 %6, %6, 0;\n\t"
        "addc.cc.u32 %7, %7, 0;\n\t"
        "addc.cc.u32 %8, %8, 0;\n\t"
        "addc.cc.u32 %9, %9, 0;\n\t"
        "addc.u32 %10, %10, 0;"
        : "+r"(R[0]), "+r"(R[1]), "+r"(R[2]), "+r"(R[3]), "+r"(R[4]), "+r"(R[5]), "+r"(R[6]),
          "+r"(R[7]), "+r"(R[8]), "+r"(R[9]), "+r"(R[10])
        : "r"(x0), "r"(x1), "r"(x2));
}

// Squaring: R = 2 R + sum_(k<4) a_k^2 2^(64k) over 11 limbs.
__device__ __forceinline__ void double_add_squares(u32* R, const u32* a) {
#pragma unroll
    for (int k = 10; k >= 1; --k) R[k] = fshl(R[k - 1], R[k], 1);
    R[0] <<= 1;
    u32 S[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        S[2 * k] = a[k] * a[k];
        S[2 * k + 1] = __umulhi(a[k], a[k]);
    }
    asm("add.cc.u32 %0, %0, %11;\n\t"
        "addc.cc.u32 %1, %1, %12;\n\t"
        "addc.cc.u32 %2, %2, %13;\n\t"
        "addc.cc.u32 %3, %3, %14;\n\t"
        "addc.cc.u32 %4, %4, %15;\n\t"
        "addc.cc.u32 %5, %5, %16;\n\t"
        "addc.cc.u32 %6, %6, %17;\n\t"
        "addc.cc.u32 %7, %7, %18;\n\t"
        "addc.cc.u32 %8, %8, 0;\n\t"
        "addc.cc.u32 %9, %9, 0;\n\t"
        "addc.u32 %10, %10, 0;"
        : "+r"(R[0]), "+r"(R[1]), "+r"(R[2]), "+r"(R[3]), "+r"(R[4]), "+r"(R[5]), "+r"(R[6]),
          "+r"(R[7]), "+r"(R[8]), "+r"(R[9]), "+r"(R[10])
        : "r"(S[0]), "r"(S[1]), "r"(S[2]), "r"(S[3]), "r"(S[4]), "r"(S[5]), "r"(S[6]), "r"(S[7]));
}

// Eight limbs of an output row at pos (zeros at and past len), for a window
// the emission reads later in the same diagonal.  The loads are volatile with a
// memory clobber so that they stay at this point of the diagonal: hoisted to
// the top of the unrolled diagonals they would hold three windows' registers.
__device__ __forceinline__ void prefetch8(const u32* row, int pos, int len, bool vec, u32 v[8]) {
    if (vec && pos + 8 <= len) {
        asm volatile("ld.global.v4.u32 {%0, %1, %2, %3}, [%8];\n\t"
                     "ld.global.v4.u32 {%4, %5, %6, %7}, [%8+16];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                       "=r"(v[7])
                     : "l"(row + pos)
                     : "memory");
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            u32 x = 0;
            if (pos + k < len) asm volatile("ld.global.u32 %0, [%1];" : "=r"(x) : "l"(row + pos + k) : "memory");
            v[k] = x;
        }
    }
}

// Karatsuba combine of one window: res = tw + xw + (sub ? -R : R) + carry over
// eight limbs; carry (signed, |carry| <= 3) becomes the window's overflow.
// -R is ~R + 1 - 2^256, so one add chain with carry-in (sub & 1) serves both
// signs; a negative incoming carry enters as its 256-bit two's complement.
__device__ __forceinline__ void combine_window(const u32 tw[8], const u32 xw[8], const u32 R[8], u32 sub,
                                               int& carry, u32 res[8]) {
    u32 S[8], Rm[8];
    u32 c = add4c(tw, xw, 0u, S);
    c = add4c(tw + 4, xw + 4, c, S + 4);
    int top = (int)c - (int)(sub & 1u);
#pragma unroll
    for (int j = 0; j < 8; ++j) Rm[j] = R[j] ^ sub;
    c = add4c(S, Rm, sub & 1u, res);
    c = add4c(S + 4, Rm + 4, c, res + 4);
    top += (int)c;
    const u32 ext = carry < 0 ? ~0u : 0u;
    u32 co;
    asm("add.cc.u32 %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, %10;\n\t"
        "addc.cc.u32 %2, %2, %10;\n\t"
        "addc.cc.u32 %3, %3, %10;\n\t"
        "addc.cc.u32 %4, %4, %10;\n\t"
        "addc.cc.u32 %5, %5, %10;\n\t"
        "addc.cc.u32 %6, %6, %10;\n\t"
        "addc.cc.u32 %7, %7, %10;\n\t"
        "addc.u32 %8, 0, 0;"
        : "+r"(res[0]), "+r"(res[1]), "+r"(res[2]), "+r"(res[3]), "+r"(res[4]), "+r"(res[5]),
          "+r"(res[6]), "+r"(res[7]), "=r"(co)
        : "r"((u32)carry), "r"(ext));
    carry = top + (int)co - (carry < 0 ? 1 : 0);
}

// r[0, k) = |r[0, k) - r[k, k + n1)| in place (the second operand is zero past
// n1 <= k; k and n1 multiples of 4, r 16-byte aligned shared memory); returns 1
// when the difference was negative.
__device__ __forceinline__ u32 abs_diff_inplace(u32* r, int k, int n1) {
    u32 br = 0;
    for (int i = 0; i < k; i += 4) {
        const uint4 x = ld4(r + i);
        const uint4 y = i < n1 ? ld4(r + k + i) : make_uint4(0u, 0u, 0u, 0u);
        const u32 xa[4] = {x.x, x.y, x.z, x.w}, ya[4] = {y.x, y.y, y.z, y.w};
        u32 d[4];
        br = sub4b(xa, ya, br, d);
        st4(r + i, d);
    }
    if (br) {  // negate: ~d + 1
        u32 c = 1;
        for (int i = 0; i < k; i += 4) {
            const uint4 x = ld4(r + i);
            u32 d[4] = {~x.x, ~x.y, ~x.z, ~x.w};
            c = inc4(d, c);
            st4(r + i, d);
        }
    }
    return br;
}

// One anti-diagonal of the pair kernel; OFF is the ring offset of the window's
// column 0 among the twelve accumulator slots (slot (OFF + k) mod 12 holds
// column 8D + 4h + k).
template <bool SQ>
struct PairDiag {
    const u32* ra;
    const u32* rb;
    u32* out;
    int T, h;
    bool emit, aligned;
    int out_len;
    // Karatsuba sweeps (out = the product row, out_len = 2s): mode 1 is P2,
    // whose windows land on columns 2k + 8D and whose low half L2 becomes
    // T = H0 + L2 on the fly (stored at k + 8D and 2k + 8D); mode 2 is the
    // combine of P1's windows into columns k + 8D (see combine_window).
    int mode;
    int ks, T0;   // split column k and tiles of a0
    u32 sub;      // all ones: the middle product is subtracted
    int carry;    // mode 1: T's carry chain; mode 2: signed carry between windows
    int cT;       // carry out of T

    template <int OFF>
    __device__ __forceinline__ void step(int D, u32 (&lo)[12], u32 (&mid)[12], u32 (&hi)[12],
                                         u32 (&cin)[3]) {
        auto S = [](int k) { return (OFF + k) % 12; };
        // the output windows this diagonal's emission reads, loaded ahead of its
        // products so that their latency overlaps them
        u32 pa[8] = {0, 0, 0, 0, 0, 0, 0, 0}, pb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (mode == 1 && emit && D < T0) prefetch8(out, ks + 8 * D, out_len, aligned, pa);      // H0
        if (mode == 2 && emit) {
            prefetch8(out, ks + 8 * D, out_len, aligned, pa);                                   // T
            prefetch8(out, D < T0 ? 8 * D : 2 * ks + 8 * D, out_len, aligned, pb);              // L0, H2
        }
        const int Ilo = D - T + 1 > 0 ? D - T + 1 : 0;
        int Ihi = D < T - 1 ? D : T - 1;
        if (SQ && Ihi > D / 2) Ihi = D / 2;
        for (int I = Ilo; I <= Ihi; ++I) {
            const int J = D - I;
            const uint4 av = ld4(ra + 8 * I + 4 * h);
            const uint4 b0 = ld4(rb + 8 * J), b1 = ld4(rb + 8 * J + 4);
            const u32 a4[4] = {av.x, av.y, av.z, av.w};
            const u32 b8[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
            if (SQ && I == J) {
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        mac96(lo[S(r + c)], mid[S(r + c)], hi[S(r + c)], a4[r], c > 4 * h + r ? b8[c] : 0u);
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) mac96(lo[S(r + c)], mid[S(r + c)], hi[S(r + c)], a4[r], b8[c]);
            }
        }
        // the odd lane's columns 0..7 join the even lane's columns 4..11
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const u32 pl = __shfl_down_sync(FULL, lo[S(k)], 1);
            const u32 pm = __shfl_down_sync(FULL, mid[S(k)], 1);
            const u32 ph = __shfl_down_sync(FULL, hi[S(k)], 1);
            if (h == 0) add96(lo[S(k + 4)], mid[S(k + 4)], hi[S(k + 4)], pl, pm, ph);
        }
        // columns 8D .. 8D+7 (even lane): the limbs of sum_k (lo_k + mid_k 2^32 + hi_k 2^64)
        // 2^(32k), k < 8, by two carry chains.  What spills past column 8D+7 (three
        // words) is the next diagonal's carry: added into column 8 (the next window's
        // column 0), or, when squaring, kept apart because the columns get doubled.
        const u32 wl[8] = {lo[S(0)], lo[S(1)], lo[S(2)], lo[S(3)], lo[S(4)], lo[S(5)], lo[S(6)], lo[S(7)]};
        const u32 wm[8] = {mid[S(0)], mid[S(1)], mid[S(2)], mid[S(3)], mid[S(4)], mid[S(5)], mid[S(6)], mid[S(7)]};
        const u32 wh[8] = {hi[S(0)], hi[S(1)], hi[S(2)], hi[S(3)], hi[S(4)], hi[S(5)], hi[S(6)], hi[S(7)]};
        u32 R[11];
        add8_shifted(wl, wm, wh, R);
        if (SQ) {
            const uint4 sq = ld4(ra + 4 * D);  // a_(4D + k/2) for the even columns (zeros past s)
            const u32 sqv[4] = {sq.x, sq.y, sq.z, sq.w};
            double_add_squares(R, sqv);
            add3_into11(R, cin[0], cin[1], cin[2]);
            cin[0] = R[8]; cin[1] = R[9]; cin[2] = R[10];
        } else if (h == 0) {
            add96(lo[S(8)], mid[S(8)], hi[S(8)], R[8], R[9], R[10]);
        }
        if (emit) {
            // whole windows below 3k <= 2s: the T windows and the combined ones
            auto put8 = [&](u32* dst, const u32* v) {
                if (aligned) {
                    st4(dst, v);
                    st4(dst + 4, v + 4);
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) dst[j] = v[j];
                }
            };
            if (mode == 2) {
                if (D == T0) carry += cT;
                u32 res[8];
                combine_window(pa, pb, R, sub, carry, res);
                put8(out + ks + 8 * D, res);
            } else if (mode == 1 && D < T0) {
                u32 t[8];
                u32 c = add4c(pa, R, (u32)carry, t);
                carry = (int)add4c(pa + 4, R + 4, c, t + 4);
                put8(out + ks + 8 * D, t);
                put8(out + 2 * ks + 8 * D, t);
                if (D == T0 - 1) cT = carry;
            } else {
                const int c0 = (mode == 1 ? 2 * ks : 0) + 8 * D;
                if (aligned && c0 + 8 <= out_len) {
                    st4(out + c0, R);
                    st4(out + c0 + 4, R + 4);
                } else {
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (c0 + k < out_len) out[c0 + k] = R[k];
                }
            }
        }
        // columns 0..7 are done: their slots become columns 4..11 of the next window
#pragma unroll
        for (int k = 0; k < 8; ++k) { lo[S(k)] = 0; mid[S(k)] = 0; hi[S(k)] = 0; }
    }
};

template <bool SQ, bool KARA>
__global__ void __launch_bounds__(32 * PAIR_WARPS)
leaf_pair_kernel(const u32* __restrict__ A, long lda, const u32* __restrict__ Bm, long ldb,
                 u32* __restrict__ OUT, long ldo, int s, long P, int vec) {
    extern __shared__ __align__(16) u32 psm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int T = (s + 7) / 8, sp = pair_stride(s);
    u32* sa = psm + (long)warp * (SQ ? 1 : 2) * 16 * sp;
    u32* sb = SQ ? sa : sa + 16 * sp;
    const long pw = ((long)blockIdx.x * PAIR_WARPS + warp) * 16;  // first product of the warp
    if (vec) {
        // aligned rows: asynchronous 16-byte copies straight into shared memory, all in
        // flight together; the bytes past a row's end (or of a missing product) are zero
        for (int q = 0; q < 16; ++q) {
            const long pq = pw + q;
            const bool ok = pq < P;
            const u32* ra = A + (ok ? pq : 0) * lda;
            const u32* rb = Bm + (ok ? pq : 0) * ldb;
            for (int i = 4 * lane; i < 8 * T; i += 128) {
                const int left = ok ? s - i : 0;
                const unsigned bytes = left >= 4 ? 16u : left > 0 ? 4u * left : 0u;
                const u32* ga = bytes ? ra + i : ra;
                const u32* gb = bytes ? rb + i : rb;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                             :: "r"((unsigned)__cvta_generic_to_shared(sa + q * sp + i)), "l"(ga), "r"(bytes));
                if (!SQ)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                                 :: "r"((unsigned)__cvta_generic_to_shared(sb + q * sp + i)), "l"(gb), "r"(bytes));
            }
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
    } else {
        for (int q = 0; q < 16; ++q) {
            const long pq = pw + q;
            const bool ok = pq < P;
            const u32* ra = A + (ok ? pq : 0) * lda;
            const u32* rb = Bm + (ok ? pq : 0) * ldb;
            for (int i = 4 * lane; i < 8 * T; i += 128) {
                u32 va[4], vb[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    va[j] = ok && i + j < s ? ra[i + j] : 0u;
                    if (!SQ) vb[j] = ok && i + j < s ? rb[i + j] : 0u;
                }
                st4(sa + q * sp + i, va);
                if (!SQ) st4(sb + q * sp + i, vb);
            }
        }
    }
    __syncwarp();

    const int q = lane >> 1, h = lane & 1;
    const long p = pw + q;
    const bool emit = p < P && h == 0;
    const u32* ra = sa + q * sp;
    const u32* rb = sb + q * sp;
    u32* out = OUT + (p < P ? p : 0) * ldo;
    const bool aligned = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
    // Karatsuba: a0 = the first T0 tiles of a row, a1 = the other T - T0
    const int T0 = KARA ? (T + 1) / 2 : T, k = 8 * T0;
    PairDiag<SQ> pd{ra, rb, out, T0, h, emit, aligned, 2 * s, 0, k, T0, 0u, 0, 0};
#pragma unroll 1
    for (int part = 0; part < (KARA ? 3 : 1); ++part) {
        if (KARA && part == 1) {          // P2 = a1 b1 -> columns [2k, 2s), T = H0 + L2
            pd.ra = ra + k;
            pd.rb = rb + k;
            pd.T = T - T0;
            pd.mode = 1;
        } else if (KARA && part == 2) {   // P1 = |a0 - a1| |b0 - b1|, combined
            __syncwarp();
            u32 neg = 0;
            if (!SQ || h == 0) neg = abs_diff_inplace(const_cast<u32*>(h == 0 ? ra : rb), k, 8 * (T - T0));
            const u32 other = __shfl_xor_sync(FULL, neg, 1);
            pd.sub = (SQ || neg == other) ? ~0u : 0u;
            __syncwarp();
            pd.ra = ra;
            pd.rb = rb;
            pd.T = T0;
            pd.mode = 2;
            pd.carry = 0;
        }
        u32 lo[12], mid[12], hi[12], cin[3] = {0, 0, 0};
#pragma unroll
        for (int j = 0; j < 12; ++j) { lo[j] = 0; mid[j] = 0; hi[j] = 0; }
        // The twelve slots are a ring that advances by eight per diagonal, so three
        // consecutive diagonals (ring offsets 0, 8, 4) run unrolled with fixed
        // register names instead of moving the window.
        const int TT = pd.T;
        int D = 0;
        for (; D + 3 <= 2 * TT; D += 3) {
            pd.template step<0>(D, lo, mid, hi, cin);
            pd.template step<8>(D + 1, lo, mid, hi, cin);
            pd.template step<4>(D + 2, lo, mid, hi, cin);
        }
        if (D < 2 * TT) pd.template step<0>(D++, lo, mid, hi, cin);
        if (D < 2 * TT) pd.template step<8>(D++, lo, mid, hi, cin);
    }
    if (KARA && emit) {  // the last window's carry and T's second carry into H2's columns
        int c = pd.carry + pd.cT;
        for (int i = 3 * k; i < 2 * s && c != 0; ++i) {
            const long long v = (long long)out[i] + c;
            out[i] = (u32)v;
            c = (int)(v >> 32);
        }
    }
}

// Products at or above this count use the lane-per-product kernels: a lane
// pair per product with the rows in shared memory while a block's rows fit,
// else one lane per product reading its rows from global memory.
constexpr long LANE_KERNEL_MIN = 4096;
constexpr size_t PAIR_SMEM_MAX = 200 * 1024;

static int g_kara_min_limbs = TC_LEAF_KARATSUBA_DEFAULT;   // tc_set_leaf_karatsuba

static bool pair_karatsuba(int s) {
    const int T = (s + 7) / 8, k = 8 * ((T + 1) / 2);
    return g_kara_min_limbs > 0 && s >= g_kara_min_limbs && s >= PAIR_KARA_MIN_LIMBS && 2 * s >= 3 * k;
}

static bool pair_kernel_fits(int s, bool square) {
    return (size_t)(square ? 1 : 2) * 16 * pair_stride(s) * 4 * PAIR_WARPS <= PAIR_SMEM_MAX;
}

double leaf_limb_products(int s, long P) {
    if (P >= LANE_KERNEL_MIN && pair_kernel_fits(s, false) && pair_karatsuba(s)) {
        const double k = 8.0 * (((s + 7) / 8 + 1) / 2);
        return (double)P * (2.0 * k * k + (s - k) * (s - k));
    }
    return (double)P * s * s;
}


cudaError_t launch_leaf(const u32* A, long lda, const u32* Bm, long ldb, u32* OUT, long ldo,
                        int s, long P, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    const bool square = (A == Bm && lda == ldb);
    if (P >= LANE_KERNEL_MIN) {
        const bool vec = ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Bm)) & 15u) == 0 &&
                         lda % 4 == 0 && ldb % 4 == 0;
        const size_t per_warp = (size_t)(square ? 1 : 2) * 16 * pair_stride(s) * 4;
        if (per_warp * PAIR_WARPS <= PAIR_SMEM_MAX) {
            static std::once_flag pair_once;
            std::call_once(pair_once, [] {
                cudaFuncSetAttribute(leaf_pair_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, PAIR_SMEM_MAX);
                cudaFuncSetAttribute(leaf_pair_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, PAIR_SMEM_MAX);
                cudaFuncSetAttribute(leaf_pair_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, PAIR_SMEM_MAX);
                cudaFuncSetAttribute(leaf_pair_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, PAIR_SMEM_MAX);
            });
            const unsigned grid = (unsigned)((P + 16 * PAIR_WARPS - 1) / (16 * PAIR_WARPS));
            const size_t smem = per_warp * PAIR_WARPS;
            const bool kara = pair_karatsuba(s);
#define TC_PAIR_LAUNCH(SQ_, K_)                                                                        \
    do {                                                                                               \
        note_kernel("leaf_pair_kernel<" #SQ_ ", " #K_ ">");                                            \
        leaf_pair_kernel<SQ_, K_><<<grid, 32 * PAIR_WARPS, smem, st>>>(A, lda, Bm, ldb, OUT, ldo, s, P, vec); \
    } while (0)
            if (square) {
                if (kara) TC_PAIR_LAUNCH(true, true); else TC_PAIR_LAUNCH(true, false);
            } else {
                if (kara) TC_PAIR_LAUNCH(false, true); else TC_PAIR_LAUNCH(false, false);
            }
#undef TC_PAIR_LAUNCH
            return cudaGetLastError();
        }
        const unsigned grid = (unsigned)((P + 127) / 128);
        if (square) {
            note_kernel("leaf_lane_kernel<true>");
            leaf_lane_kernel<true><<<grid, 128, 0, st>>>(A, lda, Bm, ldb, OUT, ldo, s, P, vec);
        } else {
            note_kernel("leaf_lane_kernel<false>");
            leaf_lane_kernel<false><<<grid, 128, 0, st>>>(A, lda, Bm, ldb, OUT, ldo, s, P, vec);
        }
        return cudaGetLastError();
    }
    LeafGeom g = leaf_geom(s);
    const int tiles = g.RB * g.CT;
    const size_t smem_max = 220 * 1024;
    int ppc = tiles >= 256 ? 1 : 256 / tiles;
    while (ppc > 1 && (size_t)ppc * g.words * 4 > smem_max) --ppc;
    if ((size_t)g.words * 4 > smem_max) return cudaErrorInvalidValue;
    int threads = tiles * ppc >= 256 ? 256 : ((tiles * ppc + 31) / 32) * 32;
    if (threads < 64) threads = 64;
    const size_t smem = (size_t)ppc * g.words * 4;
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        cudaFuncSetAttribute(leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    });
    const long grid = (P + ppc - 1) / ppc;
    note_kernel("leaf_kernel");
    leaf_kernel<<<(unsigned)grid, threads, smem, st>>>(A, lda, Bm, ldb, OUT, ldo, g, P, ppc);
    return cudaGetLastError();
}

}  // namespace tc

extern "C" tc_status tc_set_leaf_karatsuba(int min_limbs) {
    if (min_limbs < 0 || (min_limbs > 0 && min_limbs < tc::PAIR_KARA_MIN_LIMBS)) return TC_EINVAL;
    tc::g_kara_min_limbs = min_limbs;
    return TC_OK;
}
