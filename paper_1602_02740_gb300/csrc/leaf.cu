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
// window of columns per row block; a warp per product then sums the row
// blocks per output limb and resolves carries with the warp scans.
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

    const int warp = tid >> 5, nwarps = nt >> 5, lane = tid & 31;
    const int out_len = 2 * g.s;
    for (int k = warp; k < np; k += nwarps) {
        const u32* part = sm + k * g.words + g.sa_len + g.sb_len;
        u32* out = OUT + (p0 + k) * ldo;
        const bool aligned = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
        SignedNorm st{0, 0};
        for (int base = 0; base < out_len; base += CH) {
            i64 cols[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int c = base + 4 * lane + jj;
                u64 S = 0;
                for (int r = 0; r < g.RB; ++r) {
                    const int x = c - r * g.H;
                    if (x >= 0 && x < g.NW) S += part[(0 * g.RB + r) * g.NW + x];
                    if (x - 1 >= 0 && x - 1 < g.NW) S += part[(1 * g.RB + r) * g.NW + x - 1];
                    if (x - 2 >= 0 && x - 2 < g.NW) S += part[(2 * g.RB + r) * g.NW + x - 2];
                }
                cols[jj] = (i64)S;
            }
            u32 d[4];
            warp_norm_signed(cols, st, d);
            const int pos = base + 4 * lane;
            if (aligned && pos + 4 <= out_len) {
                st4(out + pos, d);
            } else {
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (pos + jj < out_len) out[pos + jj] = d[jj];
            }
        }
    }
}

cudaError_t launch_leaf(const u32* A, long lda, const u32* Bm, long ldb, u32* OUT, long ldo,
                        int s, long P, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    LeafGeom g = leaf_geom(s);
    const int tiles = g.RB * g.CT;
    const size_t smem_max = 220 * 1024;
    int ppc = tiles >= 256 ? 1 : 256 / tiles;
    while (ppc > 1 && (size_t)ppc * g.words * 4 > smem_max) --ppc;
    if ((size_t)g.words * 4 > smem_max) return cudaErrorInvalidValue;
    int threads = tiles * ppc >= 256 ? 256 : ((tiles * ppc + 31) / 32) * 32;
    if (threads < 64) threads = 64;
    const size_t smem = (size_t)ppc * g.words * 4;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr_set = true;
    }
    const long grid = (P + ppc - 1) / ppc;
    leaf_kernel<<<(unsigned)grid, threads, smem, st>>>(A, lda, Bm, ldb, OUT, ldo, g, P, ppc);
    return cudaGetLastError();
}

}  // namespace tc
