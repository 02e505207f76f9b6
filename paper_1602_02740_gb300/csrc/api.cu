// C-ABI entry points (include/tc.h): context, plans, scratch, level schedule.
#include <algorithm>
#include <memory>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tc.h"
#include "tc_device.cuh"
#include "tc_internal.h"
#include "tc_ctx.h"

using namespace tc;

static thread_local int g_last_cuda_error = 0;

tc_status tc_fail_cuda(cudaError_t e) {
    g_last_cuda_error = (int)e;
    return e == cudaErrorMemoryAllocation ? TC_ENOMEM : TC_EDEVICE;
}

#define CK(x)                                         \
    do {                                              \
        cudaError_t _e = (x);                         \
        if (_e != cudaSuccess) return tc_fail_cuda(_e); \
    } while (0)

extern "C" const char* tc_strerror(tc_status s) {
    switch (s) {
        case TC_OK: return "ok";
        case TC_EINVAL: return "invalid argument";
        case TC_ENOMEM: return "scratch budget exceeded or device allocation failed";
        case TC_EBUSY: return "not admitted: budget or slots full";
        case TC_ETIMEOUT: return "bounded wait gave up";
        case TC_EDEVICE: return "CUDA error";
        case TC_EPENDING: return "pending";
    }
    return "unknown status";
}

extern "C" int tc_last_cuda_error(void) { return g_last_cuda_error; }

// ---------------------------------------------------------------------------
// Plans
// ---------------------------------------------------------------------------
namespace tc {

// Built-in rule: pick B per level so the recursion ends near 64-128 limbs.
tc_opts default_plan(size_t s) {
    tc_opts o;
    memset(&o, 0, sizeof(o));
    size_t L = s;
    while (L > 128 && o.levels < TC_MAX_LEVELS) {
        int B = L > 16384 ? 16 : L > 2048 ? 8 : L > 512 ? 4 : 3;
        o.B[o.levels++] = B;
        LevelGeom g = make_level((int)L, B);
        L = (size_t)g.e;
    }
    return o;
}

bool plan_valid(const tc_opts& o, size_t s) {
    if (o.levels < 0 || o.levels > TC_MAX_LEVELS) return false;
    if (o.base != TC_BASE_SCHOOLBOOK && o.base != TC_BASE_NTT) return false;
    size_t L = s;
    for (int l = 0; l < o.levels; ++l) {
        if (o.B[l] < 2 || o.B[l] > 32) return false;
        if ((size_t)o.B[l] > L) return false;
        LevelGeom g = make_level((int)L, o.B[l]);
        L = (size_t)g.e;
    }
    if (o.base == TC_BASE_NTT) return L <= (size_t)NTT_MAX_LIMBS;
    return o.levels == 0 || L <= (size_t)LEAF_MAX;  // no levels: plain schoolbook, any length
}

tc_opts plan_for(tc_ctx* ctx, size_t s) {
    if (ctx) {
        for (auto& row : ctx->table)
            if (s <= row.first && plan_valid(row.second, s)) return row.second;
    }
    return default_plan(s);
}


BatchLayout layout_for(size_t count, size_t s, const tc_opts& o, bool square) {
    BatchLayout L;
    size_t off = 0;
    long P = (long)count;
    int sl = (int)s;
    for (int l = 0; l < o.levels; ++l) {
        LevelGeom g = make_level(sl, o.B[l]);
        const long Pn = P * (2 * g.B - 1);
        L.g.push_back(g);
        L.P.push_back(P);
        L.evalU.push_back(off); off = align256(off + (size_t)Pn * g.estride * 4);
        L.evalV.push_back(off); if (!square) off = align256(off + (size_t)Pn * g.estride * 4);
        L.sgnU.push_back(off); off = align256(off + (size_t)Pn);
        L.sgnV.push_back(off); if (!square) off = align256(off + (size_t)Pn);
        L.prod.push_back(off); off = align256(off + (size_t)Pn * g.ystride * 4);
        L.work.push_back(off); off = align256(off + (size_t)P * interp_work_bytes(g, P));
        L.evwork.push_back(off);
        if (use_wide_eval(g, P)) off = align256(off + wide_eval_work_bytes(g, P));
        P = Pn;
        sl = g.e;
    }
    L.P.push_back(P);
    L.base = o.base;
    if (o.base == TC_BASE_NTT) {  // transform scratch of the base products
        L.ntt = off;
        off = align256(off + ntt_work_bytes(sl, P, square));
        L.total = off;
        return L;
    }
    if (o.levels == 0 && s > (size_t)LEAF_MAX) {  // column buffer of the large schoolbook
        L.work.push_back(off);
        off = align256(off + schoolbook_big_bytes((int)s, (long)count));
    }
    L.total = off;
    return L;
}

tc_status ensure_arena(tc_ctx* ctx, size_t bytes, cudaStream_t st) {
    if (bytes <= ctx->arena_bytes) return TC_OK;
    if (bytes > ctx->budget) return TC_ENOMEM;
    CK(cudaStreamSynchronize(st));
    if (ctx->arena) cudaFree(ctx->arena);
    ctx->arena = nullptr;
    ctx->arena_bytes = 0;
    size_t want = std::min(ctx->budget, std::max(bytes, bytes + bytes / 4));
    cudaError_t e = cudaMalloc(&ctx->arena, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&ctx->arena, bytes);
        if (e != cudaSuccess) { cudaGetLastError(); ctx->arena = nullptr; return TC_ENOMEM; }
        want = bytes;
    }
    ctx->arena_bytes = want;
    return TC_OK;
}

// Phase timing: events around each launch when the context asks for it.
struct PhaseTimer {
    tc_ctx* ctx;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    int kind = 0, level = 0;
    double bytes = 0, lp = 0;
    static cudaEvent_t get(tc_ctx* c) {
        if (!c->event_pool.empty()) {
            cudaEvent_t e = c->event_pool.back();
            c->event_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void begin(int k, int l, double by, double p) {
        if (!ctx || !ctx->profile) return;
        kind = k; level = l; bytes = by; lp = p;
        a = get(ctx);
        cudaEventRecord(a, st);
    }
    void end() {
        if (!ctx || !ctx->profile || !a) return;
        cudaEvent_t b = get(ctx);
        cudaEventRecord(b, st);
        ctx->recs.push_back({kind, level, a, b, bytes, lp, g_kernel_name});
        a = nullptr;
    }
};

cudaError_t StreamFan::init() {
    if (ready) return cudaSuccess;
    cudaError_t e = cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming);
    for (int i = 0; i < K && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join_ev[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        destroy();
        return e;
    }
    ready = true;
    return cudaSuccess;
}

void StreamFan::destroy() {
    for (int i = 0; i < K; ++i) {
        if (s[i]) {
            cudaStreamSynchronize(s[i]);
            cudaStreamDestroy(s[i]);
        }
        if (join_ev[i]) cudaEventDestroy(join_ev[i]);
        s[i] = nullptr;
        join_ev[i] = nullptr;
    }
    if (fork_ev) cudaEventDestroy(fork_ev);
    fork_ev = nullptr;
    ready = false;
}

cudaError_t StreamFan::fork(cudaStream_t st) {
    cudaError_t e = cudaEventRecord(fork_ev, st);
    for (int i = 0; i < K && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(s[i], fork_ev, 0);
    return e;
}

cudaError_t StreamFan::join(cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < K && e == cudaSuccess; ++i) {
        e = cudaEventRecord(join_ev[i], s[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, join_ev[i], 0);
    }
    return e;
}

// Run a uniform batch whose scratch is `base` laid out by `L`.
static __global__ void or_error_kernel(int* sticky, const int* word) {
    if (threadIdx.x == 0 && *word) atomicOr(sticky, TC_STICKY_TIMEOUT);
}

cudaError_t launch_or_error(int* sticky, const int* word, cudaStream_t st) {
    or_error_kernel<<<1, 32, 0, st>>>(sticky, word);
    return cudaGetLastError();
}

tc_status run_uniform(const BatchLayout& L, char* base, size_t count, size_t s, const u32* A,
                      long lda, const u32* Bm, long ldb, u32* OUT, long ldo, bool square,
                      cudaStream_t st, tc_ctx* ctx, int* sticky) {
    PhaseTimer pt{ctx, st};
    const int D = (int)L.g.size();
    if (D == 0) {
        pt.begin(1, 0, 4.0 * count * 4 * s, leaf_limb_products(s, count));
        if (L.base == TC_BASE_NTT)
            CK(launch_ntt_mul(A, lda, square ? A : Bm, square ? lda : ldb, OUT, ldo, (int)s,
                              (long)count, square, base + L.ntt, st));
        else if (s > (size_t)LEAF_MAX)
            CK(launch_schoolbook_big(A, lda, square ? A : Bm, square ? lda : ldb, OUT, ldo, (int)s,
                                     (long)count, reinterpret_cast<u32*>(base + L.work[0]), st));
        else
            CK(launch_leaf(A, lda, square ? A : Bm, square ? lda : ldb, OUT, ldo, (int)s, (long)count, st));
        pt.end();
        return TC_OK;
    }
    const u32* inU = A;
    const u32* inV = square ? A : Bm;
    long strU = lda, strV = square ? lda : ldb;
    for (int l = 0; l < D; ++l) {
        const LevelGeom& g = L.g[l];
        u32* eU = reinterpret_cast<u32*>(base + L.evalU[l]);
        uint8_t* sU = reinterpret_cast<uint8_t*>(base + L.sgnU[l]);
        const double eval_bytes = 4.0 * L.P[l] * (g.s + (2.0 * g.B - 1) * g.estride) +
                                  (2.0 * g.B - 1) * L.P[l];
        void* evw = base + L.evwork[l];
        if (!square) {  // both operands (one launch for few rows)
            u32* eV = reinterpret_cast<u32*>(base + L.evalV[l]);
            uint8_t* sV = reinterpret_cast<uint8_t*>(base + L.sgnV[l]);
            pt.begin(0, l, 2 * eval_bytes, 0);
            CK(launch_eval2(inU, strU, eU, sU, inV, strV, eV, sV, g, L.P[l], evw, st));
            pt.end();
            inU = eU;
            strU = g.estride;
            inV = eV;
            strV = g.estride;
        } else {
            pt.begin(0, l, eval_bytes, 0);
            CK(launch_eval(inU, strU, g, eU, sU, L.P[l], evw, st));
            pt.end();
            inU = eU;
            strU = g.estride;
            inV = inU;
            strV = strU;
        }
    }
    const LevelGeom& gl = L.g[D - 1];
    pt.begin(1, D, 4.0 * L.P[D] * 4 * gl.e, leaf_limb_products(gl.e, L.P[D]));
    if (L.base == TC_BASE_NTT)
        CK(launch_ntt_mul(inU, strU, inV, strV, reinterpret_cast<u32*>(base + L.prod[D - 1]),
                          gl.ystride, gl.e, L.P[D], square, base + L.ntt, st));
    else
        CK(launch_leaf(inU, strU, inV, strV, reinterpret_cast<u32*>(base + L.prod[D - 1]), gl.ystride,
                       gl.e, L.P[D], st));
    pt.end();
    for (int l = D - 1; l >= 0; --l) {
        const LevelGeom& g = L.g[l];
        u32* out;
        long ostr;
        if (l == 0) {
            out = OUT;
            ostr = ldo;
        } else {
            out = reinterpret_cast<u32*>(base + L.prod[l - 1]);
            ostr = L.g[l - 1].ystride;
        }
        // squaring: every pointwise product U(x)^2 is non-negative, so no signs are passed
        const uint8_t* sU = square ? nullptr : reinterpret_cast<const uint8_t*>(base + L.sgnU[l]);
        const uint8_t* sV = square ? nullptr : reinterpret_cast<const uint8_t*>(base + L.sgnV[l]);
        u32* work = interp_work_bytes(g, L.P[l]) ? reinterpret_cast<u32*>(base + L.work[l]) : nullptr;
        pt.begin(2, l, 4.0 * L.P[l] * ((2.0 * g.B - 1) * 2 * g.e + 2.0 * g.s) +
                           (square ? 0.0 : 2.0 * (2 * g.B - 1) * L.P[l]), 0);
        CK(launch_interp(g, reinterpret_cast<const u32*>(base + L.prod[l]), sU, sV, out, ostr,
                         2 * g.s, work, L.P[l], st));
        pt.end();
    }
    // segment-parallel levels: a bounded wait that gave up (never expected) is
    // carried into the caller's sticky word by a kernel; nothing waits here
    if (sticky) {
        for (int l = 0; l < D; ++l) {
            if (use_wide(L.g[l], L.P[l]))
                CK(launch_or_error(sticky, wide_error_word(base + L.work[l], L.g[l], L.P[l]), st));
            if (use_wide_eval(L.g[l], L.P[l]))
                CK(launch_or_error(sticky, wide_eval_error_word(base + L.evwork[l], L.g[l], L.P[l]),
                                   st));
        }
    }
    return TC_OK;
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
static bool load_table(const char* path, std::vector<std::pair<size_t, tc_opts>>& out) {
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        unsigned long long mx;
        int lv, n = 0, pos = 0;
        if (sscanf(line, "%llu %d%n", &mx, &lv, &n) != 2) continue;
        pos = n;
        tc_opts o;
        memset(&o, 0, sizeof o);
        if (lv < 0 || lv > TC_MAX_LEVELS) continue;
        o.levels = lv;
        bool ok = true;
        for (int l = 0; l < lv; ++l) {
            if (sscanf(line + pos, "%d%n", &o.B[l], &n) != 1) { ok = false; break; }
            pos += n;
        }
        char word[16];
        if (ok && sscanf(line + pos, "%15s", word) == 1 && strcmp(word, "ntt") == 0) o.base = TC_BASE_NTT;
        if (ok) out.push_back({(size_t)mx, o});
    }
    fclose(f);
    return true;
}

extern "C" tc_status tc_create(tc_ctx** ctx, int device, size_t hbm_budget_bytes,
                               const char* tune_table_path) {
    if (!ctx) return TC_EINVAL;
    *ctx = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return TC_EINVAL;
    CK(cudaSetDevice(device));
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    tc_ctx* c = new tc_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes ? hbm_budget_bytes : fr / 4 * 3;
    if (tune_table_path && !load_table(tune_table_path, c->table)) {
        delete c;
        return TC_EINVAL;
    }
    cudaError_t e = cudaMalloc(&c->err_dev, 256);
    if (e == cudaSuccess) e = cudaMemset(c->err_dev, 0, 256);
    if (e != cudaSuccess) {
        if (c->err_dev) cudaFree(c->err_dev);
        delete c;
        return tc_fail_cuda(e);
    }
    *ctx = c;
    return TC_OK;
}

extern "C" void tc_destroy(tc_ctx* ctx) {
    if (!ctx) return;
    tc_serve_stop(ctx);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto& r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->arena) cudaFree(ctx->arena);
    if (ctx->aux) cudaFree(ctx->aux);
    if (ctx->err_dev) cudaFree(ctx->err_dev);
    ctx->fan.destroy();
    for (int i = 0; i < 2; ++i) {
        if (ctx->pin[i]) cudaFreeHost(ctx->pin[i]);
        if (ctx->pin_ev[i]) cudaEventDestroy(ctx->pin_ev[i]);
    }
    delete ctx;
}

extern "C" tc_status tc_plan_for(tc_ctx* ctx, size_t limbs, tc_opts* plan_out) {
    if (!plan_out || limbs == 0) return TC_EINVAL;
    *plan_out = plan_for(ctx, limbs);
    return TC_OK;
}

static tc_status resolve_plan(tc_ctx* ctx, size_t s, const tc_opts* opts, tc_opts& o) {
    o = opts ? *opts : plan_for(ctx, s);
    return plan_valid(o, s) ? TC_OK : TC_EINVAL;
}

extern "C" tc_status tc_scratch_bytes(tc_ctx* ctx, size_t count, size_t limbs, const tc_opts* opts,
                                      size_t* bytes_out) {
    if (!bytes_out || limbs == 0) return TC_EINVAL;
    tc_opts o;
    tc_status s = resolve_plan(ctx, limbs, opts, o);
    if (s) return s;
    *bytes_out = layout_for(count, limbs, o, false).total;
    return TC_OK;
}

// Uniform batch with the context's arena.
static tc_status mul_uniform(tc_ctx* ctx, size_t count, size_t limbs, const u32* A, size_t lda,
                             const u32* Bm, size_t ldb, u32* OUT, size_t ldo, const tc_opts* opts,
                             bool square, cudaStream_t st) {
    if (count == 0) return TC_OK;
    if (limbs == 0) return TC_OK;  // products of zero limbs have zero limbs
    tc_opts o;
    tc_status s = resolve_plan(ctx, limbs, opts, o);
    if (s) return s;
    BatchLayout L = layout_for(count, limbs, o, square);
    s = ensure_arena(ctx, L.total, st);
    if (s) return s;
    return run_uniform(L, (char*)ctx->arena, count, limbs, A, (long)lda, Bm, (long)ldb, OUT,
                       (long)ldo, square, st, ctx, ctx->err_dev);
}

extern "C" tc_status tc_mul_uniform(tc_ctx* ctx, size_t count, size_t limbs, const uint32_t* A,
                                    size_t lda, const uint32_t* Bv, size_t ldb, uint32_t* OUT,
                                    size_t ldo, const tc_opts* opts, void* stream) {
    if (!ctx || (count && (!A || !Bv || !OUT))) return TC_EINVAL;
    if (count > 1 && (lda < limbs || ldb < limbs || ldo < 2 * limbs)) return TC_EINVAL;
    CK(cudaSetDevice(ctx->device));
    const bool sq = (A == Bv && lda == ldb);
    return mul_uniform(ctx, count, limbs, A, lda, Bv, ldb, OUT, ldo, opts, sq, (cudaStream_t)stream);
}

extern "C" tc_status tc_mul_uniform_host(tc_ctx* ctx, size_t count, size_t limbs,
                                         const uint32_t* A, const uint32_t* Bv, uint32_t* OUT,
                                         const tc_opts* opts, void* stream) {
    if (!ctx || (count && (!A || !Bv || !OUT))) return TC_EINVAL;
    if (count == 0) return TC_OK;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t in_bytes = count * limbs * 4, out_bytes = count * 2 * limbs * 4;
    const size_t need = 2 * align256(in_bytes) + align256(out_bytes);
    if (need > ctx->aux_bytes) {
        CK(cudaStreamSynchronize(st));
        if (ctx->aux) cudaFree(ctx->aux);
        ctx->aux = nullptr;
        ctx->aux_bytes = 0;
        if (need > ctx->budget) return TC_ENOMEM;
        cudaError_t e = cudaMalloc(&ctx->aux, need);
        if (e != cudaSuccess) { cudaGetLastError(); return TC_ENOMEM; }
        ctx->aux_bytes = need;
    }
    char* base = (char*)ctx->aux;
    u32* dA = (u32*)base;
    u32* dB = (u32*)(base + align256(in_bytes));
    u32* dO = (u32*)(base + 2 * align256(in_bytes));
    CK(cudaMemcpyAsync(dA, A, in_bytes, cudaMemcpyHostToDevice, st));
    if (Bv != A) CK(cudaMemcpyAsync(dB, Bv, in_bytes, cudaMemcpyHostToDevice, st));
    tc_status s = mul_uniform(ctx, count, limbs, dA, limbs, Bv == A ? dA : dB, limbs, dO,
                              2 * limbs, opts, Bv == A, st);
    if (s) return s;
    CK(cudaMemcpyAsync(OUT, dO, out_bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return TC_OK;
}

// ---------------------------------------------------------------------------
// Pipelined host-buffer batches: two batches in flight, batch i+1's copy-in and
// batch i-1's copy-out overlap batch i's kernels.  Three streams ordered by
// events; device inputs, outputs and level scratch owned by the pipe.
// ---------------------------------------------------------------------------
struct tc_pipe {
    int device = 0;
    size_t count = 0, limbs = 0;
    bool square = false;
    BatchLayout L;
    char* mem = nullptr;  // level scratch, then per slot: A, B, OUT
    size_t in_bytes = 0, out_bytes = 0, scratch = 0;
    cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
    cudaEvent_t in_done[2] = {}, run_done[2] = {}, out_done[2] = {};
    int* err_dev = nullptr;  // sticky bounded-wait error word of the pipe's batches
    long submitted = 0;
    u32* slot_ptr(int slot, int which) const {  // which: 0 A, 1 B, 2 OUT
        const size_t per = 2 * align256(in_bytes) + align256(out_bytes);
        char* b = mem + scratch + slot * per;
        return (u32*)(which == 0 ? b : which == 1 ? b + align256(in_bytes) : b + 2 * align256(in_bytes));
    }
};

static void pipe_free(tc_pipe* p) {
    if (!p) return;
    cudaSetDevice(p->device);
    for (cudaStream_t s : {p->s_in, p->s_run, p->s_out})
        if (s) cudaStreamSynchronize(s);
    for (int i = 0; i < 2; ++i) {
        if (p->in_done[i]) cudaEventDestroy(p->in_done[i]);
        if (p->run_done[i]) cudaEventDestroy(p->run_done[i]);
        if (p->out_done[i]) cudaEventDestroy(p->out_done[i]);
    }
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_run) cudaStreamDestroy(p->s_run);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    if (p->mem) cudaFree(p->mem);
    if (p->err_dev) cudaFree(p->err_dev);
    delete p;
}

extern "C" tc_status tc_pipe_create(tc_ctx* ctx, size_t count, size_t limbs, int square,
                                    const tc_opts* opts, tc_pipe** out) {
    if (!ctx || !out || count == 0 || limbs == 0 || limbs > (1u << 30)) return TC_EINVAL;
    *out = nullptr;
    CK(cudaSetDevice(ctx->device));
    tc_opts o;
    tc_status s = resolve_plan(ctx, limbs, opts, o);
    if (s) return s;
    std::unique_ptr<tc_pipe, void (*)(tc_pipe*)> p(new tc_pipe, pipe_free);
    p->device = ctx->device;
    p->count = count;
    p->limbs = limbs;
    p->square = square != 0;
    p->L = layout_for(count, limbs, o, p->square);
    p->scratch = align256(p->L.total);
    p->in_bytes = count * limbs * 4;
    p->out_bytes = count * 2 * limbs * 4;
    const size_t need = p->scratch + 2 * (2 * align256(p->in_bytes) + align256(p->out_bytes));
    if (need > ctx->budget) return TC_ENOMEM;
    if (cudaMalloc(&p->mem, need) != cudaSuccess) {
        cudaGetLastError();
        p->mem = nullptr;
        return TC_ENOMEM;
    }
    CK(cudaMalloc(&p->err_dev, 256));
    CK(cudaMemset(p->err_dev, 0, 256));
    CK(cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&p->s_run, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
        CK(cudaEventCreateWithFlags(&p->in_done[i], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&p->run_done[i], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&p->out_done[i], cudaEventDisableTiming));
    }
    *out = p.release();
    return TC_OK;
}

extern "C" tc_status tc_pipe_submit(tc_ctx* ctx, tc_pipe* p, const uint32_t* A, const uint32_t* Bv,
                                    uint32_t* OUT) {
    if (!ctx || !p || !A || !OUT || (!p->square && !Bv)) return TC_EINVAL;
    if (ctx->device != p->device) return TC_EINVAL;
    CK(cudaSetDevice(p->device));
    const int slot = (int)(p->submitted & 1);
    u32* dA = p->slot_ptr(slot, 0);
    u32* dB = p->square ? dA : p->slot_ptr(slot, 1);
    u32* dO = p->slot_ptr(slot, 2);
    // copy-in: after the kernels of the batch two back stopped reading this slot
    CK(cudaStreamWaitEvent(p->s_in, p->run_done[slot], 0));
    CK(cudaMemcpyAsync(dA, A, p->in_bytes, cudaMemcpyHostToDevice, p->s_in));
    if (!p->square) CK(cudaMemcpyAsync(dB, Bv, p->in_bytes, cudaMemcpyHostToDevice, p->s_in));
    CK(cudaEventRecord(p->in_done[slot], p->s_in));
    // kernels: after this batch's copy-in and the copy-out of the batch two back
    CK(cudaStreamWaitEvent(p->s_run, p->in_done[slot], 0));
    CK(cudaStreamWaitEvent(p->s_run, p->out_done[slot], 0));
    tc_status s = run_uniform(p->L, p->mem, p->count, p->limbs, dA, (long)p->limbs, dB,
                              (long)p->limbs, dO, (long)(2 * p->limbs), p->square, p->s_run, ctx,
                              p->err_dev);
    if (s) return s;
    CK(cudaEventRecord(p->run_done[slot], p->s_run));
    // copy-out
    CK(cudaStreamWaitEvent(p->s_out, p->run_done[slot], 0));
    CK(cudaMemcpyAsync(OUT, dO, p->out_bytes, cudaMemcpyDeviceToHost, p->s_out));
    CK(cudaEventRecord(p->out_done[slot], p->s_out));
    ++p->submitted;
    return TC_OK;
}

extern "C" tc_status tc_pipe_wait(tc_pipe* p) {
    if (!p) return TC_EINVAL;
    CK(cudaSetDevice(p->device));
    CK(cudaStreamSynchronize(p->s_out));  // its last copy waits on every earlier step
    CK(cudaStreamSynchronize(p->s_run));
    CK(cudaStreamSynchronize(p->s_in));
    int flag = 0;
    CK(cudaMemcpy(&flag, p->err_dev, sizeof flag, cudaMemcpyDeviceToHost));
    if (flag) {
        CK(cudaMemset(p->err_dev, 0, sizeof flag));
        return TC_ETIMEOUT;
    }
    return TC_OK;
}

extern "C" void tc_pipe_destroy(tc_pipe* p) { pipe_free(p); }

// ---------------------------------------------------------------------------
// General products: gather into padded rows per size class, run, scatter.
// ---------------------------------------------------------------------------
namespace {

__global__ void gather_rows(const u32* src, const int64_t* off, const int64_t* len, int s,
                            u32* dst, int count) {
    const int k = blockIdx.y;
    if (k >= count) return;
    const u32* a = src + off[k];
    const int64_t L = len[k];
    u32* d = dst + (long)k * s;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s; i += gridDim.x * blockDim.x)
        d[i] = i < L ? a[i] : 0u;
}

__global__ void scatter_rows(const u32* src, int stride, const int64_t* off, const int64_t* len,
                             u32* dst, int count) {
    const int k = blockIdx.y;
    if (k >= count) return;
    const u32* s = src + (long)k * stride;
    u32* d = dst + off[k];
    const int64_t L = len[k];
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < L; i += (long)gridDim.x * blockDim.x)
        d[i] = s[i];
}

// Device tables (tc_mul_batch_dev): row k of the padded batch from product k's
// operand, or zeros and the sticky "invalid" bit when the entry is out of range.
__global__ void gather_rows_checked(const u32* src, const int64_t* off, const int64_t* len, int s,
                                    int64_t max_len, u32* dst, int count, int* sticky) {
    const int k = blockIdx.y;
    if (k >= count) return;
    const int64_t L = len[k], o = off[k];
    const bool ok = L >= 0 && L <= max_len && o >= 0;
    if (!ok && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(sticky, TC_STICKY_INVALID);
    const u32* a = src + (ok ? o : 0);
    u32* d = dst + (long)k * s;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s; i += gridDim.x * blockDim.x)
        d[i] = ok && i < L ? a[i] : 0u;
}

__global__ void scatter_rows_checked(const u32* src, int stride, const int64_t* off, const int64_t* alen,
                                     const int64_t* blen, int64_t max_len, u32* dst, int count) {
    const int k = blockIdx.y;
    if (k >= count) return;
    const int64_t la = alen[k], lb = blen[k], o = off[k];
    if (la < 0 || lb < 0 || la > max_len || lb > max_len || o < 0) return;  // reported by the gather
    const u32* s = src + (long)k * stride;
    u32* d = dst + o;
    const int64_t L = la + lb;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < L; i += (long)gridDim.x * blockDim.x)
        d[i] = s[i];
}

}  // namespace

size_t tc::size_class(size_t L) {
    // classes 2^k and 3 * 2^(k-1): at most 50% padding
    size_t c = 32;
    while (c < L) {
        size_t mid = c + c / 2;
        if (mid >= L) return mid;
        c *= 2;
    }
    return c;
}

// Host index arrays of a packed batch: every offset >= 0 and below 2^40 limbs,
// every length in [0, 2^28] limbs (the serving limit), checked before any launch
// so that no gather or scatter is given an address outside the caller's buffers'
// possible range.
static bool batch_tables_valid(size_t count, const int64_t* a_off, const int64_t* a_len,
                               const int64_t* b_off, const int64_t* b_len, const int64_t* out_off) {
    const int64_t kMaxLen = (int64_t)1 << 28, kMaxOff = (int64_t)1 << 40;
    for (size_t k = 0; k < count; ++k) {
        if (a_len[k] < 0 || b_len[k] < 0 || a_len[k] > kMaxLen || b_len[k] > kMaxLen) return false;
        if (a_off[k] < 0 || b_off[k] < 0 || out_off[k] < 0) return false;
        if (a_off[k] > kMaxOff || b_off[k] > kMaxOff || out_off[k] > kMaxOff) return false;
    }
    return true;
}

// Pinned host staging for `bytes` of index tables (one of two buffers, in turn).
// A buffer is rewritten only after the copy that last read it has completed:
// the copy was enqueued ahead of that call's kernels, so this waits for at most
// the work enqueued before the previous call, never for the previous call itself.
static tc_status stage_tables(tc_ctx* ctx, size_t bytes, void** host) {
    const int t = ctx->pin_turn;
    if (ctx->pin_ev[t]) CK(cudaEventSynchronize(ctx->pin_ev[t]));
    else CK(cudaEventCreateWithFlags(&ctx->pin_ev[t], cudaEventDisableTiming));
    if (bytes > ctx->pin_bytes[t]) {  // grow (allocation path)
        if (ctx->pin[t]) CK(cudaFreeHost(ctx->pin[t]));
        ctx->pin[t] = nullptr;
        ctx->pin_bytes[t] = 0;
        const size_t want = std::max(bytes, (size_t)64 << 10);
        CK(cudaHostAlloc(&ctx->pin[t], want, cudaHostAllocDefault));
        ctx->pin_bytes[t] = want;
    }
    *host = ctx->pin[t];
    return TC_OK;
}

// Products listed by (offset, length) triples; all device limb buffers, host index arrays
// (validated by batch_tables_valid).  Asynchronous: the tables of every size class
// go to the device in one copy from pinned staging; the classes are independent, so
// each gets its own scratch region and they run concurrently on the context's stream
// fan (a class of a few hundred products alone leaves most of the GPU idle).
static tc_status mul_general(tc_ctx* ctx, size_t count, const u32* A, const int64_t* a_off,
                             const int64_t* a_len, const u32* Bm, const int64_t* b_off,
                             const int64_t* b_len, u32* OUT, const int64_t* out_off,
                             const tc_opts* opts, cudaStream_t st) {
    // classes by padded balanced length
    struct Item { size_t k, cls; };
    std::vector<Item> items;
    items.reserve(count);
    for (size_t k = 0; k < count; ++k) {
        const size_t L = (size_t)std::max(a_len[k], b_len[k]);
        if (a_len[k] == 0 || b_len[k] == 0) {
            const size_t n = (size_t)(a_len[k] + b_len[k]);
            if (n) CK(cudaMemsetAsync(OUT + out_off[k], 0, n * 4, st));
            continue;
        }
        items.push_back({k, size_class(L)});
    }
    if (items.empty()) return TC_OK;
    std::sort(items.begin(), items.end(), [](const Item& x, const Item& y) { return x.cls < y.cls; });
    struct Class { size_t s, cnt, first, off; BatchLayout L; };
    std::vector<Class> classes;
    size_t need = 0;  // sum of the classes' regions
    for (size_t i = 0; i < items.size();) {
        size_t j = i;
        while (j < items.size() && items[j].cls == items[i].cls) ++j;
        Class c;
        c.s = items[i].cls;
        c.cnt = j - i;
        c.first = i;
        // a caller's plan applies to every size class it is valid for
        const tc_opts o = (opts && plan_valid(*opts, c.s)) ? *opts : plan_for(ctx, c.s);
        c.L = layout_for(c.cnt, c.s, o, false);
        c.off = need;
        need += align256(c.L.total + 2 * align256(c.cnt * c.s * 4) + align256(c.cnt * 2 * c.s * 4));
        classes.push_back(std::move(c));
        i = j;
    }
    // index tables: aoff, alen, boff, blen, ooff, olen, each N long, in class order
    const size_t N = items.size();
    const size_t tab_bytes = 6 * N * 8;
    tc_status e = ensure_arena(ctx, align256(need) + align256(tab_bytes), st);
    if (e) return e;
    void* hv = nullptr;
    if ((e = stage_tables(ctx, tab_bytes, &hv))) return e;
    int64_t* h = static_cast<int64_t*>(hv);
    for (size_t t = 0; t < N; ++t) {
        const size_t k = items[t].k;
        h[t] = a_off[k];
        h[N + t] = a_len[k];
        h[2 * N + t] = b_off[k];
        h[3 * N + t] = b_len[k];
        h[4 * N + t] = out_off[k];
        h[5 * N + t] = a_len[k] + b_len[k];
    }
    char* arena = (char*)ctx->arena;
    int64_t* dtab = (int64_t*)(arena + align256(need));
    CK(cudaMemcpyAsync(dtab, h, tab_bytes, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(ctx->pin_ev[ctx->pin_turn], st));
    ctx->pin_turn ^= 1;
    const bool fan = classes.size() > 1;
    if (fan) {
        CK(ctx->fan.init());
        CK(ctx->fan.fork(st));
    }
    // the largest classes first, each on the next stream of the fan
    for (size_t ci = classes.size(); ci-- > 0;) {
        const Class& c = classes[ci];
        const cudaStream_t cs = fan ? ctx->fan.s[(classes.size() - 1 - ci) % StreamFan::K] : st;
        char* base = arena + c.off;
        const size_t s = c.s, cnt = c.cnt;
        u32* rA = (u32*)(base + c.L.total);
        u32* rB = (u32*)((char*)rA + align256(cnt * s * 4));
        u32* rO = (u32*)((char*)rB + align256(cnt * s * 4));
        const int64_t* aoff = dtab + c.first;
        const int64_t* alen = dtab + N + c.first;
        const int64_t* boff = dtab + 2 * N + c.first;
        const int64_t* blen = dtab + 3 * N + c.first;
        const int64_t* ooff = dtab + 4 * N + c.first;
        const int64_t* olen = dtab + 5 * N + c.first;
        for (size_t c0 = 0; c0 < cnt; c0 += 65535) {
            const int cc = (int)std::min<size_t>(65535, cnt - c0);
            dim3 grid((unsigned)std::min<size_t>((s + 255) / 256, 64), cc);
            gather_rows<<<grid, 256, 0, cs>>>(A, aoff + c0, alen + c0, (int)s, rA + c0 * s, cc);
            gather_rows<<<grid, 256, 0, cs>>>(Bm, boff + c0, blen + c0, (int)s, rB + c0 * s, cc);
        }
        CK(cudaGetLastError());
        e = run_uniform(c.L, base, cnt, s, rA, (long)s, rB, (long)s, rO, (long)(2 * s), false, cs, ctx,
                        ctx->err_dev);
        if (e) return e;
        for (size_t c0 = 0; c0 < cnt; c0 += 65535) {
            const int cc = (int)std::min<size_t>(65535, cnt - c0);
            dim3 grid((unsigned)std::min<size_t>((2 * s + 255) / 256, 64), cc);
            scatter_rows<<<grid, 256, 0, cs>>>(rO + c0 * 2 * s, (int)(2 * s), ooff + c0, olen + c0,
                                               OUT, cc);
        }
        CK(cudaGetLastError());
    }
    if (fan) CK(ctx->fan.join(st));
    return TC_OK;
}

extern "C" tc_status tc_mul_batch(tc_ctx* ctx, size_t count, const uint32_t* A, const int64_t* a_off,
                                  const int64_t* a_len, const uint32_t* Bv, const int64_t* b_off,
                                  const int64_t* b_len, uint32_t* OUT, const int64_t* out_off,
                                  const tc_opts* opts, void* stream) {
    if (!ctx) return TC_EINVAL;
    if (count == 0) return TC_OK;
    if (!A || !Bv || !OUT || !a_off || !a_len || !b_off || !b_len || !out_off) return TC_EINVAL;
    if (!batch_tables_valid(count, a_off, a_len, b_off, b_len, out_off)) return TC_EINVAL;
    CK(cudaSetDevice(ctx->device));
    return mul_general(ctx, count, A, a_off, a_len, Bv, b_off, b_len, OUT, out_off, opts,
                       (cudaStream_t)stream);
}

// Products listed by DEVICE (offset, length) tables: the host never reads them.
// Every product is padded to the balanced size class of max_limbs; entries out of
// range are skipped on the device and raise the context's "invalid" bit.
extern "C" tc_status tc_mul_batch_dev(tc_ctx* ctx, size_t count, const uint32_t* A,
                                      const int64_t* a_off, const int64_t* a_len, const uint32_t* Bv,
                                      const int64_t* b_off, const int64_t* b_len, uint32_t* OUT,
                                      const int64_t* out_off, size_t max_limbs, const tc_opts* opts,
                                      void* stream) {
    if (!ctx) return TC_EINVAL;
    if (count == 0) return TC_OK;
    if (!A || !Bv || !OUT || !a_off || !a_len || !b_off || !b_len || !out_off) return TC_EINVAL;
    if (max_limbs == 0 || max_limbs > ((size_t)1 << 28) || count > ((size_t)1 << 31)) return TC_EINVAL;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t s = size_class(max_limbs);
    tc_opts o;
    tc_status e = resolve_plan(ctx, s, opts, o);
    if (e) return e;
    const BatchLayout L = layout_for(count, s, o, false);
    const size_t rows_bytes = align256(count * s * 4);
    e = ensure_arena(ctx, L.total + 2 * rows_bytes + align256(count * 2 * s * 4), st);
    if (e) return e;
    char* base = (char*)ctx->arena;
    u32* rA = (u32*)(base + L.total);
    u32* rB = (u32*)((char*)rA + rows_bytes);
    u32* rO = (u32*)((char*)rB + rows_bytes);
    for (size_t c0 = 0; c0 < count; c0 += 65535) {
        const int cc = (int)std::min<size_t>(65535, count - c0);
        dim3 grid((unsigned)std::min<size_t>((s + 255) / 256, 64), cc);
        gather_rows_checked<<<grid, 256, 0, st>>>(A, a_off + c0, a_len + c0, (int)s, (int64_t)max_limbs,
                                                  rA + c0 * s, cc, ctx->err_dev);
        gather_rows_checked<<<grid, 256, 0, st>>>(Bv, b_off + c0, b_len + c0, (int)s, (int64_t)max_limbs,
                                                  rB + c0 * s, cc, ctx->err_dev);
    }
    CK(cudaGetLastError());
    e = run_uniform(L, base, count, s, rA, (long)s, rB, (long)s, rO, (long)(2 * s), false, st, ctx,
                    ctx->err_dev);
    if (e) return e;
    for (size_t c0 = 0; c0 < count; c0 += 65535) {
        const int cc = (int)std::min<size_t>(65535, count - c0);
        dim3 grid((unsigned)std::min<size_t>((2 * s + 255) / 256, 64), cc);
        scatter_rows_checked<<<grid, 256, 0, st>>>(rO + c0 * 2 * s, (int)(2 * s), out_off + c0,
                                                   a_len + c0, b_len + c0, (int64_t)max_limbs, OUT, cc);
    }
    CK(cudaGetLastError());
    return TC_OK;
}

// ---------------------------------------------------------------------------
// Prepared batches: the host work of tc_mul_batch (grouping into size
// classes, index tables, scratch) done once, so that running the batch is
// kernel launches and memsets only, with no host synchronisation: it can be
// captured into a CUDA graph and replayed.
// ---------------------------------------------------------------------------
struct tc_batch {
    int device = 0;
    struct Class {
        size_t s = 0, cnt = 0;
        BatchLayout L;
        size_t tab = 0;  // first entry of this class in each index table
        size_t off = 0;  // this class's region of the scratch
    };
    std::vector<Class> classes;
    std::vector<std::pair<int64_t, int64_t>> zeros;  // (out offset, limbs) of empty products
    int64_t* tables = nullptr;  // device: aoff, alen, boff, blen, ooff, olen (each `total` long)
    size_t total = 0;
    char* scratch = nullptr;    // device: one region per class (level scratch + rows + outputs)
    size_t scratch_bytes = 0;
    int* err_dev = nullptr;     // device: sticky bounded-wait error word of the runs
    StreamFan fan;              // the classes run concurrently on these
};

extern "C" void tc_batch_destroy(tc_batch* bt);

static size_t class_extra(size_t cnt, size_t s) {
    return 2 * align256(cnt * s * 4) + align256(cnt * 2 * s * 4);
}

extern "C" tc_status tc_batch_prepare(tc_ctx* ctx, size_t count, const int64_t* a_off,
                                      const int64_t* a_len, const int64_t* b_off,
                                      const int64_t* b_len, const int64_t* out_off,
                                      const tc_opts* opts, tc_batch** out) {
    if (!ctx || !out || (count && (!a_off || !a_len || !b_off || !b_len || !out_off))) return TC_EINVAL;
    *out = nullptr;
    if (!batch_tables_valid(count, a_off, a_len, b_off, b_len, out_off)) return TC_EINVAL;
    CK(cudaSetDevice(ctx->device));
    std::unique_ptr<tc_batch> bt(new tc_batch);
    bt->device = ctx->device;
    struct Item { size_t k, cls; };
    std::vector<Item> items;
    for (size_t k = 0; k < count; ++k) {
        if (a_len[k] == 0 || b_len[k] == 0) {
            if (a_len[k] + b_len[k]) bt->zeros.push_back({out_off[k], a_len[k] + b_len[k]});
            continue;
        }
        items.push_back({k, size_class((size_t)std::max(a_len[k], b_len[k]))});
    }
    std::sort(items.begin(), items.end(), [](const Item& x, const Item& y) { return x.cls < y.cls; });
    std::vector<int64_t> h(6 * items.size());
    const size_t N = items.size();
    size_t need = 0;
    for (size_t i = 0; i < N;) {
        size_t j = i;
        while (j < N && items[j].cls == items[i].cls) ++j;
        tc_batch::Class c;
        c.s = items[i].cls;
        c.cnt = j - i;
        c.tab = i;
        const tc_opts o = (opts && plan_valid(*opts, c.s)) ? *opts : plan_for(ctx, c.s);
        c.L = layout_for(c.cnt, c.s, o, false);
        c.off = need;
        need += align256(c.L.total + class_extra(c.cnt, c.s));
        for (size_t t = i; t < j; ++t) {
            const size_t k = items[t].k;
            h[t] = a_off[k];
            h[N + t] = a_len[k];
            h[2 * N + t] = b_off[k];
            h[3 * N + t] = b_len[k];
            h[4 * N + t] = out_off[k];
            h[5 * N + t] = a_len[k] + b_len[k];
        }
        bt->classes.push_back(c);
        i = j;
    }
    if (need > ctx->budget) return TC_ENOMEM;
    bt->total = N;
    // on any failure below the partly built batch is released with its device memory
    auto fail = [&](tc_status st) {
        tc_batch_destroy(bt.release());
        return st;
    };
    if (cudaMalloc(&bt->err_dev, 256) != cudaSuccess) { cudaGetLastError(); return fail(TC_ENOMEM); }
    cudaError_t e = cudaMemset(bt->err_dev, 0, 256);
    if (e != cudaSuccess) return fail(tc_fail_cuda(e));
    if (bt->classes.size() > 1 && (e = bt->fan.init()) != cudaSuccess) return fail(tc_fail_cuda(e));
    if (N) {
        if (cudaMalloc(&bt->tables, h.size() * 8) != cudaSuccess) {
            cudaGetLastError();
            return fail(TC_ENOMEM);
        }
        if (cudaMalloc(&bt->scratch, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(TC_ENOMEM);
        }
        bt->scratch_bytes = need;
        e = cudaMemcpy(bt->tables, h.data(), h.size() * 8, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(tc_fail_cuda(e));
    }
    *out = bt.release();
    return TC_OK;
}

extern "C" tc_status tc_batch_run(tc_ctx* ctx, const tc_batch* bt, const uint32_t* A,
                                  const uint32_t* Bv, uint32_t* OUT, void* stream) {
    if (!ctx || !bt || bt->device != ctx->device) return TC_EINVAL;
    if (bt->total && (!A || !Bv || !OUT)) return TC_EINVAL;
    if (!bt->total && !bt->zeros.empty() && !OUT) return TC_EINVAL;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    for (const auto& z : bt->zeros) CK(cudaMemsetAsync(OUT + z.first, 0, (size_t)z.second * 4, st));
    const size_t N = bt->total;
    // the classes are independent: each on the next stream of the fan (largest first)
    tc::StreamFan& fan = const_cast<tc::StreamFan&>(bt->fan);
    const bool fanned = fan.ready;
    if (fanned) CK(fan.fork(st));
    for (size_t ci = bt->classes.size(); ci-- > 0;) {
        const auto& c = bt->classes[ci];
        const cudaStream_t cs = fanned ? fan.s[(bt->classes.size() - 1 - ci) % StreamFan::K] : st;
        char* base = bt->scratch + c.off;
        u32* rA = (u32*)(base + c.L.total);
        u32* rB = (u32*)((char*)rA + align256(c.cnt * c.s * 4));
        u32* rO = (u32*)((char*)rB + align256(c.cnt * c.s * 4));
        const int64_t* aoff = bt->tables + c.tab;
        const int64_t* alen = bt->tables + N + c.tab;
        const int64_t* boff = bt->tables + 2 * N + c.tab;
        const int64_t* blen = bt->tables + 3 * N + c.tab;
        const int64_t* ooff = bt->tables + 4 * N + c.tab;
        const int64_t* olen = bt->tables + 5 * N + c.tab;
        for (size_t c0 = 0; c0 < c.cnt; c0 += 65535) {
            const int cc = (int)std::min<size_t>(65535, c.cnt - c0);
            dim3 grid((unsigned)std::min<size_t>((c.s + 255) / 256, 64), cc);
            gather_rows<<<grid, 256, 0, cs>>>(A, aoff + c0, alen + c0, (int)c.s, rA + c0 * c.s, cc);
            gather_rows<<<grid, 256, 0, cs>>>(Bv, boff + c0, blen + c0, (int)c.s, rB + c0 * c.s, cc);
        }
        CK(cudaGetLastError());
        // no context: no phase events and no host read-back inside a possibly captured run
        tc_status e = run_uniform(c.L, base, c.cnt, c.s, rA, (long)c.s, rB, (long)c.s, rO,
                                  (long)(2 * c.s), false, cs, nullptr, bt->err_dev);
        if (e) return e;
        for (size_t c0 = 0; c0 < c.cnt; c0 += 65535) {
            const int cc = (int)std::min<size_t>(65535, c.cnt - c0);
            dim3 grid((unsigned)std::min<size_t>((2 * c.s + 255) / 256, 64), cc);
            scatter_rows<<<grid, 256, 0, cs>>>(rO + c0 * 2 * c.s, (int)(2 * c.s), ooff + c0,
                                               olen + c0, OUT, cc);
        }
        CK(cudaGetLastError());
    }
    if (fanned) CK(fan.join(st));
    return TC_OK;
}

extern "C" size_t tc_batch_scratch_bytes(const tc_batch* bt) { return bt ? bt->scratch_bytes : 0; }

// After a run (direct or replayed) has completed on `stream`: TC_ETIMEOUT if a
// bounded wait of a segment-parallel level gave up in any run since the last
// check (the word is cleared), else TC_OK.  Synchronises.
extern "C" tc_status tc_batch_check(tc_ctx* ctx, const tc_batch* bt, void* stream) {
    if (!ctx || !bt || bt->device != ctx->device) return TC_EINVAL;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(st));
    int flag = 0;
    CK(cudaMemcpy(&flag, bt->err_dev, sizeof flag, cudaMemcpyDeviceToHost));
    if (flag) {
        CK(cudaMemset(bt->err_dev, 0, sizeof flag));
        return TC_ETIMEOUT;
    }
    return TC_OK;
}

/* The context's sticky bounded-wait error word: waits for `stream`, then
 * TC_ETIMEOUT (and clears the word) if a segment-parallel level of any call on
 * this context since the last check gave up a wait. */
extern "C" tc_status tc_check(tc_ctx* ctx, void* stream) {
    if (!ctx) return TC_EINVAL;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    int flag = 0;
    CK(cudaMemcpy(&flag, ctx->err_dev, sizeof flag, cudaMemcpyDeviceToHost));
    if (flag) {
        CK(cudaMemset(ctx->err_dev, 0, sizeof flag));
        return (flag & TC_STICKY_INVALID) ? TC_EINVAL : TC_ETIMEOUT;
    }
    return TC_OK;
}

extern "C" void tc_batch_destroy(tc_batch* bt) {
    if (!bt) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(bt->device);
    bt->fan.destroy();
    if (bt->tables) cudaFree(bt->tables);
    if (bt->scratch) cudaFree(bt->scratch);
    if (bt->err_dev) cudaFree(bt->err_dev);
    cudaSetDevice(cur);
    delete bt;
}

extern "C" tc_status tc_mul(tc_ctx* ctx, const uint32_t* a, size_t na, const uint32_t* b, size_t nb,
                            uint32_t* out, const tc_opts* opts, void* stream) {
    if (!ctx || !out || (na && !a) || (nb && !b)) return TC_EINVAL;
    if (na > ((size_t)1 << 30) || nb > ((size_t)1 << 30)) return TC_EINVAL;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (na == 0 || nb == 0) {
        if (na + nb) CK(cudaMemsetAsync(out, 0, (na + nb) * 4, st));
        return TC_OK;
    }
    if (na == nb) {
        const bool sq = (a == b);
        return mul_uniform(ctx, 1, na, a, na, b, nb, out, 2 * na, opts, sq, st);
    }
    const size_t lo = std::min(na, nb), hi = std::max(na, nb);
    const uint32_t* longp = na >= nb ? a : b;
    const uint32_t* shortp = na >= nb ? b : a;
    if (hi < 2 * lo) {
        int64_t ao = 0, al = (int64_t)na, bo = 0, bl = (int64_t)nb, oo = 0;
        return mul_general(ctx, 1, a, &ao, &al, b, &bo, &bl, out, &oo, opts, st);
    }
    // slices of the longer operand, each lo limbs (last one shorter), as one batch
    const size_t pieces = (hi + lo - 1) / lo;
    // one uniform batch of `pieces` products lo x lo (the short operand replicated by stride 0)
    tc_opts o;
    tc_status s = resolve_plan(ctx, lo, opts, o);
    if (s) return s;
    BatchLayout L = layout_for(pieces, lo, o, false);
    const size_t rows_bytes = align256(pieces * lo * 4);
    const size_t outs_bytes = align256(pieces * 2 * lo * 4);
    s = ensure_arena(ctx, L.total + rows_bytes + outs_bytes, st);
    if (s) return s;
    char* base = (char*)ctx->arena;
    u32* rA = (u32*)(base + L.total);
    u32* rO = (u32*)(base + L.total + rows_bytes);
    CK(cudaMemsetAsync(rA, 0, pieces * lo * 4, st));
    CK(cudaMemcpyAsync(rA, longp, hi * 4, cudaMemcpyDeviceToDevice, st));
    s = run_uniform(L, base, pieces, lo, rA, (long)lo, shortp, 0, rO, (long)(2 * lo), false, st, ctx,
                    ctx->err_dev);
    if (s) return s;
    CK(launch_overlap_add(rO, (long)(2 * lo), (int)(2 * lo), (int)pieces, (long)lo, out,
                          (long)(na + nb), st));
    return TC_OK;
}

extern "C" tc_status tc_sqr(tc_ctx* ctx, const uint32_t* a, size_t na, uint32_t* out,
                            const tc_opts* opts, void* stream) {
    return tc_mul(ctx, a, na, a, na, out, opts, stream);
}

// ---------------------------------------------------------------------------
// Steps of one level
// ---------------------------------------------------------------------------
extern "C" tc_status tc_schoolbook(size_t count, size_t limbs, const uint32_t* A, size_t lda,
                                   const uint32_t* Bv, size_t ldb, uint32_t* OUT, size_t ldo,
                                   void* stream) {
    if (count == 0) return TC_OK;
    if (!A || !Bv || !OUT || limbs == 0 || limbs > (size_t)LEAF_MAX) return TC_EINVAL;
    if (count > 1 && (lda < limbs || ldb < limbs || ldo < 2 * limbs)) return TC_EINVAL;
    CK(launch_leaf(A, (long)lda, Bv, (long)ldb, OUT, (long)ldo, (int)limbs, (long)count,
                   (cudaStream_t)stream));
    return TC_OK;
}

extern "C" tc_status tc_toom_evaluate(size_t count, size_t limbs, int B, const uint32_t* U,
                                      size_t ld, uint32_t* OUT, size_t estride, uint8_t* SGN,
                                      void* stream) {
    if (count == 0) return TC_OK;
    if (!U || !OUT || !SGN || B < 2 || B > 32 || limbs == 0 || limbs > (1u << 30))
        return TC_EINVAL;
    LevelGeom g = make_level((int)limbs, B);
    if (estride < (size_t)g.e || estride % 4 || (reinterpret_cast<uintptr_t>(OUT) & 15u))
        return TC_EINVAL;
    if (count > 1 && ld < limbs) return TC_EINVAL;
    g.estride = (int)estride;
    CK(launch_eval(U, (long)ld, g, OUT, SGN, (long)count, nullptr, (cudaStream_t)stream));
    return TC_OK;
}

extern "C" size_t tc_toom_interpolate_work_bytes(size_t count, size_t limbs, int B) {
    if (B < 2 || B > 32 || limbs == 0 || limbs > (1u << 30)) return 0;
    return count * interp_work_bytes(make_level((int)limbs, B), (long)count);
}

extern "C" tc_status tc_toom_interpolate(size_t count, size_t limbs, int B, const uint32_t* Y,
                                         size_t ystride, const uint8_t* SGN_U,
                                         const uint8_t* SGN_V, uint32_t* OUT, size_t ldo,
                                         void* work, void* stream) {
    if (count == 0) return TC_OK;
    if (!Y || !OUT || B < 2 || B > 32 || limbs == 0 || limbs > (1u << 30)) return TC_EINVAL;
    LevelGeom g = make_level((int)limbs, B);
    if (ystride < (size_t)(2 * g.e) || ystride % 4) return TC_EINVAL;
    if (((reinterpret_cast<uintptr_t>(Y) | reinterpret_cast<uintptr_t>(work)) & 15u) != 0)
        return TC_EINVAL;
    if (count > 1 && ldo < 2 * limbs) return TC_EINVAL;
    if (interp_work_bytes(g, (long)count) && !work) return TC_EINVAL;
    g.ystride = (int)ystride;
    CK(launch_interp(g, Y, SGN_U, SGN_V, OUT, (long)ldo, 2 * g.s, (u32*)work, (long)count,
                     (cudaStream_t)stream));
    return TC_OK;
}

// ---------------------------------------------------------------------------
// Phase timing
// ---------------------------------------------------------------------------
extern "C" tc_status tc_profile_enable(tc_ctx* ctx, int on) {
    if (!ctx) return TC_EINVAL;
    CK(cudaSetDevice(ctx->device));
    for (auto& r : ctx->recs) {
        cudaEventSynchronize(r.b);
        ctx->event_pool.push_back(r.a);
        ctx->event_pool.push_back(r.b);
    }
    ctx->recs.clear();
    ctx->profile = on != 0;
    return TC_OK;
}

extern "C" tc_status tc_profile_read(tc_ctx* ctx, tc_phase_stat* out, int cap, int* n) {
    if (!ctx || !n || (cap > 0 && !out)) return TC_EINVAL;
    CK(cudaSetDevice(ctx->device));
    std::vector<tc_phase_stat> acc;
    for (auto& r : ctx->recs) {
        CK(cudaEventSynchronize(r.b));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        tc_phase_stat* p = nullptr;
        for (auto& x : acc)
            if (x.kind == r.kind && x.level == r.level) p = &x;
        if (!p) {
            tc_phase_stat x;
            memset(&x, 0, sizeof x);
            x.kind = r.kind;
            x.level = r.level;
            snprintf(x.kernel, sizeof x.kernel, "%s", r.kernel ? r.kernel : "");
            acc.push_back(x);
            p = &acc.back();
        }
        p->launches += 1;
        p->ms += ms;
        p->bytes += r.bytes;
        p->limb_products += r.lp;
    }
    std::sort(acc.begin(), acc.end(), [](const tc_phase_stat& x, const tc_phase_stat& y) {
        return x.kind != y.kind ? x.kind < y.kind : x.level < y.level;
    });
    int k = 0;
    for (; k < cap && k < (int)acc.size(); ++k) out[k] = acc[k];
    *n = k;
    return TC_OK;
}
