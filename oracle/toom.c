/*
 * Oracle: plain recursive B-way Toom-Cook multiplication in C.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline and reference legs may load this code.  The
 * library's product path never calls it, and it shares no code with the
 * library.
 *
 * The same method as oracle/toom.py (which works on Python integers), written
 * out on limb arrays so that products of 2^24 to 2^27 bits finish in seconds.
 * The steps are taken in the paper's order and notation, one level at a time:
 *
 *  1. Split (Section 1, eq. 1.1-1.3): u = U(2^(32 b)) with B blocks u_0..u_n of
 *     b = ceil(L / B) limbs, n = B - 1, the top block zero-padded.
 *  2. Evaluate (Section 4, eq. 4.1; the points of Section 6): for x = 2^j,
 *     j = 0..n-1, the even part E = sum_{i even} u_i x^i and the odd part
 *     O = sum_{i odd} u_i x^i; U(x) = E + O and U(-x) = E - O kept as a
 *     magnitude and a sign; U(0) = u_0.  Point order 0, +1, -1, +2, -2, ...
 *     Every value fits e = b + ceil((n(n-1)+1)/32) limbs.
 *  3. Pointwise products y = U(x) V(x) (Section 1): the magnitudes are
 *     multiplied by this same procedure with the next B of the plan, and below
 *     the last level by the plain schoolbook (schoolbook.c); the sign of y is
 *     the product of the signs.
 *  4. Even-odd combine (Section 4, eq. 4.5-4.6): ye_0 = y(0), yo_0 = 0, and for
 *     x = 2^(k-1): ye_k = (W(x) + W(-x)) / 2, yo_k = x (W(x) - W(-x)) / 2.
 *  5. Newton divided differences (Section 3, Theorem 3.2) on the nodes
 *     X = 0, 1, 4, ..., 4^(n-1): column k of the table at positions k..n,
 *     entry m + k = (previous entry m + k - previous entry m + k - 1) divided
 *     by X_(m+k) - X_m.  Each division is plain long division by the whole
 *     divisor (up to 2^62 at B = 32), from the top limb down, and its
 *     remainder must be zero.
 *  6. Newton basis to monomial basis (Section 3, Theorem 3.3): for m = n-1
 *     down to 0 and k = m..n-1, beta_k -= X_m beta_(k+1) (old values), the
 *     product X_m beta_(k+1) formed by multiplying by the word X_m.
 *  7. Re-interleave (eq. 4.3): w_(2i) = ce_i, w_(2i+1) = co_(i+1); recompose
 *     w = sum_k w_k 2^(32 b k) into exactly 2L limbs.
 *
 * Every subtraction must not underflow (with non-negative blocks every
 * interpolation intermediate is non-negative), every division must be exact,
 * every value must fit its stated length, and the recomposition must fit 2L
 * limbs; a violation makes the call return a nonzero code instead of a result.
 *
 * oracle_toom_mul runs the 2B-1 top-level products on up to `threads` POSIX
 * threads, the paper's own parallel scheme (Section 2: the products of the
 * top level are independent); below the top level everything is sequential.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void oracle_schoolbook(const uint32_t *a, size_t na, const uint32_t *b, size_t nb, uint32_t *out);

typedef unsigned __int128 u128;

enum {
    T_OK = 0,
    T_UNDERFLOW = 1,   /* a subtraction went below zero */
    T_INEXACT = 2,     /* a division left a remainder */
    T_OVERFLOW = 3,    /* a value did not fit its stated length */
    T_NOMEM = 4,
    T_BADPLAN = 5
};

/* ---------------------------------------------------------------- limb arithmetic
 * Fixed-length little-endian arrays of N limbs. */

/* r += x (N limbs); returns the carry out. */
static uint32_t nat_add(uint32_t *r, const uint32_t *x, size_t N)
{
    uint64_t c = 0;
    for (size_t i = 0; i < N; ++i) {
        c += (uint64_t)r[i] + x[i];
        r[i] = (uint32_t)c;
        c >>= 32;
    }
    return (uint32_t)c;
}

/* r -= x (N limbs); returns the borrow out. */
static uint32_t nat_sub(uint32_t *r, const uint32_t *x, size_t N)
{
    uint64_t bw = 0;
    for (size_t i = 0; i < N; ++i) {
        const uint64_t t = (uint64_t)r[i] - x[i] - bw;
        r[i] = (uint32_t)t;
        bw = (t >> 32) ? 1 : 0;
    }
    return (uint32_t)bw;
}

/* -1, 0 or 1 as x <, =, > y (N limbs). */
static int nat_cmp(const uint32_t *x, const uint32_t *y, size_t N)
{
    for (size_t i = N; i-- > 0;)
        if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    return 0;
}

/* acc (N limbs) += x (nx limbs) * 2^s, s in bits; returns nonzero if the sum
 * does not fit N limbs. */
static int nat_add_shifted(uint32_t *acc, size_t N, const uint32_t *x, size_t nx, size_t s)
{
    const size_t q = s / 32;
    const unsigned r = (unsigned)(s % 32);
    uint64_t c = 0;
    uint32_t lower = 0;  /* the limb of x below the current one */
    for (size_t i = 0; i <= nx; ++i) {
        const uint32_t cur = i < nx ? x[i] : 0;
        const uint32_t piece = r ? (uint32_t)((cur << r) | (lower >> (32 - r))) : cur;
        lower = cur;
        const size_t pos = q + i;
        if (pos >= N) {
            if (piece) return 1;
            continue;
        }
        c += (uint64_t)acc[pos] + piece;
        acc[pos] = (uint32_t)c;
        c >>= 32;
    }
    for (size_t pos = q + nx + 1; c && pos < N; ++pos) {
        c += acc[pos];
        acc[pos] = (uint32_t)c;
        c >>= 32;
    }
    return c != 0;
}

/* r = x * m (N limbs, m < 2^63); returns nonzero if the product does not fit. */
static int nat_mul_word(uint32_t *r, const uint32_t *x, size_t N, uint64_t m)
{
    u128 c = 0;
    for (size_t i = 0; i < N; ++i) {
        c += (u128)x[i] * m;
        r[i] = (uint32_t)c;
        c >>= 32;
    }
    return c != 0;
}

/* r = x / d by long division from the top limb down (N limbs, 0 < d < 2^63);
 * returns the remainder. */
static uint64_t nat_div_word(uint32_t *r, const uint32_t *x, size_t N, uint64_t d)
{
    u128 rem = 0;
    for (size_t i = N; i-- > 0;) {
        const u128 cur = (rem << 32) | x[i];
        r[i] = (uint32_t)(cur / d);   /* cur < d 2^32: the quotient limb fits */
        rem = cur % d;
    }
    return (uint64_t)rem;
}

static int nat_is_zero(const uint32_t *x, size_t N)
{
    for (size_t i = 0; i < N; ++i)
        if (x[i]) return 0;
    return 1;
}

/* ---------------------------------------------------------------- one level */

static size_t ceil_div(size_t a, size_t b) { return (a + b - 1) / b; }

/* Extra limbs of an evaluation value over the block: |U(+-2^j)| < 2^(32b + n(n-1) + 1). */
static size_t growth_limbs(int B)
{
    const size_t n = (size_t)B - 1;
    return ceil_div(n * (n - 1) + 1, 32);
}

/* Node X_i of the even-odd method: X_0 = 0, X_i = 4^(i-1). */
static uint64_t node(int i) { return i == 0 ? 0 : (uint64_t)1 << (2 * (i - 1)); }

static int toom_rec(const uint32_t *u, const uint32_t *v, size_t L, const int *plan, int nlev,
                    uint32_t *w);

/* Block i of an L-limb operand split into b-limb blocks, zero-padded: copied into dst. */
static void block(const uint32_t *u, size_t L, size_t b, int i, uint32_t *dst)
{
    memset(dst, 0, b * 4);
    const size_t lo = (size_t)i * b;
    if (lo < L) memcpy(dst, u + lo, (L - lo < b ? L - lo : b) * 4);
}

/* Step 2: the 2B-1 values U(x) (magnitudes of e limbs, signs 0/1) of u. */
static int evaluate(const uint32_t *u, size_t L, int B, size_t b, size_t e, uint32_t *val,
                    unsigned char *sgn)
{
    const int n = B - 1;
    uint32_t *blk = calloc(b, 4), *E = calloc(e, 4), *O = calloc(e, 4);
    int st = T_OK;
    if (!blk || !E || !O) { st = T_NOMEM; goto done; }
    /* U(0) = u_0 */
    block(u, L, b, 0, blk);
    memset(val, 0, e * 4);
    memcpy(val, blk, b * 4);
    sgn[0] = 0;
    for (int j = 0; j < n; ++j) {
        memset(E, 0, e * 4);
        memset(O, 0, e * 4);
        for (int i = 0; i < B; ++i) {
            block(u, L, b, i, blk);
            if (nat_add_shifted(i % 2 == 0 ? E : O, e, blk, b, (size_t)j * (size_t)i)) {
                st = T_OVERFLOW;
                goto done;
            }
        }
        uint32_t *plus = val + (size_t)(2 * j + 1) * e, *minus = val + (size_t)(2 * j + 2) * e;
        memcpy(plus, E, e * 4);                     /* U(+x) = E + O */
        if (nat_add(plus, O, e)) { st = T_OVERFLOW; goto done; }
        sgn[2 * j + 1] = 0;
        if (nat_cmp(E, O, e) >= 0) {                /* U(-x) = E - O */
            memcpy(minus, E, e * 4);
            nat_sub(minus, O, e);
            sgn[2 * j + 2] = 0;
        } else {
            memcpy(minus, O, e * 4);
            nat_sub(minus, E, e);
            sgn[2 * j + 2] = 1;
        }
    }
done:
    free(blk); free(E); free(O);
    return st;
}

/* Steps 4-7 for one product: y holds the 2B-1 magnitudes (2e limbs each) and
 * ysgn their signs; writes w = u v into 2L limbs. */
static int interpolate(const uint32_t *y, const unsigned char *ysgn, int B, size_t L, size_t b,
                       size_t e, uint32_t *w)
{
    const int n = B - 1;
    const size_t V = 2 * e + 2;  /* every intermediate is below 2^(32 (2e + 1)) */
    uint32_t *ye = calloc((size_t)(n + 1) * V, 4), *yo = calloc((size_t)(n + 1) * V, 4);
    uint32_t *prev = calloc((size_t)(n + 1) * V, 4), *t1 = calloc(V, 4), *t2 = calloc(V, 4);
    int st = T_OK;
    if (!ye || !yo || !prev || !t1 || !t2) { st = T_NOMEM; goto done; }

    /* step 4: even-odd combine */
    memcpy(ye, y, 2 * e * 4);
    for (int k = 1; k <= n; ++k) {
        const uint32_t *wp = y + (size_t)(2 * k - 1) * 2 * e, *wm = y + (size_t)(2 * k) * 2 * e;
        const int neg = ysgn[2 * k];
        memset(t1, 0, V * 4);                       /* t1 = W(x) + W(-x) */
        memcpy(t1, wp, 2 * e * 4);
        memset(t2, 0, V * 4);                       /* t2 = W(x) - W(-x) */
        memcpy(t2, wp, 2 * e * 4);
        memset(prev, 0, V * 4);
        memcpy(prev, wm, 2 * e * 4);
        if (neg) {
            if (nat_sub(t1, prev, V)) { st = T_UNDERFLOW; goto done; }
            nat_add(t2, prev, V);
        } else {
            nat_add(t1, prev, V);
            if (nat_sub(t2, prev, V)) { st = T_UNDERFLOW; goto done; }
        }
        if (nat_div_word(ye + (size_t)k * V, t1, V, 2)) { st = T_INEXACT; goto done; }
        if (nat_div_word(t1, t2, V, 2)) { st = T_INEXACT; goto done; }
        if (nat_mul_word(yo + (size_t)k * V, t1, V, (uint64_t)1 << (k - 1))) {
            st = T_OVERFLOW;
            goto done;
        }
    }

    /* steps 5 and 6 on each polynomial */
    for (int p = 0; p < 2; ++p) {
        uint32_t *col = p == 0 ? ye : yo;
        /* Theorem 3.2 */
        for (int k = 1; k <= n; ++k) {
            memcpy(prev, col, (size_t)(n + 1) * V * 4);
            for (int pos = k; pos <= n; ++pos) {
                const int m = pos - k;
                memcpy(t1, prev + (size_t)pos * V, V * 4);
                if (nat_sub(t1, prev + (size_t)(pos - 1) * V, V)) { st = T_UNDERFLOW; goto done; }
                if (nat_div_word(col + (size_t)pos * V, t1, V, node(pos) - node(m))) {
                    st = T_INEXACT;
                    goto done;
                }
            }
        }
        /* Theorem 3.3 */
        for (int m = n - 1; m >= 0; --m) {
            memcpy(prev, col, (size_t)(n + 1) * V * 4);
            for (int k = m; k <= n - 1; ++k) {
                if (nat_mul_word(t1, prev + (size_t)(k + 1) * V, V, node(m))) {
                    st = T_OVERFLOW;
                    goto done;
                }
                if (nat_sub(col + (size_t)k * V, t1, V)) { st = T_UNDERFLOW; goto done; }
            }
        }
        for (int k = 0; k <= n; ++k)
            if (col[(size_t)k * V + V - 1]) { st = T_OVERFLOW; goto done; }
    }
    if (!nat_is_zero(yo, V)) { st = T_INEXACT; goto done; }  /* co_0 = 0 */

    /* step 7: w = sum_k w_k 2^(32 b k), w_(2i) = ce_i, w_(2i+1) = co_(i+1) */
    memset(w, 0, 2 * L * 4);
    for (int t = 0; t <= 2 * n; ++t) {
        const uint32_t *wt = t % 2 == 0 ? ye + (size_t)(t / 2) * V : yo + (size_t)(t / 2 + 1) * V;
        if (nat_add_shifted(w, 2 * L, wt, V, 32 * b * (size_t)t)) {
            st = T_OVERFLOW;
            goto done;
        }
    }
done:
    free(ye); free(yo); free(prev); free(t1); free(t2);
    return st;
}

/* Step 3 for points [p0, p1): y_p = |U_p| |V_p| by the rest of the plan. */
static int products(const uint32_t *uval, const uint32_t *vval, size_t e, const int *plan, int nlev,
                    int p0, int p1, uint32_t *y)
{
    for (int p = p0; p < p1; ++p) {
        const int st = toom_rec(uval + (size_t)p * e, vval + (size_t)p * e, e, plan, nlev,
                                y + (size_t)p * 2 * e);
        if (st) return st;
    }
    return T_OK;
}

struct job {
    const uint32_t *uval, *vval;
    size_t e;
    const int *plan;
    int nlev, p0, p1, step;
    uint32_t *y;
    int st;
};

static void *job_run(void *arg)
{
    struct job *j = arg;
    j->st = T_OK;
    for (int p = j->p0; p < j->p1 && !j->st; p += j->step)
        j->st = products(j->uval, j->vval, j->e, j->plan, j->nlev, p, p + 1, j->y);
    return NULL;
}

/* One level with B = plan[0], then the rest of the plan below; `threads` > 1
 * spreads this level's 2B-1 products over that many threads. */
static int toom_level(const uint32_t *u, const uint32_t *v, size_t L, const int *plan, int nlev,
                      uint32_t *w, int threads)
{
    const int B = plan[0];
    if (B < 2 || B > 32 || (size_t)B > L) return T_BADPLAN;
    const int npts = 2 * B - 1;
    const size_t b = ceil_div(L, (size_t)B), e = b + growth_limbs(B);
    uint32_t *uval = malloc((size_t)npts * e * 4), *vval = malloc((size_t)npts * e * 4);
    uint32_t *y = malloc((size_t)npts * 2 * e * 4);
    unsigned char *us = malloc(npts), *vs = malloc(npts), *ys = malloc(npts);
    int st = T_OK;
    if (!uval || !vval || !y || !us || !vs || !ys) { st = T_NOMEM; goto done; }
    if ((st = evaluate(u, L, B, b, e, uval, us))) goto done;
    if ((st = evaluate(v, L, B, b, e, vval, vs))) goto done;
    if (threads <= 1) {
        st = products(uval, vval, e, plan + 1, nlev - 1, 0, npts, y);
    } else {
        const int nt = threads < npts ? (threads < 64 ? threads : 64) : npts;
        pthread_t tid[64];
        struct job jobs[64];
        int ok[64];
        for (int t = 0; t < nt; ++t) {
            jobs[t] = (struct job){uval, vval, e, plan + 1, nlev - 1, t, npts, nt, y, T_OK};
            ok[t] = pthread_create(&tid[t], NULL, job_run, &jobs[t]) == 0;
            if (!ok[t]) job_run(&jobs[t]);   /* no thread: run this share here */
        }
        for (int t = 0; t < nt; ++t) {
            if (ok[t]) pthread_join(tid[t], NULL);
            if (jobs[t].st && !st) st = jobs[t].st;
        }
    }
    if (st) goto done;
    for (int p = 0; p < npts; ++p) {
        const int zero = nat_is_zero(y + (size_t)p * 2 * e, 2 * e);
        ys[p] = (unsigned char)(zero ? 0 : (us[p] ^ vs[p]));
    }
    st = interpolate(y, ys, B, L, b, e, w);
done:
    free(uval); free(vval); free(y); free(us); free(vs); free(ys);
    return st;
}

static int toom_rec(const uint32_t *u, const uint32_t *v, size_t L, const int *plan, int nlev,
                    uint32_t *w)
{
    if (nlev == 0) {
        oracle_schoolbook(u, L, v, L, w);
        return T_OK;
    }
    return toom_level(u, v, L, plan, nlev, w, 1);
}

/* ---------------------------------------------------------------- entry points */

/* out[0 .. 2L) = a[0 .. L) * b[0 .. L) by B-way Toom-Cook with B = plan[l] at
 * level l (nlev levels, 0 = plain schoolbook), the top level's products on up
 * to `threads` threads.  Returns 0, or the code of the first violated
 * invariant (1 underflow, 2 inexact division, 3 overflow, 4 no memory, 5 bad
 * plan). */
int oracle_toom_mul(const uint32_t *a, const uint32_t *b, size_t L, const int *plan, int nlev,
                    uint32_t *out, int threads)
{
    if (nlev < 0 || (nlev > 0 && !plan)) return T_BADPLAN;
    if (L == 0) return T_OK;
    if (nlev == 0) {
        oracle_schoolbook(a, L, b, L, out);
        return T_OK;
    }
    return toom_level(a, b, L, plan, nlev, out, threads);
}

struct batch_job {
    size_t first, count, step, L;
    const uint32_t *A, *B;
    const int *plan;
    int nlev;
    uint32_t *OUT;
    int st;
};

static void *batch_run(void *arg)
{
    struct batch_job *j = arg;
    j->st = T_OK;
    for (size_t k = j->first; k < j->count && !j->st; k += j->step)
        j->st = oracle_toom_mul(j->A + k * j->L, j->B + k * j->L, j->L, j->plan, j->nlev,
                                j->OUT + k * 2 * j->L, 1);
    return NULL;
}

/* `count` independent products of rows of L limbs (A, B packed; OUT rows of
 * 2L limbs), whole products spread over up to `threads` threads. */
int oracle_toom_mul_batch(size_t count, const uint32_t *A, const uint32_t *B, size_t L,
                          const int *plan, int nlev, uint32_t *OUT, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if ((size_t)threads > count) threads = (int)(count ? count : 1);
    pthread_t tid[256];
    struct batch_job jobs[256];
    int ok[256];
    int st = T_OK;
    for (int t = 0; t < threads; ++t) {
        jobs[t] = (struct batch_job){(size_t)t, count, (size_t)threads, L, A, B, plan, nlev, OUT,
                                     T_OK};
        ok[t] = pthread_create(&tid[t], NULL, batch_run, &jobs[t]) == 0;
        if (!ok[t]) batch_run(&jobs[t]);
    }
    for (int t = 0; t < threads; ++t) {
        if (ok[t]) pthread_join(tid[t], NULL);
        if (jobs[t].st && !st) st = jobs[t].st;
    }
    return st;
}
