/*
 * tc.h - exact B-way Toom-Cook multiplication of large unsigned integers on
 * an NVIDIA GB300 (sm_103a).  C ABI; every entry point is extern "C".
 *
 * The operation is the product w = u v of two unsigned integers (Section 1 of
 * Kronenburg, "Toom-Cook Multiplication: Some Theoretical and Practical
 * Aspects", arXiv:1602.02740: u = U(2^b), v = V(2^b), w = W(2^b)), computed by
 * B-way Toom-Cook: split into B blocks, evaluate at the 2B-1 points 0 and
 * +-2^j (Section 6), multiply pointwise (recursively), interpolate with the
 * even-odd method (Section 4) and Newton's divided differences with exact
 * divisions (Section 3, Theorems 3.2 and 3.3), and recompose.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - An integer is a little-endian array of uint32 limbs: limb i holds bits
 *   [32 i, 32 i + 32).  Lengths are in limbs.
 * - "Device pointer" means memory the CUDA device can read (cudaMalloc,
 *   managed, or a torch CUDA tensor's storage) on the context's device.
 *   "Host pointer" means ordinary or pinned host memory.
 * - Output buffers must not overlap input buffers.
 * - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *   stream.  Calls are asynchronous with respect to the host unless stated;
 *   results are valid once the stream has completed.  The multiply calls
 *   (tc_mul, tc_sqr, tc_mul_uniform, tc_mul_batch) never wait for the device,
 *   except when the context's scratch or pinned staging has to grow (the
 *   first call of a larger shape allocates); so they can be captured into a
 *   CUDA graph once the context has run the same shape outside the capture.
 * - Levels with few huge products run segment-parallel with bounded device
 *   waits.  A wait that gives up (never expected: it needs a stalled GPU) sets
 *   a sticky error word of the context instead of hanging; tc_check reports it.
 * - The caller owns every buffer it passes.  The context owns its scratch
 *   memory (allocated with cudaMalloc, never above the context's budget).
 * - Errors are returned as tc_status; nothing aborts, traps or throws.
 *   Argument errors are detected on the host before any launch.
 * - Calls that share one context must not run concurrently (they share its
 *   scratch); use one context per concurrent stream.  The serving calls are
 *   the exception: they are thread-safe.
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_ctx tc_ctx;

typedef enum {
    TC_OK = 0,
    TC_EINVAL = -1,     /* bad argument (null pointer, size, plan) */
    TC_ENOMEM = -2,     /* scratch would exceed the context budget, or cudaMalloc failed */
    TC_EBUSY = -3,      /* serving: not admitted now (budget or slots full) */
    TC_ETIMEOUT = -4,   /* a bounded wait gave up */
    TC_EDEVICE = -5,    /* a CUDA call failed; see tc_last_cuda_error */
    TC_EPENDING = 1     /* serving: request still running */
} tc_status;

#define TC_MAX_LEVELS 8

/*
 * Recursion plan.  levels = number of Toom levels above the base product
 * (0 = the base product alone); B[l] is the number of blocks at level l
 * (2 <= B[l] <= 32).  Block size at a level of operand length s is
 * b = ceil(s / B); each evaluation value has e = b + ceil((n(n-1)+1)/32)
 * limbs (n = B-1), which is the operand length of the next level.
 * base selects the product below the last level: TC_BASE_SCHOOLBOOK (the
 * plain schoolbook of Section 6; leaves of at most 1024 limbs when levels > 0)
 * or TC_BASE_NTT (an exact number-theoretic-transform product: Toom-Cook as
 * the parallel wrapper around a fast multiply, Section 5; leaves of at most
 * 2^24 limbs).  Passing NULL for a `const tc_opts*` lets the library choose
 * the plan (autotuned table if loaded, else a built-in rule).
 */
#define TC_BASE_SCHOOLBOOK 0
#define TC_BASE_NTT 1
typedef struct {
    int levels;
    int B[TC_MAX_LEVELS];
    int base;
} tc_opts;

/* Create a context on CUDA device `device` whose scratch never exceeds
 * `hbm_budget_bytes` (0 = 3/4 of the device's free memory).
 * `tune_table_path` (nullable) names a plan table written by the autotuner:
 * text lines "<max_limbs> <levels> <B0> <B1> ... [ntt]", ascending max_limbs
 * ("ntt" selects the transform base product).
 * On success *ctx is set and TC_OK returned. */
tc_status tc_create(tc_ctx **ctx, int device, size_t hbm_budget_bytes,
                    const char *tune_table_path);

/* Free the context and its scratch (synchronises the device first). */
void tc_destroy(tc_ctx *ctx);

/* Wait for `stream`, then report the context's sticky device error word (the
 * word is cleared by the report): TC_EINVAL if a device-side table entry of
 * tc_mul_batch_dev was out of range, else TC_ETIMEOUT if a segment-parallel
 * level of any multiply call on this context since the last check gave up a
 * wait -- those results are invalid -- else TC_OK.  Prepared batches and pipes
 * keep their own words (tc_batch_check, tc_pipe_wait). */
tc_status tc_check(tc_ctx *ctx, void *stream);

/* The plan the library would use for balanced operands of `limbs` limbs. */
tc_status tc_plan_for(tc_ctx *ctx, size_t limbs, tc_opts *plan_out);

/* Scratch bytes a balanced batch of `count` products of `limbs` limbs needs
 * under `opts` (NULL = the library's plan). */
tc_status tc_scratch_bytes(tc_ctx *ctx, size_t count, size_t limbs, const tc_opts *opts,
                           size_t *bytes_out);

/*
 * The product w = u v of Section 1 (u = U(2^b), v = V(2^b), w = W(2^b)) by
 * B-way Toom-Cook with the context's plan: evaluation at the 2B-1 points of
 * Section 6 by the even-odd parts (Section 4, eq. 4.1-4.2), pointwise products
 * recursively (Section 2), interpolation by the even-odd combine (eq. 4.5-4.6)
 * and Newton's divided differences (Theorems 3.2 and 3.3), recomposition.
 * out[0 .. na+nb) = a[0 .. na) * b[0 .. nb)   (device pointers).
 * Exactly na+nb limbs are written (leading zeros kept).  na == 0 or nb == 0
 * zero-fills out.  a == b with na == nb selects the squaring path.
 * Unbalanced operands: the shorter operand is zero-padded when the ratio is
 * below 2; otherwise the longer one is cut into pieces of the shorter's
 * length, the pieces are multiplied as one balanced batch, and the partial
 * products are added at their offsets.  na and nb at most 2^30 limbs, else
 * TC_EINVAL.
 */
tc_status tc_mul(tc_ctx *ctx, const uint32_t *a, size_t na, const uint32_t *b, size_t nb,
                 uint32_t *out, const tc_opts *opts, void *stream);

/* out[0 .. 2 na) = a^2 (device pointers): tc_mul with U = V, one evaluation
 * per level and squares in the base case (all pointwise products are >= 0). */
tc_status tc_sqr(tc_ctx *ctx, const uint32_t *a, size_t na, uint32_t *out,
                 const tc_opts *opts, void *stream);

/*
 * `count` independent products in one call: the paper runs the 2B-1 top-level
 * products of one multiplication in parallel (Section 2, eq. 2.5); here every
 * product of a list is batched level by level.  A, Bv and OUT are device limb
 * buffers; a_off/a_len, b_off/b_len and out_off are HOST int64 arrays of
 * limb offsets and lengths.  Product k reads A[a_off[k] .. +a_len[k]) and
 * Bv[b_off[k] .. +b_len[k]) and writes OUT[out_off[k] .. +a_len[k]+b_len[k]).
 * Products are grouped into size classes; each class runs level by level
 * (breadth first) with every product of the class in the same launches, and
 * the classes run concurrently on streams of the context (each in its own
 * region of the context's scratch; the call's stream waits for all of them).
 * TC_EINVAL (before any launch) if an offset is negative or above 2^40, or a
 * length is negative or above 2^28 limbs.
 */
tc_status tc_mul_batch(tc_ctx *ctx, size_t count,
                       const uint32_t *A, const int64_t *a_off, const int64_t *a_len,
                       const uint32_t *Bv, const int64_t *b_off, const int64_t *b_len,
                       uint32_t *OUT, const int64_t *out_off,
                       const tc_opts *opts, void *stream);

/*
 * The same products with DEVICE int64 tables a_off/a_len, b_off/b_len and
 * out_off (built on the device, read only by kernels: the call never waits for
 * the device and can be captured into a CUDA graph once the context has run the
 * same count and max_limbs).  Without the lengths on the host the products
 * cannot be grouped into size classes: every product is padded to the one
 * balanced class that holds `max_limbs` (0 < max_limbs <= 2^28), so uneven
 * batches do more work than with tc_mul_batch or a prepared batch.  A product
 * whose offset is negative or whose length is negative or above max_limbs is
 * skipped on the device (its output is not written) and tc_check then reports
 * TC_EINVAL.
 */
tc_status tc_mul_batch_dev(tc_ctx *ctx, size_t count,
                           const uint32_t *A, const int64_t *a_off, const int64_t *a_len,
                           const uint32_t *Bv, const int64_t *b_off, const int64_t *b_len,
                           uint32_t *OUT, const int64_t *out_off, size_t max_limbs,
                           const tc_opts *opts, void *stream);

/*
 * Prepared batches (the scheduler's work lists; CUDA-graph replay).  The
 * paper runs the top-level products of one multiplication in parallel
 * threads (Section 2, eq. 2.5); here any list of products is batched level by
 * level.  tc_batch_prepare does the host side of tc_mul_batch once for a
 * fixed list: it groups the products into size classes (padded balanced
 * lengths), picks each class's plan (`opts` as in tc_mul_batch), uploads the
 * index tables and allocates one scratch region per class -- device memory
 * owned by the batch, at most the context's budget (else TC_ENOMEM) -- and the
 * streams its classes run on concurrently (a captured run becomes parallel
 * branches of the graph).  Offsets
 * and lengths are host int64 arrays read during the call only.
 * tc_batch_run then enqueues kernels and memsets on `stream` and nothing else
 * (no allocation, no host memory, no synchronisation), so it may be captured
 * into a CUDA graph and replayed; A, Bv and OUT are device buffers addressed by
 * the prepared offsets (products of length 0 get zero-filled outputs).  Runs of
 * one batch must not overlap in time: they share its scratch.
 * tc_batch_check waits for `stream` and returns TC_ETIMEOUT if a bounded wait
 * of a segment-parallel level gave up in any run since the last check (and
 * clears that state), else TC_OK.
 * tc_batch_destroy frees the batch (NULL is ignored).
 */
typedef struct tc_batch tc_batch;
tc_status tc_batch_prepare(tc_ctx *ctx, size_t count, const int64_t *a_off, const int64_t *a_len,
                           const int64_t *b_off, const int64_t *b_len, const int64_t *out_off,
                           const tc_opts *opts, tc_batch **out);
tc_status tc_batch_run(tc_ctx *ctx, const tc_batch *batch, const uint32_t *A, const uint32_t *Bv,
                       uint32_t *OUT, void *stream);
tc_status tc_batch_check(tc_ctx *ctx, const tc_batch *batch, void *stream);
size_t tc_batch_scratch_bytes(const tc_batch *batch);
void tc_batch_destroy(tc_batch *batch);

/*
 * Uniform batch: `count` balanced products of `limbs` x `limbs` limbs stored
 * as rows.  A row k is A[k * lda .. k * lda + limbs), likewise B; the result
 * row is OUT[k * ldo .. k * ldo + 2 limbs).  Device pointers.
 */
tc_status tc_mul_uniform(tc_ctx *ctx, size_t count, size_t limbs,
                         const uint32_t *A, size_t lda, const uint32_t *Bv, size_t ldb,
                         uint32_t *OUT, size_t ldo, const tc_opts *opts, void *stream);

/*
 * Same as tc_mul_uniform but A, Bv and OUT are HOST pointers (pinned memory
 * gives full copy speed).  Copies in, multiplies, copies out and waits for
 * the stream before returning.
 */
tc_status tc_mul_uniform_host(tc_ctx *ctx, size_t count, size_t limbs,
                              const uint32_t *A, const uint32_t *Bv, uint32_t *OUT,
                              const tc_opts *opts, void *stream);

/*
 * Pipelined host-buffer batches (the same products as tc_mul_uniform_host,
 * Section 1 with the context's plan: `count` rows of `limbs` x `limbs` limbs,
 * packed, results 2*limbs limbs a row; the pipelining is scheduling only).
 * The pipe owns device memory for two batches in flight plus its own level
 * scratch (so its batches do not contend with other calls on the context for
 * the context's scratch), and three streams: copy-in, kernels, copy-out.  tc_pipe_submit
 * enqueues one batch and returns without waiting: batch i+1's copy-in and
 * batch i-1's copy-out overlap batch i's kernels.  A, Bv and OUT are HOST
 * pointers (pinned memory for asynchronous, full-speed copies) that must stay
 * valid and unmodified (OUT unread) until tc_pipe_wait returns.  `square`
 * fixes at creation whether batches are squares (Bv ignored, A == Bv
 * semantics) or products.  tc_pipe_wait blocks until every submitted batch is
 * complete; it returns TC_ETIMEOUT if a bounded wait of a segment-parallel
 * level gave up in any batch since the last wait.  Errors: TC_EINVAL (null or
 * zero arguments, a context of another device), TC_ENOMEM (the pipe's memory
 * exceeds the context's budget), TC_EDEVICE; after an error from
 * tc_pipe_submit or tc_pipe_wait the pipe's state is undefined: destroy it.
 * tc_pipe_destroy waits for the pipe and
 * frees it (NULL ignored).
 */
typedef struct tc_pipe tc_pipe;
tc_status tc_pipe_create(tc_ctx *ctx, size_t count, size_t limbs, int square,
                         const tc_opts *opts, tc_pipe **out);
tc_status tc_pipe_submit(tc_ctx *ctx, tc_pipe *pipe, const uint32_t *A, const uint32_t *Bv,
                         uint32_t *OUT);
tc_status tc_pipe_wait(tc_pipe *pipe);
void tc_pipe_destroy(tc_pipe *pipe);

/* ---------------------------------------------------------------------
 * The steps of one Toom level, exported for testing and for callers that
 * schedule levels themselves.  All pointers are device pointers.
 * ------------------------------------------------------------------- */

/*
 * Plain schoolbook products (the base case): `count` rows of `limbs` x
 * `limbs` limbs, row k of A at A + k*lda, of B at Bv + k*ldb; 2*limbs limbs
 * written at OUT + k*ldo.  limbs <= 1024.
 */
tc_status tc_schoolbook(size_t count, size_t limbs, const uint32_t *A, size_t lda,
                        const uint32_t *Bv, size_t ldb, uint32_t *OUT, size_t ldo,
                        void *stream);

/*
 * Base product by number-theoretic transform (the fast multiply that Section 5
 * wraps in Toom-Cook; the paper's is GMP's FFT, this one is exact by
 * construction): `count` rows of `limbs` x `limbs` limbs as in tc_schoolbook
 * (limbs <= 2^24), 2*limbs limbs written at OUT + k*ldo.  Each operand is
 * read as 16-bit digits; the digit vectors are convolved by a transform of
 * N = 2^n >= 4*limbs points modulo the prime p = 2^64 - 2^32 + 1 (every
 * convolution coefficient is below N 2^32 < p, so the result is exact), and
 * the coefficients are carried into limbs.  A == Bv with lda == ldb squares
 * (one forward transform).  `work` is device scratch of
 * tc_ntt_work_bytes(count, limbs) bytes, 16-byte aligned; otherwise
 * TC_EINVAL.  The first call for a transform length uploads that length's
 * root tables (a small device allocation kept until exit).
 */
tc_status tc_ntt_mul(size_t count, size_t limbs, const uint32_t *A, size_t lda,
                     const uint32_t *Bv, size_t ldb, uint32_t *OUT, size_t ldo, void *work,
                     void *stream);
size_t tc_ntt_work_bytes(size_t count, size_t limbs);

/* Host only: the primitive 2^log2n-th root of unity modulo p = 2^64 - 2^32 + 1
 * the transform uses (7^((p-1)/2^log2n), 7 generating the multiplicative
 * group); TC_EINVAL unless 0 <= log2n <= 32. */
tc_status tc_ntt_root(int log2n, uint64_t *root);

/*
 * Evaluation (Section 4, eq. 4.1-4.2; points of Section 6).  Each of `count`
 * operand rows of `limbs` limbs (row k at U + k*ld) is split into B blocks
 * of b = ceil(limbs/B) limbs and evaluated at the 2B-1 points in the order
 * 0, +1, -1, +2, -2, ..., +2^(B-2), -2^(B-2).  Value p of row k is written
 * as a magnitude of `estride` limbs at OUT + (k*(2B-1) + p) * estride, and
 * its sign (1 = negative) at SGN[k*(2B-1) + p].  estride must be >= e (the
 * evaluation length) and a multiple of 4, and OUT 16-byte aligned (the
 * kernels store 4 limbs at a time); otherwise TC_EINVAL.
 */
tc_status tc_toom_evaluate(size_t count, size_t limbs, int B, const uint32_t *U, size_t ld,
                           uint32_t *OUT, size_t estride, uint8_t *SGN, void *stream);

/*
 * Interpolation and recomposition of one level (Section 4 even-odd
 * combine, Theorem 3.2 divided differences with exact division, Theorem 3.3
 * Newton-to-monomial, recomposition W(2^(32 b))).  For each of `count`
 * products of operands of `limbs` limbs: the 2B-1 pointwise products are
 * magnitudes of 2e limbs at Y + (k*(2B-1) + p) * ystride with signs
 * SGN_U[k*(2B-1)+p] xor SGN_V[k*(2B-1)+p] (either may be NULL = all
 * positive); 2*limbs result limbs are written at OUT + k*ldo.  `work` is
 * device scratch of tc_toom_interpolate_work_bytes(count, limbs, B) bytes (may
 * be NULL when that is 0).  ystride >= 2e, multiple of 4; Y and work
 * 16-byte aligned (4-limb loads and stores); otherwise TC_EINVAL.
 */
tc_status tc_toom_interpolate(size_t count, size_t limbs, int B,
                              const uint32_t *Y, size_t ystride,
                              const uint8_t *SGN_U, const uint8_t *SGN_V,
                              uint32_t *OUT, size_t ldo, void *work, void *stream);

/*
 * The same interpolation and recomposition by the inverse Vandermonde matrix
 * (the alternative that closes Section 3): each coefficient is computed in
 * one pass as w_i = (sum_p M_ip W(x_p)) / (2^s_i d_i) from the integer form
 * of row i of V^-1 (see tc_interp_matrix_table), with no even-odd combine and
 * no Newton stages.  Same arguments, layout and result as tc_toom_interpolate
 * minus `work` (no scratch).  Supported: B <= 6 and 2e + 2 <= 1024 (values of
 * at most 1024 limbs, e the evaluation length); otherwise TC_EINVAL.
 */
tc_status tc_toom_interpolate_matrix(size_t count, size_t limbs, int B,
                                     const uint32_t *Y, size_t ystride,
                                     const uint8_t *SGN_U, const uint8_t *SGN_V,
                                     uint32_t *OUT, size_t ldo, void *stream);

/*
 * Host only (no GPU needed): the integer form of V^-1 for B blocks (2 <= B <= 6)
 * on the points 0, +1, -1, +2, -2, ..., +-2^(B-2): for coefficient i and
 * point p, M[i*(2B-1) + p] = M_ip, and V^-1[i][p] = M_ip / (2^shift[i] odd[i])
 * with odd[i] odd, shift[i] and odd[i] the smallest that make row i integral.
 * M holds (2B-1)^2 entries, shift and odd 2B-1; TC_EINVAL on bad arguments.
 */
tc_status tc_interp_matrix_table(int B, int64_t *M, int *shift, uint32_t *odd);

/* Scratch bytes tc_toom_interpolate needs for `count` products of `limbs`
 * limbs split into B blocks (0 when it runs in shared memory). */
size_t tc_toom_interpolate_work_bytes(size_t count, size_t limbs, int B);

/*
 * Interpolation without any device allocation (the paper has no counterpart:
 * this is an integration convenience).  For callers that must not allocate
 * device memory while they run -- e.g. a service that reserved all GPU memory
 * for its own pool at start-up, or a latency-critical loop where
 * cudaMalloc/cudaFree (which may synchronise the device) is not acceptable.
 *
 * Computes exactly what tc_toom_interpolate computes, with the same arguments
 * minus `work`: the scratch comes from one fixed device array of
 * TC_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads the
 * library holds until the process exits.  Calls needing more scratch than
 * that (tc_toom_interpolate_work_bytes(count, limbs, B) > TC_NOALLOC_SCRATCH_BYTES)
 * are rejected with TC_ENOMEM before any launch; nothing is allocated, by
 * this library or any other, on any path.  The first call that needs scratch
 * on a device looks up the array's device address for that device (make that
 * first call before any stream capture); later calls reuse it.
 * Every call on a device shares the one array and it keeps the last call's
 * contents (nothing in it needs to start at zero: each call writes all the
 * scratch it reads).  Calls whose GPU work overlaps in time race on the
 * array: serialise them, e.g. on one stream.
 */
#define TC_NOALLOC_SCRATCH_BYTES (16u << 20)
tc_status tc_toom_interpolate_noalloc(size_t count, size_t limbs, int B,
                                      const uint32_t *Y, size_t ystride,
                                      const uint8_t *SGN_U, const uint8_t *SGN_V,
                                      uint32_t *OUT, size_t ldo, void *stream);

/* ---------------------------------------------------------------------
 * Serving: a request loop on a host thread that admits products while the
 * scratch budget and a slot allow, groups them by size class, and keeps the
 * GPU busy with several groups in flight.  Thread-safe.
 * ------------------------------------------------------------------- */

/* Submit u*v (device pointers; they must stay valid until tc_serve_poll
 * reports completion).  TC_EBUSY = not admitted now (retry later). */
tc_status tc_serve_submit(tc_ctx *ctx, const uint32_t *a, size_t na, const uint32_t *b,
                          size_t nb, uint32_t *out, uint64_t *ticket);

/* TC_OK when the ticket's product is complete in `out`, TC_EPENDING while it
 * runs, or the request's error status.  The call that reports a final state
 * (TC_OK or an error) releases the ticket: polling it again returns TC_EINVAL.
 * tc_serve_stop may run concurrently with tc_serve_submit, tc_serve_poll and
 * tc_serve_stats (after a stop they see no server: TC_EINVAL for poll). */
tc_status tc_serve_poll(tc_ctx *ctx, uint64_t ticket);

/* Latency percentiles (submit -> completion seen by the loop) and sustained
 * product-bits per second over the completed requests so far.  Product bits
 * of a request = 32 (na + nb). */
tc_status tc_serve_stats(tc_ctx *ctx, double *p50_ms, double *p99_ms, double *bits_per_s,
                         uint64_t *completed);

/* Stop the serving loop: pending requests complete first, then the loop's
 * tickets and statistics are discarded (the next submit starts a new loop). */
tc_status tc_serve_stop(tc_ctx *ctx);

/* ---------------------------------------------------------------------
 * Phase timing.  When enabled, every evaluate / base-case / interpolate
 * launch of tc_mul* calls on this context is bracketed by CUDA events
 * recorded on the launching stream, and its algorithmic work is recorded:
 * bytes = limbs the step must read plus limbs it must write (x4), and
 * limb_products = the s*s limb products of each schoolbook product.
 * ------------------------------------------------------------------- */
typedef struct {
    int kind;              /* 0 evaluate, 1 base-case product, 2 interpolate+recompose */
    int level;             /* Toom level (base case: number of levels) */
    int launches;
    double ms;             /* summed event time */
    double bytes;          /* summed algorithmic bytes */
    double limb_products;  /* summed limb products (base case only) */
    char kernel[48];       /* name of the kernel (or kernel sequence) the step launched */
} tc_phase_stat;

/* Turn phase timing on (1) or off (0); turning it on clears the records. */
tc_status tc_profile_enable(tc_ctx *ctx, int on);

/* Wait for the recorded events and report up to `cap` phases in *out
 * (one entry per kind and level); *n receives the number written. */
tc_status tc_profile_read(tc_ctx *ctx, tc_phase_stat *out, int cap, int *n);

/*
 * Integer ceiling of the base case (a measurement kernel; the paper has no
 * counterpart).  Enqueues on `stream` `blocks` CTAs of 256 threads, each
 * thread running `iters` iterations of 64 register-only limb products, each
 * added into a 96-bit column sum by the base case's own instruction sequence
 * (mad.lo.cc, madc.hi.cc, addc).  *limb_products receives the number of limb
 * products the launch performs; time the launch with events on `stream` to
 * get limb products per second.  `sink` is a device buffer of blocks * 256
 * uint32 (one checksum per thread, so the work cannot be elided).  TC_EINVAL
 * for non-positive sizes or null pointers.
 */
tc_status tc_peak_madc(int blocks, int iters, uint32_t *sink, void *stream, double *limb_products);

/*
 * Failure-detection test hook (the paper has no counterpart).  On the current
 * device, from the next launch on: every bounded wait of the segment-parallel
 * passes gives up after `polls` polls of at least 64 ns (0 restores the default
 * of 2^22 polls, about a quarter second), and if `withhold` is nonzero the first
 * segment of every segment-parallel add/subtract chain does not publish its
 * carry, so the waits behind it run out and the calls report TC_ETIMEOUT
 * (tc_check, tc_batch_check, tc_pipe_wait, a serving poll) instead of
 * hanging.  Results computed while `withhold` is set are wrong by design.  Not
 * for concurrent use with other work on the device.  TC_EINVAL if polls < 0.
 */
tc_status tc_test_bounded_waits(int polls, int withhold);

/*
 * Base-case variant (tuning and test hook; the paper has none).  The
 * lane-pair base case (4096 or more products of up to 792 limbs) runs one
 * Karatsuba level inside the kernel (Section 1's B = 2 split taken below the
 * Toom threshold: three products of half-length rows instead of one) for rows
 * of at least `min_limbs` limbs; 0 turns it off.  Both variants give the same
 * limbs.  The default, TC_LEAF_KARATSUBA_DEFAULT, is where it measured faster
 * on GB300.  Process-wide, from the next launch on; not for concurrent use
 * with other work.  TC_EINVAL if min_limbs < 0 or 0 < min_limbs < 49 (the split
 * needs seven 8-limb tiles).
 */
#define TC_LEAF_KARATSUBA_DEFAULT 384
tc_status tc_set_leaf_karatsuba(int min_limbs);

/* Message for a status code (static string). */
const char *tc_strerror(tc_status s);

/* cudaError_t of the last TC_EDEVICE on this thread (0 if none). */
int tc_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TC_H */
