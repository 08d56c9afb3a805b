/*
 * mont.h -- C ABI of the GB300 (sm_103a) Montgomery multiplication library.
 *
 * Montgomery multiplication of 32-bit residues after L. Meng, "Automatic
 * Generation of Vectorized Montgomery Algorithm", Sec. 3.1 (Alg. 2, REDC) and
 * Sec. 3.2 (its data-parallel form), with R = 2^32 and P' = -P^-1 mod R.
 *
 * Conventions shared by every entry point:
 *  - Data pointers are DEVICE pointers (or memory the device can address,
 *    e.g. pinned host memory) owned by the caller; the library never frees
 *    them.  Elements are uint32 residues, contiguous, in [0, P).  Inputs
 *    outside [0, P) give unspecified (but in-bounds, non-faulting) results.
 *  - Calls are asynchronous on `stream` (0 = the legacy default stream) of
 *    the current device; they return once the work is queued.
 *  - Return value: MONT_OK (0) or a negative MONT_E* code.  Argument errors
 *    are detected on the host before anything is queued; a launch failure
 *    returns MONT_ECUDA.  No C++ exception crosses this boundary.
 *  - n == 0 is a no-op returning MONT_OK.
 *  - Elementwise calls allow out to equal an input (in place); any other
 *    overlap of an output with an input is rejected with MONT_EINVAL.
 */
#ifndef GB300_MONT_H
#define GB300_MONT_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MONT_OK = 0,
    MONT_EINVAL = -1,      /* bad argument (modulus, pointer, size, overlap, flags)   */
    MONT_ENOMEM = -2,      /* device or host allocation failed                         */
    MONT_ERANGE = -3,      /* size (or, for mont_check_residues, a value) out of range */
    MONT_ETIMEOUT = -4,    /* a bounded device-side wait gave up                       */
    MONT_ECUDA = -5,       /* a CUDA runtime call or kernel launch failed              */
    MONT_EUNSUPPORTED = -6 /* valid request this build does not implement              */
};

/*
 * Montgomery context (Sec. 3.1: "P' with R R^-1 - P P' = 1", residues
 * i-bar = iR mod P).  Plain caller-owned POD; filled by mont_setup and
 * validated by every call that takes it.
 *   p        odd modulus, 3 <= p < 2^31 (so 2P < R and the REDC sum fits 32 bits)
 *   p_prime  P' = -P^-1 mod 2^32
 *   r_mod_p  R mod P  (the Montgomery form of 1)
 *   r2_mod_p R^2 mod P (to_mont multiplies by it through REDC)
 */
typedef struct mont_ctx {
    uint32_t p;
    uint32_t p_prime;
    uint32_t r_mod_p;
    uint32_t r2_mod_p;
} mont_ctx;

/* Host only, no device work.  MONT_EINVAL if p is even, p < 3, p >= 2^31 or out is NULL. */
int mont_setup(uint32_t p, mont_ctx *out);

/*
 * out[i] = in[i] R mod P  (Sec. 3.1 residue map), computed as REDC(in[i] * (R^2 mod P)).
 */
int to_mont(const mont_ctx *ctx, const uint32_t *in, uint32_t *out, size_t n, cudaStream_t stream);

/* out[i] = in[i] R^-1 mod P, computed as REDC(in[i] * 1). */
int from_mont(const mont_ctx *ctx, const uint32_t *in, uint32_t *out, size_t n, cudaStream_t stream);

/*
 * out[i] = REDC(a[i], b[i]) = a[i] b[i] R^-1 mod P, fully reduced to [0, P)
 * (Alg. 2: T = ab; m = (T mod R) P' mod R; t = (T + mP)/R; one conditional
 * subtract).  With Montgomery-form operands a = xR, b = yR the result is xyR.
 */
int mont_mul(const mont_ctx *ctx, const uint32_t *a, const uint32_t *b, uint32_t *out, size_t n,
             cudaStream_t stream);

/*
 * out[i] = (REDC(a[i], b[i]) + c[i]) mod P: a Montgomery multiply followed by
 * a modular add, which Sec. 3.1 notes is unchanged by the representation.
 * With a = xR, b = yR, c = zR the result is (xy + z)R mod P.
 */
int mont_fma(const mont_ctx *ctx, const uint32_t *a, const uint32_t *b, const uint32_t *c,
             uint32_t *out, size_t n, cudaStream_t stream);

/*
 * out[i] = a[i] b[i] mod p on plain residues by Barrett reduction (Alg. 1):
 * k = ceil(log2 p), P' = floor(2^(2k) / p), m = floor(ab / 2^k),
 * q = floor(m P' / 2^k), t = ab - qP, subtract P while t >= P (at most 3
 * times).  p odd, 3 <= p < 2^31, else MONT_EINVAL.
 */
int barrett_mulmod(uint32_t p, const uint32_t *a, const uint32_t *b, uint32_t *out, size_t n,
                   cudaStream_t stream);

/*
 * out[i] = a[i] b[i] R^-1 mod P (the value REDC returns) by Montgomery
 * reduction over a Fourier prime P = c 2^n + 1 (Alg. 3): multiplies by c 2^n
 * replace the multiply by P', and sign masks replace the compare.  Needs
 * 2n >= 32 and, for the 31-bit sign tests to hold, P < 2^30 (so not
 * 2013265921); otherwise MONT_ERANGE.
 */
int fourier_redc_mul(const mont_ctx *ctx, const uint32_t *a, const uint32_t *b, uint32_t *out, size_t n,
                     cudaStream_t stream);

/*
 * Checks the precondition every entry point states for its inputs: REDC
 * (Alg. 2) and the transforms take residues of Z_P (Sec. 3.1), so each word
 * must lie in [0, p).  Returns MONT_OK if x[i] < p for every i < n (and for
 * n == 0), MONT_ERANGE if some word is >= p, MONT_EINVAL for p even, p < 3,
 * p >= 2^31, or x NULL with n > 0.  One read of x (4 B per element).
 * Unlike every other call it is SYNCHRONOUS: it runs on `stream` after the
 * work queued there, reads its result back and returns once the stream has
 * drained.  A debugging aid for callers whose data did not come from this
 * library; the product calls never run it.
 */
int mont_check_residues(uint32_t p, const uint32_t *x, size_t n, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Number-theoretic transform and polynomial multiplication.
 *
 * The modular FFT over Z_P that the paper's generated libraries compute
 * (Sec. 1 and 5; the paper does not restate it): X_k = sum_j x_j w^(jk) mod P
 * for N = 2^log2n, w = g^((P-1)/N), g the smallest primitive root of P.
 * The butterflies multiply by Montgomery-form twiddles with REDC (Alg. 2);
 * data stay in plain (non-Montgomery) form in [0, P).
 * ------------------------------------------------------------------------ */

/* Opaque plan: prime, size and the library-owned, device-resident twiddle
 * tables of the device current at creation.  Create and destroy on the host;
 * use only with that device current. */
typedef struct ntt_plan ntt_plan;

/* Flag for ntt_fwd: leave the output in bit-reversed order.
 * Flag for ntt_inv: the input is in bit-reversed order. */
#define NTT_BITREV 1

/* p prime, 3 <= p < 2^31, 2^log2n divides p - 1, log2n <= 24.  Builds (or
 * reuses) the twiddle tables with cudaMalloc/cudaMemcpy (synchronous; do not
 * call during stream capture).  MONT_EINVAL for a bad prime or NULL out,
 * MONT_ERANGE for an unsupported size, MONT_ENOMEM / MONT_ECUDA on failure. */
int ntt_plan_create(uint32_t p, uint32_t log2n, ntt_plan **out);

/* Frees the plan object (NULL is a no-op).  Its twiddle tables (the
 * Montgomery-form roots w^i R mod P of Sec. 3.1's residue map) stay cached
 * in device memory for later plans and products of the same (device, p) and
 * are released with the process; work already queued with the plan may
 * still run. */
void ntt_plan_destroy(ntt_plan *plan);

/* In-place forward transform of `batch` contiguous rows of N residues
 * ([batch][N] row-major).  Natural order in; natural order out unless
 * flags has NTT_BITREV.  N <= 2^14 runs in one kernel per batch; larger N
 * runs column and row kernels in place (plus a bit-reversal pass for
 * natural order), needing no scratch. */
int ntt_fwd(const ntt_plan *plan, uint32_t *data, size_t batch, int flags, cudaStream_t stream);

/* In-place inverse transform including the factor N^-1: ntt_inv(ntt_fwd(x)) = x.
 * Natural-order input unless flags has NTT_BITREV; natural-order output. */
int ntt_inv(const ntt_plan *plan, uint32_t *data, size_t batch, int flags, cudaStream_t stream);

/* c = a * b mod p (polynomials, coefficient 0 first), c has la + lb - 1
 * coefficients; a, b in [0, p).  Computed as forward NTTs of both operands
 * zero-padded to N = 2^ceil(log2(la + lb - 1)), a pointwise REDC product and
 * an inverse NTT, fused per product.  la, lb >= 1 (else MONT_EINVAL); c may
 * not overlap a or b.  The twiddle tables are built on first use for
 * (device, p, N): make the first call outside stream capture. */
int polymul(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c,
            cudaStream_t stream);

/* `count` independent products of the same shape: a is [count][la], b is
 * [count][lb], c is [count][la + lb - 1], all row-major and contiguous.
 * N <= 2^14 runs one fused kernel per batch.  Larger N (up to 2^24) runs
 * column / row / column kernels through a scratch buffer of 2N words per
 * product; polymul and polymul_many take it from a library-owned buffer per
 * (device, stream), at most 1 GiB (larger batches run in chunks), allocated
 * or grown with cudaMalloc on first need: size it outside stream capture.
 * Concurrent calls on different streams use different buffers; calls that
 * share a stream must come from one host thread at a time (a call that
 * grows the buffer frees the one another call is about to use). */
int polymul_many(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c,
                 size_t count, cudaStream_t stream);

/* polymul_many with Alg. 3 (FourierREDC, Sec. 3.1) in place of Alg. 2 for
 * every twiddle, scaling and pointwise multiply of the same fused kernels.
 * Same layout and results (bit for bit) as polymul_many; for comparing the
 * two reductions.  p must be a Fourier prime c 2^n + 1 with 2n >= 32 and
 * p < 2^30 (Alg. 3's 31-bit sign tests), else MONT_ERANGE; N <= 2^14 only,
 * else MONT_EUNSUPPORTED; other errors as polymul_many. */
int polymul_many_fourier(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c,
                         size_t count, cudaStream_t stream);

/* Scratch bytes polymul_many_ws needs for `count` products of this shape
 * (0 when N <= 2^14). */
size_t polymul_workspace_bytes(size_t la, size_t lb, size_t count);

/* polymul_many with caller-owned scratch: workspace is a 16-byte aligned
 * device buffer of ws_bytes.  With less than polymul_workspace_bytes(la, lb,
 * count) the products run in chunks that fit; less than one product's share
 * (or a misaligned pointer) is MONT_EINVAL.  The buffer must not be used by
 * other work until the queued kernels finish. */
int polymul_many_ws(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c,
                    size_t count, void *workspace, size_t ws_bytes, cudaStream_t stream);

/*
 * polymul without any allocation.  (No counterpart in the paper: this is a
 * service to callers of this library that cannot call cudaMalloc -- code being
 * recorded into a CUDA graph, code inside a framework whose allocator owns the
 * device memory, or latency-critical paths that cannot take cudaMalloc's
 * implicit device synchronisation.)
 *
 * Same result as polymul(plan's prime, a, la, b, lb, c, stream).  The
 * twiddle tables come from `plan` (created beforehand with ntt_plan_create,
 * on the current device, for a size 2^k >= la + lb - 1 of the same prime:
 * larger plans serve smaller products).  Products with N > 2^14 use a fixed
 * 2 MiB scratch array in the library's device memory instead of allocating:
 * la + lb - 1 must be <= 2^18 (else MONT_ERANGE; also MONT_ERANGE if the
 * plan's tables are too short).  Calls no cudaMalloc/cudaFree.  The first
 * call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process: make that
 * first call before any stream capture, and do not call this entry point
 * again on a device after cudaDeviceReset (or anything else that destroys
 * the device's primary context) in the same process, since the array may
 * then sit at another address.  Every call on a device shares the one array,
 * so calls whose kernels overlap on the GPU (e.g. on different streams) race
 * and must be ordered by the caller; no state carries over from one call to
 * the next.
 */
int polymul_noalloc(const ntt_plan *plan, const uint32_t *a, size_t la, const uint32_t *b, size_t lb,
                    uint32_t *c, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Uneven batches: many products of different lengths and primes in one
 * persistent kernel launch, or in the phased form's few kernels (optionally
 * replayed from a CUDA graph).  The data-parallel REDC of Sec. 3.2 taken from
 * vector lanes to whole products: every product is the fused NTT product
 * above (Sec. 1 and 5: the modular FFT libraries), and the autotuner plays the
 * part of the generator's search over implementations (Sec. 4, 5).
 * ------------------------------------------------------------------------ */

/* One product of a batch: c[0 .. la+lb-1) = a * b mod p.  a, b, c are device
 * pointers (c must not overlap a or b); p prime, 3 <= p < 2^31;
 * la + lb - 1 <= 2^21 and 2^ceil(log2(la+lb-1)) must divide p - 1. */
typedef struct polymul_desc {
    const uint32_t *a;
    const uint32_t *b;
    uint32_t *c;
    uint32_t la;
    uint32_t lb;
    uint32_t p;
    uint32_t reserved;   /* must be 0 */
} polymul_desc;

/* Launch shape of a batch: CTAs per SM of the persistent grid (0 = as many
 * as fit), the job order, the kernel variant and the transform form.
 * Truncated transforms (the TFT of J. van der Hoeven, "The truncated Fourier
 * transform and applications", 2004, which the polynomial libraries of
 * Sec. 1 use to avoid power-of-two padding): a product of N = 2^K, split into
 * 2^(K-13) rows of 2^13, computes only the first ceil((la + lb - 1) / 2^13)
 * rows of the forward transforms (the first outputs in bit-reversed order)
 * and recovers c from them by an inverse TFT over each column; the results
 * are the same, bit for bit.
 * Kernel forms: the persistent kernel (0, 1) claims jobs from one list and
 * waits, bounded, on per-product counters; the phased form (2) runs each job
 * kind as its own kernel with its own register budget, one CTA per job, in
 * stream order on `stream` (the forward columns, rows and output columns of
 * every product above 2^13) plus a side stream the plan owns (the products
 * up to 2^13, one kernel per size), joined back before the call's work
 * ends: no device-side waits, and the same results.  Products up to 2^13 run
 * whole in one CTA, products of 2^14 and 2^15 as one whole-product job each,
 * larger ones as column-tile, row and output-tile jobs.  Orders: 0: column
 * tiles first, then whole-product and small jobs, then rows and output
 * tiles; 1: whole-product and small jobs first; 2, 3: software-pipelined,
 * rows of one product beside the column tiles of a later one, lag 32 or 64
 * products.  Chosen by polymul_batch_plan_tune. */
typedef struct polymul_batch_config {
    int ctas_per_sm;
    int order;
    int kernel;            /* 0: persistent kernel, registers budgeted for 2 CTAs per SM; 1: for 3;
                              2: phased form, one kernel per job kind (ctas_per_sm and order unused) */
    int full_transforms;   /* 0 (default): products of N = 2^15 .. 2^17 whose length leaves rows of
                              2^13 unused run as truncated transforms (below); 1: every product is
                              padded to its full power-of-two transform */
} polymul_batch_config;

/* Library-owned plan: device copies of the job list and the product table,
 * synchronisation counters, scratch (2N words per product with N > 2^13),
 * resident twiddle tables and, once used, a CUDA graph.  Creation allocates
 * and copies synchronously (not during stream capture).  Up to 8 distinct
 * primes per batch (else MONT_EUNSUPPORTED). */
typedef struct polymul_batch_plan polymul_batch_plan;

int polymul_batch_plan_create(const polymul_desc *descs, size_t count, polymul_batch_plan **out);

/* Host only, no device work: the job list the batch kernel runs for these
 * descriptors in job order `order` (0 .. 3), for inspection and tests.  The
 * first min(cap, *njobs) jobs go to jobs, 4 words each: kind (0: single-CTA
 * products, the job covering `count` consecutive products; 1: column tile;
 * 2: row; 3: output tile; 4: whole product), log2 N, product, and the tile
 * or row index (kind 0: the product count).  Products are numbered in the
 * kernel's order (single-CTA products first, by size, then the others in
 * descriptor order); prods, if not NULL, receives 4 words per product:
 * log2 N, column tiles, rows computed, and 1 if the product runs as a
 * truncated transform.  full_transforms as in polymul_batch_config.
 * *njobs gets the full job count.  Errors as polymul_batch_plan_create's
 * descriptor checks; MONT_EINVAL for a bad order or full_transforms. */
int polymul_batch_describe(const polymul_desc *descs, size_t count, int order, int full_transforms, uint32_t *jobs,
                           size_t cap, uint32_t *prods, size_t *njobs);
/* Frees the plan and its device tables (NULL is a no-op); queued runs of it
 * must have finished. */
void polymul_batch_plan_destroy(polymul_batch_plan *plan);
/* Bytes of scratch the plan holds (2N words per product with N > 2^13). */
size_t polymul_batch_plan_workspace_bytes(const polymul_batch_plan *plan);
/* The plan's current launch configuration; set_config checks the fields
 * (MONT_EINVAL: ctas_per_sm < 0, order not 0 .. 3, kernel not 0 .. 2,
 * full_transforms not 0 or 1) and takes effect on the next run. */
int polymul_batch_plan_get_config(const polymul_batch_plan *plan, polymul_batch_config *cfg);
int polymul_batch_plan_set_config(polymul_batch_plan *plan, const polymul_batch_config *cfg);

/* Queue the whole batch on `stream`: one memset of the counters and one
 * persistent kernel launch (kernel 0, 1), or the phased form's kernels on
 * `stream` and the plan's side stream, joined back into `stream`
 * (kernel 2).  The operands must be ready when it runs.  Runs of one plan
 * share its counters, scratch and side stream: two of them must not be in
 * flight at once (queue them on one stream, or order them with events);
 * distinct plans are independent. */
int polymul_batch_run(polymul_batch_plan *plan, cudaStream_t stream);

/* Same work replayed from a CUDA graph captured on first use (re-captured
 * when the configuration changes). */
int polymul_batch_run_graph(polymul_batch_plan *plan, cudaStream_t stream);

/* Synchronises `stream`, then reports MONT_OK, or MONT_ETIMEOUT when a
 * bounded wait inside the last run of the plan expired (its results are
 * then incomplete; the device context stays usable). */
int polymul_batch_status(polymul_batch_plan *plan, cudaStream_t stream);

/* Autotuner (the generator's timing search of Sec. 4, 5, over launch shapes
 * instead of code variants): runs the batch `trials` times per launch shape
 * (persistent kernel variant x CTAs per SM x job order, and the phased
 * form), keeps the fastest (CUDA-event timed on `stream`) and caches it for
 * batches with the same size histogram on this device; the plan's
 * full_transforms choice is kept.  Synchronous.  Returns the status of the
 * last run. */
int polymul_batch_plan_tune(polymul_batch_plan *plan, cudaStream_t stream, int trials);

/* One-shot batch without a plan: the same kernels and results as
 * polymul_batch_plan_create + polymul_batch_run, in the phased form with
 * truncated transforms (every kernel in order on `stream`), with every
 * device table of the batch in the caller's workspace.  Each call validates
 * the descriptors, builds the job lists on the host, queues copies of them
 * and of the product table from pageable host memory into the workspace (so
 * not during stream capture; a plan can be captured), and launches the
 * kernels.
 * workspace: device memory, 256-byte aligned (as cudaMalloc returns), at
 * least polymul_batch_workspace_bytes(descs, count) bytes; it must not be
 * used by other work until the queued kernel finishes (calls on one stream
 * may share it).  Descriptor errors as polymul_batch_plan_create;
 * MONT_EINVAL for a missing, misaligned or short workspace.  The twiddle
 * tables of each prime are built on first use (make the first call outside
 * stream capture).  count == 0 is a no-op. */
int polymul_batch(const polymul_desc *descs, size_t count, void *workspace, size_t ws_bytes, cudaStream_t stream);

/* Host only: workspace bytes polymul_batch needs for these descriptors
 * (counters, product table, the phased form's job lists and 2N words of
 * scratch per product with N > 2^13); 0 for count == 0 or invalid
 * descriptors. */
size_t polymul_batch_workspace_bytes(const polymul_desc *descs, size_t count);

/* Synchronises `stream`, then reports the status word of the last
 * polymul_batch run on this workspace: MONT_OK (the phased form has no
 * device-side waits, so nothing sets MONT_ETIMEOUT there). */
int polymul_batch_check(const void *workspace, cudaStream_t stream);

/* Bound of every device-side wait of the plan (default 2^22 polls, 2 s). */
int polymul_batch_plan_set_wait_limit(polymul_batch_plan *plan, uint32_t iterations, uint64_t nanoseconds);

/* Failure-detection test hook: makes the first product with N > 2^15 wait
 * for a column tile that does not exist, so its bounded waits expire and
 * polymul_batch_status reports MONT_ETIMEOUT.  MONT_EINVAL if the batch has
 * no product with N > 2^15 (smaller ones run without cross-CTA waits). */
int polymul_batch_plan_inject_stall(polymul_batch_plan *plan);

/* ------------------------------------------------------------------------
 * Continuous-batching request server (one device).  The caller drives it
 * from one host thread; internally one launcher thread per slot builds and
 * queues its batches.
 * ------------------------------------------------------------------------ */

/* One request: c[0 .. la+lb-1) = a * b mod p.  a, b, c may be host memory
 * (pinned for asynchronous copies) or device memory; they must stay valid
 * until the request's completion is reported.  id is returned with it. */
typedef struct mont_request {
    const uint32_t *a;
    const uint32_t *b;
    uint32_t *c;
    uint32_t la;
    uint32_t lb;
    uint32_t p;
    uint32_t reserved;   /* must be 0 */
    uint64_t id;
} mont_request;

typedef struct mont_completion {
    uint64_t id;
    int status;          /* MONT_OK, MONT_ETIMEOUT or MONT_ECUDA */
    int reserved;
} mont_completion;

typedef struct mont_server_stats {
    uint64_t submitted, admitted, launched, completed, batches;   /* running totals */
    uint64_t queued, admitted_waiting, in_flight;                   /* current requests per stage */
    uint64_t bytes_in_use, peak_bytes, budget_bytes;                /* device-memory budget */
} mont_server_stats;

typedef struct mont_server mont_server;

/* Server for the given primes (at most 8; twiddle tables for N up to
 * 2^max_log2n, max_log2n <= 21, built now and kept resident), a device-memory
 * budget of budget_bytes (one allocation made now) that holds every admitted
 * request's operands, result and scratch, `slots` streams (batches in flight
 * at once) and at most max_batch_coeffs input coefficients per batch (a single
 * larger request still forms a batch of its own). */
int mont_server_create(const uint32_t *primes, int nprimes, uint32_t max_log2n, size_t budget_bytes, int slots,
                       size_t max_batch_coeffs, mont_server **out);

/* Waits for the work in flight, then frees everything. */
void mont_server_destroy(mont_server *server);

/* Queues n requests (no device work).  The whole call is rejected with
 * MONT_EINVAL (bad pointer, length, or a prime the server was not created
 * for) or MONT_ERANGE (N beyond max_log2n, or a request larger than the
 * whole budget). */
int mont_server_submit(mont_server *server, const mont_request *reqs, size_t n);

/* Non-blocking step: retires finished batches (their memory returns to the
 * budget), admits queued requests in order while memory allows, launches the
 * admitted requests on every idle slot, and copies up to cap completions
 * into done (*ndone of them).  Call it repeatedly from one thread. */
int mont_server_progress(mont_server *server, mont_completion *done, size_t cap, size_t *ndone);

int mont_server_get_stats(const mont_server *server, mont_server_stats *out);

/* Frees the library-owned scratch buffers (waits for the device). */
int mont_release_workspaces(void);

/* ------------------------------------------------------------------------
 * Measurement support: integer-pipe throughput probes.  (The paper reports
 * no measurements; these give the roofline of Alg. 2's arithmetic and of the
 * NTT butterflies built on it a measured ceiling on the device at hand.)
 * ------------------------------------------------------------------------ */

/* Probe kinds: one instruction form each (32-bit multiply-add, high-word
 * multiply-add, 32x32->64 multiply-add, three-input add), one REDC (Alg. 2,
 * result fully reduced), and the NTT butterflies as the transform kernels
 * run them: Cooley-Tukey with a twiddle (REDC of y by w, lazy [0, 2P)
 * values), with twiddle 1, with twiddle 1 on reduced inputs (level 0), and
 * Gentleman-Sande with a twiddle and with twiddle 1. */
enum {
    MONT_PROBE_IMAD = 0,
    MONT_PROBE_IMAD_HI = 1,
    MONT_PROBE_IMAD_WIDE = 2,
    MONT_PROBE_IADD3 = 3,
    MONT_PROBE_REDC = 4,
    MONT_PROBE_CT = 5,
    MONT_PROBE_CT_ONE = 6,
    MONT_PROBE_CT_FIRST = 7,
    MONT_PROBE_GS = 8,
    MONT_PROBE_GS_ONE = 9
};

/* Queues one probe kernel on `stream`: a grid of ctas_per_sm CTAs per SM
 * (0 = as many as fit; 256 threads each), every thread applying the
 * operation `kind` to 8 independent register chains 16 x iterations times,
 * with no memory traffic.  *ops_per_launch (if not NULL) receives the number
 * of operations the launch performs (instructions, REDCs or butterflies);
 * divided by the launch's duration it is the throughput.  p: odd modulus,
 * 3 <= p < 2^31, used by the REDC and butterfly kinds.  sink: a device word
 * the kernel may write (keeps the chains live).  MONT_EINVAL for an unknown
 * kind, a bad p, iterations == 0 or a NULL sink. */
int mont_int_probe(int kind, uint32_t p, uint32_t iterations, uint32_t ctas_per_sm, uint32_t *sink,
                   uint64_t *ops_per_launch, cudaStream_t stream);

/* Static description of a return code (the MONT_E* codes above; the paper
 * defines no error model); never NULL. */
const char *mont_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
