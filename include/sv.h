/*
 * sv.h -- C ABI of the GB300 (sm_103a) squarefree + power-of-two verifier.
 *
 * The operation (C. Hercher, "On the Sum of Squarefree Integers and a Power of
 * Two", arXiv 2411.01964): for every odd n > 1 find the smallest k >= 1 such
 * that n - 2^k is a positive squarefree integer (the Conjecture in Sec. 1 and
 * the Theorem in Sec. 4), called mink(n) below.  The library computes it with
 * Algorithm 1 (a sieve of the odd squarefree integers, Sec. 3) followed by
 * Algorithm 2 (the per-n search over k, Sec. 3), and aggregates the results the
 * way Sec. 3 "Collecting the results" does (sum and maximum of k), extended to
 * a histogram over k, first occurrences (the records of Table 3) and lists.
 *
 * Conventions shared by every entry point
 *   - All arithmetic is exact unsigned 64-bit integer arithmetic: the device
 *     code uses no floating point at all (square roots are integer Newton
 *     iterations).  The host uses floating point only for estimates that never
 *     change a result: buffer sizes, and the first guess of an integer square
 *     root that exact integer steps then correct.
 *   - Every entry point makes the context's CUDA device current while it runs
 *     and gives the calling thread its own current device back afterwards.
 *   - squarefree(s): s >= 1 and no prime p with p^2 | s.  1 is squarefree.
 *   - mink(n) = min{ k >= 1 : 2^k < n and n - 2^k squarefree }.  If no such k
 *     exists n is a "failure" (the case Algorithm 2 prints as "no
 *     representation found"; it never occurred in the paper).
 *   - A range [lo, hi) is half-open (Algorithm 1's "[start; end[") and covers
 *     the odd n with max(lo, 3) <= n < hi (the Conjecture asks n > 1).
 *   - Limits: hi <= 2^62, and the prime table set up by sv_init_primes(max_hi)
 *     must cover the request: hi <= max_hi (else SV_ERANGE).
 *   - Every call returns an sv_status; the library never aborts, traps or
 *     exits the process.  Device faults are reported as SV_ECUDA.
 *   - Ownership: the context owns all device memory it allocates; caller
 *     buffers (host or device, as documented per call) stay owned by the caller
 *     and are only written, never freed or retained past the call (sv_submit:
 *     past completion).
 *   - Threading: one context may be used from several host threads for
 *     sv_submit / sv_poll / sv_cancel.  The blocking calls (sv_verify_range,
 *     sv_verify_batch, sv_min_k, sv_sieve_bitmap) and the device-resident
 *     calls are serialised per context by an internal mutex.
 */
#ifndef SV_H
#define SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sv_status {
    SV_OK = 0,
    SV_EINVAL = 1,      /* invalid argument (NULL pointer, lo > hi, bad config) */
    SV_ERANGE = 2,      /* hi beyond 2^62 or beyond the prime table (sv_init_primes) */
    SV_ENOMEM = 3,      /* host or device allocation failed; admission refused */
    SV_EAGAIN = 4,      /* sv_poll: the request has not finished yet */
    SV_ETIMEDOUT = 5,   /* a bounded wait ran out */
    SV_ECANCELLED = 6,  /* the request was cancelled */
    SV_ECUDA = 7,       /* a CUDA runtime call or kernel failed */
    SV_ENOPRIMES = 8,   /* sv_init_primes has not been called */
    SV_ENOTFOUND = 9,   /* unknown ticket */
    SV_EOVERFLOW = 10   /* an internal device buffer overflowed and the retry failed */
} sv_status;

typedef struct sv_ctx sv_ctx; /* opaque: prime table, scratch, streams, graphs, server */

/*
 * Tuning knobs.  Every field may be 0, meaning "choose automatically" (the
 * built-in defaults, or the values found by sv_autotune).  None of them
 * changes any result; they only change speed and memory.
 */
typedef struct sv_config {
    uint32_t tile_log2;          /* odd numbers per shared-memory tile = 2^tile_log2 (14..20) */
    uint32_t margin_log2;        /* look-back below each tile, in integers: W = 2^margin_log2
                                    (6..tile_log2+1).  n - 2^k with 2^k <= W is read from the
                                    tile's own window; larger k go to the exact straggler test */
    uint32_t threads;            /* threads per CTA of the tile kernel (256, 512 or 1024) */
    uint32_t large_prime_min;    /* lower bound of the bucket threshold: primes from the threshold on
                                    are delivered through per-tile buckets.  The library raises the
                                    threshold to about sqrt(range length / 128) and keeps at most 2048
                                    primes between the dense ones and it */
    uint32_t bucket_capacity;    /* entries per tile bucket (grown automatically on overflow) */
    uint32_t record_k_threshold; /* T: every n with mink(n) >= T is listed (default 6) */
    uint32_t ctas_per_sm;        /* resident tile CTAs per SM (1 or 2) */
    uint32_t stamp_primes;       /* how many of the smallest odd primes (3, 5, 7, ...) are applied as
                                    computed word patterns instead of atomic strikes: 2, 4, 6 or 8 */
    uint64_t list_capacity;      /* device list entries per range (grown on overflow) */
    uint64_t device_mem_budget;  /* bytes the serving loop may hold for requests in flight */
    void *cuda_stream;           /* cudaStream_t used for all work; NULL = a library stream */
    uint32_t list_stage_capacity;/* listed n a tile may stage for the ordered list (1..128; 0 = 128).
                                    A tile with more repeats the launch through the unordered list
                                    path; results never depend on it (small values exercise that path) */
    uint32_t mult_prime_log2;    /* multiplier threshold: bucket primes p >= 2^mult_prime_log2 reach the
                                    buckets by enumerating the odd multipliers j of j p^2 in the range
                                    (cheap for many short ranges far up); smaller bucket primes take one
                                    Barrett reduction per range (10..31; 0 = 18) */
    uint32_t serve_slots;        /* launches the serving loop keeps in flight, each on its own stream
                                    with its own device workspace (1..8; 0 = 4) */
    uint32_t reserved1;
} sv_config;

/*
 * Result of one range, filled by sv_verify_range / sv_verify_batch / sv_poll.
 * The caller sets the buffer pointers and capacities (any may be NULL with
 * capacity 0) before the call; everything else is written by the library.
 * Entries of list / list_k past min(list_len, list_cap) are unspecified (the
 * library may write there, never past list_cap).  For a call of one range
 * whose list / list_k are page-locked host memory (cudaHostAlloc or
 * cudaHostRegister), the list is copied from the device straight into them;
 * other buffers receive it through the library's own staging.
 */
typedef struct sv_range_result {
    uint64_t lo, hi;          /* echoed */
    uint64_t n_odd;           /* number of odd n in [max(lo,3), hi) */
    uint64_t hist[64];        /* hist[k] = #odd n with mink(n) = k (hist[0] unused) */
    uint64_t first_n[64];     /* smallest n with mink(n) = k; UINT64_MAX if none */
    uint64_t ksum;            /* sum of mink over the range (Sec. 3 "Collecting the results") */
    uint64_t kmax;            /* largest mink in the range (same section) */
    uint64_t *list;           /* caller-owned, ascending: every n with mink(n) >= T */
    uint8_t *list_k;          /* caller-owned: mink of list[i] (may be NULL) */
    uint64_t list_cap;        /* capacity of list / list_k */
    uint64_t list_len;        /* entries found; may exceed list_cap (then truncated) */
    uint64_t *failures;       /* caller-owned, ascending: odd n without any k */
    uint64_t fail_cap;
    uint64_t fail_len;        /* failures found; may exceed fail_cap (then truncated) */
    uint8_t *per_n_k;         /* optional, caller-owned HOST buffer of n_odd bytes: mink of the
                                 i-th odd n of the range at index i; 255 = failure; NULL = skip */
    uint64_t list_overflow;   /* 1 if list_len > list_cap */
} sv_range_result;

typedef enum sv_request_kind { SV_REQ_RANGE = 0, SV_REQ_POINTS = 1 } sv_request_kind;

/* One serving request (sv_submit). Buffers must stay valid until sv_poll
 * returns SV_OK or SV_ECANCELLED for its ticket. */
typedef struct sv_request {
    uint32_t kind;            /* sv_request_kind */
    uint32_t reserved;
    uint64_t lo, hi;          /* SV_REQ_RANGE */
    sv_range_result *result;  /* SV_REQ_RANGE: caller-owned host result */
    const uint64_t *points;   /* SV_REQ_POINTS: caller-owned host array */
    uint64_t n_points;
    uint8_t *out_k;           /* SV_REQ_POINTS: caller-owned host output, n_points bytes */
} sv_request;

/* Serving counters (sv_server_stats). Latencies in microseconds. */
typedef struct sv_server_stats {
    uint64_t submitted, completed, cancelled, refused;
    uint64_t odd_n_done;      /* odd n verified by completed range requests + points */
    uint64_t launches;        /* batched device launches issued */
    uint64_t in_flight;       /* requests admitted and not yet completed */
    uint64_t queued;          /* requests waiting for admission */
    double p50_us, p99_us;    /* over completed requests since start */
    uint64_t peak_mem_in_flight; /* largest device memory (the admission estimate) of the launches in
                                    flight at one time; at most device_mem_budget unless a single
                                    launch alone needs more */
    double wall_us;           /* time since the server started or the stats were reset */
    double loop_busy_us;      /* of that, time the serving thread spent packing, launching and
                                 collecting (the rest it waited for work or for the GPU) */
} sv_server_stats;

/* Human-readable name of a status (static string, never NULL). */
const char *sv_strerror(sv_status s);

/*
 * Create a context on the current CUDA device.  cfg may be NULL (all
 * automatic).  On success *ctx owns a stream (unless cfg->cuda_stream is set)
 * and no prime table yet.  Errors: SV_EINVAL, SV_ENOMEM, SV_ECUDA.
 */
sv_status sv_create(sv_ctx **ctx, const sv_config *cfg);

/* Stop the server (pending requests complete as SV_ECANCELLED), free all
 * device memory.  NULL is allowed. */
void sv_destroy(sv_ctx *ctx);

/* The effective configuration (after automatic choices). */
sv_status sv_get_config(const sv_ctx *ctx, sv_config *out);

/*
 * Algorithm 1 needs every prime 3 <= p < sqrt(end) (Sec. 3).  Builds, on the
 * device, the table of all odd primes p <= isqrt(max_hi - 1) with the
 * constants the kernels use, and keeps it resident.  max_hi <= 2^62.  Calling
 * it again with a larger max_hi rebuilds the table; a smaller one is a no-op.
 * Errors: SV_EINVAL, SV_ERANGE, SV_ENOMEM, SV_ECUDA.
 */
sv_status sv_init_primes(sv_ctx *ctx, uint64_t max_hi);

/* Number of odd primes in the resident table and the largest one. */
sv_status sv_prime_count(const sv_ctx *ctx, uint64_t *count, uint64_t *largest);

/*
 * Copies the resident table (the primes of Algorithm 1, Sec. 3) into HOST
 * arrays owned by the caller, for inspection: p[i] (ascending odd primes) and
 * mu[i] = floor((2^64-1) / p^2) for i < min(cap, count); inv[i] = p^-1 mod
 * 2^64 and lim[i] = floor((2^64-1) / p) for i < min(cap, *n_div), the primes
 * that carry divisibility constants (all p < 2^21 of the table).  Any array
 * pointer may be NULL.  Blocking.  Errors: SV_EINVAL, SV_ENOPRIMES, SV_ECUDA.
 */
sv_status sv_prime_table_copy(sv_ctx *ctx, uint32_t *p, uint64_t *mu, uint64_t *inv, uint64_t *lim,
                              uint64_t cap, uint64_t *n_div);

/*
 * Verify one range (Algorithms 1 and 2, Sec. 3): mink of every odd n in
 * [max(lo,3), hi), aggregated into *out.  Blocking.  out's buffers are HOST
 * memory owned by the caller.  lo >= hi gives an empty result.
 * Errors: SV_EINVAL, SV_ERANGE, SV_ENOPRIMES, SV_ENOMEM, SV_ECUDA, SV_EOVERFLOW.
 */
sv_status sv_verify_range(sv_ctx *ctx, uint64_t lo, uint64_t hi, sv_range_result *out);

/*
 * Verify `count` independent ranges [lo[i], hi[i]) in one batched, persistent,
 * CUDA-graph launch (all tiles of all ranges share one work queue).  out[i]
 * as for sv_verify_range.  Blocking.
 */
sv_status sv_verify_batch(sv_ctx *ctx, const uint64_t *lo, const uint64_t *hi, size_t count,
                          sv_range_result *out);

/*
 * mink of single points (Algorithm 2 for one n, with every n - 2^k decided by
 * an exact squarefree test).  points and out_k are HOST arrays of `count`
 * entries.  out_k[i] = mink(points[i]); 0 if points[i] is even or < 3; 255 if
 * no k with 2^k < n works.  Every point must be < the table's max_hi.
 * Errors: SV_EINVAL, SV_ERANGE, SV_ENOPRIMES, SV_ENOMEM, SV_ECUDA.
 */
sv_status sv_min_k(sv_ctx *ctx, const uint64_t *points, size_t count, uint8_t *out_k);

/*
 * Algorithm 1 alone: the squarefree flags of the odd integers of [lo, hi)
 * into d_bitmap, a DEVICE buffer of sv_bitmap_words(lo, hi) uint32 words.
 * Bit b of word i describes the odd integer m = 64*(floor(lo/64) + i) + 2b + 1
 * (1 = squarefree); bits for m outside [lo, hi) are 0.  Blocking.
 */
sv_status sv_sieve_bitmap(sv_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t *d_bitmap);
uint64_t sv_bitmap_words(uint64_t lo, uint64_t hi);

/*
 * The plain (unfused) form of sv_verify_range, with the bitmap through device
 * memory as Sec. 3 describes it: Algorithm 1 writes the squarefree flags of
 * the odd integers from the range's look-back margin up to hi into a bitmap in
 * device memory (one bit per odd integer, 128-bit bulk stores from shared
 * memory), then Algorithm 2 reads them back tile by tile (bulk loads into
 * shared memory) and finds mink.  Results are identical to sv_verify_range;
 * the fused path is faster because its bitmap never leaves shared memory.
 * The bitmap (about (hi - lo) / 16 bytes) is owned by the context and kept
 * for the next call.  out as for sv_verify_range (HOST buffers).  Blocking.
 * Errors: as sv_verify_range, and SV_ETIMEDOUT if a bulk copy did not
 * complete within about a second.
 */
sv_status sv_verify_range_plain(sv_ctx *ctx, uint64_t lo, uint64_t hi, sv_range_result *out);

/* Device-resident form of sv_verify_range_plain: both passes are enqueued on
 * the context's stream without waiting; sv_fetch_range collects the result.
 * d_per_n_k as for sv_launch_range. */
sv_status sv_launch_range_plain(sv_ctx *ctx, uint64_t lo, uint64_t hi, uint8_t *d_per_n_k);

/*
 * Device-resident form of sv_verify_range: enqueue the whole range on the
 * context's stream and return without waiting; results stay in device memory
 * until sv_fetch_range.  d_per_n_k is an optional caller-owned DEVICE buffer
 * of n_odd bytes (NULL = skip).  One range may be pending per context.
 */
sv_status sv_launch_range(sv_ctx *ctx, uint64_t lo, uint64_t hi, uint8_t *d_per_n_k);

/* Wait for the pending sv_launch_range (or sv_launch_range_plain) and copy its aggregates to *out
 * (out->per_n_k is ignored: the per-n values are already in the device
 * buffer given to sv_launch_range). */
sv_status sv_fetch_range(sv_ctx *ctx, sv_range_result *out);

/*
 * Device-resident form of sv_verify_batch: enqueue the batch as one replay of
 * the captured launch graph and return without waiting (list capacity per
 * range: sv_config.list_capacity).  sv_fetch_batch waits and copies the
 * aggregates into out[0..count) (count must match).  One launch may be
 * pending per context (a range or a batch).
 */
sv_status sv_launch_batch(sv_ctx *ctx, const uint64_t *lo, const uint64_t *hi, size_t count);
sv_status sv_fetch_batch(sv_ctx *ctx, sv_range_result *out, size_t count);

/* Device-resident form of sv_min_k: d_points / d_out_k are DEVICE arrays;
 * enqueued on the context's stream, no wait. */
sv_status sv_min_k_device(sv_ctx *ctx, const uint64_t *d_points, size_t count, uint8_t *d_out_k);

/* Wait until all work enqueued on the context's stream has finished. */
sv_status sv_synchronize(sv_ctx *ctx);

/*
 * Autotuner (coordinate descent, two rounds): times candidate values of each
 * knob in turn -- tile shape (tile_log2, threads, ctas_per_sm), stamped
 * primes, look-back margin, bucket threshold (large_prime_min), multiplier
 * threshold (mult_prime_log2) and bucket depth (bucket_capacity) -- with the
 * others held, and keeps the fastest configuration in the context (and in
 * *chosen, if not NULL).  The work timed is the device time (CUDA events on the
 * context's stream, best of three after a warm-up) of [lo, hi) as one launch
 * (sv_autotune) or of the `count` ranges as one batched launch
 * (sv_autotune_batch), a sample of the target workload.  Never changes
 * results.  Errors: as sv_verify_range / sv_verify_batch.
 */
sv_status sv_autotune(sv_ctx *ctx, uint64_t lo, uint64_t hi, sv_config *chosen);
sv_status sv_autotune_batch(sv_ctx *ctx, const uint64_t *lo, const uint64_t *hi, size_t count, sv_config *chosen);

/*
 * Serving.  sv_submit admits a range or point request into the request loop
 * (continuous batching: requests that arrive while others are on the GPU are
 * packed into the next launches as device memory and launch slots free up;
 * long ranges are split so that they do not block short ones).  *ticket
 * identifies it.  Admission is by device memory: the launches in flight stay
 * within sv_config.device_mem_budget, and a request waits until its next unit
 * of work fits.  SV_ENOMEM: even the request's smallest unit of work (its
 * first chunk of at most 2^30 integers, or one launch's points) exceeds the
 * budget, or the queue is full; nothing is queued then.
 */
sv_status sv_submit(sv_ctx *ctx, const sv_request *req, uint64_t *ticket);

/*
 * Several requests at once (a burst from one client): each is checked and
 * queued as by sv_submit, all under one lock.  status[i] receives request i's
 * outcome and tickets[i] its ticket where status[i] is SV_OK; the call returns
 * the first failing status, or SV_OK.  reqs, tickets and status are HOST
 * arrays of `count` entries.
 */
sv_status sv_submit_many(sv_ctx *ctx, const sv_request *reqs, size_t count, uint64_t *tickets, sv_status *status);

/* SV_OK when the request has finished (its result is written), SV_EAGAIN if
 * still pending after timeout_us microseconds (0 = do not wait, < 0 = wait
 * without limit), SV_ECANCELLED, SV_ENOTFOUND.  A finished ticket is
 * released by the call that reports it. */
sv_status sv_poll(sv_ctx *ctx, uint64_t ticket, int64_t timeout_us);

/* Cancel a request that has not started on the device yet (a running one
 * completes normally).  SV_OK if cancelled, SV_EAGAIN if already running. */
sv_status sv_cancel(sv_ctx *ctx, uint64_t ticket);

/* Serving counters since the server started (first sv_submit) or since the
 * last sv_server_stats_reset. */
sv_status sv_server_stats_get(sv_ctx *ctx, sv_server_stats *out);

/* Restarts the serving counters and latency samples (requests in flight are
 * not affected; their completions count in the new period). */
sv_status sv_server_stats_reset(sv_ctx *ctx);

/* Replace the tuning knobs (same rules as sv_create; the stream is kept). */
sv_status sv_set_config(sv_ctx *ctx, const sv_config *cfg);

/* Bytes the last blocking call copied host->device and device->host
 * (inputs, descriptors, aggregates, lists, per-n values). */
sv_status sv_last_transfer(const sv_ctx *ctx, uint64_t *h2d_bytes, uint64_t *d2h_bytes);

/*
 * sv_verify_range for callers that cannot allocate memory when they verify.
 * Such callers include a process whose GPU memory is already held by a caching
 * allocator (PyTorch's, for one), where a cudaMalloc by this library would
 * fail; latency-critical loops, because cudaMalloc and cudaFree can
 * synchronise the whole device and take milliseconds; and services whose
 * memory budget is fixed at start-up.  The paper has no counterpart: this is
 * a property of this library's interface, not of the method.
 *
 * It computes exactly what sv_verify_range computes, with the same kernels,
 * and allocates nothing: no cudaMalloc, cudaFree or cudaMallocHost and no
 * other allocating routine.  All scratch memory (launch header, descriptor,
 * result slot, tile buckets, straggler queue, list and failure arenas) comes
 * from one fixed 8 MiB array in device memory that the library declares at
 * file scope; every GPU that loads the library holds those 8 MiB until the
 * process exits.  Results are written into the caller's buffers in *out
 * (HOST memory, as for sv_verify_range).  The call blocks: it waits for the
 * context's stream and copies the results back through small host stack
 * buffers before it returns.
 *
 * Limits and rules:
 *   - hi - lo <= 2^32, and the range's tile buckets must fit the array (true
 *     for every such range with the default tile size); otherwise SV_ERANGE.
 *   - At most 65536 listed n (mink >= T) and 1024 failures per call, and a
 *     straggler queue (n whose n - 2^k leaves a tile's look-back window) of
 *     at least 4096 entries: what the array holds after the other parts.  More
 *     listed n or more stragglers give SV_EOVERFLOW (sv_verify_range would
 *     grow its buffers instead).  out->per_n_k must be NULL (SV_EINVAL).
 *   - sv_init_primes must have been called before (it allocates, once, at
 *     set-up): SV_ENOPRIMES otherwise.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture begins.
 *   - Every call shares the one array, which keeps the previous call's
 *     contents (the call clears what must start at zero).  Calls that overlap
 *     on the GPU -- from different contexts or threads on the same device --
 *     race on it and must not be issued; calls through one context are
 *     serialised by the context.
 * Errors: SV_EINVAL, SV_ERANGE, SV_ENOPRIMES, SV_ECUDA, SV_EOVERFLOW.
 */
sv_status sv_verify_range_noalloc(sv_ctx *ctx, uint64_t lo, uint64_t hi, sv_range_result *out);

/*
 * Measured peaks of this GPU for the rooflines of the tile kernel (Algorithms 1
 * and 2 of Sec. 3 fused): the strikes of Algorithm 1 are shared-memory atomics
 * and the word-parallel Algorithm 2 is integer work.  Rates are for the whole
 * GPU (every SM at full occupancy), per second.
 */
typedef struct sv_peaks {
    double smem_atomic_per_s;        /* 32-bit shared-memory atomicAnd, the 32 lanes of a warp on 32 banks */
    double smem_atomic_strike_per_s; /* the same in the dense-strike pattern: lanes q = p^2 bits apart */
    double scan_mix_ops_per_s;       /* funnel shift, AND-NOT, popcount, add (one scan step = 4 ops) */
    double int_alu_ops_per_s;        /* three-input logic and 32-bit add */
    double popc_per_s;               /* population counts, in a loop of one popcount per four operations */
    double sm_clock_max_mhz;         /* the device's maximum SM clock (attribute, not measured) */
    uint32_t sms;                    /* streaming multiprocessors */
    uint32_t reserved;
} sv_peaks;

/*
 * Runs the microbenchmarks behind sv_peaks on the context's device: each probe
 * kernel runs a few milliseconds on every SM, timed with CUDA events on the
 * context's stream (best of five after a warm-up).  Allocates a small scratch
 * buffer; changes no device setting.  Errors: SV_EINVAL, SV_ENOMEM, SV_ECUDA.
 */
sv_status sv_measure_peaks(sv_ctx *ctx, sv_peaks *out);

/*
 * Test hook for the failure paths: the next `count` device or pinned-host
 * buffer allocations the library makes (in any context of the process) fail
 * as if memory were exhausted; the calls that needed them return SV_ENOMEM
 * (a served request completes with SV_ENOMEM) and the library stays usable.
 * count = 0 clears the hook.  No GPU operation is affected: the failure is
 * made on the host, before the allocation call.
 */
sv_status sv_inject_alloc_failures(sv_ctx *ctx, uint32_t count);

/*
 * Test hook for the bounded waits: the next `count` plain-path launches of
 * this context (sv_verify_range_plain, sv_launch_range_plain) leave out their
 * bulk window loads and wait at most about half a millisecond for them, so
 * every block's bounded wait runs out; the call returns SV_ETIMEDOUT and the
 * context stays usable.  Nothing is in flight when a block gives up: no GPU
 * fault, trap or hang is involved.  count = 0 clears the hook.
 */
sv_status sv_inject_bulk_timeout(sv_ctx *ctx, uint32_t count);

/* Number of kernels this context has launched so far. */
uint64_t sv_kernel_launches(const sv_ctx *ctx);

/* Per-kernel timing: when enabled, each launch of a timed kernel is
 * bracketed by CUDA events recorded on the stream it is launched on.  A
 * launch replayed from a captured graph times only its tile kernel (id 2),
 * through event-record nodes given fresh events at every replay; the others
 * in it are not timed, so sv_launch_range takes the graph path only while no
 * other kernel is timed.  enable: 0 off, -1 every
 * kernel, otherwise a bit mask of kernel ids (bit i: id i); every call resets
 * the totals.  Kernel ids: 0 init, 1 bucket fill, 2 tile (sieve + scan),
 * 3 stragglers, 4 points, 5 ordered-list compaction, 6 tile kernel of the
 * plain path's sieve pass, 7 tile kernel of the plain path's scan pass. */
sv_status sv_kernel_timing(sv_ctx *ctx, int enable);

/* Total milliseconds and launch count of one kernel id since the last reset
 * (waits for the context's stream). */
sv_status sv_kernel_time(sv_ctx *ctx, int kernel, double *total_ms, uint64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* SV_H */
