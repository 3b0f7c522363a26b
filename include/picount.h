/*
 * picount.h -- C ABI of the GB300 (sm_103a) prime-counting library.
 *
 * The library computes pi(x), the number of primes <= x, and the partial
 * sieve function phi(x, a) (the count of 1 <= n <= x coprime to the first a
 * primes, defined in Section 3 of Staple, "The combinatorial algorithm for
 * computing pi(x)", arXiv:1503.01839) by the combinatorial method the paper
 * refines (Sections 2-4): ordinary leaves, special leaves split into
 * trivial / easy / hard leaves, and the second partial sum P2.  The hard
 * special leaves are resolved by a segmented sieve held in GPU shared memory
 * (the main sieve of Section 3), whose per-segment counts are stitched
 * together by a device-wide carry scan (the tallies of Section 3).
 *
 * Conventions shared by every call:
 *   - Arithmetic is exact integer arithmetic.  Results never depend on the
 *     tuning parameters (segment size, alpha, c): Section 5 uses exactly this
 *     invariance as a check.
 *   - x/n means floor(x/n).  iroot3 and isqrt are exact integer roots.
 *   - x must satisfy x < 2^63, else PC_ERANGE.
 *   - Host pointers are caller-owned and are written only on success.
 *   - A context is not thread-safe: use one context per host thread.
 *   - Every function returns PC_OK (0) or a negative PC_E* code; the message
 *     of the last failure is available from pc_last_error().
 *   - All GPU work of a context runs on one CUDA stream (pc_set_stream), and
 *     each call synchronizes that stream before it returns.
 */
#ifndef PICOUNT_H
#define PICOUNT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define PC_OK 0
#define PC_EINVAL (-1)    /* argument outside its documented domain */
#define PC_ERANGE (-2)    /* x >= 2^63 */
#define PC_ENOMEM (-3)    /* device or host allocation failed */
#define PC_ECUDA (-4)     /* a CUDA call failed (message in pc_last_error) */
#define PC_ETIMEOUT (-5)  /* a bounded device-side wait gave up */
#define PC_EOVERFLOW (-6) /* an intermediate exceeded its integer width */

/* Signed 128-bit integer, two's complement: value = hi * 2^64 + (uint64_t)lo. */
typedef struct pc_i128 {
    int64_t lo;
    int64_t hi;
} pc_i128;

/* Tuning parameters; zero selects the built-in default of each field.
 * None of them changes any result. */
typedef struct pc_params {
    uint32_t seg_bytes;   /* bytes of shared-memory bitset per sieve segment:
                             1024, 2048, or a multiple of 4096 up to 131072;
                             one byte holds 30 consecutive integers (mod-30
                             wheel) */
    uint32_t ctas_per_sm; /* resident sieve CTAs per SM (1..4) */
    uint32_t threads;     /* reserved (the sieve uses one warp per warp_bytes) */
    uint32_t alpha;       /* default alpha of pc_pi_count (y = alpha*iroot3(x)) */
    uint32_t c;           /* default wheel depth c of pc_pi_count (0..7) */
    uint32_t warp_bytes;  /* bytes of a segment each warp of the hard-leaf sieve
                             owns: 1024, 2048, 4096 or 8192, and at most 16
                             warps per segment */
    uint32_t streams;     /* concurrent query slots of pc_pi_count_batch and of
                             the server (1..64): each slot is one host thread
                             with its own CUDA stream and scratch; default 8 */
    uint32_t pi_gather;   /* how the easy leaves read pi(u): 0 = the popcount pi
                             table (one 16-byte record per 240 integers, the
                             default); 1 = the sampled table of Section 2.1
                             (pi at every floor(log2 y)-th integer, then a walk
                             along the primes) */
    uint32_t m_source;    /* how the list of squarefree m <= y (lpf > p_c, with
                             lpf, mu and gpf) is built: 0 = a sieve of least and
                             greatest prime factors per integer (the default);
                             1 = the nested loops of Section 2.2 over products of
                             distinct primes, mu = (-1)^(number of primes), with
                             no per-integer table.  Both give the same list. */
    uint32_t batch_launch; /* how pc_pi_count_batch runs its one schedule: 0 = the
                             device work of every phase captured into one CUDA
                             graph and launched once (the default); 1 = the same
                             kernels launched one by one */
    uint32_t p2_bucket;   /* the P2 sieve of pc_pi_count / pc_p2: 0 = every segment
                             visits every sieving prime (the default); 1 = the
                             bucket sieve of Section 2.3: segments of seg_bytes
                             (default 4096 = 2^15 bits) taken in waves, and each
                             prime p > seg_bytes (at most one multiple per residue
                             class in a segment) visits only the segments holding
                             its multiples, filed in per-segment buckets before
                             each wave.  Same results.  The batch keeps the
                             default. */
} pc_params;

/* Counters and phase times of the last successful call. */
typedef struct pc_stats {
    uint64_t x, y, z;       /* argument, y, z = x / y */
    uint64_t a;             /* pi(y) (or the a of pc_phi) */
    uint64_t B;             /* pi(isqrt(z)): sieving primes of the hard-leaf sieve */
    uint32_t c;
    uint32_t seg_bytes;
    uint64_t segments;      /* hard-leaf sieve segments */
    uint64_t steps;         /* (segment, prime) steps of the hard-leaf sieve */
    uint64_t hard_leaves;   /* hard special leaves resolved by the sieve */
    uint64_t clears;        /* multiples crossed off by the hard-leaf sieve */
    uint64_t work_items;    /* sieve work items (segments, heavy ones split into replicas) */
    uint64_t item_steps;    /* (work item, prime) steps the work items own: every (segment,
                               prime) step once, heavy segments split among replicas */
    uint64_t kernel_launches;
    double ms_tables, ms_s1, ms_trivial, ms_easy, ms_hard, ms_p2, ms_total;
    double ms_hard_sieve;   /* the segmented sieve kernel alone (CUDA events) */
    uint64_t warp_steps;      /* (warp sub-range, prime) steps with work in the hard-leaf sieve */
    uint64_t leaf_warp_steps; /* of which resolved leaves */
    double ms_easy_kernel;    /* the easy-leaf kernel alone (CUDA events) */
    double ms_p2_kernel;      /* the P2 sieve kernel alone (CUDA events) */
    uint64_t easy_leaves;     /* easy leaves resolved one at a time */
    uint64_t easy_runs;       /* runs of clustered easy leaves: with the odd-number pi table, the
                                 (b, pi value) pairs taken (one division and one pi lookup each,
                                 empty runs included); otherwise the runs walked */
    uint64_t easy_run_leaves; /* easy leaves those runs cover */
    uint64_t p2_clears;       /* multiples crossed off by the P2 sieve */
    uint64_t presieve_steps;  /* hard-leaf sieve: steps that replicas of heavy segments cross
                                 off, with no counts, before the steps they own */
    uint64_t graph_launches;  /* pc_pi_count_batch: CUDA graphs launched (the schedule's
                                 kernels, counted in kernel_launches, are its nodes) */
    uint64_t graph_nodes;     /* nodes of that graph (kernels and memsets) */
} pc_stats;

typedef struct pc_ctx pc_ctx;

/* Create a context on CUDA device `device`.  p may be NULL (defaults).
 * The context owns its device tables and scratch; it allocates device memory
 * lazily, on the first call that needs it.  On success *out is set. */
int pc_create(pc_ctx** out, int device, const pc_params* p);

/* Free every device and host resource of ctx.  NULL is accepted. */
void pc_destroy(pc_ctx* ctx);

/* Use CUDA stream `stream` (a cudaStream_t, NULL = the context's own stream)
 * for all later work of ctx. */
int pc_set_stream(pc_ctx* ctx, void* stream);

/* pi(x): pi(x) = phi(x, a) + a - 1 - P2(x, a) with a = pi(y),
 * y = min(alpha * iroot3(x), isqrt(x)) (Section 2: y_max = alpha x^(1/3)).
 * alpha = 0 selects the built-in choice.  pi(0) = pi(1) = 0. */
int pc_pi_count(pc_ctx* ctx, uint64_t x, uint32_t alpha, uint64_t* out_pi);

/* phi(x, a) (Section 3 definition).  phi(x, 0) = x, phi(0, a) = 0;
 * a >= pi(isqrt x) uses phi = max(1, pi(x) - a + 1) for x >= 1 (the
 * Legendre case of Section 4); otherwise the combinatorial tree truncated
 * at p_a.  a may be any value; out_phi receives the exact count. */
int pc_phi(pc_ctx* ctx, uint64_t x, uint64_t a, uint64_t* out_phi);

/* S2_hard(x, y, c): the sum of -mu(m) * phi(x / (p_b m), b - 1) over the hard
 * special leaves (b, m): c < b <= pi(y), m squarefree, lpf(m) > p_b,
 * y / p_b < m <= y, and u = x / (p_b m) >= min(p_b^2, y).  These are the
 * leaves that need the main sieve of Section 3.
 * Requires iroot3(x) <= y <= isqrt(x) and 0 <= c <= min(7, pi(y)), else
 * PC_EINVAL.  *out receives the exact signed 128-bit sum. */
int pc_s2_hard(pc_ctx* ctx, uint64_t x, uint64_t y, uint32_t c, pc_i128* out);

/* Shard k of n of S2_hard(x, y, c): the hard special leaves whose u falls in
 * the k-th of n equal runs of sieve segments, plus (k = 0 only) the
 * closed-form leaves with b <= 3.  The n shards are independent -- no shard
 * needs another's counts -- because each starts its carries from the
 * starting values phi(L - 1, b) of Section 4 (pc_phi_starts), and their sum
 * is exactly pc_s2_hard(x, y, c).  Same domain as pc_s2_hard; 0 <= k < n. */
int pc_s2_hard_shard(pc_ctx* ctx, uint64_t x, uint64_t y, uint32_t c, uint32_t k, uint32_t n, pc_i128* out);

/* Starting values of Section 4: out[b - c] = phi(m, b) for every
 * c <= b <= b_max, from phi(m, c) and the recurrence (4.1), the subtracted
 * terms phi(m / p_b, b - 1) taken as 0, 1, Legendre's pi(m / p_b) - b + 2
 * (when m / p_b < p_b^2) or a phi computation, as the paper's case split
 * prescribes.  c <= 7; out has b_max - c + 1 entries. */
int pc_phi_starts(pc_ctx* ctx, uint64_t m, uint32_t c, uint64_t b_max, uint64_t* out);

/* P2(x, a) with a = pi(y): sum over primes y < p <= isqrt(x) of
 * (pi(x / p) - pi(p) + 1).  Requires iroot3(x) <= y <= isqrt(x).
 * The value fits in uint64_t for x < 2^63. */
int pc_p2(pc_ctx* ctx, uint64_t x, uint64_t y, uint64_t* out);

/* The five parts of phi(x, a) = S1 + S2_triv + S2_easy + S2_hard and P2(x, a)
 * for a given (x, y, c, a): out[0] = S1 (ordinary leaves), out[1] = trivial,
 * out[2] = easy, out[3] = hard special leaves, out[4] = P2.  a = 0 selects
 * a = pi(y); otherwise 1 <= a <= pi(y), c <= a, and the tree is truncated at
 * p_a.  Requires 1 <= y <= isqrt(x) and c <= 7. */
int pc_leaf_sums(pc_ctx* ctx, uint64_t x, uint64_t y, uint32_t c, uint64_t a, pc_i128 out[5]);

/* pi(x_i) for n queries of arbitrary, mixed sizes (the batched pattern built
 * on Sections 2-4; the paper runs one query at a time).  With stream == NULL,
 * xs and out are host arrays; otherwise they are device arrays, read and
 * written in order on that stream.  The tables (pi table, primes, m-list)
 * are built once for the whole batch and shared read-only by every query;
 * the queries, largest first, are drained by `streams` slots (pc_params),
 * each a host thread with its own CUDA stream and scratch, so that the
 * kernels of different queries overlap on the GPU.  When at least 64 queries
 * have x < 2^32, the pi table is extended to the largest of them (at most
 * 286 MB) and those queries are answered by one lookup kernel.  Every result
 * equals pc_pi_count(x_i, 0).  out is written only if every query succeeded;
 * otherwise the first failure's code is returned. */
int pc_pi_count_batch(pc_ctx* ctx, const uint64_t* xs, size_t n, uint64_t* out, void* stream);

/* Autotuner for pi(x) queries with alpha = 0 (the built-in choice): for every
 * decade of x in [x_lo, x_hi], times pi(3 * 10^(d-1)) for alphas around the
 * built-in one (alpha/2 .. 2 alpha) and hard-leaf segments of 16, 32 and
 * 64 KiB, `reps` timed runs each (0 = 2), and keeps the fastest pair for that
 * decade in ctx; pc_pi_count(x, 0), the batch and the server then use it.
 * A fixed pc_params alpha or seg_bytes is kept fixed.  No result depends on
 * the choice (every candidate's pi is compared; a mismatch is PC_EOVERFLOW).
 * The paper tunes alpha by hand (Section 5, y_max = alpha x^(1/3)). */
int pc_autotune(pc_ctx* ctx, uint64_t x_lo, uint64_t x_hi, uint32_t reps);
/* The alpha and segment bytes pc_pi_count(x, 0) uses now. */
int pc_tuned(pc_ctx* ctx, uint64_t x, uint32_t* alpha, uint32_t* seg_bytes);

/* Autotuner of the batched schedule (pc_pi_count_batch): its one hard-leaf sieve
 * launch over every query's segments shares one segment size and residency, which
 * the per-decade tuning of pc_autotune cannot pick, and the alphas that suit single
 * queries need not suit the batch's throughput.  Runs the batch xs[0..n) with the
 * alphas of pc_autotune or the built-in ones, and hard-leaf segments of 16 KiB (as
 * many resident CTAs per SM as fit, or 8) or 32 KiB (as many as fit), reps + 1
 * times each (the first untimed; reps 0 = 1), and keeps the fastest in ctx for
 * later batches.  Every candidate's results must agree (else PC_EOVERFLOW and the
 * defaults).  A fixed pc_params alpha, seg_bytes or ctas_per_sm is kept fixed.  The paper schedules blocks dynamically by their
 * measured run times (Section 3); here the geometry is measured, the schedule
 * planned on the device. */
int pc_autotune_batch(pc_ctx* ctx, const uint64_t* xs, size_t n, uint32_t reps);
/* The batched schedule's choice now: segment bytes, resident CTAs per SM (0 = as
 * many as fit), and 1 if it uses the built-in alphas (0: pc_autotune's). */
int pc_tuned_batch(pc_ctx* ctx, uint32_t* seg_bytes, uint32_t* ctas_per_sm, uint32_t* builtin_alpha);

/* ---------------------------------------------------------------------------
 * Served queries: continuous batching over the context's tables.
 *
 * A server admits pi(x) and phi(x, a) requests as they arrive.  A request
 * starts as soon as a slot is free (pc_params.streams slots) and its device
 * scratch estimate (pc_server_footprint) fits, with those of the requests
 * already running, in mem_budget bytes.  The waiting requests form one queue:
 * in arrival order (PC_SERVE_FIFO), or by x, smallest first, arrival order
 * among equal x (PC_SERVE_SMALL_FIRST: lower median latency under overload;
 * a large request waits while smaller ones keep arriving).  Only the head of
 * the queue may start.
 * Requests in different slots run concurrently on the GPU, each on its own
 * stream.  Tables for every x <= x_max and a <= a_max are built when the
 * server is created and stay resident until it is destroyed; a request
 * outside those bounds is rejected at submission (PC_EINVAL), one whose
 * estimate alone exceeds the budget with PC_ENOMEM.  Results are the exact
 * values pc_pi_count(x, 0) / pc_phi(x, a) return.  The paper has no
 * counterpart: it is a serving layer over the method. */
typedef struct pc_server pc_server;

#define PC_SERVE_FIFO 0
#define PC_SERVE_SMALL_FIRST 1

#define PC_QUERY_PI 0   /* value = pi(x) */
#define PC_QUERY_PHI 1  /* value = phi(x, a) */

typedef struct pc_result {
    uint64_t tag;         /* the caller's tag from pc_server_submit */
    uint64_t x, a;        /* the request (a = 0 for pi) */
    uint64_t value;       /* the result, valid when status == PC_OK */
    int32_t kind;         /* PC_QUERY_PI or PC_QUERY_PHI */
    int32_t status;       /* PC_OK or the failure's code */
    double t_submit_ms;   /* times since the server was created */
    double t_start_ms;
    double t_done_ms;
} pc_result;

typedef struct pc_server_stats {
    uint64_t submitted, completed, failed;
    uint64_t max_running;      /* most requests ever running at once */
    uint64_t max_bytes;        /* largest sum of running footprints */
    uint64_t mem_budget;
} pc_server_stats;

/* Start a server on ctx (which it uses exclusively until pc_server_destroy).
 * mem_budget = 0 selects half of the device memory free at creation. */
int pc_server_create(pc_ctx* ctx, uint64_t x_max, uint64_t a_max, uint64_t mem_budget, uint32_t policy,
                     pc_server** out);
/* Queue one request; returns at once.  kind is PC_QUERY_PI or PC_QUERY_PHI. */
int pc_server_submit(pc_server* s, int kind, uint64_t x, uint64_t a, uint64_t tag);
/* Move up to max finished results into out (completion order); waits up to
 * timeout_ms (< 0: until one is ready or nothing is pending) when none is
 * ready yet.  *n_out receives the number written. */
int pc_server_poll(pc_server* s, pc_result* out, size_t max, int timeout_ms, size_t* n_out);
int pc_server_get_stats(pc_server* s, pc_server_stats* out);
/* Device scratch estimate (bytes) the server charges a request against the budget. */
uint64_t pc_server_footprint(pc_server* s, int kind, uint64_t x, uint64_t a);
/* Finish every queued request, stop the slots and free the server (results
 * not yet polled are dropped).  NULL is accepted. */
void pc_server_destroy(pc_server* s);

/* ---------------------------------------------------------------------------
 * P2 for callers that cannot allocate device memory.
 *
 * The paper has no counterpart to this entry point; it exists for library
 * users, not for the method.  Some callers must not call cudaMalloc: a serving
 * process whose device memory is carved up in advance by its own pool
 * allocator (an allocation outside the pool could exceed the budget), or a
 * latency-critical path that cannot afford the device-wide synchronization a
 * cudaMalloc or cudaFree may trigger.  pc_p2_noalloc allocates nothing and
 * needs no context: the caller passes the inputs and the output as device
 * memory it already owns, and the per-segment scratch lives in one fixed
 * array inside the library (PC_NOALLOC_MAX_SEGMENTS * 16 bytes + 256 bytes,
 * 512 KiB), which every GPU that loads the library keeps until the process
 * exits.
 *
 * Computes P2(x, a), a = pi(y), as pc_p2 does:
 *   x, y       iroot3(x) <= y <= isqrt(x), x < 2^63 (PC_ERANGE otherwise);
 *   primes     device array of the primes 2, 3, 5, ... in ascending order,
 *              n_primes entries, every prime <= isqrt(x); the last entry
 *              must be >= isqrt(x) (then the array provably covers isqrt(x));
 *   out        device uint64_t that receives P2; it receives UINT64_MAX if
 *              the last entry of primes is below isqrt(x);
 *   stream     cudaStream_t (NULL = legacy default stream) of the current
 *              device.
 * The work is enqueued on `stream` and the call returns without waiting; *out
 * is valid once the stream reaches that point.  Size limit: z = x / y must
 * give z / PC_NOALLOC_SEG_SPAN + 1 <= PC_NOALLOC_MAX_SEGMENTS segments
 * (z < 3.2e10) and z >= 25; larger or smaller problems return PC_EINVAL and
 * leave *out untouched.  The first call on a device looks up the scratch
 * array's device address once (cudaGetSymbolAddress); make that first call
 * before any stream capture begins.  All calls on a device share the one
 * scratch array: calls that overlap on the GPU (concurrent streams, or host
 * threads racing) race on it and give wrong results -- order them on one
 * stream.  Each call clears the part of the scratch that must start at zero.
 */
#define PC_NOALLOC_MAX_SEGMENTS 32768
#define PC_NOALLOC_SEG_SPAN 983040   /* integers per segment (32 KiB, mod-30 wheel) */
int pc_p2_noalloc(uint64_t x, uint64_t y, const uint32_t* primes, uint64_t n_primes, uint64_t* out, void* stream);

/* The resident CTAs per SM of the hard-leaf sieve that pi(x) calls use for x's decade:
 * the autotuned value (pc_autotune tries the most that fit, 2, 4 and 6 after choosing alpha
 * and the segment size), else 0 = as many as registers and shared memory allow (or the
 * context's ctas_per_sm when set). */
int pc_tuned_ctas(pc_ctx* ctx, uint64_t x, uint32_t* ctas_per_sm);

/* Counters of the last successful call. */
int pc_last_stats(pc_ctx* ctx, pc_stats* out);

/* Static description of an error code. */
const char* pc_strerror(int code);

/* Message of the last failure on ctx ("" if none). */
const char* pc_last_error(pc_ctx* ctx);

/* Library version string. */
const char* pc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PICOUNT_H */
