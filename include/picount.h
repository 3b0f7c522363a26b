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
 * (the "main sieve" of Section 3), whose per-segment counts are stitched
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
    uint32_t reserved[2];
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
    uint64_t item_steps;    /* (work item, prime) steps actually run, replicas included */
    uint64_t kernel_launches;
    double ms_tables, ms_s1, ms_trivial, ms_easy, ms_hard, ms_p2, ms_total;
    double ms_hard_sieve;   /* the segmented sieve kernel alone (CUDA events) */
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

/* pi(x_i) for n queries.  With stream == NULL, xs and out are host arrays;
 * otherwise they are device arrays and the call runs on that stream.  Tables
 * are built once for the largest query and shared by all of them. */
int pc_pi_count_batch(pc_ctx* ctx, const uint64_t* xs, size_t n, uint64_t* out, void* stream);

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
 *              n_primes entries: every prime <= isqrt(x) and at least one
 *              prime above it (so the array provably covers isqrt(x));
 *   out        device uint64_t that receives P2; it receives UINT64_MAX if
 *              the last entry of primes is not above isqrt(x);
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
