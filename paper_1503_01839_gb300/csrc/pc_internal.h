// pc_internal.h -- host-side declarations shared by the library's .cu files.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <vector>
#include <cuda_runtime.h>

#include "picount.h"
#include "pc_common.cuh"

// ------------------------------------------------------------------ errors
// Every CUDA call goes through PC_CUDA; on failure the enclosing function
// returns PC_ECUDA after recording the message in the context.
void pc_set_error(pc_ctx* ctx, const char* fmt, ...);

#define PC_CUDA(ctx, call)                                                     \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            pc_set_error((ctx), "%s failed: %s (%s:%d)", #call,                \
                         cudaGetErrorString(e_), __FILE__, __LINE__);          \
            return PC_ECUDA;                                                   \
        }                                                                      \
    } while (0)

#define PC_TRY(expr)                                                           \
    do {                                                                       \
        int r_ = (expr);                                                       \
        if (r_ != PC_OK) return r_;                                            \
    } while (0)

// Launch check: a launch error (bad configuration) is reported at once.
#define PC_LAUNCHED(ctx) PC_CUDA(ctx, cudaGetLastError())

// --------------------------------------------------------------- buffers
// Grow-only device buffer owned by the context.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    template <class T> T* as() const { return (T*)p; }
};

int buf_reserve(pc_ctx* ctx, DevBuf& b, size_t bytes);
void buf_free(DevBuf& b);

// ----------------------------------------------------------------- tables
struct Tables {
    // primes <= 65536 (bootstrap), u32, ascending, 0-based
    DevBuf small_primes;
    u32 n_small = 0;
    // pi table over [0, pi_limit]
    u64 pi_limit = 0;
    DevBuf pi_rec;   // PiRec per 240 numbers
    // primes[1..nprimes] (u32), primes[0] = 1, primes[nprimes+1] = next prime
    u64 prime_limit = 0;
    u64 nprimes = 0;
    DevBuf primes;
    DevBuf primes_rcp;   // floor((2^64 - 1) / p_k), same indexing as primes
    DevBuf primes_dv;    // p_k | floor((2^(32+s) - 1) / p_k) << 32, s = floor(log2 p_k) (div_dv)
    // squarefree m-list over [2, ml_limit] with lpf > p_cmin
    u64 ml_limit = 0;
    u32 ml_cmin = 99;
    u64 ml_n = 0;
    DevBuf ml_m, ml_info, ml_gpf, ml_rcp, rank_bits, rank_cnt;
    // sub-lists of the m-list: entries with lpf index > sl_K[k] (ascending K), so
    // that the leaves of a prime p_b with b >= K need not skip entries with lpf <= p_K
    static constexpr int NSUB = 4;
    DevBuf sl_m[NSUB], sl_info[NSUB], sl_gpf[NSUB], sl_rcp[NSUB], sl_bits[NSUB], sl_cnt[NSUB];
    u32 sl_K[NSUB] = {0, 0, 0, 0};
    u64 sl_n[NSUB] = {0, 0, 0, 0};
    u32 n_sl = 0;
    // sampled pi table (Section 2.1): samp[j] = pi(j * samp_s), covering every v <= samp_limit
    DevBuf samp;
    u32 samp_s = 0;
    u64 samp_limit = 0;
    // presieve pattern of the primes 7, 11, 13, 17, 19 (WHEEL19_PERIOD bytes of the mod-30
    // bitset, then a copy of its start so that any 128 KiB slice is contiguous)
    DevBuf wheel19;
    // odd-number pi table over [0, podd_limit] (pi_odd): one uint2 per 64 integers
    DevBuf pi_odd;
    u64 podd_limit = 0;
    // phi(., c) residue tables for the primorial of c (c = 0..7)
    DevBuf phiT[8];
    bool phiT_ok[8] = {false, false, false, false, false, false, false, false};

    PiTable pi() const { return PiTable{pi_rec.as<PiRec>(), pi_limit}; }
    RankTable rank() const { return RankTable{rank_bits.as<u64>(), rank_cnt.as<u32>(), ml_limit}; }
    MList mlist() const
    {
        return MList{ml_m.as<u32>(), ml_info.as<u32>(), ml_gpf.as<u32>(), ml_rcp.as<u64>(), ml_n, ml_limit, ml_cmin};
    }
    MList sublist(int k) const
    {
        return MList{sl_m[k].as<u32>(), sl_info[k].as<u32>(), sl_gpf[k].as<u32>(), sl_rcp[k].as<u64>(), sl_n[k],
                     ml_limit, sl_K[k]};
    }
    RankTable subrank(int k) const { return RankTable{sl_bits[k].as<u64>(), sl_cnt[k].as<u32>(), ml_limit}; }
};

// ---------------------------------------------------------------- context
struct pc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;   // stream every kernel of this context uses
    cudaStream_t own_stream = nullptr;
    pc_params params{};
    int sm_count = 0;
    size_t smem_optin = 0;
    Tables T;
    // scratch (grow-only)
    DevBuf seg_b, seg_off, counts, tallies, acc_seg, partials, result, misc, scan_tmp, queue;
    DevBuf easy_rng, easy_chunk_off, easy_cmap, starts;
    DevBuf mq_q, mq_pref, mq_e, mq_h, mq_hq, mq_p;   // batched queries (pc_pi_count_batch)
    DevBuf p2_bkt;   // P2 bucket sieve: the buckets of one wave of segments and their fill counts
    // pinned host staging for small results
    void* host_stage = nullptr;
    pc_stats stats{};
    char errmsg[512] = {0};
    cudaEvent_t ev[16];
    bool ev_ok = false;
    // A worker context borrows the tables of its parent (shallow copy of T):
    // it never grows or frees them.  Batched and served queries run on
    // workers, one host thread and one stream each, so that their kernels
    // overlap on the device.
    bool borrowed = false;
    std::vector<pc_ctx*> workers;
    // autotuned alpha and segment bytes per decimal digit count of x (0 = not tuned)
    u32 tuned_alpha[21] = {0};
    u32 tuned_seg[21] = {0};
    u32 seg_call = 0;   // segment bytes chosen for the running pi(x) call (0 = default)
    u32 tuned_ctas[21] = {0};   // autotuned resident CTAs per SM of the hard-leaf sieve (0 = most)
    u32 ctas_call = 0;          // the value for the running call
    // device counters of the running call (easy leaves, runs, their leaves, P2 crossings),
    // beside the result slots; null outside a leaf-sum call
    unsigned long long* dstat = nullptr;
    bool easy_timed = false, p2_timed = false;   // ev[2..3] / ev[4..5] hold kernel times
    // How the batched phases (mq_*) run: MQ_DIRECT launches as it goes; MQ_PREPARE reserves
    // scratch, uploads the arrays built on the host and reads back table values, with no
    // device work; MQ_CAPTURE then enqueues only device work (kernels, memsets), into a
    // CUDA graph, and must not grow any scratch
    int mq_mode = 0;
    u64 mq_p2_pv[2] = {0, 0};   // pi values mq_p2 needs, read in the prepare pass
    // hard-leaf sieve geometry of the batched schedule (pc_autotune_batch; 0 = default:
    // 16 KiB segments, as many resident CTAs per SM as fit)
    u32 batch_seg = 0, batch_ctas = 0;
    bool batch_builtin_alpha = false;   // the batch uses the built-in alphas, not pc_autotune's
    void* mq_hard_kern = nullptr;   // the batched sieve's instantiation and resident CTAs per SM,
    int mq_hard_per_sm = 0;         // chosen (and its shared-memory limit set) before any capture
};

enum { MQ_DIRECT = 0, MQ_PREPARE = 1, MQ_CAPTURE = 2 };
inline bool mq_device_work(const pc_ctx* c) { return c->mq_mode != MQ_PREPARE; }
inline bool mq_host_upload(const pc_ctx* c) { return c->mq_mode != MQ_CAPTURE; }

u32 default_alpha(u64 x);
int decimal_digits(u64 x);
u32 choose_alpha(const pc_ctx* ctx, u64 x);

// Worker contexts of ctx (created on first use, tables refreshed from ctx).
int workers_ensure(pc_ctx* ctx, int n);
void workers_destroy(pc_ctx* ctx);
// Build every table that queries up to x_max (pi(x) with the built-in alpha,
// and phi(x, a) for a <= a_max) need, so that workers never grow them.
int tables_for_queries(pc_ctx* ctx, const u64* xs, size_t n, u64 a_max);
int pi_count_impl(pc_ctx* ctx, u64 x, u32 alpha, u64* out);
int phi_impl(pc_ctx* ctx, u64 x, u64 a, u64* out);

// ------------------------------------------------------------------- util
// out[i] = sum_{j<i} in[j] for i < n, and out[n] = total (out has n+1 slots).
int scan_exclusive_u32_to_u32(pc_ctx* ctx, const u32* in, u32* out, u64 n);
int scan_exclusive_u32_to_u64(pc_ctx* ctx, const u32* in, u64* out, u64 n);
// *out = sum of n i128 values
int reduce_i128(pc_ctx* ctx, const I128Pair* in, u64 n, I128Pair* out);
int copy_to_host(pc_ctx* ctx, void* dst, const void* src, size_t bytes);  // synchronizes

// ----------------------------------------------------------------- tables
// Make sure tables cover pi lookups up to pi_limit, primes up to
// prime_limit (plus one sentinel prime), and the m-list up to ml_limit with
// lpf(m) > p_cmin.
int tables_ensure(pc_ctx* ctx, u64 pi_limit, u64 prime_limit, u64 ml_limit, u32 cmin);
// the presieve pattern of the primes 7..19 (Tables::wheel19), built once by a context that
// owns its tables (tables_ensure does); a no-op for one that borrows them
static constexpr u32 WHEEL19_PERIOD = 7u * 11u * 13u * 17u * 19u;   // bytes (30 integers each)
int tables_wheel19(pc_ctx* ctx);
int tables_phi_c(pc_ctx* ctx, u32 c);   // phi(., c) residue table
// values of pi(v) for a handful of v (v <= pi_limit), synchronizing
int tables_pi_values(pc_ctx* ctx, const u64* v, u64* out, int n);
// pi(v) for any number of v (every v <= the table limit), synchronizing
int tables_pi_many(pc_ctx* ctx, const u64* v, u64* out, size_t n);

// ----------------------------------------------------------------- leaves
struct LeafProblem {
    u64 x, y, z;
    u32 c;        // ordinary-leaf wheel depth
    u64 a;        // leaves use primes p_b with c < b <= a
    bool trunc;   // a < pi(y): filter gpf(m) <= p_a
    u64 piy;      // pi(y)
    u64 B;        // pi(isqrt z)
    // hard-leaf sieve over segments [shard_k * nseg / shard_n, (shard_k + 1) * nseg / shard_n) only
    // (shard_n = 0: all of them); the leaves' carries then start from phi(L - 1, b)
    u32 shard_k = 0, shard_n = 0;
};

// phi(m, b) for every c <= b <= b_max (Section 4 starting values): out[b - c]
int phi_starts(pc_ctx* ctx, u64 m, u32 c, u64 b_max, u64* out);
// segments of the hard-leaf sieve for (x, z) in the context's geometry
u64 hard_segments(pc_ctx* ctx, u64 z);

// Each adds its sum to *out (device I128Pair) -- out must be zeroed first.
int run_s1(pc_ctx* ctx, const LeafProblem& P, I128Pair* out);
int run_trivial(pc_ctx* ctx, const LeafProblem& P, I128Pair* out);
int run_easy(pc_ctx* ctx, const LeafProblem& P, I128Pair* out);
int run_hard_smallb(pc_ctx* ctx, const LeafProblem& P, I128Pair* out);
int run_hard_sieve(pc_ctx* ctx, const LeafProblem& P, I128Pair* out);
int run_p2(pc_ctx* ctx, u64 x, u64 y, u64 a, I128Pair* out);

// ------------------------------------------------------- batched queries
// One pi(x) query of a batched launch (pc_pi_count_batch): its parameters, and the
// table values the batch reads back once for all queries.
struct MQ {
    u64 x, y, z;
    u64 a;      // pi(y)
    u64 B;      // pi(isqrt z)
    u64 K;      // pi(isqrt x)
    u64 nlim;   // m-list entries with m <= y
    u64 E;      // pi(iroot3 x): the easy leaves have b <= E
    u32 c;
    u32 pad;
};

// The parts of every query of a batch, [q][0..4] = S1, trivial, easy, hard, P2, summed
// exactly by atomic_add_i128 (any order).
struct MQPlan {
    u32 Q = 0;
    const MQ* dq = nullptr;      // device copy of hq
    I128Pair* parts = nullptr;   // device, Q x 5
    std::vector<MQ> hq;
};

__device__ __forceinline__ void mq_atomic_add_i128(I128Pair* p, i128 v)
{
    // the low words add with wrap-around; every addition sends its own carry to the high word
    const unsigned long long lo = (unsigned long long)(u64)v;
    const unsigned long long old = atomicAdd((unsigned long long*)&p->lo, lo);
    const u64 carry = old + lo < old ? 1u : 0u;
    atomicAdd((unsigned long long*)&p->hi, (unsigned long long)((u64)(i64)(v >> 64) + carry));
}

// the last index k < n with pref[k] <= v (pref ascending, pref[0] <= v)
__device__ __forceinline__ u64 mq_find(const u64* pref, u64 n, u64 v)
{
    u64 lo = 0, hi = n;
    while (hi - lo > 1) {
        const u64 mid = (lo + hi) >> 1;
        if (pref[mid] <= v) lo = mid; else hi = mid;
    }
    return lo;
}

int mq_info(pc_ctx* ctx, MQPlan& P);          // fills a, B, K, nlim, E (one read-back for the batch)
int mq_s1_trivial(pc_ctx* ctx, const MQPlan& P);
int mq_easy(pc_ctx* ctx, const MQPlan& P);
int mq_hard(pc_ctx* ctx, const MQPlan& P);
int mq_p2(pc_ctx* ctx, const MQPlan& P);

// segment geometry shared by the sieve kernels
struct SegGeom {
    u32 seg_bytes;   // bytes per segment (multiple of 128)
    u64 span;        // numbers per segment = 30 * seg_bytes
    u64 nseg;
    int threads;
    int ctas;
    size_t smem;
};

// segment bytes: the context's fixed size, else the tuned one of the call, else dflt
u32 pc_seg_bytes(pc_ctx* ctx, u32 dflt);
