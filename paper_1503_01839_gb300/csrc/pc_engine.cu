// pc_engine.cu -- context, orchestration and the C ABI of picount.h.
//
// pi(x) = S1 + S2_triv + S2_easy + S2_hard + a - 1 - P2(x, a),  a = pi(y),
// y = min(alpha * iroot3(x), isqrt(x)) (Section 2: y_max = alpha x^(1/3));
// with y >= x^(1/3) the third partial sum P3 vanishes.  Every part is an
// exact integer computed on the GPU; the host adds the five i128 parts and a - 1.
// (The host also picks y, z and the launch sizes, and reads back the handful of
// table values, such as pi(y), that size them.)
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "pc_internal.h"


static const char* kVersion = "picount-gb300 0.1 (sm_103a)";

static i128 from_pair(const I128Pair& p) { return ((i128)p.hi << 64) | (i128)(u64)p.lo; }

static pc_i128 to_pc(i128 v)
{
    pc_i128 r;
    r.lo = (int64_t)(u64)v;
    r.hi = (int64_t)(v >> 64);
    return r;
}

struct Timer {
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double ms() const
    {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

// -------------------------------------------------------------- context
extern "C" int pc_create(pc_ctx** out, int device, const pc_params* p)
{
    if (!out) return PC_EINVAL;
    pc_ctx* ctx = new (std::nothrow) pc_ctx();
    if (!ctx) return PC_ENOMEM;
    ctx->device = device;
    if (p) ctx->params = *p;
    const uint32_t sb = ctx->params.seg_bytes;
    const uint32_t wb = ctx->params.warp_bytes;
    if (ctx->params.c > 7 || (sb && sb != 1024 && sb != 2048 && (sb % 4096 || sb > 131072)) ||
        (wb && wb != 1024 && wb != 2048 && wb != 4096 && wb != 8192) ||
        ctx->params.ctas_per_sm > 4 || ctx->params.pi_gather > 1 || ctx->params.m_source > 1 || ctx->params.batch_launch > 1 || ctx->params.p2_bucket > 1 ||
        (ctx->params.threads && (ctx->params.threads % 32 || ctx->params.threads < 128 || ctx->params.threads > 1024))) {
        delete ctx;
        return PC_EINVAL;
    }
    cudaError_t e = cudaSetDevice(device);
    cudaDeviceProp prop;
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->host_stage, 1 << 16);
    if (e == cudaSuccess) {
        for (int i = 0; i < 16 && e == cudaSuccess; i++) e = cudaEventCreate(&ctx->ev[i]);
        ctx->ev_ok = e == cudaSuccess;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return e == cudaErrorMemoryAllocation ? PC_ENOMEM : PC_ECUDA;
    }
    ctx->sm_count = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    ctx->stream = ctx->own_stream;
    *out = ctx;
    return PC_OK;
}

extern "C" void pc_destroy(pc_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    workers_destroy(ctx);
    DevBuf* bufs[] = {&ctx->seg_b, &ctx->seg_off, &ctx->counts, &ctx->tallies,
                      &ctx->acc_seg, &ctx->partials, &ctx->result, &ctx->misc, &ctx->scan_tmp, &ctx->queue,
                      &ctx->easy_rng, &ctx->easy_chunk_off, &ctx->easy_cmap, &ctx->starts,
                      &ctx->mq_q, &ctx->mq_pref, &ctx->mq_e, &ctx->mq_h, &ctx->mq_hq, &ctx->mq_p,
                      &ctx->p2_bkt};
    for (DevBuf* b : bufs) buf_free(*b);
    if (!ctx->borrowed) {
        Tables& T = ctx->T;
        DevBuf* tabs[] = {&T.small_primes, &T.pi_rec, &T.primes, &T.primes_rcp, &T.ml_m, &T.ml_info,
                          &T.ml_gpf, &T.ml_rcp, &T.rank_bits, &T.rank_cnt, &T.samp, &T.primes_dv, &T.pi_odd, &T.wheel19};
        for (DevBuf* b : tabs) buf_free(*b);
        for (int c = 0; c < 8; c++) buf_free(T.phiT[c]);
        for (int k = 0; k < Tables::NSUB; k++) {
            DevBuf* sb[] = {&T.sl_m[k], &T.sl_info[k], &T.sl_gpf[k], &T.sl_rcp[k], &T.sl_bits[k], &T.sl_cnt[k]};
            for (DevBuf* b : sb) buf_free(*b);
        }
    }
    if (ctx->ev_ok)
        for (int i = 0; i < 16; i++) cudaEventDestroy(ctx->ev[i]);
    if (ctx->host_stage) cudaFreeHost(ctx->host_stage);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}

extern "C" int pc_set_stream(pc_ctx* ctx, void* stream)
{
    if (!ctx) return PC_EINVAL;
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    return PC_OK;
}

extern "C" const char* pc_strerror(int code)
{
    switch (code) {
    case PC_OK: return "ok";
    case PC_EINVAL: return "invalid argument";
    case PC_ERANGE: return "x out of range (x must be < 2^63)";
    case PC_ENOMEM: return "out of memory";
    case PC_ECUDA: return "CUDA error";
    case PC_ETIMEOUT: return "device-side wait timed out";
    case PC_EOVERFLOW: return "integer overflow";
    default: return "unknown error";
    }
}

extern "C" const char* pc_last_error(pc_ctx* ctx) { return ctx ? ctx->errmsg : ""; }

extern "C" const char* pc_version(void) { return kVersion; }

extern "C" int pc_last_stats(pc_ctx* ctx, pc_stats* out)
{
    if (!ctx || !out) return PC_EINVAL;
    *out = ctx->stats;
    return PC_OK;
}

// ------------------------------------------------------------ helpers
static void stats_begin(pc_ctx* ctx, u64 x)
{
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.x = x;
}

// Result slots 0..7 hold i128 parts; slots 8..15 (as u64) the call's counters.
static int result_slots(pc_ctx* ctx, int n, I128Pair** d)
{
    (void)n;
    PC_TRY(buf_reserve(ctx, ctx->result, 16 * sizeof(I128Pair)));
    PC_CUDA(ctx, cudaMemsetAsync(ctx->result.p, 0, 16 * sizeof(I128Pair), ctx->stream));
    *d = ctx->result.as<I128Pair>();
    ctx->dstat = (unsigned long long*)(ctx->result.as<I128Pair>() + 8);
    ctx->easy_timed = ctx->p2_timed = false;
    return PC_OK;
}

static int read_slots(pc_ctx* ctx, int n, i128* out)
{
    I128Pair h[16];
    PC_TRY(copy_to_host(ctx, h, ctx->result.p, 16 * sizeof(I128Pair)));
    for (int i = 0; i < n; i++) out[i] = from_pair(h[i]);
    const u64* c = (const u64*)(h + 8);
    ctx->stats.easy_leaves += c[0];
    ctx->stats.easy_runs += c[1];
    ctx->stats.easy_run_leaves += c[2];
    ctx->stats.p2_clears += c[3];
    float ms = 0;
    if (ctx->easy_timed && cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]) == cudaSuccess) ctx->stats.ms_easy_kernel += ms;
    if (ctx->p2_timed && cudaEventElapsedTime(&ms, ctx->ev[4], ctx->ev[5]) == cudaSuccess) ctx->stats.ms_p2_kernel += ms;
    ctx->easy_timed = ctx->p2_timed = false;
    ctx->dstat = nullptr;
    return PC_OK;
}

static int sync_timed(pc_ctx* ctx, double* acc, Timer& t)
{
    PC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *acc += t.ms();
    t = Timer();
    return PC_OK;
}

// p_a by binary search on the pi table (smallest v with pi(v) >= a)
__global__ void nth_prime_kernel(PiTable pit, u64 a, u64 hi, u64* out)
{
    u64 lo = 2;
    while (lo < hi) {
        u64 mid = lo + (hi - lo) / 2;
        if (pi_lookup(pit, mid) >= a) hi = mid; else lo = mid + 1;
    }
    *out = lo;
}

u32 default_alpha(u64 x)
{
    // y = alpha x^(1/3): the hard-leaf sieve and P2 shrink with alpha while the
    // easy leaves grow; values from sweeps of pi(10^n) on GB300
    int d = 0;
    for (u64 t = x; t >= 10; t /= 10) d++;
    if (d <= 8) return 2;
    if (d == 9) return 4;
    if (d <= 11) return 6;
    if (d <= 13) return 16;
    if (d == 14) return 24;
    if (d == 15) return 20;
    if (d == 16) return 32;
    if (d == 17) return 40;
    return 56;
}

int decimal_digits(u64 x)
{
    int d = 1;
    for (u64 t = x; t >= 10; t /= 10) d++;
    return d;
}

// alpha of a query: the context's fixed alpha, else the autotuned one for
// x's decade, else the built-in table
u32 choose_alpha(const pc_ctx* ctx, u64 x)
{
    if (ctx->params.alpha) return ctx->params.alpha;
    const u32 t = ctx->tuned_alpha[decimal_digits(x)];
    return t ? t : default_alpha(x);
}

// segment bytes of the hard-leaf sieve for a query (0 = built-in default)
static u32 choose_seg(const pc_ctx* ctx, u64 x)
{
    if (ctx->params.seg_bytes) return 0;
    return ctx->tuned_seg[decimal_digits(x)];
}

// Leaf decomposition of phi(x, a) and P2(x, a); a == 0 selects pi(y).
// parts: S1, trivial, easy, hard, P2 (P2 only when want_p2).
static int leaf_parts(pc_ctx* ctx, u64 x, u64 y, u32 c, u64 a, bool want_p2, i128 parts[5], u64* a_out)
{
    if (y < 1 || y > pc_isqrt(x) || c > 7) {
        pc_set_error(ctx, "leaf sums need 1 <= y <= isqrt(x) and c <= 7");
        return PC_EINVAL;
    }
    Timer t;
    const u64 z = x / y;
    const u64 r = pc_isqrt(x);
    PC_TRY(tables_ensure(ctx, r > y ? r : y, pc_max(y, pc_isqrt(z)), y, c));
    u64 vals[2] = {y, pc_isqrt(z)}, pv[2];
    PC_TRY(tables_pi_values(ctx, vals, pv, 2));
    const u64 piy = pv[0], B = pv[1];
    if (a == 0) a = piy;
    if (a > piy || c > a) {
        pc_set_error(ctx, "need c <= a <= pi(y) (c=%u, a=%llu, pi(y)=%llu)", c, (unsigned long long)a,
                     (unsigned long long)piy);
        return PC_EINVAL;
    }
    PC_TRY(sync_timed(ctx, &ctx->stats.ms_tables, t));
    LeafProblem P{x, y, z, c, a, a < piy, piy, B};
    ctx->stats.y = y;
    ctx->stats.z = z;
    ctx->stats.a = a;
    ctx->stats.B = B;
    ctx->stats.c = c;
    I128Pair* d;
    PC_TRY(result_slots(ctx, 5, &d));
    PC_TRY(run_s1(ctx, P, d + 0));
    PC_TRY(sync_timed(ctx, &ctx->stats.ms_s1, t));
    PC_TRY(run_trivial(ctx, P, d + 1));
    PC_TRY(sync_timed(ctx, &ctx->stats.ms_trivial, t));
    PC_TRY(run_easy(ctx, P, d + 2));
    PC_TRY(sync_timed(ctx, &ctx->stats.ms_easy, t));
    PC_TRY(run_hard_smallb(ctx, P, d + 3));
    PC_TRY(run_hard_sieve(ctx, P, d + 3));
    PC_TRY(sync_timed(ctx, &ctx->stats.ms_hard, t));
    if (want_p2) {
        PC_TRY(run_p2(ctx, x, y, a, d + 4));
        PC_TRY(sync_timed(ctx, &ctx->stats.ms_p2, t));
    }
    PC_TRY(read_slots(ctx, 5, parts));
    if (!want_p2) parts[4] = 0;
    if (a_out) *a_out = a;
    return PC_OK;
}

// ------------------------------------------------------------- C ABI
extern "C" int pc_leaf_sums(pc_ctx* ctx, uint64_t x, uint64_t y, uint32_t c, uint64_t a, pc_i128 out[5])
{
    if (!ctx || !out) return PC_EINVAL;
    if (x >> 63) return PC_ERANGE;
    PC_CUDA(ctx, cudaSetDevice(ctx->device));
    stats_begin(ctx, x);
    Timer t;
    i128 parts[5];
    PC_TRY(leaf_parts(ctx, x, y, c, a, true, parts, nullptr));
    for (int i = 0; i < 5; i++) out[i] = to_pc(parts[i]);
    ctx->stats.ms_total = t.ms();
    return PC_OK;
}

static int s2_hard_impl(pc_ctx* ctx, uint64_t x, uint64_t y, uint32_t c, u32 shard_k, u32 shard_n, pc_i128* out);

extern "C" int pc_s2_hard(pc_ctx* ctx, uint64_t x, uint64_t y, uint32_t c, pc_i128* out)
{
    return s2_hard_impl(ctx, x, y, c, 0, 0, out);
}

extern "C" int pc_s2_hard_shard(pc_ctx* ctx, uint64_t x, uint64_t y, uint32_t c, uint32_t k, uint32_t n,
                                pc_i128* out)
{
    if (n == 0 || k >= n) return PC_EINVAL;
    return s2_hard_impl(ctx, x, y, c, k, n, out);
}

static int s2_hard_impl(pc_ctx* ctx, uint64_t x, uint64_t y, uint32_t c, u32 shard_k, u32 shard_n, pc_i128* out)
{
    if (!ctx || !out) return PC_EINVAL;
    if (x >> 63) return PC_ERANGE;
    if (x < 1 || y < pc_iroot3(x) || y > pc_isqrt(x) || c > 7) {
        pc_set_error(ctx, "s2_hard needs iroot3(x) <= y <= isqrt(x) and c <= 7");
        return PC_EINVAL;
    }
    PC_CUDA(ctx, cudaSetDevice(ctx->device));
    stats_begin(ctx, x);
    Timer t, ph;
    const u64 z = x / y;
    const u64 r = pc_isqrt(x);
    PC_TRY(tables_ensure(ctx, r > y ? r : y, pc_max(y, pc_isqrt(z)), y, c));
    u64 vals[2] = {y, pc_isqrt(z)}, pv[2];
    PC_TRY(tables_pi_values(ctx, vals, pv, 2));
    const u64 piy = pv[0], B = pv[1];
    if (c > piy) {
        pc_set_error(ctx, "c=%u exceeds pi(y)=%llu", c, (unsigned long long)piy);
        return PC_EINVAL;
    }
    PC_TRY(sync_timed(ctx, &ctx->stats.ms_tables, ph));
    LeafProblem P{x, y, z, c, piy, false, piy, B};
    P.shard_k = shard_k;
    P.shard_n = shard_n;
    ctx->stats.y = y;
    ctx->stats.z = z;
    ctx->stats.a = piy;
    ctx->stats.B = B;
    ctx->stats.c = c;
    I128Pair* d;
    PC_TRY(result_slots(ctx, 1, &d));
    if (shard_n == 0 || shard_k == 0)
        PC_TRY(run_hard_smallb(ctx, P, d));   // closed-form leaves (b <= 3): counted once, in shard 0
    PC_TRY(run_hard_sieve(ctx, P, d));
    i128 v;
    PC_TRY(read_slots(ctx, 1, &v));
    ctx->stats.ms_hard = ph.ms();
    *out = to_pc(v);
    ctx->stats.ms_total = t.ms();
    return PC_OK;
}

extern "C" int pc_p2(pc_ctx* ctx, uint64_t x, uint64_t y, uint64_t* out)
{
    if (!ctx || !out) return PC_EINVAL;
    if (x >> 63) return PC_ERANGE;
    if (x < 1 || y < pc_iroot3(x) || y > pc_isqrt(x)) {
        pc_set_error(ctx, "p2 needs iroot3(x) <= y <= isqrt(x)");
        return PC_EINVAL;
    }
    PC_CUDA(ctx, cudaSetDevice(ctx->device));
    stats_begin(ctx, x);
    Timer t;
    const u64 z = x / y;
    const u64 r = pc_isqrt(x);
    PC_TRY(tables_ensure(ctx, r > y ? r : y, pc_max(y, pc_isqrt(z)), 0, 7));
    u64 vals[1] = {y}, pv[1];
    PC_TRY(tables_pi_values(ctx, vals, pv, 1));
    I128Pair* d;
    PC_TRY(result_slots(ctx, 1, &d));
    PC_TRY(run_p2(ctx, x, y, pv[0], d));
    i128 v;
    PC_TRY(read_slots(ctx, 1, &v));
    if (v < 0 || (v >> 64) != 0) return PC_EOVERFLOW;
    *out = (uint64_t)v;
    ctx->stats.ms_p2 = t.ms();
    ctx->stats.ms_total = t.ms();
    return PC_OK;
}

int pi_count_impl(pc_ctx* ctx, u64 x, u32 alpha, u64* out)
{
    if (x < 2) {
        *out = 0;
        return PC_OK;
    }
    if (x < (1ull << 20)) {
        // small x: read pi(x) from the device pi table (built by sieving on the GPU)
        PC_TRY(tables_ensure(ctx, x, 64, 0, 7));
        u64 v[1] = {x};
        return tables_pi_values(ctx, v, out, 1);
    }
    if (alpha == 0) alpha = choose_alpha(ctx, x);
    ctx->seg_call = choose_seg(ctx, x);
    ctx->ctas_call = ctx->params.ctas_per_sm ? 0 : ctx->tuned_ctas[decimal_digits(x)];
    const u64 r = pc_isqrt(x);
    u64 y = (u64)alpha * pc_iroot3(x);
    if (y > r) y = r;
    if (y < 1) y = 1;
    // c = min(default c, pi(y)); pi(y) >= 5 for y >= 11
    u32 c = ctx->params.c ? ctx->params.c : 5;
    if (y < 17) {
        PC_TRY(tables_ensure(ctx, r, y, 0, 0));
        u64 v[1] = {y}, pv[1];
        PC_TRY(tables_pi_values(ctx, v, pv, 1));
        if (c > pv[0]) c = (u32)pv[0];
    }
    i128 parts[5];
    u64 a = 0;
    const int rc = leaf_parts(ctx, x, y, c, 0, true, parts, &a);
    ctx->seg_call = 0;
    ctx->ctas_call = 0;
    if (rc != PC_OK) return rc;
    i128 pi = parts[0] + parts[1] + parts[2] + parts[3] + (i128)a - 1 - parts[4];
    if (pi < 0 || (pi >> 64) != 0) {
        pc_set_error(ctx, "pi(x) out of range: internal inconsistency");
        return PC_EOVERFLOW;
    }
    *out = (u64)pi;
    return PC_OK;
}

extern "C" int pc_pi_count(pc_ctx* ctx, uint64_t x, uint32_t alpha, uint64_t* out_pi)
{
    if (!ctx || !out_pi) return PC_EINVAL;
    if (x >> 63) return PC_ERANGE;
    PC_CUDA(ctx, cudaSetDevice(ctx->device));
    stats_begin(ctx, x);
    Timer t;
    u64 v = 0;
    PC_TRY(pi_count_impl(ctx, x, alpha, &v));
    *out_pi = v;
    ctx->stats.ms_total = t.ms();
    return PC_OK;
}

int phi_impl(pc_ctx* ctx, u64 x, u64 a, u64* out_phi)
{
    Timer t;
    if (a == 0 || x == 0) {
        *out_phi = a == 0 ? x : 0;
        return PC_OK;
    }
    const u64 r = pc_isqrt(x);
    PC_TRY(tables_ensure(ctx, r, 64, 0, 7));
    u64 v[1] = {r}, pv[1];
    PC_TRY(tables_pi_values(ctx, v, pv, 1));
    const u64 K = pv[0];
    if (a >= K) {
        // every n in (1, x] coprime to p_1..p_a is a prime > p_a (Section 4)
        u64 pix = 0;
        PC_TRY(pi_count_impl(ctx, x, 0, &pix));
        *out_phi = pix + 1 > a ? pix - a + 1 : 1;
        ctx->stats.ms_total = t.ms();
        return PC_OK;
    }
    // p_a < isqrt(x): truncated tree with y in [p_a, isqrt x]
    PC_TRY(buf_reserve(ctx, ctx->misc, 64 * sizeof(u64)));
    nth_prime_kernel<<<1, 1, 0, ctx->stream>>>(ctx->T.pi(), a, r, ctx->misc.as<u64>());
    PC_LAUNCHED(ctx);
    u64 pa = 0;
    PC_TRY(copy_to_host(ctx, &pa, ctx->misc.p, sizeof(u64)));
    u64 y = (u64)choose_alpha(ctx, x) * pc_iroot3(x);
    if (y < pa) y = pa;
    if (y > r) y = r;
    u32 c = a < 5 ? (u32)a : 5;
    i128 parts[5];
    PC_TRY(leaf_parts(ctx, x, y, c, a, false, parts, nullptr));
    i128 phi = parts[0] + parts[1] + parts[2] + parts[3];
    if (phi < 0 || (phi >> 64) != 0) return PC_EOVERFLOW;
    *out_phi = (u64)phi;
    ctx->stats.ms_total = t.ms();
    return PC_OK;
}

extern "C" int pc_phi(pc_ctx* ctx, uint64_t x, uint64_t a, uint64_t* out_phi)
{
    if (!ctx || !out_phi) return PC_EINVAL;
    if (x >> 63) return PC_ERANGE;
    PC_CUDA(ctx, cudaSetDevice(ctx->device));
    stats_begin(ctx, x);
    u64 v = 0;
    PC_TRY(phi_impl(ctx, x, a, &v));
    *out_phi = v;
    return PC_OK;
}
