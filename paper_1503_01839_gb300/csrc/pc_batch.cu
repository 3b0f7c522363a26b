// pc_batch.cu -- many queries at once: the batched call and the server.
//
// Both run queries on worker contexts.  A worker borrows the parent's tables
// (read-only, built up front for every query it will see) and owns a CUDA
// stream, scratch buffers and a host thread, so the kernels of different
// queries overlap on the GPU while each query's own launches stay in order.
// The arithmetic of a query is exactly that of pc_pi_count / pc_phi.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "pc_internal.h"

static int slots_of(const pc_ctx* ctx)
{
    int n = (int)ctx->params.streams;
    if (n <= 0) n = 8;
    if (n > 64) n = 64;
    return n;
}

// ------------------------------------------------------------- workers
int workers_ensure(pc_ctx* ctx, int n)
{
    while ((int)ctx->workers.size() < n) {
        pc_ctx* w = nullptr;
        pc_params p = ctx->params;
        const int rc = pc_create(&w, ctx->device, &p);
        if (rc != PC_OK) {
            pc_set_error(ctx, "worker context: %s", pc_strerror(rc));
            return rc;
        }
        w->borrowed = true;
        ctx->workers.push_back(w);
    }
    for (pc_ctx* w : ctx->workers) {
        w->T = ctx->T;   // shallow: the parent owns every table buffer
        w->params = ctx->params;
        memcpy(w->tuned_alpha, ctx->tuned_alpha, sizeof(ctx->tuned_alpha));
        memcpy(w->tuned_seg, ctx->tuned_seg, sizeof(ctx->tuned_seg));
        memcpy(w->tuned_ctas, ctx->tuned_ctas, sizeof(ctx->tuned_ctas));
    }
    return PC_OK;
}

void workers_destroy(pc_ctx* ctx)
{
    for (pc_ctx* w : ctx->workers) pc_destroy(w);
    ctx->workers.clear();
}

// ------------------------------------------------------ table requirements
// What the tables must cover for a set of queries.  This mirrors the table
// requests of pi_count_impl, phi_impl and leaf_parts; a query that needs more
// fails on its worker with PC_EINVAL instead of growing shared tables.
struct TableNeeds {
    u64 pi = 0, prime = 0, ml = 0;
    u32 cmin = 7;
    void add(u64 pi_, u64 prime_, u64 ml_, u32 c)
    {
        pi = pc_max(pi, pi_);
        prime = pc_max(prime, prime_);
        if (ml_) {
            ml = pc_max(ml, ml_);
            cmin = c < cmin ? c : cmin;
        }
    }
};

// primes p_1..p_n by a host sieve (n is small: the largest a of phi queries)
static std::vector<u64> first_primes(u64 n)
{
    std::vector<u64> ps;
    u64 lim = 64;
    while (true) {
        std::vector<char> comp(lim + 1, 0);
        ps.clear();
        for (u64 i = 2; i <= lim && ps.size() < n + 1; i++) {
            if (comp[i]) continue;
            ps.push_back(i);
            for (u64 j = i * i; j <= lim; j += i) comp[j] = 1;
        }
        if (ps.size() >= n + 1) break;
        lim *= 2;
    }
    return ps;   // ps[k] = p_{k+1}; n + 1 entries
}

static u32 pi_small(u64 v)   // pi(v) for v < 17
{
    static const u32 t[17] = {0, 0, 1, 2, 2, 3, 3, 4, 4, 4, 4, 5, 5, 6, 6, 6, 6};
    return t[v < 17 ? v : 16];
}

// alpha of a query of the batched schedule: the built-in table when pc_autotune_batch found it
// faster for the batch than the per-decade alphas pc_autotune picked for single queries
static u32 batch_alpha(const pc_ctx* ctx, u64 x)
{
    return ctx->batch_builtin_alpha && !ctx->params.alpha ? default_alpha(x) : choose_alpha(ctx, x);
}

static void needs_pi(const pc_ctx* ctx, u64 x, TableNeeds& N, bool batched = false)
{
    if (x < 2) return;
    if (x < (1ull << 20)) {
        N.add(x, 64, 0, 7);
        return;
    }
    const u64 r = pc_isqrt(x);
    u64 y = (u64)(batched ? batch_alpha(ctx, x) : choose_alpha(ctx, x)) * pc_iroot3(x);
    if (y > r) y = r;
    if (y < 1) y = 1;
    u32 c = ctx->params.c ? ctx->params.c : 5;
    if (y < 17 && c > pi_small(y)) c = pi_small(y);
    N.add(r, pc_max(y, pc_isqrt(x / y)), y, c);
}

// phi(x, a) with p_a, p_{a+1} known on the host
static void needs_phi(const pc_ctx* ctx, u64 x, u64 a, u64 pa, u64 pa1, TableNeeds& N)
{
    if (a == 0 || x == 0) return;
    const u64 r = pc_isqrt(x);
    N.add(r, 64, 0, 7);
    if (pa1 > r) {   // a >= pi(isqrt x): the pi(x) branch
        needs_pi(ctx, x, N);
        return;
    }
    u64 y = (u64)choose_alpha(ctx, x) * pc_iroot3(x);
    if (y < pa) y = pa;
    if (y > r) y = r;
    const u32 c = a < 5 ? (u32)a : 5;
    N.add(pc_max(r, y), pc_max(y, pc_isqrt(x / y)), y, c);
}

static int build_needs(pc_ctx* ctx, const TableNeeds& N)
{
    if (N.pi == 0) return PC_OK;
    // slack for isqrt(x / y), which is not monotone in x at cube boundaries
    const u64 prime = N.prime + N.prime / 64 + 64;
    PC_TRY(tables_ensure(ctx, pc_max(N.pi, prime + 2048), prime, N.ml, N.cmin));
    for (u32 c = 1; c <= 7; c++) PC_TRY(tables_phi_c(ctx, c));
    PC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PC_OK;
}

// ------------------------------------------------------------- run queries
struct Query {
    u32 kind;   // PC_QUERY_PI / PC_QUERY_PHI
    u64 x, a;
};

static int run_one(pc_ctx* w, const Query& q, u64* out)
{
    memset(&w->stats, 0, sizeof(w->stats));
    w->stats.x = q.x;
    w->errmsg[0] = 0;
    return q.kind == PC_QUERY_PI ? pi_count_impl(w, q.x, 0, out) : phi_impl(w, q.x, q.a, out);
}

// Runs every query on min(slots, n) workers, largest x first.
static int run_queries(pc_ctx* ctx, const std::vector<Query>& q, std::vector<u64>& out)
{
    const size_t n = q.size();
    const int W = (int)std::min<size_t>((size_t)slots_of(ctx), n);
    PC_TRY(workers_ensure(ctx, W));
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t i, size_t j) { return q[i].x > q[j].x; });
    std::atomic<size_t> next{0};
    std::atomic<int> first_rc{PC_OK};
    std::mutex mu;
    std::vector<pc_stats> st(W);
    auto body = [&](int k) {
        pc_ctx* w = ctx->workers[k];
        if (cudaSetDevice(ctx->device) != cudaSuccess) {
            first_rc = PC_ECUDA;
            return;
        }
        pc_stats acc{};
        for (;;) {
            const size_t i = next.fetch_add(1);
            if (i >= n || first_rc.load() != PC_OK) break;
            const size_t j = order[i];
            u64 v = 0;
            const int rc = run_one(w, q[j], &v);
            if (rc != PC_OK) {
                std::lock_guard<std::mutex> g(mu);
                if (first_rc.load() == PC_OK) {
                    first_rc = rc;
                    pc_set_error(ctx, "query x=%llu: %s", (unsigned long long)q[j].x, w->errmsg);
                }
                break;
            }
            out[j] = v;
            acc.kernel_launches += w->stats.kernel_launches;
            acc.hard_leaves += w->stats.hard_leaves;
            acc.clears += w->stats.clears;
            acc.steps += w->stats.steps;
            acc.segments += w->stats.segments;
        }
        st[k] = acc;
    };
    std::vector<std::thread> th;
    for (int k = 1; k < W; k++) th.emplace_back(body, k);
    body(0);
    for (auto& t : th) t.join();
    pc_stats agg{};
    for (const pc_stats& s : st) {
        agg.kernel_launches += s.kernel_launches;
        agg.hard_leaves += s.hard_leaves;
        agg.clears += s.clears;
        agg.steps += s.steps;
        agg.segments += s.segments;
    }
    ctx->stats = agg;
    return first_rc.load();
}

int mq_final(pc_ctx* ctx, const MQPlan& P, u64* d_out, int* d_bad);

// The pi(x) queries of a batch with 2^20 <= x < MQ_MAX as one schedule: every phase
// (ordinary and trivial leaves, easy leaves, the hard-leaf sieve, P2, the final sums)
// is one launch over all queries, on the context's stream, after one read-back of
// the table values every query needs (pi(y), pi(isqrt z), ...).  The queries are
// sorted largest first, so that the sieve launches start on the longest segments.
static constexpr u64 MQ_MAX = 10000000000000000ull;   // 1e16: larger ones run one by one

// every phase after the read-back of mq_info, in the context's mode (ctx->mq_mode)
static int mq_phases(pc_ctx* ctx, const MQPlan& P, u64* d_out, int* d_bad)
{
    PC_TRY(mq_s1_trivial(ctx, P));
    PC_TRY(mq_easy(ctx, P));
    PC_TRY(mq_hard(ctx, P));
    PC_TRY(mq_p2(ctx, P));
    return mq_final(ctx, P, d_out, d_bad);
}

// The phases' device work (kernels and memsets, no host copies: the prepare pass made
// those), captured from the context's stream into one executable graph.  The capture
// is always ended, so the stream leaves capture mode on every path.
static int mq_capture(pc_ctx* ctx, const MQPlan& P, u64* d_out, int* d_bad, cudaGraphExec_t* out)
{
    PC_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    ctx->mq_mode = MQ_CAPTURE;
    const int rc = mq_phases(ctx, P, d_out, d_bad);
    ctx->mq_mode = MQ_DIRECT;
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(ctx->stream, &g);
    if (rc != PC_OK || ec != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        if (rc != PC_OK) return rc;
        pc_set_error(ctx, "batch graph capture: %s", cudaGetErrorString(ec));
        return PC_ECUDA;
    }
    size_t nodes = 0;
    cudaGraphGetNodes(g, nullptr, &nodes);
    const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        pc_set_error(ctx, "batch graph instantiate: %s", cudaGetErrorString(ei));
        return PC_ECUDA;
    }
    ctx->stats.graph_nodes = nodes;
    return PC_OK;
}

static int multi_batch(pc_ctx* ctx, const std::vector<u64>& xs, std::vector<u64>& out)
{
    const u32 n = (u32)xs.size();
    std::vector<u32> order(n);
    for (u32 i = 0; i < n; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](u32 i, u32 j) { return xs[i] > xs[j]; });
    MQPlan P;
    P.Q = n;
    P.hq.resize(n);
    TableNeeds N;
    for (u32 k = 0; k < n; k++) {
        const u64 x = xs[order[k]];
        const u64 r = pc_isqrt(x);
        u64 y = (u64)batch_alpha(ctx, x) * pc_iroot3(x);
        if (y > r) y = r;
        MQ& m = P.hq[k];
        memset(&m, 0, sizeof(m));
        m.x = x;
        m.y = y;
        m.z = x / y;
        m.c = 5;   // pi(y) >= 5 for every x >= 2^20
        needs_pi(ctx, x, N, true);
    }
    PC_TRY(build_needs(ctx, N));
    // mq_q: queries (n MQ) | parts (5 n I128Pair) | results (n u64) | overflow flag
    const size_t o_parts = ((size_t)n * sizeof(MQ) + 15) / 16 * 16;
    const size_t o_out = o_parts + (size_t)n * 5 * sizeof(I128Pair), o_bad = o_out + (size_t)n * 8;
    PC_TRY(buf_reserve(ctx, ctx->mq_q, o_bad + 16));
    unsigned char* base = ctx->mq_q.as<unsigned char>();
    P.dq = (const MQ*)base;
    P.parts = (I128Pair*)(base + o_parts);
    u64* d_out = (u64*)(base + o_out);
    int* d_bad = (int*)(base + o_bad);
    PC_CUDA(ctx, cudaMemcpyAsync(base, P.hq.data(), n * sizeof(MQ), cudaMemcpyHostToDevice, ctx->stream));
    PC_CUDA(ctx, cudaMemsetAsync(P.parts, 0, (size_t)n * 5 * sizeof(I128Pair) + (size_t)n * 8 + 16, ctx->stream));
    PC_TRY(mq_info(ctx, P));   // the batch's one read-back before the leaf sums
    cudaGraphExec_t exec = nullptr;
    if (ctx->params.batch_launch == 0) {
        // prepare (scratch, uploads, table reads), then capture the device work of every
        // phase into one graph and launch it
        ctx->mq_mode = MQ_PREPARE;
        const int rc = mq_phases(ctx, P, d_out, d_bad);
        ctx->mq_mode = MQ_DIRECT;
        PC_TRY(rc);
        PC_TRY(mq_capture(ctx, P, d_out, d_bad, &exec));
        const cudaError_t e = cudaGraphLaunch(exec, ctx->stream);
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(exec);
            pc_set_error(ctx, "batch graph launch: %s", cudaGetErrorString(e));
            return PC_ECUDA;
        }
        ctx->stats.graph_launches++;
    } else {
        PC_TRY(mq_phases(ctx, P, d_out, d_bad));
    }
    std::vector<u64> res(n);
    int bad = 0;
    cudaError_t e1 = cudaMemcpyAsync(res.data(), d_out, n * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e1 == cudaSuccess) e1 = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(ctx->stream);
    if (exec) cudaGraphExecDestroy(exec);   // after the stream has drained
    if (e1 != cudaSuccess) {
        pc_set_error(ctx, "batch read-back: %s", cudaGetErrorString(e1));
        return PC_ECUDA;
    }
    if (bad) {
        pc_set_error(ctx, "batch: pi(x) out of range (internal inconsistency)");
        return PC_EOVERFLOW;
    }
    for (u32 k = 0; k < n; k++) out[order[k]] = res[k];
    return PC_OK;
}

extern "C" int pc_pi_count_batch(pc_ctx* ctx, const uint64_t* xs, size_t n, uint64_t* out, void* stream)
{
    if (!ctx || (n && (!xs || !out))) return PC_EINVAL;
    if (n == 0) return PC_OK;
    if (ctx->borrowed) return PC_EINVAL;
    PC_CUDA(ctx, cudaSetDevice(ctx->device));
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<u64> hx(n), hout(n, 0);
    if (stream) {
        PC_CUDA(ctx, cudaMemcpyAsync(hx.data(), xs, n * sizeof(u64), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
        PC_CUDA(ctx, cudaStreamSynchronize((cudaStream_t)stream));
    } else {
        memcpy(hx.data(), xs, n * sizeof(u64));
    }
    for (size_t i = 0; i < n; i++)
        if (hx[i] >> 63) return PC_ERANGE;
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    // x < 2^20: one pi-table lookup, as pc_pi_count answers them; 2^20 <= x < 1e16: the
    // batched launches; larger x: one at a time (they fill the GPU on their own)
    std::vector<u64> sx, mx, bx;
    std::vector<size_t> si, mi, bi;
    TableNeeds N;
    for (size_t i = 0; i < n; i++) {
        if (hx[i] < 2) {
            hout[i] = 0;
        } else if (hx[i] < (1ull << 20)) {
            sx.push_back(hx[i]);
            si.push_back(i);
            N.add(hx[i], 64, 0, 7);
        } else if (hx[i] < MQ_MAX && ctx->params.pi_gather == 0) {
            mx.push_back(hx[i]);
            mi.push_back(i);
        } else {
            bx.push_back(hx[i]);
            bi.push_back(i);
        }
    }
    if (!sx.empty()) {
        PC_TRY(build_needs(ctx, N));
        std::vector<u64> sv(sx.size());
        PC_TRY(tables_pi_many(ctx, sx.data(), sv.data(), sx.size()));
        for (size_t k = 0; k < sx.size(); k++) hout[si[k]] = sv[k];
        ctx->stats.kernel_launches++;
    }
    u64 launches = ctx->stats.kernel_launches, glaunch = 0, gnodes = 0;
    if (!mx.empty()) {
        std::vector<u64> mv(mx.size());
        PC_TRY(multi_batch(ctx, mx, mv));
        for (size_t k = 0; k < mx.size(); k++) hout[mi[k]] = mv[k];
        launches = ctx->stats.kernel_launches;
        glaunch = ctx->stats.graph_launches;
        gnodes = ctx->stats.graph_nodes;
    }
    for (size_t k = 0; k < bx.size(); k++) {
        u64 v = 0;
        memset(&ctx->stats, 0, sizeof(ctx->stats));
        PC_TRY(pi_count_impl(ctx, bx[k], 0, &v));
        hout[bi[k]] = v;
        launches += ctx->stats.kernel_launches;
    }
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.kernel_launches = launches;
    ctx->stats.graph_launches = glaunch;
    ctx->stats.graph_nodes = gnodes;
    if (stream) {
        PC_CUDA(ctx, cudaMemcpyAsync(out, hout.data(), n * sizeof(u64), cudaMemcpyHostToDevice, (cudaStream_t)stream));
        PC_CUDA(ctx, cudaStreamSynchronize((cudaStream_t)stream));
    } else {
        memcpy(out, hout.data(), n * sizeof(u64));
    }
    ctx->stats.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return PC_OK;
}

// ------------------------------------------------------------------ server
struct Request {
    pc_result r;
    u64 foot;
};

struct pc_server {
    pc_ctx* ctx = nullptr;
    u64 x_max = 0, a_max = 0, budget = 0;
    u32 policy = PC_SERVE_FIFO;
    std::vector<u64> primes;   // p_1..p_{a_max+1}
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::deque<pc_result> done;
    std::vector<std::thread> threads;
    u64 in_use = 0, running = 0, pending = 0;
    bool stop = false;
    pc_server_stats st{};
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double now_ms() const
    {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

// pi(n) <= 1.26 n / ln n for n > 1 (Rosser and Schoenfeld 1962).  Used only
// to size scratch estimates, never in a count.
static double pi_upper(double n) { return n < 17 ? 7.0 : 1.26 * n / std::log(n); }

// Device scratch of one query: the hard-leaf count and tally rows (at most
// segments x pi(isqrt z) u32 pairs), per-segment and per-work-item arrays,
// the easy-leaf ranges (one per b <= pi(y)) and the P2 segment results.
static u64 footprint(const pc_server* s, int kind, u64 x, u64 a)
{
    const pc_ctx* ctx = s->ctx;
    if (x < (1ull << 20)) return 1ull << 20;
    const u64 r = pc_isqrt(x);
    u64 y = (u64)choose_alpha(ctx, x) * pc_iroot3(x);
    if (kind == PC_QUERY_PHI && a >= 1 && a <= s->a_max && s->primes[a] <= r) y = pc_max(y, s->primes[a - 1]);
    if (y > r) y = r;
    const u64 z = x / y;
    u32 sb = ctx->params.seg_bytes ? ctx->params.seg_bytes : ctx->tuned_seg[decimal_digits(x)];
    if (sb == 0) sb = 32768;
    const double nseg = (double)(z / (30ull * sb) + 1);
    const double B = pi_upper((double)pc_isqrt(z));
    const double rows = nseg * B;
    const double bytes = rows * 8.0 + nseg * 64.0 + pi_upper((double)y) * 32.0 + (double)(z / 983040 + 1) * 48.0 +
                         (double)(4u << 20);
    return (u64)bytes;
}

extern "C" uint64_t pc_server_footprint(pc_server* s, int kind, uint64_t x, uint64_t a)
{
    if (!s) return 0;
    return footprint(s, kind, x, a);
}

static void server_slot(pc_server* s, int k)
{
    pc_ctx* w = s->ctx->workers[k];
    const bool dev_ok = cudaSetDevice(s->ctx->device) == cudaSuccess;
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // the head request starts when it fits in the budget beside the running ones
        s->cv_work.wait(lk, [&] {
            return (!s->queue.empty() && s->in_use + s->queue.front().foot <= s->budget) ||
                   (s->stop && s->queue.empty());
        });
        if (s->queue.empty()) break;
        Request rq = s->queue.front();
        s->queue.pop_front();
        s->in_use += rq.foot;
        s->running++;
        s->st.max_running = pc_max(s->st.max_running, s->running);
        s->st.max_bytes = pc_max(s->st.max_bytes, s->in_use);
        rq.r.t_start_ms = s->now_ms();
        lk.unlock();
        // another request may fit beside this one
        s->cv_work.notify_one();
        u64 v = 0;
        const int rc = dev_ok ? run_one(w, Query{(u32)rq.r.kind, rq.r.x, rq.r.a}, &v) : PC_ECUDA;
        lk.lock();
        rq.r.status = rc;
        rq.r.value = rc == PC_OK ? v : 0;
        rq.r.t_done_ms = s->now_ms();
        s->in_use -= rq.foot;
        s->running--;
        s->pending--;
        s->st.completed++;
        if (rc != PC_OK) s->st.failed++;
        s->done.push_back(rq.r);
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

extern "C" int pc_server_create(pc_ctx* ctx, uint64_t x_max, uint64_t a_max, uint64_t mem_budget, uint32_t policy,
                                pc_server** out)
{
    if (!ctx || !out || ctx->borrowed || policy > PC_SERVE_SMALL_FIRST) return PC_EINVAL;
    if (x_max >> 63) return PC_ERANGE;
    if (a_max > 100000000ull) {
        pc_set_error(ctx, "a_max above 1e8");
        return PC_EINVAL;
    }
    PC_CUDA(ctx, cudaSetDevice(ctx->device));
    pc_server* s = new (std::nothrow) pc_server();
    if (!s) return PC_ENOMEM;
    s->ctx = ctx;
    s->policy = policy;
    s->x_max = x_max;
    s->a_max = a_max;
    s->primes = first_primes(a_max + 1);
    // the requirements grow with x inside each decade (alpha is constant there)
    TableNeeds N;
    std::vector<u64> reps;
    for (u64 p = 10; p - 1 < x_max; p *= 10) {
        reps.push_back(p - 1);
        if (p > x_max / 10) break;
    }
    reps.push_back(x_max);
    for (u64 x : reps) {
        needs_pi(ctx, x, N);
        if (a_max) {
            // y is smallest for a = 1 (covered by pi(x)) and largest for a = a_max
            needs_phi(ctx, x, a_max, s->primes[a_max - 1], s->primes[a_max], N);
            for (u64 a = 1; a <= a_max && a <= 8; a++) needs_phi(ctx, x, a, s->primes[a - 1], s->primes[a], N);
        }
    }
    int rc = build_needs(ctx, N);
    if (rc == PC_OK) rc = workers_ensure(ctx, slots_of(ctx));
    if (rc == PC_OK && mem_budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) rc = PC_ECUDA;
        mem_budget = fr / 2;
    }
    if (rc != PC_OK) {
        delete s;
        return rc;
    }
    s->budget = mem_budget;
    s->st.mem_budget = mem_budget;
    for (int k = 0; k < slots_of(ctx); k++) s->threads.emplace_back(server_slot, s, k);
    *out = s;
    return PC_OK;
}

extern "C" int pc_server_submit(pc_server* s, int kind, uint64_t x, uint64_t a, uint64_t tag)
{
    if (!s || (kind != PC_QUERY_PI && kind != PC_QUERY_PHI)) return PC_EINVAL;
    if (x >> 63) return PC_ERANGE;
    if (x > s->x_max || (kind == PC_QUERY_PHI && a > s->a_max)) return PC_EINVAL;
    Request rq{};
    rq.r.tag = tag;
    rq.r.kind = kind;
    rq.r.x = x;
    rq.r.a = kind == PC_QUERY_PHI ? a : 0;
    rq.foot = footprint(s, kind, x, rq.r.a);
    if (rq.foot > s->budget) return PC_ENOMEM;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stop) return PC_EINVAL;
        rq.r.t_submit_ms = s->now_ms();
        if (s->policy == PC_SERVE_SMALL_FIRST) {
            // ordered by x (the work grows with x), arrival order among equals
            auto at = std::upper_bound(s->queue.begin(), s->queue.end(), rq,
                                       [](const Request& a, const Request& b) { return a.r.x < b.r.x; });
            s->queue.insert(at, rq);
        } else {
            s->queue.push_back(rq);
        }
        s->pending++;
        s->st.submitted++;
    }
    s->cv_work.notify_one();
    return PC_OK;
}

extern "C" int pc_server_poll(pc_server* s, pc_result* out, size_t max, int timeout_ms, size_t* n_out)
{
    if (!s || !n_out || (max && !out)) return PC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] { return !s->done.empty() || s->pending == 0; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, ready);
    else if (timeout_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    size_t k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = k;
    return PC_OK;
}

extern "C" int pc_server_get_stats(pc_server* s, pc_server_stats* out)
{
    if (!s || !out) return PC_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->st;
    return PC_OK;
}

extern "C" void pc_server_destroy(pc_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->threads) t.join();
    delete s;
}

// ---------------------------------------------------------------- autotune
// For every decade of x in [x_lo, x_hi] (x >= 2^20), time pi(x) at a
// representative x for a few alphas around the built-in choice and a few
// hard-leaf segment sizes, and keep the fastest pair for that decade.  Every
// candidate must return the same pi(x); a mismatch is reported as an error.
extern "C" int pc_autotune(pc_ctx* ctx, uint64_t x_lo, uint64_t x_hi, uint32_t reps)
{
    if (!ctx || ctx->borrowed || x_lo > x_hi) return PC_EINVAL;
    if (x_hi >> 63) return PC_ERANGE;
    PC_CUDA(ctx, cudaSetDevice(ctx->device));
    if (reps == 0) reps = 2;
    const u32 fixed_alpha = ctx->params.alpha, fixed_seg = ctx->params.seg_bytes;
    const int d0 = decimal_digits(pc_max(x_lo, 1ull << 20)), d1 = decimal_digits(x_hi);
    for (int d = d0; d <= d1 && d <= 19; d++) {
        // 3 * 10^(d-1): the geometric middle of the decade, inside [x_lo, x_hi]
        u64 x = 3;
        for (int k = 1; k < d; k++) x *= 10;
        x = pc_min(pc_max(x, x_lo), x_hi);
        if (x < (1ull << 20) || decimal_digits(x) != d) continue;
        const u32 a0 = default_alpha(x);
        u32 alphas[5] = {a0 / 2 ? a0 / 2 : 1u, (2 * a0) / 3 ? (2 * a0) / 3 : 1u, a0, (3 * a0 + 1) / 2, 2 * a0};
        const u32 segs[3] = {16384, 32768, 65536};
        double best_ms = 1e300;
        u32 best_a = 0, best_s = 0;
        u64 want = 0;
        bool have = false;
        ctx->tuned_alpha[d] = ctx->tuned_seg[d] = 0;
        for (u32 ai = 0; ai < 5; ai++) {
            if (fixed_alpha && alphas[ai] != fixed_alpha) continue;
            if (ai && alphas[ai] == alphas[ai - 1]) continue;
            for (u32 si = 0; si < 3; si++) {
                if (fixed_seg && si) continue;
                ctx->tuned_seg[d] = fixed_seg ? 0 : segs[si];
                double ms = 1e300;
                for (u32 r = 0; r <= reps; r++) {   // the first run builds tables and is not timed
                    const auto t0 = std::chrono::steady_clock::now();
                    u64 v = 0;
                    memset(&ctx->stats, 0, sizeof(ctx->stats));
                    PC_TRY(pi_count_impl(ctx, x, alphas[ai], &v));
                    const double dt =
                        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
                    if (!have) {
                        want = v;
                        have = true;
                    } else if (v != want) {
                        ctx->tuned_seg[d] = 0;
                        pc_set_error(ctx, "autotune: pi(%llu) differs between settings", (unsigned long long)x);
                        return PC_EOVERFLOW;
                    }
                    if (r && dt < ms) ms = dt;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best_a = alphas[ai];
                    best_s = fixed_seg ? 0 : segs[si];
                }
            }
        }
        ctx->tuned_alpha[d] = fixed_alpha ? 0 : best_a;
        ctx->tuned_seg[d] = best_s;
        // then the resident CTAs per SM of the hard-leaf sieve at that alpha and segment size
        ctx->tuned_ctas[d] = 0;
        if (!ctx->params.ctas_per_sm) {
            const u32 ctas[4] = {0, 2, 4, 6};
            double best_c = 1e300;
            u32 best_k = 0;
            for (u32 ci = 0; ci < 4; ci++) {
                ctx->tuned_ctas[d] = ctas[ci];
                double ms = 1e300;
                for (u32 r = 0; r <= reps; r++) {
                    const auto t0 = std::chrono::steady_clock::now();
                    u64 v = 0;
                    memset(&ctx->stats, 0, sizeof(ctx->stats));
                    PC_TRY(pi_count_impl(ctx, x, best_a, &v));
                    const double dt =
                        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
                    if (!have) {   // a fixed alpha none of the candidates matched: nothing timed yet
                        want = v;
                        have = true;
                    } else if (v != want) {
                        ctx->tuned_ctas[d] = 0;
                        pc_set_error(ctx, "autotune: pi(%llu) differs between settings (alpha %u, segment %u, %u CTAs per SM)",
                                     (unsigned long long)x, best_a, best_s, ctas[ci]);
                        return PC_EOVERFLOW;
                    }
                    if (r && dt < ms) ms = dt;
                }
                if (ms < best_c) {
                    best_c = ms;
                    best_k = ctas[ci];
                }
            }
            ctx->tuned_ctas[d] = best_k;
        }
    }
    return PC_OK;
}

// The batched schedule's alphas and sieve geometry: every candidate (the per-decade alphas of
// pc_autotune or the built-in ones; hard-leaf segments of 16 or 32 KiB, resident CTAs per SM
// as many as fit or 8) runs the whole batch reps + 1 times (the first untimed), the results
// must agree, and the fastest is kept for later batches.
extern "C" int pc_autotune_batch(pc_ctx* ctx, const uint64_t* xs, size_t n, uint32_t reps)
{
    if (!ctx || (n && !xs) || ctx->borrowed) return PC_EINVAL;
    if (n == 0) return PC_OK;
    if (reps == 0) reps = 1;
    struct Cand {
        u32 seg, ctas;
        bool builtin;
    };
    static const Cand cands[] = {{16384, 0, false}, {16384, 8, false}, {32768, 0, false},
                                 {16384, 0, true},  {16384, 8, true},  {32768, 0, true}};
    std::vector<uint64_t> want(n), got(n);
    double best_ms = 1e300;
    Cand best = {0, 0, false};
    bool have = false;
    for (const Cand& c : cands) {
        if (ctx->params.seg_bytes && c.seg != 16384) continue;   // a fixed segment size stays fixed
        if (ctx->params.ctas_per_sm && c.ctas) continue;
        ctx->batch_seg = c.seg;
        ctx->batch_ctas = c.ctas;
        ctx->batch_builtin_alpha = c.builtin;
        double ms = 1e300;
        for (u32 r = 0; r <= reps; r++) {
            const auto t0 = std::chrono::steady_clock::now();
            const int rc = pc_pi_count_batch(ctx, xs, n, got.data(), nullptr);
            const double dt = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (rc != PC_OK) {
                ctx->batch_seg = ctx->batch_ctas = 0;
                ctx->batch_builtin_alpha = false;
                return rc;
            }
            if (!have) {
                want = got;
                have = true;
            } else if (got != want) {
                ctx->batch_seg = ctx->batch_ctas = 0;
                ctx->batch_builtin_alpha = false;
                pc_set_error(ctx, "autotune_batch: results differ between settings (segment %u, %u CTAs per SM)",
                             c.seg, c.ctas);
                return PC_EOVERFLOW;
            }
            if (r && dt < ms) ms = dt;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    ctx->batch_seg = best.seg;
    ctx->batch_ctas = best.ctas;
    ctx->batch_builtin_alpha = best.builtin;
    return PC_OK;
}

extern "C" int pc_tuned_batch(pc_ctx* ctx, uint32_t* seg_bytes, uint32_t* ctas_per_sm, uint32_t* builtin_alpha)
{
    if (!ctx || !seg_bytes || !ctas_per_sm || !builtin_alpha) return PC_EINVAL;
    *builtin_alpha = ctx->batch_builtin_alpha && !ctx->params.alpha ? 1u : 0u;
    *seg_bytes = ctx->params.seg_bytes ? ctx->params.seg_bytes : (ctx->batch_seg ? ctx->batch_seg : 16384);
    *ctas_per_sm = ctx->params.ctas_per_sm ? ctx->params.ctas_per_sm : ctx->batch_ctas;
    return PC_OK;
}

extern "C" int pc_tuned_ctas(pc_ctx* ctx, uint64_t x, uint32_t* ctas_per_sm)
{
    if (!ctx || !ctas_per_sm) return PC_EINVAL;
    *ctas_per_sm = ctx->params.ctas_per_sm ? ctx->params.ctas_per_sm : ctx->tuned_ctas[decimal_digits(x)];
    return PC_OK;
}

extern "C" int pc_tuned(pc_ctx* ctx, uint64_t x, uint32_t* alpha, uint32_t* seg_bytes)
{
    if (!ctx || !alpha || !seg_bytes) return PC_EINVAL;
    const int d = decimal_digits(x);
    *alpha = choose_alpha(ctx, x);
    *seg_bytes = ctx->params.seg_bytes ? ctx->params.seg_bytes : (ctx->tuned_seg[d] ? ctx->tuned_seg[d] : 32768);
    return PC_OK;
}

// ------------------------------------------------------- starting values
// phi(m, b) for every c <= b <= b_max, by the recurrence (4.1)
//   phi(m, b) = phi(m, b-1) - phi(m / p_b, b-1)
// with the case split of Section 4 for the subtracted term, v = m / p_b:
//   p_b > m:               phi(v, b-1) = phi(0, b-1) = 0;
//   sqrt(m) < p_b <= m:    v < p_b, only 1 survives: phi(v, b-1) = 1;
//   v < p_b^2 (Legendre):  every composite <= v has a prime factor < p_b, so
//                          phi(v, b-1) = pi(v) - (b - 1) + 1, pi(v) from the pi table;
//   otherwise:             phi(v, b-1) by the combinatorial algorithm (pc_phi),
//                          these queries running concurrently on the worker slots.
// v < p_b^2 holds exactly when p_b > iroot3(m), so the combinatorial terms are those of
// c < b <= pi(iroot3 m).  The first value phi(m, c) is itself a pc_phi query.  The other
// terms and the running differences are computed on the device.

// term[b - c] for pi(iroot3 m) < b <= b_max (the ones below are the phi queries' values)
__global__ void phi_terms_kernel(const u32* primes, PiTable pit, u64 m, u32 c, u64 b_max, u64 b3, u64* term)
{
    const u64 b = b3 + 1 + (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > b_max) return;
    const u64 p = primes[b];
    u64 t;
    if (p > m) t = 0;
    else if (p * p > m) t = 1;
    else t = pi_lookup(pit, m / p) - b + 2;
    term[b - c] = t;
}

// out[i] = first - sum_{1 <= j <= i} term[j], i < n, by one CTA of 1024 threads
__global__ void __launch_bounds__(1024) phi_sweep_kernel(const u64* term, u64 first, u64 n, u64* out)
{
    __shared__ u64 wsum[32];
    __shared__ u64 s_run;
    const u32 lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_run = 0;
    __syncthreads();
    for (u64 base = 0; base < n; base += 1024) {
        const u64 i = base + threadIdx.x;
        const u64 v = (i < n && i > 0) ? term[i] : 0;
        u64 incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const u64 t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const u64 w = wsum[lane];
            u64 wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const u64 t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            wsum[lane] = wi - w;
        }
        __syncthreads();
        const u64 run = s_run;
        if (i < n) out[i] = first - (run + wsum[wid] + incl);
        __syncthreads();
        if (threadIdx.x == 1023) s_run = run + wsum[wid] + incl;
        __syncthreads();
    }
}

int phi_starts(pc_ctx* ctx, u64 m, u32 c, u64 b_max, u64* out)
{
    if (ctx->borrowed || c > b_max) return PC_EINVAL;
    const u64 n = b_max - c + 1;
    if (m == 0) {
        for (u64 i = 0; i < n; i++) out[i] = 0;
        return PC_OK;
    }
    {
        // p_b <= b (ln b + ln ln b) for b >= 6 (Rosser); only sizes the prime table
        const double bb = (double)pc_max(b_max, (u64)6);
        const u64 plim = (u64)(bb * (std::log(bb) + std::log(std::log(bb)))) + 64;
        PC_TRY(tables_ensure(ctx, pc_max(plim + 4096, pc_iroot3(m) * pc_iroot3(m) + 4096), plim, 0, 7));
    }
    if (ctx->T.nprimes < b_max) {
        pc_set_error(ctx, "phi starts: %llu primes needed", (unsigned long long)b_max);
        return PC_EINVAL;
    }
    // the combinatorial terms: c < b <= b3 = min(pi(iroot3 m), b_max)
    u64 b3 = 0;
    {
        const u64 v[1] = {pc_iroot3(m)};
        PC_TRY(tables_pi_values(ctx, v, &b3, 1));
        b3 = pc_min(pc_max(b3, (u64)c), b_max);
    }
    // p_0 .. p_{max(b3, c + 1)} (the table ends with a sentinel prime past b_max): the
    // queries' arguments m / p_b, and p_a, p_{a+1} to size their tables
    const u64 np = pc_max(b3, (u64)c + 1) + 1;
    std::vector<u32> P(np);
    PC_CUDA(ctx, cudaMemcpy(P.data(), ctx->T.primes.p, np * sizeof(u32), cudaMemcpyDeviceToHost));
    std::vector<Query> q;
    q.push_back(Query{PC_QUERY_PHI, m, c});   // phi(m, c)
    for (u64 b = (u64)c + 1; b <= b3; b++) q.push_back(Query{PC_QUERY_PHI, m / P[b], b - 1});
    TableNeeds N;
    for (const Query& qq : q) {
        const u64 a = qq.a;
        if (a == 0) continue;
        needs_phi(ctx, qq.x, a, P[a], P[a + 1], N);   // a + 1 <= max(b3, c + 1)
    }
    PC_TRY(build_needs(ctx, N));
    std::vector<u64> qv(q.size(), 0);
    const pc_stats keep = ctx->stats;   // the queries run on the worker slots; keep the caller's counters
    const int rq = run_queries(ctx, q, qv);
    ctx->stats = keep;
    PC_TRY(rq);
    // term[b - c]: the queries' values for b <= b3, the rest on the device; then the sweep
    PC_TRY(buf_reserve(ctx, ctx->misc, 2 * n * sizeof(u64) + 64));
    u64* d_term = ctx->misc.as<u64>();
    u64* d_out = d_term + n;
    if (b3 > c)
        PC_CUDA(ctx, cudaMemcpyAsync(d_term + 1, qv.data() + 1, (b3 - c) * sizeof(u64), cudaMemcpyHostToDevice,
                                     ctx->stream));
    if (b_max > b3) {
        phi_terms_kernel<<<(unsigned)((b_max - b3 + 255) / 256), 256, 0, ctx->stream>>>(
            ctx->T.primes.as<u32>(), ctx->T.pi(), m, c, b_max, b3, d_term);
        PC_LAUNCHED(ctx);
    }
    phi_sweep_kernel<<<1, 1024, 0, ctx->stream>>>(d_term, qv[0], n, d_out);
    PC_LAUNCHED(ctx);
    PC_CUDA(ctx, cudaMemcpyAsync(out, d_out, n * sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
    PC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PC_OK;
}

extern "C" int pc_phi_starts(pc_ctx* ctx, uint64_t m, uint32_t c, uint64_t b_max, uint64_t* out)
{
    if (!ctx || !out || c > 7 || b_max < c) return PC_EINVAL;
    if (m >> 63) return PC_ERANGE;
    PC_CUDA(ctx, cudaSetDevice(ctx->device));
    std::vector<u64> v(b_max - c + 1);
    PC_TRY(phi_starts(ctx, m, c, b_max, v.data()));
    memcpy(out, v.data(), v.size() * sizeof(u64));
    return PC_OK;
}
