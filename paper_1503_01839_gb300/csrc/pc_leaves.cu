// pc_leaves.cu -- the leaf sums that need no sieve.
//
// phi(x, a) = S1 + S2 with (combinatorial method of Section 2, tree
// truncated at p_a):
//   S1 = sum over squarefree n <= y, n = 1 or lpf(n) > p_c, gpf(n) <= p_a of
//        mu(n) * phi(x/n, c)                                 (ordinary leaves)
//   S2 = sum over c < b <= a, squarefree m with lpf(m) > p_b, gpf(m) <= p_a,
//        y/p_b < m <= y, of -mu(m) * phi(x/(p_b m), b-1)     (special leaves)
// For a special leaf let u = x/(p_b m).  u < p_b: phi(u, b-1) = 1 (trivial).
// p_b <= u < min(p_b^2, y): phi(u, b-1) = pi(u) - b + 2 (easy; the Legendre
// case of Section 4, with pi(u) from the pi table).  Everything else is a
// hard leaf, resolved by the main sieve (pc_hard.cu); those with b <= 3 have
// the closed forms phi(u,0) = u, phi(u,1) = u - u/2, phi(u,2) = u - u/2 - u/3 + u/6.
// The easy leaves are embarrassingly parallel (Section 3).
#include "pc_internal.h"

struct LeafArgs {
    u64 x, y;
    u32 c;
    u64 a;
    bool trunc;
    PiTable pit;
    RankTable rk;
    MList ml;
    // sub-lists of the m-list (lpf index > slK[k]); the easy leaves of p_b are read from
    // the last one with slK <= b, else from ml
    MList sl[Tables::NSUB];
    RankTable srk[Tables::NSUB];
    u32 slK[Tables::NSUB];
    const u32* primes;
    const u64* primes_rcp;   // floor((2^64 - 1) / p_k)
    const u64* primes_dv;    // p_k and its 32-bit reciprocal (div_dv)
    const uint2* podd;       // odd-number pi table (pi_odd) over [0, y]
    u64 n_lim;   // list entries with m <= y: [0, n_lim)
    // easy-leaf gathers from the sampled table of Section 2.1 instead of the pi table
    const u32* samp;
    u32 samp_s;
    u32 sampled;
    u32 clust_chunk;   // leaves per clustered chunk (a multiple of 32)
};

// pi(v) and p_pi(v) from the sampled table: start at pi(floor(v/s) * s), then
// step along the primes while the next one is <= v (on average about
// s / ln v < 1 step; the prime table ends with a sentinel prime above every v).
__device__ __forceinline__ u64 pi_sampled(const LeafArgs& A, u64 v, u64* pv)
{
    u64 k = A.samp[v / A.samp_s];
    u64 nxt = A.primes[k + 1];
    while (nxt <= v) {
        k++;
        nxt = A.primes[k + 1];
    }
    *pv = A.primes[k];
    return k;
}

// a lane walks clust_chunk / 32 primes of a clustered chunk: long slices keep
// more of a run in one lane, short ones balance the warps when there are few
PC_HD u32 clust_chunk_for(u64 x) { return x >= 100000000000000000ull ? 16384 : 8192; }

static LeafArgs make_args(pc_ctx* ctx, const LeafProblem& P, u64 n_lim)
{
    LeafArgs A;
    A.x = P.x;
    A.y = P.y;
    A.c = P.c;
    A.a = P.a;
    A.trunc = P.trunc;
    A.pit = ctx->T.pi();
    A.rk = ctx->T.rank();
    A.ml = ctx->T.mlist();
    for (int k = 0; k < Tables::NSUB; k++) {
        A.sl[k] = ctx->T.sublist(k);
        A.srk[k] = ctx->T.subrank(k);
        A.slK[k] = k < (int)ctx->T.n_sl ? ctx->T.sl_K[k] : ~0u;
    }
    A.primes = ctx->T.primes.as<u32>();
    A.primes_rcp = ctx->T.primes_rcp.as<u64>();
    A.primes_dv = ctx->T.primes_dv.as<u64>();
    A.podd = ctx->T.pi_odd.as<uint2>();
    A.n_lim = n_lim;
    A.samp = ctx->T.samp.as<u32>();
    A.samp_s = ctx->T.samp_s;
    A.sampled = ctx->params.pi_gather == 1;
    A.clust_chunk = clust_chunk_for(P.x);
    return A;
}

// list index range of entries with m <= y
__global__ void rank_of_kernel(RankTable rk, u64 v, u64* out) { *out = rank_lookup(rk, v); }

static int list_count_upto(pc_ctx* ctx, u64 y, u64* n)
{
    PC_TRY(buf_reserve(ctx, ctx->misc, 64 * sizeof(u64)));
    rank_of_kernel<<<1, 1, 0, ctx->stream>>>(ctx->T.rank(), y, ctx->misc.as<u64>());
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    return copy_to_host(ctx, n, ctx->misc.p, sizeof(u64));
}

static int grid_for(pc_ctx* ctx) { return ctx->sm_count * 4; }

// ------------------------------------------------------------------- S1
__global__ void s1_kernel(LeafArgs A, const u32* phiT, u32 Q, I128Pair* part)
{
    __shared__ i128 scratch[32];
    i128 s = 0;
    auto phic = [&](u64 v) -> u64 {
        if (A.c == 0) return v;
        u64 q = v / Q;
        u32 r = (u32)(v - q * Q);
        return q * phiT[Q] + phiT[r + 1];
    };
    u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) s += (i128)phic(A.x);   // n = 1
    for (u64 i = tid; i < A.n_lim; i += (u64)gridDim.x * blockDim.x) {
        u32 info = A.ml.info[i];
        if ((info >> 1) <= A.c) continue;
        if (A.trunc && A.ml.gpf[i] > A.a) continue;
        u64 m = A.ml.m[i];
        u64 f = phic(A.x / m);
        if (info & 1) s -= (i128)f; else s += (i128)f;
    }
    s = block_sum_i128(s, scratch);
    if (threadIdx.x == 0) store_i128(part + blockIdx.x, s);
}

int run_s1(pc_ctx* ctx, const LeafProblem& P, I128Pair* out)
{
    PC_TRY(tables_phi_c(ctx, P.c));
    u64 n_lim = 0;
    PC_TRY(list_count_upto(ctx, P.y, &n_lim));
    int g = grid_for(ctx);
    PC_TRY(buf_reserve(ctx, ctx->partials, g * sizeof(I128Pair)));
    u32 Q = 1;
    static const u32 P8[8] = {1, 2, 3, 5, 7, 11, 13, 17};
    for (u32 i = 1; i <= P.c; i++) Q *= P8[i];
    s1_kernel<<<g, 256, 0, ctx->stream>>>(make_args(ctx, P, n_lim), P.c ? ctx->T.phiT[P.c].as<u32>() : nullptr, Q,
                                          ctx->partials.as<I128Pair>());
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    return reduce_i128(ctx, ctx->partials.as<I128Pair>(), g, out);
}

// -------------------------------------------------------------- trivial
// For m the trivial leaves are the b with max(c, pi(T)) < b < lpf_index(m),
// b <= a, T = max(y/m, isqrt(x/m)): p_b > y/m makes m > y/p_b, and
// p_b > isqrt(x/m) makes p_b^2 m > x, i.e. u < p_b.
__global__ void trivial_kernel(LeafArgs A, I128Pair* part)
{
    __shared__ i128 scratch[32];
    i64 s = 0;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < A.n_lim; i += (u64)gridDim.x * blockDim.x) {
        u32 info = A.ml.info[i];
        u64 k = info >> 1;
        if (k <= A.c + 1) continue;
        if (A.trunc && A.ml.gpf[i] > A.a) continue;
        u64 m = A.ml.m[i];
        u64 T = pc_max(A.y / m, pc_isqrt(A.x / m));
        u64 hi = pc_min(k - 1, A.a);
        u64 lo = A.c;
        if (T >= 2) {
            u64 pt = pi_lookup(A.pit, T);
            if (pt > lo) lo = pt;
        }
        if (hi > lo) {
            i64 cnt = (i64)(hi - lo);
            s += (info & 1) ? cnt : -cnt;
        }
    }
    i128 v = block_sum_i128((i128)s, scratch);
    if (threadIdx.x == 0) store_i128(part + blockIdx.x, v);
}

int run_trivial(pc_ctx* ctx, const LeafProblem& P, I128Pair* out)
{
    u64 n_lim = 0;
    PC_TRY(list_count_upto(ctx, P.y, &n_lim));
    int g = grid_for(ctx);
    PC_TRY(buf_reserve(ctx, ctx->partials, g * sizeof(I128Pair)));
    trivial_kernel<<<g, 256, 0, ctx->stream>>>(make_args(ctx, P, n_lim), ctx->partials.as<I128Pair>());
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    return reduce_i128(ctx, ctx->partials.as<I128Pair>(), g, out);
}

// ----------------------------------------------------------------- easy
// Leaf ranges per b, then fixed-size chunks of leaves over all b.
//
// Clustered easy leaves: when m is a prime q and u = x/(p_b q) is well below
// q, consecutive q share the same pi(u).  With l = pi(u), every prime q' >= q
// with q' <= (x/p_b) / p_l has pi(x/(p_b q')) = l as well (u only falls as q'
// grows, and stays >= p_l), so the whole run counts (run length) * (l - b + 2).
// Those leaves (q^2 >= CLUST_K * x/p_b, i.e. u <= q / CLUST_K) are taken run by
// run; the rest one leaf per thread.  With the odd-number pi table the runs are
// taken by their value l, 31 consecutive l per warp pass: the run of l holds the
// clustered q with (x/p_b)/p_(l+1) < q <= (x/p_b)/p_l, so its length is a
// difference of two pi lookups that neighbouring lanes share, and p_l's record is
// read with its neighbours'.  Otherwise each thread walks the runs of a contiguous
// slice of q, one pi lookup and two quotients per run.  Chunks go to warps one at
// a time.
static constexpr u32 EASY_CHUNK = 4096;     // leaves per chunk of the rest (128 per lane)
static constexpr u64 CLUST_K = 2;   // measured: 2 beats 1 and 3 by about 1 % at pi(10^18)

struct EasyRange {
    u64 i0, i1;   // list indices [i0, i1) or prime indices (i0, i1] shifted to [i0+1, i1+1)
    u64 im;       // first index of the clustered part (src 1), else i1
    u32 src;      // 0: m-list, 1: primes
    u32 l0, l1;   // clustered part: pi(u) runs from l0 (largest q) to l1 (smallest q)
    u32 ls;       // src 0: the list read, 0 for the m-list, k + 1 for its sub-list k
};

// Clustered chunks taken by pi value (clust_chunk = 0, the odd-table path): the
// clustered leaves of p_b with pi(u) = l, for every l in [l0, l1], CLUST_L values a chunk.
static constexpr u32 CLUST_L = 31 * 128;

__host__ __device__ inline u64 easy_chunks(const EasyRange& r, u32 clust_chunk)
{
    const u64 nclust = r.i1 <= r.im ? 0
                       : clust_chunk ? (r.i1 - r.im + clust_chunk - 1) / clust_chunk
                                     : ((u64)r.l1 - r.l0 + CLUST_L) / CLUST_L;
    return (r.im - r.i0 + EASY_CHUNK - 1) / EASY_CHUNK + nclust;
}

// The easy leaves of prime p_b for a query (x, y, a): list indices [i0, i1) of the
// m-list, or of the primes when p_b^2 > y, and where the clustered part starts.
__device__ __forceinline__ EasyRange easy_range(const LeafArgs& A, u64 x, u64 y, u64 a, u64 b)
{
    const u64 p = A.primes[b];
    const u64 xp = x / p;
    const u64 T = pc_min(p * p, y);
    const u64 lo = pc_max(y / p, xp / T);
    const u64 hi = pc_min(y, xp / p);
    EasyRange r{0, 0, 0, 0, 0, 0, 0};
    if (hi > lo) {
        if (p * p > y) {
            // lpf(m) > p_b and m <= y < p_b^2: m is a prime q, p_b < q <= p_a
            u64 k0 = pc_max(pi_lookup(A.pit, lo), b);
            u64 k1 = pc_min(pi_lookup(A.pit, hi), a);
            if (k1 > k0) {
                r.i0 = k0 + 1;
                r.i1 = k1 + 1;
                r.src = 1;
                // clustered from the first prime q with q^2 >= CLUST_K * x/p_b
                const u64 qc = xp > ~0ull / CLUST_K ? hi + 1 : pc_isqrt(CLUST_K * xp - 1) + 1;
                r.im = qc > hi ? r.i1 : pc_min(pc_max(pi_lookup(A.pit, qc - 1) + 1, r.i0), r.i1);
                if (r.im < r.i1) {
                    // u = x/(p_b q) <= q/3 < y: pi at the smallest and the largest clustered q
                    r.l0 = (u32)pi_lookup(A.pit, xp / A.primes[r.i1 - 1]);
                    r.l1 = (u32)pi_lookup(A.pit, xp / A.primes[r.im]);
                }
            }
        } else {
            // the last sub-list whose entries all have lpf index > K, K <= b: it holds every
            // leaf of p_b and fewer entries to skip (lpf <= p_b) than the whole m-list
            u32 li = 0;
            for (int k = 0; k < Tables::NSUB; k++)
                if (A.slK[k] <= b) li = k + 1;
            const RankTable& R = li ? A.srk[li - 1] : A.rk;
            r.i0 = rank_lookup(R, lo);
            r.i1 = rank_lookup(R, hi);
            r.src = 0;
            r.ls = li;
        }
    }
    if (r.src == 0) r.im = r.i1;
    return r;
}

__global__ void easy_ranges_kernel(LeafArgs A, u64 b_lo, u64 nb, EasyRange* rng, u32* nchunk)
{
    u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    const EasyRange r = easy_range(A, A.x, A.y, A.a, b_lo + t);
    rng[t] = r;
    nchunk[t] = (u32)easy_chunks(r, A.clust_chunk);
}

// chunk -> index t = b - b_lo of the prime whose leaves it holds
__global__ void easy_chunk_map_kernel(u64 nb, const u64* choff, u32* cmap)
{
    const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    for (u64 ch = choff[t]; ch < choff[t + 1]; ch++) cmap[ch] = (u32)t;
}

// How an easy leaf reads pi(u): from the popcount pi table (PI_REC), from the
// sampled table of Section 2.1 (PI_SAMPLED), or from the odd-number table with
// the 32-bit reciprocal divisions of div_dv (PI_ODD, for y < 2^29: every
// quotient taken, u < y and the run bound (x/p_b)/p_l < 2.3 y, stays below 2^31).
enum { PI_REC = 0, PI_SAMPLED = 1, PI_ODD = 2 };
static constexpr u64 PI_ODD_Y = 1ull << 29;

// One chunk of the easy leaves of p_b (query x, a): chunk c of range r, walked by the
// 32 lanes of a warp; adds this lane's share of the sum to s.
template <int MODE>
__device__ __forceinline__ void easy_chunk(const LeafArgs& A, u64 x, u64 a, u64 b, const EasyRange& r, u64 c, u32 cc,
                                           u32 lane, i64& s, u32& n_one, u32& n_runs, u32& n_run_leaves)
{
    const u64 nsp = (r.im - r.i0 + EASY_CHUNK - 1) / EASY_CHUNK;
    const u64 p = A.primes[b];
    const u64 xp = div_rcp(x, p, A.primes_rcp[b]);
    if (c >= nsp) {
        if (MODE == PI_ODD && cc == 0) {
            // Clustered chunk by pi value.  With G(l) = the number of clustered q (prime
            // indices [im, i1)) with q <= (x/p_b)/p_l, exactly G(l) - G(l + 1) of them have
            // pi(x/(p_b q)) = l, each adding l - b + 2.  Lane k takes l = base + k; lanes 0..30
            // take their G(l + 1) from the next lane, so a pass covers 31 values of l, and
            // each G costs one division (p_l's record, read coalesced) and one pi lookup.
            const u32 lbase = r.l0 + (u32)(c - nsp) * CLUST_L;
            const u32 lend = (u32)pc_min((u64)r.l1, (u64)lbase + CLUST_L - 1);   // inclusive
            const u32 im = (u32)r.im, nq = (u32)(r.i1 - r.im);
            const u64 qlast = A.primes[r.i1 - 1];
            // sum over the lane's l of n_l * l; the - (b - 2) n_l part is added per chunk, from
            // sum n_l = G(lbase) - G(lend + 1) (the differences telescope)
            u64 nl = 0;
            u32 g_first = 0, g_last = 0;
            for (u32 l0 = lbase; l0 <= lend; l0 += 31) {
                const u32 l = l0 + lane;
                u32 G = 0;
                if (l <= lend + 1) {   // p_l's record exists: l <= l1 + 1 <= pi(y) + 1
                    // (x/p_b)/p_l < 2.3 y < 2^31; below qlast <= y it is inside the pi table
                    const u32 v = div_dv(xp, A.primes_dv[l]);
                    if (v >= qlast) {
                        G = nq;
                    } else {
                        const i32 k = (i32)pi_odd(A.podd, v) - (i32)im + 1;   // v >= q_im / 2 >= 2
                        G = k <= 0 ? 0u : ((u32)k > nq ? nq : (u32)k);
                    }
                }
                const u32 Gn = __shfl_down_sync(0xffffffffu, G, 1);
                if (lane < 31 && l <= lend) nl += (u64)(G - Gn) * l;
                if (l0 == lbase && lane == 0) g_first = G;
                if (l == lend + 1) g_last = G;
            }
            // G(lbase) sits in lane 0, G(lend + 1) in the lane that computed it
            const u32 gsum = __reduce_add_sync(0xffffffffu, g_last);
            const u32 leaves = __shfl_sync(0xffffffffu, g_first, 0) - gsum;
            s += (i64)nl;
            if (lane == 0) {
                s -= (i64)leaves * ((i64)b - 2);
                n_runs += lend - lbase + 1;   // pi values taken
                n_run_leaves += leaves;
            }
            return;
        }
        // clustered chunk: each thread walks the runs of its slice of primes q
        const u64 per = cc / 32;
        const u64 start = r.im + (c - nsp) * cc + lane * per;
        const u64 end = pc_min(r.i1, start + per);
        if (start >= end) return;
        const u64 qlast = A.primes[end - 1];
        for (u64 i = start; i < end;) {
            const u64 u = div_rcp(xp, A.primes[i], A.primes_rcp[i]);
            u64 l, pl = 0, w = 0, bits = 0;
            u32 hb0 = 0;
            if (MODE == PI_SAMPLED) {
                l = pi_sampled(A, u, &pl);
            } else {
                // pi(u) from u's record (u >= p_b >= 13, so 2, 3 and 5 all count)
                // u < y < 2^32: the record is u / 240, its bit from u / 30 and u % 30
                const u32 u32v = (u32)u, q30 = u32v / 30;
                w = q30 >> 3;
                const u32 e = 8 * (q30 & 7) + cntle30(u32v - 30 * q30);
                const uint4 rq = __ldg((const uint4*)(A.pit.rec + w));
                // the bits of the primes <= u, at the top of the word (shifted by 64 - e)
                bits = low_bits_top((u64)rq.x | ((u64)rq.y << 32), e);
                l = 3 + rq.z + __popcll(bits);
                hb0 = e - 1;
            }
            u64 n = 1;
            if (i + 1 < end) {
                if (MODE == PI_REC) {
                    // p_l, the largest prime <= u, from the same record when it holds one
                    if (bits) {
                        const u32 hb = hb0 - __clzll((long long)bits);   // its bit in the record
                        pl = 240 * w + 30 * (hb >> 3) + r8(hb & 7);
                    } else {
                        pl = A.primes[l];
                    }
                }
                // the run: primes q' <= (x/p_b) / p_l, by the reciprocal of p_l (its index is l)
                const u64 bound = div_rcp(xp, pl, A.primes_rcp[l]);
                u64 pb;
                n = bound >= qlast ? end - i
                                   : (MODE == PI_SAMPLED ? pi_sampled(A, bound, &pb) : pi_lookup(A.pit, bound)) - i + 1;
            }
            s += (i64)n * ((i64)l - (i64)b + 2);
            n_runs++;
            n_run_leaves += (u32)n;
            i += n;
        }
        return;
    }
    const u32 start = (u32)(r.i0 + c * EASY_CHUNK);   // list and prime indices are below 2^32
    const u32 end = (u32)pc_min(r.im, (u64)start + EASY_CHUNK);
    if (MODE == PI_ODD && r.src) {
        // m = q prime: every leaf adds pi(u) - b + 2
        u64 sum = 0;
        u32 k = 0;
        for (u32 i = start + lane; i < end; i += 32, k++) sum += pi_odd(A.podd, div_dv(xp, A.primes_dv[i]));
        s += (i64)sum - (i64)k * ((i64)b - 2);
        n_one += k;
        return;
    }
    for (u32 i = start + lane; i < end; i += 32) {
        u64 m, v;
        bool neg = true;
        if (r.src) {
            m = A.primes[i];
            v = A.primes_rcp[i];
        } else {
            const MList& ml = r.ls ? A.sl[r.ls - 1] : A.ml;
            const u32 info = ml.info[i];
            if ((info >> 1) <= b) continue;
            if (A.trunc && ml.gpf[i] > a) continue;
            m = ml.m[i];
            v = ml.rcp[i];
            neg = info & 1;
        }
        // easy: p_b <= u < y < 2^32; for b > 3, u >= 7 and pi(u) counts 2, 3, 5
        const u32 u = (u32)div_rcp(xp, m, v);
        u64 piu;
        if (MODE == PI_SAMPLED) {
            u64 pv;
            piu = pi_sampled(A, u, &pv);
        } else if (MODE == PI_ODD) {
            piu = pi_odd(A.podd, u);   // u >= p_b >= 2
        } else {
            const u32 q30 = u / 30, w = q30 >> 3;
            const u32 e = 8 * (q30 & 7) + cntle30(u - 30 * q30);   // 0..64
            const uint4 q = __ldg((const uint4*)(A.pit.rec + w));
            const u32 c = __popcll(low_bits_top((u64)q.x | ((u64)q.y << 32), e));
            const u32 small = b > 3 ? 3u : (u >= 2) + (u >= 3) + (u >= 5);
            piu = small + q.z + c;
        }
        const i64 t2 = (i64)piu - (i64)b + 2;
        s += neg ? t2 : -t2;
        n_one++;
    }
}

// MODE: how pi(u) is read (PI_REC, PI_SAMPLED, PI_ODD)
template <int MODE>
__global__ void easy_kernel(LeafArgs A, u64 b_lo, const EasyRange* rng, const u64* choff, const u32* cmap,
                            u64 nchunks, unsigned long long* queue, I128Pair* part, unsigned long long* stat)
{
    __shared__ i128 scratch[32];
    const u32 lane = threadIdx.x & 31;
    i64 s = 0;
    u32 n_one = 0, n_runs = 0, n_run_leaves = 0;   // counters: leaves one at a time, runs, leaves in runs
    // chunks are handed out one at a time to warps (their costs differ widely)
    for (;;) {
        u64 ch = 0;
        if (lane == 0) ch = atomicAdd(queue, 1ull);
        ch = __shfl_sync(0xffffffffu, ch, 0);
        if (ch >= nchunks) break;
        const u64 t = cmap[ch];
        const EasyRange r = rng[t];
        easy_chunk<MODE>(A, A.x, A.a, b_lo + t, r, ch - choff[t], A.clust_chunk, lane, s, n_one, n_runs,
                            n_run_leaves);
    }
    if (stat) {
        const u32 a0 = __reduce_add_sync(0xffffffffu, n_one), a1 = __reduce_add_sync(0xffffffffu, n_runs);
        const u32 a2 = __reduce_add_sync(0xffffffffu, n_run_leaves);
        if (lane == 0) {
            if (a0) atomicAdd(stat, (unsigned long long)a0);
            if (a1) atomicAdd(stat + 1, (unsigned long long)a1);
            if (a2) atomicAdd(stat + 2, (unsigned long long)a2);
        }
    }
    i128 v = block_sum_i128((i128)s, scratch);
    if (threadIdx.x == 0) store_i128(part + blockIdx.x, v);
}

int run_easy(pc_ctx* ctx, const LeafProblem& P, I128Pair* out)
{
    u64 b_lo = (u64)P.c + 1;
    if (P.a < b_lo) return PC_OK;
    u64 nb = P.a - b_lo + 1;
    PC_TRY(buf_reserve(ctx, ctx->easy_rng, nb * sizeof(EasyRange)));
    PC_TRY(buf_reserve(ctx, ctx->easy_chunk_off, (nb + 1) * sizeof(u64) + (nb + 1) * sizeof(u32)));
    u64* choff = ctx->easy_chunk_off.as<u64>();
    u32* nch = (u32*)(choff + nb + 1);
    LeafArgs A = make_args(ctx, P, 0);
    const bool odd = !A.sampled && P.y < PI_ODD_Y && ctx->T.podd_limit >= P.y;
    if (odd) A.clust_chunk = 0;   // clustered chunks by pi value
    easy_ranges_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, ctx->stream>>>(A, b_lo, nb,
                                                                              ctx->easy_rng.as<EasyRange>(), nch);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    PC_TRY(scan_exclusive_u32_to_u64(ctx, nch, choff, nb));
    u64 nchunks = 0;
    PC_TRY(copy_to_host(ctx, &nchunks, choff + nb, sizeof(u64)));
    if (nchunks == 0) return PC_OK;
    if (nchunks >> 32) {
        pc_set_error(ctx, "easy leaves: %llu chunks", (unsigned long long)nchunks);
        return PC_EOVERFLOW;
    }
    PC_TRY(buf_reserve(ctx, ctx->easy_cmap, nchunks * sizeof(u32)));
    easy_chunk_map_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, ctx->stream>>>(nb, choff,
                                                                                 ctx->easy_cmap.as<u32>());
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    int g = (int)pc_min((u64)ctx->sm_count * 8, nchunks);
    PC_TRY(buf_reserve(ctx, ctx->partials, g * sizeof(I128Pair)));
    PC_TRY(buf_reserve(ctx, ctx->queue, 64));
    PC_CUDA(ctx, cudaMemsetAsync(ctx->queue.p, 0, 64, ctx->stream));
    PC_CUDA(ctx, cudaEventRecord(ctx->ev[2], ctx->stream));
    const EasyRange* rng = ctx->easy_rng.as<EasyRange>();
    const u32* cmap = ctx->easy_cmap.as<u32>();
    unsigned long long* queue = (unsigned long long*)ctx->queue.p;
    if (A.sampled)
        easy_kernel<PI_SAMPLED><<<g, 256, 0, ctx->stream>>>(A, b_lo, rng, choff, cmap, nchunks, queue,
                                                            ctx->partials.as<I128Pair>(), ctx->dstat);
    else if (odd)
        easy_kernel<PI_ODD><<<g, 256, 0, ctx->stream>>>(A, b_lo, rng, choff, cmap, nchunks, queue,
                                                        ctx->partials.as<I128Pair>(), ctx->dstat);
    else
        easy_kernel<PI_REC><<<g, 256, 0, ctx->stream>>>(A, b_lo, rng, choff, cmap, nchunks, queue,
                                                        ctx->partials.as<I128Pair>(), ctx->dstat);
    PC_LAUNCHED(ctx);
    PC_CUDA(ctx, cudaEventRecord(ctx->ev[3], ctx->stream));
    ctx->easy_timed = true;
    ctx->stats.kernel_launches++;
    return reduce_i128(ctx, ctx->partials.as<I128Pair>(), g, out);
}

// ------------------------------------------------------- hard, b <= 3
__global__ void hard_smallb_kernel(LeafArgs A, u64 b, u64 i0, u64 i1, I128Pair* part)
{
    __shared__ i128 scratch[32];
    i128 s = 0;
    u64 p = A.primes[b];
    u64 xp = A.x / p;
    for (u64 i = i0 + (u64)blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += (u64)gridDim.x * blockDim.x) {
        u32 info = A.ml.info[i];
        if ((info >> 1) <= b) continue;
        if (A.trunc && A.ml.gpf[i] > A.a) continue;
        u64 u = xp / A.ml.m[i];
        u64 ph;
        if (b == 1) ph = u;
        else if (b == 2) ph = u - u / 2;
        else ph = u - u / 2 - u / 3 + u / 6;
        if (info & 1) s += (i128)ph; else s -= (i128)ph;
    }
    s = block_sum_i128(s, scratch);
    if (threadIdx.x == 0) store_i128(part + blockIdx.x, load_i128(part + blockIdx.x) + s);
}

__global__ void smallb_range_kernel(LeafArgs A, u64 b, u64* out)
{
    u64 p = A.primes[b];
    u64 xp = A.x / p;
    u64 T = pc_min(p * p, A.y);
    u64 lo = A.y / p;
    u64 hi = pc_min(A.y, xp / T);
    out[0] = rank_lookup(A.rk, lo);
    out[1] = hi > lo ? rank_lookup(A.rk, hi) : out[0];
}

int run_hard_smallb(pc_ctx* ctx, const LeafProblem& P, I128Pair* out)
{
    if (P.c >= 3) return PC_OK;
    int g = grid_for(ctx);
    PC_TRY(buf_reserve(ctx, ctx->partials, g * sizeof(I128Pair)));
    PC_CUDA(ctx, cudaMemsetAsync(ctx->partials.p, 0, g * sizeof(I128Pair), ctx->stream));
    LeafArgs A = make_args(ctx, P, 0);
    for (u64 b = (u64)P.c + 1; b <= 3 && b <= P.a; b++) {
        PC_TRY(buf_reserve(ctx, ctx->misc, 64 * sizeof(u64)));
        smallb_range_kernel<<<1, 1, 0, ctx->stream>>>(A, b, ctx->misc.as<u64>());
        PC_LAUNCHED(ctx);
        u64 r[2];
        PC_TRY(copy_to_host(ctx, r, ctx->misc.p, 2 * sizeof(u64)));
        if (r[1] > r[0]) {
            hard_smallb_kernel<<<g, 256, 0, ctx->stream>>>(A, b, r[0], r[1], ctx->partials.as<I128Pair>());
            PC_LAUNCHED(ctx);
            ctx->stats.kernel_launches++;
        }
        ctx->stats.kernel_launches++;
    }
    return reduce_i128(ctx, ctx->partials.as<I128Pair>(), g, out);
}

// ----------------------------------------------------------- many queries at once
// The leaf sums of the pi(x) queries of a batch, each phase one launch over all of
// them: the same arithmetic as the single-query kernels above, with each query's
// x, y, a, c read from its MQ record and its sums added to its parts.

static LeafArgs table_args(pc_ctx* ctx)
{
    LeafProblem P{};
    P.x = 0;
    return make_args(ctx, P, 0);
}

// per query: pi(y), pi(isqrt z), pi(isqrt x), the m-list entries up to y, pi(iroot3 x);
// and the ordinary leaf n = 1, phi(x, c), into S1
__global__ void mq_info_kernel(PiTable pit, RankTable rk, MQ* qs, u32 Q, const u32* phiT, u32 Qc, I128Pair* parts)
{
    const u32 q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    MQ m = qs[q];
    m.a = pi_lookup(pit, m.y);
    m.B = pi_lookup(pit, pc_isqrt(m.z));
    m.K = pi_lookup(pit, pc_isqrt(m.x));
    m.nlim = rank_lookup(rk, m.y);
    m.E = pi_lookup(pit, pc_iroot3(m.x));
    qs[q] = m;
    const u64 v = m.x / Qc;
    const u32 r = (u32)(m.x - v * Qc);
    store_i128(parts + 5 * q, (i128)(v * phiT[Qc] + phiT[r + 1]));   // n = 1 (c = 5 for every batched query)
}

int mq_info(pc_ctx* ctx, MQPlan& P)
{
    PC_TRY(tables_phi_c(ctx, 5));
    mq_info_kernel<<<(P.Q + 127) / 128, 128, 0, ctx->stream>>>(ctx->T.pi(), ctx->T.rank(), (MQ*)P.dq, P.Q,
                                                               ctx->T.phiT[5].as<u32>(), 2310, P.parts);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    PC_CUDA(ctx, cudaMemcpyAsync(P.hq.data(), P.dq, P.Q * sizeof(MQ), cudaMemcpyDeviceToHost, ctx->stream));
    PC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PC_OK;
}

// S1 (ordinary leaves n = m > 1) and the trivial leaves of every m-list entry m <= y of
// every query; thread k takes a contiguous run of the flattened (query, entry) space
__global__ void mq_s1_trivial_kernel(LeafArgs T, const MQ* qs, const u64* pref, u32 Q, const u32* phiT, u32 Qc,
                                     I128Pair* parts)
{
    const u64 total = pref[Q];
    const u64 nth = (u64)gridDim.x * blockDim.x, k = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    const u64 per = (total + nth - 1) / nth;
    u64 g = k * per;
    const u64 gend = pc_min(g + per, total);
    if (g >= gend) return;
    u64 q = mq_find(pref, Q + 1, g);
    while (g < gend) {
        const MQ m = qs[q];
        const u64 qend = pc_min(gend, pref[q + 1]);
        i128 s1 = 0;
        i64 tr = 0;
        for (; g < qend; g++) {
            const u64 i = g - pref[q];
            const u32 info = T.ml.info[i];
            const u64 kb = info >> 1;
            if (kb <= m.c) continue;
            const u64 mv = T.ml.m[i], rc = T.ml.rcp[i];
            const u64 xm = div_rcp(m.x, mv, rc);
            const u64 v = xm / Qc;
            const u64 f = v * phiT[Qc] + phiT[(u32)(xm - v * Qc) + 1];
            s1 += (info & 1) ? -(i128)f : (i128)f;
            if (kb > m.c + 1) {   // trivial leaves of m: max(c, pi(T)) < b < lpf index, b <= a
                const u64 Tm = pc_max(div_rcp(m.y, mv, rc), pc_isqrt(xm));
                const u64 hi = pc_min(kb - 1, m.a);
                u64 lo = m.c;
                if (Tm >= 2) lo = pc_max(lo, pi_lookup(T.pit, Tm));
                if (hi > lo) tr += (info & 1) ? (i64)(hi - lo) : -(i64)(hi - lo);
            }
        }
        if (s1) mq_atomic_add_i128(parts + 5 * q + 0, s1);
        if (tr) mq_atomic_add_i128(parts + 5 * q + 1, (i128)tr);
        q++;
    }
}

int mq_s1_trivial(pc_ctx* ctx, const MQPlan& P)
{
    std::vector<u64> pref(P.Q + 1, 0);
    for (u32 q = 0; q < P.Q; q++) pref[q + 1] = pref[q] + P.hq[q].nlim;
    PC_TRY(buf_reserve(ctx, ctx->mq_pref, (P.Q + 1) * sizeof(u64)));
    if (mq_host_upload(ctx))
        PC_CUDA(ctx, cudaMemcpyAsync(ctx->mq_pref.p, pref.data(), (P.Q + 1) * sizeof(u64), cudaMemcpyHostToDevice,
                                     ctx->stream));
    if (pref[P.Q] == 0 || !mq_device_work(ctx)) return PC_OK;
    const int g = ctx->sm_count * 8;
    mq_s1_trivial_kernel<<<g, 256, 0, ctx->stream>>>(table_args(ctx), P.dq, ctx->mq_pref.as<u64>(), P.Q,
                                                     ctx->T.phiT[5].as<u32>(), 2310, P.parts);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    return PC_OK;
}

// easy ranges of every (query, b), c < b <= min(a, E): pair g of query q is b = c + 1 + g - pref[q]
__global__ void mq_easy_ranges_kernel(LeafArgs T, const MQ* qs, const u64* pref, u32 Q, EasyRange* rng, u32* nch)
{
    const u64 g = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= pref[Q]) return;
    const u64 q = mq_find(pref, Q + 1, g);
    const MQ m = qs[q];
    const EasyRange r = easy_range(T, m.x, m.y, m.a, m.c + 1 + (g - pref[q]));
    rng[g] = r;
    nch[g] = (u32)easy_chunks(r, 0);   // clustered chunks by pi value (odd-table path)
}

// every chunk of every (query, b), handed out to warps one at a time
__global__ void mq_easy_kernel(LeafArgs T, const MQ* qs, const u64* pref, u32 Q, const EasyRange* rng,
                               const u64* choff, u64 npairs, unsigned long long* queue, I128Pair* parts)
{
    const u32 lane = threadIdx.x & 31;
    const u64 nchunks = choff[npairs];
    for (;;) {
        u64 ch = 0;
        if (lane == 0) ch = atomicAdd(queue, 1ull);
        ch = __shfl_sync(0xffffffffu, ch, 0);
        if (ch >= nchunks) break;
        const u64 g = mq_find(choff, npairs + 1, ch);   // the pair of the chunk
        const u64 q = mq_find(pref, Q + 1, g);
        const MQ m = qs[q];
        const EasyRange r = rng[g];
        i64 s = 0;
        u32 n1 = 0, nr = 0, nrl = 0;
        easy_chunk<PI_ODD>(T, m.x, m.a, m.c + 1 + (g - pref[q]), r, ch - choff[g], 0, lane, s,
                          n1, nr, nrl);
        s = warp_sum_i64(s);
        if (lane == 0 && s) mq_atomic_add_i128(parts + 5 * q + 2, (i128)s);
    }
}

int mq_easy(pc_ctx* ctx, const MQPlan& P)
{
    std::vector<u64> pref(P.Q + 1, 0);
    for (u32 q = 0; q < P.Q; q++) {
        const MQ& m = P.hq[q];
        const u64 top = pc_min(m.a, m.E);
        pref[q + 1] = pref[q] + (top > m.c ? top - m.c : 0);
    }
    const u64 np = pref[P.Q];
    if (np == 0) return PC_OK;
    // the batch's x < 10^16 keeps y <= isqrt(x) < 2^29 (PI_ODD)
    for (u32 q = 0; q < P.Q; q++)
        if (P.hq[q].y >= PI_ODD_Y || P.hq[q].y > ctx->T.podd_limit) {
            pc_set_error(ctx, "batched easy leaves: y = %llu beyond the odd-number pi table",
                         (unsigned long long)P.hq[q].y);
            return PC_EINVAL;
        }
    // layout of mq_e: pref (Q+1 u64) | ranges (np) | chunk counts (np u32) | chunk offsets (np+1 u64) | queue
    const size_t o_rng = ((P.Q + 1) * sizeof(u64) + 15) / 16 * 16;
    const size_t o_nch = o_rng + np * sizeof(EasyRange);
    const size_t o_off = (o_nch + np * sizeof(u32) + 15) / 16 * 16;
    const size_t o_q = (o_off + (np + 1) * sizeof(u64) + 15) / 16 * 16;
    PC_TRY(buf_reserve(ctx, ctx->mq_e, o_q + 64));
    unsigned char* base = ctx->mq_e.as<unsigned char>();
    u64* dpref = (u64*)base;
    EasyRange* rng = (EasyRange*)(base + o_rng);
    u32* nch = (u32*)(base + o_nch);
    u64* choff = (u64*)(base + o_off);
    unsigned long long* queue = (unsigned long long*)(base + o_q);
    if (mq_host_upload(ctx))
        PC_CUDA(ctx, cudaMemcpyAsync(dpref, pref.data(), (P.Q + 1) * sizeof(u64), cudaMemcpyHostToDevice,
                                     ctx->stream));
    if (!mq_device_work(ctx)) return scan_exclusive_u32_to_u64(ctx, nch, choff, np);   // its scratch only
    PC_CUDA(ctx, cudaMemsetAsync(queue, 0, 64, ctx->stream));
    const LeafArgs T = table_args(ctx);
    mq_easy_ranges_kernel<<<(unsigned)((np + 255) / 256), 256, 0, ctx->stream>>>(T, P.dq, dpref, P.Q, rng, nch);
    PC_LAUNCHED(ctx);
    PC_TRY(scan_exclusive_u32_to_u64(ctx, nch, choff, np));
    mq_easy_kernel<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(T, P.dq, dpref, P.Q, rng, choff, np, queue, P.parts);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches += 2;
    return PC_OK;
}
