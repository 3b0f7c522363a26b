// pc_hard.cu -- the hard special leaves: the main sieve of Section 3 on the GPU.
//
// The interval [0, z] (z = x/y) is cut into segments; a segment is split
// into sub-ranges of sub_bytes bytes (30*sub_bytes integers, mod-30 wheel),
// one per warp of the CTA that owns the segment.  Each warp walks the primes
// p_b in order, b = k0+1 .. B_s, over its own sub-range only:
//
//   1. leaves of b (b > c): its bitset holds the integers of the sub-range
//      coprime to p_1..p_{b-1}, so for a hard leaf (b, m) with
//      u = x/(p_b m) in the sub-range, phi(u, b-1) = phi(L_w - 1, b-1) +
//      local(u), local(u) = set bits in [L_w, u].  The warp adds
//      -mu(m) * local(u) to its sum and -mu(m) to its tally for b: the unknown
//      phi(L_w - 1, b-1) is recorded, not needed, exactly as the tallies of
//      Section 3.
//   2. cross off the multiples of p_b in the sub-range, then record its count
//      of set bits.
//
// Warps never wait for one another inside a batch of primes (only
// __syncwarp); once per batch the CTA folds the warps' counts and tallies
// into segment rows and settles the carries between its own sub-ranges.
// Across segments, phi(L_s - 1, b - 1) = sum_{s' < s} count(s', b - 1) is an
// exclusive scan (the carries), and
//   S2_hard = sum (local sums) + sum_{s,b} tally(s, b) * phi(L_s - 1, b - 1).
// All segments are sieved at once, so the per-round synchronization of the
// blocks in Section 3 becomes one scan.
//
// A hard leaf (b, m) has u < x / p_b^2, so a segment starting at L only
// needs the primes p_b <= isqrt(x / L): B_s = pi(isqrt(x/L)).
//
// Load balance: hard leaves crowd near u = y (their density falls like
// 1/u^2), so one segment can hold a large share of them.  A pre-pass counts
// the leaves of every segment; heavy segments are handed to several CTAs
// ("replicas"), each of which sieves the whole segment but resolves only its
// share of every step's leaves (Section 3 mentions dynamic block scheduling;
// here the schedule is a list of work items ordered by estimated cost,
// planned on the device).
#include <algorithm>
#include <cmath>
#include <vector>

#include "pc_internal.h"
#include "pc_sieve.cuh"

static constexpr u32 BATCH = 64;
// below this a warp crosses off whole wheel rounds per lane and recounts its blocks after;
// from here on lanes take (class, round) pairs and decrement the block counters (64 against
// 128: S2_hard(1e18) kernel 66.3 -> 65.0 ms)
static constexpr u32 RECOUNT_P = 64;
static constexpr u32 GROUP_P = 128;     // smallest prime crossed off in groups of leaf-free steps
static_assert(GROUP_P >= RECOUNT_P, "grouped steps keep their block counters up to date");
static constexpr u32 MAX_NW = 16;       // warps (sub-ranges) per segment
static constexpr u32 MAX_SUB = 8192;    // bytes per sub-range: up to 256 blocks of 256 bits
static constexpr u32 MAX_SEG = 131072;  // bytes per segment
// Steps of primes p >= sub-range bytes >> RUN_SHIFT (at most 2^RUN_SHIFT multiples per
// residue class in a sub-range) with p^3 above the segment are taken in runs (sparse_runs):
// (runs of 32 steps with up to 512 leaves measured fastest on GB300, against 32 to 256
// leaves and thresholds of 1, 1/4 and 1/8 of the sub-range)
static constexpr u32 RUN_SHIFT = 1;
static constexpr u32 RUN_LEAVES = 512;             // a run ends after the step that brings its leaves to this many
static constexpr u32 LOG_CAP = 512;                // hit log entries per warp (a run's crossings are bounded by it)

// A work item: the steps b_lo <= b < b_hi (and b <= B_s) of segment s.  A light
// segment is one item with all its steps; a heavy one is split into replicas that
// each own a run of consecutive steps (see plan_bsplit_kernel).
struct HardItem {
    u32 s;      // segment
    u32 b_lo;   // first step
    u32 b_hi;   // one past the last step (~0: to the segment's last)
    u32 pad;
};

struct HardArgs {
    u64 x, y, z;
    u32 c, k0, kleaf, bmax;
    u64 a;
    bool trunc;
    u64 nseg;
    u64 s0, s1;   // the segments [s0, s1) of this run (a shard, or all of them)
    u32 seg_bytes, sub_bytes, nw, sub_shift;   // sub_bits = 1 << sub_shift
    u64 span;     // integers per segment
    u64 dspan;    // integers per sub-range
    PiTable pit;
    RankTable rk;
    MList ml;
    // sub-lists of the m-list (lpf index > slK[k]); a prime p_b reads its leaves
    // from the last one with slK <= b, else from ml
    MList sl[Tables::NSUB];
    RankTable srk[Tables::NSUB];
    u32 slK[Tables::NSUB];
    u32 nsl;
    const u32* primes;
    const u64* primes_rcp;
    u64 rcp_y;          // floor((2^64 - 1) / y)
    const u32* segB;
    const u64* rcp_seg;   // per segment: reciprocals of L_s and L_s + span (0 for L = 0)
    const u64* off;
    const u64* start;   // phi(L_{s0} - 1, b) for b = k0 .. bmax (index b - k0), or null for s0 = 0
    u32* counts;
    i32* tallies;
    const HardItem* items;
    const unsigned long long* nitems;   // number of items, written by the planner
    I128Pair* acc;                 // one slot per CTA
    u32* queue;
    unsigned long long* stat;      // [0] hard leaves, [1] multiples crossed off
};

struct __align__(16) StepInfo {
    u64 xp;        // x / p_b
    u64 q;         // L / p_b
    u64 mlo, mhi;  // leaf window m in (mlo, mhi]
    u64 vp;        // floor((2^64 - 1) / p_b)
    u32 p;
    u32 r0;        // L mod p_b
    u32 coff[8];   // floor(p * R8[j] / 30): byte offset of class j inside a wheel round
    u8 cbit[8];    // bit of class j inside its byte
    u32 flags;     // bit 0: leaves are primes, bit 1: step has leaves, bits 2-4: m-list (0 = all, k = sub-list k-1),
                   // bit 5: p >= GROUP_P and p^3 > the last integer of the segment (see group_cross),
                   // bit 6: bit 5 and p >= the sub-range's bytes >> RUN_SHIFT (see sparse_runs)
    u32 pself;     // segment bit of p_b itself, or ~0
    u32 row;       // off[b - k0]: start of the count / tally rows of b
    u32 runcap;    // bit 6: bound of the step's log entries, 8 ceil(sub_bytes / p) + 1
    u32 pad[2];
};

// leaf range of prime b in the segment [L, L + span): m in (mlo, mhi].
// vp, vL, vLs: reciprocals of p, L (0 when L = 0) and L + span.
__device__ __forceinline__ bool leaf_window(const HardArgs& A, u64 p, u64 vp, u64 xp, u64 L, u64 vL, u64 vLs,
                                            u64& mlo, u64& mhi)
{
    // hard: u >= min(p^2, y); xp / p^2 = floor(floor(xp / p) / p)
    const u64 xT = p * p <= A.y ? div_rcp(div_rcp(xp, p, vp), p, vp) : div_rcp(xp, A.y, A.rcp_y);
    mhi = pc_min(A.y, xT);
    if (L) mhi = pc_min(mhi, div_rcp(xp, L, vL));                        // u >= L
    mlo = pc_max(div_rcp(A.y, p, vp), div_rcp(xp, L + A.span, vLs));     // u < L + span, m > y / p
    return mhi > mlo;
}

// A warp owns its sub-range, so crossing off one prime needs no atomics on
// the bitset.  For p < RECOUNT_P (64) the lanes take whole wheel rounds (30 p
// integers, p bytes), even rounds first, then odd ones, so lanes of one pass
// touch words at least 2p bytes apart; for larger p a lane takes one residue
// class in every fourth round, and two of its crossings by different lanes are
// at least 4 bytes apart (classes of one round are >= floor(2p/30) bytes apart,
// neighbouring rounds >= p - floor(29p/30) + floor(p/30); both are >= 4 for p >= 60).  Runs of steps crossed off together (group_cross) mix
// primes in one pass and use atomics on the words.  Block counters take
// shared-memory atomics, since lanes of one pass may share a block.
// Instantiated for several (threads, resident CTAs) launch bounds: fewer
// registers per thread buy more resident warps to hide shared-memory latency.
// A launch over the segments of many queries (the batched form): item g is segment
// g - qpref[q] of query q, qpref[q] <= g < qpref[q + 1], with arguments qargs[q] and its
// local sums added to qacc[q].  Queries keep their segments whole (no replicas).
struct MultiArgs {
    const HardArgs* qargs;
    const u32* qpref;   // nq + 1 entries
    u32 nq;
    unsigned long long items;
    I128Pair* qacc;     // query q's sum goes to qacc[q * qstride]
    u32 qstride;
};

template <int MAXT, int MINB, bool MULTI>
__global__ void __launch_bounds__(MAXT, MINB) hard_sieve_kernel(HardArgs A0, MultiArgs M)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // blocks of 256 bits (four 64-bit words); each lane owns bpl consecutive blocks
    const u32 nw = A0.nw, sub_bytes = A0.sub_bytes, sub_words = sub_bytes >> 2, nbw = sub_bytes >> 5, bpl = nbw >> 5;
    const u32 sub_bits = sub_bytes << 3;
    StepInfo* st = (StepInfo*)smem_raw;
    u32* bits = (u32*)(smem_raw + BATCH * sizeof(StepInfo));
    u16* blk = (u16*)(bits + (A0.seg_bytes >> 2));  // nw * nbw block counters
    u16* pre = blk + nw * nbw;                     // nw * nbw prefix counts
    u32* I = (u32*)(pre + nw * nbw);               // BATCH * (nw + 1)
    u32* cw = I + BATCH * (nw + 1);                // BATCH * nw
    i32* tw = (i32*)(cw + BATCH * nw);             // BATCH * nw
    i32* basew = tw + BATCH * nw;                  // BATCH * nw
    u8* kmodw = (u8*)(basew + BATCH * nw);         // BATCH * nw
    u16* hitlog = (u16*)(kmodw + BATCH * nw);      // nw * LOG_CAP

    __shared__ u32 patw[80];
    __shared__ u32 prev[MAX_NW];
    __shared__ u64 rLk[MAX_NW + 1];   // reciprocals of L + k * dspan, k = 0..nw
    __shared__ u32 s_item;
    __shared__ i128 red[32];
    // the m-lists a step may read its leaves from: index 0 the whole list, k the sub-list k-1
    __shared__ const u32* lst_info[1 + Tables::NSUB];
    __shared__ const u32* lst_m[1 + Tables::NSUB];
    __shared__ const u32* lst_gpf[1 + Tables::NSUB];
    __shared__ const u64* lst_rcp[1 + Tables::NSUB];
    __shared__ RankTable lst_rank[1 + Tables::NSUB];

    const u32 tid = threadIdx.x, lane = tid & 31, w = tid >> 5, NT = blockDim.x;
    make_pattern_words(patw, A0.k0);
    if (tid <= Tables::NSUB) {
        const MList& l = tid == 0 ? A0.ml : A0.sl[tid - 1];
        lst_info[tid] = l.info;
        lst_m[tid] = l.m;
        lst_gpf[tid] = l.gpf;
        lst_rcp[tid] = l.rcp;
        lst_rank[tid] = tid == 0 ? A0.rk : A0.srk[tid - 1];
    }
    u32* my = bits + w * sub_words;
    const u64* my64 = (const u64*)my;
    u16* myblk = blk + w * nbw;
    u32* myblk32 = (u32*)myblk;
    u16* mypre = pre + w * nbw;
    u16* lg = hitlog + w * LOG_CAP;

    // count the set bits of every 256-bit block of the sub-range into myblk;
    // returns this lane's share of the total.  Lanes read consecutive 16-byte
    // halves of blocks (no bank conflicts) and pairs of lanes add up a block.
    auto count_blocks = [&]() -> u32 {
        u32 tot = 0;
        const ulonglong2* h2 = (const ulonglong2*)my;
        for (u32 k = lane; k < 2 * nbw; k += 32) {
            const ulonglong2 v = h2[k];
            u32 c = __popcll(v.x) + __popcll(v.y);
            tot += c;
            c += __shfl_xor_sync(0xffffffffu, c, 1);
            if (!(k & 1)) myblk[k >> 1] = (u16)c;
        }
        return tot;
    };
    i64 acc = 0;
    unsigned long long nleaves = 0, nclears = 0, nbusy = 0, nleafy = 0;

    __shared__ __align__(16) unsigned char sA_raw[MULTI ? sizeof(HardArgs) : 16];
    __shared__ u32 s_q;
    u32 cur_q = ~0u;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(A0.queue, 1u);
        __syncthreads();
        const u64 item = s_item;
        u64 s;
        u32 it_lo, it_hi;
        if (MULTI) {
            if (item >= M.items) break;
            if (tid == 0) {   // the item's query: the last q with qpref[q] <= item
                u32 lo = 0, hi = M.nq;
                while (hi - lo > 1) {
                    const u32 mid = (lo + hi) >> 1;
                    if (M.qpref[mid] <= item) lo = mid; else hi = mid;
                }
                s_q = lo;
            }
            __syncthreads();
            const u32 q = s_q;
            if (q != cur_q) {   // the previous query's sums, then this query's arguments
                if (cur_q != ~0u) {
                    const i128 tq = block_sum_i128((i128)acc, red);
                    if (tid == 0) mq_atomic_add_i128(M.qacc + (u64)cur_q * M.qstride, tq);
                    acc = 0;
                }
                const u32* src = (const u32*)(M.qargs + q);
                for (u32 k = tid; k < sizeof(HardArgs) / 4; k += NT) ((u32*)sA_raw)[k] = src[k];
                cur_q = q;
                __syncthreads();
            }
            s = item - M.qpref[q];
            it_lo = ((const HardArgs*)sA_raw)->k0 + 1;
            it_hi = ~0u;
        } else {
            if (item >= *A0.nitems) break;
            const HardItem it = A0.items[item];
            s = it.s;
            it_lo = it.b_lo;
            it_hi = it.b_hi;
        }
        const HardArgs& A = MULTI ? *(const HardArgs*)sA_raw : A0;
        const u32 Bs = A.segB[s];
        const u32 b_first = it_lo, b_last = it_hi - 1 < Bs ? it_hi - 1 : Bs;   // this item's steps
        const u64 L = s * A.span;
        const u64 Lw = L + w * A.dspan;

        fill_pattern(bits, A.seg_bytes >> 2, L, patw, A.k0);
        if (tid <= nw) {
            const u64 Lk = L + tid * A.dspan;
            rLk[tid] = Lk ? ~0ull / Lk : 0;
        }
        if (b_first > A.k0 + 1 && b_first <= b_last) {
            // A replica that starts at step b_first needs the state after p_{b_first - 1}:
            // the primes before it are crossed off in any order, with no counts (the
            // replica that owns those steps records them), then the blocks are counted.
            __syncthreads();
            auto none = [](u32) {};
            u32 b = A.k0 + 1;
            for (; b < b_first; b++) {   // small primes: the whole CTA, lanes over wheel rounds
                const u32 p = A.primes[b];
                if (p >= 512) break;
                u64 ks = L ? div_rcp(L + p - 1, p, A.primes_rcp[b]) : 0;
                if (ks < p) ks = p;
                cross_off_coop(bits, A.seg_bytes, L, p, ks, tid, NT, none);
            }
            for (u32 task = tid; task < 8 * (b_first - b); task += NT) {   // one thread per (prime, class)
                const u32 bq = b + (task >> 3);
                const u64 p = A.primes[bq];
                u64 ks = L ? div_rcp(L + p - 1, p, A.primes_rcp[bq]) : 0;
                if (ks < p) ks = p;
                cross_off_class(bits, A.seg_bytes, L, (u32)p, ks, task & 7, none);
            }
            for (u32 bq = A.k0 + 1 + tid; bq < b_first; bq += NT) {   // the primes themselves (first segment)
                const u64 p = A.primes[bq];
                if (p >= L + A.span) break;
                if (p >= L) {
                    const u32 pos = seg_pos(p, L);
                    atomicAnd(&bits[pos >> 5], ~(1u << (pos & 31)));
                }
            }
        }
        __syncthreads();
        u32 cnt = __reduce_add_sync(0xffffffffu, count_blocks());
        if (lane == 0) prev[w] = cnt;
        __syncthreads();
        if (tid == 0 && b_first == A.k0 + 1) {
            u32 t = 0;
            for (u32 k = 0; k < nw; k++) t += prev[k];
            A.counts[A.off[0] + (s - A.s0)] = t;
        }

        for (u32 bb = b_first; bb <= b_last; bb += BATCH) {
            const u32 nb = b_last - bb + 1 < BATCH ? b_last - bb + 1 : BATCH;
            __syncthreads();
            // A: per-prime data of the batch
            for (u32 t = tid; t < nb; t += NT) {
                const u32 b = bb + t;
                StepInfo si;
                const u64 p = A.primes[b];
                const u64 vp = A.primes_rcp[b];
                si.p = (u32)p;
                si.vp = vp;
                si.xp = div_rcp(A.x, p, vp);
                si.q = div_rcp(L, p, vp);
                si.r0 = (u32)(L - si.q * p);
                si.row = (u32)A.off[b - A.k0];
                si.runcap = si.pad[0] = si.pad[1] = 0;
                si.flags = 0;
                si.mlo = si.mhi = 0;
                si.pself = (p >= L && p < L + A.span) ? seg_pos(p, L) : ~0u;
                if (b > A.kleaf && b <= A.a && leaf_window(A, p, vp, si.xp, L, rLk[0], rLk[nw], si.mlo, si.mhi))
                {
                    u32 li = 0;
                    for (u32 k = 0; k < A.nsl; k++)
                        if (A.slK[k] <= b) li = k + 1;
                    si.flags = 2u | (p * p > A.y ? 1u : 0u) | (li << 2);
                }
                if (p >= GROUP_P && p * p > div_rcp(L + A.span - 1, p, vp)) {
                    si.flags |= 32u;
                    if (p >= (A.sub_bytes >> RUN_SHIFT)) {
                        si.flags |= 64u;
                        si.runcap = 8 * ((A.sub_bytes + (u32)p - 1) / (u32)p) + 1;
                    }
                }
                for (int j = 0; j < 8; j++) {
                    const u32 pr = (u32)p * r8(j);
                    si.coff[j] = pr / 30;
                    si.cbit[j] = (u8)idx30(pr % 30);
                }
                st[t] = si;
            }
            __syncthreads();
            // B: leaf index boundaries of every sub-range, and first wheel rounds
            for (u32 idx = tid; idx < nb * (nw + 1); idx += NT) {
                const u32 t = idx / (nw + 1), k = idx - t * (nw + 1);
                const StepInfo& si = st[t];
                u32 v32 = 0;
                if (si.flags & 2u) {
                    u64 v;
                    if (k == 0) v = si.mhi;
                    else if (k == nw) v = si.mlo;
                    else v = pc_max(pc_min(div_rcp(si.xp, L + k * A.dspan, rLk[k]), si.mhi), si.mlo);
                    if (si.flags & 1u) {
                        const u64 b = bb + t;
                        v32 = (u32)(pc_min(pc_max(pi_lookup(A.pit, v), b), A.a) + 1);
                    } else {
                        v32 = (u32)rank_lookup(lst_rank[(si.flags >> 2) & 7u], v);
                    }
                }
                I[idx] = v32;
            }
            for (u32 idx = tid; idx < nb * nw; idx += NT) {
                const u32 t = idx / nw, k = idx - t * nw;
                const StepInfo& si = st[t];
                if (bb + t >= Bs) continue;
                const u64 p = si.p;
                u64 klo = si.q + div_rcp((u64)si.r0 + k * A.dspan + p - 1, p, si.vp);   // ceil(L_k / p)
                if (klo < p) klo = p;
                const u64 qa = klo / 30;
                const u32 kmod = (u32)(klo - 30 * qa);
                i64 base = (i64)(p * qa) - (i64)(L / 30 + (u64)k * sub_bytes);
                if (p >= 128 && base < (i64)sub_bytes) {
                    // a large prime often has no multiple in the sub-range although a
                    // wheel round overlaps it: look at the first multiple of every class
                    i64 first = (i64)sub_bytes;
#pragma unroll
                    for (u32 j = 0; j < 8; j++) {
                        const i64 fj = base + (i64)si.coff[j] + (r8(j) < kmod ? (i64)p : 0);
                        first = fj < first ? fj : first;
                    }
                    if (first >= (i64)sub_bytes) base = sub_bytes;
                }
                basew[idx] = base > (i64)sub_bytes ? (i32)sub_bytes : (i32)base;
                kmodw[idx] = (u8)kmod;
            }
            __syncthreads();
            // C: every warp runs the batch over its own sub-range.  Steps that touch
            // neither its leaves nor its integers are skipped: the warp marks its
            // busy steps (and those with leaves, and those it may cross off in a
            // group) with ballots and fills the skipped counts afterwards.
            auto leaf_range = [&](u32 t, u32& j0, u32& j1) {
                j0 = I[t * (nw + 1) + w + 1];
                j1 = I[t * (nw + 1) + w];
            };
            u64 busy = 0, leafy = 0, grp = 0, sparse = 0;
            u32 lj0[BATCH / 32], lj1[BATCH / 32];   // leaf range of step h*32 + lane
#pragma unroll
            for (u32 h = 0; h < BATCH / 32; h++) {
                const u32 t = h * 32 + lane;
                bool on = false, g = false, sq = false;
                lj0[h] = lj1[h] = 0;
                if (t < nb) {
                    const u32 b = bb + t, fl = st[t].flags, ps = st[t].pself;
                    sq = (fl & 64u) != 0;
                    if (b < Bs) {
                        if (basew[t * nw + w] < (i32)sub_bytes) on = true;
                        if (ps != ~0u && (ps >> A.sub_shift) == w) on = true;
                        g = (fl & 32u) != 0;
                    }
                    if (b > A.kleaf && (fl & 2u)) {
                        leaf_range(t, lj0[h], lj1[h]);
                        if (lj1[h] > lj0[h]) on = true;
                    }
                    if (b > A.kleaf) tw[t * nw + w] = 0;
                }
                busy |= (u64)__ballot_sync(0xffffffffu, on) << (h * 32);
                leafy |= (u64)__ballot_sync(0xffffffffu, lj1[h] > lj0[h]) << (h * 32);
                grp |= (u64)__ballot_sync(0xffffffffu, g) << (h * 32);
                sparse |= (u64)__ballot_sync(0xffffffffu, sq) << (h * 32);
            }
            // the sparse steps are a suffix of the batch (both of their conditions grow with p):
            // steps below t_sp go one by one or in groups, the rest in runs
            const u32 t_sp = sparse ? (u32)__ffsll((long long)sparse) - 1 : nb;
            const u64 lomask = t_sp >= 64 ? ~0ull : (1ull << t_sp) - 1;
            grp &= busy & ~leafy & lomask;
            // Leaf data (m, its reciprocal, lpf index and mu) does not depend on the
            // sieve, so the first 32 leaves of the next leaf step are loaded ahead,
            // while the warp is still crossing off earlier primes.
            u32 pf_info = 0, pf_m = 0, pf_gpf = 0;
            u64 pf_v = 0;
            auto leaf_bounds = [&](u32 t, u32& j0, u32& j1) {
                const u32 h = t >> 5;
                j0 = __shfl_sync(0xffffffffu, h ? lj0[1] : lj0[0], t & 31);
                j1 = __shfl_sync(0xffffffffu, h ? lj1[1] : lj1[0], t & 31);
            };
            auto prefetch = [&](u32 t) {
                u32 j0, j1;
                leaf_bounds(t, j0, j1);
                const u32 i = j0 + lane;
                pf_m = 0;
                if (i < j1) {
                    if (st[t].flags & 1u) {
                        pf_info = ~0u;   // a prime: lpf = itself, mu = -1
                        pf_m = A.primes[i];
                        pf_v = A.primes_rcp[i];
                        pf_gpf = 0;
                    } else {
                        const u32 li = (st[t].flags >> 2) & 7u;
                        pf_info = lst_info[li][i];
                        pf_m = lst_m[li][i];
                        pf_v = lst_rcp[li][i];
                        pf_gpf = A.trunc ? lst_gpf[li][i] : 0;
                    }
                }
            };
            // prefix counts of the 256-bit blocks of the sub-range (from the block counters)
            auto block_prefix = [&]() {
                if (bpl == 8) {   // one 16-byte load and store per lane
                    const uint4 q = ((const uint4*)myblk)[lane];
                    const u32 c01 = (q.x & 0xFFFFu) + (q.x >> 16), c23 = (q.y & 0xFFFFu) + (q.y >> 16);
                    const u32 c45 = (q.z & 0xFFFFu) + (q.z >> 16), c67 = (q.w & 0xFFFFu) + (q.w >> 16);
                    const u32 own = c01 + c23 + c45 + c67;
                    u32 incl = own;
                    for (int o = 1; o < 32; o <<= 1) {
                        u32 v = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += v;
                    }
                    const u32 r0 = incl - own, r2 = r0 + c01, r4 = r2 + c23, r6 = r4 + c45;
                    uint4 o4;
                    o4.x = r0 | ((r0 + (q.x & 0xFFFFu)) << 16);
                    o4.y = r2 | ((r2 + (q.y & 0xFFFFu)) << 16);
                    o4.z = r4 | ((r4 + (q.z & 0xFFFFu)) << 16);
                    o4.w = r6 | ((r6 + (q.w & 0xFFFFu)) << 16);
                    ((uint4*)mypre)[lane] = o4;
                } else {
                    u32 run = 0;
                    for (u32 k = 0; k < bpl; k++) run += myblk[lane * bpl + k];
                    u32 incl = run;
                    for (int o = 1; o < 32; o <<= 1) {
                        u32 v = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += v;
                    }
                    run = incl - run;
                    for (u32 k = 0; k < bpl; k++) {
                        const u32 bi = lane * bpl + k;
                        mypre[bi] = (u16)run;
                        run += myblk[bi];
                    }
                }
                __syncwarp();
            };
            // set bits of the sub-range up to the count end e (0 < e <= sub_bits; other lanes
            // read clamped, in-bounds words and add what they like)
            auto count_to = [&](u32 e) -> u32 {
                u32 bi = e >> 8;
                if (bi >= nbw) bi = nbw - 1;
                // set bits of block bi below the end (0..256 of them): both halves
                // of the block at once, no data-dependent loop.  Word i keeps its
                // bits below rem - 64 i by a left shift of 64 (i + 1) - rem, taken
                // as at least 0; PTX clamps a 64-bit shift above 64 to 64 (result 0).
                const u32 rem = e - (bi << 8);
                const ulonglong2 h0 = ((const ulonglong2*)my64)[2 * bi];
                const ulonglong2 h1 = ((const ulonglong2*)my64)[2 * bi + 1];
                auto part = [&](u64 wv, u32 i) -> u32 {
                    i32 sh = (i32)(64 * i + 64) - (i32)rem;
                    sh = sh < 0 ? 0 : (sh > 64 ? 64 : sh);
                    u64 r;
                    asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(wv), "r"(sh));
                    return __popcll(r);
                };
                return mypre[bi] + part(h0.x, 0) + part(h0.y, 1) + part(h1.x, 2) + part(h1.y, 3);
            };
            nbusy += __popcll(busy);
            nleafy += __popcll(leafy);
            if (leafy & lomask) prefetch(__ffsll((long long)(leafy & lomask)) - 1);
            __syncwarp();
            // A run of consecutive busy steps without leaves in this sub-range, all of
            // primes p with p >= GROUP_P and p^3 > every integer of the segment, is
            // crossed off in one go: lane = (step of the run, residue class j), four
            // steps per pass.  A bit still set here is 1, a prime, or a product of primes
            // that are all >= the run's first prime; below that prime cubed it has at
            // most two of them, so exactly one lane of the run reaches it: the one of its
            // least prime factor q, at the cofactor n / q >= q.  That lane's decrement is
            // therefore the one the steps would make in order, and the per-step counts
            // follow by a prefix sum.  Lanes of different primes may share a word, hence
            // the atomics.
            auto group_cross = [&](u64 run) {
                const u32 nr = __popcll(run), lo32 = (u32)run, hi32 = (u32)(run >> 32), nlo = __popc(lo32);
                const u32 slot = lane >> 3, j = lane & 7;
                for (u32 c = 0; c < nr; c += 4) {
                    const u32 n = c + slot;
                    u32 d = 0, tt = 0;
                    if (n < nr) {
                        tt = n < nlo ? __fns(lo32, 0, (int)n + 1) : 32 + __fns(hi32, 0, (int)(n - nlo) + 1);
                        const i32 p = (i32)st[tt].p;
                        const u32 kmod = kmodw[tt * nw + w];
                        const u32 bj = st[tt].cbit[j];
                        i32 by = basew[tt * nw + w] + (i32)st[tt].coff[j] + (r8(j) < kmod ? p : 0);
                        for (; by < (i32)sub_bytes; by += p) {
                            const u32 pos = ((u32)by << 3) + bj, mask = 1u << (pos & 31);
                            const u32 hit = (atomicAnd(&my[pos >> 5], ~mask) & mask) ? 1u : 0u;
                            d += hit;
                            atomicSub(&myblk32[pos >> 9], hit << (16 * ((pos >> 8) & 1)));   // 0 or 1
                            nclears++;
                        }
                        const u32 ps = st[tt].pself;
                        if (j == 0 && ps != ~0u && (ps >> A.sub_shift) == w) {   // p itself
                            const u32 pos = ps & (sub_bits - 1), mask = 1u << (pos & 31);
                            if (atomicAnd(&my[pos >> 5], ~mask) & mask) {
                                d++;
                                atomicSub(&myblk32[pos >> 9], 1u << (16 * ((pos >> 8) & 1)));
                            }
                        }
                    }
                    // lanes 8s .. 8s+7 hold step c+s: an inclusive scan over the warp gives,
                    // at lane 8s+7, the decrement of the steps up to c+s
                    u32 incl = d;
                    for (int o = 1; o < 32; o <<= 1) {
                        const u32 up = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += up;
                    }
                    if (j == 7 && n < nr) cw[tt * nw + w] = cnt - incl;
                    cnt -= __shfl_sync(0xffffffffu, incl, 31);
                }
                __syncwarp();
            };
            // Runs of sparse steps (p >= the sub-range's bytes >> RUN_SHIFT, so each residue
            // class has at most 2^RUN_SHIFT multiples in the sub-range, and p^3 above the
            // segment's last integer).  As in group_cross, a bit still set when the run starts
            // is reached by exactly one crossing of the run, that of its least prime factor, so
            // every crossing of every step of the run is found against the bitset as it is at
            // the run's start, in parallel: lane = (step, residue class), four steps per pass.
            // The crossings that hit a set bit go to a log, ordered by step.  A leaf of step t
            // needs the count of set bits up to u after the steps before t; that is the count on
            // the run's starting bitset less the logged hits of the run's steps before t below
            // u.  So the leaves of all steps of a run share 32-lane passes, one block prefix
            // serves the whole run, and the logged bits are cleared once at its end.  A run ends
            // after the step that brings its leaves to RUN_LEAVES, at 32 steps, or where the
            // log could overflow, which keeps the log scans short.
            auto sparse_runs = [&](u32 t0) {
                while (t0 < nb) {
                    // the leaf ranges of the next (up to) 32 steps, one per lane
                    const u32 ts = t0 + lane;
                    u32 j0 = 0, j1 = 0;
                    {
                        const u32 src = ts & 31;
                        const u32 a0 = __shfl_sync(0xffffffffu, lj0[0], src), a1 = __shfl_sync(0xffffffffu, lj0[1], src);
                        const u32 c0 = __shfl_sync(0xffffffffu, lj1[0], src), c1 = __shfl_sync(0xffffffffu, lj1[1], src);
                        if (ts < nb) {
                            j0 = ts >= 32 ? a1 : a0;
                            j1 = ts >= 32 ? c1 : c0;
                        }
                    }
                    const u32 n = j1 - j0;   // 0 for steps without leaves in this sub-range (or share)
                    u32 incl = n;
                    for (int o = 1; o < 32; o <<= 1) {
                        const u32 v = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += v;
                    }
                    u32 cap = ts < nb ? st[ts].runcap : 0;   // log entries the step may add
                    for (int o = 1; o < 32; o <<= 1) {
                        const u32 v = __shfl_up_sync(0xffffffffu, cap, o);
                        if (lane >= o) cap += v;
                    }
                    u32 avail = nb - t0 < 32 ? nb - t0 : 32;
                    const u32 fits = __popc(__ballot_sync(0xffffffffu, lane < avail && cap <= LOG_CAP));
                    if (fits < avail) avail = fits;   // at least 1: a step adds at most 8 * 2^RUN_SHIFT + 1
                    const u32 enough = __ballot_sync(0xffffffffu, lane < avail && incl >= RUN_LEAVES);
                    const u32 len = enough ? (u32)__ffs(enough) : avail;   // steps t0 .. t0 + len - 1
                    const u32 TL = __shfl_sync(0xffffffffu, incl, len - 1);
                    const u32 loff = incl - n;                             // first leaf of step t0 + lane
                    // leaf g of the run: its step i (the last i < len with loff_i <= g) and its
                    // m-list data (nothing for g >= TL)
                    auto run_leaf = [&](u32 g, u32& i, u32& info, u32& m32, u64& v, u32& gpf) {
                        i = 0;
                        for (u32 stp = 16; stp; stp >>= 1) {
                            const u32 cand = i + stp;
                            const u32 vv = __shfl_sync(0xffffffffu, loff, cand & 31);
                            if (cand < len && vv <= g) i = cand;
                        }
                        const u32 ji = __shfl_sync(0xffffffffu, j0, i);
                        const u32 li = __shfl_sync(0xffffffffu, loff, i);
                        const u32 fl = st[t0 + i].flags;
                        info = 0, m32 = 0, gpf = 0;
                        v = 0;
                        if (g < TL) {
                            const u32 idx = ji + (g - li);
                            if (fl & 1u) {
                                info = ~0u;   // a prime: lpf = itself, mu = -1
                                m32 = A.primes[idx];
                                v = A.primes_rcp[idx];
                            } else {
                                const u32 li2 = (fl >> 2) & 7u;
                                info = lst_info[li2][idx];
                                m32 = lst_m[li2][idx];
                                v = lst_rcp[li2][idx];
                                gpf = A.trunc ? lst_gpf[li2][idx] : 0;
                            }
                        }
                    };

                    // crossings against the starting bitset; hits logged in step order: each lane
                    // counts its hits, a warp scan gives its log offset, then it writes them
                    u32 nent = 0, hoff = 0;                                // hoff: log entries before step t0 + lane
                    for (u32 c = 0; c < len; c += 4) {
                        const u32 sl = lane >> 3, j = lane & 7, i = c + sl, t = t0 + i;
                        i32 by = (i32)sub_bytes, p = 0;
                        u32 bj = 0, pp = ~0u;
                        if (i < len && bb + t < Bs) {
                            p = (i32)st[t].p;
                            by = basew[t * nw + w] + (i32)st[t].coff[j] + (r8(j) < kmodw[t * nw + w] ? p : 0);
                            bj = st[t].cbit[j];
                            const u32 ps = st[t].pself;
                            if (j == 0 && ps != ~0u && (ps >> A.sub_shift) == w) pp = ps & (sub_bits - 1);   // p itself
                        }
                        if (st[t0 + c].p >= sub_bytes) {
                            // every prime of the pass has at most one multiple per class in the
                            // sub-range: hits found in one go, offsets from two ballots
                            u32 h = 0, pa = 0, pb = 0;
                            if (by < (i32)sub_bytes) {
                                const u32 pos = ((u32)by << 3) + bj;
                                nclears++;
                                if ((my[pos >> 5] >> (pos & 31)) & 1u) {
                                    pa = pos;
                                    h = 1;
                                }
                            }
                            if (pp != ~0u && ((my[pp >> 5] >> (pp & 31)) & 1u)) {
                                if (h) pb = pp; else pa = pp;
                                h++;
                            }
                            const u32 m1 = __ballot_sync(0xffffffffu, h >= 1), m2 = __ballot_sync(0xffffffffu, h >= 2);
                            const u32 below = (1u << lane) - 1u;
                            const u32 off = nent + __popc(m1 & below) + __popc(m2 & below);
                            if (h >= 1) lg[off] = (u16)pa;
                            if (h >= 2) lg[off + 1] = (u16)pb;
                            const u32 first = __shfl_sync(0xffffffffu, off, ((lane - c) & 3) * 8);
                            if (lane >= c && lane < c + 4) hoff = first;
                            nent += __popc(m1) + __popc(m2);
                            continue;
                        }
                        u32 h = 0;
                        for (i32 q = by; q < (i32)sub_bytes; q += p) {
                            const u32 pos = ((u32)q << 3) + bj;
                            h += (my[pos >> 5] >> (pos & 31)) & 1u;
                            nclears++;
                        }
                        if (pp != ~0u) h += (my[pp >> 5] >> (pp & 31)) & 1u;
                        u32 hin = h;
                        for (int o = 1; o < 32; o <<= 1) {
                            const u32 v = __shfl_up_sync(0xffffffffu, hin, o);
                            if (lane >= o) hin += v;
                        }
                        u32 off = nent + hin - h;
                        // step c + s starts at the entry offset of lane 8 s
                        const u32 first = __shfl_sync(0xffffffffu, off, ((lane - c) & 3) * 8);
                        if (lane >= c && lane < c + 4) hoff = first;
                        if (h) {
                            for (i32 q = by; q < (i32)sub_bytes; q += p) {
                                const u32 pos = ((u32)q << 3) + bj;
                                if ((my[pos >> 5] >> (pos & 31)) & 1u) lg[off++] = (u16)pos;
                            }
                            if (pp != ~0u && ((my[pp >> 5] >> (pp & 31)) & 1u)) lg[off] = (u16)pp;
                        }
                        nent += __shfl_sync(0xffffffffu, hin, 31);
                    }
                    __syncwarp();
                    if (TL) {
                        block_prefix();   // of the run's starting bitset
                        // each pass's m-list loads are issued one pass ahead (S2_hard(1e17) kernel
                        // 13.62 -> 13.30 ms with the same for steps taken one at a time)
                        u32 ci, cinfo, cm, cgpf;
                        u64 cv;
                        run_leaf(lane, ci, cinfo, cm, cv, cgpf);
                        for (u32 g0 = 0; g0 < TL; g0 += 32) {
                            u32 i, info, m32, gpf;
                            u64 v;
                            i = ci, info = cinfo, m32 = cm, gpf = cgpf, v = cv;
                            if (g0 + 32 < TL) run_leaf(g0 + 32 + lane, ci, cinfo, cm, cv, cgpf);   // next pass in flight
                            const u32 hi = __shfl_sync(0xffffffffu, hoff, i);
                            const u32 t = t0 + i, b = bb + t;
                            const u64 xp = st[t].xp;
                            const bool valid = m32 && (info >> 1) > b && !(A.trunc && gpf > A.a);
                            const u32 e = seg_count_end(div_rcp(xp, m32, v), Lw);
                            u32 below = 0;   // hits of the run's earlier steps below the count end
                            for (u32 k = 0; k < hi; k++) below += lg[k] < e ? 1u : 0u;
                            const u32 cnt_u = count_to(e) - below;
                            const i64 sg = valid ? ((info & 1u) ? 1 : -1) : 0;
                            acc += sg * (i64)cnt_u;
                            if (valid) atomicAdd(&tw[t * nw + w], (i32)sg);
                            nleaves += valid;
                        }
                        __syncwarp();
                    }
                    // clear the logged bits; counts after every step of the run
                    for (u32 k = lane; k < nent; k += 32) {
                        const u32 pos = lg[k];
                        atomicAnd(&my[pos >> 5], ~(1u << (pos & 31)));
                        atomicSub(&myblk32[pos >> 9], 1u << (16 * ((pos >> 8) & 1)));
                    }
                    const u32 hnext = __shfl_down_sync(0xffffffffu, hoff, 1);
                    if (lane < len) cw[(t0 + lane) * nw + w] = cnt - (lane + 1 < len ? hnext : nent);
                    cnt -= nent;
                    __syncwarp();
                    t0 += len;
                }
            };
            const u32 cnt0 = cnt;
            for (u64 todo = busy & lomask; todo;) {
                const u32 t = __ffsll((long long)todo) - 1;
                if ((grp >> t) & 1u) {
                    // the run ends below the next busy step that is not in grp
                    const u64 stop = busy & ~grp & (~0ull << t);
                    const u64 run = grp & (~0ull << t) & (stop ? (stop & (0ull - stop)) - 1 : ~0ull);
                    group_cross(run);
                    todo &= ~run;
                    continue;
                }
                todo &= todo - 1;
                const u32 b = bb + t;
                // the step's data, all loaded at once rather than as a chain of loads
                const u32 fl = st[t].flags, p = st[t].p, ps = st[t].pself;
                const i32 base = basew[t * nw + w];
                const u32 kmod = kmodw[t * nw + w];
                const i32 cj = (i32)st[t].coff[lane & 7];
                const u32 bj = st[t].cbit[lane & 7];
                if (b > A.kleaf) {
                    int tl = 0;
                    if ((leafy >> t) & 1u) {
                        u32 j0, j1;
                        leaf_bounds(t, j0, j1);
                        block_prefix();
                        const u64 xp = st[t].xp;
                        auto one_leaf = [&](u32 info, u32 m32, u64 v, u32 gpf) {
                            // no early exit: a lane without a leaf of b (no entry, lpf <= p_b, or
                            // gpf > p_a) runs the same code and adds 0; its block index is clamped
                            // below and its shifts to 0..64, so its reads stay inside the sub-range
                            const bool valid = m32 && (info >> 1) > b && !(A.trunc && gpf > A.a);
                            const bool neg = info & 1u;
                            const u64 u = div_rcp(xp, m32, v);
                            const u32 c = count_to(seg_count_end(u, Lw));
                            const i64 sg = valid ? (neg ? 1 : -1) : 0;
                            acc += sg * (i64)c;
                            tl += (int)sg;
                            nleaves += valid;
                        };
                        auto load_at = [&](u32 base, u32& info, u32& m32, u64& v, u32& gpf) {
                            const u32 i = base + lane;
                            info = 0, m32 = 0, gpf = 0;
                            v = 0;
                            if (i < j1) {
                                if (fl & 1u) {
                                    info = ~0u;
                                    m32 = A.primes[i];
                                    v = A.primes_rcp[i];
                                } else {
                                    const u32 li = (fl >> 2) & 7u;
                                    info = lst_info[li][i];
                                    m32 = lst_m[li][i];
                                    v = lst_rcp[li][i];
                                    gpf = A.trunc ? lst_gpf[li][i] : 0;
                                }
                            }
                        };
                        u32 ninfo = 0, nm = 0, ngpf = 0;
                        u64 nv = 0;
                        if (j0 + 32 < j1) load_at(j0 + 32, ninfo, nm, nv, ngpf);        // second 32 in flight
                        one_leaf(pf_info, pf_m, pf_v, pf_gpf);                        // first 32, loaded ahead
                        const u64 later = leafy & lomask & ~((2ull << t) - 1);
                        if (later) prefetch(__ffsll((long long)later) - 1);           // next leaf step
                        for (u32 base = j0 + 32; base < j1; base += 32) {             // the rest
                            u32 info, m32, gpf;
                            u64 v;
                            info = ninfo, m32 = nm, gpf = ngpf, v = nv;
                            if (base + 32 < j1) load_at(base + 32, ninfo, nm, nv, ngpf);   // next 32 in flight
                            one_leaf(info, m32, v, gpf);
                        }
                        tl = __reduce_add_sync(0xffffffffu, (u32)tl);
                        if (lane == 0) tw[t * nw + w] = tl;   // steps without leaves keep the 0 set above
                    }
                }
                if (b < Bs) {
                    const bool recount = p < RECOUNT_P;
                    u32 dec = 0;
                    auto clear_bit = [&](u32 pos) {   // pos: bit inside this warp's sub-range
                        const u32 mask = 1u << (pos & 31);
                        const u32 old = my[pos >> 5];
                        my[pos >> 5] = old & ~mask;   // written back whether or not the bit was set
                        const u32 hit = (old & mask) ? 1u : 0u;
                        dec += hit;
                        if (!recount) atomicSub(&myblk32[pos >> 9], hit << (16 * ((pos >> 8) & 1)));
                    };
                    {
                        if (base < (i32)sub_bytes) {
                            if (p >= RECOUNT_P) {
                                // lane = (class j, round offset o): four rounds per pass.
                                // Two crossings of one prime p >= 64 by different lanes
                                // are >= 4 bytes apart, so no two lanes share a word.
                                const u32 j = lane & 7, o = lane >> 3;
                                // round o, or o + 4 when round 0 starts below the first cofactor;
                                // every byte reached from there is >= 0 (k >= klo)
                                const i32 step4 = 4 * (i32)p;
                                i32 by = base + (i32)p * (i32)o + cj;
                                if (o == 0 && r8(j) < kmod) by += step4;
                                u32 n = 0;
                                // two rounds at a time, both words loaded before either is written
                                // (they are 4p bytes apart, so never the same word)
                                for (; by + step4 < (i32)sub_bytes; by += 2 * step4, n += 2) {
                                    const u32 pa = ((u32)by << 3) + bj, pb = ((u32)(by + step4) << 3) + bj;
                                    const u32 ma = 1u << (pa & 31), mb = 1u << (pb & 31);
                                    // no branch on whether the bit was still set: the word is
                                    // written back either way and the block counter takes 0 or 1
                                    const u32 oa = my[pa >> 5], ob = my[pb >> 5];
                                    my[pa >> 5] = oa & ~ma;
                                    my[pb >> 5] = ob & ~mb;
                                    const u32 ca = (oa & ma) ? 1u : 0u, cb = (ob & mb) ? 1u : 0u;
                                    dec += ca + cb;
                                    atomicSub(&myblk32[pa >> 9], ca << (16 * ((pa >> 8) & 1)));
                                    atomicSub(&myblk32[pb >> 9], cb << (16 * ((pb >> 8) & 1)));
                                }
                                if (by < (i32)sub_bytes) {
                                    clear_bit(((u32)by << 3) + bj);
                                    n++;
                                }
                                nclears += n;
                            } else {
                                const uint2 bv = *(const uint2*)st[t].cbit;
                                const uint4 c0 = *(const uint4*)st[t].coff, c1 = *(const uint4*)(st[t].coff + 4);
                                const u32 cw8[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
                                // lane = whole wheel rounds, even rounds first, then odd ones.
                                // The blocks are recounted afterwards (p < RECOUNT_P), so a bit is
                                // simply cleared; a lane takes rounds r and r + 64 together
                                // (64 p bytes apart: never the same word) to overlap their loads.
                                for (u32 ph = 0; ph < 2; ph++) {
                                    for (u32 r = 2 * lane + ph;; r += 128) {
                                        const i32 b0 = base + (i32)(p * r);
                                        if (b0 >= (i32)sub_bytes) break;
                                        const i32 b1 = b0 + 64 * (i32)p;
#pragma unroll
                                        for (int jj = 0; jj < 8; jj++) {
                                            const i32 by0 = b0 + (i32)cw8[jj], by1 = b1 + (i32)cw8[jj];
                                            const bool ok0 = by0 < (i32)sub_bytes && !(r == 0 && r8(jj) < kmod);
                                            const bool ok1 = by1 < (i32)sub_bytes;
                                            const u32 bit = ((jj < 4 ? bv.x : bv.y) >> (8 * (jj & 3))) & 0xFFu;
                                            const u32 q0 = ((u32)by0 << 3) + bit, q1 = ((u32)by1 << 3) + bit;
                                            u32 w0 = 0, w1 = 0;
                                            if (ok0) w0 = my[q0 >> 5];
                                            if (ok1) w1 = my[q1 >> 5];
                                            if (ok0) my[q0 >> 5] = w0 & ~(1u << (q0 & 31));
                                            if (ok1) my[q1 >> 5] = w1 & ~(1u << (q1 & 31));
                                            nclears += (u32)ok0 + (u32)ok1;
                                        }
                                    }
                                    __syncwarp();
                                }
                            }
                        }
                    }
                    __syncwarp();
                    if (lane == 0 && ps != ~0u && (ps >> A.sub_shift) == w) clear_bit(ps & (sub_bits - 1));
                    if (recount) {
                        __syncwarp();
                        cnt = __reduce_add_sync(0xffffffffu, count_blocks());
                    } else {
                        cnt -= __reduce_add_sync(0xffffffffu, dec);
                    }
                }
                if (lane == 0) cw[t * nw + w] = cnt;
                __syncwarp();
            }
            if (t_sp < nb) sparse_runs(t_sp);
            for (u32 t = lane; t < t_sp; t += 32) {
                if ((busy >> t) & 1u) continue;
                const u64 before = busy & ((1ull << t) - 1);
                cw[t * nw + w] = before ? cw[(63 - __clzll((long long)before)) * nw + w] : cnt0;
            }
            __syncthreads();
            // D: segment rows, and the carries between the CTA's sub-ranges
            for (u32 t = tid; t < nb; t += NT) {
                const u32 b = bb + t;
                u32 C = 0;
                for (u32 k = 0; k < nw; k++) C += cw[t * nw + k];
                const u64 row = st[t].row;
                if (b < Bs) A.counts[row + (s - A.s0)] = C;
                if (b > A.kleaf) {
                    const u32* cp = t ? cw + (t - 1) * nw : prev;
                    i32 T = 0;
                    i64 intra = 0, run = 0;
                    for (u32 k = 0; k < nw; k++) {
                        const i32 tk = tw[t * nw + k];
                        T += tk;
                        intra += (i64)tk * run;
                        run += cp[k];
                    }
                    if (T) atomicAdd(&A.tallies[row + (s - A.s0)], T);
                    acc += intra;
                }
            }
            __syncthreads();
            if (tid < nw) prev[tid] = cw[(nb - 1) * nw + tid];
        }
    }
    i128 tot = block_sum_i128((i128)acc, red);
    if (MULTI) {
        if (tid == 0 && cur_q != ~0u) mq_atomic_add_i128(M.qacc + (u64)cur_q * M.qstride, tot);
    } else {
        if (tid == 0) store_i128(A0.acc + blockIdx.x, tot);
    }
    for (int o = 16; o; o >>= 1) {
        nleaves += __shfl_xor_sync(0xffffffffu, nleaves, o);
        nclears += __shfl_xor_sync(0xffffffffu, nclears, o);
    }
    if (lane == 0 && nleaves) atomicAdd(A0.stat, nleaves);
    if (lane == 0 && nclears) atomicAdd(A0.stat + 1, nclears);
    if (lane == 0 && nbusy) atomicAdd(A0.stat + 2, nbusy);     // busy (warp, step) pairs
    if (lane == 0 && nleafy) atomicAdd(A0.stat + 3, nleafy);   // of which with leaves
}

// ---------------------------------------------------------- schedule
__global__ void seg_b_kernel(u64 x, u64 nseg, u64 span, u32 bmax, PiTable pit, u32* segB, u64* rcp_seg)
{
    u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    rcp_seg[2 * s] = s ? ~0ull / (s * span) : 0;
    rcp_seg[2 * s + 1] = ~0ull / ((s + 1) * span);
    u32 B = bmax;
    if (s > 0) {
        u64 L = s * span;
        u64 r = pc_isqrt(x / L);
        u64 pr = pi_lookup(pit, r);
        if (pr < B) B = (u32)pr;
    }
    segB[s] = B;
}

// S_b = number of segments in [s0, s1) with B_s >= b (B_s is non-increasing in s)
__global__ void row_len_kernel(const u32* segB, u64 nseg, u64 s0, u64 s1, u32 k0, u32 bmax, u32* len)
{
    u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    u32 b = k0 + t;
    if (b > bmax) return;
    u64 lo = 0, hi = nseg;   // first s with segB[s] < b
    while (lo < hi) {
        u64 mid = (lo + hi) >> 1;
        if (segB[mid] >= b) lo = mid + 1; else hi = mid;
    }
    len[t] = (u32)(pc_min(pc_max(lo, s0), s1) - s0);
}

// Upper bound of the hard leaves of every segment (the lpf filter of the
// m-list is not applied): a warp per segment s in [s0, s1), its lanes over the
// segment's leaf primes b (kleaf < b <= min(B_s, a)), one store per segment.
__global__ void hard_estimate_kernel(HardArgs A, unsigned long long* est)
{
    const u64 s = A.s0 + ((u64)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const u32 lane = threadIdx.x & 31;
    if (s >= A.s1) return;   // the whole warp
    const u64 L = s * A.span, vL = A.rcp_seg[2 * s], vLs = A.rcp_seg[2 * s + 1];
    const u64 bhi = pc_min((u64)A.segB[s], A.a);
    u64 n = 0;
    for (u64 b = A.kleaf + 1 + lane; b <= bhi; b += 32) {
        const u64 p = A.primes[b];
        const u64 vp = A.primes_rcp[b];
        const u64 xp = div_rcp(A.x, p, vp);
        u64 mlo, mhi;
        if (!leaf_window(A, p, vp, xp, L, vL, vLs, mlo, mhi)) continue;
        if (p * p > A.y) {
            const u64 k0 = pc_min(pc_max(pi_lookup(A.pit, mlo), b), A.a);
            const u64 k1 = pc_min(pc_max(pi_lookup(A.pit, mhi), b), A.a);
            n += k1 - k0;
        } else {
            n += rank_lookup(A.rk, mhi) - rank_lookup(A.rk, mlo);
        }
    }
    for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0) est[s] = n;
}

// S2_hard carries: for each leaf prime b, the exclusive scan over segments
// of count(., b-1) dotted with tally(., b).
template <int NT>
__global__ void __launch_bounds__(NT) hard_combine_kernel(HardArgs A, I128Pair* part)
{
    __shared__ u64 wsum[NT / 32];
    __shared__ u64 s_carry;
    __shared__ i128 red[32];
    const u32 lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    i128 dot = 0;
    for (u32 b = A.kleaf + 1 + blockIdx.x; b <= A.bmax; b += gridDim.x) {
        const u64 row = A.off[b - A.k0];
        const u64 Sb = A.off[b - A.k0 + 1] - row;
        const u64 prow = A.off[b - 1 - A.k0];
        if (threadIdx.x == 0) s_carry = A.start ? A.start[b - 1 - A.k0] : 0;
        __syncthreads();
        for (u64 base = 0; base < Sb; base += NT) {
            const u64 s = base + threadIdx.x;
            const u64 v = s < Sb ? (u64)A.counts[prow + s] : 0;
            u64 incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                u64 t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) wsum[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                u64 w = lane < NT / 32 ? wsum[lane] : 0, wi = w;
                for (int o = 1; o < 32; o <<= 1) {
                    u64 t = __shfl_up_sync(0xffffffffu, wi, o);
                    if (lane >= o) wi += t;
                }
                if (lane < NT / 32) wsum[lane] = wi - w;
            }
            __syncthreads();
            const u64 c0 = s_carry;
            const u64 carry = c0 + wsum[wid] + incl - v;
            if (s < Sb) {
                const i32 tl = A.tallies[row + s];
                if (tl) dot += (i128)tl * (i128)carry;
            }
            __syncthreads();
            if (threadIdx.x == NT - 1) s_carry = c0 + wsum[wid] + incl;
            __syncthreads();
        }
    }
    dot = block_sum_i128(dot, red);
    if (threadIdx.x == 0) store_i128(part + blockIdx.x, dot);
}

// ---------------------------------------------------------------- host
u32 pc_seg_bytes(pc_ctx* ctx, u32 dflt)
{
    u32 sb = ctx->params.seg_bytes ? ctx->params.seg_bytes : ctx->seg_call;
    if (sb == 0) sb = dflt;
    if (sb < 1024) sb = 1024;
    if (sb > MAX_SEG) sb = MAX_SEG;
    if (sb > 4096) sb = sb / 4096 * 4096;
    else if (sb > 2048) sb = 4096 > sb ? 2048 : 4096;   // sub-ranges are powers of two
    else sb = sb / 1024 * 1024;
    return sb;
}

// bytes per warp sub-range: a power of two dividing seg_bytes, at most 16 warps
static u32 pc_sub_bytes(pc_ctx* ctx, u32 seg_bytes)
{
    u32 wb = ctx->params.warp_bytes ? ctx->params.warp_bytes : 8192;
    if (wb > MAX_SUB) wb = MAX_SUB;
    if (wb > seg_bytes) wb = seg_bytes;
    while (seg_bytes % wb) wb >>= 1;
    while (seg_bytes / wb > MAX_NW) wb <<= 1;
    return wb;
}

// Work items: segments, heavy ones split into replicas; sorted by estimated
// cost, heaviest first.  Costs in units of one leaf: one (segment, prime)
// step of all warps costs about STEP_COST leaves, one crossing-off about
// CLEAR_COST.  A segment's crossings are estimated by Mertens' theorem,
// span * 8/30 * sum_{13 <= p <= P} 1/p ~ span * 8/30 * (ln ln P - 1.0056),
// P = isqrt(x / L), the largest prime the segment sieves with.
// Work items, planned on the device.  Cost of a segment (arbitrary units): its
// (segment, prime) steps, its crossings (span * 8/30 * the sum of 1/p over its
// primes, about ln ln P - ln ln 11 for primes up to P) and its estimated hard
// leaves.  A segment whose leaves outweigh both its sieve and a fair share of
// the launch (total / (4 * resident CTAs)) becomes R replicas that share its
// leaves.  Items are handed out largest first from an atomic counter, ordered
// by cost in buckets of a quarter octave (the order only balances the load).
static constexpr int PLAN_BUCKETS = 128;

struct PlanScratch {
    double total;                 // cost of every segment of the run
    unsigned long long nitems;    // items planned
    u32 cnt[PLAN_BUCKETS];        // items per cost bucket
    u32 cur[PLAN_BUCKETS];        // next free slot of each bucket
    u32 nheavy;                   // segments split into replicas
    u32 pad;
};

struct HeavySeg {
    u32 s;     // segment
    u32 pos;   // its first item
    u32 R;     // its replicas (items pos .. pos + R - 1)
    u32 pad;
};

struct PlanArgs {
    const u32* segB;
    const unsigned long long* est;
    u32 k0;
    double x, z;
    u64 span, s0, s1;
    double inv_ctas4;           // 1 / (4 * resident CTAs)
    u64 cap;                    // slots in items
    PlanScratch* scr;
    u32* split;                 // per segment: R | bucket << 16 (R = 0: no item)
    HardItem* items;
    HeavySeg* heavy;            // the segments with R > 1
    unsigned long long* stat;   // [4] items, [5] item steps, [6] set when cap was too small,
                                // [7] steps replicas cross off before their own
};

__device__ __forceinline__ double seg_cost(const PlanArgs& P, u64 s)
{
    const double steps = (double)(P.segB[s] - P.k0);
    const double sz = sqrt(P.z);
    const double pm = s ? fmin(sqrt(P.x / ((double)s * (double)P.span)), sz) : sz;
    const double ll = pm > 16.0 ? log(log(pm)) - 1.0056 : 0.0;
    return 128.0 * steps + 0.08 * (double)P.span * (8.0 / 30.0) * (ll > 0.0 ? ll : 0.0);
}

__global__ void plan_cost_kernel(PlanArgs P)
{
    __shared__ double part[32];
    double t = 0;
    for (u64 s = P.s0 + (u64)blockIdx.x * blockDim.x + threadIdx.x; s < P.s1; s += (u64)gridDim.x * blockDim.x)
        if (P.segB[s] > P.k0) t += seg_cost(P, s) + (double)P.est[s];
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0;
        for (u32 k = 0; k < blockDim.x / 32; k++) b += part[k];
        atomicAdd(&P.scr->total, b);
    }
}

// R and the cost bucket of every segment, decided once and stored
__global__ void plan_split_kernel(PlanArgs P)
{
    const double target = fmax(P.scr->total * P.inv_ctas4, 1.0);
    for (u64 s = P.s0 + (u64)blockIdx.x * blockDim.x + threadIdx.x; s < P.s1; s += (u64)gridDim.x * blockDim.x) {
        u32 v = 0;
        if (P.segB[s] > P.k0) {
            const double base = seg_cost(P, s), e = (double)P.est[s];
            u32 R = 1;
            if (base + e > target && e > base) {
                const double room = fmax(target - base, base);
                R = (u32)fmin(1024.0, ceil(e / fmax(room, 1.0)));
                if (R < 1) R = 1;
            }
            const int k = (int)floor(4.0 * log2((base + e) / R));   // a replica's share
            const u32 key = (u32)(k < 0 ? 0 : (k >= PLAN_BUCKETS ? PLAN_BUCKETS - 1 : k));
            v = R | (key << 16);
            atomicAdd(&P.scr->cnt[key], R);
            atomicAdd(&P.stat[5], (unsigned long long)(P.segB[s] - P.k0));
        }
        P.split[s] = v;
    }
}

// first slot of every bucket, the most costly bucket first (one block)
__global__ void plan_offsets_kernel(PlanArgs P)
{
    if (threadIdx.x != 0) return;
    unsigned long long run = 0;
    for (int k = PLAN_BUCKETS - 1; k >= 0; k--) {
        P.scr->cur[k] = (u32)run;
        run += P.scr->cnt[k];
    }
    if (run > P.cap) {   // cannot happen with cap = segments + 8 * CTAs; the run reports it
        P.stat[6] = 1;
        run = 0;
    }
    P.scr->nitems = run;
    P.stat[4] = run;
}

__global__ void plan_scatter_kernel(PlanArgs P)
{
    if (P.stat[6]) return;
    for (u64 s = P.s0 + (u64)blockIdx.x * blockDim.x + threadIdx.x; s < P.s1; s += (u64)gridDim.x * blockDim.x) {
        const u32 v = P.split[s], R = v & 0xFFFFu;
        if (!R) continue;
        const u32 pos = atomicAdd(&P.scr->cur[v >> 16], R);
        // replica 0 starts at the first step; the others get their steps in plan_bsplit_kernel
        for (u32 r = 0; r < R; r++) P.items[pos + r] = HardItem{(u32)s, r ? ~0u : P.k0 + 1, ~0u, 0u};
        if (R > 1) P.heavy[atomicAdd(&P.scr->nheavy, 1u)] = HeavySeg{(u32)s, pos, R, 0u};
    }
}

// Estimated cost of step b of the segment [L, L + span), in the units of seg_cost (one
// leaf = 1): 128 for the step, 0.08 per crossing, plus its hard leaves (upper bound, as in
// hard_estimate_kernel).  Integer, so that prefix sums are exact.
__device__ __forceinline__ unsigned long long step_cost(const HardArgs& A, u32 b, u64 L, u64 vL, u64 vLs)
{
    const u64 p = A.primes[b], vp = A.primes_rcp[b];
    unsigned long long c = 128 + (16ull * A.seg_bytes / p) / 25;
    if (b > A.kleaf && b <= A.a) {
        const u64 xp = div_rcp(A.x, p, vp);
        u64 mlo, mhi;
        if (leaf_window(A, p, vp, xp, L, vL, vLs, mlo, mhi)) {
            if (p * p > A.y) {
                const u64 k0 = pc_min(pc_max(pi_lookup(A.pit, mlo), b), A.a);
                const u64 k1 = pc_min(pc_max(pi_lookup(A.pit, mhi), b), A.a);
                c += k1 - k0;
            } else {
                c += rank_lookup(A.rk, mhi) - rank_lookup(A.rk, mlo);
            }
        }
    }
    return c;
}

// The steps of a heavy segment's replicas: replica r owns the steps from the first b
// whose cost before it reaches r / R of the segment's total (one CTA per segment; a
// prefix sum of exact integer costs, so every step goes to exactly one replica).
__global__ void __launch_bounds__(256) plan_bsplit_kernel(HardArgs A, PlanArgs P)
{
    __shared__ unsigned long long wsum[8];
    __shared__ unsigned long long s_tot;
    const u32 tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (P.stat[6]) return;
    const u32 nh = P.scr->nheavy;
    for (u32 h = blockIdx.x; h < nh; h += gridDim.x) {
        const HeavySeg hs = P.heavy[h];
        const u64 s = hs.s, L = s * A.span, R = hs.R;
        const u32 Bs = A.segB[s];
        const u64 vL = L ? ~0ull / L : 0, vLs = ~0ull / (L + A.span);
        const u32 nsteps = Bs - A.k0, per = (nsteps + 255) / 256;
        const u32 b0 = pc_min((u64)A.k0 + 1 + (u64)tid * per, (u64)Bs + 1), b1 = pc_min((u64)b0 + per, (u64)Bs + 1);
        unsigned long long mine = 0;
        for (u32 b = b0; b < b1; b++) mine += step_cost(A, b, L, vL, vLs);
        unsigned long long incl = mine;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (tid == 0) {
            unsigned long long run = 0;
            for (u32 k = 0; k < 8; k++) {
                const unsigned long long v = wsum[k];
                wsum[k] = run;
                run += v;
            }
            s_tot = run;
        }
        __syncthreads();
        const unsigned long long T = s_tot;
        unsigned long long before = wsum[wid] + incl - mine;
        for (u32 b = b0; b < b1; b++) {
            const unsigned long long after = before + step_cost(A, b, L, vL, vLs);
            // replicas r with R * before < r * T <= R * after start right after step b
            u64 r_hi = R * after / T;
            if (r_hi > R - 1) r_hi = R - 1;
            for (u64 r = R * before / T + 1; r <= r_hi; r++) {
                P.items[hs.pos + r].b_lo = b + 1;
                P.items[hs.pos + r - 1].b_hi = b + 1;
                if (b + 1 <= Bs) atomicAdd(&P.stat[7], (unsigned long long)(b - A.k0));
            }
            before = after;
        }
        __syncthreads();
    }
}

static size_t hard_smem(const HardArgs& A)
{
    static_assert(sizeof(StepInfo) % 16 == 0, "StepInfo must keep 16-byte alignment");
    return BATCH * sizeof(StepInfo) + A.seg_bytes + (size_t)A.nw * (A.sub_bytes >> 5) * 4 +
           (size_t)BATCH * (A.nw + 1) * 4 + 3 * (size_t)BATCH * A.nw * 4 + (size_t)BATCH * A.nw +
           (size_t)A.nw * LOG_CAP * sizeof(u16);
}

// The instantiation: the most resident warps (registers and shared memory permitting), or
// at least ctas_per_sm resident CTAs when that is set; *per_sm its resident CTAs (<= 8).
template <bool MULTI>
static int choose_hard_kernel(pc_ctx* ctx, const HardArgs& A, size_t smem, void (**out)(HardArgs, MultiArgs),
                              int* out_per_sm)
{
    struct Variant {
        void (*fn)(HardArgs, MultiArgs);
        int maxt, minb;
    };
    static const Variant variants[] = {{hard_sieve_kernel<512, 1, MULTI>, 512, 1},
                                       {hard_sieve_kernel<256, 3, MULTI>, 256, 3},
                                       {hard_sieve_kernel<512, 2, MULTI>, 512, 2},
                                       {hard_sieve_kernel<256, 4, MULTI>, 256, 4}};
    const int nt = 32 * (int)A.nw;
    const int want = (int)(ctx->params.ctas_per_sm ? ctx->params.ctas_per_sm : ctx->ctas_call);
    void (*kern)(HardArgs, MultiArgs) = nullptr;
    int per_sm = 0;
    for (const Variant& v : variants) {
        if (nt > v.maxt) continue;
        // The limit is a property of the kernel, shared by every host thread of the
        // process: always raise it to the device maximum (never to this call's size),
        // so that a concurrent query with larger segments is not cut short.
        cudaFuncAttributes fa;
        PC_CUDA(ctx, cudaFuncGetAttributes(&fa, v.fn));
        const size_t dyn_max = ctx->smem_optin - fa.sharedSizeBytes;
        if (smem > dyn_max) {
            pc_set_error(ctx, "hard-leaf sieve: %zu bytes of shared memory per CTA", smem);
            return PC_EINVAL;
        }
        cudaError_t ea = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
        if (ea != cudaSuccess) {
            pc_set_error(ctx, "cudaFuncSetAttribute(smem=%zu): %s", dyn_max, cudaGetErrorString(ea));
            return PC_ECUDA;
        }
        int fit = 0;   // resident CTAs the SM can hold (registers and shared memory)
        PC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, v.fn, nt, smem));
        if (fit < 1) continue;
        if (want) {
            // the least register-constrained variant reaching the requested residency
            if (!kern || (per_sm < want && fit > per_sm)) {
                kern = v.fn;
                per_sm = fit;
            }
        } else if (fit > per_sm) {
            kern = v.fn;
            per_sm = fit;
        }
    }
    if (!kern) {
        pc_set_error(ctx, "hard-leaf sieve: no launch configuration fits (smem=%zu, threads=%d)", smem, nt);
        return PC_EINVAL;
    }
    if (want && per_sm > want) per_sm = want;
    if (per_sm > 8) per_sm = 8;   // 32 KiB segments fit 4; smaller ones (autotuned, or set) up to 8
    *out = kern;
    *out_per_sm = per_sm;
    return PC_OK;
}

int run_hard_sieve(pc_ctx* ctx, const LeafProblem& P, I128Pair* out)
{
    HardArgs A{};
    A.x = P.x;
    A.y = P.y;
    A.z = P.z;
    A.c = P.c;
    A.k0 = P.c >= 5 ? 5 : (P.c == 4 ? 4 : 3);
    A.kleaf = P.c > A.k0 ? P.c : A.k0;
    A.a = P.a;
    A.trunc = P.trunc;
    const u64 bmax = P.B < P.a ? P.B : P.a;
    if (bmax <= A.kleaf) return PC_OK;   // no hard leaf needs the sieve
    A.bmax = (u32)bmax;
    // 32 KiB segments of four 8 KiB warp sub-ranges: four CTAs fit on an SM
    A.seg_bytes = pc_seg_bytes(ctx, 32768);
    A.sub_bytes = pc_sub_bytes(ctx, A.seg_bytes);
    A.nw = A.seg_bytes / A.sub_bytes;
    A.sub_shift = 3;
    while ((1u << A.sub_shift) < A.sub_bytes * 8) A.sub_shift++;
    A.span = 30ull * A.seg_bytes;
    A.dspan = 30ull * A.sub_bytes;
    A.nseg = P.z / A.span + 1;
    A.s0 = 0;
    A.s1 = A.nseg;
    std::vector<u64> hstart;
    if (P.shard_n) {
        A.s0 = A.nseg * P.shard_k / P.shard_n;
        A.s1 = A.nseg * (P.shard_k + 1) / P.shard_n;
        if (A.s1 <= A.s0) return PC_OK;   // an empty shard
        if (A.s0) {
            // carries into the shard: phi(L - 1, b) for every b (Section 4), computed
            // before this run claims the context's scratch
            hstart.resize(bmax - A.k0 + 1);
            PC_TRY(phi_starts(ctx, A.s0 * A.span - 1, A.k0, bmax, hstart.data()));
        }
    }
    A.pit = ctx->T.pi();
    A.rk = ctx->T.rank();
    A.ml = ctx->T.mlist();
    A.nsl = ctx->T.n_sl;
    for (int k = 0; k < Tables::NSUB; k++) {
        A.sl[k] = ctx->T.sublist(k);
        A.srk[k] = ctx->T.subrank(k);
        A.slK[k] = k < (int)A.nsl ? ctx->T.sl_K[k] : ~0u;
    }
    A.primes = ctx->T.primes.as<u32>();
    A.primes_rcp = ctx->T.primes_rcp.as<u64>();

    const u64 nrows = bmax - A.k0 + 1;
    PC_TRY(buf_reserve(ctx, ctx->seg_b, A.nseg * sizeof(u32) + (nrows + 1) * sizeof(u32)));
    PC_TRY(buf_reserve(ctx, ctx->seg_off, (nrows + 1) * sizeof(u64) + 3 * A.nseg * sizeof(u64) + A.nseg * sizeof(u32) +
                                              A.nseg * sizeof(HeavySeg) + 16));
    u32* segB = ctx->seg_b.as<u32>();
    u32* rowlen = segB + A.nseg;
    u64* off = ctx->seg_off.as<u64>();
    unsigned long long* est = (unsigned long long*)(off + nrows + 1);
    u64* rcp_seg = (u64*)(est + A.nseg);
    u32* split = (u32*)(rcp_seg + 2 * A.nseg);   // the work-item split of every segment
    HeavySeg* heavy = (HeavySeg*)(((uintptr_t)(split + A.nseg) + 15) & ~(uintptr_t)15);
    A.rcp_seg = rcp_seg;
    A.rcp_y = ~0ull / P.y;
    seg_b_kernel<<<(unsigned)((A.nseg + 255) / 256), 256, 0, ctx->stream>>>(P.x, A.nseg, A.span, A.bmax, A.pit, segB,
                                                                            rcp_seg);
    PC_LAUNCHED(ctx);
    row_len_kernel<<<(unsigned)((nrows + 255) / 256), 256, 0, ctx->stream>>>(segB, A.nseg, A.s0, A.s1, A.k0, A.bmax,
                                                                              rowlen);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches += 2;
    PC_TRY(scan_exclusive_u32_to_u64(ctx, rowlen, off, nrows));
    A.segB = segB;
    A.off = off;
    A.start = nullptr;
    if (!hstart.empty()) {
        PC_TRY(buf_reserve(ctx, ctx->starts, hstart.size() * sizeof(u64)));
        PC_CUDA(ctx, cudaMemcpyAsync(ctx->starts.p, hstart.data(), hstart.size() * sizeof(u64),
                                     cudaMemcpyHostToDevice, ctx->stream));
        A.start = ctx->starts.as<u64>();
    }
    u64 total = 0;
    PC_TRY(copy_to_host(ctx, &total, off + nrows, sizeof(u64)));
    if (total >> 32) {
        pc_set_error(ctx, "hard-leaf sieve: %llu count rows exceed 32-bit offsets", (unsigned long long)total);
        return PC_EOVERFLOW;
    }

    const size_t smem = hard_smem(A);
    void (*kern)(HardArgs, MultiArgs) = nullptr;
    int per_sm = 0;
    PC_TRY(choose_hard_kernel<false>(ctx, A, smem, &kern, &per_sm));
    int ctas = ctx->sm_count * per_sm;

    // per-segment leaf estimate, then the work items, all on the device
    PC_CUDA(ctx, cudaMemsetAsync(est, 0, A.nseg * sizeof(u64), ctx->stream));
    if (A.s1 > A.s0) {
        hard_estimate_kernel<<<(unsigned)(((A.s1 - A.s0) * 32 + 255) / 256), 256, 0, ctx->stream>>>(A, est);
        PC_LAUNCHED(ctx);
        ctx->stats.kernel_launches++;
    }
    const u64 cap = (A.s1 - A.s0) + 8ull * (u64)ctas + 64;
    const size_t items_bytes = (size_t)ctas * sizeof(I128Pair) + cap * sizeof(HardItem);
    PC_TRY(buf_reserve(ctx, ctx->counts, total * sizeof(u32)));
    PC_TRY(buf_reserve(ctx, ctx->tallies, total * sizeof(i32)));
    PC_TRY(buf_reserve(ctx, ctx->acc_seg, (items_bytes + 15) / 16 * 16 + sizeof(PlanScratch)));
    PC_TRY(buf_reserve(ctx, ctx->queue, 128));
    HardItem* ditems = (HardItem*)(ctx->acc_seg.as<I128Pair>() + ctas);
    PlanScratch* scr = (PlanScratch*)(ctx->acc_seg.as<unsigned char>() + (items_bytes + 15) / 16 * 16);
    A.counts = ctx->counts.as<u32>();
    A.tallies = ctx->tallies.as<i32>();
    A.items = ditems;
    A.nitems = &scr->nitems;
    A.acc = ctx->acc_seg.as<I128Pair>();
    A.queue = ctx->queue.as<u32>();
    A.stat = (unsigned long long*)(ctx->queue.as<u32>() + 2);
    PC_CUDA(ctx, cudaMemsetAsync(ctx->queue.p, 0, 128, ctx->stream));
    PC_CUDA(ctx, cudaMemsetAsync(scr, 0, sizeof(PlanScratch), ctx->stream));
    PC_CUDA(ctx, cudaMemsetAsync(ctx->tallies.p, 0, total * sizeof(i32), ctx->stream));
    PlanArgs PA{segB, est, A.k0, (double)P.x, (double)P.z, A.span, A.s0, A.s1, 1.0 / (4.0 * ctas), cap,
                scr, split, ditems, heavy, A.stat};
    const unsigned pg = (unsigned)pc_min((A.s1 - A.s0 + 255) / 256, (u64)ctx->sm_count * 4);
    plan_cost_kernel<<<pg, 256, 0, ctx->stream>>>(PA);
    PC_LAUNCHED(ctx);
    plan_split_kernel<<<pg, 256, 0, ctx->stream>>>(PA);
    PC_LAUNCHED(ctx);
    plan_offsets_kernel<<<1, 32, 0, ctx->stream>>>(PA);
    PC_LAUNCHED(ctx);
    plan_scatter_kernel<<<pg, 256, 0, ctx->stream>>>(PA);
    PC_LAUNCHED(ctx);
    plan_bsplit_kernel<<<ctx->sm_count * 2, 256, 0, ctx->stream>>>(A, PA);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches += 5;

    cudaEvent_t e0 = ctx->ev[0], e1 = ctx->ev[1];
    PC_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
    kern<<<ctas, 32 * A.nw, smem, ctx->stream>>>(A, MultiArgs{});
    PC_LAUNCHED(ctx);
    PC_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    ctx->stats.kernel_launches++;

    int g = (int)pc_min(bmax - A.kleaf, 4096);
    PC_TRY(buf_reserve(ctx, ctx->partials, g * sizeof(I128Pair)));
    hard_combine_kernel<256><<<g, 256, 0, ctx->stream>>>(A, ctx->partials.as<I128Pair>());
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    PC_TRY(reduce_i128(ctx, ctx->partials.as<I128Pair>(), g, out));
    PC_TRY(reduce_i128(ctx, A.acc, ctas, out));

    u64 nl[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    PC_TRY(copy_to_host(ctx, nl, A.stat, 8 * sizeof(u64)));
    if (nl[6]) {
        pc_set_error(ctx, "hard-leaf sieve: work items exceed the planned %llu slots", (unsigned long long)cap);
        return PC_EOVERFLOW;
    }
    ctx->stats.work_items = nl[4];
    ctx->stats.item_steps += nl[5];
    ctx->stats.presieve_steps += nl[7];
    ctx->stats.warp_steps += nl[2];
    ctx->stats.leaf_warp_steps += nl[3];
    float ms = 0;
    PC_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
    ctx->stats.ms_hard_sieve = ms;
    ctx->stats.hard_leaves += nl[0];
    ctx->stats.clears += nl[1];
    ctx->stats.segments = A.nseg;
    ctx->stats.steps = total;
    ctx->stats.seg_bytes = A.seg_bytes;
    return PC_OK;
}

// ------------------------------------------------------- many queries at once
// The hard leaves of every pi(x) query of a batch in one sieve launch over all their
// segments (largest queries first, since the batch sorts them so), with the segment
// schedule and the count rows of every query built by one launch each.

// B_s and the reciprocals of L_s, L_s + span for segment g - pref[q] of query q
__global__ void mq_seg_b_kernel(const HardArgs* qa, const u64* pref, u32 Q, u32* segB, u64* rcp_seg)
{
    const u64 g = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= pref[Q]) return;
    const u64 q = mq_find(pref, Q + 1, g);
    const HardArgs& A = qa[q];
    const u64 s = g - pref[q];
    rcp_seg[2 * g] = s ? ~0ull / (s * A.span) : 0;
    rcp_seg[2 * g + 1] = ~0ull / ((s + 1) * A.span);
    u32 B = A.bmax;
    if (s > 0) {
        const u64 r = pc_isqrt(A.x / (s * A.span));
        const u64 pr = pi_lookup(A.pit, r);
        if (pr < B) B = (u32)pr;
    }
    segB[g] = B;
}

// row b = k0 + g - rpref[q] of query q: the number of its segments with B_s >= b
__global__ void mq_row_len_kernel(const HardArgs* qa, const u64* rpref, u32 Q, u32* len)
{
    const u64 g = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= rpref[Q]) return;
    const u64 q = mq_find(rpref, Q + 1, g);
    const HardArgs& A = qa[q];
    const u32 b = A.k0 + (u32)(g - rpref[q]);
    u64 lo = 0, hi = A.nseg;   // first s with segB[s] < b
    while (lo < hi) {
        const u64 mid = (lo + hi) >> 1;
        if (A.segB[mid] >= b) lo = mid + 1; else hi = mid;
    }
    len[g] = (u32)lo;
}

// the carries: a warp per (query, b), kleaf < b <= bmax: the exclusive scan over
// segments of count(., b - 1) dotted with tally(., b), into the query's hard part
__global__ void mq_combine_kernel(const HardArgs* qa, const u64* cpref, u32 Q, I128Pair* parts)
{
    const u32 lane = threadIdx.x & 31;
    const u64 gw = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 g = gw; g < cpref[Q]; g += nwarps) {
        const u64 q = mq_find(cpref, Q + 1, g);
        const HardArgs& A = qa[q];
        const u32 b = A.kleaf + 1 + (u32)(g - cpref[q]);
        const u64 row = A.off[b - A.k0], Sb = A.off[b - A.k0 + 1] - row, prow = A.off[b - 1 - A.k0];
        u64 carry = 0;
        i128 dot = 0;
        for (u64 base = 0; base < Sb; base += 32) {
            const u64 s = base + lane;
            const u64 v = s < Sb ? (u64)A.counts[prow + s] : 0;
            u64 incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                const u64 t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (s < Sb) {
                const i32 tl = A.tallies[row + s];
                if (tl) dot += (i128)tl * (i128)(carry + incl - v);
            }
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        dot = warp_sum_i128(dot);
        if (lane == 0 && dot != 0) mq_atomic_add_i128(parts + 5 * q + 3, dot);
    }
}

int mq_hard(pc_ctx* ctx, const MQPlan& P)
{
    const u32 Q = P.Q;
    HardArgs T{};   // what every query of the batch shares: tables, geometry, queue, counters
    T.k0 = 5;
    T.kleaf = 5;
    T.seg_bytes = pc_seg_bytes(ctx, ctx->batch_seg ? ctx->batch_seg : 16384);
    T.sub_bytes = pc_sub_bytes(ctx, T.seg_bytes);
    T.nw = T.seg_bytes / T.sub_bytes;
    T.sub_shift = 3;
    while ((1u << T.sub_shift) < T.sub_bytes * 8) T.sub_shift++;
    T.span = 30ull * T.seg_bytes;
    T.dspan = 30ull * T.sub_bytes;
    T.pit = ctx->T.pi();
    T.rk = ctx->T.rank();
    T.ml = ctx->T.mlist();
    T.nsl = ctx->T.n_sl;
    for (int k = 0; k < Tables::NSUB; k++) {
        T.sl[k] = ctx->T.sublist(k);
        T.srk[k] = ctx->T.subrank(k);
        T.slK[k] = k < (int)T.nsl ? ctx->T.sl_K[k] : ~0u;
    }
    T.primes = ctx->T.primes.as<u32>();
    T.primes_rcp = ctx->T.primes_rcp.as<u64>();
    // per query: segments, count rows b = k0 .. bmax, carried rows b = kleaf + 1 .. bmax
    std::vector<u64> spref(Q + 1, 0), rpref(Q + 1, 0), cpref(Q + 1, 0);
    std::vector<u32> ipref(Q + 1, 0);
    u64 bound = 0;   // count-row entries: at most segments x rows per query
    for (u32 q = 0; q < Q; q++) {
        const MQ& m = P.hq[q];
        const u64 bmax = m.B < m.a ? m.B : m.a;
        const bool work = m.c == 5 && bmax > T.kleaf;
        const u64 nseg = work ? m.z / T.span + 1 : 0;
        const u64 nrows = work ? bmax - T.k0 + 1 : 0;
        spref[q + 1] = spref[q] + nseg;
        rpref[q + 1] = rpref[q] + nrows;
        cpref[q + 1] = cpref[q] + (work ? bmax - T.kleaf : 0);
        bound += nseg * nrows;
    }
    const u64 S = spref[Q], R = rpref[Q];
    if (S == 0) return PC_OK;
    if (bound >> 32 || S >> 32) {
        pc_set_error(ctx, "batch: %llu count-row entries exceed 32-bit offsets", (unsigned long long)bound);
        return PC_EOVERFLOW;
    }
    for (u32 q = 0; q <= Q; q++) ipref[q] = (u32)spref[q];
    // mq_h: spref | rpref | cpref (Q+1 u64 each) | ipref (Q+1 u32) | segB (S u32) | rcp_seg (2S u64) |
    // rowlen (R u32) | off (R+1 u64) | queue + counters (128 B)
    auto al = [](size_t v) { return (v + 15) / 16 * 16; };
    const size_t o_r = al((Q + 1) * 8), o_c = o_r + al((Q + 1) * 8), o_i = o_c + al((Q + 1) * 8);
    const size_t o_sb = o_i + al((Q + 1) * 4), o_rc = o_sb + al(S * 4), o_rl = o_rc + al(2 * S * 8);
    const size_t o_off = o_rl + al(R * 4), o_q = o_off + al((R + 1) * 8), total = o_q + 128;
    PC_TRY(buf_reserve(ctx, ctx->mq_h, total));
    PC_TRY(buf_reserve(ctx, ctx->mq_hq, Q * sizeof(HardArgs)));
    PC_TRY(buf_reserve(ctx, ctx->counts, bound * sizeof(u32)));
    PC_TRY(buf_reserve(ctx, ctx->tallies, bound * sizeof(i32)));
    unsigned char* base = ctx->mq_h.as<unsigned char>();
    u64* d_spref = (u64*)base;
    u64* d_rpref = (u64*)(base + o_r);
    u64* d_cpref = (u64*)(base + o_c);
    u32* d_ipref = (u32*)(base + o_i);
    u32* d_segB = (u32*)(base + o_sb);
    u64* d_rcp = (u64*)(base + o_rc);
    u32* d_rowlen = (u32*)(base + o_rl);
    u64* d_off = (u64*)(base + o_off);
    u32* d_queue = (u32*)(base + o_q);
    HardArgs* d_qa = ctx->mq_hq.as<HardArgs>();
    std::vector<HardArgs> qa(Q, T);
    for (u32 q = 0; q < Q; q++) {
        const MQ& m = P.hq[q];
        HardArgs& A = qa[q];
        A.x = m.x;
        A.y = m.y;
        A.z = m.z;
        A.c = m.c;
        A.a = m.a;
        A.trunc = false;
        const u64 bmax = m.B < m.a ? m.B : m.a;
        A.bmax = (u32)pc_max(bmax, T.k0);
        A.nseg = spref[q + 1] - spref[q];
        A.s0 = 0;
        A.s1 = A.nseg;
        A.rcp_y = ~0ull / m.y;
        A.segB = d_segB + spref[q];
        A.rcp_seg = d_rcp + 2 * spref[q];
        A.off = d_off + rpref[q];
        A.start = nullptr;
        A.counts = ctx->counts.as<u32>();
        A.tallies = ctx->tallies.as<i32>();
        A.queue = d_queue;
        A.stat = (unsigned long long*)(d_queue + 2);
    }
    cudaStream_t st = ctx->stream;
    if (mq_host_upload(ctx)) {
        PC_CUDA(ctx, cudaMemcpyAsync(d_qa, qa.data(), Q * sizeof(HardArgs), cudaMemcpyHostToDevice, st));
        PC_CUDA(ctx, cudaMemcpyAsync(d_spref, spref.data(), (Q + 1) * 8, cudaMemcpyHostToDevice, st));
        PC_CUDA(ctx, cudaMemcpyAsync(d_rpref, rpref.data(), (Q + 1) * 8, cudaMemcpyHostToDevice, st));
        PC_CUDA(ctx, cudaMemcpyAsync(d_cpref, cpref.data(), (Q + 1) * 8, cudaMemcpyHostToDevice, st));
        PC_CUDA(ctx, cudaMemcpyAsync(d_ipref, ipref.data(), (Q + 1) * 4, cudaMemcpyHostToDevice, st));
    }
    // the sieve's instantiation (its shared-memory attribute set outside any capture)
    T.queue = d_queue;
    T.stat = (unsigned long long*)(d_queue + 2);
    const size_t smem = hard_smem(T);
    if (ctx->mq_mode != MQ_CAPTURE) {
        void (*kern)(HardArgs, MultiArgs) = nullptr;
        int per_sm = 0;
        ctx->ctas_call = ctx->batch_ctas;   // the batch's tuned residency (0: as many as fit)
        const int rc = choose_hard_kernel<true>(ctx, T, smem, &kern, &per_sm);
        ctx->ctas_call = 0;
        PC_TRY(rc);
        ctx->mq_hard_kern = (void*)kern;
        ctx->mq_hard_per_sm = per_sm;
    }
    if (!mq_device_work(ctx)) return scan_exclusive_u32_to_u64(ctx, d_rowlen, d_off, R);   // its scratch only
    PC_CUDA(ctx, cudaMemsetAsync(d_queue, 0, 128, st));
    PC_CUDA(ctx, cudaMemsetAsync(ctx->tallies.p, 0, bound * sizeof(i32), st));
    mq_seg_b_kernel<<<(unsigned)((S + 255) / 256), 256, 0, st>>>(d_qa, d_spref, Q, d_segB, d_rcp);
    PC_LAUNCHED(ctx);
    mq_row_len_kernel<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(d_qa, d_rpref, Q, d_rowlen);
    PC_LAUNCHED(ctx);
    PC_TRY(scan_exclusive_u32_to_u64(ctx, d_rowlen, d_off, R));
    // the sieve: items are the segments of every query, handed out in order
    void (*kern)(HardArgs, MultiArgs) = (void (*)(HardArgs, MultiArgs))ctx->mq_hard_kern;
    const int per_sm = ctx->mq_hard_per_sm;
    const u64 ctas = pc_min((u64)ctx->sm_count * per_sm, S);
    MultiArgs M{d_qa, d_ipref, Q, (unsigned long long)S, P.parts + 3, 5u};
    kern<<<(unsigned)ctas, 32 * T.nw, smem, st>>>(T, M);
    PC_LAUNCHED(ctx);
    if (cpref[Q]) {
        mq_combine_kernel<<<ctx->sm_count * 8, 256, 0, st>>>(d_qa, d_cpref, Q, P.parts);
        PC_LAUNCHED(ctx);
    }
    ctx->stats.kernel_launches += 4;
    return PC_OK;
}
