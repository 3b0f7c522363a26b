// pc_p2.cu -- P2(x, a) = sum over primes y < p <= isqrt(x) of (pi(x/p) - pi(p) + 1).
//
// The values pi(x/p) lie in [isqrt x, z], z = x/y.  The interval [0, z] is
// sieved in the same mod-30 shared-memory segments as the hard-leaf sieve,
// by every prime <= isqrt(z), in any order (no leaf needs an intermediate
// state, so the crossing off is order-free).  In the final state a segment
// holds phi(., B) locally, B = pi(isqrt z), and for v >= p_B
//   pi(v) = phi(v, B) + B - 1.
// Each segment answers the p with x/p inside it by a local count plus a
// tally of how many p it answered; a scan of the per-segment totals then
// supplies phi(L_s - 1, B).  The p themselves are read from the pi table.
#include "pc_internal.h"
#include "pc_sieve.cuh"

struct P2Args {
    u64 x, y, z, r;   // r = isqrt(x)
    u32 B, k0;
    u32 b_mid, b_big;   // first prime index >= P2_COOP_P, and with 8 p > seg_bytes
    u64 nseg;         // segments sieved: s0 .. s0 + nseg - 1 (arrays below indexed from s0)
    u64 s0;           // first segment sieved: those below isqrt(x) hold no x/p (x/p >= isqrt x)
    u32 seg_bytes;
    u64 span;
    PiTable pit;
    const u32* primes;
    const u64* primes_rcp;   // floor((2^64 - 1) / p_b)
    u32* cnt;         // set bits per segment (final state)
    u32* tally;       // number of p answered per segment
    I128Pair* acc;    // sum of local counts per segment
    u32* queue;
    unsigned long long* stat;   // [3]: multiples crossed off (or null)
    const u32* pat;   // presieve pattern of the primes 7..19 (k0 = 8), or null (7 and 11 from patw)
    // bucket sieve (Section 2.3), or null: the primes p_b, b >= b_bkt, are not visited by every
    // segment; segment s crosses off only the bit positions filed in its bucket,
    // bkt[s * bkt_cap + i] for i < bkt_n[s]
    const u32* bkt;
    const u32* bkt_n;
    u32 bkt_cap;
    u32 b_bkt;
};

// Primes below P2_COOP_P have many wheel rounds per segment and are crossed
// off by the whole CTA at once; the medium ones by one thread per (prime,
// residue class); those with fewer than one round per 8 bytes by one thread
// per prime.
static constexpr u32 P2_COOP_P = 512;

// The crossing walks of pc_sieve.cuh with 32-bit offsets, for p < 2^29: a byte offset
// below 2^17 plus p, or an integer offset below 30 * 2^17 plus 6 p, stays below 2^32.
// (P2's primes are at most isqrt(z) < 2^21 whenever y >= iroot3(x).)
#ifndef P2_NARROW
#define P2_NARROW 1
#endif
__device__ __forceinline__ u32 p2_cross_class(u32* bits, u32 seg_bytes, u64 L, u32 p, u64 kstart, u32 j)
{
    const u32 rj = r8(j);
    u64 q = kstart / 30;
    if (30 * q + rj < kstart) q++;
    const u32 pr = p * rj;
    const u32 bit = idx30(pr % 30);
    const u64 byte64 = (u64)p * q + pr / 30;
    const u64 Lb = L / 30;
    if (byte64 < Lb || byte64 - Lb >= seg_bytes) return 0;
    u32 n = 0;
    for (u32 by = (u32)(byte64 - Lb); by < seg_bytes; by += p, n++) {
        const u32 pos = (by << 3) + bit;
        atomicAnd(&bits[pos >> 5], ~(1u << (pos & 31)));
    }
    return n;
}

__device__ __forceinline__ u32 p2_cross_single(u32* bits, u32 seg_bytes, u64 L, u32 p, u64 kstart)
{
    const u64 k = coprime30_at_or_after(kstart);
    const u64 n0 = (u64)p * k;
    const u32 span = 30 * seg_bytes;
    if (n0 - L >= span) return 0;
    u32 r = (u32)(k % 30), rel = (u32)(n0 - L), cnt = 0;
    while (rel < span) {
        cnt++;
        const u32 q30 = rel / 30;
        const u32 pos = q30 * 8 + idx30(rel - 30 * q30);
        atomicAnd(&bits[pos >> 5], ~(1u << (pos & 31)));
        const u32 d = next30(r);
        r += d;
        if (r >= 30) r -= 30;
        rel += p * d;
    }
    return cnt;
}

// A launch over the segments of many queries (the batched form): item g is segment
// g - qpref[q] of query q, with arguments qargs[q] (all with the same segment geometry).
struct P2Multi {
    const P2Args* qargs;
    const u32* qpref;   // nq + 1 entries
    u32 nq;
    unsigned long long items;
};

// Four resident CTAs per SM (32 registers a thread, a few bytes spilled): the barriers
// between a segment's phases then leave other CTAs to issue (P2 of pi(10^18) 7.8 ms against
// 8.4 with three CTAs at 38 registers, 10.4 with two; earlier builds: 27.9 ms with the one
// CTA the registers allowed when unbounded)
template <int NT, bool MULTI>
__global__ void __launch_bounds__(NT, 4) p2_sieve_kernel(P2Args A0, P2Multi M)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u32* bits = (u32*)smem_raw;
    const u32 seg_words = A0.seg_bytes >> 2;
    const u32 nblk = A0.seg_bytes >> 7;
    u32* blk = bits + seg_words;
    u32* pre = blk + nblk;
    const u64* bits64 = (const u64*)bits;
    __shared__ u32 patw[80];
    __shared__ u32 wsum[32];
    __shared__ u32 s_seg;
    __shared__ i128 red[32];
    const u32 tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    make_pattern_words(patw, A0.k0);
    __shared__ __align__(16) unsigned char sA_raw[MULTI ? sizeof(P2Args) : 16];
    __shared__ u32 s_q;
    u32 cur_q = ~0u;

    for (;;) {
        if (tid == 0) s_seg = atomicAdd(A0.queue, 1u);
        __syncthreads();
        u64 s = s_seg;
        __syncthreads();
        if (MULTI) {
            if (s >= M.items) break;
            if (tid == 0) {   // the item's query: the last q with qpref[q] <= item
                u32 lo = 0, hi = M.nq;
                while (hi - lo > 1) {
                    const u32 mid = (lo + hi) >> 1;
                    if (M.qpref[mid] <= s) lo = mid; else hi = mid;
                }
                s_q = lo;
            }
            __syncthreads();
            const u32 q = s_q;
            if (q != cur_q) {
                const u32* src = (const u32*)(M.qargs + q);
                for (u32 k = tid; k < sizeof(P2Args) / 4; k += NT) ((u32*)sA_raw)[k] = src[k];
                cur_q = q;
                __syncthreads();
            }
            s -= M.qpref[q];
        } else if (s >= A0.nseg) {
            break;
        }
        const P2Args& A = MULTI ? *(const P2Args*)sA_raw : A0;
        const u64 L = (s + A.s0) * A.span;
        if (A.pat) fill_pattern_global(bits, seg_words, L, A.pat, WHEEL19_PERIOD);
        else fill_pattern(bits, seg_words, L, patw, A.k0);
        u32 ncl = 0;
        __syncthreads();
        const u64 end = L + A.span;
        // cross off p_b, k0 < b <= B (the prime itself included)
        auto none = [](u32) {};
        for (u32 b = A.k0 + 1; b < A.b_mid; b++) {
            const u64 p = A.primes[b];
            u64 ks = L ? div_rcp(L + p - 1, p, A.primes_rcp[b]) : 0;
            if (ks < p) ks = p;
            ncl += cross_off_coop(bits, A.seg_bytes, L, (u32)p, ks, tid, NT, none);
        }
        for (u32 task = tid; task < 8 * (A.b_big - A.b_mid); task += NT) {
            const u32 bb = A.b_mid + (task >> 3);
            const u64 p = A.primes[bb];
            u64 ks = L ? div_rcp(L + p - 1, p, A.primes_rcp[bb]) : 0;
            if (ks < p) ks = p;
            ncl += P2_NARROW && p < (1u << 29) ? p2_cross_class(bits, A.seg_bytes, L, (u32)p, ks, task & 7)
                             : cross_off_class(bits, A.seg_bytes, L, (u32)p, ks, task & 7, none);
        }
        const u32 b_end = A.bkt ? A.b_bkt : A.B + 1;
        for (u32 bb = A.b_big + tid; bb < b_end; bb += NT) {
            const u64 p = A.primes[bb];
            u64 ks = L ? div_rcp(L + p - 1, p, A.primes_rcp[bb]) : 0;
            if (ks < p) ks = p;
            ncl += P2_NARROW && p < (1u << 29) ? p2_cross_single(bits, A.seg_bytes, L, (u32)p, ks)
                             : cross_off_single(bits, A.seg_bytes, L, (u32)p, ks, none);
        }
        if (A.bkt) {   // the larger primes: only the multiples filed in this segment's bucket
            const u32 nf = pc_min(A.bkt_n[s], A.bkt_cap);
            const u32* e = A.bkt + s * A.bkt_cap;
            for (u32 i = tid; i < nf; i += NT) {
                const u32 pos = e[i];
                atomicAnd(&bits[pos >> 5], ~(1u << (pos & 31)));
                ncl++;
            }
        }
        // the sieving primes themselves (only in the first segments)
        for (u32 bb = A.k0 + 1 + tid; bb <= A.B; bb += NT) {
            const u64 p = A.primes[bb];
            if (p >= end) break;
            if (p >= L) {
                u32 pos = seg_pos(p, L);
                atomicAnd(&bits[pos >> 5], ~(1u << (pos & 31)));
            }
        }
        if (A.stat) {
            ncl = __reduce_add_sync(0xffffffffu, ncl);
            if (lane == 0 && ncl) atomicAdd(A.stat + 3, (unsigned long long)ncl);
        }
        __syncthreads();
        for (u32 k = wid; k < nblk; k += NT / 32) {   // a warp per 1024-bit block: no bank conflicts
            const u32 c = __reduce_add_sync(0xffffffffu, (u32)__popc(bits[32 * k + lane]));
            if (lane == 0) blk[k] = c;
        }
        __syncthreads();
        // exclusive scan of the block counts
        {
            const u32 per = (nblk + NT - 1) / NT;
            u32 b0 = tid * per, b1 = b0 + per < nblk ? b0 + per : nblk;
            u32 loc = 0;
            for (u32 k = b0; k < b1; k++) loc += blk[k];
            u32 incl = loc;
            for (int o = 1; o < 32; o <<= 1) {
                u32 v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) wsum[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                u32 w = lane < NT / 32 ? wsum[lane] : 0, wi = w;
                for (int o = 1; o < 32; o <<= 1) {
                    u32 v = __shfl_up_sync(0xffffffffu, wi, o);
                    if (lane >= o) wi += v;
                }
                if (lane < NT / 32) wsum[lane] = wi - w;
            }
            __syncthreads();
            u32 run = wsum[wid] + incl - loc;
            for (u32 k = b0; k < b1; k++) {
                pre[k] = run;
                run += blk[k];
            }
            if (tid == NT - 1) pre[nblk] = run;
        }
        __syncthreads();
        // the p with x/p in [L, end): p in (x/end, x/L], y < p <= r
        u64 plo = pc_max(A.x / end, A.y);       // exclusive
        u64 phi = L ? pc_min(A.x / L, A.r) : A.r;
        i64 acc = 0;
        u32 tl = 0;
        if (phi > plo) {
            const u64 w0 = (plo + 1) / 240, w1 = phi / 240;
            for (u64 w = w0 + tid; w <= w1; w += NT) {
                u64 v = A.pit.rec[w].bits;
                while (v) {
                    int bi = __ffsll((long long)v) - 1;
                    v &= v - 1;
                    u64 p = 240 * w + 30 * (u64)(bi >> 3) + r8(bi & 7);
                    if (p <= plo || p > phi) continue;
                    u64 q = A.x / p;
                    u32 e = seg_count_end(q, L);
                    u32 eb = e >> 10, ew = e >> 6;
                    u32 c = pre[eb];
                    for (u32 ww = eb << 4; ww < ew; ww++) c += __popcll(bits64[ww]);
                    if (e & 63) c += __popcll(bits64[ew] & ((1ull << (e & 63)) - 1));
                    acc += c;
                    tl++;
                }
            }
        }
        for (int o = 16; o; o >>= 1) tl += __shfl_xor_sync(0xffffffffu, tl, o);
        __syncthreads();
        if (lane == 0) wsum[wid] = tl;
        __syncthreads();
        i128 tot = block_sum_i128((i128)acc, red);
        if (tid == 0) {
            u32 t = 0;
            for (u32 w = 0; w < NT / 32; w++) t += wsum[w];
            A.tally[s] = t;
            A.cnt[s] = pre[nblk];
            store_i128(A.acc + s, tot);
        }
    }
}

// sum_s acc[s] + tally[s] * phi(L_s - 1, B), phi(L_s - 1, B) = sum_{s'<s} cnt[s']
__global__ void p2_combine_kernel(P2Args A, I128Pair* out)
{
    __shared__ u64 wsum[32];
    __shared__ u64 s_carry;
    __shared__ i128 red[32];
    const u32 lane = threadIdx.x & 31, wid = threadIdx.x >> 5, NT = blockDim.x;
    if (threadIdx.x == 0) {
        // phi(L_s0 - 1, B) for the segments not sieved: L_s0 - 1 < isqrt(x) < p_(B+1)^2, so it is
        // pi(L_s0 - 1) - B + 1 from the pi table, or 1 (the integer 1 alone) below p_B
        u64 c = 0;
        if (A.s0) {
            const u64 v = A.s0 * A.span - 1;
            c = v >= A.primes[A.B] ? pi_lookup(A.pit, v) - A.B + 1 : 1;
        }
        s_carry = c;
    }
    __syncthreads();
    i128 dot = 0;
    for (u64 base = 0; base < A.nseg; base += NT) {
        const u64 s = base + threadIdx.x;
        const u64 v = s < A.nseg ? A.cnt[s] : 0;
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
        if (s < A.nseg) dot += load_i128(A.acc + s) + (i128)A.tally[s] * (i128)carry;
        __syncthreads();
        if (threadIdx.x == NT - 1) s_carry = c0 + wsum[wid] + incl;
        __syncthreads();
    }
    dot = block_sum_i128(dot, red);
    if (threadIdx.x == 0) store_i128(out, load_i128(out) + dot);
}

// tiny z (fewer than 3 sieving primes): every pi(x/p) straight from the pi table
__global__ void p2_lookup_kernel(u64 x, u64 y, u64 r, PiTable pit, I128Pair* out)
{
    __shared__ i128 red[32];
    i128 s = 0;
    for (u64 p = y + 1 + threadIdx.x; p <= r; p += blockDim.x) {
        u64 pp = pi_lookup(pit, p);
        if (pp == pi_lookup(pit, p - 1)) continue;   // p not prime
        s += (i128)pi_lookup(pit, x / p) - (i128)pp + 1;
    }
    s = block_sum_i128(s, red);
    if (threadIdx.x == 0) store_i128(out, load_i128(out) + s);
}

// The constant part of P2, (K - a)(B - 1) - sum_{k=a+1}^{K} (k - 1), K = pi(isqrt x),
// B = pi(isqrt z), added to *out: every pi(x/p_k) = phi(x/p_k, B) + B - 1 and pi(p_k) = k.
__global__ void p2_constant_kernel(u64 K, u64 a, u64 B, I128Pair* out)
{
    const i128 n = (i128)(K - a);
    const i128 sum_k1 = ((i128)K * (i128)(K - 1) - (i128)a * (i128)(a ? a - 1 : 0)) / 2;   // sum_{k=a+1}^{K} (k - 1)
    store_i128(out, load_i128(out) + n * (i128)(B - 1) - sum_k1);
}

// ------------------------------------------------------------- bucket sieve
// Section 2.3 suggests a bucket sieve: each sieving prime waits in the bucket of the next
// interval that holds one of its multiples, so an interval meets only the primes that cross
// something off in it.  Here the buckets are filled a wave of segments at a time: one
// thread per (prime, residue class) walks the class's multiples k p (k >= p) inside the wave
// and files each under its segment; the sieve kernel then applies them.  The primes taken
// this way are those above the segment's bytes, which have at most one multiple per residue
// class in a segment.

// Bound on the entries one segment's bucket can receive: a prime p has m = floor((span - 1)
// / p) + 1 or fewer multiples k p among span consecutive integers, with consecutive k; for
// p > seg_bytes, m <= 30, and at most 8 of 30 consecutive k are coprime to 30, so at most
// min(m, 8) of them are filed.  One CTA.
__global__ void p2_bucket_bound_kernel(P2Args A, unsigned long long* out)
{
    __shared__ unsigned long long part[32];
    unsigned long long s = 0;
    for (u32 b = A.b_bkt + threadIdx.x; b <= A.B; b += blockDim.x) {
        const u64 m = (A.span - 1) / A.primes[b] + 1;
        s += m < 8 ? m : 8;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (u32 w = 0; w < blockDim.x / 32; w++) t += part[w];
        *out = t;
    }
}

// Work of the fill: the multiples of one (prime, residue class) inside a wave are cut into
// chunks of at most P2_FILL_CHUNK, one thread each, so that the threads of small primes (many
// multiples per wave) do not hold up the launch.  pref[i] counts the threads of the bucket
// primes before p_(b_bkt + i): 8 classes x ceil((floor(W span / (30 p)) + 1) / P2_FILL_CHUNK).
static constexpr u32 P2_FILL_CHUNK = 64;
__global__ void p2_bucket_chunks_kernel(P2Args A, u32 W, u32* nthr)
{
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > A.B - A.b_bkt) return;
    const u64 p = A.primes[A.b_bkt + i];
    const u64 mult = (u64)W * A.span / (30 * p) + 1;   // multiples of one class in a wave, at most
    nthr[i] = 8 * (u32)((mult + P2_FILL_CHUNK - 1) / P2_FILL_CHUNK);
}

// Files the multiples k p (k >= p, k = R8[j] mod 30) of the bucket primes that lie in the
// segments w0 .. w0 + W - 1 of A (W * span < 2^32, W <= P2_WAVE_MAX): thread t takes chunk c
// of (prime p_b, class j), found from pref (nb + 1 entries).  A CTA first counts its entries
// per segment in shared memory, reserves a range of every segment's bucket with one global
// atomic, then files its entries there, so the global atomics do not grow with the entries.
// A full bucket sets *err and drops the entry (the bound of p2_bucket_bound_kernel rules that
// out).
static constexpr u32 P2_WAVE_MAX = 4096;
__global__ void __launch_bounds__(256) p2_bucket_fill_kernel(P2Args A, u64 w0, u32 W, const u32* pref, u32 nb,
                                                             u32* bkt, u32* bkt_n, u32 cap, int* err)
{
    __shared__ u32 hist[P2_WAVE_MAX], base[P2_WAVE_MAX];
    for (u32 i = threadIdx.x; i < W; i += blockDim.x) hist[i] = 0;
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    const u64 Lw = (A.s0 + w0) * A.span;   // the wave's first integer
    const u32 wspan = W * (u32)A.span;     // its length
    u64 rel_lo = wspan, rel_hi = wspan;    // this thread's offsets in the wave (none)
    u32 step = 0;
    if (t < pref[nb]) {
        u32 lo = 0, hi = nb;               // the last i with pref[i] <= t
        while (hi - lo > 1) {
            const u32 mid = (lo + hi) >> 1;
            if (pref[mid] <= t) lo = mid; else hi = mid;
        }
        const u32 r = t - pref[lo], j = r & 7, c = r >> 3, b = A.b_bkt + lo;
        const u64 p = A.primes[b];
        u64 k = Lw ? div_rcp(Lw + p - 1, p, A.primes_rcp[b]) : 0;
        if (k < p) k = p;
        const u32 rj = r8(j);
        u64 q = k / 30;
        if (30 * q + rj < k) q++;
        step = 30 * (u32)p;
        const u64 n0 = (30 * q + rj) * p + (u64)c * P2_FILL_CHUNK * step;
        if (n0 - Lw < wspan) {
            rel_lo = n0 - Lw;
            rel_hi = pc_min((u64)wspan, rel_lo + (u64)P2_FILL_CHUNK * step);
        }
    }
    __syncthreads();
    const u32 sp = (u32)A.span;
    for (u64 rel = rel_lo; rel < rel_hi; rel += step) atomicAdd(&hist[(u32)rel / sp], 1u);
    __syncthreads();
    for (u32 i = threadIdx.x; i < W; i += blockDim.x) {
        const u32 h = hist[i];
        base[i] = h ? atomicAdd(&bkt_n[i], h) : 0;
        hist[i] = 0;
    }
    __syncthreads();
    for (u64 rel = rel_lo; rel < rel_hi; rel += step) {
        const u32 sl = (u32)rel / sp, r = (u32)rel - sl * sp;
        const u32 pos = (r / 30) * 8 + idx30(r % 30);
        const u32 slot = base[sl] + atomicAdd(&hist[sl], 1u);
        if (slot < cap) bkt[(u64)sl * cap + slot] = pos;
        else *err = 1;
    }
}

// The sieve of P2 with bucket primes: waves of W segments, each with its buckets filed
// first; W from the bound on a bucket's entries and a budget of 2^26 entries (256 MiB), so
// the buckets' memory does not grow with the number of segments.
static int run_p2_buckets(pc_ctx* ctx, const P2Args& A, int ctas, size_t smem)
{
    PC_TRY(buf_reserve(ctx, ctx->p2_bkt, 256));
    p2_bucket_bound_kernel<<<1, 1024, 0, ctx->stream>>>(A, ctx->p2_bkt.as<unsigned long long>());
    PC_LAUNCHED(ctx);
    u64 cap = 0;
    PC_TRY(copy_to_host(ctx, &cap, ctx->p2_bkt.p, sizeof(u64)));
    // bucket entries per wave: 2^26 (256 MiB; with the fill one thread per (prime, class),
    // pi(1e18)'s P2 at 4 KiB segments took 70.7 ms with 2^24, 57.9 with 2^26, 55.6 with 2^27)
    constexpr u64 P2_BKT_BUDGET = 1ull << 26;
    if (cap == 0 || cap > P2_BKT_BUDGET) {
        pc_set_error(ctx, "p2 buckets: %llu entries per segment", (unsigned long long)cap);
        return PC_EINVAL;
    }
    u64 W = P2_BKT_BUDGET / cap;
    W = pc_min(W, A.nseg);
    W = pc_min(W, (u64)0xFFFFFFFFu / A.span);   // the fill kernel's offsets inside a wave are 32-bit
    W = pc_min(W, (u64)P2_WAVE_MAX);              // and its per-segment counters fit in shared memory
    if (W == 0) W = 1;
    const u32 nb = A.B + 1 - A.b_bkt;            // bucket primes
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t o_cnt = 256, o_pref = o_cnt + al((size_t)(nb + 1) * sizeof(u32));
    const size_t o_bkt = o_pref + al((size_t)(nb + 1) * sizeof(u32));
    const size_t o_n = o_bkt + al((size_t)(W * cap * sizeof(u32)));
    const size_t o_err = o_n + al((size_t)W * sizeof(u32));
    PC_TRY(buf_reserve(ctx, ctx->p2_bkt, o_err + 256));
    unsigned char* base = ctx->p2_bkt.as<unsigned char>();
    u32* d_cnt = (u32*)(base + o_cnt);
    u32* d_pref = (u32*)(base + o_pref);
    u32* d_bkt = (u32*)(base + o_bkt);
    u32* d_n = (u32*)(base + o_n);
    int* d_err = (int*)(base + o_err);
    // the fill's threads: chunks of every (prime, class), the same layout for every wave
    p2_bucket_chunks_kernel<<<(nb + 255) / 256, 256, 0, ctx->stream>>>(A, (u32)W, d_cnt);
    PC_LAUNCHED(ctx);
    PC_TRY(scan_exclusive_u32_to_u32(ctx, d_cnt, d_pref, nb));
    u32 threads = 0;
    PC_TRY(copy_to_host(ctx, &threads, d_pref + nb, sizeof(u32)));
    PC_CUDA(ctx, cudaMemsetAsync(d_err, 0, sizeof(int), ctx->stream));
    PC_CUDA(ctx, cudaEventRecord(ctx->ev[4], ctx->stream));
    for (u64 w0 = 0; w0 < A.nseg; w0 += W) {
        const u32 Wc = (u32)pc_min(W, A.nseg - w0);
        PC_CUDA(ctx, cudaMemsetAsync(d_n, 0, Wc * sizeof(u32), ctx->stream));
        p2_bucket_fill_kernel<<<(threads + 255) / 256, 256, 0, ctx->stream>>>(A, w0, Wc, d_pref, nb, d_bkt, d_n,
                                                                            (u32)cap, d_err);
        PC_LAUNCHED(ctx);
        PC_CUDA(ctx, cudaMemsetAsync(A.queue, 0, 64, ctx->stream));
        P2Args Aw = A;
        Aw.s0 = A.s0 + w0;
        Aw.nseg = Wc;
        Aw.cnt = A.cnt + w0;
        Aw.tally = A.tally + w0;
        Aw.acc = A.acc + w0;
        Aw.bkt = d_bkt;
        Aw.bkt_n = d_n;
        Aw.bkt_cap = (u32)cap;
        p2_sieve_kernel<512, false><<<(unsigned)pc_min((u64)ctas, (u64)Wc), 512, smem, ctx->stream>>>(Aw,
                                                                                                     P2Multi{});
        PC_LAUNCHED(ctx);
        ctx->stats.kernel_launches += 2;
    }
    PC_CUDA(ctx, cudaEventRecord(ctx->ev[5], ctx->stream));
    int err = 0;
    PC_TRY(copy_to_host(ctx, &err, d_err, sizeof(int)));
    if (err) {
        pc_set_error(ctx, "p2 buckets: a bucket overflowed its bound (internal)");
        return PC_EOVERFLOW;
    }
    ctx->stats.kernel_launches += 1;
    return PC_OK;
}

int run_p2(pc_ctx* ctx, u64 x, u64 y, u64 a, I128Pair* out)
{
    const u64 r = pc_isqrt(x);
    if (r <= y) return PC_OK;
    const u64 z = x / y;
    u64 vals[3] = {r, pc_isqrt(z), 0};
    u64 pv[3];
    PC_TRY(tables_pi_values(ctx, vals, pv, 2));
    const u64 K = pv[0], B = pv[1];
    if (K <= a) return PC_OK;
    if (B < 3) {
        p2_lookup_kernel<<<1, 256, 0, ctx->stream>>>(x, y, r, ctx->T.pi(), out);
        PC_LAUNCHED(ctx);
        ctx->stats.kernel_launches++;
        return PC_OK;
    }
    P2Args A{};
    A.x = x;
    A.y = y;
    A.z = z;
    A.r = r;
    A.B = (u32)B;
    // 7..19 from the presieve pattern when they are all sieving primes (k0 = 8),
    // else 7 and 11 from the small pattern
    A.k0 = B >= 5 ? 5 : (u32)B;
    A.pat = nullptr;
    if (B >= 8 && ctx->T.wheel19.bytes) {
        A.k0 = 8;
        A.pat = ctx->T.wheel19.as<u32>();
    }
    // 32 KiB segments up to z = 2^30, 64 KiB up to 2^32, 48 KiB beyond (measured on
    // GB300: the small segments win by a third at z ~ 1e8 and lose a few percent at
    // z ~ 1.5e9; 48 KiB against 64 KiB: pi(1e17) P2 2.45 -> 2.38 ms, pi(1e18) 8.9 -> 8.5 ms)
    const bool bucket = ctx->params.p2_bucket != 0;
    A.seg_bytes = bucket ? pc_seg_bytes(ctx, 4096)
                         : pc_seg_bytes(ctx, A.z < (1ull << 30) ? 32768 : A.z < (1ull << 32) ? 65536 : 49152);
    A.span = 30ull * A.seg_bytes;
    {
        u64 v2[2] = {P2_COOP_P - 1, A.seg_bytes / 8}, pv2[2];
        PC_TRY(tables_pi_values(ctx, v2, pv2, 2));
        A.b_mid = (u32)pc_min(pc_max(pv2[0] + 1, (u64)A.k0 + 1), B + 1);
        A.b_big = (u32)pc_min(pc_max(pv2[1] + 1, (u64)A.b_mid), B + 1);
    }
    A.s0 = r / A.span;                   // r <= z since y < r
    A.nseg = z / A.span + 1 - A.s0;
    A.bkt = nullptr;
    A.bkt_n = nullptr;
    A.bkt_cap = 0;
    A.b_bkt = (u32)B + 1;
    if (bucket) {   // bucket primes: p > seg_bytes, at most one multiple per residue class in a segment
        u64 v1 = A.seg_bytes, pv1 = 0;
        PC_TRY(tables_pi_values(ctx, &v1, &pv1, 1));
        A.b_bkt = (u32)pc_min(pc_max(pv1 + 1, (u64)A.b_big), B + 1);
    }
    A.pit = ctx->T.pi();
    A.primes = ctx->T.primes.as<u32>();
    A.primes_rcp = ctx->T.primes_rcp.as<u64>();
    PC_TRY(buf_reserve(ctx, ctx->counts, A.nseg * 2 * sizeof(u32)));
    PC_TRY(buf_reserve(ctx, ctx->acc_seg, A.nseg * sizeof(I128Pair)));
    PC_TRY(buf_reserve(ctx, ctx->queue, 64));
    PC_CUDA(ctx, cudaMemsetAsync(ctx->queue.p, 0, 64, ctx->stream));
    A.cnt = ctx->counts.as<u32>();
    A.tally = A.cnt + A.nseg;
    A.acc = ctx->acc_seg.as<I128Pair>();
    A.queue = ctx->queue.as<u32>();
    const u32 nblk = A.seg_bytes >> 7;
    size_t smem = A.seg_bytes + (2 * (size_t)nblk + 2) * sizeof(u32);
    // the kernel's limit is shared by every host thread: set the device maximum
    cudaFuncAttributes fa;
    PC_CUDA(ctx, cudaFuncGetAttributes(&fa, p2_sieve_kernel<512, false>));
    const size_t dyn_max = ctx->smem_optin - fa.sharedSizeBytes;
    if (smem > dyn_max) {
        pc_set_error(ctx, "p2 sieve: %zu bytes of shared memory per CTA", smem);
        return PC_EINVAL;
    }
    cudaError_t e = cudaFuncSetAttribute(p2_sieve_kernel<512, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn_max);
    if (e != cudaSuccess) {
        pc_set_error(ctx, "p2 smem attribute: %s", cudaGetErrorString(e));
        return PC_ECUDA;
    }
    int per_sm = (int)(ctx->smem_optin / (smem + 4096));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 4) per_sm = 4;
    int ctas = ctx->sm_count * per_sm;
    if ((u64)ctas > A.nseg) ctas = (int)A.nseg;
    A.stat = ctx->dstat;
    if (A.b_bkt <= B) {
        PC_TRY(run_p2_buckets(ctx, A, ctas, smem));
    } else {
        PC_CUDA(ctx, cudaEventRecord(ctx->ev[4], ctx->stream));
        p2_sieve_kernel<512, false><<<ctas, 512, smem, ctx->stream>>>(A, P2Multi{});
        PC_LAUNCHED(ctx);
        PC_CUDA(ctx, cudaEventRecord(ctx->ev[5], ctx->stream));
    }
    ctx->p2_timed = true;
    p2_combine_kernel<<<1, 1024, 0, ctx->stream>>>(A, out);
    PC_LAUNCHED(ctx);
    p2_constant_kernel<<<1, 1, 0, ctx->stream>>>(K, a, B, out);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches += 3;
    return PC_OK;
}

// ------------------------------------------------------- many queries at once
// P2 of every query of a batch: one sieve launch over the segments of all their
// intervals [0, z], then a warp per query for its carries and the closed-form part.

// query q: sum_s acc[s] + tally[s] * phi(L_s - 1, B) + (K - a)(B - 1) - sum_{k=a+1}^{K} (k - 1)
__global__ void mq_p2_combine_kernel(const P2Args* qa, const MQ* qs, u32 Q, I128Pair* parts)
{
    const u32 lane = threadIdx.x & 31;
    const u64 q = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;
    const P2Args& A = qa[q];
    const MQ m = qs[q];
    if (m.K <= m.a || A.nseg == 0) return;
    u64 carry = 0;
    i128 dot = 0;
    for (u64 base = 0; base < A.nseg; base += 32) {
        const u64 s = base + lane;
        const u64 v = s < A.nseg ? (u64)A.cnt[s] : 0;
        u64 incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const u64 t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (s < A.nseg) dot += load_i128(A.acc + s) + (i128)A.tally[s] * (i128)(carry + incl - v);
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    dot = warp_sum_i128(dot);
    if (lane == 0) {
        const i128 K = (i128)m.K, a = (i128)m.a;
        dot += (K - a) * (i128)(m.B - 1) - (K * (K - 1) - a * (a ? a - 1 : 0)) / 2;
        store_i128(parts + 5 * q + 4, dot);
    }
}

// pi(x) = S1 + S2_triv + S2_easy + S2_hard + a - 1 - P2 for every query
__global__ void mq_final_kernel(const MQ* qs, u32 Q, const I128Pair* parts, u64* out, int* bad)
{
    const u32 q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    const I128Pair* pq = parts + 5 * q;
    const i128 pi = load_i128(pq) + load_i128(pq + 1) + load_i128(pq + 2) + load_i128(pq + 3) + (i128)qs[q].a - 1 -
                    load_i128(pq + 4);
    if (pi < 0 || (pi >> 64) != 0) *bad = 1;
    out[q] = (u64)pi;
}

int mq_final(pc_ctx* ctx, const MQPlan& P, u64* d_out, int* d_bad)
{
    if (!mq_device_work(ctx)) return PC_OK;
    mq_final_kernel<<<(P.Q + 127) / 128, 128, 0, ctx->stream>>>(P.dq, P.Q, P.parts, d_out, d_bad);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    return PC_OK;
}

int mq_p2(pc_ctx* ctx, const MQPlan& P)
{
    const u32 Q = P.Q;
    P2Args T{};
    T.k0 = 5;
    T.seg_bytes = 32768;
    T.span = 30ull * T.seg_bytes;
    T.pit = ctx->T.pi();
    T.primes = ctx->T.primes.as<u32>();
    T.primes_rcp = ctx->T.primes_rcp.as<u64>();
    u64 v2[2] = {P2_COOP_P - 1, T.seg_bytes / 8}, pv2[2];
    if (ctx->mq_mode == MQ_CAPTURE) {   // a read-back: taken in the prepare pass
        pv2[0] = ctx->mq_p2_pv[0];
        pv2[1] = ctx->mq_p2_pv[1];
    } else {
        PC_TRY(tables_pi_values(ctx, v2, pv2, 2));
        ctx->mq_p2_pv[0] = pv2[0];
        ctx->mq_p2_pv[1] = pv2[1];
    }
    std::vector<u64> spref(Q + 1, 0);
    for (u32 q = 0; q < Q; q++) {
        const MQ& m = P.hq[q];
        const bool work = m.c == 5 && m.K > m.a && m.B >= 5;
        spref[q + 1] = spref[q] + (work ? m.z / T.span + 1 : 0);
    }
    const u64 S = spref[Q];
    if (S >> 32) {
        pc_set_error(ctx, "batch: %llu P2 segments", (unsigned long long)S);
        return PC_EOVERFLOW;
    }
    // mq_p: per-query arguments (Q P2Args) | ipref (Q+1 u32) | cnt, tally (S u32 each) |
    // acc (S I128Pair) | queue (64 B)
    auto al = [](size_t v) { return (v + 15) / 16 * 16; };
    const size_t o_ip = al(Q * sizeof(P2Args));
    const size_t o_cnt = o_ip + al((Q + 1) * 4), o_tl = o_cnt + al(S * 4), o_acc = o_tl + al(S * 4);
    const size_t o_q = o_acc + al(S * sizeof(I128Pair)), total = o_q + 64;
    PC_TRY(buf_reserve(ctx, ctx->mq_p, total));
    unsigned char* base = ctx->mq_p.as<unsigned char>();
    P2Args* d_qa = (P2Args*)base;
    u32* d_ipref = (u32*)(base + o_ip);
    u32* d_cnt = (u32*)(base + o_cnt);
    u32* d_tally = (u32*)(base + o_tl);
    I128Pair* d_acc = (I128Pair*)(base + o_acc);
    u32* d_queue = (u32*)(base + o_q);
    std::vector<P2Args> qa(Q, T);
    std::vector<u32> ipref(Q + 1);
    for (u32 q = 0; q <= Q; q++) ipref[q] = (u32)spref[q];
    for (u32 q = 0; q < Q; q++) {
        const MQ& m = P.hq[q];
        P2Args& A = qa[q];
        A.x = m.x;
        A.y = m.y;
        A.z = m.z;
        A.r = pc_isqrt(m.x);
        A.B = (u32)m.B;
        A.b_mid = (u32)pc_min(pc_max(pv2[0] + 1, (u64)A.k0 + 1), m.B + 1);
        A.b_big = (u32)pc_min(pc_max(pv2[1] + 1, (u64)A.b_mid), m.B + 1);
        A.nseg = spref[q + 1] - spref[q];
        A.cnt = d_cnt + spref[q];
        A.tally = d_tally + spref[q];
        A.acc = d_acc + spref[q];
        A.queue = d_queue;
        A.stat = nullptr;
    }
    cudaStream_t st = ctx->stream;
    if (mq_host_upload(ctx)) {
        PC_CUDA(ctx, cudaMemcpyAsync(d_qa, qa.data(), Q * sizeof(P2Args), cudaMemcpyHostToDevice, st));
        PC_CUDA(ctx, cudaMemcpyAsync(d_ipref, ipref.data(), (Q + 1) * 4, cudaMemcpyHostToDevice, st));
    }
    const u32 nblk = T.seg_bytes >> 7;
    const size_t smem = T.seg_bytes + (2 * (size_t)nblk + 2) * sizeof(u32);
    if (S && ctx->mq_mode != MQ_CAPTURE) {   // the shared-memory limit, set outside any capture
        cudaFuncAttributes fa;
        PC_CUDA(ctx, cudaFuncGetAttributes(&fa, p2_sieve_kernel<512, true>));
        const size_t dyn_max = ctx->smem_optin - fa.sharedSizeBytes;
        if (smem > dyn_max) return PC_EINVAL;
        PC_CUDA(ctx, cudaFuncSetAttribute(p2_sieve_kernel<512, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)dyn_max));
    }
    if (!mq_device_work(ctx)) return PC_OK;
    PC_CUDA(ctx, cudaMemsetAsync(d_queue, 0, 64, st));
    if (S) {
        int per_sm = (int)(ctx->smem_optin / (smem + 4096));
        if (per_sm < 1) per_sm = 1;
        if (per_sm > 4) per_sm = 4;
        const u64 ctas = pc_min((u64)ctx->sm_count * per_sm, S);
        T.queue = d_queue;
        T.nseg = 0;
        p2_sieve_kernel<512, true><<<(unsigned)ctas, 512, smem, st>>>(T, P2Multi{d_qa, d_ipref, Q, S});
        PC_LAUNCHED(ctx);
    }
    mq_p2_combine_kernel<<<(unsigned)((Q * 32 + 255) / 256), 256, 0, st>>>(d_qa, P.dq, Q, P.parts);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches += 2;
    return PC_OK;
}
