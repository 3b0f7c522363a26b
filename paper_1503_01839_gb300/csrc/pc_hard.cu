// pc_hard.cu -- the hard special leaves: the main sieve of Section 3 on the GPU.
//
// The interval [0, z] (z = x/y) is cut into segments of 30*seg_bytes
// integers.  Each CTA owns one segment at a time as a mod-30 bitset in shared
// memory and walks the primes p_b in order, b = k0+1 .. B_s:
//
//   1. leaves of b (b > c): the segment's bitset holds the integers of the
//      segment coprime to p_1..p_{b-1}, so for a hard leaf (b, m) with
//      u = x/(p_b m) in the segment, phi(u, b-1) = phi(L-1, b-1) + local(u),
//      local(u) = set bits in [L, u].  The CTA adds -mu(m) * local(u) to its
//      sum and -mu(m) to tally(s, b): the unknown phi(L-1, b-1) is recorded,
//      not needed, exactly as the tallies of Section 3.
//   2. cross off the multiples of p_b, then record count(s, b), the set bits
//      left in the segment.
//
// Afterwards phi(L_s - 1, b-1) = sum_{s' < s} count(s', b-1) is an exclusive
// scan over segments (the carries), and
//   S2_hard = sum_s acc(s) + sum_{s,b} tally(s, b) * phi(L_s - 1, b - 1).
// Segments are independent, so all SMs sieve at once and the sequential
// "synchronization after each round" of Section 3 becomes one scan.
//
// local(u) uses per-1024-bit block counters, decremented when a bit is
// cleared (or recounted after a small prime), a CTA scan of the block
// counters when a step has leaves, and __popcll over the words of u's block.
//
// A hard leaf (b, m) has u < x / p_b^2, so a segment starting at L only
// needs the primes p_b <= isqrt(x / L): B_s = pi(isqrt(x/L)).
#include "pc_internal.h"
#include "pc_sieve.cuh"

static constexpr u32 BATCH = 128;
static constexpr u32 RECOUNT_P = 256;   // primes below this recount block counters

struct HardArgs {
    u64 x, y, z;
    u32 c, k0, kleaf, bmax;
    u64 a;
    bool trunc;
    u64 nseg;
    u32 seg_bytes;
    u64 span;
    PiTable pit;
    RankTable rk;
    MList ml;
    const u32* primes;
    const u32* segB;
    const u64* off;
    u32* counts;
    i32* tallies;
    I128Pair* acc;
    u32* queue;
    unsigned long long* nleaves;   // [0] hard leaves, [1] multiples crossed off
};

struct StepInfo {
    u64 xp;       // x / p_b
    u64 kstart;   // first cofactor to cross off: max(p_b, ceil(L / p_b))
    u64 i0, i1;   // leaf index range
    u32 p;
    u32 src;      // 0: m-list, 1: primes
};

// exclusive scan of blk[0..n) into pre[0..n], by the whole CTA
template <int NT>
__device__ __forceinline__ void cta_scan_blocks(const u32* blk, u32* pre, u32 n, u32* wsum)
{
    const u32 per = (n + NT - 1) / NT;
    const u32 t = threadIdx.x, lane = t & 31, wid = t >> 5;
    u32 b0 = t * per, b1 = b0 + per < n ? b0 + per : n;
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
    if (t == NT - 1) pre[n] = run;
    __syncthreads();
}

template <int NT>
__global__ void __launch_bounds__(NT) hard_sieve_kernel(HardArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepInfo* step = (StepInfo*)smem_raw;
    u32* bits = (u32*)(smem_raw + BATCH * sizeof(StepInfo));
    const u32 seg_words = A.seg_bytes >> 2;
    const u32 nblk = A.seg_bytes >> 7;      // 1024-bit blocks
    u32* blk = bits + seg_words;
    u32* pre = blk + nblk;                  // nblk + 1 entries
    const u64* bits64 = (const u64*)bits;

    __shared__ u32 patw[80];
    __shared__ u32 wsum[32];
    __shared__ u32 s_seg, s_total;
    __shared__ u32 s_dec[2];
    __shared__ int s_tally;
    __shared__ i128 red[32];

    const u32 tid = threadIdx.x, lane = tid & 31;
    make_pattern_words(patw, A.k0);
    if (tid == 0) {
        s_dec[0] = s_dec[1] = 0;
        s_tally = 0;
    }
    unsigned long long nleaves = 0, nclears = 0;

    for (;;) {
        if (tid == 0) {
            s_seg = atomicAdd(A.queue, 1u);
            s_total = 0;
        }
        __syncthreads();
        const u64 s = s_seg;
        __syncthreads();
        if (s >= A.nseg) break;
        const u32 Bs = A.segB[s];
        if (Bs <= A.k0) continue;
        const u64 L = s * A.span;

        fill_pattern(bits, seg_words, L, patw, A.k0);
        __syncthreads();
        {
            u32 tot = 0;
            for (u32 k = tid; k < nblk; k += NT) {
                u32 c = 0;
                for (u32 w = 0; w < 32; w++) c += __popc(bits[32 * k + w]);
                blk[k] = c;
                tot += c;
            }
            for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
            if (lane == 0) atomicAdd(&s_total, tot);
        }
        __syncthreads();
        if (tid == 0) A.counts[A.off[0] + s] = s_total;

        i64 acc = 0;
        for (u32 bb = A.k0 + 1; bb <= Bs; bb += BATCH) {
            const u32 nb = Bs - bb + 1 < BATCH ? Bs - bb + 1 : BATCH;
            __syncthreads();
            if (tid < nb) {
                const u32 b = bb + tid;
                StepInfo si;
                const u64 p = A.primes[b];
                si.p = (u32)p;
                si.xp = A.x / p;
                u64 ks = L ? (L + p - 1) / p : 0;
                si.kstart = ks < p ? p : ks;
                si.i0 = si.i1 = 0;
                si.src = 0;
                if (b > A.kleaf && b <= A.a) {
                    const u64 T = pc_min(p * p, A.y);
                    u64 mhi = pc_min(A.y, si.xp / T);
                    if (L) mhi = pc_min(mhi, si.xp / L);
                    const u64 mlo = pc_max(A.y / p, si.xp / (L + A.span));
                    if (mhi > mlo) {
                        if (p * p > A.y) {
                            u64 k0 = pc_max(pi_lookup(A.pit, mlo), b);
                            u64 k1 = pc_min(pi_lookup(A.pit, mhi), A.a);
                            if (k1 > k0) {
                                si.i0 = k0 + 1;
                                si.i1 = k1 + 1;
                                si.src = 1;
                            }
                        } else {
                            si.i0 = rank_lookup(A.rk, mlo);
                            si.i1 = rank_lookup(A.rk, mhi);
                        }
                    }
                }
                step[tid] = si;
            }
            __syncthreads();

            for (u32 t = 0; t < nb; t++) {
                const u32 b = bb + t;
                const u64 p = step[t].p;
                if (b > A.kleaf) {
                    const u64 i0 = step[t].i0, i1 = step[t].i1;
                    if (i1 > i0) {
                        cta_scan_blocks<NT>(blk, pre, nblk, wsum);
                        const u64 xp = step[t].xp;
                        const u32 src = step[t].src;
                        int tl = 0;
                        u32 nl = 0;
                        for (u64 i = i0 + tid; i < i1; i += NT) {
                            u64 m;
                            bool neg;
                            if (src) {
                                m = A.primes[i];
                                neg = true;
                            } else {
                                const u32 info = A.ml.info[i];
                                if ((info >> 1) <= b) continue;
                                if (A.trunc && A.ml.gpf[i] > A.a) continue;
                                m = A.ml.m[i];
                                neg = info & 1;
                            }
                            const u64 u = xp / m;
                            const u32 e = seg_count_end(u, L);
                            const u32 eb = e >> 10, ew = e >> 6;
                            u32 cnt = pre[eb];
                            for (u32 w = eb << 4; w < ew; w++) cnt += __popcll(bits64[w]);
                            if (e & 63) cnt += __popcll(bits64[ew] & ((1ull << (e & 63)) - 1));
                            acc += neg ? (i64)cnt : -(i64)cnt;
                            tl += neg ? 1 : -1;
                            nl++;
                        }
                        for (int o = 16; o; o >>= 1) {
                            tl += __shfl_xor_sync(0xffffffffu, tl, o);
                            nl += __shfl_xor_sync(0xffffffffu, nl, o);
                        }
                        if (lane == 0) {
                            if (tl) atomicAdd(&s_tally, tl);
                            nleaves += nl;
                        }
                        __syncthreads();
                        if (tid == 0) {
                            A.tallies[A.off[b - A.k0] + s] = s_tally;
                            s_tally = 0;
                        }
                    } else if (tid == 0) {
                        A.tallies[A.off[b - A.k0] + s] = 0;
                    }
                }
                if (b < Bs) {
                    const u64 ks = step[t].kstart;
                    u32 dec = 0;
                    if (p < RECOUNT_P) {
                        auto none = [](u32) {};
                        nclears += cross_off_coop(bits, A.seg_bytes, L, (u32)p, ks, tid, NT, none);
                        if (tid == 0 && p >= L && p < L + A.span) {
                            u32 pos = seg_pos(p, L);
                            atomicAnd(&bits[pos >> 5], ~(1u << (pos & 31)));
                        }
                        __syncthreads();
                        for (u32 k = tid; k < nblk; k += NT) {
                            u32 c = 0;
                            for (u32 w = 0; w < 32; w++) c += __popc(bits[32 * k + w]);
                            dec += blk[k] - c;
                            blk[k] = c;
                        }
                    } else {
                        auto newly = [&](u32 pos) {
                            atomicSub(&blk[pos >> 10], 1u);
                            dec++;
                        };
                        const u64 rounds = A.seg_bytes / p + 2;
                        u32 nt = rounds * 8 >= NT ? NT : (u32)((rounds * 8 + 31) & ~31ull);
                        if (tid < nt) nclears += cross_off_coop(bits, A.seg_bytes, L, (u32)p, ks, tid, nt, newly);
                        if (tid == 0 && p >= L && p < L + A.span) {
                            u32 pos = seg_pos(p, L);
                            u32 msk = 1u << (pos & 31);
                            if (atomicAnd(&bits[pos >> 5], ~msk) & msk) newly(pos);
                        }
                    }
                    for (int o = 16; o; o >>= 1) dec += __shfl_xor_sync(0xffffffffu, dec, o);
                    if (lane == 0 && dec) atomicAdd(&s_dec[b & 1], dec);
                    __syncthreads();
                    if (tid == 0) {
                        s_total -= s_dec[b & 1];
                        s_dec[b & 1] = 0;
                        A.counts[A.off[b - A.k0] + s] = s_total;
                    }
                }
            }
        }
        i128 tot = block_sum_i128((i128)acc, red);
        if (tid == 0) store_i128(A.acc + s, tot);
    }
    for (int o = 16; o; o >>= 1) {
        nleaves += __shfl_xor_sync(0xffffffffu, nleaves, o);
        nclears += __shfl_xor_sync(0xffffffffu, nclears, o);
    }
    if (lane == 0 && nleaves) atomicAdd(A.nleaves, nleaves);
    if (lane == 0 && nclears) atomicAdd(A.nleaves + 1, nclears);
}

// ---------------------------------------------------------- schedule
__global__ void seg_b_kernel(u64 x, u64 nseg, u64 span, u32 bmax, PiTable pit, u32* segB)
{
    u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    u32 B = bmax;
    if (s > 0) {
        u64 L = s * span;
        u64 r = pc_isqrt(x / L);
        u64 pr = pi_lookup(pit, r);
        if (pr < B) B = (u32)pr;
    }
    segB[s] = B;
}

// S_b = number of segments with B_s >= b (B_s is non-increasing in s)
__global__ void row_len_kernel(const u32* segB, u64 nseg, u32 k0, u32 bmax, u32* len)
{
    u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    u32 b = k0 + t;
    if (b > bmax) return;
    u64 lo = 0, hi = nseg;   // first s with segB[s] < b
    while (lo < hi) {
        u64 mid = (lo + hi) >> 1;
        if (segB[mid] >= b) lo = mid + 1; else hi = mid;
    }
    len[t] = (u32)lo;
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
        if (threadIdx.x == 0) s_carry = 0;
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
u32 pc_seg_bytes(pc_ctx* ctx)
{
    u32 sb = ctx->params.seg_bytes;
    if (sb == 0) sb = 65536;
    sb = (sb + 1023) & ~1023u;
    if (sb < 1024) sb = 1024;
    if (sb > 196608) sb = 196608;
    return sb;
}

template <int NT>
static int launch_hard(pc_ctx* ctx, const HardArgs& A, int ctas, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(hard_sieve_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        pc_set_error(ctx, "cudaFuncSetAttribute(smem=%zu): %s", smem, cudaGetErrorString(e));
        return PC_ECUDA;
    }
    hard_sieve_kernel<NT><<<ctas, NT, smem, ctx->stream>>>(A);
    PC_LAUNCHED(ctx);
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
    u64 bmax = P.B < P.a ? P.B : P.a;
    if (bmax <= A.kleaf) return PC_OK;   // no hard leaf needs the sieve
    A.bmax = (u32)bmax;
    A.seg_bytes = pc_seg_bytes(ctx);
    A.span = 30ull * A.seg_bytes;
    A.nseg = P.z / A.span + 1;
    A.pit = ctx->T.pi();
    A.rk = ctx->T.rank();
    A.ml = ctx->T.mlist();
    A.primes = ctx->T.primes.as<u32>();

    const u64 nrows = bmax - A.k0 + 1;
    PC_TRY(buf_reserve(ctx, ctx->seg_b, A.nseg * sizeof(u32) + (nrows + 1) * sizeof(u32)));
    PC_TRY(buf_reserve(ctx, ctx->seg_off, (nrows + 1) * sizeof(u64)));
    u32* segB = ctx->seg_b.as<u32>();
    u32* rowlen = segB + A.nseg;
    u64* off = ctx->seg_off.as<u64>();
    seg_b_kernel<<<(unsigned)((A.nseg + 255) / 256), 256, 0, ctx->stream>>>(P.x, A.nseg, A.span, A.bmax, A.pit, segB);
    PC_LAUNCHED(ctx);
    row_len_kernel<<<(unsigned)((nrows + 255) / 256), 256, 0, ctx->stream>>>(segB, A.nseg, A.k0, A.bmax, rowlen);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches += 2;
    PC_TRY(scan_exclusive_u32_to_u64(ctx, rowlen, off, nrows));
    u64 total = 0;
    PC_TRY(copy_to_host(ctx, &total, off + nrows, sizeof(u64)));
    PC_TRY(buf_reserve(ctx, ctx->counts, total * sizeof(u32)));
    PC_TRY(buf_reserve(ctx, ctx->tallies, total * sizeof(i32)));
    PC_TRY(buf_reserve(ctx, ctx->acc_seg, A.nseg * sizeof(I128Pair)));
    PC_TRY(buf_reserve(ctx, ctx->queue, 64));
    PC_CUDA(ctx, cudaMemsetAsync(ctx->queue.p, 0, 64, ctx->stream));
    PC_CUDA(ctx, cudaMemsetAsync(ctx->acc_seg.p, 0, A.nseg * sizeof(I128Pair), ctx->stream));
    A.segB = segB;
    A.off = off;
    A.counts = ctx->counts.as<u32>();
    A.tallies = ctx->tallies.as<i32>();
    A.acc = ctx->acc_seg.as<I128Pair>();
    A.queue = ctx->queue.as<u32>();
    A.nleaves = (unsigned long long*)(ctx->queue.as<u32>() + 2);

    int nt = ctx->params.threads ? (int)ctx->params.threads : 512;
    int per_sm = ctx->params.ctas_per_sm ? (int)ctx->params.ctas_per_sm : 0;
    const u32 nblk = A.seg_bytes >> 7;
    size_t smem = BATCH * sizeof(StepInfo) + A.seg_bytes + (2 * (size_t)nblk + 2) * sizeof(u32);
    if (per_sm == 0) {
        per_sm = (int)(ctx->smem_optin / (smem + 4096));
        if (per_sm < 1) per_sm = 1;
        if (per_sm > 4) per_sm = 4;
    }
    int ctas = ctx->sm_count * per_sm;
    if ((u64)ctas > A.nseg) ctas = (int)A.nseg;

    cudaEvent_t e0 = ctx->ev[0], e1 = ctx->ev[1];
    PC_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
    int rc;
    if (nt <= 256) rc = launch_hard<256>(ctx, A, ctas, smem);
    else if (nt <= 512) rc = launch_hard<512>(ctx, A, ctas, smem);
    else rc = launch_hard<1024>(ctx, A, ctas, smem);
    if (rc) return rc;
    PC_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    ctx->stats.kernel_launches++;

    int g = (int)pc_min(bmax - A.kleaf, 4096);
    PC_TRY(buf_reserve(ctx, ctx->partials, g * sizeof(I128Pair)));
    hard_combine_kernel<256><<<g, 256, 0, ctx->stream>>>(A, ctx->partials.as<I128Pair>());
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    PC_TRY(reduce_i128(ctx, ctx->partials.as<I128Pair>(), g, out));
    PC_TRY(reduce_i128(ctx, A.acc, A.nseg, out));

    u64 nl[2] = {0, 0};
    PC_TRY(copy_to_host(ctx, nl, A.nleaves, 2 * sizeof(u64)));
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
