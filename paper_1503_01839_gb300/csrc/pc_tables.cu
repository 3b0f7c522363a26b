// pc_tables.cu -- device table builders (all on the GPU).
//
//  * bootstrap primes <= 65536
//  * pi table: mod-30 prime bitset over [0, pi_limit] plus per-word prefix
//    counts, giving pi(v) in O(1) (the role of the pi(y) table of Section 2;
//    the popcount bitset is this library's GPU form of Section 2.1's idea of
//    a sampled table completed by a short local count)
//  * primes p_1..p_n as a dense array (Section 2: table of primes p_b)
//  * the squarefree m-list with lpf / mu / gpf (Section 2.2: the p_min(y)
//    and mu(y) data the leaf sums iterate over), plus a rank bitset giving
//    the list index of any m in O(1)
//  * phi(., c) residue tables for the primorial of c (the wheel of Section 4)
#include "pc_internal.h"
#include "pc_sieve.cuh"


// ------------------------------------------------------ bootstrap primes
__global__ void small_primes_kernel(u32* out, u32* count)
{
    // thread t owns the 64 integers [64t, 64t+64) of [0, 65536)

    __shared__ u32 wsum[32];
    const u32 t = threadIdx.x;
    u64 mask = 0;
    for (u32 i = 0; i < 64; i++) {
        u32 n = 64 * t + i;
        bool pr = n >= 2;
        for (u32 d = 2; pr && d * d <= n; d++)
            if (n % d == 0) pr = false;
        if (pr) mask |= 1ull << i;
    }
    u32 c = __popcll(mask);
    // block exclusive scan of c
    u32 lane = t & 31, wid = t >> 5;
    u32 incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        u32 v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        u32 w = wsum[lane], wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            u32 v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        wsum[lane] = wi - w;
        if (lane == 31) *count = wi;
    }
    __syncthreads();
    u32 pos = wsum[wid] + incl - c;

    while (mask) {
        int i = __ffsll((long long)mask) - 1;
        mask &= mask - 1;
        out[pos++] = 64 * t + (u32)i;
    }
}

// ------------------------------------------------------------- pi table
// One CTA per segment of PI_SEG_BYTES bytes: cross off multiples k*p,
// k >= p (primes stay set), then write the words and their popcounts.
static constexpr u32 PI_SEG_BYTES = 16384;

__global__ void pi_sieve_kernel(const u32* sp, u32 nsp, u64 limit, u64 nwords64, u64* words, u32* wcnt)
{
    __shared__ u32 bits[PI_SEG_BYTES / 4];
    const u64 L = (u64)blockIdx.x * (30ull * PI_SEG_BYTES);
    const u64 end = L + 30ull * PI_SEG_BYTES;   // exclusive
    for (u32 w = threadIdx.x; w < PI_SEG_BYTES / 4; w += blockDim.x) bits[w] = 0xFFFFFFFFu;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) bits[0] &= ~1u;   // 1 is not prime
    __syncthreads();
    u64 hi = end - 1 < limit ? end - 1 : limit;
    u64 r = pc_isqrt(hi);
    auto none = [](u32) {};
    // primes 7.. (sp[0..2] = 2, 3, 5)
    for (u32 i = 3; i < nsp; i++) {
        u32 p = sp[i];
        if (p > r) break;
        u64 kstart = (L + p - 1) / p;
        if (kstart < p) kstart = p;
        if ((u64)p * 8 <= PI_SEG_BYTES) {
            cross_off_coop(bits, PI_SEG_BYTES, L, p, kstart, threadIdx.x, blockDim.x, none);
        } else if (threadIdx.x < 32) {
            cross_off_coop(bits, PI_SEG_BYTES, L, p, kstart, threadIdx.x, 32, none);
        }
    }
    __syncthreads();
    const u64* b64 = (const u64*)bits;
    u64 w0 = (u64)blockIdx.x * (PI_SEG_BYTES / 8);
    for (u32 w = threadIdx.x; w < PI_SEG_BYTES / 8; w += blockDim.x) {
        u64 gw = w0 + w;
        if (gw < nwords64) {
            u64 v = b64[w];
            words[gw] = v;
            wcnt[gw] = __popcll(v);
        }
    }
}

// ------------------------------------------------------------- primes[]
// primes[k] = p_k for 1 <= k <= n_out; primes[0] = 1.
__global__ void extract_primes_kernel(const PiRec* rec, u64 nwords, u32* primes, u64 n_out)
{
    u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (w == 0) {
        primes[0] = 1;
        if (n_out >= 1) primes[1] = 2;
        if (n_out >= 2) primes[2] = 3;
        if (n_out >= 3) primes[3] = 5;
    }
    if (w >= nwords) return;
    u64 v = rec[w].bits;
    u64 idx = 3 + rec[w].cnt;
    while (v) {
        int b = __ffsll((long long)v) - 1;
        v &= v - 1;
        idx++;
        if (idx > n_out) return;
        u64 n = 240 * w + 30 * (u64)(b >> 3) + r8(b & 7);
        primes[idx] = (u32)n;
    }
}

// --------------------------------------------------------------- m-list
// One CTA per ML_CHUNK integers [lo, lo + ML_CHUNK).  Every prime p <= sqrt(Y)
// is applied to its multiples with shared-memory atomics (order free):
// lpf = min, largest small factor = max, parity of the number of small
// factors, product of small factors, and a square-factor flag.  What is left
// after dividing out the small factors is 1 or one prime > sqrt(Y).
static constexpr u32 ML_CHUNK = 2048;

__global__ void mlist_kernel(const u32* sp, u32 nsp, u64 Y, u32 pcmin, PiTable pit,
                             u64* info_tmp, u64* rbits)
{
    __shared__ u32 prod[ML_CHUNK];
    __shared__ u32 lpf[ML_CHUNK];
    __shared__ u32 gsm[ML_CHUNK];
    __shared__ u32 flg[ML_CHUNK];
    const u64 lo = (u64)blockIdx.x * ML_CHUNK;
    for (u32 i = threadIdx.x; i < ML_CHUNK; i += blockDim.x) {
        prod[i] = 1;
        lpf[i] = 0xFFFFFFFFu;
        gsm[i] = 0;
        flg[i] = 0;
    }
    __syncthreads();
    u64 hi = lo + ML_CHUNK - 1 < Y ? lo + ML_CHUNK - 1 : Y;
    u32 r = (u32)pc_isqrt(Y);
    // primes with many multiples: all threads per prime
    u32 i = 0;
    for (; i < nsp; i++) {
        u32 p = sp[i];
        if (p > r || p * 8 > ML_CHUNK) break;
        u64 first = (lo + p - 1) / p * p;
        if (first < p) first = p;
        for (u64 n = first + (u64)threadIdx.x * p; n <= hi; n += (u64)blockDim.x * p) {
            u32 k = (u32)(n - lo);
            u64 q = n / p;
            if (q % p == 0) atomicOr(&flg[k], 2u);
            atomicMin(&lpf[k], p);
            atomicMax(&gsm[k], p);
            atomicXor(&flg[k], 1u);
            u32 cur = prod[k], seen;
            do {
                seen = cur;
                cur = atomicCAS(&prod[k], seen, seen * p);
            } while (cur != seen);
        }
    }
    // primes with few multiples: one thread per prime
    for (u32 j = i + threadIdx.x; j < nsp; j += blockDim.x) {
        u32 p = sp[j];
        if (p > r) break;
        u64 first = (lo + p - 1) / p * p;
        if (first < p) first = p;
        for (u64 n = first; n <= hi; n += p) {
            u32 k = (u32)(n - lo);
            u64 q = n / p;
            if (q % p == 0) atomicOr(&flg[k], 2u);
            atomicMin(&lpf[k], p);
            atomicMax(&gsm[k], p);
            atomicXor(&flg[k], 1u);
            u32 cur = prod[k], seen;
            do {
                seen = cur;
                cur = atomicCAS(&prod[k], seen, seen * p);
            } while (cur != seen);
        }
    }
    __syncthreads();
    // finalize: one thread per integer, 64 integers per rank word
    for (u32 k = threadIdx.x; k < ML_CHUNK; k += blockDim.x) {
        u64 n = lo + k;
        bool entry = false;
        u64 packed = 0;
        if (n >= 2 && n <= Y && !(flg[k] & 2u)) {
            u32 par = flg[k] & 1u;
            u64 l = lpf[k], g = gsm[k];
            u64 big = n / prod[k];
            if (big > 1) {
                par ^= 1u;
                g = big;
                if (big < l) l = big;
            }
            if (l > pcmin) {
                entry = true;
                u64 li = pi_lookup(pit, l), gi = pi_lookup(pit, g);
                packed = (li << 1) | (u64)par | (gi << 32);
            }
        }
        if (n <= Y) info_tmp[n] = packed;
        unsigned bal = __ballot_sync(0xffffffffu, entry);
        // two warps-worth of 32 integers make one 64-bit rank word
        if ((k & 31) == 0) {
            u64 word_idx = n >> 6;
            u32 half = (u32)(n >> 5) & 1u;
            if (n <= Y) atomicOr((unsigned long long*)&rbits[word_idx], (u64)bal << (32 * half));
        }
    }
}

__global__ void popc_words_kernel(const u64* w, u64 n, u32* out)
{
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __popcll(w[i]);
}

__global__ void mlist_scatter_kernel(const u64* info_tmp, const u64* rbits, const u32* rcnt, u64 Y,
                                     u32* mm, u32* minfo, u32* mgpf)
{
    u64 n = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (n > Y) return;
    u64 w = rbits[n >> 6];
    u32 b = (u32)(n & 63);
    if (!((w >> b) & 1)) return;
    u64 idx = rcnt[n >> 6] + __popcll(w & ((1ull << b) - 1));
    u64 packed = info_tmp[n];
    mm[idx] = (u32)n;
    minfo[idx] = (u32)packed;          // (lpf_index << 1) | parity
    mgpf[idx] = (u32)(packed >> 32);
}

// reciprocals v = floor((2^64 - 1) / d) of a u32 array (d >= 1; d = 0 gives 0)
__global__ void reciprocal_kernel(const u32* d, u64 n, u64* v)
{
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = d[i] ? ~0ull / d[i] : 0;
}

// the 32-bit reciprocal records of div_dv
__global__ void dv_kernel(const u32* d, u64 n, u64* dv)
{
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dv[i] = pc_dv(d[i]);
}

// odd-number pi table (pi_odd) over [0, 64 n): a thread per odd number 2t + 1,
// a warp per record (blocks of 256 threads keep a record in one warp)
__global__ void pi_odd_kernel(PiTable pit, u64 n, uint2* out)
{
    const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    const u64 w = t >> 5, v = 2 * t + 1;
    bool prime = false;
    if (v <= 5) {
        prime = true;   // 1 stands for 2; 3 and 5
    } else if (v <= pit.limit) {
        const u32 r = (u32)(v % 30);
        if (coprime30(r)) {
            const u64 q30 = v / 30;
            prime = (pit.rec[q30 >> 3].bits >> (8 * (q30 & 7) + idx30(r))) & 1;
        }
    }
    const u32 bits = __ballot_sync(0xffffffffu, prime);
    if ((threadIdx.x & 31) == 0 && w < n) out[w] = make_uint2(bits, w ? (u32)pi_lookup(pit, 64 * w - 1) : 0u);
}

static int build_pi_odd(pc_ctx* ctx, u64 limit)
{
    Tables& T = ctx->T;
    const u64 n = limit / 64 + 1;
    PC_TRY(buf_reserve(ctx, T.pi_odd, n * sizeof(uint2)));
    pi_odd_kernel<<<(unsigned)((32 * n + 255) / 256), 256, 0, ctx->stream>>>(T.pi(), n, T.pi_odd.as<uint2>());
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    T.podd_limit = limit;
    return PC_OK;
}

// ------------------------------------------------------------ phi tables
__global__ void coprime_flags_kernel(u32 Q, u32 c, const u32* sp, u32* flags)
{
    u32 r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Q) return;
    u32 f = r >= 1;
    for (u32 i = 0; i < c; i++)
        if (r % sp[i] == 0) f = 0;
    flags[r] = f;
}

// ------------------------------------------------------------------ host
static int ensure_small(pc_ctx* ctx)
{
    Tables& T = ctx->T;
    if (T.n_small) return PC_OK;
    PC_TRY(buf_reserve(ctx, T.small_primes, 8192 * sizeof(u32)));
    PC_TRY(buf_reserve(ctx, ctx->misc, 64));
    small_primes_kernel<<<1, 1024, 0, ctx->stream>>>(T.small_primes.as<u32>(), ctx->misc.as<u32>());
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    u32 n = 0;
    PC_TRY(copy_to_host(ctx, &n, ctx->misc.p, sizeof(u32)));
    T.n_small = n;
    return PC_OK;
}

__global__ void pack_pi_kernel(const u64* words, const u32* pcnt, u64 n, PiRec* rec)
{
    u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (w < n) {
        PiRec r;
        r.bits = words[w];
        r.cnt = pcnt[w];
        r.pad = 0;
        rec[w] = r;
    }
}

static int build_pi(pc_ctx* ctx, u64 limit)
{
    Tables& T = ctx->T;
    u64 nwords = limit / 240 + 1;
    u64 nseg = (limit + 30ull * PI_SEG_BYTES) / (30ull * PI_SEG_BYTES);
    u64 nw_alloc = nseg * (PI_SEG_BYTES / 8);
    PC_TRY(buf_reserve(ctx, T.pi_rec, nwords * sizeof(PiRec)));
    DevBuf words, cnt, pcnt;
    int rc = buf_reserve(ctx, words, nw_alloc * sizeof(u64));
    if (rc == PC_OK) rc = buf_reserve(ctx, cnt, (nwords + 1) * sizeof(u32));
    if (rc == PC_OK) rc = buf_reserve(ctx, pcnt, (nwords + 1) * sizeof(u32));
    if (rc == PC_OK) {
        pi_sieve_kernel<<<(unsigned)nseg, 256, 0, ctx->stream>>>(T.small_primes.as<u32>(), T.n_small, limit, nwords,
                                                                words.as<u64>(), cnt.as<u32>());
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) rc = scan_exclusive_u32_to_u32(ctx, cnt.as<u32>(), pcnt.as<u32>(), nwords);
        else {
            pc_set_error(ctx, "pi_sieve_kernel launch: %s", cudaGetErrorString(e));
            rc = PC_ECUDA;
        }
        if (rc == PC_OK) {
            pack_pi_kernel<<<(unsigned)((nwords + 255) / 256), 256, 0, ctx->stream>>>(
                words.as<u64>(), pcnt.as<u32>(), nwords, T.pi_rec.as<PiRec>());
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) {
                pc_set_error(ctx, "pi table build: %s", cudaGetErrorString(e));
                rc = PC_ECUDA;
            }
        }
    }
    buf_free(words);
    buf_free(cnt);
    buf_free(pcnt);
    ctx->stats.kernel_launches += 2;
    if (rc == PC_OK) T.pi_limit = limit;
    return rc;
}

static int build_primes(pc_ctx* ctx, u64 prime_limit)
{
    Tables& T = ctx->T;
    // pi(prime_limit) and one sentinel prime above it (gap < 2048 below 2^64)
    u64 v[1] = {prime_limit};
    u64 np = 0;
    PC_TRY(tables_pi_values(ctx, v, &np, 1));
    u64 n_out = np + 1;
    PC_TRY(buf_reserve(ctx, T.primes, (n_out + 2) * sizeof(u32)));
    u64 wlim = (prime_limit + 2048) / 240 + 1;
    u64 wmax = T.pi_limit / 240 + 1;
    if (wlim > wmax) wlim = wmax;
    extract_primes_kernel<<<(unsigned)((wlim + 255) / 256), 256, 0, ctx->stream>>>(
        T.pi_rec.as<PiRec>(), wlim, T.primes.as<u32>(), n_out);
    PC_LAUNCHED(ctx);
    PC_TRY(buf_reserve(ctx, T.primes_rcp, (n_out + 2) * sizeof(u64)));
    reciprocal_kernel<<<(unsigned)((n_out + 1 + 255) / 256), 256, 0, ctx->stream>>>(T.primes.as<u32>(), n_out + 1,
                                                                                   T.primes_rcp.as<u64>());
    PC_LAUNCHED(ctx);
    PC_TRY(buf_reserve(ctx, T.primes_dv, (n_out + 2) * sizeof(u64)));
    dv_kernel<<<(unsigned)((n_out + 1 + 255) / 256), 256, 0, ctx->stream>>>(T.primes.as<u32>(), n_out + 1,
                                                                            T.primes_dv.as<u64>());
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches += 3;
    T.nprimes = np;
    T.prime_limit = prime_limit;
    return PC_OK;
}

// ------------------------------------------- presieve pattern of 7..19
// Byte g holds the integers 30 g + R8[j]; bit j is cleared when one of 7, 11, 13,
// 17, 19 divides it (the primes themselves included).  The pattern repeats every
// 7 * 11 * 13 * 17 * 19 bytes; the array runs 128 KiB + 8 bytes past one period, so
// that a segment's words are one contiguous slice read at any phase.
__global__ void wheel19_kernel(u32* words, u32 nwords)
{
    const u32 w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwords) return;
    u32 v = 0;
    for (u32 i = 0; i < 4; i++) {
        const u32 g = (4 * w + i) % WHEEL19_PERIOD;
        u32 byte = 0xFFu;
        for (u32 j = 0; j < 8; j++) {
            const u32 n = 30 * g + r8(j);   // < 2^24: no overflow
            if (n % 7 == 0 || n % 11 == 0 || n % 13 == 0 || n % 17 == 0 || n % 19 == 0) byte &= ~(1u << j);
        }
        v |= byte << (8 * i);
    }
    words[w] = v;
}

int tables_wheel19(pc_ctx* ctx)
{
    Tables& T = ctx->T;
    const u32 nwords = (WHEEL19_PERIOD + 131072 + 8 + 3) / 4;
    if (T.wheel19.bytes >= nwords * sizeof(u32) || ctx->borrowed) return PC_OK;
    PC_TRY(buf_reserve(ctx, T.wheel19, nwords * sizeof(u32)));
    wheel19_kernel<<<(nwords + 255) / 256, 256, 0, ctx->stream>>>(T.wheel19.as<u32>(), nwords);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    return PC_OK;
}

// ------------------------------------------------------ sampled pi table
__global__ void sampled_kernel(PiTable pit, u64 n, u32 step, u32* samp)
{
    const u64 j = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) samp[j] = (u32)pi_lookup(pit, j * step);
}

// pi at every step-th integer up to limit, step = floor(log2 limit) (Section 2.1).
static int build_sampled(pc_ctx* ctx, u64 limit)
{
    Tables& T = ctx->T;
    u32 step = 0;
    for (u64 v = limit; v > 1; v >>= 1) step++;   // floor(log2 limit)
    if (step < 1) step = 1;
    const u64 n = limit / step + 1;
    PC_TRY(buf_reserve(ctx, T.samp, n * sizeof(u32)));
    sampled_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(T.pi(), n, step, T.samp.as<u32>());
    PC_LAUNCHED(ctx);
    PC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->stats.kernel_launches++;
    T.samp_s = step;
    T.samp_limit = limit;   // every v <= limit has v / step < n
    return PC_OK;
}

// ------------------------------------------------------------ sub-lists
__global__ void sub_flags_kernel(const u32* info, u64 n, u32 K, u32* flags)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = (info[i] >> 1) > K ? 1u : 0u;
}

__global__ void sub_scatter_kernel(MList src, const u32* flags, const u32* pos, u32* m, u32* info, u32* gpf, u64* rcp,
                                   u64* bits)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= src.n || !flags[i]) return;
    const u32 j = pos[i];
    const u32 mi = src.m[i];
    m[j] = mi;
    info[j] = src.info[i];
    gpf[j] = src.gpf[i];
    rcp[j] = src.rcp[i];
    atomicOr((unsigned long long*)bits + (mi >> 6), 1ull << (mi & 63));
}

// The entries of the m-list with lpf index > K, for a few K, each with its own
// rank table over [0, ml_limit]: the leaves of p_b, b >= K, are read from the
// largest such list (same order, fewer entries to skip).
static int build_sublists(pc_ctx* ctx)
{
    Tables& T = ctx->T;
    T.n_sl = 0;
    static const u32 KS[Tables::NSUB] = {8, 24, 72, 216};
    const u64 n = T.ml_n, Y = T.ml_limit;
    if (n == 0) return PC_OK;
    const u64 nrw = Y / 64 + 1;
    DevBuf flags, pos, wc;
    int rc = buf_reserve(ctx, flags, (n + 1) * sizeof(u32));
    if (rc == PC_OK) rc = buf_reserve(ctx, pos, (n + 1) * sizeof(u32));
    if (rc == PC_OK) rc = buf_reserve(ctx, wc, (nrw + 1) * sizeof(u32));
    for (int k = 0; k < Tables::NSUB && rc == PC_OK; k++) {
        const u32 K = KS[k];
        if (K <= T.ml_cmin) continue;
        sub_flags_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(T.ml_info.as<u32>(), n, K, flags.as<u32>());
        rc = scan_exclusive_u32_to_u32(ctx, flags.as<u32>(), pos.as<u32>(), n);
        u32 cnt = 0;
        if (rc == PC_OK) rc = copy_to_host(ctx, &cnt, pos.as<u32>() + n, sizeof(u32));
        if (rc != PC_OK) break;
        const int s = T.n_sl;
        rc = buf_reserve(ctx, T.sl_m[s], ((u64)cnt + 1) * sizeof(u32));
        if (rc == PC_OK) rc = buf_reserve(ctx, T.sl_info[s], ((u64)cnt + 1) * sizeof(u32));
        if (rc == PC_OK) rc = buf_reserve(ctx, T.sl_gpf[s], ((u64)cnt + 1) * sizeof(u32));
        if (rc == PC_OK) rc = buf_reserve(ctx, T.sl_rcp[s], ((u64)cnt + 1) * sizeof(u64));
        if (rc == PC_OK) rc = buf_reserve(ctx, T.sl_bits[s], nrw * sizeof(u64));
        if (rc == PC_OK) rc = buf_reserve(ctx, T.sl_cnt[s], (nrw + 1) * sizeof(u32));
        if (rc != PC_OK) break;
        cudaError_t e = cudaMemsetAsync(T.sl_bits[s].p, 0, nrw * sizeof(u64), ctx->stream);
        if (e == cudaSuccess) {
            sub_scatter_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
                T.mlist(), flags.as<u32>(), pos.as<u32>(), T.sl_m[s].as<u32>(), T.sl_info[s].as<u32>(),
                T.sl_gpf[s].as<u32>(), T.sl_rcp[s].as<u64>(), T.sl_bits[s].as<u64>());
            popc_words_kernel<<<(unsigned)((nrw + 255) / 256), 256, 0, ctx->stream>>>(T.sl_bits[s].as<u64>(), nrw,
                                                                                      wc.as<u32>());
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            pc_set_error(ctx, "m-list sub-lists: %s", cudaGetErrorString(e));
            rc = PC_ECUDA;
            break;
        }
        rc = scan_exclusive_u32_to_u32(ctx, wc.as<u32>(), T.sl_cnt[s].as<u32>(), nrw);
        if (rc != PC_OK) break;
        T.sl_K[s] = K;
        T.sl_n[s] = cnt;
        T.n_sl = s + 1;
        ctx->stats.kernel_launches += 3;
    }
    if (rc == PC_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            pc_set_error(ctx, "m-list sub-lists: %s", cudaGetErrorString(e));
            rc = PC_ECUDA;
        }
    }
    if (rc != PC_OK) T.n_sl = 0;
    buf_free(flags);
    buf_free(pos);
    buf_free(wc);
    return rc;
}

// ------------------------------------------ m-list by nested loops (Section 2.2)
// The same list without a table of least prime factors: the squarefree m <= Y with
// lpf(m) > p_cmin are the products p_b1 p_b2 ... p_bn of distinct primes, cmin < b1 <
// b2 < ... < bn, and mu(m) = (-1)^n.  They are enumerated level by level.  A prefix
// P = p_b1 ... p_bk (P = 1 at level 0, with b_k read as cmin) owns the entries P p_j for
// every prime index j > b_k with P p_j <= Y, each with lpf index b1 (j at level 0), gpf
// index j and n = k + 1 factors; P p_j is a prefix of the next level when it still has
// an entry, P p_j p_(j+1) <= Y.  A level with no prefixes ends the loops (at most 15
// levels below 2^64, since 2 * 3 * ... * 53 > 2^64).  The entries are then placed in
// ascending order through the rank bitset of the members: set, counted, and every entry
// written at its rank.
struct NestPrefix {
    u64 P;     // product of the prefix's primes (1 at level 0)
    u32 lpf;   // index of its least prime (unused at level 0)
    u32 gi;    // index of its largest prime (cmin at level 0)
    u32 nf;    // number of primes
    u32 pad;
};

// children of each prefix: the j in (gi, J] with p_j p_(j+1) <= Y / P (a monotone test)
__global__ void nest_children_kernel(const NestPrefix* lv, u32 n, const u32* primes, PiTable pit, u64 Y, u32* cnt)
{
    const u32 k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const NestPrefix q = lv[k];
    const u64 R = Y / q.P;
    // p_j^2 < p_j p_(j+1) <= R bounds j by pi(isqrt R)
    u64 lo = q.gi, hi = pi_lookup(pit, pc_isqrt(R));   // the answer J lies in [gi, hi]
    while (hi > lo) {
        const u64 mid = lo + (hi - lo + 1) / 2;
        if ((u64)primes[mid] * primes[mid + 1] <= R) lo = mid;
        else hi = mid - 1;
    }
    cnt[k] = (u32)(lo - q.gi);
}

__global__ void nest_expand_kernel(const NestPrefix* lv, u32 n, const u32* off, const u32* primes, NestPrefix* next)
{
    const u32 k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const NestPrefix q = lv[k];
    const u32 c = off[k + 1] - off[k];
    for (u32 t = 0; t < c; t++) {
        const u32 j = q.gi + 1 + t;
        next[off[k] + t] = NestPrefix{q.P * primes[j], q.nf ? q.lpf : j, j, q.nf + 1, 0};
    }
}

// entries of each prefix: the j in (gi, pi(Y / P)]
__global__ void nest_entries_kernel(const NestPrefix* all, u64 n, PiTable pit, u64 Y, u32* cnt)
{
    const u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const u64 hi = pi_lookup(pit, Y / all[k].P);
    cnt[k] = hi > all[k].gi ? (u32)(hi - all[k].gi) : 0u;
}

// entry g: its prefix (the last k with eoff[k] <= g), its prime index and its m
__device__ __forceinline__ void nest_entry(const NestPrefix* all, u64 n, const u64* eoff, const u32* primes, u64 g,
                                           NestPrefix& q, u32& j, u64& m)
{
    u64 lo = 0, hi = n;
    while (hi - lo > 1) {
        const u64 mid = (lo + hi) >> 1;
        if (eoff[mid] <= g) lo = mid;
        else hi = mid;
    }
    q = all[lo];
    j = q.gi + 1 + (u32)(g - eoff[lo]);
    m = q.P * primes[j];
}

__global__ void nest_mark_kernel(const NestPrefix* all, u64 n, const u64* eoff, const u32* primes, u64* rbits)
{
    const u64 g = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= eoff[n]) return;
    NestPrefix q;
    u32 j;
    u64 m;
    nest_entry(all, n, eoff, primes, g, q, j, m);
    atomicOr((unsigned long long*)&rbits[m >> 6], 1ull << (m & 63));
}

__global__ void nest_scatter_kernel(const NestPrefix* all, u64 n, const u64* eoff, const u32* primes,
                                    const u64* rbits, const u32* rcnt, u32* mm, u32* minfo, u32* mgpf)
{
    const u64 g = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= eoff[n]) return;
    NestPrefix q;
    u32 j;
    u64 m;
    nest_entry(all, n, eoff, primes, g, q, j, m);
    const u64 idx = rcnt[m >> 6] + __popcll(rbits[m >> 6] & ((1ull << (m & 63)) - 1));
    mm[idx] = (u32)m;
    minfo[idx] = ((q.nf ? q.lpf : j) << 1) | ((q.nf + 1) & 1u);   // mu = -1 for an odd count of primes
    mgpf[idx] = j;
}

static int build_mlist_nested(pc_ctx* ctx, u64 Y, u32 cmin)
{
    Tables& T = ctx->T;
    // the entries' largest primes reach Y / p_(cmin+1): the prime table must cover Y
    if (T.prime_limit < Y) {
        if (Y + 2048 > T.pi_limit) {
            pc_set_error(ctx, "nested m-list: the pi table ends below %llu", (unsigned long long)(Y + 2048));
            return PC_EINVAL;
        }
        PC_TRY(build_primes(ctx, Y));
    }
    const u32* primes = T.primes.as<u32>();
    // the prefixes, level by level, appended to one array
    std::vector<u32> level_n;
    DevBuf all, nxt, cnt;
    u64 n_all = 1, cap = 1024;
    int rc = buf_reserve(ctx, all, cap * sizeof(NestPrefix));
    if (rc) return rc;
    {
        const NestPrefix root{1, 0, cmin, 0, 0};
        rc = cudaMemcpyAsync(all.p, &root, sizeof(root), cudaMemcpyHostToDevice, ctx->stream) == cudaSuccess
                 ? PC_OK : PC_ECUDA;
    }
    u64 lv0 = 0, lvn = 1;   // the current level: all[lv0, lv0 + lvn)
    int levels = 0;
    while (rc == PC_OK && lvn > 0) {
        if (++levels > 16) {
            pc_set_error(ctx, "nested m-list: more than 16 levels");
            rc = PC_EOVERFLOW;
            break;
        }
        rc = buf_reserve(ctx, cnt, (lvn + 1) * 2 * sizeof(u32));
        if (rc) break;
        u32* c = cnt.as<u32>();
        u32* off = c + lvn + 1;
        NestPrefix* cur = all.as<NestPrefix>() + lv0;
        nest_children_kernel<<<(unsigned)((lvn + 255) / 256), 256, 0, ctx->stream>>>(cur, (u32)lvn, primes, T.pi(),
                                                                                     Y, c);
        rc = scan_exclusive_u32_to_u32(ctx, c, off, lvn);
        u32 nn = 0;
        if (rc == PC_OK) rc = copy_to_host(ctx, &nn, off + lvn, sizeof(u32));
        if (rc || nn == 0) break;
        if (n_all + nn > cap) {
            // grow the prefix array (the current level is copied along)
            u64 ncap = cap;
            while (n_all + nn > ncap) ncap *= 2;
            rc = buf_reserve(ctx, nxt, ncap * sizeof(NestPrefix));
            if (rc == PC_OK && cudaMemcpyAsync(nxt.p, all.p, n_all * sizeof(NestPrefix), cudaMemcpyDeviceToDevice,
                                               ctx->stream) != cudaSuccess)
                rc = PC_ECUDA;
            if (rc) break;
            std::swap(all, nxt);
            buf_free(nxt);
            cap = ncap;
            cur = all.as<NestPrefix>() + lv0;
        }
        nest_expand_kernel<<<(unsigned)((lvn + 255) / 256), 256, 0, ctx->stream>>>(cur, (u32)lvn, off, primes,
                                                                                   all.as<NestPrefix>() + n_all);
        ctx->stats.kernel_launches += 2;
        lv0 = n_all;
        lvn = nn;
        n_all += nn;
    }
    // entries per prefix, their offsets, then the rank bitset and the list
    u64 nrw = Y / 64 + 1, total = 0;
    if (rc == PC_OK) rc = buf_reserve(ctx, cnt, (n_all + 1) * sizeof(u32) + (n_all + 1) * sizeof(u64) + 8);
    u32* ec = cnt.as<u32>();
    u64* eoff = (u64*)(((uintptr_t)(ec + n_all + 1) + 7) & ~(uintptr_t)7);
    if (rc == PC_OK) {
        nest_entries_kernel<<<(unsigned)((n_all + 255) / 256), 256, 0, ctx->stream>>>(all.as<NestPrefix>(), n_all,
                                                                                      T.pi(), Y, ec);
        rc = scan_exclusive_u32_to_u64(ctx, ec, eoff, n_all);
    }
    if (rc == PC_OK) rc = copy_to_host(ctx, &total, eoff + n_all, sizeof(u64));
    if (rc == PC_OK && total > 0xFFFFFFFFull) {
        pc_set_error(ctx, "nested m-list: %llu entries", (unsigned long long)total);
        rc = PC_EOVERFLOW;
    }
    if (rc == PC_OK) rc = buf_reserve(ctx, T.rank_bits, nrw * sizeof(u64));
    if (rc == PC_OK) rc = buf_reserve(ctx, T.rank_cnt, (nrw + 1) * sizeof(u32));
    if (rc == PC_OK && cudaMemsetAsync(T.rank_bits.p, 0, nrw * sizeof(u64), ctx->stream) != cudaSuccess) rc = PC_ECUDA;
    const unsigned eg = (unsigned)((total + 255) / 256);
    if (rc == PC_OK && total)
        nest_mark_kernel<<<eg, 256, 0, ctx->stream>>>(all.as<NestPrefix>(), n_all, eoff, primes,
                                                      T.rank_bits.as<u64>());
    DevBuf tmp;
    if (rc == PC_OK) rc = buf_reserve(ctx, tmp, (nrw + 1) * sizeof(u32));
    if (rc == PC_OK) {
        popc_words_kernel<<<(unsigned)((nrw + 255) / 256), 256, 0, ctx->stream>>>(T.rank_bits.as<u64>(), nrw,
                                                                                 tmp.as<u32>());
        rc = scan_exclusive_u32_to_u32(ctx, tmp.as<u32>(), T.rank_cnt.as<u32>(), nrw);
    }
    u32 members = 0;
    if (rc == PC_OK) rc = copy_to_host(ctx, &members, T.rank_cnt.as<u32>() + nrw, sizeof(u32));
    if (rc == PC_OK && members != total) {
        // two entries with the same m would mean a product enumerated twice
        pc_set_error(ctx, "nested m-list: %llu entries but %u distinct m", (unsigned long long)total, members);
        rc = PC_EOVERFLOW;
    }
    if (rc == PC_OK) rc = buf_reserve(ctx, T.ml_m, (total + 1) * sizeof(u32));
    if (rc == PC_OK) rc = buf_reserve(ctx, T.ml_info, (total + 1) * sizeof(u32));
    if (rc == PC_OK) rc = buf_reserve(ctx, T.ml_gpf, (total + 1) * sizeof(u32));
    if (rc == PC_OK) rc = buf_reserve(ctx, T.ml_rcp, (total + 1) * sizeof(u64));
    if (rc == PC_OK && total) {
        nest_scatter_kernel<<<eg, 256, 0, ctx->stream>>>(all.as<NestPrefix>(), n_all, eoff, primes,
                                                         T.rank_bits.as<u64>(), T.rank_cnt.as<u32>(),
                                                         T.ml_m.as<u32>(), T.ml_info.as<u32>(), T.ml_gpf.as<u32>());
        reciprocal_kernel<<<eg, 256, 0, ctx->stream>>>(T.ml_m.as<u32>(), total, T.ml_rcp.as<u64>());
        ctx->stats.kernel_launches += 3;
    }
    if (rc == PC_OK) {
        const cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            pc_set_error(ctx, "nested m-list build: %s", cudaGetErrorString(e));
            rc = PC_ECUDA;
        }
    }
    buf_free(tmp);
    buf_free(cnt);
    buf_free(all);
    ctx->stats.kernel_launches += 2;
    if (rc == PC_OK) {
        T.ml_limit = Y;
        T.ml_cmin = cmin;
        T.ml_n = total;
    }
    return rc;
}

static int build_mlist(pc_ctx* ctx, u64 Y, u32 cmin)
{
    Tables& T = ctx->T;
    u32 pcmin = 1;   // lpf must exceed p_cmin (p_0 = 1)
    {
        static const u32 P8[8] = {1, 2, 3, 5, 7, 11, 13, 17};
        pcmin = P8[cmin];
    }
    u64 nrw = Y / 64 + 1;
    DevBuf info_tmp;
    int rc = buf_reserve(ctx, info_tmp, (Y + 1) * sizeof(u64));
    if (rc) return rc;
    PC_TRY(buf_reserve(ctx, T.rank_bits, nrw * sizeof(u64)));
    PC_TRY(buf_reserve(ctx, T.rank_cnt, (nrw + 1) * sizeof(u32)));
    PC_CUDA(ctx, cudaMemsetAsync(T.rank_bits.p, 0, nrw * sizeof(u64), ctx->stream));
    u64 nchunks = Y / ML_CHUNK + 1;
    mlist_kernel<<<(unsigned)nchunks, 256, 0, ctx->stream>>>(T.small_primes.as<u32>(), T.n_small, Y, pcmin,
                                                             T.pi(), info_tmp.as<u64>(), T.rank_bits.as<u64>());
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        buf_free(info_tmp);
        pc_set_error(ctx, "mlist_kernel launch: %s", cudaGetErrorString(e));
        return PC_ECUDA;
    }
    DevBuf tmp;
    rc = buf_reserve(ctx, tmp, (nrw + 1) * sizeof(u32));
    if (rc) { buf_free(info_tmp); return rc; }
    popc_words_kernel<<<(unsigned)((nrw + 255) / 256), 256, 0, ctx->stream>>>(T.rank_bits.as<u64>(), nrw, tmp.as<u32>());
    rc = scan_exclusive_u32_to_u32(ctx, tmp.as<u32>(), T.rank_cnt.as<u32>(), nrw);
    u32 total = 0;
    if (rc == PC_OK) rc = copy_to_host(ctx, &total, T.rank_cnt.as<u32>() + nrw, sizeof(u32));
    if (rc == PC_OK) rc = buf_reserve(ctx, T.ml_m, ((u64)total + 1) * sizeof(u32));
    if (rc == PC_OK) rc = buf_reserve(ctx, T.ml_info, ((u64)total + 1) * sizeof(u32));
    if (rc == PC_OK) rc = buf_reserve(ctx, T.ml_gpf, ((u64)total + 1) * sizeof(u32));
    if (rc == PC_OK) rc = buf_reserve(ctx, T.ml_rcp, ((u64)total + 1) * sizeof(u64));
    if (rc == PC_OK) {
        mlist_scatter_kernel<<<(unsigned)((Y + 256) / 256), 256, 0, ctx->stream>>>(
            info_tmp.as<u64>(), T.rank_bits.as<u64>(), T.rank_cnt.as<u32>(), Y, T.ml_m.as<u32>(),
            T.ml_info.as<u32>(), T.ml_gpf.as<u32>());
        e = cudaGetLastError();
        if (e == cudaSuccess && total) {
            reciprocal_kernel<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(T.ml_m.as<u32>(), total,
                                                                                      T.ml_rcp.as<u64>());
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            pc_set_error(ctx, "m-list build: %s", cudaGetErrorString(e));
            rc = PC_ECUDA;
        }
    }
    buf_free(tmp);
    buf_free(info_tmp);
    ctx->stats.kernel_launches += 3;
    if (rc == PC_OK) {
        T.ml_limit = Y;
        T.ml_cmin = cmin;
        T.ml_n = total;
    }
    return rc;
}

int tables_ensure(pc_ctx* ctx, u64 pi_limit, u64 prime_limit, u64 ml_limit, u32 cmin)
{
    Tables& T = ctx->T;
    if (prime_limit < 64) prime_limit = 64;
    if (pi_limit < prime_limit + 2048) pi_limit = prime_limit + 2048;
    if (pi_limit < 65536) pi_limit = 65536;
    if (ctx->borrowed) {
        // a worker reads its parent's tables and must find them big enough
        if (T.n_small && pi_limit <= T.pi_limit && prime_limit <= T.prime_limit &&
            (ml_limit == 0 || (ml_limit <= T.ml_limit && cmin >= T.ml_cmin && ml_limit <= T.podd_limit &&
                               (ctx->params.pi_gather == 0 || ml_limit <= T.samp_limit))))
            return PC_OK;
        pc_set_error(ctx, "query needs tables beyond those prepared for the batch");
        return PC_EINVAL;
    }
    PC_TRY(ensure_small(ctx));
    PC_TRY(tables_wheel19(ctx));
    bool new_pi = false;
    // The table is sieved with the bootstrap primes <= 65536, which suffice up to
    // 65536^2 = 2^32 (every query x < 2^63 needs at most isqrt(x) < 3.04e9).
    static constexpr u64 PI_TABLE_MAX = (1ull << 32) - 1;
    if (pi_limit > PI_TABLE_MAX) {
        pc_set_error(ctx, "pi table limited to 2^32 - 1 (asked for %llu)", (unsigned long long)pi_limit);
        return PC_EINVAL;
    }
    if (pi_limit > T.pi_limit) {
        // grow geometrically so that a rising sequence of queries rebuilds rarely
        u64 lim = pi_limit;
        if (T.pi_limit && lim < T.pi_limit + T.pi_limit / 2) lim = T.pi_limit + T.pi_limit / 2;
        if (lim > PI_TABLE_MAX) lim = PI_TABLE_MAX;
        PC_TRY(build_pi(ctx, lim));
        new_pi = true;
    }
    if (new_pi || prime_limit > T.prime_limit) {
        u64 lim = prime_limit;
        if (T.prime_limit && lim < T.prime_limit + T.prime_limit / 2) lim = T.prime_limit + T.prime_limit / 2;
        if (lim + 2048 > T.pi_limit) lim = T.pi_limit - 2048;
        if (lim < prime_limit) lim = prime_limit;
        PC_TRY(build_primes(ctx, lim));
    }
    if (ml_limit > 0 && (ml_limit > T.ml_limit || cmin < T.ml_cmin)) {
        u64 lim = ml_limit;
        if (T.ml_limit && lim < T.ml_limit + T.ml_limit / 2 && cmin >= T.ml_cmin) lim = T.ml_limit + T.ml_limit / 2;
        if (lim > T.pi_limit) lim = T.pi_limit;
        if (lim < ml_limit) lim = ml_limit;
        u32 cm = cmin < T.ml_cmin ? cmin : T.ml_cmin;
        if (T.ml_limit == 0) cm = cmin;
        PC_TRY(ctx->params.m_source == 1 ? build_mlist_nested(ctx, lim, cm) : build_mlist(ctx, lim, cm));
        PC_TRY(build_sublists(ctx));
    }
    // the odd-number pi table serves the easy leaves, whose u stays below the m-list limit y
    if (ml_limit > 0 && T.ml_limit > T.podd_limit) PC_TRY(build_pi_odd(ctx, T.ml_limit));
    // the sampled table serves the easy leaves, whose u stays below the m-list limit y
    if (ctx->params.pi_gather == 1 && ml_limit > 0 && T.ml_limit > T.samp_limit)
        PC_TRY(build_sampled(ctx, T.ml_limit));
    return PC_OK;
}

__global__ void pi_values_kernel(PiTable t, const u64* v, u64* out, int n)
{
    int i = threadIdx.x;
    if (i < n) out[i] = pi_lookup(t, v[i]);
}

int tables_pi_values(pc_ctx* ctx, const u64* v, u64* out, int n)
{
    if (n > 32) return PC_EINVAL;
    for (int i = 0; i < n; i++)
        if (v[i] > ctx->T.pi_limit) {
            pc_set_error(ctx, "pi lookup %llu beyond table %llu", (unsigned long long)v[i],
                         (unsigned long long)ctx->T.pi_limit);
            return PC_EINVAL;
        }
    PC_TRY(buf_reserve(ctx, ctx->misc, 64 * sizeof(u64)));
    u64* d = ctx->misc.as<u64>();
    PC_CUDA(ctx, cudaMemcpyAsync(d, v, n * sizeof(u64), cudaMemcpyHostToDevice, ctx->stream));
    pi_values_kernel<<<1, 32, 0, ctx->stream>>>(ctx->T.pi(), d, d + 32, n);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches++;
    return copy_to_host(ctx, out, d + 32, n * sizeof(u64));
}

__global__ void pi_many_kernel(PiTable t, const u64* v, u64* out, u64 n)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = pi_lookup(t, v[i]);
}

int tables_pi_many(pc_ctx* ctx, const u64* v, u64* out, size_t n)
{
    if (n == 0) return PC_OK;
    for (size_t i = 0; i < n; i++)
        if (v[i] > ctx->T.pi_limit) {
            pc_set_error(ctx, "pi lookup %llu beyond table %llu", (unsigned long long)v[i],
                         (unsigned long long)ctx->T.pi_limit);
            return PC_EINVAL;
        }
    DevBuf tmp;
    int rc = buf_reserve(ctx, tmp, 2 * n * sizeof(u64));
    if (rc != PC_OK) return rc;
    u64* d = tmp.as<u64>();
    cudaError_t e = cudaMemcpyAsync(d, v, n * sizeof(u64), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        pi_many_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(ctx->T.pi(), d, d + n, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d + n, n * sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    buf_free(tmp);
    ctx->stats.kernel_launches++;
    if (e != cudaSuccess) {
        pc_set_error(ctx, "pi lookups: %s", cudaGetErrorString(e));
        return PC_ECUDA;
    }
    return PC_OK;
}

int tables_phi_c(pc_ctx* ctx, u32 c)
{
    Tables& T = ctx->T;
    if (c == 0 || T.phiT_ok[c]) return PC_OK;
    if (ctx->borrowed) {
        pc_set_error(ctx, "phi(., %u) table was not prepared for the batch", c);
        return PC_EINVAL;
    }
    PC_TRY(ensure_small(ctx));
    u32 Q = 1;
    static const u32 P8[8] = {1, 2, 3, 5, 7, 11, 13, 17};
    for (u32 i = 1; i <= c; i++) Q *= P8[i];
    DevBuf flags;
    PC_TRY(buf_reserve(ctx, flags, (Q + 1) * sizeof(u32)));
    int rc = buf_reserve(ctx, T.phiT[c], (Q + 1) * sizeof(u32));
    if (rc == PC_OK) {
        coprime_flags_kernel<<<(Q + 255) / 256, 256, 0, ctx->stream>>>(Q, c, T.small_primes.as<u32>(), flags.as<u32>());
        rc = scan_exclusive_u32_to_u32(ctx, flags.as<u32>(), T.phiT[c].as<u32>(), Q);
        if (rc == PC_OK) {
            cudaError_t e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) {
                pc_set_error(ctx, "phi table: %s", cudaGetErrorString(e));
                rc = PC_ECUDA;
            }
        }
    }
    buf_free(flags);
    ctx->stats.kernel_launches++;
    if (rc == PC_OK) T.phiT_ok[c] = true;
    return rc;
}
