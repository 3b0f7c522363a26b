// pc_noalloc.cu -- P2(x, a) without any device allocation.
//
// Some callers cannot call cudaMalloc: a serving process whose device memory
// is owned up front by a pool allocator (a cudaMalloc outside the pool could
// exceed its budget), or a latency-critical path that cannot risk the implicit
// device-wide synchronization cudaMalloc / cudaFree may cause.  They own their
// inputs and outputs; this entry point adds no allocation of its own.  Its
// per-segment scratch lives in one file-scope __device__ array of fixed size,
// which every GPU that loads the library holds until the process exits.
//
// The computation is the P2 sieve of pc_p2.cu (same segments, same final-state
// counting, same carries), except that the primes come from the caller's
// array instead of the context's tables, so the query primes are found by
// binary search in that array.
#include <mutex>

#include "pc_internal.h"
#include "pc_sieve.cuh"

static constexpr u32 NA_SEG_BYTES = PC_NOALLOC_SEG_SPAN / 30;   // 32 KiB segments
static constexpr u32 NA_MAX_SEG = PC_NOALLOC_MAX_SEGMENTS;
static constexpr int NA_THREADS = 512;

struct NoAllocScratch {
    u32 queue;              // next segment to sieve (cleared by every call)
    u32 pad[63];
    u32 cnt[NA_MAX_SEG];    // set bits per segment in the final state
    u32 tally[NA_MAX_SEG];  // query primes answered per segment
    i64 acc[NA_MAX_SEG];    // sum of their local counts
};

// 512 KiB + 256 B of scratch, shared by all calls on a device.
static __device__ __align__(256) NoAllocScratch g_p2_scratch;

// number of entries of P[0..n) that are <= v (P ascending)
__device__ __forceinline__ u64 count_le(const u32* P, u64 n, u64 v)
{
    u64 lo = 0, hi = n;
    while (lo < hi) {
        u64 mid = (lo + hi) >> 1;
        if ((u64)P[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

struct NaArgs {
    u64 x, y, z, r;
    const u32* P;   // P[0] = 2, P[k-1] = p_k
    u64 n;
    u64 nseg;
    NoAllocScratch* S;
};

__global__ void __launch_bounds__(NA_THREADS) na_p2_sieve_kernel(NaArgs A)
{
    constexpr u32 seg_bytes = NA_SEG_BYTES, seg_words = seg_bytes / 4, nblk = seg_bytes / 128;
    constexpr u64 span = 30ull * seg_bytes;
    __shared__ __align__(16) u32 bits[seg_words];
    __shared__ u32 blk[nblk];
    __shared__ u32 pre[nblk + 1];
    __shared__ u32 patw[80];
    __shared__ u32 wsum[32];
    __shared__ i64 wacc[32];
    __shared__ u32 s_seg;
    __shared__ u64 s_B, s_a, s_K;
    const u64* bits64 = (const u64*)bits;
    const u32 tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        s_B = count_le(A.P, A.n, pc_isqrt(A.z));
        s_a = count_le(A.P, A.n, A.y);
        s_K = count_le(A.P, A.n, A.r);
    }
    __syncthreads();
    const u64 B = s_B, a = s_a, K = s_K;
    const int k0 = B >= 5 ? 5 : (int)B;
    make_pattern_words(patw, k0);
    for (;;) {
        if (tid == 0) s_seg = atomicAdd(&A.S->queue, 1u);
        __syncthreads();
        const u64 s = s_seg;
        __syncthreads();
        if (s >= A.nseg) break;
        const u64 L = s * span, end = L + span;
        fill_pattern(bits, seg_words, L, patw, k0);
        __syncthreads();
        auto none = [](u32) {};
        u64 b = k0 + 1;
        for (; b <= B; b++) {
            const u64 p = A.P[b - 1];
            if (p * 8 > seg_bytes) break;
            u64 ks = L ? (L + p - 1) / p : 0;
            if (ks < p) ks = p;
            cross_off_coop(bits, seg_bytes, L, (u32)p, ks, tid, NA_THREADS, none);
        }
        for (u64 bb = b + tid; bb <= B; bb += NA_THREADS) {
            const u64 p = A.P[bb - 1];
            u64 ks = L ? (L + p - 1) / p : 0;
            if (ks < p) ks = p;
            cross_off_single(bits, seg_bytes, L, (u32)p, ks, none);
        }
        for (u64 bb = k0 + 1 + tid; bb <= B; bb += NA_THREADS) {
            const u64 p = A.P[bb - 1];
            if (p >= end) break;
            if (p >= L) {
                u32 pos = seg_pos(p, L);
                atomicAnd(&bits[pos >> 5], ~(1u << (pos & 31)));
            }
        }
        __syncthreads();
        // one warp per 1024-bit block: lane l reads word 32k + l (32 banks, no conflict)
        for (u32 k = wid; k < nblk; k += NA_THREADS / 32) {
            const u32 c = __reduce_add_sync(0xffffffffu, (u32)__popc(bits[32 * k + lane]));
            if (lane == 0) blk[k] = c;
        }
        __syncthreads();
        if (wid == 0) {   // nblk = 256: eight blocks per lane
            u32 loc = 0;
            for (u32 k = 8 * lane; k < 8 * lane + 8; k++) loc += blk[k];
            u32 incl = loc;
            for (int o = 1; o < 32; o <<= 1) {
                u32 v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            u32 run = incl - loc;
            for (u32 k = 8 * lane; k < 8 * lane + 8; k++) {
                pre[k] = run;
                run += blk[k];
            }
            if (lane == 31) pre[nblk] = run;
        }
        __syncthreads();
        // query primes p_k, a < k <= K, with x/p_k in [L, end)
        const u64 plo = pc_max(A.x / end, A.y);
        const u64 phi = L ? pc_min(A.x / L, A.r) : A.r;
        i64 acc = 0;
        u32 tl = 0;
        if (phi > plo) {
            u64 k_lo = count_le(A.P, K, plo);   // primes <= plo (>= a since plo >= y)
            u64 k_hi = count_le(A.P, K, phi);
            for (u64 k = k_lo + tid; k < k_hi; k += NA_THREADS) {
                const u64 q = A.x / A.P[k];
                const u32 e = seg_count_end(q, L);
                const u32 eb = e >> 10, ew = e >> 6;
                u32 c = pre[eb];
                for (u32 ww = eb << 4; ww < ew; ww++) c += __popcll(bits64[ww]);
                if (e & 63) c += __popcll(bits64[ew] & ((1ull << (e & 63)) - 1));
                acc += c;
                tl++;
            }
        }
        (void)a;
        for (int o = 16; o; o >>= 1) {
            tl += __shfl_xor_sync(0xffffffffu, tl, o);
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
        }
        __syncthreads();
        if (lane == 0) {
            wsum[wid] = tl;
            wacc[wid] = acc;
        }
        __syncthreads();
        if (tid == 0) {
            u32 t = 0;
            i64 sa = 0;
            for (u32 w = 0; w < NA_THREADS / 32; w++) {
                t += wsum[w];
                sa += wacc[w];
            }
            A.S->tally[s] = t;
            A.S->cnt[s] = pre[nblk];
            A.S->acc[s] = sa;
        }
        __syncthreads();
    }
}

// P2 = sum_s (acc[s] + tally[s] * phi(L_s - 1, B)) + (K - a)(B - 1) - sum_{k=a+1}^{K} (k - 1)
__global__ void __launch_bounds__(1024) na_p2_combine_kernel(NaArgs A, u64* out)
{
    __shared__ u64 wsum[32];
    __shared__ u64 s_carry;
    __shared__ i128 red[32];
    const u32 lane = threadIdx.x & 31, wid = threadIdx.x >> 5, NT = blockDim.x;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    i128 dot = 0;
    for (u64 base = 0; base < A.nseg; base += NT) {
        const u64 s = base + threadIdx.x;
        const u64 v = s < A.nseg ? A.S->cnt[s] : 0;
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
        if (s < A.nseg) dot += (i128)A.S->acc[s] + (i128)A.S->tally[s] * (i128)carry;
        __syncthreads();
        if (threadIdx.x == NT - 1) s_carry = c0 + wsum[wid] + incl;
        __syncthreads();
    }
    dot = block_sum_i128(dot, red);
    if (threadIdx.x == 0) {
        const u64 B = count_le(A.P, A.n, pc_isqrt(A.z));
        const u64 a = count_le(A.P, A.n, A.y);
        const u64 K = count_le(A.P, A.n, A.r);
        const bool ok = A.n > 0 && (u64)A.P[A.n - 1] >= A.r;   // the caller's primes reach isqrt(x)
        i128 v = dot;
        if (K > a) {
            const i128 nq = (i128)(K - a);
            const i128 sk = ((i128)K * (i128)(K - 1) - (i128)a * (i128)(a ? a - 1 : 0)) / 2;
            v += nq * (i128)(B - 1) - sk;
        } else {
            v = 0;
        }
        *out = ok ? (u64)v : ~0ull;
    }
}

// one-time, per-device address of the scratch array
static std::mutex g_na_mutex;
static void* g_na_ptr[128];
static bool g_na_ok[128];

extern "C" int pc_p2_noalloc(uint64_t x, uint64_t y, const uint32_t* primes, uint64_t n_primes, uint64_t* out,
                             void* stream)
{
    if (!primes || !out || n_primes == 0) return PC_EINVAL;
    if (x >> 63) return PC_ERANGE;
    if (x < 1 || y < pc_iroot3(x) || y > pc_isqrt(x)) return PC_EINVAL;
    const u64 z = x / y;
    if (z < 25) return PC_EINVAL;                                  // fewer than three sieving primes
    const u64 nseg = z / PC_NOALLOC_SEG_SPAN + 1;
    if (nseg > NA_MAX_SEG) return PC_EINVAL;                       // beyond the fixed scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return PC_ECUDA;
    void* ptr = nullptr;
    {
        std::lock_guard<std::mutex> g(g_na_mutex);
        if (!g_na_ok[dev]) {
            if (cudaGetSymbolAddress(&g_na_ptr[dev], g_p2_scratch) != cudaSuccess) return PC_ECUDA;
            g_na_ok[dev] = true;
        }
        ptr = g_na_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    NaArgs A;
    A.x = x;
    A.y = y;
    A.z = z;
    A.r = pc_isqrt(x);
    A.P = primes;
    A.n = n_primes;
    A.nseg = nseg;
    A.S = (NoAllocScratch*)ptr;
    if (cudaMemsetAsync(&A.S->queue, 0, sizeof(u32), st) != cudaSuccess) return PC_ECUDA;
    int ctas = 0, sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PC_ECUDA;
    ctas = sms * 2;
    if ((u64)ctas > nseg) ctas = (int)nseg;
    na_p2_sieve_kernel<<<ctas, NA_THREADS, 0, st>>>(A);
    if (cudaGetLastError() != cudaSuccess) return PC_ECUDA;
    na_p2_combine_kernel<<<1, 1024, 0, st>>>(A, (u64*)out);
    if (cudaGetLastError() != cudaSuccess) return PC_ECUDA;
    return PC_OK;
}
