// pc_common.cuh -- shared device/host helpers for the picount CUDA library.
//
// Number layout used by every sieve in this library ("mod-30 wheel"): byte i
// of a bitset stands for the numbers 30*i .. 30*i+29, and bit j of that byte
// for 30*i + R8[j], R8 = {1,7,11,13,17,19,23,29} (the residues coprime to
// 2*3*5).  Multiples of 2, 3, 5 are never stored.  This is the wheel of
// Section 2.1 / 2.2 with c = 3; deeper wheels (7, 11) are applied as
// periodic byte patterns.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

typedef unsigned long long u64;
typedef long long i64;
typedef unsigned int u32;
typedef int i32;
typedef unsigned short u16;
typedef unsigned char u8;
typedef __int128 i128;
typedef unsigned __int128 u128;

#define PC_HD __host__ __device__ __forceinline__

// ------------------------------------------------------------- wheel residues
// R8MASK has bit r set for the residues r mod 30 that are coprime to 30,
// R8PACK holds R8[0..7] in 5-bit fields.  Everything below is bit
// arithmetic, so lanes with different residues never serialize on a table.
#define PC_R8MASK 0x208A2882u
#define PC_R8PACK (1ull | 7ull << 5 | 11ull << 10 | 13ull << 15 | 17ull << 20 | 19ull << 25 | 23ull << 30 | 29ull << 35)

__device__ __forceinline__ u32 r8(u32 j) { return (u32)(PC_R8PACK >> (5 * j)) & 31u; }            // R8[j]
__device__ __forceinline__ bool coprime30(u32 r) { return (PC_R8MASK >> r) & 1u; }                  // gcd(r, 30) == 1
__device__ __forceinline__ u32 cntle30(u32 r) { return __popc(PC_R8MASK & ((2u << r) - 1u)); }      // #R8 <= r
__device__ __forceinline__ u32 idx30(u32 r) { return cntle30(r) - 1u; }                               // j with R8[j] == r
__device__ __forceinline__ u32 next30(u32 r)                                                          // to next coprime > r
{
    const u32 m = PC_R8MASK >> (r + 1);
    return m ? (u32)__ffs(m) : 31u - r;
}

// ------------------------------------------------------ exact integer roots
PC_HD int pc_bitlen(u64 n) { int k = 0; while (n) { k++; n >>= 1; } return k; }

// floor(sqrt(n)) by integer Newton iteration from an upper bound (no FP).
PC_HD u64 pc_isqrt(u64 n)
{
    if (n < 2) return n;
    u64 x = 1ull << ((pc_bitlen(n) + 1) / 2);
    for (;;) {
        u64 y = (x + n / x) >> 1;
        if (y >= x) break;
        x = y;
    }
    return x;
}

// floor(cbrt(n)) by integer Newton iteration plus an exact correction.
PC_HD u64 pc_iroot3(u64 n)
{
    if (n < 8) return n ? 1 : 0;
    u64 x = 1ull << ((pc_bitlen(n) + 2) / 3);
    for (;;) {
        u64 y = (2 * x + n / (x * x)) / 3;
        if (y >= x) break;
        x = y;
    }
    while ((u128)x * x * x > n) x--;
    while ((u128)(x + 1) * (x + 1) * (x + 1) <= n) x++;
    return x;
}

PC_HD u64 pc_min(u64 a, u64 b) { return a < b ? a : b; }

// Division by an invariant divisor through a precomputed reciprocal
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): v = floor((2^64 - 1) / d) for d >= 1.  For
// n < 2^63, n / d - 1 < n * v / 2^64 <= n / d (v > (2^64 - 1 - d) / d and
// (1 + d) / d <= 2 give n * v / 2^64 > n / d - n / 2^63), so
// q = floor(n * v / 2^64) is floor(n / d) or one less, and one remainder test
// fixes it.  Every dividend in this library is at most x < 2^63.
__device__ __forceinline__ u64 div_rcp(u64 n, u64 d, u64 v)
{
    const u64 q = __umul64hi(n, v);
    return n - q * d >= d ? q + 1 : q;
}
PC_HD u64 pc_max(u64 a, u64 b) { return a > b ? a : b; }

// floor(n / d) for d = low word of dv, v = high word = floor((2^(32+s) - 1) / d),
// s = floor(log2 d), whenever the quotient is below 2^31.  v < 2^32 and
// v > 2^(32+s)/d - 1, so n v / 2^(32+s) falls short of n/d by less than
// n / 2^(32+s) < 2 (n/d) / 2^32 < 1: the estimate is the quotient or one less,
// and one remainder test settles it.  Two 32x32 -> 64-bit products instead of
// the 64-bit high product of div_rcp.
__device__ __forceinline__ u32 div_dv(u64 n, u64 dv)
{
    const u32 d = (u32)dv, v = (u32)(dv >> 32);
    const u64 lo = (u64)(u32)n * v;
    const u64 hi = (u64)(u32)(n >> 32) * v + (lo >> 32);   // floor(n v / 2^32)
    u32 q = (u32)(hi >> (31 - __clz(d)));
    if (n - (u64)q * d >= d) q++;
    return q;
}
PC_HD u64 pc_dv(u32 d)
{
    if (d == 0) return 0;
    int s = 31;
    while (!((d >> s) & 1u)) s--;
    return (u64)d | ((((1ull << (32 + s)) - 1) / d) << 32);
}

// ----------------------------------------------------------- lookup tables
// pi table: mod-30 bitset of the primes in [0, limit] (1 is cleared), one
// record per 240 numbers: the 64-bit word and the number of set bits in all
// earlier words, so that one 16-byte load answers a lookup.
struct __align__(16) PiRec {
    u64 bits;
    u32 cnt;
    u32 pad;
};

struct PiTable {
    const PiRec* rec;
    u64 limit;
};

// The low e bits (0 <= e <= 64) of w, moved to the top of the word: a left
// shift by 64 - e, which PTX clamps at 64 (the result is then 0).
__device__ __forceinline__ u64 low_bits_top(u64 w, u32 e)
{
    u64 r;
    asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(w), "r"(64u - e));
    return r;
}

// pi(v) for 0 <= v <= limit.
__device__ __forceinline__ u64 pi_lookup(const PiTable& t, u64 v)
{
    // v <= limit < 2^32; one division by 30 gives the record (8 groups of 30
    // integers each) and the bit inside it
    const u32 v32 = (u32)v, q30 = v32 / 30;
    const u64 small = (v32 >= 2) + (v32 >= 3) + (v32 >= 5);
    const u32 e = 8 * (q30 & 7) + cntle30(v32 - 30 * q30);
    const uint4 q = __ldg((const uint4*)(t.rec + (q30 >> 3)));
    return small + q.z + __popcll(low_bits_top((u64)q.x | ((u64)q.y << 32), e));
}

// Odd-number pi table: record w covers [64w, 64w + 64); .x holds one bit per
// odd number 64w + 2j + 1 (j = 0..31) that is prime, with bit 0 of record 0
// (the number 1) standing for the prime 2, and .y = pi(64w - 1).  pi(u) for
// 2 <= u <= limit is .y plus the bits of the odd numbers <= u: a shift, an
// 8-byte load and one 32-bit popcount, with no division and no wheel residue.
__device__ __forceinline__ u32 pi_odd(const uint2* t, u32 u)
{
    const uint2 r = __ldg(t + (u >> 6));
    const u32 e = ((u & 63u) + 1u) >> 1;   // odd numbers <= u in the record, 0..32
    return r.y + __popc(__funnelshift_lc(0u, r.x, 32u - e));   // r.x << (32 - e), 0 when e = 0
}

// rank structure over a plain bitset of [0, limit]: rank(v) = #set bits <= v.
struct RankTable {
    const u64* bits;
    const u32* cnt;   // set bits in words < w
    u64 limit;
};

__device__ __forceinline__ u64 rank_lookup(const RankTable& t, u64 v)
{
    if (v > t.limit) v = t.limit;
    u64 w = v >> 6;
    u32 sh = (u32)(v & 63);
    u64 mask = sh == 63 ? ~0ull : ((1ull << (sh + 1)) - 1);
    return t.cnt[w] + __popcll(__ldg(t.bits + w) & mask);
}

// squarefree m-list, ascending m.  info = (lpf_index << 1) | (mu == -1).
struct MList {
    const u32* m;
    const u32* info;
    const u32* gpf;   // prime index of the greatest prime factor
    const u64* rcp;   // floor((2^64 - 1) / m)
    u64 n;
    u64 limit;        // every squarefree m <= limit with lpf(m) > p_cmin is listed
    u32 cmin;
};

// ------------------------------------------------------------- reductions
__device__ __forceinline__ i64 warp_sum_i64(i64 v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ i128 warp_sum_i128(i128 v)
{
    u64 lo = (u64)v;
    i64 hi = (i64)(v >> 64);
    for (int o = 16; o; o >>= 1) {
        u64 lo2 = __shfl_xor_sync(0xffffffffu, lo, o);
        i64 hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
        u64 s = lo + lo2;
        hi = hi + hi2 + (s < lo);
        lo = s;
    }
    return ((i128)hi << 64) | (i128)lo;
}

// CTA-wide i128 sum; result valid in thread 0.  scratch: >= 32 i128.
__device__ __forceinline__ i128 block_sum_i128(i128 v, i128* scratch)
{
    v = warp_sum_i128(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    i128 r = 0;
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? scratch[lane] : (i128)0;
        r = warp_sum_i128(r);
    }
    return r;
}

// --------------------------------------------------------------- results
// Partial sums are written as i128 into per-block slots and summed by
// reduce_i128_kernel (pc_engine.cu).
struct I128Pair { i64 lo; i64 hi; };

__device__ __forceinline__ void store_i128(I128Pair* p, i128 v)
{
    p->lo = (i64)(u64)v;
    p->hi = (i64)(v >> 64);
}

__device__ __forceinline__ i128 load_i128(const I128Pair* p)
{
    return ((i128)p->hi << 64) | (i128)(u64)p->lo;
}
