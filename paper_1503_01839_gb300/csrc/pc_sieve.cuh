// pc_sieve.cuh -- crossing off multiples in a mod-30 shared-memory segment.
//
// A segment covers the integers [L, L + 30*seg_bytes) with L a multiple of
// 30; byte i of the segment holds L + 30*i + R8[j] in bit j (see
// pc_common.cuh).  Multiples n = k*p of a prime p >= 7 that are coprime to 30
// are exactly those with k coprime to 30, so crossing off p means visiting
// k = 30*q + R8[j].  For fixed j the byte index advances by p per step of q
// and the bit inside the byte stays fixed at idx((p*R8[j]) mod 30).
#pragma once

#include "pc_common.cuh"

// first k >= k0 that is coprime to 30
__device__ __forceinline__ u64 coprime30_at_or_after(u64 k0)
{
    u32 r = (u32)(k0 % 30);
    return coprime30(r) ? k0 : k0 + next30(r);
}

// Cooperative cross-off of the multiples k*p, k >= kstart, k coprime to 30,
// inside the segment, by `nt` threads (t = 0..nt-1, nt a multiple of 8).
// Each thread handles one residue class j and every (nt/8)-th wheel round;
// consecutive threads take one class in consecutive rounds, p bytes apart (a
// warp of 256 or more threads: 32 rounds of one class), so that they spread
// over the banks instead of crowding into the words of one round.
// NEWLY(bitpos) is invoked for every bit that was set before this call
// cleared it (bit position relative to the segment).
template <class F>
__device__ __forceinline__ u32 cross_off_coop(u32* bits, u32 seg_bytes, u64 L, u32 p, u64 kstart,
                                               int t, int nt, F&& newly)
{
    const u32 rounds = (u32)nt >> 3;
    const int j = (u32)t / rounds;
    const u32 o = (u32)t % rounds;
    const u32 rj = r8(j);
    const u64 q0 = kstart / 30;
    const u32 pr = p * rj;                 // p < 2^27 here, so no overflow
    const u32 bit = idx30(pr % 30);
    const u64 Lb = L / 30;
    // byte(q) = p*q + pr/30 - L/30 for k = 30*q + rj
    u64 q = q0 + o;
    if (30 * q + rj < kstart) q += rounds;
    const u64 byte64 = (u64)p * q + pr / 30;
    if (byte64 < Lb || byte64 - Lb >= seg_bytes) return 0;   // the first cannot happen for kstart*p >= L
    // byte offsets inside the segment in 32 bits: below seg_bytes + step < 2^32
    const u32 step = p * rounds;
    u32 n = 0;
    for (u32 by = (u32)(byte64 - Lb); by < seg_bytes; by += step) {
        u32 pos = (by << 3) + bit;
        u32 mask = 1u << (pos & 31);
        u32 old = atomicAnd(&bits[pos >> 5], ~mask);
        if (old & mask) newly(pos);
        n++;
    }
    return n;   // multiples crossed off by this thread
}

// One thread crosses off the multiples k*p of one residue class,
// k = 30 q + R8[j] >= kstart: one per wheel round, p bytes apart.
// Returns the number of multiples crossed off.
template <class F>
__device__ __forceinline__ u32 cross_off_class(u32* bits, u32 seg_bytes, u64 L, u32 p, u64 kstart, u32 j,
                                               F&& newly)
{
    const u32 rj = r8(j);
    u64 q = kstart / 30;
    if (30 * q + rj < kstart) q++;
    const u32 pr = p * rj;                 // p < 2^27 here, so no overflow
    const u32 bit = idx30(pr % 30);
    const u64 byte64 = (u64)p * q + pr / 30;
    const u64 Lb = L / 30;
    if (byte64 < Lb || byte64 - Lb >= seg_bytes) return 0;   // the first cannot happen for kstart*p >= L
    u32 n = 0;
    for (u64 by = byte64 - Lb; by < seg_bytes; by += p, n++) {   // 64-bit: p may be near 2^32
        const u32 pos = ((u32)by << 3) + bit;
        const u32 mask = 1u << (pos & 31);
        const u32 old = atomicAnd(&bits[pos >> 5], ~mask);
        if (old & mask) newly(pos);
    }
    return n;
}

// One thread crosses off all multiples k*p (k >= kstart, k coprime to 30)
// of a large prime by walking k along the wheel.  Returns their number.
template <class F>
__device__ __forceinline__ u32 cross_off_single(u32* bits, u32 seg_bytes, u64 L, u32 p, u64 kstart,
                                                F&& newly)
{
    const u64 end = L + 30ull * seg_bytes;
    u64 k = coprime30_at_or_after(kstart);
    u32 r = (u32)(k % 30);
    u64 n = (u64)p * k;
    u32 cnt = 0;
    while (n < end) {
        cnt++;
        u32 rel = (u32)(n - L);
        u32 pos = (rel / 30) * 8 + idx30(rel % 30);
        u32 mask = 1u << (pos & 31);
        u32 old = atomicAnd(&bits[pos >> 5], ~mask);
        if (old & mask) newly(pos);
        u32 d = next30(r);
        r += d;
        if (r >= 30) r -= 30;
        n += (u64)p * d;
    }
    return cnt;
}

// Bit position of the integer n (coprime to 30) in the segment starting at L.
__device__ __forceinline__ u32 seg_pos(u64 n, u64 L)
{
    u32 rel = (u32)(n - L);
    return (rel / 30) * 8 + idx30(rel % 30);
}

// Number of bits before the first bit of integers > v, i.e. the count end
// for "integers in [L, v]" (v >= L).
__device__ __forceinline__ u32 seg_count_end(u64 v, u64 L)
{
    u32 rel = (u32)(v - L);
    return (rel / 30) * 8 + cntle30(rel % 30);
}

// Byte value of the wheel pattern of the primes 7 (depth 4) or 7 and 11
// (depth 5) for the 30 integers 30*g .. 30*g+29.
__device__ __forceinline__ u32 pattern_byte(u64 g, int depth)
{
    u32 v = 0xFF;
    if (depth >= 4) {
        u32 r7 = (u32)(g % 7);
        for (int j = 0; j < 8; j++)
            if ((30 * r7 + r8(j)) % 7 == 0) v &= ~(1u << j);
    }
    if (depth >= 5) {
        u32 r11 = (u32)(g % 11);
        for (int j = 0; j < 8; j++)
            if ((30 * r11 + r8(j)) % 11 == 0) v &= ~(1u << j);
    }
    return v;
}

// Fill the segment with the wheel state after the first `depth` primes
// (depth 3: 2,3,5 only; 4: also 7; 5: also 7 and 11).  patw must hold the
// 77 precomputed pattern words (see make_pattern_words).
__device__ __forceinline__ void fill_pattern(u32* bits, u32 seg_words, u64 L, const u32* patw, int depth)
{
    const u32 period = depth >= 5 ? 77 : (depth == 4 ? 7 : 1);
    const u64 gb = L / 30;   // first byte index
    for (u32 w = threadIdx.x; w < seg_words; w += blockDim.x) {
        u32 v;
        if (period == 1) v = 0xFFFFFFFFu;
        else v = patw[(u32)((gb + 4ull * w) % period)];
        bits[w] = v;
    }
}

// Fill from a pattern in global memory whose bytes repeat every `period` bytes and
// which runs at least seg_words + 1 words past any phase: the segment's bytes are one
// contiguous slice, read as aligned words and shifted by the phase's byte offset.
__device__ __forceinline__ void fill_pattern_global(u32* bits, u32 seg_words, u64 L, const u32* pat, u32 period)
{
    const u32 o = (u32)((L / 30) % period);
    const u32* src = pat + (o >> 2);
    const u32 sh = 8 * (o & 3);
    for (u32 w = threadIdx.x; w < seg_words; w += blockDim.x) bits[w] = __funnelshift_r(src[w], src[w + 1], sh);
}

// patw[ph] = 4 consecutive pattern bytes starting at phase ph (mod period)
__device__ __forceinline__ void make_pattern_words(u32* patw, int depth)
{
    const u32 period = depth >= 5 ? 77 : (depth == 4 ? 7 : 1);
    for (u32 ph = threadIdx.x; ph < period; ph += blockDim.x) {
        u32 v = 0;
        for (u32 i = 0; i < 4; i++) v |= pattern_byte((ph + i) % period, depth) << (8 * i);
        patw[ph] = v;
    }
}
