"""The bound on a P2 bucket's entries (the bucket sieve of Section 2.3), on CPU.

This checks the counting argument, restated here in Python, not the kernel: the kernel's
buckets never overflowing is checked on the GPU by tests/test_gpu_p2_bucket.py (an overflow
there sets an error flag and the call fails).

A bucket prime p (p > seg_bytes) has its multiples k p, k >= p and k coprime to 30, filed
under the segment [L, L + span) that holds them, span = 30 seg_bytes.  The multiples in
one segment have consecutive k, at most m = floor((span - 1) / p) + 1 of them; m <= 30
since p > seg_bytes, and any 30 consecutive integers hold exactly 8 coprime to 30, so a
segment receives at most min(m, 8) entries from p.  Brute force over 400 segments from p^2
on, for 400 primes at three segment sizes, confirms it (and the sharper count of the densest
run of m consecutive integers), and that some segment meets it."""
import math


def primes_upto(n):
    sieve = bytearray([1]) * (n + 1)
    sieve[0:2] = b"\x00\x00"
    for i in range(2, math.isqrt(n) + 1):
        if sieve[i]:
            sieve[i * i :: i] = bytearray(len(sieve[i * i :: i]))
    return [i for i in range(n + 1) if sieve[i]]


def entries(p, L, span):
    """Multiples k p in [L, L + span) with k >= p and gcd(k, 30) = 1."""
    k0 = max(p, -(-L // p))
    k1 = (L + span - 1) // p
    return sum(1 for k in range(k0, k1 + 1) if math.gcd(k, 30) == 1)


def bound(p, span):
    return min((span - 1) // p + 1, 8)


def densest(m):
    """Most integers coprime to 30 among m consecutive integers."""
    return max(sum(1 for k in range(r, r + m) if math.gcd(k, 30) == 1) for r in range(30))


def test_bucket_bound_holds():
    ps = primes_upto(40000)
    for seg_bytes in (64, 128, 1024):
        span = 30 * seg_bytes
        bucket = [p for p in ps if p > seg_bytes][:400]
        attained = 0
        for p in bucket:
            m = (span - 1) // p + 1
            assert m <= 30
            assert densest(m) <= bound(p, span)
            worst = max(entries(p, s * span, span) for s in range(p * p // span, p * p // span + 400))
            assert worst <= densest(m) <= bound(p, span), (p, seg_bytes, worst)
            attained += worst == bound(p, span)
        assert attained > 0   # the bound is met by some segment of some prime


def test_bucket_entries_sum_to_crossings():
    # over a whole range, the entries filed for p are exactly its multiples with a cofactor
    # coprime to 30 from p^2 on: the crossings the plain sieve makes
    span = 30 * 128
    for p in (131, 257, 1021, 4093):
        nseg = 300
        filed = sum(entries(p, s * span, span) for s in range(nseg))
        direct = sum(1 for k in range(p, (nseg * span - 1) // p + 1) if math.gcd(k, 30) == 1)
        assert filed == direct, p
