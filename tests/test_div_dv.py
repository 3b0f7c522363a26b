"""The arithmetic of the 32-bit reciprocal division of the easy leaves, on CPU.

This restates in Python the formula of div_dv and pc_dv (pc_common.cuh), not
the kernel: the kernels' results are checked on the GPU by the pi(x) parity
tests.  For a divisor d with s = floor(log2 d), the record holds
v = floor((2^(32+s) - 1) / d) < 2^32; the estimate floor(n v / 2^(32+s)),
taken as floor(floor(n v / 2^32) / 2^s) from two 32x32-bit products, is the
quotient floor(n / d) or one less whenever that quotient is below 2^31, so one
remainder test gives the quotient exactly."""
import random


def dv(d):
    s = d.bit_length() - 1
    v = ((1 << (32 + s)) - 1) // d
    assert v < (1 << 32)
    return v, s


def estimate(n, d):
    v, s = dv(d)
    lo = (n & 0xFFFFFFFF) * v
    hi = (n >> 32) * v + (lo >> 32)
    assert hi < (1 << 64)
    return hi >> s


def div_dv(n, d):
    q = estimate(n, d)
    if n - q * d >= d:
        q += 1
    return q


def check(n, d):
    q = n // d
    e = estimate(n, d)
    assert e in (q - 1, q), (n, d, e, q)
    assert div_dv(n, d) == q


def test_estimate_within_one_random():
    rng = random.Random(11)
    for _ in range(200000):
        d = rng.randrange(2, 1 << 30)
        q = rng.randrange(0, 1 << 31)
        n = q * d + rng.randrange(0, d)
        if n >= 1 << 64:
            continue
        check(n, d)


def test_estimate_at_the_edges():
    # powers of two and their neighbours, the largest quotient, the largest remainder
    ds = [2, 3, 5, 7, 13]
    for s in range(2, 31):
        ds += [(1 << s) - 1, 1 << s, (1 << s) + 1]
    for d in ds:
        for q in (0, 1, 2, (1 << 31) - 1, (1 << 31) - 2, (1 << 30), 12345):
            for r in (0, 1, d - 1):
                n = q * d + r
                if r < d and n < (1 << 64):
                    check(n, d)


def test_easy_leaf_quotients():
    # the shapes of the easy leaves at x = 10^18, y = 4.8e7: x/p_b up to 2^43, q <= y
    rng = random.Random(5)
    for _ in range(100000):
        xp = rng.randrange(1 << 30, 1 << 43)
        q = rng.randrange(7, 48000000)
        if xp // q < (1 << 31):
            check(xp, q)
