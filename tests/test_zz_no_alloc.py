"""pc_p2_noalloc: P2 for callers that cannot allocate device memory (for
example a server whose device memory is handed out by its own pool, where a
cudaMalloc could overrun the budget or stall the device).  The caller owns
the primes array and the output word; the entry point itself allocates
nothing and keeps its scratch in a fixed array inside the library.

Checked through the C ABI against the CPU oracle's P2 and against the
ordinary pc_p2 entry point, exactly, on calls in a row (each call reuses the
scratch the previous one left behind), including the edges of its domain:
the smallest z it accepts, y = isqrt(x) (no query primes), a primes array
that ends exactly at a prime isqrt(x), and z at the largest segment count the
fixed scratch holds.  This file is collected last on purpose."""
import bisect

import numpy as np
import pytest

import oracle
import paper_1503_01839_gb300 as pc

pytestmark = pytest.mark.gpu


def primes_upto(n):
    f = np.ones(n + 1, dtype=bool)
    f[:2] = False
    for p in range(2, int(n ** 0.5) + 1):
        if f[p]:
            f[p * p::p] = False
    return np.nonzero(f)[0].astype(np.uint32)


def iroot3(n):
    r = int(round(n ** (1.0 / 3)))
    while r ** 3 > n:
        r -= 1
    while (r + 1) ** 3 <= n:
        r += 1
    return r


def isqrt(n):
    import math
    return math.isqrt(n)


def run_noalloc(x, y, P, out):
    import torch
    stream = torch.cuda.current_stream()
    rc = pc.lib().pc_p2_noalloc(x, y, P.data_ptr(), P.numel(), out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return rc, int(out.item()) & ((1 << 64) - 1)


def test_p2_noalloc_matches_oracle_and_p2():
    import torch
    cases = [(10 ** 14, 2 * iroot3(10 ** 14)),           # many segments
             (2 ** 40 + 12345, 3 * iroot3(2 ** 40 + 12345)),
             (10 ** 12, 10 ** 6),                         # y = isqrt(x): no query prime, P2 = 0
             (125, 5),                                    # the smallest z accepted: z = 25
             (10 ** 11 + 7, iroot3(10 ** 11 + 7))]        # y at its lower bound
    top = 2 * max(isqrt(x) + 2 for x, _ in cases)
    PR = primes_upto(top)
    P = torch.from_numpy(PR.view(np.int32)).cuda()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pc.Context(0) as ctx:
        for x, y in cases:                      # calls in a row on the shared scratch
            a = bisect.bisect_right(PR.tolist(), y)
            want = oracle.p2(x, a)
            assert ctx.p2(x, y) == want, (x, y)
            rc, got = run_noalloc(x, y, P, out)
            assert rc == 0
            assert got == want, (x, y, got, want)
            assert run_noalloc(x, y, P, out) == (0, want)   # again, on what the last call left


def test_p2_noalloc_primes_ending_at_isqrt():
    import torch
    # isqrt(x) = 997 is prime: an array that ends exactly there covers it
    x, y = 997 * 997, 100
    PR = primes_upto(997)
    assert int(PR[-1]) == 997
    P = torch.from_numpy(PR.view(np.int32)).cuda()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc, got = run_noalloc(x, y, P, out)
    assert rc == 0 and got == oracle.p2(x, bisect.bisect_right(PR.tolist(), y))


def test_p2_noalloc_at_the_segment_limit():
    import torch
    span, max_seg = 983040, 32768
    z_max = max_seg * span - 1               # z / span + 1 == max_seg
    y = 10 ** 6
    x = z_max * y + y - 1                    # x // y == z_max, iroot3(x) <= y <= isqrt(x)
    assert x // y == z_max and iroot3(x) <= y <= isqrt(x)
    P = torch.from_numpy(primes_upto(isqrt(x) + 1000).view(np.int32)).cuda()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pc.Context(0) as ctx:
        want = ctx.p2(x, y)
    assert run_noalloc(x, y, P, out) == (0, want)
    # one integer more needs one segment more than the scratch holds: refused, out untouched
    x2 = (z_max + 1) * y
    out.fill_(7)
    rc, got = run_noalloc(x2, y, P, out)
    assert rc == -1 and got == 7


def test_p2_noalloc_flags_short_primes_array():
    import torch
    x, y = 10 ** 12, 2 * 10 ** 4
    P = torch.from_numpy(primes_upto(999983).view(np.int32)).cuda()   # stops below isqrt(x) = 10^6
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert pc.lib().pc_p2_noalloc(x, y, P.data_ptr(), P.numel(), out.data_ptr(), 0) == 0
    torch.cuda.synchronize()
    assert int(out.item()) == -1   # UINT64_MAX


def test_p2_noalloc_rejects_out_of_domain():
    import torch
    P = torch.from_numpy(primes_upto(1000).view(np.int32)).cuda()
    out = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    L = pc.lib()
    x = 10 ** 18
    # z = x / iroot3(x) = 1e12 needs far more segments than the fixed scratch holds
    assert L.pc_p2_noalloc(x, iroot3(x), P.data_ptr(), P.numel(), out.data_ptr(), 0) == -1
    # z = 24 < 25
    assert L.pc_p2_noalloc(120, 5, P.data_ptr(), P.numel(), out.data_ptr(), 0) == -1
    torch.cuda.synchronize()
    assert int(out.item()) == 7
