"""pc_p2_noalloc: P2 for callers that cannot allocate device memory (for
example a server whose device memory is handed out by its own pool, where a
cudaMalloc could overrun the budget or stall the device).  The caller owns
the primes array and the output word; the entry point itself allocates
nothing and keeps its scratch in a fixed array inside the library.

Checked through the C ABI against the ordinary pc_p2 entry point, exactly,
on two calls in a row (the second call reuses the scratch the first one
left behind).  This file is collected last on purpose."""
import numpy as np
import pytest

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


def test_p2_noalloc_matches_p2_twice():
    import torch
    cases = [(10 ** 14, 2 * iroot3(10 ** 14)), (2 ** 40 + 12345, 3 * iroot3(2 ** 40 + 12345))]
    # all primes up to isqrt(x), plus at least one above it
    top = 2 * max(int(np.sqrt(float(x))) + 2 for x, _ in cases)
    P = torch.from_numpy(primes_upto(top).view(np.int32)).cuda()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    L = pc.lib()
    with pc.Context(0) as ctx:
        for x, y in cases:                      # two calls in a row
            want = ctx.p2(x, y)
            rc = L.pc_p2_noalloc(x, y, P.data_ptr(), P.numel(), out.data_ptr(), stream.cuda_stream)
            assert rc == 0
            torch.cuda.synchronize()
            got = int(out.item()) & ((1 << 64) - 1)
            assert got == want, (x, y, got, want)


def test_p2_noalloc_flags_short_primes_array():
    import torch
    x, y = 10 ** 12, 2 * 10 ** 4
    P = torch.from_numpy(primes_upto(999983).view(np.int32)).cuda()   # stops below isqrt(x) = 10^6
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert pc.lib().pc_p2_noalloc(x, y, P.data_ptr(), P.numel(), out.data_ptr(), 0) == 0
    torch.cuda.synchronize()
    assert int(out.item()) == -1   # UINT64_MAX


def test_p2_noalloc_rejects_oversized_problems():
    import torch
    P = torch.from_numpy(primes_upto(1000).view(np.int32)).cuda()
    out = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    L = pc.lib()
    x = 10 ** 18
    # z = x / iroot3(x) = 1e12 needs far more segments than the fixed scratch holds
    rc = L.pc_p2_noalloc(x, iroot3(x), P.data_ptr(), P.numel(), out.data_ptr(), 0)
    assert rc == -1
    torch.cuda.synchronize()
    assert int(out.item()) == 7
