"""GPU parity: every part of the CUDA path against the CPU oracle, through
the C ABI, bit for bit (all quantities are exact integers)."""
import math
import random

import pytest

import oracle as o
import paper_1503_01839_gb300 as pc
from conftest import read_table

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx_small():
    # 1 KiB segments = 30720 integers: small inputs still span many segments
    with pc.Context(0, seg_bytes=1024, ctas_per_sm=4, threads=256) as c:
        yield c


@pytest.fixture(scope="module")
def ctx():
    with pc.Context(0) as c:
        yield c


def y_for(x, alpha):
    return min(alpha * o.iroot3(x), o.isqrt(x))


CASES = [(10 ** 6, 1), (10 ** 6, 10), (3 * 10 ** 7, 2), (10 ** 9, 1), (10 ** 9, 5), (10 ** 10, 1),
         (10 ** 10, 4), (2 ** 35, 3), (10 ** 11, 2), (10 ** 12, 1), (10 ** 12, 6)]


@pytest.mark.parametrize("x,alpha", CASES)
def test_leaf_sums_parity(ctx_small, ctx, x, alpha):
    y = y_for(x, alpha)
    for c in (0, 2, 3, 5, 7):
        want = o.leaf_sums(x, y, c)
        for cx in (ctx_small, ctx):
            got = cx.leaf_sums(x, y, c)
            for k in ("S1", "S2_triv", "S2_easy", "S2_hard", "P2"):
                assert got[k] == want[k], (x, y, c, k, got[k], want[k])


@pytest.mark.parametrize("x,alpha", CASES[:8])
def test_s2_hard_parity(ctx_small, x, alpha):
    y = y_for(x, alpha)
    for c in range(0, 8):
        want = o.leaf_sums(x, y, c)["S2_hard"]
        assert ctx_small.s2_hard(x, y, c) == want, (x, y, c)


def test_s2_hard_many_segment_sizes():
    x, y, c = 10 ** 11, 4641 * 2, 5
    want = o.leaf_sums(x, y, c)["S2_hard"]
    for sb, cps, wb in [(1024, 1, 0), (2048, 2, 0), (4096, 4, 0), (8192, 0, 0), (16384, 3, 0), (65536, 0, 0),
                        (65536, 1, 0), (65536, 0, 8192), (131072, 0, 8192), (131072, 0, 4096), (32768, 0, 1024),
                        (16384, 0, 2048)]:
        with pc.Context(0, seg_bytes=sb, ctas_per_sm=cps, warp_bytes=wb) as cx:
            assert cx.s2_hard(x, y, c) == want, (sb, cps, wb)


def test_planner_item_bound():
    # the device planner's work items (segments, heavy ones split into replicas) stay
    # within the buffer it is given, segments + 8 x resident CTAs + 64, on inputs whose
    # leaves crowd into a few segments (alpha 1: every special leaf is hard) and on
    # ordinary ones; the results stay exact
    import torch
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    for x, alpha, sb in [(10 ** 12, 1, 1024), (10 ** 12, 1, 32768), (10 ** 11, 6, 4096), (10 ** 14, 1, 131072),
                         (10 ** 10, 1, 1024)]:
        y = y_for(x, alpha)
        want = o.leaf_sums(x, y, 5)["S2_hard"] if x <= 10 ** 12 else None
        with pc.Context(0, seg_bytes=sb) as cx:
            got = cx.s2_hard(x, y, 5)
            st = cx.stats()
        if want is not None:
            assert got == want, (x, alpha, sb)
        assert 1 <= st["work_items"] <= st["segments"] + 8 * 8 * n_sm + 64, (x, alpha, sb, st)
        # every (segment, prime) step belongs to exactly one item (the step count also
        # holds one wheel-count row entry per segment)
        assert st["item_steps"] + st["segments"] >= st["steps"]


def test_truncated_phi_parts(ctx_small):
    # phi(x, a) = S1 + S2 with the tree truncated at p_a (gpf(m) <= p_a)
    for x, y, a, c in [(10 ** 7, 300, 30, 5), (10 ** 9, 1000, 100, 5), (10 ** 9, 1000, 168, 3),
                       (10 ** 10, 2154, 7, 2), (10 ** 10, 5000, 300, 5)]:
        want = o.leaf_sums(x, y, c, a)
        got = ctx_small.leaf_sums(x, y, c, a)
        for k in ("S1", "S2_triv", "S2_easy", "S2_hard"):
            assert got[k] == want[k], (x, y, a, c, k)


def test_p2_parity(ctx_small, ctx):
    for x, alpha in CASES:
        y = y_for(x, alpha)
        a = o.pi_sieve(y)
        want = o.p2(x, a)
        assert ctx_small.p2(x, y) == want
        assert ctx.p2(x, y) == want


def test_p2_first_sieved_segment(ctx, ctx_small):
    # P2 sieves from the segment that holds isqrt(x), its starting count phi(L - 1, B) taken
    # from the pi table: x at and around squares of the segment span (30 * 32768 bytes for
    # the default context below z = 2^30, 30 * 1024 for the small one)
    for cx, span in ((ctx, 30 * 32768), (ctx_small, 30 * 1024)):
        for k, d in ((1, -1), (1, 0), (1, 1), (2, 0), (3, 7)):
            x = (k * span) ** 2 + d
            y = max(20000, o.iroot3(x) + 1)   # the domain of pc_p2: iroot3(x) <= y <= isqrt(x)
            if y > math.isqrt(x):
                continue
            assert cx.p2(x, y) == o.p2(x, o.pi_sieve(y)), (x, y, span)


def test_pi_count_table1(ctx, pi_pow10):
    for n in range(1, 19):
        assert ctx.pi_count(10 ** n) == pi_pow10[n], n


def test_pi_count_table2(ctx, pi_pow2):
    for m in range(1, 63):
        assert ctx.pi_count(2 ** m) == pi_pow2[m], m


def test_pi_count_alpha_segment_invariance(pi_pow10):
    # Section 5: the same value with different (alpha, c, L)
    x = 10 ** 14
    for sb, alpha, c in [(1024, 1, 5), (8192, 3, 3), (65536, 8, 7), (4096, 20, 5), (32768, 40, 4)]:
        with pc.Context(0, seg_bytes=sb, c=c) as cx:
            assert cx.pi_count(x, alpha) == pi_pow10[14], (sb, alpha, c)


def test_pi_count_small_x_exhaustive(ctx):
    rng = random.Random(3)
    xs = list(range(0, 200)) + [rng.randrange(200, 1 << 22) for _ in range(60)] + \
        [(1 << 20) - 1, 1 << 20, (1 << 20) + 1]
    for x in xs:
        assert ctx.pi_count(x) == o.pi_sieve(x), x


def test_pi_count_random_mid(ctx_small, ctx):
    rng = random.Random(4)
    for _ in range(12):
        x = rng.randrange(1 << 21, 10 ** 10)
        want = o.pi_meissel(x)
        assert ctx.pi_count(x) == want, x
        assert ctx_small.pi_count(x, rng.randrange(1, 8)) == want, x


def test_phi_vs_oracle(ctx):
    rng = random.Random(5)
    for _ in range(40):
        x = rng.randrange(0, 3 * 10 ** 6)
        a = rng.randrange(0, 250)
        assert ctx.phi(x, a) == o.phi_brute(x, a), (x, a)
    for a in (10, 100, 1000):
        assert ctx.phi(10 ** 12, a) == o.phi_rec(10 ** 12, a), a


def test_phi_1e14_recurrence(ctx):
    # Eq. (4.1) at full size: phi(x, a) = phi(x, a-1) - phi(x/p_a, a-1)
    x = 10 ** 14
    for a in (10, 100, 1000):
        pa = o.nth_prime(a)
        assert ctx.phi(x, a) == ctx.phi(x, a - 1) - ctx.phi(x // pa, a - 1), a


def test_phi_legendre_branch(ctx, pi_pow10):
    # a >= pi(isqrt x): phi(x, a) = pi(x) - a + 1 (Section 4)
    x = 10 ** 12
    a = o.pi_sieve(10 ** 6)
    assert ctx.phi(x, a) == pi_pow10[12] - a + 1
    # p_a > x: only n = 1 is left
    assert ctx.phi(x, 10 ** 11) == 1
    assert ctx.phi(x, 10 ** 9) == pi_pow10[12] - 10 ** 9 + 1


def test_s2_hard_tiny_inputs(ctx_small):
    for x in list(range(8, 400, 7)) + [1000, 4096, 10007, 65536]:
        for y in sorted({o.iroot3(x), o.isqrt(x)}):
            a = o.pi_sieve(y)
            for c in range(0, min(7, a) + 1):
                assert ctx_small.s2_hard(x, y, c) == o.leaf_sums(x, y, c)["S2_hard"], (x, y, c)


def test_errors(ctx):
    with pytest.raises(pc.PicountError) as e:
        ctx.pi_count(1 << 63)
    assert e.value.code == -2
    with pytest.raises(pc.PicountError) as e:
        ctx.s2_hard(10 ** 10, 10, 5)       # y < iroot3(x)
    assert e.value.code == -1
    with pytest.raises(pc.PicountError) as e:
        ctx.s2_hard(10 ** 10, 2154, 8)     # c > 7
    assert e.value.code == -1
    # the context stays usable after an error
    assert ctx.pi_count(10 ** 9) == 50847534


def test_batch_matches_single(ctx):
    rng = random.Random(6)
    xs = [int(10 ** rng.uniform(3, 12)) for _ in range(40)]
    got = ctx.pi_count_batch(xs)
    assert got == [ctx.pi_count(x) for x in xs]


def test_full_size_pins(pi_pow10, pi_pow2):
    # the largest workloads, in the launch configuration the benchmark uses
    with pc.Context(0) as cx:
        for alpha in (20, 30, 40):
            assert cx.pi_count(10 ** 18, alpha) == pi_pow10[18], alpha
        for alpha in (20, 30):
            assert cx.pi_count(2 ** 59, alpha) == pi_pow2[59], alpha
        # S2_hard at 1e18 cannot be brute-forced: it must not depend on the
        # segment geometry
        y = 20 * 10 ** 6
        h = cx.s2_hard(10 ** 18, y, 5)
    with pc.Context(0, seg_bytes=32768, ctas_per_sm=1) as cx:
        assert cx.s2_hard(10 ** 18, y, 5) == h


def _phi_wheel(x, a):
    """phi(x, a) for a <= 7 from the textbook periodicity: with P the product of
    the first a primes, phi(x, a) = (x // P) * phi(P, a) + phi(x mod P, a)."""
    ps = [2, 3, 5, 7, 11, 13, 17][:a]
    P = 1
    for p in ps:
        P *= p
    r = x % P
    ok = [all(n % p for p in ps) for n in range(1, P + 1)]
    return (x // P) * sum(ok) + sum(ok[:r])


def test_full_size_phi_properties(pi_pow10):
    # properties that hold at any size, at the largest x of the benchmark
    x = 10 ** 18
    with pc.Context(0) as cx:
        for a in (1, 3, 5, 7):
            assert cx.phi(x, a) == _phi_wheel(x, a), a
        for a in (100, 1000):
            pa = o.nth_prime(a)
            assert cx.phi(x, a) == cx.phi(x, a - 1) - cx.phi(x // pa, a - 1), a
        # a >= pi(isqrt x): phi(x, a) = pi(x) - a + 1 (Section 4)
        a = 50847534 + 10   # pi(10^9) + 10
        assert cx.phi(x, a) == pi_pow10[18] - a + 1


def test_largest_x_is_consistent():
    # x = 2^63 - 1, the top of the domain: every alpha and segment size must agree
    x = (1 << 63) - 1
    with pc.Context(0) as cx:
        v = cx.pi_count(x, 0)
        assert cx.pi_count(x, 12) == v
    with pc.Context(0, seg_bytes=65536) as cx:
        assert cx.pi_count(x, 30) == v
    with pc.Context(0) as cx:
        assert cx.pi_count(1 << 62, 0) < v


@pytest.mark.parametrize("x,alpha", [(10 ** 9, 5), (10 ** 11, 2), (10 ** 12, 6), (2 ** 35, 3)])
def test_sampled_pi_table_parity(x, alpha):
    # easy leaves reading pi(u) from the sampled table of Section 2.1 instead of the popcount table
    y = y_for(x, alpha)
    with pc.Context(0, pi_gather=1) as cx:
        for c in (0, 3, 5):
            want = o.leaf_sums(x, y, c)
            got = cx.leaf_sums(x, y, c)
            for k in ("S1", "S2_triv", "S2_easy", "S2_hard", "P2"):
                assert got[k] == want[k], (x, y, c, k, got[k], want[k])


@pytest.mark.parametrize("x,alpha", [(10 ** 9, 5), (10 ** 11, 2), (10 ** 12, 6), (2 ** 35, 3), (10 ** 10, 40)])
def test_nested_mlist_parity(x, alpha):
    # the m-list built by the nested loops of Section 2.2 (products of distinct primes,
    # mu = (-1)^n) instead of the sieve of least prime factors: every leaf sum as the oracle's
    y = y_for(x, alpha)
    with pc.Context(0, m_source=1) as cx:
        for c in (0, 3, 5, 7):
            want = o.leaf_sums(x, y, c)
            got = cx.leaf_sums(x, y, c)
            for k in ("S1", "S2_triv", "S2_easy", "S2_hard", "P2"):
                assert got[k] == want[k], (x, y, c, k, got[k], want[k])


def test_nested_mlist_full_size(pi_pow10):
    with pc.Context(0, m_source=1) as cx:
        assert cx.pi_count(10 ** 16) == pi_pow10[16]
        assert cx.pi_count(10 ** 18) == pi_pow10[18]
        xs = [10 ** 9 + 7, 10 ** 11 + 1, 10 ** 15 + 3]
        assert cx.pi_count_batch(xs) == [o.pi_meissel(x) if x <= 10 ** 11 + 1 else cx.pi_count(x) for x in xs]


def test_sampled_pi_table_full_size(pi_pow10):
    with pc.Context(0, pi_gather=1) as cx:
        assert cx.pi_count(10 ** 16) == pi_pow10[16]
        assert cx.pi_count(10 ** 18, 48) == pi_pow10[18]
