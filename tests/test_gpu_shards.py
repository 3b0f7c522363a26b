"""Independent shards of the hard-leaf sieve (Section 4): starting values
phi(m, b) for every b, and S2_hard split into shards that never exchange
counts, whose sum must equal the unsplit sum (and the oracle's)."""
import pytest

import oracle as o
import paper_1503_01839_gb300 as pc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    with pc.Context(0, streams=8) as c:
        yield c


@pytest.mark.parametrize("m", [1, 2, 30, 1000, 10 ** 6 + 7, 3 * 10 ** 6 - 1])
def test_phi_starts_vs_brute_force(ctx, m):
    c = 5
    bmax = 120
    got = ctx.phi_starts(m, c, bmax)
    assert len(got) == bmax - c + 1
    for b in list(range(c, 40)) + [60, 87, 119, 120]:
        assert got[b - c] == o.phi_brute(m, b), (m, b)


def test_phi_starts_large_vs_phi(ctx):
    # every case of the split at once: combinatorial (small p_b), Legendre
    # (m^(1/3) < p_b <= sqrt m), and p_b > sqrt m
    m = 5 * 10 ** 9 + 11
    c, bmax = 3, 6000          # p_6000 = 59359 < sqrt(m) = 70710 < p_7400
    got = ctx.phi_starts(m, c, bmax)
    for b in (3, 4, 10, 100, 300, 800, 2000, 5999, 6000):
        assert got[b - c] == ctx.phi(m, b), b
    bmax2 = 7400               # beyond pi(sqrt m): each further prime removes only itself
    got2 = ctx.phi_starts(m, c, bmax2)
    assert got2[:len(got)] == got
    assert got2[-1] == ctx.phi(m, bmax2)


@pytest.mark.parametrize("x,alpha", [(10 ** 11, 2), (3 * 10 ** 12, 4), (10 ** 13, 6)])
def test_shards_sum_to_whole_small(ctx, x, alpha):
    y = min(alpha * o.iroot3(x), o.isqrt(x))
    c = 5
    whole = ctx.s2_hard(x, y, c)
    if x <= 3 * 10 ** 12:
        assert whole == o.leaf_sums(x, y, c)["S2_hard"]
    for n in (2, 3, 7):
        parts = [ctx.s2_hard_shard(x, y, c, k, n) for k in range(n)]
        assert sum(parts) == whole, (x, n, parts)


def test_shards_sum_to_whole_large(ctx):
    x, y, c = 10 ** 16, 20 * 215443, 5
    whole = ctx.s2_hard(x, y, c)
    assert sum(ctx.s2_hard_shard(x, y, c, k, 4) for k in range(4)) == whole


def test_shard_errors(ctx):
    with pytest.raises(pc.PicountError):
        ctx.s2_hard_shard(10 ** 12, 10 ** 4, 5, 3, 3)
    with pytest.raises(pc.PicountError):
        ctx.s2_hard_shard(10 ** 12, 10 ** 4, 5, 0, 0)
