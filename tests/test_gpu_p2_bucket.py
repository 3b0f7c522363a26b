"""GPU parity of the bucket sieve of Section 2.3 (pc_params.p2_bucket = 1) in P2: the
primes above the segment's bytes cross off only the multiples filed in each segment's
bucket, a wave of segments at a time.  The results must equal the oracle's P2, the
default P2 path, and pi(x) of the paper's Table 1."""
import pytest

import oracle as o
import paper_1503_01839_gb300 as pc

pytestmark = pytest.mark.gpu

CASES = [(10 ** 8, 1), (10 ** 9, 1), (10 ** 9, 5), (10 ** 10, 1), (10 ** 10, 4), (2 ** 35, 3), (10 ** 11, 2),
         (10 ** 12, 1), (10 ** 12, 6)]


def y_for(x, alpha):
    return min(alpha * o.iroot3(x), o.isqrt(x))


@pytest.fixture(scope="module")
def plain():
    with pc.Context(0) as c:
        yield c


@pytest.mark.parametrize("seg", [1024, 2048, 4096])
def test_p2_bucket_matches_oracle(plain, seg):
    with pc.Context(0, p2_bucket=1, seg_bytes=seg) as cx:
        for x, alpha in CASES:
            y = y_for(x, alpha)
            want = o.p2(x, o.pi_sieve(y))
            assert cx.p2(x, y) == want, (x, y, seg)
            assert plain.p2(x, y) == want


def test_p2_bucket_uses_waves(plain):
    # 1 KiB segments at x = 1e14, alpha = 1: z = 2.2e9 (about 7e4 segments), primes up to
    # 46 000 (about 4 600 of them above 1024): the buckets are filled in many waves
    x, y = 10 ** 14, o.iroot3(10 ** 14)
    with pc.Context(0, p2_bucket=1, seg_bytes=1024) as cx:
        got = cx.p2(x, y)
        launches = cx.stats()["kernel_launches"]
    assert got == plain.p2(x, y)
    assert launches > 20   # two launches per wave


def test_p2_bucket_first_segments(plain):
    # x at and around squares of the segment span: P2 sieves from the segment of isqrt(x)
    span = 30 * 2048
    with pc.Context(0, p2_bucket=1, seg_bytes=2048) as cx:
        for k, d in ((1, -1), (1, 0), (1, 1), (2, 0), (3, 7), (17, 5)):
            x = (k * span) ** 2 + d
            y = max(20000, o.iroot3(x) + 1)
            if y > o.isqrt(x):
                continue
            assert cx.p2(x, y) == o.p2(x, o.pi_sieve(y)), (x, y)


def test_pi_count_bucket_table1(pi_pow10, pi_pow2):
    # the default bucket segment (4 KiB = 2^15 bits) through pc_pi_count
    with pc.Context(0, p2_bucket=1) as cx:
        for n in (10, 12, 14, 16, 17, 18):
            assert cx.pi_count(10 ** n) == pi_pow10[n], n
        assert cx.pi_count(10 ** 14, 1) == pi_pow10[14]
        assert cx.pi_count(2 ** 59) == pi_pow2[59]
        assert cx.pi_count(2 ** 62) == pi_pow2[62]
