"""Pins for the CPU oracle: each function is checked against something other
than itself -- the values printed in Tables 1 and 2, brute force on small
inputs, exact root identities, and the recurrence/identities of Sections 3-4.
"""
import math
import random

import pytest

import oracle as o
from conftest import read_table


def small_primes(n):
    f = bytearray([1]) * (n + 1)
    f[0:2] = b"\x00\x00"
    for p in range(2, math.isqrt(n) + 1):
        if f[p]:
            f[p * p::p] = bytearray(len(f[p * p::p]))
    return [i for i in range(n + 1) if f[i]]


PR = small_primes(2100000)


def pi_small(v):
    import bisect
    return bisect.bisect_right(PR, v)


# ---------------------------------------------------------------- roots

def test_isqrt_exhaustive_small():
    for n in range(0, 200000):
        assert o.isqrt(n) == math.isqrt(n)


def test_iroot3_exhaustive_small():
    r = 0
    for n in range(0, 200000):
        while (r + 1) ** 3 <= n:
            r += 1
        assert o.iroot3(n) == r


def test_roots_near_powers_up_to_2_63():
    rng = random.Random(7)
    ks = [rng.randrange(2, 3037000499) for _ in range(2000)] + [3037000499, 2, 3, 1 << 31]
    for k in ks:
        for n in (k * k - 1, k * k, k * k + 1):
            if n < 1 << 63:
                assert o.isqrt(n) == math.isqrt(n)
    for k in [rng.randrange(2, 2097151) for _ in range(2000)] + [2097151, 2, 3]:
        for n in (k ** 3 - 1, k ** 3, k ** 3 + 1):
            if n < 1 << 63:
                r = o.iroot3(n)
                assert r ** 3 <= n < (r + 1) ** 3
    top = (1 << 63) - 1
    assert o.isqrt(top) == math.isqrt(top)
    r = o.iroot3(top)
    assert r ** 3 <= top < (r + 1) ** 3


# ------------------------------------------------------------------ O-A

def test_pi_sieve_table1(pi_pow10):
    for n in range(1, 10):
        assert o.pi_sieve(10 ** n) == pi_pow10[n], n


@pytest.mark.slow
def test_pi_sieve_table1_1e10(pi_pow10):
    # the brute-force check of the smallest workload, pi(10^10)
    assert o.pi_sieve(10 ** 10) == pi_pow10[10]


def test_pi_sieve_table2(pi_pow2):
    for m in range(1, 31):
        assert o.pi_sieve(2 ** m) == pi_pow2[m], m


def test_pi_sieve_small_exhaustive():
    for x in range(0, 5000):
        assert o.pi_sieve(x) == pi_small(x)


def test_nth_prime_vs_sieve_list():
    # p_k by the plain sieve list: every k up to 2000, then a sample up to 10^4
    for k in range(1, 2001):
        assert o.nth_prime(k) == PR[k - 1], k
    rng = random.Random(11)
    for k in rng.sample(range(2001, 10001), 300) + [10000]:
        assert o.nth_prime(k) == PR[k - 1], k


def test_nth_prime_table1(pi_pow10):
    # Table 1 fixes p_k at k = pi(10^n): the largest prime <= 10^n, the next one above it
    assert o.nth_prime(168) == 997 and pi_pow10[3] == 168
    assert o.nth_prime(78498) == 999983 and pi_pow10[6] == 78498
    for n in range(1, 9):
        k = pi_pow10[n]
        assert o.nth_prime(k) <= 10 ** n < o.nth_prime(k + 1), n


def test_s2_hard_range_splits_add_up():
    # a shard's hard leaves (its range sieved alone, carries from the recursion of
    # Eq. (4.1)) over any split of [1, z] add up to the whole S2_hard and leaf count
    rng = random.Random(3)
    for x, y, c in [(10 ** 9, 1000, 5), (10 ** 10, 4308, 5), (10 ** 10, 2154, 3), (3 * 10 ** 9, 1442 * 3, 7)]:
        whole = o.leaf_sums(x, y, c)
        z = x // y
        cuts = sorted({1, z + 1, *[rng.randrange(2, z) for _ in range(5)]})
        parts = [o.s2_hard_range(x, y, c, lo, hi) for lo, hi in zip(cuts[:-1], cuts[1:])]
        assert sum(p[0] for p in parts) == whole["S2_hard"], (x, y, c)
        assert sum(p[1] for p in parts) == whole["n_hard"], (x, y, c)


def test_phi_brute_definition_small():
    # direct gcd count against the definition of phi(x, a) (Section 3)
    for x in range(0, 400, 7):
        for a in range(0, 8):
            prod = 1
            for p in PR[:a]:
                prod *= p
            want = sum(1 for n in range(1, x + 1) if math.gcd(n, prod) == 1)
            assert o.phi_brute(x, a) == want


def test_phi_brute_closed_forms():
    # phi(x, pi(sqrt x)) = pi(x) - pi(sqrt x) + 1 (Legendre)
    for x in [10 ** 5, 123457, 999999]:
        a = pi_small(math.isqrt(x))
        assert o.phi_brute(x, a) == pi_small(x) - a + 1
    # phi(k * 30030, 6) = k * phi(30030) with phi(30030) = 5760
    for k in (1, 2, 17):
        assert o.phi_brute(k * 30030, 6) == k * 5760


# ------------------------------------------------------------------ O-B

def test_phi_rec_vs_brute_random():
    rng = random.Random(11)
    for _ in range(300):
        x = rng.randrange(0, 10 ** 6)
        a = rng.randrange(0, 120)
        assert o.phi_rec(x, a) == o.phi_brute(x, a), (x, a)


def test_phi_rec_small_table_forces_recursion():
    # a tiny pi table makes the recursion do almost all the work
    rng = random.Random(12)
    for _ in range(100):
        x = rng.randrange(0, 3 * 10 ** 5)
        a = rng.randrange(0, 60)
        assert o.phi_rec(x, a, 64) == o.phi_brute(x, a)


def test_phi_rec_edges():
    assert o.phi_rec(0, 5) == 0
    assert o.phi_rec(12345, 0) == 12345
    assert o.phi_rec(1, 100) == 1
    assert o.phi_rec(10 ** 6, 168) == pi_small(10 ** 6) - 168 + 1


def test_pi_meissel_table1(pi_pow10):
    for n in range(1, 13):
        assert o.pi_meissel(10 ** n) == pi_pow10[n], n


def test_pi_meissel_table2(pi_pow2):
    for m in range(1, 41):
        assert o.pi_meissel(2 ** m) == pi_pow2[m], m


def test_pi_meissel_small_exhaustive():
    for x in range(0, 3000):
        assert o.pi_meissel(x) == pi_small(x), x


def test_identity_several_y(pi_pow10, pi_pow2):
    # pi(x) = phi(x, a) + a - 1 - P2(x, a), a = pi(y), any iroot3 <= y <= isqrt
    cases = [(10 ** 8, pi_pow10[8]), (10 ** 9, pi_pow10[9]), (2 ** 33, pi_pow2[33])]
    for x, want in cases:
        lo, hi = o.iroot3(x), o.isqrt(x)
        for y in sorted({lo, 2 * lo, 5 * lo, (lo + hi) // 2, hi}):
            a = o.pi_sieve(y)
            assert o.phi_rec(x, a) + a - 1 - o.p2(x, a) == want, (x, y)


def test_p2_by_definition_small():
    for x in [1000, 12345, 10 ** 5, 777777]:
        for a in range(0, 12):
            r = math.isqrt(x)
            want = sum(pi_small(x // PR[b - 1]) - b + 1 for b in range(a + 1, pi_small(r) + 1))
            assert o.p2(x, a) == want


# ------------------------------------------------------------------ O-C

def decomposed(s):
    return s["S1"] + s["S2_triv"] + s["S2_easy"] + s["S2_hard"] + s["a"] - 1 - s["P2"]


@pytest.mark.parametrize("n", range(4, 13))
def test_leaf_decomposition_table1(pi_pow10, n):
    x = 10 ** n
    lo, hi = o.iroot3(x), o.isqrt(x)
    for alpha in (1, 2, 4, 10):
        y = min(alpha * lo, hi)
        for c in (0, 1, 3, 5, 7):
            s = o.leaf_sums(x, y, min(c, o.pi_sieve(y)))
            assert decomposed(s) == pi_pow10[n], (n, alpha, c)


@pytest.mark.parametrize("m", [20, 27, 31, 36, 39])
def test_leaf_decomposition_table2(pi_pow2, m):
    x = 2 ** m
    y = min(3 * o.iroot3(x), o.isqrt(x))
    s = o.leaf_sums(x, y, 5)
    assert decomposed(s) == pi_pow2[m]


def test_leaf_decomposition_small_exhaustive():
    for x in range(8, 2500):
        lo, hi = o.iroot3(x), o.isqrt(x)
        for y in {lo, hi}:
            a = o.pi_sieve(y)
            c = min(2, a)
            assert decomposed(o.leaf_sums(x, y, c)) == pi_small(x), (x, y)


def test_alpha1_all_special_leaves_hard():
    # with y = iroot3(x), u >= x / y^2 >= y for every special leaf
    s = o.leaf_sums(10 ** 10, 2154, 5)
    assert s["n_triv"] == 0 and s["n_easy"] == 0 and s["n_hard"] == 51164


def test_truncated_phi_matches_recursion():
    # phi(x, a) = S1 + S2 for a < pi(y): the tree truncated at p_a
    rng = random.Random(5)
    for x in (10 ** 5, 3 * 10 ** 5, 10 ** 7):
        for y in (46, 100, 300):
            if y > o.isqrt(x):
                continue
            piy = o.pi_sieve(y)
            for a in sorted({2, 3, 5, 9, 17, 31, piy // 2, piy - 1, piy} | {rng.randrange(1, piy + 1) for _ in range(4)}):
                if a < 1 or a > piy:
                    continue
                for c in (0, 2, min(5, a)):
                    if c > a:
                        continue
                    s = o.leaf_sums(x, y, c, a)
                    got = s["S1"] + s["S2_triv"] + s["S2_easy"] + s["S2_hard"]
                    assert got == o.phi_brute(x, a), (x, y, a, c)


def test_leaf_classes_pinned_by_brute_force():
    """Each class sum of O-C equals sum(-mu * phi(u, b-1)) over leaves listed
    by an independent trial-division enumeration, with phi by brute force;
    trivial leaves have phi = 1 and easy leaves phi = pi(u) - b + 2."""
    for x, y, c, a in [(10 ** 5, 60, 2, 0), (2 * 10 ** 5, 200, 3, 0),
                       (10 ** 6, 500, 5, 0), (10 ** 6, 300, 1, 40), (777777, 91, 0, 0)]:
        s = o.leaf_sums(x, y, c, a)
        sums = [0, 0, 0]
        counts = [0, 0, 0]
        for b, m, u, mu, cls in o.list_leaves(x, y, c, a):
            ph = o.phi_brute(u, b - 1)
            if cls == 0:
                assert ph == 1
            elif cls == 1:
                assert ph == pi_small(u) - b + 2
            sums[cls] += -mu * ph
            counts[cls] += 1
        assert [s["S2_triv"], s["S2_easy"], s["S2_hard"]] == sums, (x, y, c)
        assert [s["n_triv"], s["n_easy"], s["n_hard"]] == counts


def test_ordinary_leaves_brute():
    # S1 = sum mu(n) phi(x/n, c) over n <= y, n = 1 or lpf(n) > p_c, by brute force
    for x, y, c in [(10 ** 5, 46, 3), (10 ** 6, 100, 5), (10 ** 6, 100, 7)]:
        tot = 0
        for n in range(1, y + 1):
            f, r, d, mu, sq = [], n, 2, 1, True
            while d * d <= r:
                if r % d == 0:
                    r //= d
                    if r % d == 0:
                        sq = False
                        break
                    f.append(d)
                    mu = -mu
                d += 1
            if not sq:
                continue
            if r > 1:
                f.append(r)
                mu = -mu
            if n > 1 and min(f) <= PR[c - 1] if c > 0 else False:
                continue
            tot += mu * o.phi_brute(x // n, c)
        assert o.leaf_sums(x, y, c)["S1"] == tot


def test_b_bound_counts():
    s = o.leaf_sums(10 ** 10, 2154, 5)
    assert s["z"] == 10 ** 10 // 2154 and s["B"] == pi_small(math.isqrt(s["z"]))


def test_golden_tables_shape():
    t10 = dict(read_table("pi_pow10.txt"))
    t2 = dict(read_table("pi_pow2.txt"))
    assert sorted(t10) == list(range(1, 19))
    assert sorted(t2) == list(range(1, 63))
    assert t10[18] == 24739954287740860 and t2[59] == 14458792895301660
