"""The arithmetic of the clustered easy leaves taken by their pi value, on CPU.

This restates in Python the identity the easy-leaf kernel uses (pc_leaves.cu,
the clustered chunks of easy_chunk), not the kernel: the kernel's sums are
checked on the GPU by the leaf-sum and pi(x) parity tests.  For fixed b, with
X = x / p_b and the clustered primes q_i, i in [im, i1), the leaves add
pi(X // q_i) - b + 2 each.  Grouped by l = pi(X // q_i): the q with
pi(X // q) = l are those with X // p_(l+1) < q <= X // p_l, so with
G(l) = #{i in [im, i1) : q_i <= X // p_l} the group of l has G(l) - G(l+1)
leaves, and l runs over [pi(X // q_(i1-1)), pi(X // q_im)].  A chunk of
consecutive l computes every G once and takes G(l + 1) from the next l, so the
chunks must also meet exactly at their boundaries."""
import bisect
import math
import random

N = 200000


def primes_upto(n):
    s = bytearray([1]) * (n + 1)
    s[0] = s[1] = 0
    for i in range(2, math.isqrt(n) + 1):
        if s[i]:
            s[i * i::i] = bytearray(len(s[i * i::i]))
    return [i for i in range(n + 1) if s[i]]


P = [1] + primes_upto(N)   # 1-based: P[k] = k-th prime


def pi(v):
    return bisect.bisect_right(P, v) - 1


def leaves_one_by_one(X, b, im, i1):
    return sum(pi(X // P[i]) - b + 2 for i in range(im, i1))


def leaves_by_value(X, b, im, i1, chunk):
    nq, qlast = i1 - im, P[i1 - 1]

    def G(l):
        v = X // P[l]
        if v >= qlast:
            return nq
        return min(max(pi(v) - im + 1, 0), nq)

    l0, l1 = pi(X // P[i1 - 1]), pi(X // P[im])
    total = 0
    for base in range(l0, l1 + 1, chunk):   # chunks of consecutive l, each on its own
        end = min(l1, base + chunk - 1)
        g = [G(l) for l in range(base, end + 2)]
        total += sum((g[k] - g[k + 1]) * (base + k - b + 2) for k in range(end - base + 1))
    return total


def test_runs_by_value_equal_the_leaves():
    rng = random.Random(3)
    for _ in range(300):
        b = rng.randrange(4, 60)
        p = P[b]
        X = rng.randrange(p * p, 10 ** 9) // 1
        # clustered q: prime indices above b with q^2 >= 2 X (u <= q/2), inside the table
        qc = math.isqrt(2 * X - 1) + 1
        im = max(pi(qc - 1) + 1, b + 1)
        if im >= len(P) - 2:
            continue
        top = min(len(P) - 1, im + 5000, pi(X // p) + 1)   # easy: u = X // q >= p_b
        if top <= im + 1:
            continue
        i1 = rng.randrange(im + 1, top)
        for chunk in (1, 31, 3968):
            assert leaves_by_value(X, b, im, i1, chunk) == leaves_one_by_one(X, b, im, i1), (X, b, im, i1, chunk)


def test_single_prime_and_tiny_ranges():
    # every q with u = X // q >= p_b, from one prime to just past a 31-value pass
    for b in (4, 5, 10):
        for X in (10 ** 6 + 7, 99991 * 13, 7 * 10 ** 8):
            qc = math.isqrt(2 * X - 1) + 1
            im = max(pi(qc - 1) + 1, b + 1)
            top = pi(X // P[b]) + 1
            for i1 in (im + 1, im + 2, im + 31, im + 32, top):
                if im < i1 <= top:
                    assert leaves_by_value(X, b, im, i1, 31) == leaves_one_by_one(X, b, im, i1)
