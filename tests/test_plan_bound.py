"""The arithmetic of the hard-leaf work planner's buffer bound, on CPU.

This checks the formula, restated here in Python, not the kernel: the
planner's own output (its item count on real and skewed inputs) is checked on
the GPU by tests/test_gpu_parity.py::test_planner_item_bound.

The planner (pc_hard.cu, plan_split_kernel) splits a segment whose estimated
leaves e outweigh both its sieve cost b and a fair share of the launch,
target = max(total / (4 * CTAs), 1), total = sum(b + e), into
R = min(1024, ceil(e / max(max(target - b, b), 1))) replicas.  The host sizes
the item buffer as segments + 8 * CTAs + 64 slots.  Since max(target - b, b)
>= target / 2, R <= 2 e / target + 1, and sum(e) <= total gives
sum(R) <= segments + 8 * CTAs.  This checks that bound on random and skewed
cost mixes (the kernel flags an overflow at run time as well)."""
import math
import random


def split(base, est, ctas):
    total = sum(b + e for b, e in zip(base, est))
    target = max(total / (4.0 * ctas), 1.0)
    rs = []
    for b, e in zip(base, est):
        r = 1
        if b + e > target and e > b:
            room = max(target - b, b)
            r = int(min(1024.0, math.ceil(e / max(room, 1.0))))
            r = max(r, 1)
        rs.append(r)
    return rs


def test_item_bound_random_and_skewed():
    rng = random.Random(7)
    for trial in range(400):
        n = rng.choice([1, 2, 7, 100, 5000])
        ctas = rng.choice([1, 152, 608, 1216])
        kind = trial % 4
        if kind == 0:      # uniform
            base = [rng.uniform(1e3, 1e5) for _ in range(n)]
            est = [rng.uniform(0, 1e5) for _ in range(n)]
        elif kind == 1:    # a few segments hold almost every leaf
            base = [rng.uniform(1e3, 1e4) for _ in range(n)]
            est = [rng.uniform(0, 10) for _ in range(n)]
            for i in rng.sample(range(n), min(n, 3)):
                est[i] = rng.uniform(1e8, 1e10)
        elif kind == 2:    # tiny costs: target clamps to 1
            base = [rng.uniform(0, 0.01) for _ in range(n)]
            est = [rng.uniform(0, 0.5) for _ in range(n)]
        else:              # leaves much larger than the sieve everywhere
            base = [128.0] * n
            est = [rng.uniform(1e4, 1e7) for _ in range(n)]
        rs = split(base, est, ctas)
        assert sum(rs) <= n + 8 * ctas, (trial, n, ctas, sum(rs))
        assert all(1 <= r <= 1024 for r in rs)


def test_item_bound_is_nearly_tight():
    # one segment with every leaf and a negligible sieve: R reaches about 8 * CTAs
    ctas = 16
    rs = split([1.0], [1e6], ctas)
    assert sum(rs) <= 1 + 8 * ctas
    assert sum(rs) >= 4 * ctas
