"""Seeded synthetic inputs shared by the tests and the benchmark.

The paper's workloads are integers x (the values of its Tables 1-3); there is
no dataset.  These generators only draw numbers: none of the method's
arithmetic lives here.  Floating point appears only in drawing exponents.
"""
from __future__ import annotations

import numpy as np


def log_uniform_x(n: int, lo_exp: float, hi_exp: float, seed: int) -> list[int]:
    """n integers x = floor(10^e), e ~ U(lo_exp, hi_exp), numpy default_rng(seed)."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(lo_exp, hi_exp, size=n)
    return [int(v) for v in np.floor(np.power(10.0, e))]


def batch_queries(n: int = 4096, seed: int = 0) -> list[int]:
    """The batched workload: n pi(x) queries, log10 x ~ U(8, 15)."""
    return log_uniform_x(n, 8.0, 15.0, seed)


def served_trace(n: int = 20000, rate_per_s: float = 2000.0, seed: int = 1, lo_exp: float = 9.0,
                 hi_exp: float = 17.0, phi_share: float = 0.2, a_lo: int = 5, a_hi: int = 5000) -> list[dict]:
    """A Poisson arrival stream: exponential inter-arrival times (mean 1/rate),
    a share phi_share of phi(x, a) requests with a ~ U{a_lo..a_hi}, the rest
    pi(x); log10 x ~ U(lo_exp, hi_exp).  Each entry: t_ms, kind ("pi"/"phi"),
    x, a (0 for pi)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1000.0 / rate_per_s, size=n)
    t = np.cumsum(gaps) - gaps[0]
    e = rng.uniform(lo_exp, hi_exp, size=n)
    xs = np.floor(np.power(10.0, e))
    is_phi = rng.uniform(0.0, 1.0, size=n) < phi_share
    a = rng.integers(a_lo, a_hi + 1, size=n)
    out = []
    for i in range(n):
        out.append({"t_ms": float(t[i]), "kind": "phi" if is_phi[i] else "pi", "x": int(xs[i]),
                    "a": int(a[i]) if is_phi[i] else 0})
    return out
