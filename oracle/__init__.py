"""CPU oracle for the combinatorial pi(x) method (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain,
single-threaded C written from the paper's definitions) through ctypes and
shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-Wall", "-shared", "-fPIC",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u64, i64 = ctypes.c_uint64, ctypes.c_int64
            p_i64 = ctypes.POINTER(ctypes.c_int64)
            for name, res, args in [
                ("orc_isqrt", u64, [u64]),
                ("orc_iroot3", u64, [u64]),
                ("orc_pi_sieve", u64, [u64]),
                ("orc_phi_brute", u64, [u64, u64]),
                ("orc_phi_rec", u64, [u64, u64, u64]),
                ("orc_p2", ctypes.c_int, [u64, u64, p_i64]),
                ("orc_pi_meissel", u64, [u64, u64]),
                ("orc_leaf_sums", ctypes.c_int, [u64, u64, ctypes.c_uint32, u64, p_i64]),
                ("orc_list_leaves", i64, [u64, u64, ctypes.c_uint32, u64, p_i64, i64]),
                ("orc_nth_prime", u64, [u64]),
                ("orc_s2_hard_range", ctypes.c_int, [u64, u64, ctypes.c_uint32, u64, u64, p_i64]),
            ]:
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _i128(lo: int, hi: int) -> int:
    return (hi << 64) + (lo & ((1 << 64) - 1))


def isqrt(n: int) -> int:
    return int(_load().orc_isqrt(n))


def iroot3(n: int) -> int:
    return int(_load().orc_iroot3(n))


def pi_sieve(x: int) -> int:
    """O-A: pi(x) by a segmented sieve of Eratosthenes."""
    return int(_load().orc_pi_sieve(x))


def phi_brute(x: int, a: int) -> int:
    """O-A: phi(x, a) by directly marking multiples of p_1..p_a."""
    return int(_load().orc_phi_brute(x, a))


def phi_rec(x: int, a: int, table: int = 0) -> int:
    """O-B: phi(x, a) by the naive recursion of Eq. (4.1) with textbook cut-offs."""
    return int(_load().orc_phi_rec(x, a, table))


def p2(x: int, a: int) -> int:
    """P2(x, a) = sum_{a < b <= pi(isqrt x)} (pi(x/p_b) - b + 1)."""
    out = (ctypes.c_int64 * 2)()
    _load().orc_p2(x, a, out)
    return _i128(out[0], out[1])


def pi_meissel(x: int, y: int = 0) -> int:
    """O-B: pi(x) = phi(x, a) + a - 1 - P2(x, a) with a = pi(y)."""
    return int(_load().orc_pi_meissel(x, y))


def nth_prime(k: int) -> int:
    return int(_load().orc_nth_prime(k))


def s2_hard_range(x: int, y: int, c: int, lo: int, hi: int) -> tuple:
    """The hard leaves with lo <= u < hi only, as one shard sees them: the range
    sieved alone, phi(lo - 1, b - 1) from the recursion of Eq. (4.1).
    Returns (sum, number of leaves)."""
    out = (ctypes.c_int64 * 3)()
    if _load().orc_s2_hard_range(x, y, c, lo, hi, out) != 0:
        raise ValueError("oracle domain error")
    return _i128(out[0], out[1]), out[2]


def leaf_sums(x: int, y: int, c: int, a: int = 0) -> dict:
    """O-C: per-term brute force of the leaf decomposition of phi(x, a)."""
    out = (ctypes.c_int64 * 17)()
    rc = _load().orc_leaf_sums(x, y, c, a, out)
    if rc != 0:
        raise ValueError("oracle domain error for x=%d y=%d c=%d a=%d" % (x, y, c, a))
    return {
        "S1": _i128(out[0], out[1]),
        "S2_triv": _i128(out[2], out[3]),
        "S2_easy": _i128(out[4], out[5]),
        "S2_hard": _i128(out[6], out[7]),
        "P2": _i128(out[8], out[9]),
        "a": out[10],
        "n_triv": out[11],
        "n_easy": out[12],
        "n_hard": out[13],
        "n_ord": out[14],
        "z": out[15],
        "B": out[16],
    }


def list_leaves(x: int, y: int, c: int, a: int = 0, cap: int = 1 << 20):
    """Special leaves (b, m, u, mu, cls) of phi(x, a) for tiny x, factoring
    every m by trial division.  cls: 0 trivial, 1 easy, 2 hard."""
    buf = (ctypes.c_int64 * (4 * cap))()
    n = _load().orc_list_leaves(x, y, c, a, buf, cap)
    if n < 0:
        raise ValueError("list_leaves: bad domain or cap too small")
    rows = []
    for i in range(n):
        b, m, u, t = buf[4 * i], buf[4 * i + 1], buf[4 * i + 2], buf[4 * i + 3]
        mu = 1 if t > 0 else -1
        rows.append((b, m, u, mu, abs(t) - 1))
    return rows


def pi_decomposed(x: int, y: int, c: int) -> int:
    """pi(x) = S1 + S2_triv + S2_easy + S2_hard + a - 1 - P2 from O-C."""
    s = leaf_sums(x, y, c)
    return s["S1"] + s["S2_triv"] + s["S2_easy"] + s["S2_hard"] + s["a"] - 1 - s["P2"]
