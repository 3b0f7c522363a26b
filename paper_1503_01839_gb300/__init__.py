"""Python binding of the picount C ABI (include/picount.h).

Argument marshalling only: every step of every computation runs in the CUDA
library ``libpicount.so`` built for sm_103a.  There is no CPU fallback: if
the library is missing or cannot be loaded, importing ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpicount.so")

PC_OK = 0
ERRORS = {-1: "PC_EINVAL", -2: "PC_ERANGE", -3: "PC_ENOMEM", -4: "PC_ECUDA", -5: "PC_ETIMEOUT", -6: "PC_EOVERFLOW"}

# every symbol declared in include/picount.h
SYMBOLS = ["pc_create", "pc_destroy", "pc_set_stream", "pc_pi_count", "pc_phi", "pc_s2_hard", "pc_p2",
           "pc_leaf_sums", "pc_pi_count_batch", "pc_last_stats", "pc_strerror", "pc_last_error", "pc_version",
           "pc_p2_noalloc", "pc_server_create", "pc_server_submit", "pc_server_poll", "pc_server_get_stats",
           "pc_server_footprint", "pc_server_destroy", "pc_autotune", "pc_tuned", "pc_s2_hard_shard",
           "pc_phi_starts", "pc_tuned_ctas", "pc_autotune_batch", "pc_tuned_batch"]

PC_QUERY_PI = 0
PC_QUERY_PHI = 1
PC_SERVE_FIFO = 0
PC_SERVE_SMALL_FIRST = 1


class PcI128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int64), ("hi", ctypes.c_int64)]

    def value(self) -> int:
        return (self.hi << 64) + (self.lo & ((1 << 64) - 1))


class PcParams(ctypes.Structure):
    _fields_ = [("seg_bytes", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32), ("threads", ctypes.c_uint32),
                ("alpha", ctypes.c_uint32), ("c", ctypes.c_uint32), ("warp_bytes", ctypes.c_uint32),
                ("streams", ctypes.c_uint32), ("pi_gather", ctypes.c_uint32), ("m_source", ctypes.c_uint32),
                ("batch_launch", ctypes.c_uint32), ("p2_bucket", ctypes.c_uint32)]


class PcStats(ctypes.Structure):
    _fields_ = [("x", ctypes.c_uint64), ("y", ctypes.c_uint64), ("z", ctypes.c_uint64), ("a", ctypes.c_uint64),
                ("B", ctypes.c_uint64), ("c", ctypes.c_uint32), ("seg_bytes", ctypes.c_uint32),
                ("segments", ctypes.c_uint64), ("steps", ctypes.c_uint64), ("hard_leaves", ctypes.c_uint64),
                ("clears", ctypes.c_uint64), ("work_items", ctypes.c_uint64), ("item_steps", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64),
                ("ms_tables", ctypes.c_double), ("ms_s1", ctypes.c_double), ("ms_trivial", ctypes.c_double),
                ("ms_easy", ctypes.c_double), ("ms_hard", ctypes.c_double), ("ms_p2", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_hard_sieve", ctypes.c_double),
                ("warp_steps", ctypes.c_uint64), ("leaf_warp_steps", ctypes.c_uint64),
                ("ms_easy_kernel", ctypes.c_double), ("ms_p2_kernel", ctypes.c_double),
                ("easy_leaves", ctypes.c_uint64), ("easy_runs", ctypes.c_uint64),
                ("easy_run_leaves", ctypes.c_uint64), ("p2_clears", ctypes.c_uint64),
                ("presieve_steps", ctypes.c_uint64), ("graph_launches", ctypes.c_uint64),
                ("graph_nodes", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class PcResult(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("x", ctypes.c_uint64), ("a", ctypes.c_uint64), ("value", ctypes.c_uint64),
                ("kind", ctypes.c_int32), ("status", ctypes.c_int32), ("t_submit_ms", ctypes.c_double),
                ("t_start_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class PcServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("max_running", ctypes.c_uint64), ("max_bytes", ctypes.c_uint64), ("mem_budget", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def lib():
    """Load libpicount.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libpicount.so not built: run paper_1503_01839_gb300/build.py "
                                   "(or __graft_entry__.build()) first")
            L = ctypes.CDLL(LIB_PATH)
            u64, u32, p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
            L.pc_create.argtypes = [ctypes.POINTER(p), ctypes.c_int, ctypes.POINTER(PcParams)]
            L.pc_destroy.argtypes = [p]
            L.pc_destroy.restype = None
            L.pc_set_stream.argtypes = [p, p]
            L.pc_pi_count.argtypes = [p, u64, u32, ctypes.POINTER(u64)]
            L.pc_phi.argtypes = [p, u64, u64, ctypes.POINTER(u64)]
            L.pc_s2_hard.argtypes = [p, u64, u64, u32, ctypes.POINTER(PcI128)]
            L.pc_p2.argtypes = [p, u64, u64, ctypes.POINTER(u64)]
            L.pc_leaf_sums.argtypes = [p, u64, u64, u32, u64, ctypes.POINTER(PcI128)]
            L.pc_pi_count_batch.argtypes = [p, p, ctypes.c_size_t, p, p]
            L.pc_last_stats.argtypes = [p, ctypes.POINTER(PcStats)]
            L.pc_strerror.argtypes = [ctypes.c_int]
            L.pc_strerror.restype = ctypes.c_char_p
            L.pc_last_error.argtypes = [p]
            L.pc_last_error.restype = ctypes.c_char_p
            L.pc_version.restype = ctypes.c_char_p
            L.pc_p2_noalloc.argtypes = [u64, u64, p, u64, p, p]
            L.pc_p2_noalloc.restype = ctypes.c_int
            L.pc_server_create.argtypes = [p, u64, u64, u64, u32, ctypes.POINTER(p)]
            L.pc_server_submit.argtypes = [p, ctypes.c_int, u64, u64, u64]
            L.pc_server_poll.argtypes = [p, ctypes.POINTER(PcResult), ctypes.c_size_t, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_size_t)]
            L.pc_server_get_stats.argtypes = [p, ctypes.POINTER(PcServerStats)]
            L.pc_server_footprint.argtypes = [p, ctypes.c_int, u64, u64]
            L.pc_server_footprint.restype = u64
            L.pc_autotune.argtypes = [p, u64, u64, u32]
            L.pc_s2_hard_shard.argtypes = [p, u64, u64, u32, u32, u32, ctypes.POINTER(PcI128)]
            L.pc_phi_starts.argtypes = [p, u64, u32, u64, ctypes.POINTER(u64)]
            L.pc_tuned.argtypes = [p, u64, ctypes.POINTER(u32), ctypes.POINTER(u32)]
            L.pc_tuned_ctas.argtypes = [p, u64, ctypes.POINTER(u32)]
            L.pc_autotune_batch.argtypes = [p, p, ctypes.c_size_t, u32]
            L.pc_tuned_batch.argtypes = [p, ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]
            L.pc_server_destroy.argtypes = [p]
            L.pc_server_destroy.restype = None
            for name in ("pc_create", "pc_set_stream", "pc_pi_count", "pc_phi", "pc_s2_hard", "pc_p2",
                         "pc_leaf_sums", "pc_pi_count_batch", "pc_last_stats", "pc_server_create",
                         "pc_server_submit", "pc_server_poll", "pc_server_get_stats", "pc_autotune", "pc_tuned",
                         "pc_s2_hard_shard", "pc_phi_starts", "pc_tuned_ctas", "pc_autotune_batch",
                         "pc_tuned_batch"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


class PicountError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class Context:
    """One library context (device tables + scratch) on one CUDA device."""

    def __init__(self, device: int = 0, seg_bytes: int = 0, ctas_per_sm: int = 0, threads: int = 0,
                 alpha: int = 0, c: int = 0, warp_bytes: int = 0, streams: int = 0, pi_gather: int = 0,
                 m_source: int = 0, batch_launch: int = 0, p2_bucket: int = 0):
        self._L = lib()
        prm = PcParams(seg_bytes, ctas_per_sm, threads, alpha, c, warp_bytes, streams, pi_gather, m_source,
                       batch_launch, p2_bucket)
        h = ctypes.c_void_p()
        rc = self._L.pc_create(ctypes.byref(h), device, ctypes.byref(prm))
        if rc != PC_OK:
            raise PicountError(rc, "pc_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.pc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc: int):
        if rc != PC_OK:
            raise PicountError(rc, self._L.pc_last_error(self._h).decode())

    def set_stream(self, stream_handle: int | None):
        self._check(self._L.pc_set_stream(self._h, ctypes.c_void_p(stream_handle or 0)))

    def pi_count(self, x: int, alpha: int = 0) -> int:
        out = ctypes.c_uint64()
        self._check(self._L.pc_pi_count(self._h, x, alpha, ctypes.byref(out)))
        return out.value

    def phi(self, x: int, a: int) -> int:
        out = ctypes.c_uint64()
        self._check(self._L.pc_phi(self._h, x, a, ctypes.byref(out)))
        return out.value

    def s2_hard(self, x: int, y: int, c: int) -> int:
        out = PcI128()
        self._check(self._L.pc_s2_hard(self._h, x, y, c, ctypes.byref(out)))
        return out.value()

    def s2_hard_shard(self, x: int, y: int, c: int, k: int, n: int) -> int:
        out = PcI128()
        self._check(self._L.pc_s2_hard_shard(self._h, x, y, c, k, n, ctypes.byref(out)))
        return out.value()

    def phi_starts(self, m: int, c: int, b_max: int) -> list:
        out = (ctypes.c_uint64 * (b_max - c + 1))()
        self._check(self._L.pc_phi_starts(self._h, m, c, b_max, out))
        return list(out)

    def p2(self, x: int, y: int) -> int:
        out = ctypes.c_uint64()
        self._check(self._L.pc_p2(self._h, x, y, ctypes.byref(out)))
        return out.value

    def leaf_sums(self, x: int, y: int, c: int, a: int = 0) -> dict:
        out = (PcI128 * 5)()
        self._check(self._L.pc_leaf_sums(self._h, x, y, c, a, out))
        v = [o.value() for o in out]
        return {"S1": v[0], "S2_triv": v[1], "S2_easy": v[2], "S2_hard": v[3], "P2": v[4]}

    def pi_count_batch(self, xs, out=None, stream_handle: int | None = None):
        """xs: sequence of ints (host), or a device pointer (int) with n given
        by len(out) when stream_handle is set."""
        if stream_handle is None:
            n = len(xs)
            arr = (ctypes.c_uint64 * n)(*xs)
            res = (ctypes.c_uint64 * n)()
            self._check(self._L.pc_pi_count_batch(self._h, arr, n, res, None))
            return list(res)
        xs_ptr, out_ptr, n = xs
        self._check(self._L.pc_pi_count_batch(self._h, ctypes.c_void_p(xs_ptr), n, ctypes.c_void_p(out_ptr),
                                              ctypes.c_void_p(stream_handle)))
        return None

    def autotune(self, x_lo: int, x_hi: int, reps: int = 0) -> None:
        self._check(self._L.pc_autotune(self._h, x_lo, x_hi, reps))

    def tuned(self, x: int) -> tuple:
        a, s = ctypes.c_uint32(), ctypes.c_uint32()
        self._check(self._L.pc_tuned(self._h, x, ctypes.byref(a), ctypes.byref(s)))
        return a.value, s.value

    def autotune_batch(self, xs, reps: int = 0) -> None:
        n = len(xs)
        arr = (ctypes.c_uint64 * n)(*xs)
        self._check(self._L.pc_autotune_batch(self._h, arr, n, reps))

    def tuned_batch(self) -> tuple:
        """(segment bytes, resident CTAs per SM, 1 if the built-in alphas) of the batch."""
        s, c, a = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        self._check(self._L.pc_tuned_batch(self._h, ctypes.byref(s), ctypes.byref(c), ctypes.byref(a)))
        return s.value, c.value, a.value

    def tuned_ctas(self, x: int) -> int:
        v = ctypes.c_uint32()
        self._check(self._L.pc_tuned_ctas(self._h, x, ctypes.byref(v)))
        return v.value

    def stats(self) -> dict:
        s = PcStats()
        self._check(self._L.pc_last_stats(self._h, ctypes.byref(s)))
        return s.as_dict()


class Server:
    """Continuous-batching server over a Context (pc_server_* of picount.h):
    submit() queues a pi(x) or phi(x, a) request and returns at once; poll()
    returns finished results as dicts.  The context must not be used for
    anything else while the server lives."""

    def __init__(self, ctx: Context, x_max: int, a_max: int = 0, mem_budget: int = 0, policy: int = PC_SERVE_FIFO):
        self._L = lib()
        self._ctx = ctx
        h = ctypes.c_void_p()
        rc = self._L.pc_server_create(ctx._h, x_max, a_max, mem_budget, policy, ctypes.byref(h))
        if rc != PC_OK:
            raise PicountError(rc, self._L.pc_last_error(ctx._h).decode())
        self._h = h

    def submit(self, kind: int, x: int, a: int = 0, tag: int = 0) -> None:
        rc = self._L.pc_server_submit(self._h, kind, x, a, tag)
        if rc != PC_OK:
            raise PicountError(rc, "pc_server_submit rejected the request")

    def poll(self, max_results: int = 256, timeout_ms: int = 0) -> list:
        buf = (PcResult * max_results)()
        n = ctypes.c_size_t()
        rc = self._L.pc_server_poll(self._h, buf, max_results, timeout_ms, ctypes.byref(n))
        if rc != PC_OK:
            raise PicountError(rc, "pc_server_poll failed")
        return [buf[i].as_dict() for i in range(n.value)]

    def footprint(self, kind: int, x: int, a: int = 0) -> int:
        return self._L.pc_server_footprint(self._h, kind, x, a)

    def stats(self) -> dict:
        s = PcServerStats()
        rc = self._L.pc_server_get_stats(self._h, ctypes.byref(s))
        if rc != PC_OK:
            raise PicountError(rc, "pc_server_get_stats failed")
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            self._L.pc_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def p2_noalloc(x: int, y: int, primes_ptr: int, n_primes: int, out_ptr: int, stream_handle: int = 0) -> None:
    """P2(x, pi(y)) into the device uint64 at out_ptr, with no device
    allocation: primes_ptr is a caller-owned device array of the primes
    up to isqrt(x) (uint32, ascending).  Enqueued on stream_handle."""
    rc = lib().pc_p2_noalloc(x, y, ctypes.c_void_p(primes_ptr), n_primes, ctypes.c_void_p(out_ptr),
                             ctypes.c_void_p(stream_handle or 0))
    if rc != PC_OK:
        raise PicountError(rc, "pc_p2_noalloc rejected its arguments")


def version() -> str:
    return lib().pc_version().decode()
