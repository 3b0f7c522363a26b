"""GPU tests of the batched call and the server: every result equals the same
query run alone (pc_pi_count / pc_phi) and, where the oracle is fast, the
oracle; the server's admission respects slots and its memory budget."""
import time

import pytest

import oracle as o
import paper_1503_01839_gb300 as pc
from paper_1503_01839_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def alone():
    with pc.Context(0) as c:
        yield c


def test_batch_mixed_sizes_match_alone_and_oracle(alone):
    xs = inputs.log_uniform_x(300, 3.0, 13.0, seed=11)
    xs += [0, 1, 2, 3, 4, 5, 100, (1 << 20) - 1, 1 << 20, 10 ** 10, 2 ** 40, 10 ** 13]
    with pc.Context(0, streams=8) as cx:
        got = cx.pi_count_batch(xs)
        st = cx.stats()
    assert got == [alone.pi_count(x) for x in xs]
    for x, g in zip(xs, got):
        if x <= 10 ** 7:
            assert g == o.pi_sieve(x), x
    assert got[xs.index(10 ** 10)] == 455052511
    assert st["kernel_launches"] > 0


def test_batch_graph_equals_direct_launches(alone):
    # the default runs the schedule's device work as one captured CUDA graph; the same
    # kernels launched one by one, and every query alone, give the same results
    xs = inputs.log_uniform_x(400, 7.0, 15.0, seed=31) + [1 << 20, 10 ** 10, 10 ** 15 - 1]
    with pc.Context(0) as cg, pc.Context(0, batch_launch=1) as cd:
        g1 = cg.pi_count_batch(xs)
        sg = cg.stats()
        g2 = cg.pi_count_batch(xs[::-1])   # a second graph on the same context
        d = cd.pi_count_batch(xs)
        sd = cd.stats()
    assert g1 == d == g2[::-1]
    assert g1 == [alone.pi_count(x) for x in xs]
    assert sg["graph_launches"] == 1 and 10 <= sg["graph_nodes"] <= sg["kernel_launches"] + 8
    assert sd["graph_launches"] == 0 and sd["graph_nodes"] == 0


def test_autotune_batch_keeps_results(alone):
    # the batch geometry tuner (segment size, resident CTAs) changes no result
    xs = inputs.log_uniform_x(300, 8.0, 14.0, seed=32)
    with pc.Context(0) as cx:
        assert cx.tuned_batch() == (16384, 0, 0)
        cx.autotune(min(xs), max(xs))
        before = cx.pi_count_batch(xs)
        cx.autotune_batch(xs, reps=1)
        seg, ctas, builtin = cx.tuned_batch()
        assert (seg, ctas) in [(16384, 0), (16384, 8), (32768, 0)] and builtin in (0, 1)
        after = cx.pi_count_batch(xs[::-1])[::-1]
    assert before == after == [alone.pi_count(x) for x in xs]
    with pc.Context(0, seg_bytes=65536) as cf:   # a fixed segment size stays fixed
        cf.autotune_batch(xs[:50], reps=1)
        assert cf.tuned_batch()[0] == 65536
        assert cf.pi_count_batch(xs[:50]) == before[:50]


def test_batch_device_arrays_on_stream(alone):
    torch = pytest.importorskip("torch")
    xs = inputs.log_uniform_x(64, 6.0, 12.0, seed=12)
    s = torch.cuda.Stream()
    dx = torch.tensor(xs, dtype=torch.int64, device="cuda")
    dout = torch.zeros(len(xs), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    with pc.Context(0, streams=4) as cx:
        cx.pi_count_batch((dx.data_ptr(), dout.data_ptr(), len(xs)), stream_handle=s.cuda_stream)
    s.synchronize()
    assert dout.cpu().tolist() == [alone.pi_count(x) for x in xs]


def test_batch_slot_counts_agree():
    xs = inputs.log_uniform_x(120, 8.0, 13.0, seed=13)
    res = []
    for streams in (1, 3, 16):
        with pc.Context(0, streams=streams) as cx:
            res.append(cx.pi_count_batch(xs))
    assert res[0] == res[1] == res[2]


def test_batch_reuses_context_and_grows_tables():
    with pc.Context(0, streams=4) as cx:
        small = inputs.log_uniform_x(40, 6.0, 9.0, seed=14)
        big = inputs.log_uniform_x(40, 12.0, 14.0, seed=15)
        a = cx.pi_count_batch(small)
        b = cx.pi_count_batch(big)
        a2 = cx.pi_count_batch(small)
        assert a == a2
        assert b == [cx.pi_count(x) for x in big]


def test_batch_errors():
    with pc.Context(0) as cx:
        assert cx.pi_count_batch([]) == []
        with pytest.raises(pc.PicountError) as e:
            cx.pi_count_batch([10, 1 << 63])
        assert e.value.code == -2
        # the context stays usable
        assert cx.pi_count_batch([10 ** 9]) == [50847534]


def _drain(srv, n, timeout_s=600.0):
    out = []
    t0 = time.time()
    while len(out) < n:
        out += srv.poll(256, timeout_ms=200)
        assert time.time() - t0 < timeout_s
    return out


def test_server_results_equal_alone(alone):
    trace = inputs.served_trace(160, rate_per_s=4000.0, seed=21, lo_exp=6.0, hi_exp=13.0, a_hi=3000)
    with pc.Context(0, streams=6) as cx:
        with pc.Server(cx, x_max=10 ** 13, a_max=3000) as srv:
            for i, r in enumerate(trace):
                srv.submit(pc.PC_QUERY_PHI if r["kind"] == "phi" else pc.PC_QUERY_PI, r["x"], r["a"], tag=i)
            res = _drain(srv, len(trace))
            st = srv.stats()
    assert st["completed"] == len(trace) and st["failed"] == 0
    assert st["max_running"] >= 2   # requests overlapped on the device
    by_tag = {r["tag"]: r for r in res}
    for i, r in enumerate(trace):
        g = by_tag[i]
        assert g["status"] == 0
        want = alone.phi(r["x"], r["a"]) if r["kind"] == "phi" else alone.pi_count(r["x"])
        assert g["value"] == want, (r, g)
        assert g["t_submit_ms"] <= g["t_start_ms"] <= g["t_done_ms"]
    # a few against the oracle directly
    for i, r in enumerate(trace[:40]):
        if r["x"] <= 10 ** 8:
            want = o.phi_brute(r["x"], r["a"]) if r["kind"] == "phi" else o.pi_sieve(r["x"])
            assert by_tag[i]["value"] == want


def test_server_results_equal_alone_up_to_1e16(alone):
    # the served workload's mix (80 % pi(x), 20 % phi(x, a)) with x up to 10^16
    trace = inputs.served_trace(80, rate_per_s=4000.0, seed=23, lo_exp=9.0, hi_exp=16.0, a_hi=5000)
    with pc.Context(0, streams=8) as cx:
        with pc.Server(cx, x_max=10 ** 16, a_max=5000) as srv:
            for i, r in enumerate(trace):
                srv.submit(pc.PC_QUERY_PHI if r["kind"] == "phi" else pc.PC_QUERY_PI, r["x"], r["a"], tag=i)
            res = _drain(srv, len(trace))
            st = srv.stats()
    assert st["completed"] == len(trace) and st["failed"] == 0
    by_tag = {r["tag"]: r for r in res}
    for i, r in enumerate(trace):
        want = alone.phi(r["x"], r["a"]) if r["kind"] == "phi" else alone.pi_count(r["x"])
        assert by_tag[i]["status"] == 0 and by_tag[i]["value"] == want, (r, by_tag[i])


def test_batch_across_the_schedule_boundary(alone, pi_pow10):
    # queries on both sides of the batched schedule's limit (1e16) and of the table
    # cut-over (2^20), in one call; every result equal to the query alone and to Table 1
    xs = inputs.log_uniform_x(120, 6.0, 16.6, seed=29)
    xs += [10 ** n for n in range(6, 17)] + [(1 << 20) - 1, 1 << 20, 10 ** 16 - 1, 10 ** 16 + 1]
    with pc.Context(0) as cx:
        got = cx.pi_count_batch(xs)
    assert got == [alone.pi_count(x) for x in xs]
    for n in range(6, 17):
        assert got[xs.index(10 ** n)] == pi_pow10[n], n


def test_server_memory_budget_admits_one_at_a_time():
    xs = [10 ** 12 + 7919 * k for k in range(12)]
    with pc.Context(0, streams=8) as cx:
        with pc.Server(cx, x_max=2 * 10 ** 12, a_max=0, mem_budget=1 << 40) as probe:
            foot = max(probe.footprint(pc.PC_QUERY_PI, x) for x in xs)
        with pc.Server(cx, x_max=2 * 10 ** 12, a_max=0, mem_budget=foot + foot // 2) as srv:
            for k, x in enumerate(xs):
                srv.submit(pc.PC_QUERY_PI, x, 0, tag=k)
            res = _drain(srv, len(xs))
            st = srv.stats()
            with pytest.raises(pc.PicountError) as e2:
                srv.submit(pc.PC_QUERY_PI, 10 ** 13, 0, tag=100)   # beyond x_max
            assert e2.value.code == -1
        # a request whose footprint alone exceeds the budget is refused at submission
        with pc.Server(cx, x_max=2 * 10 ** 12, a_max=0, mem_budget=foot // 2) as tiny:
            with pytest.raises(pc.PicountError) as e3:
                tiny.submit(pc.PC_QUERY_PI, xs[0], 0, tag=0)
            assert e3.value.code == -3
    assert st["max_running"] == 1
    assert st["max_bytes"] <= foot + foot // 2
    assert sorted(r["tag"] for r in res) == list(range(len(xs)))
    # FIFO admission with one request at a time: starts follow submission order
    starts = [r["t_start_ms"] for r in sorted(res, key=lambda r: r["tag"])]
    assert starts == sorted(starts)
    with pc.Context(0) as c1:
        assert [r["value"] for r in sorted(res, key=lambda r: r["tag"])] == [c1.pi_count(x) for x in xs]


def test_autotune_keeps_results(alone):
    with pc.Context(0, streams=4) as cx:
        before = {x: cx.tuned(x) for x in (10 ** 9, 3 * 10 ** 10, 10 ** 12)}
        cx.autotune(10 ** 9, 2 * 10 ** 12, reps=1)
        after = {x: cx.tuned(x) for x in before}
        for x, (al, sb) in after.items():
            assert al >= 1 and sb in (16384, 32768, 65536)
            assert cx.tuned_ctas(x) in (0, 2, 4, 6)   # resident CTAs per SM, tuned too
        xs = inputs.log_uniform_x(60, 9.0, 12.3, seed=31) + [10 ** 10, 10 ** 12]
        got = cx.pi_count_batch(xs)
        assert got == [alone.pi_count(x) for x in xs]
        assert cx.pi_count(10 ** 10) == 455052511 and cx.pi_count(10 ** 12) == 37607912018
    # a fixed alpha stays fixed
    with pc.Context(0, alpha=3) as cx:
        cx.autotune(10 ** 9, 10 ** 10, reps=1)
        assert cx.tuned(5 * 10 ** 9)[0] == 3


def test_server_small_first_policy(alone):
    xs = [10 ** 13, 10 ** 9 + 7, 10 ** 12, 10 ** 10, 3 * 10 ** 11, 10 ** 9, 2 * 10 ** 12, 5 * 10 ** 10]
    with pc.Context(0, streams=1) as cx:
        with pc.Server(cx, x_max=10 ** 13, policy=pc.PC_SERVE_SMALL_FIRST) as srv:
            for k, x in enumerate(xs):
                srv.submit(pc.PC_QUERY_PI, x, 0, tag=k)
            res = _drain(srv, len(xs))
            st = srv.stats()
    assert st["max_running"] == 1
    order = sorted(res, key=lambda r: r["t_start_ms"])
    later = [r["x"] for r in order[1:]]          # all queued while the first one ran
    assert later == sorted(later)
    for r in res:
        assert r["value"] == alone.pi_count(r["x"])


def test_concurrent_contexts_with_different_segments(alone):
    # Per-kernel launch limits are process-wide: two host threads running
    # queries with different segment sizes at once must not disturb each other.
    import threading
    x, y = 10 ** 14, 8 * 46415
    want = alone.s2_hard(x, y, 5)
    errors, results = [], []

    def run(seg):
        try:
            with pc.Context(0, seg_bytes=seg) as cx:
                for _ in range(6):
                    results.append(cx.s2_hard(x, y, 5))
                    results.append(cx.p2(x, y))
        except Exception as e:   # collected and re-raised below
            errors.append(e)

    th = [threading.Thread(target=run, args=(seg,)) for seg in (16384, 65536, 131072)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    p2 = alone.p2(x, y)
    assert all(r in (want, p2) for r in results) and results.count(want) == 18


def test_batch_after_autotune_over_many_decades(alone):
    # decades tuned to different segment sizes run concurrently in one batch
    xs = inputs.log_uniform_x(200, 8.0, 14.0, seed=41)
    with pc.Context(0, streams=8) as cx:
        cx.autotune(min(xs), max(xs), reps=1)
        got = cx.pi_count_batch(xs)
    assert got == [alone.pi_count(x) for x in xs]


def test_batch_small_queries_from_the_table(alone, pi_pow2):
    # at least 64 queries < 2^32 are answered by table lookups; mixed with larger ones
    xs = inputs.log_uniform_x(120, 8.0, 9.6, seed=51) + [1 << 31, (1 << 32) - 1, 1 << 32, 10 ** 12]
    with pc.Context(0, streams=4) as cx:
        got = cx.pi_count_batch(xs)
    assert got == [alone.pi_count(x) for x in xs]
    assert got[-4] == pi_pow2[31]          # Table 2, answered by the lookup
    assert got[-2] == pi_pow2[32]          # Table 2, just beyond the lookup range
