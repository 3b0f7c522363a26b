"""The benchmark's 4096-query batch (log10 x ~ U(8, 15), seed 0) on the GPU,
checked against the oracle (Meissel-Lehmer, plain phi recursion) on every host
core.  The oracle's cost grows about tenfold per decade (2 s at 10^12, 16 s at
10^13 on one core), so every query up to 10^11 is checked (1783 of
them); the larger ones are checked against single queries by the batch tests
and against Tables 1-2 by the parity tests."""
import concurrent.futures as cf
import multiprocessing
import os

import pytest

import oracle
import paper_1503_01839_gb300 as pc
from paper_1503_01839_gb300 import inputs

pytestmark = pytest.mark.gpu

ORACLE_MAX = 10 ** 11


def test_benchmark_batch_against_oracle_on_host_cores():
    xs = inputs.batch_queries(4096, 0)
    with pc.Context(0, streams=8) as cx:
        got = cx.pi_count_batch(xs)
    sub = [(x, g) for x, g in zip(xs, got) if x <= ORACLE_MAX]
    assert len(sub) > 1500
    oracle.build()
    # spawned workers (a fork of a process holding a CUDA context can hang); the
    # executor raises if a worker dies instead of replacing it
    cores = os.cpu_count() or 1
    with cf.ProcessPoolExecutor(cores, mp_context=multiprocessing.get_context("spawn")) as ex:
        want = list(ex.map(oracle.pi_meissel, [x for x, _ in sub], chunksize=16))
    bad = [(x, g, w) for (x, g), w in zip(sub, want) if g != w]
    assert not bad, bad[:5]
