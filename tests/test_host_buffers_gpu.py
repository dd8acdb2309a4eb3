"""Host result buffers: pinned blocks from the binding's pool, pageable buffers through the C-ABI,
and the server's pinned result pool, all against the oracle.

The binding hands out results that live in pinned host blocks and the batch copies each job's
codes while later jobs sort; these tests check that results stay intact after later calls reuse
the pool, that pageable buffers passed straight to the C-ABI get the same codes, and that served
results of very different sizes stay exact while the server recycles its pinned blocks.
"""
import ctypes

import numpy as np
import pytest

import paper_1403_1313_gb300 as m
from oracle import oracle
from paper_1403_1313_gb300 import fmgen

pytestmark = pytest.mark.gpu

# (n, t, l, d, seed): dense results (bitmap output) and sparse ones (sorted list)
SHAPES = [(6, 300, 9, 3, 71), (8, 200, 10, 3, 72), (5, 120, 8, 1, 73), (12, 400, 11, 2, 74),
          (4, 500, 9, 4, 75), (3, 60, 12, 1, 76)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1403_1313_gb300 import build
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def jobs():
    js = [fmgen.fm_job(n, t, l, d, s) for n, t, l, d, s in SHAPES]
    return js, [oracle.search(j.rows(), j.l, j.d, threads=8)[0] for j in js]


def _plans(js):
    plans = []
    for j in js:
        p = m.motif_plan_create(j.n, j.t, j.l, j.d)
        m.motif_load_seqs(p, j.seqs)
        plans.append(p)
    return plans


def test_results_survive_later_calls(jobs):
    js, refs = jobs
    plans = _plans(js)
    first = m.motif_batch_search(plans)
    singles = [m.motif_search(p) for p in plans]
    for _ in range(3):  # later calls take blocks from the same pools
        m.motif_batch_search(plans)
        for p in plans:
            m.motif_search(p)
    for a, b, r in zip(first, singles, refs):
        assert np.array_equal(a, r)
        assert np.array_equal(b, r)
    for p in plans:
        m.motif_plan_destroy(p)


def test_pageable_buffers_through_the_abi(jobs):
    js, refs = jobs
    plans = _plans(js)
    lib = m._load()
    u64p = ctypes.POINTER(ctypes.c_uint64)
    caps = [max(1, r.size) for r in refs]
    # one pageable array per job (plain numpy, not pinned)
    outs = [np.empty(c, dtype=np.uint64) for c in caps]
    for use_graph in (1, 0):
        k = len(plans)
        counts = (ctypes.c_int64 * k)()
        stats = (ctypes.c_int32 * k)()
        st = lib.motif_batch_search(k, (ctypes.c_void_p * k)(*[p.handle for p in plans]),
                                    (u64p * k)(*[o.ctypes.data_as(u64p) for o in outs]),
                                    (ctypes.c_int64 * k)(*caps), counts, stats, use_graph)
        assert st == m.OK and list(stats) == [m.OK] * k
        for o, c, r in zip(outs, counts, refs):
            assert c == r.size and np.array_equal(o[:c], r)
    for p, r in zip(plans, refs):
        out = np.empty(max(1, r.size), dtype=np.uint64)
        cnt = ctypes.c_int64(0)
        assert lib.motif_search(p, out.ctypes.data_as(u64p), out.size, ctypes.byref(cnt)) == m.OK
        assert cnt.value == r.size and np.array_equal(out[:cnt.value], r)
        m.motif_plan_destroy(p)


def test_server_result_pool_reuse(jobs):
    js, refs = jobs
    try:
        for _ in range(3):  # the same sizes again: pooled blocks come back
            ids = []
            for j in js:
                p = m.motif_plan_create(j.n, j.t, j.l, j.d)
                m.motif_load_seqs(p, j.seqs)
                ids.append(m.motif_submit(p))
                m.motif_plan_destroy(p)
            for jid, r in zip(ids, refs):
                got, _ = m.motif_poll(jid, timeout_ms=120000, capacity=max(1, r.size))
                assert np.array_equal(got, r)
    finally:
        m.motif_server_stop()
