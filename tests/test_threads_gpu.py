"""Host threads: plans used from several threads at once, concurrent submit/poll, and
concurrent batches, against the oracle.

A plan is not thread-safe, but different plans are independent; motif_submit and motif_poll are
thread-safe; batches serialise on the library's per-device batch context.  The binding's ctypes
calls release the interpreter lock, so these calls really run side by side in the library (its
shared Hamming-ball tables, kernel-attribute table, graph caches and launch counter).
"""
import random
import threading

import numpy as np
import pytest

import paper_1403_1313_gb300 as m
from oracle import oracle
from paper_1403_1313_gb300 import fmgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1403_1313_gb300 import build
    build.build()
    oracle.build()


def _jobs(seed, count):
    rng = random.Random(seed)
    out = []
    for k in range(count):
        l = rng.randint(7, 11)
        d = rng.randint(1, 3)
        job = fmgen.fm_job(rng.randint(3, 9), rng.randint(40, 220), l, d, seed * 100 + k)
        out.append((job, oracle.search(job.rows(), l, d, threads=4)[0]))
    return out


def _run_threads(targets):
    errors = []

    def wrap(f):
        try:
            f()
        except BaseException as e:  # reported below, in the test's thread
            errors.append(e)

    ts = [threading.Thread(target=wrap, args=(f,)) for f in targets]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    assert not any(t.is_alive() for t in ts), "a thread did not finish"
    if errors:
        raise errors[0]


def test_own_plans_in_parallel_threads():
    work = [_jobs(900 + w, 4) for w in range(6)]

    def worker(jobs):
        def run():
            for _ in range(3):
                for job, ref in jobs:
                    plan = m.motif_plan_create(job.n, job.t, job.l, job.d)
                    m.motif_load_seqs(plan, job.seqs)
                    got = m.motif_search(plan)
                    m.motif_plan_destroy(plan)
                    assert np.array_equal(got, ref)
        return run

    _run_threads([worker(j) for j in work])


def test_concurrent_submit_and_poll():
    work = [_jobs(950 + w, 6) for w in range(4)]

    def worker(jobs):
        def run():
            ids = []
            for job, _ in jobs:
                plan = m.motif_plan_create(job.n, job.t, job.l, job.d)
                m.motif_load_seqs(plan, job.seqs)
                ids.append(m.motif_submit(plan))
                m.motif_plan_destroy(plan)
            for jid, (_, ref) in zip(ids, jobs):
                got, _ = m.motif_poll(jid, timeout_ms=120000, capacity=max(1, ref.size))
                assert np.array_equal(got, ref)
        return run

    try:
        _run_threads([worker(j) for j in work])
    finally:
        m.motif_server_stop()


def test_concurrent_row_submissions_and_polls():
    """motif_submit_seqs from several threads at once (the server's pinned staging pool and
    submit stream are shared), each thread polling its own jobs, some with a capacity that is
    too small at first; mixed with plan submissions from another thread."""
    work = [_jobs(1010 + w, 8) for w in range(5)]

    def rows_worker(jobs):
        def run():
            for _ in range(2):
                ids = [m.motif_submit_seqs(job.seqs, job.l, job.d) for job, _ in jobs]
                for k, (jid, (_, ref)) in enumerate(zip(ids, jobs)):
                    cap = 1 if k % 2 else max(1, ref.size)  # odd jobs: grow on ERR_CAPACITY
                    got, _ = m.motif_poll(jid, timeout_ms=120000, capacity=cap)
                    assert np.array_equal(got, ref)
        return run

    def plan_worker(jobs):
        def run():
            ids = []
            for job, _ in jobs:
                plan = m.motif_plan_create(job.n, job.t, job.l, job.d)
                m.motif_load_seqs(plan, job.seqs)
                ids.append(m.motif_submit(plan))
                m.motif_plan_destroy(plan)
            for jid, (_, ref) in zip(ids, jobs):
                assert np.array_equal(m.motif_poll(jid, timeout_ms=120000)[0], ref)
        return run

    try:
        m.motif_server_start(max_active=16, step_tiles=512)
        _run_threads([rows_worker(j) for j in work[:4]] + [plan_worker(work[4])])
    finally:
        m.motif_server_stop()


def test_concurrent_batches():
    work = [_jobs(980 + w, 8) for w in range(3)]

    def worker(jobs):
        def run():
            plans = []
            for job, _ in jobs:
                plan = m.motif_plan_create(job.n, job.t, job.l, job.d)
                m.motif_load_seqs(plan, job.seqs)
                plans.append(plan)
            for use_graph in (True, False, True):
                got = m.motif_batch_search(plans, use_graph=use_graph)
                for g, (_, ref) in zip(got, jobs):
                    assert np.array_equal(g, ref)
            for p in plans:
                m.motif_plan_destroy(p)
        return run

    _run_threads([worker(j) for j in work])
