"""Serving (continuous batching) on the GPU: jobs submitted while others run are admitted into
the shared job table; every result equals the oracle's and the result of the same job served
alone (exact equality: the result is an integer set)."""
import ctypes
import random

import numpy as np
import pytest

import paper_1403_1313_gb300 as m
from oracle import oracle
from paper_1403_1313_gb300 import fmgen

pytestmark = pytest.mark.gpu


@pytest.fixture()
def server():
    from paper_1403_1313_gb300 import build
    build.build()
    yield
    try:
        m.motif_server_stop()
    except m.MotifError:
        pass


def _submit(job):
    plan = m.motif_plan_create(job.n, job.t, job.l, job.d)
    m.motif_load_seqs(plan, job.seqs)
    jid = m.motif_submit(plan)
    m.motif_plan_destroy(plan)  # the job keeps its own copy of the windows
    return jid


def _mix(seed, count):
    rng = random.Random(seed)
    jobs = []
    for j in range(count):
        l = rng.randint(7, 10)
        d = rng.randint(1, 3)
        jobs.append(fmgen.fm_job(rng.randint(3, 9), rng.randint(40, 240), l, d, 900 + j,
                                 gc=rng.choice([0.4, 0.5, 0.6])))
    return jobs


@pytest.mark.parametrize("use_graph", [1, 0])
def test_mix_equals_oracle_and_alone(server, use_graph):
    # A tiny tile budget per step forces every job to share many steps with the others.
    m.motif_server_start(max_active=6, step_tiles=64, use_graph=use_graph)
    jobs = _mix(3, 14)
    ids = [_submit(j) for j in jobs]
    mixed = []
    for jid in ids:
        res = m.motif_poll(jid, timeout_ms=120000)
        assert res is not None
        mixed.append(res[0])
    for job, got in zip(jobs, mixed):
        ref, _ = oracle.search(job.rows(), job.l, job.d, threads=8)
        assert np.array_equal(got, ref)
        assert m.motif_encode(job.consensus) in set(got.tolist())
    # The same jobs served alone give identical results.
    for job, got in zip(jobs[:4], mixed[:4]):
        alone = m.motif_poll(_submit(job), timeout_ms=120000)[0]
        assert np.array_equal(alone, got)


def test_poll_states(server):
    m.motif_server_start(max_active=2)
    job = fmgen.fm_job(8, 300, 11, 3, 5)
    jid = _submit(job)
    first = m.motif_poll(jid, timeout_ms=0)          # may still be pending
    res = first or m.motif_poll(jid, timeout_ms=120000)
    assert res is not None
    codes, stats = res
    assert m.motif_encode(job.consensus) in set(codes.tolist())
    assert stats["total_ms"] >= stats["queue_ms"] >= 0
    with pytest.raises(m.MotifError) as e:           # released after a successful poll
        m.motif_poll(jid, timeout_ms=0)
    assert e.value.status == m.ERR_NOTFOUND


def test_empty_jobs_complete_immediately(server):
    m.motif_server_start()
    job = fmgen.fm_job(2, 5, 8, 1, 1)  # t < l: no windows
    codes, _ = m.motif_poll(_submit(job), timeout_ms=10000)
    assert codes.size == 0


def test_served_matches_blocking_search_larger(server):
    m.motif_server_start(max_active=4)
    jobs = [fmgen.fm_job(12, 400, 13, 3, 70 + i) for i in range(3)]
    ids = [_submit(j) for j in jobs]
    for job, jid in zip(jobs, ids):
        got = m.motif_poll(jid, timeout_ms=120000)[0]
        plan = m.motif_plan_create(job.n, job.t, job.l, job.d)
        m.motif_load_seqs(plan, job.seqs)
        assert np.array_equal(got, m.motif_search(plan))
        m.motif_plan_destroy(plan)


@pytest.mark.parametrize("use_graph", [1, 0])
def test_dense_jobs_take_the_bitmap(server, use_graph):
    """Jobs whose codes the plan collects in a bitmap (forced, or chosen for dense results) are
    served through an ordered compaction, mixed with list jobs; one job has 262144 codes, more
    than a served job's first output buffer holds."""
    m.motif_server_start(max_active=8, step_tiles=64, use_graph=use_graph)
    rng = random.Random(17)
    cases = []
    for j in range(8):
        l = rng.randint(6, 10)
        d = rng.randint(2, 4)
        t = rng.randint(30, 120)
        rows = ["".join(rng.choice("ACGT") for _ in range(t)) for _ in range(rng.randint(2, 5))]
        cases.append((rows, l, d, [m.OUTPUT_AUTO, m.OUTPUT_LIST, m.OUTPUT_BITMAP][j % 3]))
    every = ["".join(rng.choice("ACGT") for _ in range(20)) for _ in range(3)]
    cases.append((every, 9, 9, m.OUTPUT_AUTO))  # all 4^9 codes survive: dense, AUTO -> bitmap
    ids = []
    for rows, l, d, output in cases:
        o = m.motif_opts_default()
        o.output = output
        plan = m.motif_plan_create(len(rows), len(rows[0]), l, d, o)
        m.motif_load_seqs(plan, rows)
        ids.append(m.motif_submit(plan))
        m.motif_plan_destroy(plan)
    for jid, (rows, l, d, _) in zip(ids, cases):
        got = m.motif_poll(jid, timeout_ms=120000, capacity=1 << 19)
        assert got is not None
        ref, _ = oracle.search(rows, l, d, threads=8)
        assert np.array_equal(got[0], ref)


def test_other_variant_does_not_hold_back_later_jobs(server):
    """A queued job that needs another step-kernel variant than the running table (l = 3: suffix
    length 3) does not hold back the jobs that arrive after it: they are admitted while the long
    job that fills the table still runs, the passed-over job runs once the table drains, and
    every result equals the oracle's."""
    import time
    # One tile per CTA per step, so the long (17,5) job spans hundreds of steps.
    m.motif_server_start(max_active=8, step_tiles=256)
    long_job = fmgen.single("l17d5")
    t0 = time.perf_counter()
    a = _submit(long_job)
    other = fmgen.fm_job(4, 30, 3, 0, 41)
    b = _submit(other)
    later = [fmgen.fm_job(5, 60, l, 2, 50 + l) for l in (8, 9, 10)]
    ids, t_sub = [], []
    for job in later:
        t_sub.append(1e3 * (time.perf_counter() - t0))
        ids.append(_submit(job))
    res_later = [m.motif_poll(jid, timeout_ms=120000) for jid in ids]
    codes_a, st_a = m.motif_poll(a, timeout_ms=120000)
    codes_b, st_b = m.motif_poll(b, timeout_ms=120000)
    for job, (codes, st), ts in zip(later, res_later, t_sub):
        # admitted (ts + queue_ms after the first submit) before the long job ended
        assert ts + st["queue_ms"] < st_a["total_ms"], (ts, st["queue_ms"], st_a["total_ms"])
        ref, _ = oracle.search(job.rows(), job.l, job.d, threads=8)
        assert np.array_equal(codes, ref)
    ref_b, _ = oracle.search(other.rows(), other.l, other.d)
    assert np.array_equal(codes_b, ref_b)
    assert m.motif_encode(long_job.consensus) in set(codes_a.tolist())
    for c in codes_a.tolist():
        ref, _ = oracle.search(long_job.rows(), long_job.l, long_job.d, lo=c, hi=c + 1)
        assert ref.tolist() == [c]


@pytest.mark.parametrize("use_graph", [1, 0])
def test_submit_seqs_equals_oracle_and_plan_path(server, use_graph):
    """Jobs submitted from host rows without a plan, mixed with plan-submitted jobs in one table,
    give the oracle's result and the same result as through a plan."""
    m.motif_server_start(max_active=6, step_tiles=64, use_graph=use_graph)
    jobs = _mix(11, 10)
    # alternately through a plan and straight from the rows (as strings and as a uint8 array)
    ids = []
    for i, job in enumerate(jobs):
        if i % 3 == 0:
            ids.append(_submit(job))
        elif i % 3 == 1:
            ids.append(m.motif_submit_seqs(job.rows(), job.l, job.d))
        else:
            arr = np.frombuffer("".join(job.rows()).encode(), dtype=np.uint8).reshape(job.n, job.t)
            ids.append(m.motif_submit_seqs(arr, job.l, job.d))
    got = [m.motif_poll(jid, timeout_ms=120000)[0] for jid in ids]
    for job, g in zip(jobs, got):
        ref, _ = oracle.search(job.rows(), job.l, job.d, threads=8)
        assert np.array_equal(g, ref)
    for job, g in zip(jobs[:3], got[:3]):  # each path alone
        assert np.array_equal(m.motif_poll(m.motif_submit_seqs(job.rows(), job.l, job.d),
                                           timeout_ms=120000)[0], g)
        assert np.array_equal(m.motif_poll(_submit(job), timeout_ms=120000)[0], g)


def test_submit_seqs_range_and_errors(server):
    """A sub-range through the options; lower-case rows; the host-side checks."""
    m.motif_server_start(max_active=4)
    job = fmgen.fm_job(6, 200, 9, 2, 77)
    full = m.motif_poll(m.motif_submit_seqs(job.rows(), job.l, job.d), timeout_ms=120000)[0]
    ref, _ = oracle.search(job.rows(), job.l, job.d, threads=8)
    assert np.array_equal(full, ref)
    lo, hi = 1 << 12, 3 << 15
    o = m.motif_opts_default()
    o.range_lo, o.range_hi = lo, hi
    part = m.motif_poll(m.motif_submit_seqs(job.rows(), job.l, job.d, o), timeout_ms=120000)[0]
    assert np.array_equal(part, ref[(ref >= lo) & (ref < hi)])
    lower = [r.lower() for r in job.rows()]
    assert np.array_equal(m.motif_poll(m.motif_submit_seqs(lower, job.l, job.d),
                                       timeout_ms=120000)[0], ref)
    bad = list(job.rows())
    bad[3] = bad[3][:50] + "N" + bad[3][51:]
    with pytest.raises(m.MotifError) as e:
        m.motif_submit_seqs(bad, job.l, job.d)
    assert e.value.status == m.ERR_ALPHABET
    lib = m._load()
    jid = ctypes.c_int64(-1)
    buf = "".join(job.rows()).encode()
    assert lib.motif_submit_seqs(buf, job.t - 1, job.n, job.t, job.l, job.d, None,
                                 ctypes.byref(jid)) == m.ERR_ARG          # stride < t
    assert lib.motif_submit_seqs(None, job.t, job.n, job.t, job.l, job.d, None,
                                 ctypes.byref(jid)) == m.ERR_ARG          # no rows
    assert lib.motif_submit_seqs(buf, job.t, job.n, job.t, 0, job.d, None,
                                 ctypes.byref(jid)) == m.ERR_ARG          # l < 1
    assert jid.value == -1
    # rows shorter than l: no windows, nothing survives
    short = m.motif_poll(m.motif_submit_seqs(["ACGT"] * 3, 6, 1), timeout_ms=120000)[0]
    assert short.size == 0


def test_served_overflow_paths_equal_oracle(server):
    """Results larger than a served job's first output buffer (65,536 codes): a list job grows
    its buffer and starts again, then sorts on the retirement stream (radix sort); a bitmap job
    compacts again into a larger buffer.  Mixed with small jobs in one table."""
    m.motif_server_start(max_active=8, step_tiles=256)
    dense = fmgen.fm_job(3, 100, 10, 4, 321)          # most of the 4^10 codes survive
    ref_dense, _ = oracle.search(dense.rows(), dense.l, dense.d, threads=8)
    assert ref_dense.size > 1 << 16
    as_list = m.motif_opts_default()
    as_list.output = m.OUTPUT_LIST
    as_bitmap = m.motif_opts_default()
    as_bitmap.output = m.OUTPUT_BITMAP
    small = _mix(21, 6)
    ids = [m.motif_submit_seqs(dense.rows(), dense.l, dense.d, as_list)]
    ids += [m.motif_submit_seqs(j.rows(), j.l, j.d) for j in small[:3]]
    ids.append(m.motif_submit_seqs(dense.rows(), dense.l, dense.d, as_bitmap))
    ids += [m.motif_submit_seqs(j.rows(), j.l, j.d) for j in small[3:]]
    got = [m.motif_poll(jid, timeout_ms=120000, capacity=1 << 21)[0] for jid in ids]
    assert np.array_equal(got[0], ref_dense)
    assert np.array_equal(got[4], ref_dense)
    for job, g in zip(small, got[1:4] + got[5:]):
        ref, _ = oracle.search(job.rows(), job.l, job.d, threads=8)
        assert np.array_equal(g, ref)
