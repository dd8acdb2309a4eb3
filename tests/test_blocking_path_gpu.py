"""The blocking ABI path: staged host loads and one-wait searches, against the oracle.

A small host load is validated on the host while it is copied into pinned staging, so the call
returns before the device has read it; a larger one is checked on the device.  A blocking
search reads its count and first codes back with one wait, sorts a large result once on the
host side when the plan has no multi-CTA sort scratch yet, and shares a cached sort graph with
the device path.  These tests change the caller's buffer right after a load, put bad
characters on both sides of the host-check size, alternate blocking and device searches on
one plan, and cross the one-wait and one-CTA-sort sizes.
"""
import ctypes
import random

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


def test_buffer_reuse_right_after_load():
    a = fmgen.fm_job(6, 150, 9, 2, 301)
    b = fmgen.fm_job(6, 150, 9, 2, 302)
    ref_a = oracle.search(a.rows(), 9, 2)[0]
    ref_b = oracle.search(b.rows(), 9, 2)[0]
    plan = m.motif_plan_create(6, 150, 9, 2)
    buf = np.ascontiguousarray(a.seqs).copy()
    lib = m._load()
    for _ in range(3):
        buf[:] = a.seqs
        assert lib.motif_load_seqs(plan, buf.ctypes.data_as(ctypes.c_char_p), 150) == m.OK
        buf[:] = b.seqs  # the caller's buffer changes as soon as the load returns
        assert np.array_equal(m.motif_search(plan), ref_a)
        assert lib.motif_load_seqs(plan, buf.ctypes.data_as(ctypes.c_char_p), 150) == m.OK
        buf[:] = a.seqs
        assert np.array_equal(m.motif_search(plan), ref_b)
    m.motif_plan_destroy(plan)


@pytest.mark.parametrize("n,t", [(4, 100), (8, 8192), (20, 8000)])  # 400 B, 64 KiB, 160 KB
@pytest.mark.parametrize("where", ["first", "last", "middle"])
def test_bad_characters_on_both_load_paths(n, t, where):
    rng = random.Random(n * t)
    rows = ["".join(rng.choice("ACGT") for _ in range(t)) for _ in range(n)]
    r, c = {"first": (0, 0), "last": (n - 1, t - 1), "middle": (n // 2, t // 2)}[where]
    rows[r] = rows[r][:c] + rng.choice("NXn-") + rows[r][c + 1:]
    plan = m.motif_plan_create(n, t, 8, 1)
    with pytest.raises(m.MotifError) as e:
        m.motif_load_seqs(plan, rows)
    assert e.value.status == m.ERR_ALPHABET
    with pytest.raises(m.MotifError) as e:  # the plan holds no sequences
        m.motif_search(plan)
    assert e.value.status == m.ERR_STATE
    rows[r] = rows[r][:c] + "A" + rows[r][c + 1:]  # a clean load afterwards works
    m.motif_load_seqs(plan, rows)
    m.motif_search(plan)
    m.motif_plan_destroy(plan)


def test_alternating_blocking_and_device_searches():
    torch = pytest.importorskip("torch")
    # list output with results of a few codes, a few hundred, and tens of thousands
    cases = [(fmgen.fm_job(8, 200, 10, 2, 303), m.OUTPUT_AUTO),
             (fmgen.fm_job(6, 200, 8, 2, 304), m.OUTPUT_LIST),
             (fmgen.fm_job(5, 250, 9, 3, 305), m.OUTPUT_LIST)]
    for job, output in cases:
        ref = oracle.search(job.rows(), job.l, job.d, threads=8)[0]
        o = m.torch_opts(output=output)
        plan = m.motif_plan_create(job.n, job.t, job.l, job.d, o)
        m.motif_load_seqs(plan, job.seqs)
        for cap in (max(1, ref.size), ref.size + 4097, max(1 << 16, ref.size)):
            assert np.array_equal(m.motif_search(plan), ref)
            out = torch.zeros(cap, dtype=torch.int64, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            m.motif_search_device(plan, out, cap, cnt)
            torch.cuda.synchronize()
            assert int(cnt.item()) == ref.size
            assert np.array_equal(out[:ref.size].cpu().numpy().astype(np.uint64), ref)
        assert np.array_equal(m.motif_search(plan), ref)
        m.motif_plan_destroy(plan)


# accepted codes: 507 (inside the codes read with the count), 2205 (beyond them, one-CTA sort),
# 164027 (beyond the one-CTA sort)
PEEK_JOBS = {"r507": (10, 192, 10, 3, 313), "r2205": (6, 200, 8, 2, 304),
             "r164k": (5, 250, 9, 3, 306)}


@pytest.fixture(scope="module")
def peek_refs():
    out = {}
    for key, (n, t, l, d, seed) in PEEK_JOBS.items():
        job = fmgen.fm_job(n, t, l, d, seed)
        out[key] = (job, oracle.search(job.rows(), l, d, threads=8)[0])
    return out


@pytest.mark.parametrize("key", sorted(PEEK_JOBS))
@pytest.mark.parametrize("rel", ["one", "size-1", "size", "size+1", "511", "512", "513", "4097"])
def test_capacity_protocol_around_the_peek(peek_refs, key, rel):
    job, ref = peek_refs[key]
    cap = {"one": 1, "size-1": max(1, ref.size - 1), "size": ref.size, "size+1": ref.size + 1,
           "511": 511, "512": 512, "513": 513, "4097": 4097}[rel]
    o = m.motif_opts_default()
    o.output = m.OUTPUT_LIST
    plan = m.motif_plan_create(job.n, job.t, job.l, job.d, o)
    m.motif_load_seqs(plan, job.seqs)
    lib = m._load()
    out = np.empty(cap, dtype=np.uint64)
    cnt = ctypes.c_int64(0)
    st = lib.motif_search(plan, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap,
                          ctypes.byref(cnt))
    assert cnt.value == ref.size
    if cap < ref.size:
        assert st == m.ERR_CAPACITY
    else:
        assert st == m.OK and np.array_equal(out[:ref.size], ref)
    assert np.array_equal(m.motif_search(plan), ref)  # and again, through the binding
    m.motif_plan_destroy(plan)


def test_small_results_fit_the_peek():
    # results from one code to tens of thousands: inside and beyond the codes read with the count
    rng = random.Random(307)
    for k in range(6):
        job = fmgen.fm_job(rng.randint(3, 10), rng.randint(40, 300), rng.randint(7, 10),
                           rng.randint(1, 3), 310 + k)
        ref = oracle.search(job.rows(), job.l, job.d, threads=8)[0]
        plan = m.motif_plan_create(job.n, job.t, job.l, job.d)
        m.motif_load_seqs(plan, job.seqs)
        assert np.array_equal(m.motif_search(plan), ref)
        m.motif_plan_destroy(plan)
