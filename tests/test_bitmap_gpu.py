"""GPU parity of the two output collections: LIST (append, then sort and deduplicate) and BITMAP
(one bit per code of the range, then an ordered compaction of the set bits).

Both must give exactly the oracle's ascending code set for every kernel form, on whole spaces,
unaligned sub-ranges (the bitmap is rounded out to 256-code groups), dense results that overflow
the plan's first output buffer, the capacity protocol of the blocking and device paths, and a
batch that mixes the two.
"""
import ctypes
import random

import numpy as np
import pytest

import paper_1403_1313_gb300 as m
from oracle import oracle
from paper_1403_1313_gb300 import fmgen

pytestmark = pytest.mark.gpu

VARIANTS = [
    ("tiled", dict(kernel=m.KERNEL_TILED)),
    ("group4", dict(kernel=m.KERNEL_GROUP, suffix_bases=4)),
    ("group3", dict(kernel=m.KERNEL_GROUP, suffix_bases=3)),
    ("group2", dict(kernel=m.KERNEL_GROUP, suffix_bases=2)),
    ("group1", dict(kernel=m.KERNEL_GROUP, suffix_bases=1)),
    ("cand1", dict(kernel=m.KERNEL_CAND, cands_per_thread=1)),
    ("cand4", dict(kernel=m.KERNEL_CAND, cands_per_thread=4)),
    ("bitslice2", dict(kernel=m.KERNEL_BITSLICE, cands_per_thread=2)),
]
OUTPUTS = [("list", m.OUTPUT_LIST), ("bitmap", m.OUTPUT_BITMAP)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1403_1313_gb300 import build
    build.build()
    oracle.build()


def _plan(seqs, l, d, **kw):
    o = m.motif_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    n = len(seqs)
    t = seqs.shape[1] if isinstance(seqs, np.ndarray) else len(seqs[0])
    plan = m.motif_plan_create(n, t, l, d, o)
    m.motif_load_seqs(plan, seqs)
    return plan


def _search(seqs, l, d, **kw):
    plan = _plan(seqs, l, d, **kw)
    got = m.motif_search(plan)
    m.motif_plan_destroy(plan)
    return got


def _rows(rng, n, t):
    return ["".join(rng.choice("ACGT") for _ in range(t)) for _ in range(n)]


@pytest.mark.parametrize("out_name,output", OUTPUTS, ids=[o[0] for o in OUTPUTS])
@pytest.mark.parametrize("name,kw", VARIANTS, ids=[v[0] for v in VARIANTS])
@pytest.mark.parametrize("seed", range(6))
def test_small_random_both_outputs(out_name, output, name, kw, seed):
    rng = random.Random(seed * 104729 + len(name) * 7 + output)
    l = rng.randint(2, 9)
    d = rng.randint(0, min(l, 4))
    n = rng.randint(1, 6)
    t = rng.randint(max(1, l - 1), 60)
    rows = _rows(rng, n, t)
    ref, _ = oracle.search(rows, l, d)
    assert np.array_equal(_search(rows, l, d, output=output, **kw), ref)


@pytest.mark.parametrize("name,kw", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_bitmap_unaligned_subranges(name, kw):
    job = fmgen.fm_job(5, 70, 9, 3, 77)
    rng = random.Random(17)
    for _ in range(4):
        lo = rng.randrange(0, 4 ** 9 - 1)
        hi = rng.randrange(lo + 1, min(4 ** 9, lo + 50000) + 1)
        ref, _ = oracle.search(job.rows(), 9, 3, lo=lo, hi=hi)
        got = _search(job.seqs, 9, 3, output=m.OUTPUT_BITMAP, range_lo=lo, range_hi=hi, **kw)
        assert np.array_equal(got, ref), (lo, hi)


@pytest.mark.parametrize("out_name,output", OUTPUTS, ids=[o[0] for o in OUTPUTS])
@pytest.mark.parametrize("name,kw", [VARIANTS[0], VARIANTS[3], VARIANTS[5]],
                         ids=["tiled", "group2", "cand1"])
@pytest.mark.parametrize("l,d", [(6, 6), (9, 9)])
def test_dense_results_both_outputs(out_name, output, name, kw, l, d):
    """d >= l: all 4^l codes (262144 at l = 9, more than the plan's first 65536-code buffer)."""
    rows = _rows(random.Random(l + output), 3, 20)
    got = _search(rows, l, d, output=output, **kw)
    assert np.array_equal(got, np.arange(4 ** l, dtype=np.uint64))


@pytest.mark.parametrize("out_name,output", OUTPUTS, ids=[o[0] for o in OUTPUTS])
def test_capacity_protocol_both_outputs(out_name, output):
    rows = _rows(random.Random(9), 2, 12)
    plan = _plan(rows, 5, 5, output=output)
    lib = m._load()
    out = np.empty(4 ** 5, dtype=np.uint64)
    cnt = ctypes.c_int64(0)
    ptr = out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    assert lib.motif_search(plan, ptr, 10, ctypes.byref(cnt)) == m.ERR_CAPACITY
    assert cnt.value == 4 ** 5
    assert lib.motif_search(plan, ptr, 4 ** 5, ctypes.byref(cnt)) == m.OK
    assert cnt.value == 4 ** 5 and np.array_equal(out, np.arange(4 ** 5, dtype=np.uint64))
    m.motif_plan_destroy(plan)


def test_bitmap_device_path_capacity():
    """The device path writes the first `capacity` codes in ascending order and the full count."""
    torch = pytest.importorskip("torch")
    job = fmgen.fm_job(4, 50, 8, 3, 5)
    ref, _ = oracle.search(job.rows(), 8, 3)
    assert ref.size > 40
    o = m.torch_opts()
    o.output = m.OUTPUT_BITMAP
    plan = m.motif_plan_create(job.n, job.t, 8, 3, o)
    m.motif_load_seqs_device(plan, torch.from_numpy(job.seqs.copy()).cuda())
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    small = torch.zeros(40, dtype=torch.int64, device="cuda")
    m.motif_search_device(plan, small, 40, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == ref.size
    assert np.array_equal(small.cpu().numpy().astype(np.uint64), ref[:40])
    full = torch.zeros(ref.size, dtype=torch.int64, device="cuda")
    m.motif_search_device(plan, full, ref.size, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == ref.size
    assert np.array_equal(full.cpu().numpy().astype(np.uint64), ref)
    m.motif_plan_destroy(plan)


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_mixes_outputs(use_graph):
    rng = random.Random(83)
    jobs, plans = [], []
    for j in range(9):
        l = rng.randint(6, 10)
        d = rng.randint(1, 4)
        n = rng.randint(2, 6)
        t = rng.randint(l, 120)
        output = [m.OUTPUT_AUTO, m.OUTPUT_LIST, m.OUTPUT_BITMAP][j % 3]
        job = fmgen.fm_job(n, t, l, d, 900 + j)
        jobs.append((job.rows(), l, d))
        plans.append(_plan(job.seqs, l, d, output=output))
    rows = _rows(random.Random(5), 3, 20)  # every code survives: 262144 > the first buffer
    jobs.append((rows, 9, 9))
    plans.append(_plan(rows, 9, 9, output=m.OUTPUT_BITMAP))
    outs = m.motif_batch_search(plans, use_graph=use_graph)
    for (rows_j, l, d), got in zip(jobs, outs):
        ref, _ = oracle.search(rows_j, l, d)
        assert np.array_equal(got, ref)
    for p in plans:
        m.motif_plan_destroy(p)


def test_output_argument_rules():
    rows = _rows(random.Random(1), 2, 30)
    with pytest.raises(m.MotifError) as e:
        _plan(rows, 8, 2, output=3)
    assert e.value.status == m.ERR_ARG
    with pytest.raises(m.MotifError) as e:  # 4^16 codes: more than 2^31 bits
        _plan(rows, 16, 4, output=m.OUTPUT_BITMAP)
    assert e.value.status == m.ERR_ARG
    # A sub-range of the same space fits.
    ref, _ = oracle.search(rows, 16, 9, lo=5_000_000, hi=5_300_000)
    got = _search(rows, 16, 9, output=m.OUTPUT_BITMAP, range_lo=5_000_000, range_hi=5_300_000)
    assert np.array_equal(got, ref)
