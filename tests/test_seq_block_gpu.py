"""The prefix-tiled pass split into (tile, sequence block) items, against the oracle.

A dense job with bitmap output can run its tiled pass as items of one tile and a block of
sequences, each ANDing its survivors into a bitmap that starts as all ones.  Every block size
must give exactly the oracle's code set: one sequence per item, blocks with a ragged last block,
one block of all n sequences, never split (-1), and the automatic choice; on whole code spaces
and on sub-ranges whose tiles end inside the range; through the blocking, device, batched and
served paths.
"""
import random

import numpy as np
import pytest

import paper_1403_1313_gb300 as m
from oracle import oracle
from paper_1403_1313_gb300 import fmgen

pytestmark = pytest.mark.gpu

BLOCKS = [-1, 0, 1, 2, 3, 7, 100]

# (n, t, l, d, seed): dense results (AUTO takes the bitmap) and one sparse (8-mers, 13 rows)
DENSE = [(6, 300, 9, 3, 81), (9, 260, 10, 3, 82), (4, 200, 10, 4, 83), (5, 250, 9, 4, 84),
         (13, 160, 8, 2, 85)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1403_1313_gb300 import build
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def dense():
    js = [fmgen.fm_job(n, t, l, d, s) for n, t, l, d, s in DENSE]
    return js, [oracle.search(j.rows(), j.l, j.d, threads=8)[0] for j in js]


def _plan(job, **kw):
    o = m.motif_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    p = m.motif_plan_create(job.n, job.t, job.l, job.d, o)
    m.motif_load_seqs(p, job.seqs)
    return p


@pytest.mark.parametrize("seq_block", BLOCKS)
@pytest.mark.parametrize("which", range(len(DENSE)))
def test_blocking_search(dense, which, seq_block):
    js, refs = dense
    p = _plan(js[which], kernel=m.KERNEL_TILED, output=m.OUTPUT_BITMAP, seq_block=seq_block)
    got = m.motif_search(p)
    assert m.motif_stats(p)["kernel"] == m.KERNEL_TILED
    m.motif_plan_destroy(p)
    assert np.array_equal(got, refs[which])


@pytest.mark.parametrize("seq_block", [0, 1, 4])
def test_sub_ranges(seq_block):
    # tiles of 2^16 codes: lo on a tile boundary, hi inside a tile and inside a 256-code group
    job = fmgen.fm_job(8, 300, 11, 4, 86)
    for lo, hi in [(0, 1 << 18), (1 << 16, (5 << 16) + 12345), (3 << 16, (3 << 16) + 300),
                   ((4 ** 11) - (2 << 16), 4 ** 11)]:
        ref, _ = oracle.search(job.rows(), 11, 4, lo=lo, hi=hi, threads=8)
        p = _plan(job, kernel=m.KERNEL_TILED, output=m.OUTPUT_BITMAP, seq_block=seq_block,
                  range_lo=lo, range_hi=hi)
        got = m.motif_search(p)
        m.motif_plan_destroy(p)
        assert np.array_equal(got, ref), (lo, hi)


def test_auto_splits_dense_jobs(dense):
    js, refs = dense
    for j, r in zip(js, refs):
        p = _plan(j)  # AUTO kernel, AUTO output
        got = m.motif_search(p)
        m.motif_plan_destroy(p)
        assert np.array_equal(got, r)


def test_device_path(dense):
    torch = pytest.importorskip("torch")
    js, refs = dense
    for seq_block in (0, 1, 3):
        for j, r in zip(js, refs):
            o = m.torch_opts(kernel=m.KERNEL_TILED, output=m.OUTPUT_BITMAP, seq_block=seq_block)
            p = m.motif_plan_create(j.n, j.t, j.l, j.d, o)
            m.motif_load_seqs(p, j.seqs)
            out = torch.zeros(max(1, r.size), dtype=torch.int64, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            m.motif_search_device(p, out, out.numel(), cnt)
            torch.cuda.synchronize()
            assert int(cnt.item()) == r.size
            assert np.array_equal(out[:r.size].cpu().numpy().astype(np.uint64), r)
            m.motif_plan_destroy(p)


def test_batch_mixes_split_and_whole(dense):
    js, refs = dense
    rng = random.Random(87)
    plans = [_plan(j, seq_block=rng.choice(BLOCKS)) for j in js]
    sparse = fmgen.fm_job(10, 200, 11, 2, 88)  # a list-output job in the same batch
    plans.append(_plan(sparse))
    expect = refs + [oracle.search(sparse.rows(), 11, 2, threads=8)[0]]
    for use_graph in (True, False):
        got = m.motif_batch_search(plans, use_graph=use_graph)
        for g, r in zip(got, expect):
            assert np.array_equal(g, r)
    for p in plans:
        m.motif_plan_destroy(p)


def test_served_dense_jobs(dense):
    js, refs = dense
    try:
        ids = []
        for j in js:
            p = _plan(j)
            ids.append(m.motif_submit(p))
            m.motif_plan_destroy(p)
        for jid, r in zip(ids, refs):
            got, _ = m.motif_poll(jid, timeout_ms=120000, capacity=max(1, r.size))
            assert np.array_equal(got, r)
    finally:
        m.motif_server_stop()


def test_bad_block_is_rejected():
    job = fmgen.fm_job(3, 60, 9, 2, 89)
    with pytest.raises(m.MotifError) as e:
        _plan(job, seq_block=-2)
    assert e.value.status == m.ERR_ARG


def test_split_over_a_large_range_and_served():
    # (16,7) on 4 rows of 40 bases over [0, 2^31), about 1.8 M accepted codes (bitmap output):
    # the split and whole-tile passes must agree exactly (a tiled pass takes the range as one
    # chunk), the served job must agree too, and the oracle must agree on ranges at both ends,
    # across 2^30, and around the planted consensus
    job = fmgen.fm_job(4, 40, 16, 7, 92)
    cons = m.motif_encode(job.consensus)
    assert (1 << 30) < cons < (1 << 31)
    results = {}
    for sb in (-1, 1, 2):
        p = _plan(job, kernel=m.KERNEL_TILED, output=m.OUTPUT_BITMAP, seq_block=sb,
                  range_lo=0, range_hi=1 << 31)
        results[sb] = m.motif_search(p)
        m.motif_plan_destroy(p)
    assert results[-1].size > 1_000_000
    assert np.array_equal(results[1], results[-1])
    assert np.array_equal(results[2], results[-1])
    full = results[-1]
    try:
        p = _plan(job, kernel=m.KERNEL_TILED, output=m.OUTPUT_BITMAP, seq_block=1,
                  range_lo=0, range_hi=1 << 31)
        jid = m.motif_submit(p)
        m.motif_plan_destroy(p)
        served, _ = m.motif_poll(jid, timeout_ms=120000, capacity=full.size)
        assert np.array_equal(served, full)
    finally:
        m.motif_server_stop()
    for lo, hi in [(0, 1 << 14), ((1 << 30) - (1 << 13), (1 << 30) + (1 << 13)),
                   (cons - (1 << 13), cons + (1 << 13)), ((1 << 31) - (1 << 14), 1 << 31)]:
        ref, _ = oracle.search(job.rows(), 16, 7, lo=lo, hi=hi, threads=8)
        assert np.array_equal(full[(full >= lo) & (full < hi)], ref), (lo, hi)
