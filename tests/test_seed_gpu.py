"""Candidates seeded by the d-neighbourhoods of the first sequence's windows
(MOTIF_SEED_NEIGHBOURHOOD): the result must equal the oracle's exactly (a candidate outside every
neighbourhood cannot match the first sequence), and the seed count must equal the number of range
candidates within d of some window of the first sequence, computed here from its definition.
"""
import itertools
import random

import numpy as np
import pytest

import paper_1403_1313_gb300 as m
from oracle import oracle
from paper_1403_1313_gb300 import fmgen

pytestmark = pytest.mark.gpu

KERNELS = [("cand1", m.KERNEL_CAND, 1), ("cand4", m.KERNEL_CAND, 4),
           ("bitslice2", m.KERNEL_BITSLICE, 2), ("bitslice4", m.KERNEL_BITSLICE, 4)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1403_1313_gb300 import build
    build.build()
    oracle.build()


def _plan(rows, l, d, ragged=False, **kw):
    o = m.motif_opts_default()
    o.seed = m.SEED_NEIGHBOURHOOD
    for k, v in kw.items():
        setattr(o, k, v)
    t = max(len(r) for r in rows)
    plan = m.motif_plan_create(len(rows), t, l, d, o)
    if ragged:
        m.motif_load_seqs_var(plan, rows)
    else:
        m.motif_load_seqs(plan, rows)
    return plan


def _rows(rng, n, t):
    return ["".join(rng.choice("ACGT") for _ in range(t)) for _ in range(n)]


def _neighbourhood_count(row, l, d, lo, hi):
    """Range candidates within d of some window of `row`, from the definition."""
    cands = np.array(list(itertools.product(range(4), repeat=l)), dtype=np.int8)[lo:hi]
    enc = np.array(["ACGT".index(c) for c in row], dtype=np.int8)
    win = np.stack([enc[j:j + l] for j in range(len(row) - l + 1)])
    near = ((cands[:, None, :] != win[None, :, :]).sum(-1) <= d).any(1)
    return int(near.sum())


@pytest.mark.parametrize("out_name,output", [("list", m.OUTPUT_LIST), ("bitmap", m.OUTPUT_BITMAP)])
@pytest.mark.parametrize("name,kernel,cpt", KERNELS, ids=[k[0] for k in KERNELS])
@pytest.mark.parametrize("seed", range(8))
def test_seeded_search_matches_oracle(out_name, output, name, kernel, cpt, seed):
    rng = random.Random(seed * 7 + cpt + kernel)
    l = rng.randint(2, 9)
    d = rng.randint(0, min(l, 4))
    n = rng.randint(1, 6)
    t = rng.randint(max(1, l - 1), 60)
    rows = _rows(rng, n, t)
    ref, _ = oracle.search(rows, l, d)
    plan = _plan(rows, l, d, kernel=kernel, cands_per_thread=cpt, output=output)
    assert np.array_equal(m.motif_search(plan), ref)
    m.motif_plan_destroy(plan)


@pytest.mark.parametrize("seed", range(6))
def test_seed_count_is_the_neighbourhood_union(seed):
    rng = random.Random(100 + seed)
    l = rng.randint(3, 7)
    d = rng.randint(0, 3)
    rows = _rows(rng, 3, rng.randint(l, 40))
    lo = rng.randrange(0, 4 ** l)
    hi = rng.randrange(lo + 1, 4 ** l + 1)
    plan = _plan(rows, l, d, kernel=m.KERNEL_BITSLICE, range_lo=lo, range_hi=hi)
    assert m.motif_seed_count(plan) == _neighbourhood_count(rows[0], l, d, lo, hi)
    ref, _ = oracle.search(rows, l, d, lo=lo, hi=hi)
    assert np.array_equal(m.motif_search(plan), ref)
    m.motif_plan_destroy(plan)


@pytest.mark.parametrize("name,kernel,cpt", KERNELS, ids=[k[0] for k in KERNELS])
def test_seeded_planted_and_single_sequence(name, kernel, cpt):
    job = fmgen.fm_job(6, 120, 10, 3, 55)
    ref, _ = oracle.search(job.rows(), 10, 3)
    plan = _plan(job.rows(), 10, 3, kernel=kernel, cands_per_thread=cpt)
    got = m.motif_search(plan)
    m.motif_plan_destroy(plan)
    assert np.array_equal(got, ref) and m.motif_encode(job.consensus) in set(got.tolist())
    # One sequence: the seed itself is the result.
    one = job.rows()[:1]
    ref1, _ = oracle.search(one, 10, 3)
    plan = _plan(one, 10, 3, kernel=kernel, cands_per_thread=cpt)
    assert np.array_equal(m.motif_search(plan), ref1)
    assert m.motif_seed_count(plan) == ref1.size
    m.motif_plan_destroy(plan)


def test_seeded_ragged_and_batch():
    rng = random.Random(8)
    rows = ["".join(rng.choice("ACGTN") for _ in range(rng.randint(20, 90))) for _ in range(4)]
    ref, _ = oracle.search_var(rows, 7, 2)
    plan = _plan(rows, 7, 2, ragged=True, kernel=m.KERNEL_BITSLICE)
    assert np.array_equal(m.motif_search(plan), ref)
    m.motif_plan_destroy(plan)
    jobs, plans = [], []
    for j in range(5):
        job = fmgen.fm_job(rng.randint(2, 6), rng.randint(30, 150), 9, 2, 600 + j)
        jobs.append(job)
        plans.append(_plan(job.rows(), 9, 2, kernel=[m.KERNEL_CAND, m.KERNEL_BITSLICE][j % 2]))
    for job, got in zip(jobs, m.motif_batch_search(plans)):
        assert np.array_equal(got, oracle.search(job.rows(), 9, 2)[0])
    for p in plans:
        m.motif_plan_destroy(p)


def test_full_size_sampled_l15d4():
    job = fmgen.single("l15d4")
    lo = 4 ** 15 // 3 - 12345
    hi = lo + (1 << 16)
    ref, _ = oracle.search(job.rows(), 15, 4, lo=lo, hi=hi, threads=8)
    plan = _plan(job.rows(), 15, 4, kernel=m.KERNEL_BITSLICE, cands_per_thread=4,
                 range_lo=lo, range_hi=hi)
    assert np.array_equal(m.motif_search(plan), ref)
    m.motif_plan_destroy(plan)


def test_seed_argument_rules():
    rows = _rows(random.Random(3), 2, 30)
    for kw in (dict(kernel=m.KERNEL_GROUP), dict(kernel=m.KERNEL_TILED), dict(kernel=m.KERNEL_AUTO),
               dict(kernel=m.KERNEL_CAND, seq_block=-2)):
        with pytest.raises(m.MotifError) as e:
            _plan(rows, 8, 2, **kw)
        assert e.value.status == m.ERR_ARG
    with pytest.raises(m.MotifError) as e:  # sum_k<=9 C(20,k) 3^k patterns: more than 2^24
        _plan(rows, 20, 9, kernel=m.KERNEL_CAND, range_lo=0, range_hi=1 << 20)
    assert e.value.status == m.ERR_ARG
    plan = m.motif_plan_create(2, 30, 8, 2)  # an unseeded plan has no seed count
    m.motif_load_seqs(plan, rows)
    with pytest.raises(m.MotifError) as e:
        m.motif_seed_count(plan)
    assert e.value.status == m.ERR_STATE
    m.motif_plan_destroy(plan)
