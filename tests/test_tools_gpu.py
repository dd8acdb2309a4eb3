"""GPU tests of the tooling around the search: the work counters, the autotuner and its JSON
cache, the single-process path of the sharded search, and the device-path capacity protocol."""
import itertools
import json
import random

import numpy as np
import pytest

import paper_1403_1313_gb300 as m
from oracle import oracle
from paper_1403_1313_gb300 import fmgen

pytestmark = pytest.mark.gpu
ACGT = "ACGT"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1403_1313_gb300 import build
    build.build()
    oracle.build()


def _plan(rows, l, d, **kw):
    o = m.motif_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    plan = m.motif_plan_create(len(rows), len(rows[0]), l, d, o)
    m.motif_load_seqs(plan, rows)
    return plan


def _group_tally(rows, l, d, k):
    """The GROUP formulation's canonical (group, window) tally, written out from its definition:
    groups of 4^k candidates sharing their first l-k bases; per sequence, windows left to right
    up to and including the first window after which every live candidate of the group has a
    window within d, else all W; candidates without such a window drop out; a group with none
    left stops."""
    cands = np.array(list(itertools.product(range(4), repeat=l)), dtype=np.int8)
    enc = np.array([[ACGT.index(ch) for ch in s] for s in rows], dtype=np.int8)
    W = enc.shape[1] - l + 1
    win = np.stack([enc[:, j:j + l] for j in range(W)], axis=1)        # (n, W, l)
    hit = ((cands[:, None, None, :] != win[None]).sum(-1) <= d)         # (K, n, W)
    per = 4 ** k
    total = 0
    for g in range(4 ** (l - k)):
        alive = np.ones(per, dtype=bool)
        for s in range(len(rows)):
            if not alive.any():
                break
            h = hit[g * per:(g + 1) * per, s, :]                          # (per, W)
            matched = np.zeros(per, dtype=bool)
            scanned = W
            for j in range(W):
                matched |= h[:, j]
                if np.all(matched[alive]):
                    scanned = j + 1
                    break
            total += scanned
            alive &= matched
    return total


@pytest.mark.parametrize("l,d,k,seed", [(5, 1, 2, 1), (6, 2, 3, 2), (6, 1, 4, 3), (7, 2, 4, 4)])
def test_group_unit_steps_match_definition(l, d, k, seed):
    rng = random.Random(seed)
    rows = ["".join(rng.choice(ACGT) for _ in range(rng.randint(l, 24))) for _ in range(1)]
    rows = rows * 1 + ["".join(rng.choice(ACGT) for _ in range(len(rows[0]))) for _ in range(3)]
    plan = _plan(rows, l, d, kernel=m.KERNEL_GROUP, suffix_bases=k)
    compares, unit_steps = m.motif_count_work(plan)
    m.motif_plan_destroy(plan)
    assert compares == oracle.search(rows, l, d)[1]
    assert unit_steps == _group_tally(rows, l, d, k)


@pytest.mark.parametrize("kernel", [m.KERNEL_CAND, m.KERNEL_BITSLICE])
def test_cand_unit_steps_equal_compares(kernel):
    job = fmgen.fm_job(5, 60, 7, 2, 9)
    plan = _plan(job.rows(), 7, 2, kernel=kernel)
    compares, unit_steps = m.motif_count_work(plan)
    m.motif_plan_destroy(plan)
    assert compares == unit_steps == oracle.search(job.rows(), 7, 2)[1]


def test_autotune_and_cache_roundtrip(tmp_path):
    job = fmgen.fm_job(8, 200, 11, 3, 77)
    plan = _plan(job.rows(), 11, 3)
    ref = m.motif_search(plan)
    best = m.motif_autotune(plan, 3000)
    assert best.kernel in (m.KERNEL_CAND, m.KERNEL_GROUP, m.KERNEL_TILED, m.KERNEL_BITSLICE)
    assert np.array_equal(m.motif_search(plan), ref)  # the tuned plan gives the same result
    path = str(tmp_path / "tune.json")
    m.motif_tune_cache_save(path)
    data = json.load(open(path))
    keys = [k for k in data if k.startswith("w32_l11_d3_n8")]
    assert len(keys) == 1
    entry = data[keys[0]]
    assert entry["kernel"] == best.kernel and entry["cand_per_s"] > 0
    m.motif_tune_cache_load(path)
    # A fresh plan of the same shape picks the cached choice (and runs that kernel) and agrees.
    plan2 = _plan(job.rows(), 11, 3)
    assert np.array_equal(m.motif_search(plan2), ref)
    assert m.motif_stats(plan2)["kernel"] == best.kernel
    m.motif_plan_destroy(plan)
    m.motif_plan_destroy(plan2)


def test_sharded_search_single_process_matches():
    from paper_1403_1313_gb300.shard import sharded_search
    job = fmgen.fm_job(6, 90, 8, 2, 12)
    ref, _ = oracle.search(job.rows(), 8, 2)
    assert np.array_equal(sharded_search(job.seqs, 8, 2, rank=0, world=1), ref)
    # Every rank's own range, concatenated in rank order, is the whole result.
    parts = []
    for r in range(3):
        lo, hi = m.motif_shard_range(4 ** 8, r, 3, weights=[1.0, 2.0, 3.0])
        plan = _plan(job.rows(), 8, 2, range_lo=lo, range_hi=hi)
        parts.append(m.motif_search(plan))
        m.motif_plan_destroy(plan)
    assert np.array_equal(np.concatenate(parts), ref)


def test_dynamic_sharded_search_single_process_matches():
    import torch.distributed as dist
    from paper_1403_1313_gb300.shard import dynamic_sharded_search
    job = fmgen.fm_job(6, 90, 9, 2, 13)
    ref, _ = oracle.search(job.rows(), 9, 2)
    store = dist.HashStore()
    got = dynamic_sharded_search(job.seqs, 9, 2, store, "chunks", chunk=30000)
    assert np.array_equal(got, ref)


def test_device_path_capacity_overflow_reports_count():
    torch = pytest.importorskip("torch")
    rows = ["ACGTACGTAC", "TTGACCATGA"]
    plan = m.motif_plan_create(2, 10, 5, 5, m.torch_opts())
    chars = torch.tensor([list(r.encode()) for r in rows], dtype=torch.uint8, device="cuda")
    m.motif_load_seqs_device(plan, chars)
    out = torch.zeros(100, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    m.motif_search_device(plan, out, 100, cnt)      # 1024 codes do not fit in 100
    torch.cuda.synchronize()
    assert int(cnt.item()) == 4 ** 5
    out = torch.zeros(4096, dtype=torch.int64, device="cuda")
    m.motif_search_device(plan, out, 4096, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == 4 ** 5
    assert np.array_equal(out[:1024].cpu().numpy(), np.arange(1024))
