"""GPU parity for sequences of their own lengths with masked unknown characters
(motif_load_seqs_var) against the oracle's variable-length form, element by element.

Covers every kernel form and both output collections, rows shorter than l, empty and fully
masked rows, masks at row ends and in the middle, the canonical compare tally, the device
path, batching, serving, and FASTA text end to end.
"""
import random

import numpy as np
import pytest

import paper_1403_1313_gb300 as m
from oracle import oracle

pytestmark = pytest.mark.gpu

VARIANTS = [
    ("tiled", dict(kernel=m.KERNEL_TILED)),
    ("group4", dict(kernel=m.KERNEL_GROUP, suffix_bases=4)),
    ("group2", dict(kernel=m.KERNEL_GROUP, suffix_bases=2)),
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


def _plan(rows, l, d, **kw):
    o = m.motif_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    t = max(1, max(len(r) for r in rows))
    plan = m.motif_plan_create(len(rows), t, l, d, o)
    m.motif_load_seqs_var(plan, rows)
    return plan


def _ragged(rng, n, lmin, lmax, p_mask, l):
    rows = []
    for _ in range(n):
        t = rng.randint(lmin, lmax)
        r = [rng.choice("ACGT") for _ in range(t)]
        for i in range(t):
            if rng.random() < p_mask:
                r[i] = rng.choice("NnRYX-")
        rows.append("".join(r))
    return rows


@pytest.mark.parametrize("out_name,output", OUTPUTS, ids=[o[0] for o in OUTPUTS])
@pytest.mark.parametrize("name,kw", VARIANTS, ids=[v[0] for v in VARIANTS])
@pytest.mark.parametrize("seed", range(8))
def test_ragged_masked_random(out_name, output, name, kw, seed):
    rng = random.Random(seed * 31 + len(name) + 7 * output)
    l = rng.randint(3, 10)
    d = rng.randint(0, min(l, 4))
    n = rng.randint(1, 6)
    rows = _ragged(rng, n, max(0, l - 2), 90, rng.choice([0.0, 0.01, 0.05]), l)
    ref, ref_cmp = oracle.search_var(rows, l, d)
    plan = _plan(rows, l, d, output=output, **kw)
    got = m.motif_search(plan)
    cmp = m.motif_count_compares(plan)
    m.motif_plan_destroy(plan)
    assert np.array_equal(got, ref)
    assert cmp == ref_cmp


@pytest.mark.parametrize("name,kw", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_planted_motif_survives_masking_elsewhere(name, kw):
    rng = random.Random(5)
    l, d = 9, 2
    motif = "".join(rng.choice("ACGT") for _ in range(l))
    rows = []
    for s in range(6):
        t = rng.randint(40, 160)
        r = [rng.choice("ACGT") for _ in range(t)]
        inst = list(motif)
        for p in rng.sample(range(l), d):
            inst[p] = rng.choice([c for c in "ACGT" if c != inst[p]])
        at = rng.randint(0, t - l)
        r[at:at + l] = inst
        for i in range(t):  # mask a few positions outside the planted instance
            if not at <= i < at + l and rng.random() < 0.05:
                r[i] = "N"
        rows.append("".join(r))
    ref, ref_cmp = oracle.search_var(rows, l, d)
    assert m.motif_encode(motif) in set(ref.tolist())
    plan = _plan(rows, l, d, **kw)
    assert np.array_equal(m.motif_search(plan), ref)
    assert m.motif_count_compares(plan) == ref_cmp
    m.motif_plan_destroy(plan)


@pytest.mark.parametrize("rows", [
    ["ACGTACGTAC", "ACG"],            # a row shorter than l
    ["ACGTACGTAC", ""],               # an empty row
    ["ACGTACGTAC", "NNNNNNNN"],       # a fully masked row
    ["ACGTNACGTA", "TTNNACGTNN"],     # masks everywhere but one window
], ids=["short", "empty", "all_masked", "one_window"])
def test_degenerate_rows(rows):
    l, d = 4, 1
    ref, ref_cmp = oracle.search_var(rows, l, d)
    for name, kw in VARIANTS:
        plan = _plan(rows, l, d, **kw)
        assert np.array_equal(m.motif_search(plan), ref), name
        assert m.motif_count_compares(plan) == ref_cmp, name
        m.motif_plan_destroy(plan)


def test_without_masking_unknown_characters_are_rejected():
    plan = m.motif_plan_create(2, 10, 4, 1)
    with pytest.raises(m.MotifError) as e:
        m.motif_load_seqs_var(plan, ["ACGTNACG", "ACGTAC"], mask_unknown=False)
    assert e.value.status == m.ERR_ALPHABET
    # The plan is usable again after a valid load.
    m.motif_load_seqs_var(plan, ["ACGTAACG", "acgtac"], mask_unknown=False)
    ref, _ = oracle.search_var(["ACGTAACG", "acgtac"], 4, 1, mask_unknown=False)
    assert np.array_equal(m.motif_search(plan), ref)
    m.motif_plan_destroy(plan)


def test_equal_length_load_after_a_ragged_one():
    """A plan reloaded with motif_load_seqs drops the ragged state."""
    rows = ["ACGTACGTAA", "TTGACCATGA"]
    plan = _plan(["ACGTNCGTAA", "TTG"], 4, 1)
    assert m.motif_search(plan).size == 0  # "TTG" is shorter than l
    m.motif_load_seqs(plan, rows)
    ref, ref_cmp = oracle.search(rows, 4, 1)
    assert np.array_equal(m.motif_search(plan), ref)
    assert m.motif_count_compares(plan) == ref_cmp
    m.motif_plan_destroy(plan)


def test_device_path_batch_and_serving():
    torch = pytest.importorskip("torch")
    rng = random.Random(11)
    jobs = []
    for j in range(6):
        l = rng.randint(6, 10)
        d = rng.randint(1, 3)
        jobs.append((_ragged(rng, rng.randint(2, 5), l - 1, 120, 0.03, l), l, d))
    refs = [oracle.search_var(r, l, d)[0] for r, l, d in jobs]
    # device path
    rows, l, d = jobs[0]
    plan = _plan(rows, l, d, **{"stream": torch.cuda.current_stream().cuda_stream})
    out = torch.zeros(max(1, refs[0].size), dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    m.motif_search_device(plan, out, out.numel(), cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == refs[0].size
    assert np.array_equal(out[:refs[0].size].cpu().numpy().astype(np.uint64), refs[0])
    m.motif_plan_destroy(plan)
    # batch
    plans = [_plan(r, l, d) for r, l, d in jobs]
    for got, ref in zip(m.motif_batch_search(plans), refs):
        assert np.array_equal(got, ref)
    # serving
    m.motif_server_start(max_active=8)
    try:
        ids = [m.motif_submit(p) for p in plans]
        for jid, ref in zip(ids, refs):
            res = None
            while res is None:
                res = m.motif_poll(jid, timeout_ms=5000)
            assert np.array_equal(res[0], ref)
    finally:
        m.motif_server_stop()
    for p in plans:
        m.motif_plan_destroy(p)


def test_fasta_end_to_end():
    rng = random.Random(21)
    recs = _ragged(rng, 5, 30, 200, 0.02, 8)
    text = "".join(">r%d\n%s\n" % (i, "\n".join(r[k:k + 60] for k in range(0, len(r), 60)))
                   for i, r in enumerate(recs))
    rows = m.motif_fasta_parse(text)
    assert rows == [r.encode() for r in recs]
    ref, _ = oracle.search_var(recs, 8, 2)
    plan = _plan(rows, 8, 2)
    assert np.array_equal(m.motif_search(plan), ref)
    m.motif_plan_destroy(plan)
