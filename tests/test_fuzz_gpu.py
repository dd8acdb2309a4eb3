"""Seeded random combinations of every option against the oracle, element by element.

Each case draws a kernel form, an output collection, candidate seeding (where the form allows
it), the tiled pass's sequence blocks, equal-length or ragged rows with masked symbols, a
candidate sub-range and a search path (blocking, device, or batched with its neighbours), and
compares the codes with the oracle's exactly.  The draws are fixed by the case number, so a failure names a reproducible case.
"""
import random

import numpy as np
import pytest

import paper_1403_1313_gb300 as m
from oracle import oracle

pytestmark = pytest.mark.gpu

KERNELS = [m.KERNEL_AUTO, m.KERNEL_TILED, m.KERNEL_GROUP, m.KERNEL_CAND, m.KERNEL_BITSLICE]
OUTPUTS = [m.OUTPUT_AUTO, m.OUTPUT_LIST, m.OUTPUT_BITMAP]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1403_1313_gb300 import build
    build.build()
    oracle.build()


def _draw(case):
    rng = random.Random(7919 * case + 17)
    l = rng.randint(2, 11)
    d = rng.randint(0, min(l, 5))
    n = rng.randint(1, 5)
    ragged = rng.random() < 0.4
    p_mask = rng.choice([0.0, 0.02, 0.08]) if ragged else 0.0
    if ragged:
        rows = []
        for _ in range(n):
            r = [rng.choice("ACGT") for _ in range(rng.randint(max(0, l - 2), 70))]
            rows.append("".join(rng.choice("NRY") if rng.random() < p_mask else c for c in r))
    else:
        t = rng.randint(max(1, l - 1), 70)
        rows = ["".join(rng.choice("ACGT") for _ in range(t)) for _ in range(n)]
    kernel = rng.choice(KERNELS)
    opts = dict(kernel=kernel, output=rng.choice(OUTPUTS))
    if kernel in (m.KERNEL_CAND, m.KERNEL_BITSLICE):
        opts["cands_per_thread"] = rng.choice([1, 2, 4])
        if rng.random() < 0.4:
            opts["seed"] = m.SEED_NEIGHBOURHOOD
    if kernel == m.KERNEL_GROUP:
        opts["suffix_bases"] = rng.randint(1, 4)
    if kernel in (m.KERNEL_AUTO, m.KERNEL_TILED) and rng.random() < 0.5:
        opts["seq_block"] = rng.choice([-1, 1, 2, 3])  # a dense bitmap job's tiled-pass split
    space = 4 ** l
    lo, hi = 0, space
    if rng.random() < 0.4:
        lo = rng.randrange(space)
        hi = rng.randrange(lo + 1, space + 1)
        opts["range_lo"], opts["range_hi"] = lo, hi
    path = rng.choice(["blocking", "device", "batch"])
    return rows, l, d, ragged, opts, (lo, hi), path


def _plan(rows, l, d, ragged, opts):
    o = m.torch_opts() if opts.pop("_torch", False) else m.motif_opts_default()
    for k, v in opts.items():
        setattr(o, k, v)
    t = max(1, max(len(r) for r in rows))
    plan = m.motif_plan_create(len(rows), t, l, d, o)
    if ragged:
        m.motif_load_seqs_var(plan, rows)
    else:
        m.motif_load_seqs(plan, rows)
    return plan


@pytest.mark.parametrize("case", range(160))
def test_random_option_combinations(case):
    rows, l, d, ragged, opts, (lo, hi), path = _draw(case)
    ref, _ = oracle.search_var(rows, l, d, lo=lo, hi=hi)
    if path == "device":
        torch = pytest.importorskip("torch")
        plan = _plan(rows, l, d, ragged, dict(opts, _torch=True))
        cap = max(1, ref.size)
        out = torch.zeros(cap, dtype=torch.int64, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        m.motif_search_device(plan, out, cap, cnt)
        torch.cuda.synchronize()
        assert int(cnt.item()) == ref.size, (case, opts)
        got = out[:ref.size].cpu().numpy().astype(np.uint64)
    elif path == "batch":
        plan = _plan(rows, l, d, ragged, dict(opts))
        # a neighbour job in the same batch, with the default options
        other = ["".join(random.Random(case).choice("ACGT") for _ in range(40)) for _ in range(3)]
        plan2 = m.motif_plan_create(3, 40, 6, 1)
        m.motif_load_seqs(plan2, other)
        got, got2 = m.motif_batch_search([plan, plan2])
        assert np.array_equal(got2, oracle.search(other, 6, 1)[0]), case
        m.motif_plan_destroy(plan2)
    else:
        plan = _plan(rows, l, d, ragged, dict(opts))
        got = m.motif_search(plan)
    m.motif_plan_destroy(plan)
    assert np.array_equal(got, ref), (case, l, d, ragged, opts, path)
