"""Pins of the oracle's variable-length, masked form (oracle_skipbf_var).

Reading: sequence s has t_s characters and t_s - l + 1 windows (none when t_s < l); a window
that contains a character outside ACGTacgt never matches, and the canonical tally counts every
window position the same way (j + 1 at the first match, else t_s - l + 1).  The pins compare
it with things other than itself: a numpy distance-tensor formulation of the definition (no
skip), the d = 0 intersection of substring sets, degenerate inputs, the equal-length oracle,
and a monotonicity property of masking.
"""
import itertools
import random

import numpy as np
import pytest

from oracle import oracle

ACGT = "ACGT"


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _definition(rows, l, d):
    """R and the canonical tally from the definition, with numpy over all candidates."""
    cands = np.array(list(itertools.product(range(4), repeat=l)), dtype=np.int8)   # (K, l)
    alive = np.ones(len(cands), dtype=bool)
    first = []  # per sequence: index of the first matching window per candidate, or -1
    for r in rows:
        W = len(r) - l + 1
        if W <= 0:
            first.append(np.full(len(cands), -1))
            continue
        enc = np.array([ACGT.index(c) if c in ACGT else -1 for c in r.upper()], dtype=np.int8)
        win = np.stack([enc[j:j + l] for j in range(W)])                           # (W, l)
        dist = (cands[:, None, :] != win[None, :, :]).sum(-1)                      # (K, W)
        masked = (win < 0).any(-1)                                                 # (W,)
        ok = (dist <= d) & ~masked[None, :]
        first.append(np.where(ok.any(1), ok.argmax(1), -1))
    tally = 0
    for k in range(len(cands)):
        for s, r in enumerate(rows):
            W = max(0, len(r) - l + 1)
            j = first[s][k]
            if j < 0:
                tally += W
                alive[k] = False
                break
            tally += j + 1
    codes = np.array([k for k in range(len(cands)) if alive[k]], dtype=np.uint64)
    return codes, tally


def _rand_rows(rng, n, lmin, lmax, p_mask):
    rows = []
    for _ in range(n):
        t = rng.randint(lmin, lmax)
        rows.append("".join(rng.choice("N") if rng.random() < p_mask else rng.choice(ACGT)
                            for _ in range(t)))
    return rows


@pytest.mark.parametrize("seed", range(30))
def test_matches_the_definition(seed):
    rng = random.Random(seed)
    l = rng.randint(1, 5)
    d = rng.randint(0, l)
    rows = _rand_rows(rng, rng.randint(1, 5), 0, 24, rng.choice([0.0, 0.05, 0.2]))
    got, cmp = oracle.search_var(rows, l, d)
    ref, ref_cmp = _definition(rows, l, d)
    assert np.array_equal(got, ref)
    assert cmp == ref_cmp


@pytest.mark.parametrize("seed", range(10))
def test_d0_is_the_intersection_of_unmasked_substrings(seed):
    rng = random.Random(100 + seed)
    l = rng.randint(2, 5)
    rows = _rand_rows(rng, rng.randint(1, 4), l, 40, 0.1)
    sets = [{r[j:j + l] for j in range(len(r) - l + 1) if "N" not in r[j:j + l]} for r in rows]
    common = set.intersection(*sets)
    expect = sorted(int("".join(str(ACGT.index(c)) for c in w), 4) for w in common)
    got, _ = oracle.search_var(rows, l, 0)
    assert got.tolist() == expect


def test_short_or_fully_masked_sequences_empty_the_result():
    assert oracle.search_var(["ACGTACGT", "ACG"], 4, 4)[0].size == 0      # t_s < l
    assert oracle.search_var(["ACGTACGT", "NNNNNNNN"], 4, 4)[0].size == 0  # no unmasked window
    assert oracle.search_var(["ACGTACGT", ""], 4, 4)[0].size == 0
    # ... while a single unmasked window keeps everything within d of it
    got, _ = oracle.search_var(["NNACGTNN"], 4, 0)
    assert got.tolist() == [int("0123", 4)]


@pytest.mark.parametrize("seed", range(6))
def test_equal_lengths_without_masks_equal_the_fixed_form(seed):
    rng = random.Random(200 + seed)
    l = rng.randint(3, 7)
    d = rng.randint(0, 3)
    t = rng.randint(l, 40)
    rows = ["".join(rng.choice(ACGT) for _ in range(t)) for _ in range(rng.randint(1, 6))]
    assert [x.tolist() if hasattr(x, "tolist") else x for x in oracle.search_var(rows, l, d)] == \
        [x.tolist() if hasattr(x, "tolist") else x for x in oracle.search(rows, l, d)]


@pytest.mark.parametrize("seed", range(6))
def test_unmasking_only_adds_codes(seed):
    rng = random.Random(300 + seed)
    l, d = rng.randint(3, 6), rng.randint(0, 2)
    rows = _rand_rows(rng, 3, l, 30, 0.15)
    filled = ["".join(rng.choice(ACGT) if c == "N" else c for c in r) for r in rows]
    masked, _ = oracle.search_var(rows, l, d)
    full, _ = oracle.search_var(filled, l, d)
    assert set(masked.tolist()) <= set(full.tolist())


def test_without_masking_an_unknown_character_is_an_error():
    with pytest.raises(oracle.OracleError) as e:
        oracle.search_var(["ACGTNACG"], 3, 1, mask_unknown=False)
    assert e.value.code == -2
    got, _ = oracle.search_var(["acgtacg"], 3, 0, mask_unknown=False)  # case-insensitive
    assert got.tolist() == sorted({int("".join(str(ACGT.index(c)) for c in "ACGTACG"[j:j + 3]), 4)
                                   for j in range(5)})
