"""Pins for the CPU oracle: checks it against things other than itself.

Each test ties the oracle to the paper's definitions (Perera & Ragel Sec. I.A problem, Sec.
III.A skip-BF, Sec. IV.A index ranges) through an independent route: a definition-level brute
force without the skip, set algebra for d = 0, closed forms, hand-worked fixtures, the planted
consensus of the FM model (Sec. I.B), metamorphic invariances and the closed-form expected
work.  A plausible mistake in the oracle (a dropped sequence, `<` for `<=`, an off-by-one in the
window count, a wrong base order in the code, a broken skip) fails at least one of them.
"""
import itertools
import math
import json
import os
import random
from math import comb

import numpy as np
import pytest

from oracle import oracle
from paper_1403_1313_gb300 import fmgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ACGT = "ACGT"


def naive_definition(seqs, l, d):
    """R(l,d,S) written out from Sec. I.A / III.A with no skip and no early exit: every l-mer
    in lexicographic order (itertools.product), minimum Hamming distance over every window of
    every sequence, compared with d.  Returns indices into that lexicographic enumeration."""
    out = []
    for k, tup in enumerate(itertools.product(ACGT, repeat=l)):
        ok = True
        for s in seqs:
            s = s.upper()
            dists = [sum(a != b for a, b in zip(tup, s[j:j + l])) for j in range(len(s) - l + 1)]
            if not dists or min(dists) > d:
                ok = False
        if ok:
            out.append(k)
    return out


def base4(s):
    """Base-4 number of an l-mer with A,C,G,T = 0..3, leftmost digit most significant."""
    return int(s.translate(str.maketrans(ACGT, "0123")), 4) if s else 0


def rand_seqs(rng, n, t, lower=False):
    rows = ["".join(rng.choice(ACGT) for _ in range(t)) for _ in range(n)]
    if lower:
        rows = ["".join(ch.lower() if rng.random() < 0.5 else ch for ch in r) for r in rows]
    return rows


def codes_of(seqs, l, d):
    return oracle.search(seqs, l, d)[0].tolist()


# ---- definition-level brute force ---------------------------------------------------------

@pytest.mark.parametrize("seed", range(60))
def test_matches_naive_definition(seed):
    rng = random.Random(seed)
    l = rng.randint(1, 5)
    n = rng.randint(1, 5)
    t = rng.randint(1, 14)
    d = rng.randint(0, l + 1)
    seqs = rand_seqs(rng, n, t, lower=seed % 3 == 0)
    assert codes_of(seqs, l, d) == naive_definition(seqs, l, d)


@pytest.mark.parametrize("seed", range(6))
def test_matches_naive_on_planted(seed):
    job = fmgen.fm_job(n=4, t=12, l=5, d=1 + seed % 2, seed=100 + seed)
    seqs = job.rows()
    assert codes_of(seqs, job.l, job.d) == naive_definition(seqs, job.l, job.d)


# ---- special cases with a plain definition ------------------------------------------------

@pytest.mark.parametrize("seed", range(20))
def test_d0_is_common_substrings(seed):
    rng = random.Random(1000 + seed)
    l = rng.randint(1, 6)
    n = rng.randint(2, 6)
    t = rng.randint(l, 40)
    seqs = rand_seqs(rng, n, t)
    common = set.intersection(*({s[j:j + l] for j in range(t - l + 1)} for s in seqs))
    assert codes_of(seqs, l, 0) == sorted(base4(x) for x in common)


@pytest.mark.parametrize("l,extra", [(1, 0), (3, 0), (4, 2), (6, 0)])
def test_d_at_least_l_accepts_everything(l, extra):
    seqs = rand_seqs(random.Random(l), 3, 10)
    codes, compares = oracle.search(seqs, l, l + extra)
    assert codes.tolist() == list(range(4 ** l))
    # Every candidate matches the first window of each of the 3 sequences.
    assert compares == 4 ** l * 3


@pytest.mark.parametrize("l", [2, 5, 9])
def test_short_sequences_give_nothing(l):
    seqs = rand_seqs(random.Random(l), 2, l - 1)
    codes, compares = oracle.search(seqs, l, l)
    assert codes.size == 0 and compares == 0


def test_handworked_fixtures():
    with open(os.path.join(GOLDEN, "handworked.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        got = codes_of(c["seqs"], c["l"], c["d"])
        if "codes" in c:
            assert got == c["codes"], c["name"]
        else:
            assert len(got) == c["count"], c["name"]


# ---- encoding ------------------------------------------------------------------------------

@pytest.mark.parametrize("l", [1, 2, 4, 6])
def test_index_is_lexicographic_lmer(l):
    strings = ["".join(p) for p in itertools.product(ACGT, repeat=l)]
    assert [oracle.lmer(k, l) for k in range(4 ** l)] == strings
    assert strings == sorted(strings)
    assert all(base4(s) == k for k, s in enumerate(strings))


# ---- the planted consensus is always reported (FM model, Sec. I.B / IV.B) ------------------

@pytest.mark.parametrize("l,d,n,t,seed", [(6, 1, 5, 50, 7), (8, 2, 6, 100, 8), (9, 2, 20, 600, 1),
                                          (10, 3, 8, 200, 9)])
def test_planted_consensus_survives(l, d, n, t, seed):
    job = fmgen.fm_job(n, t, l, d, seed)
    rows = job.rows()
    # The generator plants an instance at Hamming distance exactly d in every sequence.
    for s, off in enumerate(job.offsets):
        inst = rows[s][off:off + l]
        assert sum(a != b for a, b in zip(inst, job.consensus)) == d
    codes = codes_of(rows, l, d)
    assert base4(job.consensus) in codes


def test_consensus_needs_le_not_lt():
    # A single sequence whose only windows are at distance exactly d from the consensus.
    cons = "ACGTAC"
    inst = "TCGTAA"   # positions 0 and 5 mutated: distance 2
    assert codes_of([inst], 6, 2).count(base4(cons)) == 1
    assert base4(cons) not in codes_of([inst], 6, 1)


# ---- metamorphic invariances ------------------------------------------------------------------

def _perm_code(k, l, sigma):
    s = oracle.lmer(k, l)
    return base4("".join(ACGT[sigma[ACGT.index(ch)]] for ch in s))


@pytest.mark.parametrize("seed", range(8))
def test_metamorphic(seed):
    rng = random.Random(5000 + seed)
    l = rng.randint(3, 6)
    d = rng.randint(0, 2)
    n = rng.randint(2, 5)
    t = rng.randint(l + 2, 40)
    seqs = rand_seqs(rng, n, t)
    base = codes_of(seqs, l, d)
    # Base permutation sigma maps R by sigma.
    sigma = list(range(4))
    rng.shuffle(sigma)
    tr = str.maketrans(ACGT, "".join(ACGT[sigma[i]] for i in range(4)))
    assert codes_of([s.translate(tr) for s in seqs], l, d) == sorted(_perm_code(k, l, sigma) for k in base)
    # Reversing every sequence reverses every member of R.
    rev = codes_of([s[::-1] for s in seqs], l, d)
    assert rev == sorted(base4(oracle.lmer(k, l)[::-1]) for k in base)
    # Sequence order does not change R.
    shuffled = seqs[:]
    rng.shuffle(shuffled)
    assert codes_of(shuffled, l, d) == base
    # R(d) is contained in R(d+1).
    assert set(base) <= set(codes_of(seqs, l, d + 1))
    # Adding a sequence can only shrink R; duplicating one leaves it unchanged.
    assert set(codes_of(seqs + rand_seqs(rng, 1, t), l, d)) <= set(base)
    assert codes_of(seqs + [seqs[0]], l, d) == base
    # Case does not matter.
    assert codes_of([s.lower() for s in seqs], l, d) == base


def test_bad_alphabet_is_an_error():
    with pytest.raises(oracle.OracleError) as e:
        oracle.search(["ACGN"], 2, 0)
    assert e.value.code == -2


# ---- the index-range split (Sec. IV.A) ---------------------------------------------------------

@pytest.mark.parametrize("threads", [2, 3, 7])
def test_thread_split_matches_single(threads):
    job = fmgen.fm_job(8, 80, 7, 2, 42)
    rows = job.rows()
    one = oracle.search(rows, 7, 2)
    many = oracle.search(rows, 7, 2, threads=threads)
    assert one[0].tolist() == many[0].tolist() and one[1] == many[1]
    # Arbitrary sub-ranges concatenate to the whole.
    cuts = sorted({0, 4 ** 7, 1000, 5555, 9000})
    parts = [oracle.search(rows, 7, 2, lo=a, hi=b) for a, b in zip(cuts, cuts[1:])]
    assert np.concatenate([p[0] for p in parts]).tolist() == one[0].tolist()
    assert sum(p[1] for p in parts) == one[1]


# ---- the canonical compare tally --------------------------------------------------------------

def _tally_from_distance_matrix(seqs, l, d):
    """Work count from a full distance tensor D[k, s, j] (no early exits anywhere): per
    candidate, sequences in order; a sequence whose first window within d is j costs j+1, a
    sequence with none costs W and ends the candidate's scan."""
    cands = np.array(list(itertools.product(range(4), repeat=l)), dtype=np.int8)       # (K, l)
    enc = np.array([[ACGT.index(ch) for ch in s.upper()] for s in seqs], dtype=np.int8)  # (n, t)
    W = enc.shape[1] - l + 1
    win = np.stack([enc[:, j:j + l] for j in range(W)], axis=1)                          # (n, W, l)
    D = (cands[:, None, None, :] != win[None, :, :, :]).sum(-1)                            # (K, n, W)
    hit = D <= d
    total = 0
    for k in range(cands.shape[0]):
        for s in range(len(seqs)):
            row = hit[k, s]
            if row.any():
                total += int(np.argmax(row)) + 1
            else:
                total += W
                break
    return total


@pytest.mark.parametrize("seed", range(6))
def test_compare_tally_matches_distance_matrix(seed):
    rng = random.Random(77 + seed)
    l = rng.randint(2, 5)
    d = rng.randint(0, 2)
    seqs = rand_seqs(rng, rng.randint(1, 4), rng.randint(l, 20))
    assert oracle.search(seqs, l, d)[1] == _tally_from_distance_matrix(seqs, l, d)


@pytest.mark.parametrize("l,d,n,t,seed", [(9, 2, 20, 600, 11), (8, 2, 10, 300, 5)])
def test_compare_tally_near_closed_form(l, d, n, t, seed):
    """Expected compares per candidate for i.i.d. uniform text, treating windows as
    independent: p = P[Ham <= d] = sum_k C(l,k) 3^k / 4^l, A = (1 - (1-p)^W) / p per visited
    sequence, q = 1 - (1-p)^W, total A (1 - q^n) / (1 - q).  Overlapping windows make this an
    approximation, so the check is loose (3 %)."""
    seqs = fmgen.random_text(n, t, seed)
    _, compares = oracle.search(seqs, l, d, threads=8)
    p = sum(comb(l, k) * 3 ** k for k in range(d + 1)) / 4 ** l
    W = t - l + 1
    q = 1 - (1 - p) ** W
    expect = q / p * (1 - q ** n) / (1 - q)
    assert abs(compares / 4 ** l / expect - 1) < 0.03


# ---- stored expected values -------------------------------------------------------------------

def test_golden_l9d2_matches_regeneration():
    """The stored (9,2) result was written by tests/golden/make_golden.py (oracle only); the
    regenerated inputs and the oracle must reproduce it on this machine."""
    with open(os.path.join(GOLDEN, "l9d2_n20_t600_seed1.json")) as f:
        g = json.load(f)
    job = fmgen.single("l9d2")
    import hashlib
    assert hashlib.sha256(job.seqs.tobytes()).hexdigest() == g["seqs_sha256"]
    codes, compares = oracle.search(job.rows(), 9, 2, threads=4)
    assert codes.tolist() == g["codes"] and compares == g["compares"]
    assert base4(job.consensus) in g["codes"]


def test_golden_l15d4_is_consistent():
    """The stored complete (15,4) result (about 25 minutes of oracle time on 8 cores, so not
    regenerated here): same inputs, the planted consensus among the codes, every stored code
    accepted by the oracle alone, its three neighbours in the last base stored exactly when the
    oracle accepts them, and a compare tally within 0.1 % of the closed form for uniform bases
    (the skip's expected work)."""
    with open(os.path.join(GOLDEN, "l15d4_n20_t600_seed2.json")) as f:
        g = json.load(f)
    job = fmgen.single("l15d4")
    import hashlib
    assert hashlib.sha256(job.seqs.tobytes()).hexdigest() == g["seqs_sha256"]
    assert g["consensus"] == job.consensus and base4(job.consensus) in g["codes"]
    stored = set(g["codes"])
    for c in g["codes"]:
        assert oracle.search(job.rows(), 15, 4, lo=c, hi=c + 1)[0].tolist() == [c]
        for x in range(1, 4):  # the other three bases at the last position
            other = (c & ~3) | ((c + x) & 3)
            got = oracle.search(job.rows(), 15, 4, lo=other, hi=other + 1)[0].tolist()
            assert (other in stored) == (got == [other])
    l, d, n, W = 15, 4, 20, 600 - 15 + 1
    p = sum(math.comb(l, k) * 3 ** k for k in range(d + 1)) / 4 ** l
    q = 1 - (1 - p) ** W
    expect = 4 ** l * (1 - q ** n) / (1 - q) * q / p
    assert abs(g["compares"] / expect - 1) < 0.001


def test_golden_l17d5_is_consistent():
    """The stored complete (17,5) result (about 4 h of oracle time on 8 cores, so not
    regenerated here): same inputs, the planted consensus among the codes, every stored code
    accepted by the oracle alone, its three neighbours in the last base stored exactly when the
    oracle accepts them, and a compare tally within 0.1 % of the closed form for uniform bases."""
    with open(os.path.join(GOLDEN, "l17d5_n20_t600_seed3.json")) as f:
        g = json.load(f)
    job = fmgen.single("l17d5")
    import hashlib
    assert hashlib.sha256(job.seqs.tobytes()).hexdigest() == g["seqs_sha256"]
    assert g["consensus"] == job.consensus and base4(job.consensus) in g["codes"]
    stored = set(g["codes"])
    for c in g["codes"]:
        assert oracle.search(job.rows(), 17, 5, lo=c, hi=c + 1)[0].tolist() == [c]
        for x in range(1, 4):  # the other three bases at the last position
            other = (c & ~3) | ((c + x) & 3)
            got = oracle.search(job.rows(), 17, 5, lo=other, hi=other + 1)[0].tolist()
            assert (other in stored) == (got == [other])
    l, d, n, W = 17, 5, 20, 600 - 17 + 1
    p = sum(math.comb(l, k) * 3 ** k for k in range(d + 1)) / 4 ** l
    q = 1 - (1 - p) ** W
    expect = 4 ** l * (1 - q ** n) / (1 - q) * q / p
    assert abs(g["compares"] / expect - 1) < 0.001
