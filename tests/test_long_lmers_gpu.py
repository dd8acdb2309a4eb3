"""Long l-mers (l = 16 .. 31: codes wider than 32 bits, planes up to 31 bits) against the oracle.

Every kernel form, including the bit-sliced one whose candidate code spans two 32-bit words for
l > 16 and the seeded search, on candidate sub-ranges chosen so that the expected result is not
empty: around an FM-planted consensus (planted with d-1 mutations and searched at d, so that its
distance-1 neighbours in the range are accepted too), across the 2^32 code boundary (codes on
both sides accepted), and at the top of the code space (hi = 4^l).
"""
import math

import numpy as np
import pytest

import paper_1403_1313_gb300 as m
from oracle import oracle
from paper_1403_1313_gb300 import fmgen

pytestmark = pytest.mark.gpu

FORMS = [
    ("auto", dict()),
    ("tiled", dict(kernel=m.KERNEL_TILED)),
    ("group4", dict(kernel=m.KERNEL_GROUP, suffix_bases=4)),
    ("cand2", dict(kernel=m.KERNEL_CAND, cands_per_thread=2)),
    ("bitslice1", dict(kernel=m.KERNEL_BITSLICE, cands_per_thread=1)),
    ("bitslice4", dict(kernel=m.KERNEL_BITSLICE, cands_per_thread=4)),
    ("bitslice_seeded", dict(kernel=m.KERNEL_BITSLICE, seed=m.SEED_NEIGHBOURHOOD)),
    ("cand_seeded", dict(kernel=m.KERNEL_CAND, seed=m.SEED_NEIGHBOURHOOD)),
    ("bitmap", dict(kernel=m.KERNEL_TILED, output=m.OUTPUT_BITMAP)),
]


def _patterns(l, d):
    return sum(math.comb(l, k) * 3 ** k for k in range(d + 1))


def _decode(code, l):
    return "".join("ACGT"[(code >> (2 * (l - 1 - i))) & 3] for i in range(l))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1403_1313_gb300 import build
    build.build()
    oracle.build()


def _check(rows, l, d, lo, hi, kw, must_hold, tiled=False):
    ref, _ = oracle.search(rows, l, d, lo=lo, hi=hi, threads=8)
    assert set(must_hold) <= set(ref.tolist())
    o = m.motif_opts_default()
    o.range_lo, o.range_hi = lo, hi
    for k, v in kw.items():
        setattr(o, k, v)
    t = len(rows[0])
    if kw.get("seed") and _patterns(l, d) > 1 << 24:
        # the difference-pattern table of a seeded search holds at most 2^24 entries
        with pytest.raises(m.MotifError) as e:
            m.motif_plan_create(len(rows), t, l, d, o)
        assert e.value.status == m.ERR_ARG
        return
    plan = m.motif_plan_create(len(rows), t, l, d, o)
    m.motif_load_seqs(plan, rows)
    got = m.motif_search(plan)
    kernel = m.motif_stats(plan)["kernel"]
    m.motif_plan_destroy(plan)
    assert np.array_equal(got, ref)
    if tiled and kw.get("kernel") == m.KERNEL_TILED:
        assert kernel == m.KERNEL_TILED   # lo on a multiple of 2^16: the tiled pass ran


@pytest.mark.parametrize("name,kw", FORMS, ids=[f[0] for f in FORMS])
@pytest.mark.parametrize("l,d", [(16, 4), (17, 5), (20, 6), (24, 3), (31, 2)])
def test_around_a_planted_consensus(name, kw, l, d):
    job = fmgen.fm_job(5, 140, l, d - 1, 4000 + l)
    c = m.motif_encode(job.consensus)
    lo = max(0, c - (1 << 14) - 77)
    hi = min(4 ** l, c + (1 << 14) + 35)
    _check(job.rows(), l, d, lo, hi, kw, [c])


# (l, d, codes planted exactly in every row, lo, hi); lo on a multiple of 2^16 (the tiled pass
# needs its tiles of 2^16 codes aligned), hi ragged or the end of the code space
EDGES = [
    (17, 3, [(1 << 32) - 7, (1 << 32) + 5], (1 << 32) - (1 << 16), (1 << 32) + 7001),
    (20, 4, [(1 << 32) - 2, (1 << 32) + 300], (1 << 32) - (1 << 16), (1 << 32) + 12000),
    (24, 2, [4 ** 24 - 3], 4 ** 24 - (1 << 16), 4 ** 24),
    (31, 3, [4 ** 31 - 1], 4 ** 31 - (3 << 16), 4 ** 31),
]


@pytest.mark.parametrize("name,kw", FORMS, ids=[f[0] for f in FORMS])
@pytest.mark.parametrize("l,d,codes,lo,hi", EDGES, ids=[f"l{e[0]}d{e[1]}" for e in EDGES])
def test_code_space_edges(name, kw, l, d, codes, lo, hi):
    # background rows; copy j of each code sits at a seeded offset in the j-th part of every row
    n, t = 4, 120
    rows = fmgen.background(n, t, 9000 + l)
    part = t // len(codes)
    offs = fmgen.draws(9000 + l, 1, n * len(codes)) % np.uint64(part - l + 1)
    for j, code in enumerate(codes):
        cons = np.frombuffer(_decode(code, l).encode(), dtype=np.uint8)
        for s in range(n):
            o = j * part + int(offs[s * len(codes) + j])
            rows[s, o:o + l] = cons
    _check([r.tobytes().decode() for r in rows], l, d, lo, hi, kw, codes, tiled=True)


def test_l32_is_rejected():
    with pytest.raises(m.MotifError) as e:
        m.motif_plan_create(2, 40, 32, 2)
    assert e.value.status == m.ERR_ARG
