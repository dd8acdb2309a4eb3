"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

The result is an exact integer set, so the bar is bit-exact equality of the ascending code
lists (and of the canonical compare tally where it is counted).  Small cases run the oracle over
the whole candidate space and span many tiles, ragged window rows, partial groups and partial
tiles; the full-size workloads are checked on sampled candidate sub-ranges the oracle computes
directly, plus properties that hold at any size (the planted consensus is accepted, every
accepted code is accepted by the oracle one by one, the kernels agree with each other).
"""
import hashlib
import json
import os
import random

import numpy as np
import pytest

import paper_1403_1313_gb300 as m
from oracle import oracle
from paper_1403_1313_gb300 import fmgen

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

VARIANTS = [
    ("tiled", dict(kernel=m.KERNEL_TILED)),
    ("group4", dict(kernel=m.KERNEL_GROUP, suffix_bases=4)),
    ("group3", dict(kernel=m.KERNEL_GROUP, suffix_bases=3)),
    ("group2", dict(kernel=m.KERNEL_GROUP, suffix_bases=2)),
    ("group1", dict(kernel=m.KERNEL_GROUP, suffix_bases=1)),
    ("cand1", dict(kernel=m.KERNEL_CAND, cands_per_thread=1)),
    ("cand2", dict(kernel=m.KERNEL_CAND, cands_per_thread=2)),
    ("cand4", dict(kernel=m.KERNEL_CAND, cands_per_thread=4)),
    ("bitslice1", dict(kernel=m.KERNEL_BITSLICE, cands_per_thread=1)),
    ("bitslice2", dict(kernel=m.KERNEL_BITSLICE, cands_per_thread=2)),
    ("bitslice4", dict(kernel=m.KERNEL_BITSLICE, cands_per_thread=4)),
]


def _opts(**kw):
    o = m.motif_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def gpu_search(seqs, l, d, lo=0, hi=None, **kw):
    rows = [s.encode() if isinstance(s, str) else s for s in seqs] if not isinstance(seqs, np.ndarray) else seqs
    n = len(rows)
    t = rows.shape[1] if isinstance(rows, np.ndarray) else len(rows[0])
    if hi is not None or lo:
        kw["range_lo"] = lo
        kw["range_hi"] = hi if hi is not None else 4 ** l
    plan = m.motif_plan_create(n, t, l, d, _opts(**kw))
    m.motif_load_seqs(plan, seqs)
    codes = m.motif_search(plan)
    cmp = m.motif_count_compares(plan)
    m.motif_plan_destroy(plan)
    return codes, cmp


def rand_rows(rng, n, t):
    return ["".join(rng.choice("ACGT") for _ in range(t)) for _ in range(n)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1403_1313_gb300 import build
    build.build()
    oracle.build()


# ---- small cases: whole candidate space ---------------------------------------------------------

@pytest.mark.parametrize("name,kw", VARIANTS, ids=[v[0] for v in VARIANTS])
@pytest.mark.parametrize("seed", range(12))
def test_small_random(name, kw, seed):
    rng = random.Random(seed * 7919 + len(name))
    l = rng.randint(2, 8)
    d = rng.randint(0, min(l, 3))
    n = rng.randint(1, 7)
    t = rng.randint(max(1, l - 2), 70)
    rows = rand_rows(rng, n, t)
    ref, ref_cmp = oracle.search(rows, l, d)
    got, cmp = gpu_search(rows, l, d, **kw)
    assert np.array_equal(got, ref)
    assert cmp == ref_cmp


@pytest.mark.parametrize("name,kw", VARIANTS, ids=[v[0] for v in VARIANTS])
@pytest.mark.parametrize("l,d,n,t,seed", [(9, 2, 6, 100, 21), (10, 3, 5, 150, 22), (11, 3, 4, 90, 23)])
def test_fm_planted(name, kw, l, d, n, t, seed):
    job = fmgen.fm_job(n, t, l, d, seed)
    ref, ref_cmp = oracle.search(job.rows(), l, d, threads=8)
    got, cmp = gpu_search(job.seqs, l, d, **kw)
    assert np.array_equal(got, ref)
    assert m.motif_encode(job.consensus) in set(got.tolist())
    assert cmp == ref_cmp


@pytest.mark.parametrize("name,kw", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_unaligned_subranges(name, kw):
    job = fmgen.fm_job(6, 80, 9, 2, 31)
    rng = random.Random(5)
    for _ in range(4):
        lo = rng.randrange(0, 4 ** 9 - 1)
        hi = rng.randrange(lo + 1, min(4 ** 9, lo + 40000) + 1)
        ref, ref_cmp = oracle.search(job.rows(), 9, 2, lo=lo, hi=hi)
        got, cmp = gpu_search(job.seqs, 9, 2, lo=lo, hi=hi, **kw)
        assert np.array_equal(got, ref), (lo, hi)
        assert cmp == ref_cmp


@pytest.mark.parametrize("l,d", [(8, 1), (9, 2), (10, 3), (12, 4)])
def test_tiled_aligned_and_partial_ranges(l, d):
    """The prefix-tiled pass: ranges starting on a tile boundary (multiples of 4^8 candidates)
    with ragged ends, small sequence counts, and windows near the 16-bit index limit."""
    job = fmgen.fm_job(4, 70, l, d, 300 + l)
    rng = random.Random(l * 31 + d)
    tile = 4 ** 8
    for _ in range(3):
        lo = tile * rng.randrange(0, max(1, 4 ** l // tile))
        hi = min(4 ** l, lo + rng.randrange(1, 3 * tile))
        ref, ref_cmp = oracle.search(job.rows(), l, d, lo=lo, hi=hi)
        got, cmp = gpu_search(job.seqs, l, d, lo=lo, hi=hi, kernel=m.KERNEL_TILED)
        assert np.array_equal(got, ref), (lo, hi)
        assert cmp == ref_cmp


@pytest.mark.parametrize("l,d,n,t", [(8, 8, 2, 9), (9, 4, 3, 40), (11, 6, 2, 30)])
def test_tiled_every_window_listed(l, d, n, t):
    """d at or above the shared-prefix length: every window enters the filtered list."""
    rows = rand_rows(random.Random(l + d), n, t)
    ref, ref_cmp = oracle.search(rows, l, d, threads=8)
    got, cmp = gpu_search(rows, l, d, kernel=m.KERNEL_TILED)
    assert np.array_equal(got, ref)
    assert cmp == ref_cmp


@pytest.mark.parametrize("l,d,t", [(16, 5, 17), (16, 5, 1043), (16, 2, 1046), (16, 8, 40),
                                   (17, 5, 1045), (17, 6, 19), (13, 4, 1042)])
def test_tiled_prefix_filter_edges(l, d, t):
    """The tiled pass's prefix filter: l = 16 (the longest prefix it compares four windows per
    lane, a whole byte per window) and l = 17 (one window per lane); rows of 2 and 3 windows and
    of just over 1024 (a second trip of the four-window loop), with every remainder mod 4; d at
    the prefix length (every window passes).  Ranges: the two tiles from the planted
    consensus's tile, and two tiles from a random tile."""
    job = fmgen.fm_job(3, t, l, d, 400 + 8 * l + d)
    tile = 4 ** 8
    cons = m.motif_encode(job.consensus)
    rng = random.Random(t)
    for lo in (cons // tile * tile, tile * rng.randrange(4 ** l // tile)):
        hi = min(4 ** l, lo + 2 * tile)
        ref, ref_cmp = oracle.search(job.rows(), l, d, lo=lo, hi=hi, threads=8)
        plan = m.motif_plan_create(3, t, l, d, _opts(kernel=m.KERNEL_TILED, range_lo=lo,
                                                     range_hi=hi))
        m.motif_load_seqs(plan, job.seqs)
        got = m.motif_search(plan)
        assert m.motif_stats(plan)["kernel"] == m.KERNEL_TILED
        cmp = m.motif_count_compares(plan)
        m.motif_plan_destroy(plan)
        assert np.array_equal(got, ref), (lo, hi)
        assert cmp == ref_cmp
        if lo == cons // tile * tile:
            assert cons in set(ref.tolist())  # the planted consensus lies in the range


# ---- edge cases ---------------------------------------------------------------------------------

@pytest.mark.parametrize("name,kw", VARIANTS, ids=[v[0] for v in VARIANTS])
@pytest.mark.parametrize("l,d", [(6, 6), (7, 9), (9, 9)])
def test_everything_survives(name, kw, l, d):
    """d >= l: all 4^l codes; exercises the output growth and both sort paths (4096 codes,
    16384 codes, 262144 codes > the initial 65536-code buffer)."""
    rows = rand_rows(random.Random(l), 3, 20)
    got, cmp = gpu_search(rows, l, d, **kw)
    assert np.array_equal(got, np.arange(4 ** l, dtype=np.uint64))
    assert cmp == 4 ** l * 3


@pytest.mark.parametrize("name,kw", VARIANTS[:2] + VARIANTS[5:6], ids=["tiled", "group4", "cand1"])
def test_no_windows_and_single_windows(name, kw):
    rows = rand_rows(random.Random(3), 4, 5)
    got, cmp = gpu_search(rows, 6, 6, **kw)          # t < l: nothing can match
    assert got.size == 0 and cmp == 0
    rows = ["ACGTAC", "ACGTAA", "ACGTAG"]              # t == l: one window per sequence
    ref, ref_cmp = oracle.search(rows, 6, 1)
    got, cmp = gpu_search(rows, 6, 1, **kw)
    assert np.array_equal(got, ref) and cmp == ref_cmp


def test_lowercase_equals_uppercase():
    job = fmgen.fm_job(5, 60, 8, 2, 41)
    up, _ = gpu_search(job.rows(), 8, 2)
    low, _ = gpu_search([r.lower() for r in job.rows()], 8, 2)
    assert np.array_equal(up, low)


def test_bad_alphabet_is_reported():
    plan = m.motif_plan_create(2, 10, 4, 1)
    with pytest.raises(m.MotifError) as e:
        m.motif_load_seqs(plan, ["ACGTACGTAC", "ACGTNCGTAC"])
    assert e.value.status == m.ERR_ALPHABET
    with pytest.raises(m.MotifError) as e:
        m.motif_search(plan)
    assert e.value.status == m.ERR_STATE


def test_capacity_protocol():
    rows = rand_rows(random.Random(9), 2, 12)
    plan = m.motif_plan_create(2, 12, 5, 5)
    m.motif_load_seqs(plan, rows)
    import ctypes
    out = np.zeros(10, dtype=np.uint64)
    cnt = ctypes.c_int64(0)
    st = m._load().motif_search(plan, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), 10,
                                ctypes.byref(cnt))
    assert st == m.ERR_CAPACITY and cnt.value == 4 ** 5


# ---- the (9,2) workload: whole space against the stored oracle result --------------------------

@pytest.mark.parametrize("name,kw", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_l9d2_full(name, kw):
    with open(os.path.join(GOLDEN, "l9d2_n20_t600_seed1.json")) as f:
        g = json.load(f)
    job = fmgen.single("l9d2")
    got, cmp = gpu_search(job.seqs, 9, 2, **kw)
    assert got.tolist() == g["codes"]
    assert cmp == g["compares"]


# ---- device-resident path -------------------------------------------------------------------------

def test_device_path_matches_blocking_path():
    torch = pytest.importorskip("torch")
    job = fmgen.fm_job(10, 200, 10, 3, 51)
    ref, _ = oracle.search(job.rows(), 10, 3, threads=8)
    plan = m.motif_plan_create(10, 200, 10, 3, m.torch_opts())
    chars = torch.from_numpy(job.seqs.copy()).cuda()
    m.motif_load_seqs_device(plan, chars)
    out = torch.zeros(1 << 16, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(2):
        m.motif_search_device(plan, out, out.numel(), cnt)
        torch.cuda.synchronize()
        c = int(cnt.item())
        assert c == ref.size
        assert np.array_equal(out[:c].cpu().numpy().astype(np.uint64), ref)


# ---- full-size workloads: sampled parity ---------------------------------------------------------

TILE = 1 << 16  # candidates of one tile of the prefix-tiled pass (256 groups of 256 suffixes)


def _sample_ranges(l, consensus_code, seed, count=6, tiles=3):
    """Sub-ranges that start on a tile boundary and span several whole tiles (so that the
    default plan of each runs the tiled pass, as the whole-space search does), the first one
    holding the consensus's tile."""
    rng = random.Random(seed)
    ntiles = 4 ** l // TILE
    first = max(0, min(ntiles - tiles, consensus_code // TILE - tiles // 2))
    starts = [first]
    while len(starts) < count:
        t = rng.randrange(0, ntiles - tiles + 1)
        if all(abs(t - u) >= tiles for u in starts):
            starts.append(t)
    return [(t * TILE, (t + tiles) * TILE) for t in starts]


@pytest.mark.parametrize("cfg", ["l15d4", "l17d5"])
def test_full_size_sampled(cfg):
    job = fmgen.single(cfg)
    l, d = job.l, job.d
    cons = m.motif_encode(job.consensus)
    # Whole space with the default (benchmark) configuration.
    plan = m.motif_plan_create(job.n, job.t, l, d)
    m.motif_load_seqs(plan, job.seqs)
    full = m.motif_search(plan)
    m.motif_plan_destroy(plan)
    assert cons in set(full.tolist())
    # Every accepted code is accepted by the oracle on its own.
    for c in full.tolist():
        ref, _ = oracle.search(job.rows(), l, d, lo=c, hi=c + 1)
        assert ref.tolist() == [c]
    # Sampled sub-ranges: the oracle over each range, the GPU over the same range, and the
    # whole-space GPU result restricted to it.
    ranges = _sample_ranges(l, cons, seed=l * 100 + d)
    assert ranges[0][0] <= cons < ranges[0][1]
    for lo, hi in ranges:
        assert lo % TILE == 0 and hi - lo >= 2 * TILE
        ref, ref_cmp = oracle.search(job.rows(), l, d, lo=lo, hi=hi, threads=os.cpu_count() or 8)
        plan = m.motif_plan_create(job.n, job.t, l, d, _opts(range_lo=lo, range_hi=hi))
        m.motif_load_seqs(plan, job.seqs)
        sub = m.motif_search(plan)
        assert m.motif_stats(plan)["kernel"] == m.KERNEL_TILED, (lo, hi)
        cmp = m.motif_count_compares(plan)
        m.motif_plan_destroy(plan)
        assert np.array_equal(sub, ref), (lo, hi)
        assert cmp == ref_cmp
        inside = full[(full >= lo) & (full < hi)]
        assert np.array_equal(inside, ref)


FULL_GOLDEN = {"l15d4": "l15d4_n20_t600_seed2.json", "l17d5": "l17d5_n20_t600_seed3.json"}


@pytest.mark.parametrize("form", ["auto", "device", "bitslice_seeded"])
@pytest.mark.parametrize("cfg", sorted(FULL_GOLDEN))
def test_full_space_matches_stored_oracle(cfg, form):
    """The whole code space of the (15,4) and (17,5) workloads against the oracle's complete
    results (tests/golden/, written by make_golden.py from oracle/ alone): every code, none
    missing, and the canonical compare tally."""
    path = os.path.join(GOLDEN, FULL_GOLDEN[cfg])
    if not os.path.exists(path):
        pytest.skip("no stored oracle result for %s (tests/golden/make_golden.py %s)" % (cfg, cfg))
    with open(path) as f:
        g = json.load(f)
    job = fmgen.single(cfg)
    assert hashlib.sha256(job.seqs.tobytes()).hexdigest() == g["seqs_sha256"]
    if form == "device":  # the benchmark's launch configuration
        torch = pytest.importorskip("torch")
        plan = m.motif_plan_create(job.n, job.t, job.l, job.d, m.torch_opts())
        m.motif_load_seqs_device(plan, torch.from_numpy(job.seqs.copy()).cuda())
        out = torch.zeros(1 << 16, dtype=torch.int64, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        m.motif_search_device(plan, out, out.numel(), cnt)
        torch.cuda.synchronize()
        c = int(cnt.item())
        got = out[:c].cpu().numpy().astype(np.uint64)
    else:
        kw = dict(kernel=m.KERNEL_BITSLICE, seed=m.SEED_NEIGHBOURHOOD) if form != "auto" else {}
        plan = m.motif_plan_create(job.n, job.t, job.l, job.d, _opts(**kw))
        m.motif_load_seqs(plan, job.seqs)
        got = m.motif_search(plan)
    assert got.tolist() == g["codes"]
    if form == "auto":
        assert m.motif_count_compares(plan) == g["compares"]
    m.motif_plan_destroy(plan)


def test_l15d4_kernels_agree():
    job = fmgen.single("l15d4")
    res = []
    for kw in (dict(kernel=m.KERNEL_TILED), dict(kernel=m.KERNEL_GROUP, suffix_bases=4),
               dict(kernel=m.KERNEL_GROUP, suffix_bases=3), dict(kernel=m.KERNEL_CAND, cands_per_thread=2)):
        plan = m.motif_plan_create(job.n, job.t, 15, 4, _opts(**kw))
        m.motif_load_seqs(plan, job.seqs)
        res.append(m.motif_search(plan))
        m.motif_plan_destroy(plan)
    assert all(np.array_equal(res[0], r) for r in res[1:])


# ---- batching -------------------------------------------------------------------------------------

@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_oracle(use_graph):
    rng = random.Random(61)
    jobs, plans = [], []
    for j in range(10):
        l = rng.randint(6, 10)
        d = rng.randint(1, 3)
        n = rng.randint(2, 8)
        t = rng.randint(l, 160)
        job = fmgen.fm_job(n, t, l, d, 700 + j)
        plan = m.motif_plan_create(n, t, l, d)
        m.motif_load_seqs(plan, job.seqs)
        jobs.append(job)
        plans.append(plan)
    outs = m.motif_batch_search(plans, use_graph=use_graph)
    for job, got in zip(jobs, outs):
        ref, _ = oracle.search(job.rows(), job.l, job.d)
        assert np.array_equal(got, ref)


def _closed_form_compares(job):
    """Expected canonical compares of a uniform-base job (the oracle's cost estimate)."""
    import math
    p = sum(math.comb(job.l, k) * 3 ** k for k in range(min(job.d, job.l) + 1)) / 4 ** job.l
    q = 1 - (1 - p) ** (job.t - job.l + 1)
    per = (q / p) * (1 - q ** job.n) / (1 - q) if q < 1 else (job.t - job.l + 1) * job.n
    return 4 ** job.l * per


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_64_job_mix(use_graph):
    """The 64-job batch mix (seed 4: l 9..15, d 1..4, n 5..40, t 200..1000) in one batched
    search: the jobs the oracle finishes within about 2e10 compares (the 20 cheapest: l <= 12)
    equal the oracle's results, and every job equals its own one-job search."""
    jobs = fmgen.batched_jobs(seed=4, count=64)
    plans = []
    for j in jobs:
        plan = m.motif_plan_create(j.n, j.t, j.l, j.d)
        m.motif_load_seqs(plan, j.seqs)
        plans.append(plan)
    outs = m.motif_batch_search(plans, use_graph=use_graph)
    order = sorted(range(len(jobs)), key=lambda i: _closed_form_compares(jobs[i]))
    budget, checked = 2e10, 0
    for i in order:
        budget -= _closed_form_compares(jobs[i])
        if budget < 0:
            break
        ref, _ = oracle.search(jobs[i].rows(), jobs[i].l, jobs[i].d, threads=os.cpu_count() or 8)
        assert np.array_equal(outs[i], ref), (jobs[i].l, jobs[i].d, jobs[i].n, jobs[i].t)
        checked += 1
    assert checked >= 15
    for job, plan, got in zip(jobs, plans, outs):
        assert np.array_equal(got, m.motif_search(plan)), (job.l, job.d, job.n, job.t)
        assert m.motif_encode(job.consensus) in set(got.tolist())
        m.motif_plan_destroy(plan)


@pytest.mark.parametrize("l,d", [(9, 8), (12, 9)])
def test_bitslice_beyond_its_counter_falls_back_to_cand(l, d):
    """The bit-sliced counter holds distances up to 7; larger d runs the POPC compare."""
    rows = rand_rows(random.Random(l * d), 3, 25)
    plan = m.motif_plan_create(3, 25, l, d, _opts(kernel=m.KERNEL_BITSLICE))
    m.motif_load_seqs(plan, rows)
    got = m.motif_search(plan)
    assert m.motif_stats(plan)["kernel"] == m.KERNEL_CAND
    m.motif_plan_destroy(plan)
    ref, _ = oracle.search(rows, l, d)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("name,kw", VARIANTS[:1] + VARIANTS[1:2] + VARIANTS[5:6] + VARIANTS[8:9],
                         ids=["tiled", "group4", "cand1", "bitslice1"])
@pytest.mark.parametrize("output", [m.OUTPUT_LIST, m.OUTPUT_BITMAP])
def test_direct_launch_equals_oracle(name, kw, output):
    """The step kernel launched from the host once per step (MOTIF_LAUNCH_DIRECT, the form
    profilers list) gives the oracle's result, through the blocking and the device path."""
    torch = pytest.importorskip("torch")
    job = fmgen.fm_job(6, 120, 10, 2, 314)
    ref, _ = oracle.search(job.rows(), job.l, job.d)
    plan = m.motif_plan_create(job.n, job.t, job.l, job.d,
                               m.torch_opts(launch=m.LAUNCH_DIRECT, output=output, **kw))
    m.motif_load_seqs(plan, job.seqs)
    assert np.array_equal(m.motif_search(plan), ref)
    out = torch.zeros(1 << 14, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    m.motif_search_device(plan, out, out.numel(), cnt)
    torch.cuda.synchronize()
    c = int(cnt.item())
    assert np.array_equal(out[:c].cpu().numpy().astype(np.uint64), ref)
    m.motif_plan_destroy(plan)


def test_launch_option_is_checked():
    o = m.motif_opts_default()
    o.launch = 7
    with pytest.raises(m.MotifError) as e:
        m.motif_plan_create(2, 20, 8, 1, o)
    assert e.value.status == m.ERR_ARG
