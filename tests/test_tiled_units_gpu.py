"""Unit counts of the whole-tile tiled pass (motif_count_tiled_work) against a reference that
follows their definitions in motif.h step by step: per tile of 65,536 candidates sharing their
first l - 8 bases, sequences in order until no candidate of the tile is left; per visit the
windows at tile-prefix distance exactly d mark their candidate, those below d are listed (for
l <= 16 a filter lane takes four windows, and the padding slots of the last group repeat the last
window, which is then listed again when it is listed at all), and
every warp of 32 consecutive P2 values (the next 4 bases) with a live candidate scans the list 32
entries per round, a lane hitting an entry when its P2 value lies within min(d - h1, 4) of the
window's.  Candidates matched by a sequence are those within d of one of its windows (the
search's own definition, the oracle's), so the reference also carries the live sets."""
import random

import numpy as np
import pytest

import paper_1403_1313_gb300 as m
from paper_1403_1313_gb300 import fmgen

pytestmark = pytest.mark.gpu

_BASE = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}


def _ham(a, b, k):
    """Hamming distance of two arrays of k-base codes (2 bits per base)."""
    x = np.bitwise_xor(a, b)
    h = np.zeros(np.broadcast(a, b).shape, dtype=np.int64)
    for i in range(k):
        h += ((x >> (2 * i)) & 3) != 0
    return h


def reference_units(seqs, l, d, tiles=None):
    """tiles: the [first, last) tiles of a range that starts and ends on tile boundaries."""
    n, t = seqs.shape
    W = t - l + 1
    codes = np.zeros((n, W), dtype=np.int64)
    for i in range(l):
        codes = codes * 4 + np.vectorize(_BASE.get)(seqs[:, i:i + W]).astype(np.int64)
    pl = l - 8
    u = dict.fromkeys(m.TILED_UNITS, 0)
    p2 = np.arange(256, dtype=np.int64)
    sfx = np.arange(256, dtype=np.int64)
    for tile in range(*(tiles or (0, 4 ** pl))):
        alive = np.ones((256, 256), dtype=bool)  # [P2 value, suffix]
        for s in range(n):
            if not alive.any():
                break
            u["visits"] += 1
            u["windows_filtered"] += W
            w = codes[s]
            if l <= 16:  # four windows per filter lane: the padding slots repeat the last window
                w = np.concatenate([w, np.full(-W % 4, w[-1], dtype=w.dtype)])
            h1 = _ham(w >> 16, tile, pl)
            w2, ws = (w >> 8) & 0xFF, w & 0xFF
            marked = (h1 == d)
            listed = np.nonzero(h1 < d)[0]
            K = listed.size
            u["listed"] += K
            matched = np.zeros((256, 256), dtype=bool)
            mk = np.zeros((256, 256), dtype=bool)
            mk[w2[marked], ws[marked]] = True
            u["map_marks"] += int(mk.sum())
            matched |= mk
            live_lane = alive.any(axis=1)
            if K:
                r1 = d - h1[listed]
                lw2, lws = w2[listed], ws[listed]
                hit = _ham(p2[:, None], lw2[None, :], 4) <= np.minimum(r1, 4)[None, :]  # [lane, entry]
                for warp in range(8):
                    lanes = slice(32 * warp, 32 * warp + 32)
                    if not live_lane[lanes].any():
                        continue
                    for k in range(0, K, 32):
                        u["scan_rounds"] += 1
                        hh = hit[lanes, k:k + 32] & live_lane[lanes, None]
                        per_lane = hh.sum(axis=1)
                        u["warp_hit_iterations"] += int(per_lane.max())
                        u["lane_hits"] += int(per_lane.sum())
                # every candidate within d of a listed window (the whole ball, live lanes or not)
                dist = (h1[listed][None, None, :] + _ham(p2[:, None, None], lw2[None, None, :], 4)
                        + _ham(sfx[None, :, None], lws[None, None, :], 4))
                matched |= (dist <= d).any(axis=2)
            alive &= matched
    return u


@pytest.mark.parametrize("l,d,n,t,seed,tiles", [
    (9, 2, 4, 60, 3, None), (10, 3, 5, 50, 8, None), (10, 1, 6, 80, 21, None),
    (8, 2, 3, 40, 5, None), (9, 4, 3, 30, 13, None), (11, 3, 3, 41, 17, None),
    (12, 2, 3, 38, 29, None), (16, 3, 3, 40, 7, (1000, 1040)),
    (17, 3, 2, 26, 4, (5000, 5100)), (17, 5, 3, 27, 9, (777, 800)),
    (25, 4, 2, 33, 6, (12345, 12360))])  # l > 16: one window per filter lane
def test_tiled_units_match_their_definitions(l, d, n, t, seed, tiles):
    job = fmgen.fm_job(n, t, l, d, seed)
    o = m.motif_opts_default()
    o.kernel = m.KERNEL_TILED
    o.output = m.OUTPUT_LIST
    if tiles:
        o.range_lo, o.range_hi = tiles[0] << 16, tiles[1] << 16
    plan = m.motif_plan_create(n, t, l, d, o)
    m.motif_load_seqs(plan, job.seqs)
    got = m.motif_count_tiled_work(plan)
    codes = m.motif_search(plan)  # the plan still searches normally afterwards
    m.motif_plan_destroy(plan)
    if not tiles:
        assert m.motif_encode(job.consensus) in set(codes.tolist())
    assert got == reference_units(job.seqs, l, d, tiles)


def test_tiled_units_need_a_whole_tile_plan():
    job = fmgen.fm_job(4, 50, 9, 2, 1)
    o = m.motif_opts_default()
    o.kernel = m.KERNEL_CAND
    plan = m.motif_plan_create(4, 50, 9, 2, o)
    m.motif_load_seqs(plan, job.seqs)
    with pytest.raises(m.MotifError) as e:
        m.motif_count_tiled_work(plan)
    assert e.value.status == m.ERR_STATE
    m.motif_plan_destroy(plan)


def test_l15d4_units_fit_the_search():
    """On the (15,4) workload: every tile visits sequence 0, the listed and marked windows are a
    fraction of the filtered ones, and warp iterations never exceed lane hits."""
    job = fmgen.single("l15d4")
    plan = m.motif_plan_create(job.n, job.t, job.l, job.d)
    m.motif_load_seqs(plan, job.seqs)
    u = m.motif_count_tiled_work(plan)
    m.motif_plan_destroy(plan)
    tiles = 4 ** 15 // 65536
    assert tiles * 4 <= u["visits"] <= tiles * job.n
    assert u["windows_filtered"] == u["visits"] * (job.t - job.l + 1)
    assert u["listed"] + u["map_marks"] <= u["windows_filtered"]
    assert u["warp_hit_iterations"] <= u["lane_hits"]
