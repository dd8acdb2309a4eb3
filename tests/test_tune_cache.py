"""The tuning cache file, on the host (no device work): entries that parse and keep the option
rules survive a load and a save; damaged entries (an unknown kernel, a block that is not a
multiple of 32 or above 256, a candidate count per lane other than 1, 2 or 4, too many suffix
bases, negative counts, lines that do not parse) are skipped.
"""
import json

import pytest

import paper_1403_1313_gb300 as m


def _entry(kernel=2, block=256, ctas=0, cpt=0, levels=1, ks=4, rate=1.5e9):
    return {"kernel": kernel, "block": block, "ctas_per_sm": ctas, "cands_per_thread": cpt,
            "compact_levels": levels, "suffix_bases": ks, "cand_per_s": rate}


GOOD = {
    "w32_l15_d4_n20_W586_sm152": _entry(kernel=m.KERNEL_TILED),
    "w32_l11_d3_n20_W590_sm152": _entry(kernel=m.KERNEL_GROUP, ctas=2, levels=2, ks=3),
    "w64_l17_d5_n20_W584_sm152": _entry(kernel=m.KERNEL_CAND, cpt=4, ks=0),
    "w32_l9_d2_n20_W592_sm152": _entry(kernel=m.KERNEL_BITSLICE, block=128, cpt=1, ks=0),
}
BAD = {
    "bad_kernel": _entry(kernel=99),
    "bad_kernel_negative": _entry(kernel=-1),
    "bad_block_odd": _entry(block=48),
    "bad_block_big": _entry(block=512),
    "bad_block_negative": _entry(block=-32),
    "bad_cpt": _entry(kernel=m.KERNEL_CAND, cpt=3, ks=0),
    "bad_ks": _entry(ks=5),
    "bad_ctas": _entry(ctas=-1),
    "bad_levels": _entry(levels=-2),
}


def _write(path, entries, extra_lines=()):
    lines = ["{"]
    items = list(entries.items())
    for i, (k, v) in enumerate(items):
        body = ", ".join('"%s": %s' % (f, v[f]) for f in
                         ("kernel", "block", "ctas_per_sm", "cands_per_thread", "compact_levels",
                          "suffix_bases", "cand_per_s"))
        lines.append('  "%s": {%s}%s' % (k, body, "," if i + 1 < len(items) else ""))
    lines[1:1] = list(extra_lines)
    lines.append("}")
    path.write_text("\n".join(lines) + "\n")


def test_load_keeps_valid_entries_and_skips_damaged_ones(tmp_path):
    src = tmp_path / "in.json"
    out = tmp_path / "out.json"
    entries = dict(BAD)
    entries.update(GOOD)
    _write(src, entries, extra_lines=['  "truncated": {"kernel": 2, "block": 256',
                                      "  not json at all"])
    m.motif_tune_cache_load(str(src))
    m.motif_tune_cache_save(str(out))
    saved = json.loads(out.read_text())
    for k, v in GOOD.items():
        assert k in saved
        for f in ("kernel", "block", "ctas_per_sm", "cands_per_thread", "compact_levels",
                  "suffix_bases"):
            assert saved[k][f] == v[f], (k, f)
        assert saved[k]["cand_per_s"] == pytest.approx(v["cand_per_s"], rel=1e-5)
    for k in BAD:
        assert k not in saved
    assert "truncated" not in saved


def test_missing_file_and_null_path(tmp_path):
    with pytest.raises(m.MotifError) as e:
        m.motif_tune_cache_load(str(tmp_path / "does_not_exist.json"))
    assert e.value.status == m.ERR_ARG
    with pytest.raises(m.MotifError) as e:
        m.motif_tune_cache_save(str(tmp_path / "no_such_dir" / "x.json"))
    assert e.value.status == m.ERR_ARG
