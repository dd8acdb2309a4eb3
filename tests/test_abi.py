"""The C ABI on the host: the library loads, exports every symbol include/motif.h declares,
and its host-only helpers behave (no compute calls; no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_1403_1313_gb300 as m

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "motif.h")


def _header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(motif_[a-z0-9_]+)\s*\(",
                           src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(m.library_path()):
        from paper_1403_1313_gb300 import build
        build.build()
    return ctypes.CDLL(m.library_path())


def test_every_declared_symbol_is_exported(lib):
    names = _header_functions()
    expected = {"opts_default", "plan_create", "plan_destroy", "load_seqs", "load_seqs_device",
                "search", "search_device", "count_compares", "stats", "batch_search", "autotune",
                "tune_cache_save", "tune_cache_load", "server_start", "server_stop", "submit",
                "poll", "shard_range", "strerror", "encode", "decode", "probe_rate", "version",
                "count_work", "kernel_launches", "load_seqs_var", "fasta_parse",
                "sort_codes_noalloc", "seed_count"}
    assert set(names) >= {"motif_" + e for e in expected}, sorted(set(names))
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_codes_match_header(lib):
    src = open(HEADER).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"(MOTIF_(?:OK|PENDING|ERR_[A-Z]+))\s*=\s*(-?\d+)", src))
    assert codes["MOTIF_ERR_CAPACITY"] == m.ERR_CAPACITY
    assert codes["MOTIF_ERR_ALPHABET"] == m.ERR_ALPHABET
    assert codes["MOTIF_PENDING"] == m.PENDING
    for name, val in codes.items():
        assert m.motif_strerror(val) not in ("", "unknown status"), name


def test_struct_sizes_match_c_layout():
    # motif_opts: pointer, 8 int32, 2 fn pointers, ctx pointer, 2 uint64, 3 int32 (+ padding).
    assert ctypes.sizeof(m.motif_opts) == 8 + 8 * 4 + 3 * 8 + 2 * 8 + 3 * 4 + 4
    assert ctypes.sizeof(m.motif_stats_t) == 3 * 8 + 4 * 8 + 8 + 4 * 4 + 3 * 8


def test_struct_offsets_match_the_header(tmp_path):
    """Every field of the binding's structs sits at the offset the C compiler gives it."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "motif.h"', "int main(void) {"]
    for cname, py in (("motif_opts", m.motif_opts), ("motif_stats_t", m.motif_stats_t),
                      ("motif_server_opts", m.motif_server_opts)):
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f[0], cname, f[0]))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), "-o", str(exe), str(src)])
    got = {}
    for ln in subprocess.check_output([str(exe)], text=True).splitlines():
        a, b, c = ln.split()
        got[(a, b)] = int(c)
    for cname, py in (("motif_opts", m.motif_opts), ("motif_stats_t", m.motif_stats_t),
                      ("motif_server_opts", m.motif_server_opts)):
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])


def test_encode_decode_roundtrip():
    for s in ["A", "ACGT", "TTTT", "GATTACA", "ACGTACGTACGTACG", "T" * 31]:
        c = m.motif_encode(s)
        assert m.motif_decode(c, len(s)) == s
        assert c == int(s.translate(str.maketrans("ACGT", "0123")), 4)
    assert m.motif_encode("acgt") == m.motif_encode("ACGT")
    with pytest.raises(m.MotifError) as e:
        m.motif_encode("ACGN")
    assert e.value.status == m.ERR_ALPHABET
    with pytest.raises(m.MotifError):
        m.motif_decode(1 << 10, 4)  # more than 2l bits
    for bad in (lambda: m.motif_encode("A" * 32), lambda: m.motif_encode(""),
                lambda: m.motif_decode(0, 32), lambda: m.motif_decode(0, 0)):
        with pytest.raises(m.MotifError) as e:  # l outside [1, 31]
            bad()
        assert e.value.status == m.ERR_ARG


@pytest.mark.parametrize("world", [1, 2, 3, 7])
def test_shard_ranges_tile_the_space(world):
    total = 4 ** 9 + 5
    ranges = [m.motif_shard_range(total, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == total
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c and a <= b
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_weighted_shards():
    lo, hi = m.motif_shard_range(1000, 1, 2, weights=[1.0, 3.0])
    assert (lo, hi) == (250, 1000)
    with pytest.raises(m.MotifError):
        m.motif_shard_range(10, 2, 2)


def test_plan_create_rejects_bad_arguments():
    # Argument validation happens before any device call.
    for args in [(0, 10, 3, 1), (2, 0, 3, 1), (2, 10, 0, 1), (2, 10, 32, 1), (2, 10, 3, -1)]:
        with pytest.raises(m.MotifError) as e:
            m.motif_plan_create(*args)
        assert e.value.status == m.ERR_ARG


def test_version_names_the_target():
    assert "sm_103a" in m.motif_version()


def test_every_declared_symbol_has_a_binding_of_its_name():
    """The Python binding marshals arguments for every entry point, under the same name."""
    missing = [n for n in _header_functions() if not callable(getattr(m, n, None))]
    assert not missing, missing
    assert set(_header_functions()) <= set(m.__all__)
