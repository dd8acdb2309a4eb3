"""motif_fasta_parse (host-only code in the library): FASTA text to ragged rows.

Records start at lines beginning with '>' (header dropped); the residues of the following lines
are kept in order with whitespace removed; ';' lines are comments.  Runs without a GPU.
"""
import ctypes
import random

import pytest

import paper_1403_1313_gb300 as m


@pytest.fixture(scope="module")
def lib():
    from paper_1403_1313_gb300 import build
    import os
    if not os.path.exists(m.library_path()):
        build.build()
    return m._load()


def _raw(lib, data, buf_cap, max_seqs):
    n = ctypes.c_int32(-1)
    total = ctypes.c_int64(-1)
    buf = ctypes.create_string_buffer(max(1, buf_cap))
    lens = (ctypes.c_int32 * max(1, max_seqs))()
    st = lib.motif_fasta_parse(data, len(data), buf if buf_cap else None, buf_cap,
                               lens if max_seqs else None, max_seqs, ctypes.byref(n),
                               ctypes.byref(total))
    return st, n.value, total.value, buf.raw[:max(0, total.value)], list(lens)[:max(0, n.value)]


def test_records_headers_comments_and_whitespace(lib):
    text = b">s1 first\nACGT\nNNac\n;comment\n>s2 empty\n\n>s3\r\nGG TT\r\n\t a\n"
    assert m.motif_fasta_parse(text) == [b"ACGTNNac", b"", b"GGTTa"]


def test_no_trailing_newline_and_single_record(lib):
    assert m.motif_fasta_parse(b">x\nACG\nT") == [b"ACGT"]
    assert m.motif_fasta_parse(b"") == []
    assert m.motif_fasta_parse(b">only header") == [b""]


def test_residues_before_the_first_header_are_an_error(lib):
    st, *_ = _raw(lib, b"ACGT\n>x\nAC\n", 100, 10)
    assert st == m.ERR_ARG


def test_capacity_protocol(lib):
    data = b">a\nACGT\n>b\nGG\n>c\nTTTTT\n"
    st, n, total, _, _ = _raw(lib, data, 0, 0)
    assert st == m.ERR_CAPACITY and (n, total) == (3, 11)
    st, n, total, _, _ = _raw(lib, data, 11, 2)
    assert st == m.ERR_CAPACITY and (n, total) == (3, 11)
    st, n, total, _, _ = _raw(lib, data, 10, 3)
    assert st == m.ERR_CAPACITY and (n, total) == (3, 11)
    st, n, total, buf, lens = _raw(lib, data, 11, 3)
    assert st == m.OK and buf == b"ACGTGGTTTTT" and lens == [4, 2, 5]


@pytest.mark.parametrize("seed", range(5))
def test_round_trip_of_wrapped_records(lib, seed):
    rng = random.Random(seed)
    seqs = ["".join(rng.choice("ACGTNacgtn") for _ in range(rng.randint(0, 300)))
            for _ in range(rng.randint(1, 20))]
    lines = []
    for i, s in enumerate(seqs):
        lines.append(">seq%d some description" % i)
        w = rng.randint(1, 80)
        lines += [s[k:k + w] for k in range(0, len(s), w)]
    text = ("\r\n" if seed % 2 else "\n").join(lines)
    assert m.motif_fasta_parse(text) == [s.encode() for s in seqs]
