"""motif_sort_codes_noalloc: ordering codes for callers that cannot allocate device memory.

The entry point runs the sort/dedup kernels with scratch taken from a fixed array inside the
library instead of an allocation.  This test calls it through the C ABI on a shuffled, repeated
copy of a search result and checks it against the ascending, duplicate-free codes that
motif_search (which sorts with allocated scratch) returns for the same search; the result is an
integer set, so the comparison is exact.  It makes two calls in a row on each case, because
every call shares the array and inherits the previous call's contents.  The file is named to be
collected last and needs nothing from the other test files, so it runs alone in a fresh process
as well as after them.
"""
import ctypes
import gc

import numpy as np
import pytest

import paper_1403_1313_gb300 as m

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1403_1313_gb300 import build
    build.build()
    h = m._load()
    fn = h.motif_sort_codes_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                   ctypes.c_void_p]
    return h


def _search_result(l, d, n=3, t=20, seed=0):
    """The existing entry point's ascending, duplicate-free codes for an (l, d) search."""
    rng = np.random.default_rng(seed)
    rows = ["".join(rng.choice(list("ACGT"), size=t)) for _ in range(n)]
    plan = m.motif_plan_create(n, t, l, d)
    m.motif_load_seqs(plan, rows)
    codes = m.motif_search(plan)
    m.motif_plan_destroy(plan)
    return codes


@pytest.mark.parametrize("l,d,repeat", [(5, 5, 2), (7, 7, 3), (8, 2, 2), (9, 9, 1)])
def test_noalloc_sort_matches_search(lib, l, d, repeat):
    torch = pytest.importorskip("torch")
    ref = _search_result(l, d, seed=l * 10 + d)
    assert ref.size > 0
    rng = np.random.default_rng(l)
    for call in range(2):
        # A shuffled input holding every code `repeat` times.
        mixed = np.concatenate([ref] * repeat)
        rng.shuffle(mixed)
        d_codes = torch.from_numpy(mixed.astype(np.int64)).cuda()
        d_count = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        st = lib.motif_sort_codes_noalloc(d_codes.data_ptr(), mixed.size, 2 * l,
                                          d_count.data_ptr(), stream)
        assert st == m.OK, m.motif_strerror(st)
        torch.cuda.synchronize()
        cnt = int(d_count.item())
        assert cnt == ref.size, (call, cnt, ref.size)
        got = d_codes[:cnt].cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, ref), call


def test_noalloc_sort_rejects_too_many_codes(lib):
    # Checked on the host before any device work: nothing is launched or written.
    # (The pointers are placeholders that the rejected calls never dereference.)
    fake = ctypes.c_void_p(256)
    st = lib.motif_sort_codes_noalloc(fake, (1 << 18) + 1, 30, fake, None)
    assert st == m.ERR_CAPACITY
    st = lib.motif_sort_codes_noalloc(fake, 5, 0, fake, None)
    assert st == m.ERR_ARG
    st = lib.motif_sort_codes_noalloc(fake, -1, 30, fake, None)
    assert st == m.ERR_ARG


def test_noalloc_sort_through_the_binding(lib):
    torch = pytest.importorskip("torch")
    ref = _search_result(8, 3, seed=5)
    mixed = np.concatenate([ref, ref[::-1]])
    d_codes = torch.from_numpy(mixed.astype(np.int64)).cuda()
    d_count = torch.zeros(1, dtype=torch.int64, device="cuda")
    m.motif_sort_codes_noalloc(d_codes, mixed.size, 16, d_count, torch.cuda.current_stream())
    torch.cuda.synchronize()
    cnt = int(d_count.item())
    assert cnt == ref.size
    assert np.array_equal(d_codes[:cnt].cpu().numpy().astype(np.uint64), ref)
    with pytest.raises(m.MotifError) as e:  # rejected on the host, nothing launched
        m.motif_sort_codes_noalloc(256, 5, 0, 256)
    assert e.value.status == m.ERR_ARG


def test_noalloc_sort_allocates_nothing(lib):
    """After a first call (which loads the kernels and looks up the array), further calls leave
    the device's free memory exactly where it was and take nothing from torch's allocator."""
    torch = pytest.importorskip("torch")
    ref = _search_result(8, 2, seed=7)
    mixed = np.concatenate([ref, ref])
    host = torch.from_numpy(mixed.astype(np.int64))
    d_codes = host.cuda()
    d_count = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        d_codes.copy_(host)
        st = lib.motif_sort_codes_noalloc(d_codes.data_ptr(), mixed.size, 16,
                                          d_count.data_ptr(), stream)
        assert st == m.OK, m.motif_strerror(st)
        torch.cuda.synchronize()

    call()
    gc.collect()  # tensors left by earlier tests go back to torch's cache before the baseline
    free0, torch0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):
        call()
        assert int(d_count.item()) == ref.size
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() <= torch0
    assert np.array_equal(d_codes[:ref.size].cpu().numpy().astype(np.uint64), ref)
