"""GB300 (sm_103a) Skip-Brute-Force planted (l,d) motif search — Python binding.

Thin ctypes layer over ``libmotif.so``'s C ABI (``include/motif.h``): every function below has
the name of the C entry point it marshals arguments for, and every step of the search runs in
the library's CUDA kernels.  PyTorch is only used, optionally, for device memory (the caching
allocator) and streams.  Importing the package does not load the library; the first call does,
and raises ``MotifLibraryError`` if ``libmotif.so`` has not been built (there is no CPU
fallback).

Method (Perera & Ragel, Sec. III.A): every l-mer is compared with every window of each
sequence by Hamming distance; an l-mer without a window within d in some sequence is discarded
and the remaining sequences are skipped; the l-mers that match all sequences are returned as
ascending 2l-bit codes (A=0 C=1 G=2 T=3, leftmost base most significant).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "MotifError", "MotifLibraryError", "Plan", "motif_opts", "motif_stats_t",
    "motif_server_opts", "motif_opts_default", "motif_plan_create", "motif_plan_destroy",
    "motif_load_seqs", "motif_load_seqs_device", "motif_load_seqs_var", "motif_fasta_parse",
    "read_fasta", "motif_search", "motif_search_device",
    "motif_count_compares", "motif_count_work", "motif_count_tiled_work", "motif_kernel_launches", "motif_stats", "motif_batch_search", "motif_autotune",
    "motif_tune_cache_save", "motif_tune_cache_load", "motif_server_start", "motif_server_stop",
    "motif_submit", "motif_submit_seqs", "motif_poll", "motif_shard_range", "motif_strerror", "motif_encode",
    "motif_decode", "motif_probe_rate", "motif_version", "library_path", "torch_opts",
    "KERNEL_AUTO", "KERNEL_CAND", "KERNEL_GROUP", "KERNEL_TILED", "KERNEL_BITSLICE",
    "OUTPUT_AUTO", "OUTPUT_LIST", "OUTPUT_BITMAP", "SEED_ALL", "SEED_NEIGHBOURHOOD",
    "LAUNCH_GRAPH", "LAUNCH_DIRECT",
    "motif_seed_count", "motif_sort_codes_noalloc",
]

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libmotif.so")
_lock = threading.Lock()
_lib = None

OK, PENDING = 0, 1
ERR_ARG, ERR_ALPHABET, ERR_CAPACITY, ERR_OOM = -1, -2, -3, -4
ERR_CUDA, ERR_TIMEOUT, ERR_BUSY, ERR_STATE, ERR_NOTFOUND = -5, -6, -7, -8, -9
KERNEL_AUTO, KERNEL_CAND, KERNEL_GROUP, KERNEL_TILED, KERNEL_BITSLICE = 0, 1, 2, 3, 4
OUTPUT_AUTO, OUTPUT_LIST, OUTPUT_BITMAP = 0, 1, 2
SEED_ALL, SEED_NEIGHBOURHOOD = 0, 1
LAUNCH_GRAPH, LAUNCH_DIRECT = 0, 1

PROBE_KINDS = ["POPC", "LOP3", "IMNMX", "SHF", "IADD", "IMAD", "POPC_LOP3", "CMP_SPLIT",
               "CMP_FOLD", "LDS64_DIV", "ATOMS_OR", "SHFL"]

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class motif_opts(ctypes.Structure):
    _fields_ = [
        ("stream", ctypes.c_void_p), ("kernel", ctypes.c_int32), ("block", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32), ("cands_per_thread", ctypes.c_int32),
        ("compact_levels", ctypes.c_int32), ("suffix_bases", ctypes.c_int32),
        ("timeout_ms", ctypes.c_int32), ("output", ctypes.c_int32), ("alloc", _ALLOC_FN),
        ("free", _FREE_FN),
        ("alloc_ctx", ctypes.c_void_p), ("range_lo", ctypes.c_uint64),
        ("range_hi", ctypes.c_uint64), ("seed", ctypes.c_int32), ("seq_block", ctypes.c_int32),
        ("launch", ctypes.c_int32),
    ]


class motif_stats_t(ctypes.Structure):
    _fields_ = [
        ("candidates", ctypes.c_uint64), ("survivors", ctypes.c_uint64),
        ("algorithmic_compares", ctypes.c_uint64), ("search_ms", ctypes.c_double),
        ("sort_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
        ("queue_ms", ctypes.c_double), ("device_bytes", ctypes.c_int64),
        ("smem_bytes", ctypes.c_int32), ("kernel", ctypes.c_int32), ("grid", ctypes.c_int32),
        ("block", ctypes.c_int32), ("search_ms_sum", ctypes.c_double),
        ("sort_ms_sum", ctypes.c_double), ("searches", ctypes.c_int64),
    ]


class motif_server_opts(ctypes.Structure):
    _fields_ = [
        ("max_active", ctypes.c_int32), ("max_queued", ctypes.c_int32),
        ("device_budget", ctypes.c_int64), ("step_tiles", ctypes.c_int32),
        ("use_graph", ctypes.c_int32), ("timeout_ms", ctypes.c_int32),
    ]


class MotifLibraryError(RuntimeError):
    """libmotif.so is missing or cannot be loaded (build it with __graft_entry__.build())."""


class MotifError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = motif_strerror(status) if _lib is not None else "status %d" % status
        super().__init__("%s: %s (%d)" % (what or "motif", msg, status))


def library_path() -> str:
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise MotifLibraryError(
                "libmotif.so not found at %s; build it first (python -m paper_1403_1313_gb300.build)"
                % _LIB_PATH)
        try:
            lib = ctypes.CDLL(_LIB_PATH)
        except OSError as e:  # pragma: no cover - surfaced to the caller
            raise MotifLibraryError("cannot load %s: %s" % (_LIB_PATH, e)) from e
        P = ctypes.c_void_p
        i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        sig = {
            "motif_opts_default": (None, [ctypes.POINTER(motif_opts)]),
            "motif_plan_create": (ctypes.c_int, [i32, i32, i32, i32, ctypes.POINTER(motif_opts), ctypes.POINTER(P)]),
            "motif_plan_destroy": (None, [P]),
            "motif_load_seqs": (ctypes.c_int, [P, ctypes.c_char_p, i64]),
            "motif_load_seqs_device": (ctypes.c_int, [P, P, i64]),
            "motif_load_seqs_var": (ctypes.c_int, [P, ctypes.c_char_p, i64,
                                                   ctypes.POINTER(i32), i32]),
            "motif_fasta_parse": (ctypes.c_int, [ctypes.c_char_p, i64, ctypes.c_char_p, i64,
                                                 ctypes.POINTER(i32), i32,
                                                 ctypes.POINTER(i32), i64p]),
            "motif_search": (ctypes.c_int, [P, u64p, i64, i64p]),
            "motif_search_device": (ctypes.c_int, [P, P, i64, P]),
            "motif_count_compares": (ctypes.c_int, [P, u64p]),
            "motif_count_work": (ctypes.c_int, [P, u64p, u64p]),
            "motif_seed_count": (ctypes.c_int, [P, u64p]),
            "motif_sort_codes_noalloc": (ctypes.c_int, [P, i64, i32, P, P]),
            "motif_kernel_launches": (ctypes.c_uint64, []),
            "motif_stats": (ctypes.c_int, [P, ctypes.POINTER(motif_stats_t)]),
            "motif_batch_search": (ctypes.c_int, [i32, ctypes.POINTER(P), ctypes.POINTER(u64p), i64p, i64p, ctypes.POINTER(i32), i32]),
            "motif_autotune": (ctypes.c_int, [P, i32, ctypes.POINTER(motif_opts)]),
            "motif_tune_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
            "motif_tune_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
            "motif_server_start": (ctypes.c_int, [ctypes.POINTER(motif_server_opts)]),
            "motif_server_stop": (ctypes.c_int, []),
            "motif_submit": (ctypes.c_int, [P, i64p]),
            "motif_submit_seqs": (ctypes.c_int, [ctypes.c_char_p, i64, i32, i32, i32, i32,
                                                 ctypes.POINTER(motif_opts), i64p]),
            "motif_poll": (ctypes.c_int, [i64, u64p, i64, i64p, i32, ctypes.POINTER(motif_stats_t)]),
            "motif_shard_range": (ctypes.c_int, [u64, i32, i32, ctypes.POINTER(ctypes.c_double), u64p, u64p]),
            "motif_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "motif_encode": (ctypes.c_int, [ctypes.c_char_p, i32, u64p]),
            "motif_decode": (ctypes.c_int, [u64, i32, ctypes.c_char_p]),
            "motif_count_tiled_work": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_uint64)]),
            "motif_probe_rate": (ctypes.c_int, [i32, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
            "motif_version": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, what: str):
    if status != OK:
        raise MotifError(status, what)


# ---- plans -----------------------------------------------------------------------------------

class Plan:
    """Owns a motif_plan handle (and any Python callbacks its options reference)."""

    def __init__(self, handle, n, t, l, d, opts):
        self.handle = handle
        self.n, self.t, self.l, self.d = n, t, l, d
        self._opts = opts  # keeps allocator callbacks alive
        self.capacity_hint = 1 << 16  # output room for the next search (grows with results)

    def __del__(self):
        try:
            motif_plan_destroy(self)
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        if not self.handle:
            raise MotifError(ERR_STATE, "plan already destroyed")
        return self.handle


def motif_opts_default() -> motif_opts:
    o = motif_opts()
    _load().motif_opts_default(ctypes.byref(o))
    return o


def motif_plan_create(n: int, t: int, l: int, d: int, opts: motif_opts | None = None) -> Plan:
    lib = _load()
    h = ctypes.c_void_p()
    _check(lib.motif_plan_create(n, t, l, d, ctypes.byref(opts) if opts is not None else None,
                                 ctypes.byref(h)), "motif_plan_create")
    return Plan(h.value, n, t, l, d, opts)


def motif_plan_destroy(plan: Plan) -> None:
    if plan.handle:
        _load().motif_plan_destroy(plan.handle)
        plan.handle = None


def _rows(seqs, t=None):
    """(buffer, n, t) for a list of str/bytes rows or an (n, t) uint8 array; an array is passed
    by pointer (the caller keeps the returned array alive through the call)."""
    if isinstance(seqs, np.ndarray):
        a = np.ascontiguousarray(seqs, dtype=np.uint8)
        if a.ndim != 2:
            raise ValueError("expected an (n, t) array of characters")
        return a, a.shape[0], a.shape[1]
    rows = [s.encode() if isinstance(s, str) else bytes(s) for s in seqs]
    if not rows or len({len(r) for r in rows}) != 1:
        raise ValueError("expected n >= 1 rows of one common length")
    return b"".join(rows), len(rows), len(rows[0])


def motif_load_seqs(plan: Plan, seqs) -> None:
    buf, n, t = _rows(seqs)
    if (n, t) != (plan.n, plan.t):
        raise ValueError("sequences are %dx%d, plan expects %dx%d" % (n, t, plan.n, plan.t))
    ptr = buf.ctypes.data_as(ctypes.c_char_p) if isinstance(buf, np.ndarray) else buf
    _check(_load().motif_load_seqs(plan, ptr, t), "motif_load_seqs")


def motif_load_seqs_device(plan: Plan, d_seqs, stride: int | None = None) -> None:
    """d_seqs: a CUDA uint8 torch tensor of shape (n, t) (or a raw device pointer + stride)."""
    if hasattr(d_seqs, "data_ptr"):
        ptr, stride = d_seqs.data_ptr(), d_seqs.stride(0)
    else:
        ptr = int(d_seqs)
    _check(_load().motif_load_seqs_device(plan, ctypes.c_void_p(ptr), stride), "motif_load_seqs_device")


def motif_load_seqs_var(plan: Plan, seqs, mask_unknown: bool = True) -> None:
    """Sequences of their own lengths (str or bytes, each at most the plan's t); with
    mask_unknown a character outside ACGTacgt masks the windows that contain it."""
    rows = [r.encode() if isinstance(r, str) else bytes(r) for r in seqs]
    if len(rows) != plan.n:
        raise ValueError("%d sequences, plan expects %d" % (len(rows), plan.n))
    stride = max(1, plan.t)
    if any(len(r) > stride for r in rows):
        raise ValueError("a sequence is longer than the plan's t = %d" % plan.t)
    buf = b"".join(r.ljust(stride, b"A") for r in rows)
    lens = (ctypes.c_int32 * len(rows))(*[len(r) for r in rows])
    _check(_load().motif_load_seqs_var(plan, buf, stride, lens, 1 if mask_unknown else 0),
           "motif_load_seqs_var")


def motif_fasta_parse(text) -> list:
    """The residues of every record of FASTA text, as a list of bytes (headers dropped)."""
    data = text.encode() if isinstance(text, str) else bytes(text)
    lib = _load()
    n = ctypes.c_int32(0)
    total = ctypes.c_int64(0)
    st = lib.motif_fasta_parse(data, len(data), None, 0, None, 0, ctypes.byref(n),
                               ctypes.byref(total))
    if st not in (OK, ERR_CAPACITY):
        _check(st, "motif_fasta_parse")
    buf = ctypes.create_string_buffer(max(1, total.value))
    lens = (ctypes.c_int32 * max(1, n.value))()
    _check(lib.motif_fasta_parse(data, len(data), buf, total.value, lens, n.value,
                                 ctypes.byref(n), ctypes.byref(total)), "motif_fasta_parse")
    out, at = [], 0
    raw = buf.raw
    for i in range(n.value):
        out.append(raw[at:at + lens[i]])
        at += lens[i]
    return out


def read_fasta(path: str) -> list:
    """motif_fasta_parse of a file's contents."""
    with open(path, "rb") as f:
        return motif_fasta_parse(f.read())


_PINNED = None  # torch, once it is known to have a CUDA device; False where it has none


_PINNED_MIN_CODES = 1 << 17  # 1 MiB: below this a plain array costs less than a pinned block


def _host_codes(capacity: int) -> np.ndarray:
    """An uninitialised host buffer for `capacity` codes (the library writes every returned one).

    Large buffers come from torch's caching pinned-host allocator: the device copy runs at full
    link rate, and a block freed by an earlier result comes back with its pages already mapped.
    A freshly allocated pageable array instead pays the operating system's first touch of every
    page inside the copy (about 8 ms for 195 MB on a GB300 host, against 1 ms into mapped
    memory).  The returned array keeps its block alive; dropping the array gives the block back.
    Small buffers are plain arrays (small results arrive through the library's own pinned
    staging)."""
    global _PINNED
    n = max(int(capacity), 1)
    if n < _PINNED_MIN_CODES:
        return np.empty(n, dtype=np.uint64)
    if _PINNED is None:
        try:
            import torch
            _PINNED = torch if torch.cuda.is_available() else False
        except ImportError:
            _PINNED = False
    if _PINNED:
        return _PINNED.empty(n, dtype=_PINNED.int64, pin_memory=True).numpy().view(np.uint64)
    return np.empty(n, dtype=np.uint64)


def _trimmed(out: np.ndarray, count: int) -> np.ndarray:
    """The first `count` codes; a copy only when that frees most of the buffer."""
    count = int(count)
    return out[:count] if 2 * count >= out.size else out[:count].copy()


def motif_search(plan: Plan, capacity: int | None = None) -> np.ndarray:
    """Blocking search; returns the ascending accepted codes.  The output buffer starts at the
    plan's capacity hint (the size of its previous result) and grows on demand."""
    lib = _load()
    if capacity is None:
        capacity = plan.capacity_hint
    while True:
        out = _host_codes(capacity)
        cnt = ctypes.c_int64(0)
        st = lib.motif_search(plan, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), capacity,
                              ctypes.byref(cnt))
        if st == ERR_CAPACITY:
            capacity = cnt.value
            continue
        _check(st, "motif_search")
        plan.capacity_hint = max(plan.capacity_hint, int(cnt.value))
        return _trimmed(out, cnt.value)


def motif_search_device(plan: Plan, d_out, capacity: int, d_count) -> None:
    """Asynchronous search into device buffers (torch tensors: uint64/int64 codes, one int64)."""
    po = d_out.data_ptr() if hasattr(d_out, "data_ptr") else int(d_out)
    pc = d_count.data_ptr() if hasattr(d_count, "data_ptr") else int(d_count)
    _check(_load().motif_search_device(plan, ctypes.c_void_p(po), capacity, ctypes.c_void_p(pc)),
           "motif_search_device")


def motif_sort_codes_noalloc(d_codes, count: int, key_bits: int, d_unique_count,
                             stream=None) -> None:
    """Sorts `count` device codes ascending and drops repeats in place, without allocating
    device memory; the number of distinct codes goes to d_unique_count (one int64).  Tensors
    (int64/uint64 CUDA) or raw device pointers; stream: a torch stream, a raw handle or None."""
    pc = d_codes.data_ptr() if hasattr(d_codes, "data_ptr") else int(d_codes)
    pu = d_unique_count.data_ptr() if hasattr(d_unique_count, "data_ptr") else int(d_unique_count)
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(_load().motif_sort_codes_noalloc(ctypes.c_void_p(pc), int(count), int(key_bits),
                                            ctypes.c_void_p(pu),
                                            ctypes.c_void_p(s) if s else None),
           "motif_sort_codes_noalloc")


def motif_seed_count(plan: Plan) -> int:
    v = ctypes.c_uint64(0)
    _check(_load().motif_seed_count(plan, ctypes.byref(v)), "motif_seed_count")
    return int(v.value)


def motif_count_compares(plan: Plan) -> int:
    v = ctypes.c_uint64(0)
    _check(_load().motif_count_compares(plan, ctypes.byref(v)), "motif_count_compares")
    return int(v.value)


def motif_count_work(plan: Plan) -> tuple[int, int]:
    """(canonical window compares, canonical unit steps of the plan's kernel formulation)."""
    c, u = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(_load().motif_count_work(plan, ctypes.byref(c), ctypes.byref(u)), "motif_count_work")
    return int(c.value), int(u.value)


TILED_UNITS = ["visits", "windows_filtered", "map_marks", "listed", "scan_rounds",
               "warp_hit_iterations", "lane_hits"]


def motif_count_tiled_work(plan: Plan) -> dict:
    """Work units of the whole-tile tiled pass of one search (names in TILED_UNITS)."""
    u = (ctypes.c_uint64 * len(TILED_UNITS))()
    _check(_load().motif_count_tiled_work(plan, u), "motif_count_tiled_work")
    return dict(zip(TILED_UNITS, (int(x) for x in u)))


def motif_kernel_launches() -> int:
    return int(_load().motif_kernel_launches())


def _stats_dict(s: motif_stats_t) -> dict:
    return {f: getattr(s, f) for f, _ in motif_stats_t._fields_}


def motif_stats(plan: Plan) -> dict:
    s = motif_stats_t()
    _check(_load().motif_stats(plan, ctypes.byref(s)), "motif_stats")
    return _stats_dict(s)


# ---- batching and tuning ---------------------------------------------------------------------

def motif_batch_search(plans, use_graph: bool = True, capacity: int | None = None):
    """Runs loaded plans together in one persistent launch; returns the codes of each job.
    Each job's output buffer starts at its plan's capacity hint (or `capacity`)."""
    lib = _load()
    k = len(plans)
    caps = [capacity if capacity is not None else p.capacity_hint for p in plans]
    while True:
        # one host block for every job's buffer (one allocation, not k); each result is a view
        sizes = [max(int(c), 1) for c in caps]
        block = _host_codes(sum(sizes))
        ends = np.cumsum(sizes)
        outs = [block[e - n:e] for e, n in zip(ends, sizes)]
        handles = (ctypes.c_void_p * k)(*[p.handle for p in plans])
        ptrs = (ctypes.POINTER(ctypes.c_uint64) * k)(
            *[o.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) for o in outs])
        capa = (ctypes.c_int64 * k)(*caps)
        counts = (ctypes.c_int64 * k)()
        stats = (ctypes.c_int32 * k)()
        st = lib.motif_batch_search(k, handles, ptrs, capa, counts, stats, 1 if use_graph else 0)
        retry = [j for j in range(k) if stats[j] == ERR_CAPACITY]
        if retry:
            for j in retry:
                caps[j] = counts[j]
            continue
        _check(st, "motif_batch_search")
        for j, p in enumerate(plans):
            p.capacity_hint = max(p.capacity_hint, int(counts[j]))
        return [_trimmed(outs[j], counts[j]) for j in range(k)]


def motif_autotune(plan: Plan, budget_ms: int = 2000) -> motif_opts:
    best = motif_opts()
    _check(_load().motif_autotune(plan, budget_ms, ctypes.byref(best)), "motif_autotune")
    return best


def motif_tune_cache_save(path: str) -> None:
    _check(_load().motif_tune_cache_save(path.encode()), "motif_tune_cache_save")


def motif_tune_cache_load(path: str) -> None:
    _check(_load().motif_tune_cache_load(path.encode()), "motif_tune_cache_load")


# ---- serving -----------------------------------------------------------------------------------

def motif_server_start(max_active=0, max_queued=0, device_budget=0, step_tiles=0, use_graph=1,
                       timeout_ms=0) -> None:
    o = motif_server_opts(max_active, max_queued, device_budget, step_tiles, use_graph, timeout_ms)
    _check(_load().motif_server_start(ctypes.byref(o)), "motif_server_start")


def motif_server_stop() -> None:
    """Runs every submitted job to completion, then releases the server and the results not yet
    polled.  Call it once no other thread is inside motif_submit or motif_poll."""
    _check(_load().motif_server_stop(), "motif_server_stop")


def motif_submit(plan: Plan) -> int:
    j = ctypes.c_int64(0)
    _check(_load().motif_submit(plan, ctypes.byref(j)), "motif_submit")
    return int(j.value)


def motif_submit_seqs(seqs, l: int, d: int, opts: motif_opts | None = None) -> int:
    """Submits a job from host rows (a list of equal-length str/bytes rows or an (n, t) uint8
    array) without a plan; returns its id for motif_poll."""
    buf, n, t = _rows(seqs)
    ptr = buf.ctypes.data_as(ctypes.c_char_p) if isinstance(buf, np.ndarray) else buf
    j = ctypes.c_int64(0)
    _check(_load().motif_submit_seqs(ptr, t, n, t, l, d,
                                     ctypes.byref(opts) if opts is not None else None,
                                     ctypes.byref(j)), "motif_submit_seqs")
    return int(j.value)


def motif_poll(job_id: int, timeout_ms: int = 0, capacity: int = 1 << 12):
    """Returns (codes, stats dict) when the job is done, or None while it is pending.  The
    first buffer holds `capacity` codes; a larger result is polled again into one of its size
    (the job stays until its codes fit)."""
    lib = _load()
    while True:
        out = _host_codes(capacity)
        cnt = ctypes.c_int64(0)
        s = motif_stats_t()
        st = lib.motif_poll(job_id, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), capacity,
                            ctypes.byref(cnt), timeout_ms, ctypes.byref(s))
        if st == PENDING:
            return None
        if st == ERR_CAPACITY:
            capacity = cnt.value
            continue
        _check(st, "motif_poll")
        return _trimmed(out, cnt.value), _stats_dict(s)


# ---- helpers -------------------------------------------------------------------------------------

def motif_shard_range(total: int, rank: int, world: int, weights=None) -> tuple[int, int]:
    lo, hi = ctypes.c_uint64(0), ctypes.c_uint64(0)
    w = (ctypes.c_double * world)(*weights) if weights is not None else None
    _check(_load().motif_shard_range(total, rank, world, w, ctypes.byref(lo), ctypes.byref(hi)),
           "motif_shard_range")
    return int(lo.value), int(hi.value)


def motif_strerror(status: int) -> str:
    return _load().motif_strerror(status).decode()


def motif_encode(s: str) -> int:
    v = ctypes.c_uint64(0)
    _check(_load().motif_encode(s.encode(), len(s), ctypes.byref(v)), "motif_encode")
    return int(v.value)


def motif_decode(code: int, l: int) -> str:
    buf = ctypes.create_string_buffer(l + 1)
    _check(_load().motif_decode(code, l, buf), "motif_decode")
    return buf.raw[:l].decode()


def motif_probe_rate(kind, iters: int = 4096) -> tuple[float, float]:
    k = PROBE_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    r, c = ctypes.c_double(0), ctypes.c_double(0)
    _check(_load().motif_probe_rate(k, iters, ctypes.byref(r), ctypes.byref(c)), "motif_probe_rate")
    return float(r.value), float(c.value)


def motif_version() -> str:
    return _load().motif_version().decode()


# ---- PyTorch plumbing ----------------------------------------------------------------------------

def torch_opts(stream=None, use_caching_allocator: bool = True, **fields) -> motif_opts:
    """Options that run the plan on a torch CUDA stream and allocate through torch's caching
    allocator.  Extra keyword arguments set motif_opts fields (kernel=..., block=..., ...)."""
    import torch

    o = motif_opts_default()
    s = stream if stream is not None else torch.cuda.current_stream()
    o.stream = ctypes.c_void_p(s.cuda_stream)
    if use_caching_allocator:
        def _alloc(nbytes, strm, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), stream=strm or 0)
            except Exception:
                return None

        def _free(ptr, strm, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        o.alloc = _ALLOC_FN(_alloc)
        o.free = _FREE_FN(_free)
        o._keep = (o.alloc, o.free)
    for k, v in fields.items():
        setattr(o, k, v)
    return o
