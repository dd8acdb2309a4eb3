"""Seeded synthetic inputs for planted (l,d) motif search.

This module holds no arithmetic of the search method: it only draws DNA text.  Both the
library's tests/benchmark and the oracle's tests take their inputs from here.

Model (Fixed number of Mutations model, FM; Perera & Ragel Sec. I.B and Sec. IV.B):
  * n background sequences of t bases, each base i.i.d. with P(A)=P(T)=(1-g)/2 and
    P(C)=P(G)=g/2 (g = 0.5 gives the paper's 25 % each);
  * one consensus of l uniform bases per job;
  * per sequence, an instance: d distinct positions of the consensus, each replaced by a
    uniformly chosen *different* base (so the instance is at Hamming distance exactly d);
  * the instance overwrites the sequence at an offset uniform in [0, t-l] (length stays t).

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based generator: draw i of stream s is
mix(seed_s + (i+1) * 0x9E3779B97F4A7C15), which numpy evaluates vectorised and which gives
the same values on every platform.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_ALPHA = np.frombuffer(b"ACGT", dtype=np.uint8)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def draws(seed: int, stream: int, count: int) -> np.ndarray:
    """`count` 64-bit SplitMix64 outputs of sub-stream `stream` of `seed`."""
    with np.errstate(over="ignore"):
        base = _mix(np.array([(seed * 0x2545F4914F6CDD1D + stream) & (2**64 - 1)], dtype=np.uint64))[0]
        ctr = np.arange(1, count + 1, dtype=np.uint64)
        return _mix(base + ctr * _GAMMA)


def _unit(z: np.ndarray) -> np.ndarray:
    """53-bit uniform doubles in [0, 1)."""
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _below(z: np.ndarray, bound) -> np.ndarray:
    """Integers uniform in [0, bound) from the top 32 bits (multiply-shift)."""
    hi = (z >> np.uint64(32)).astype(np.uint64)
    return ((hi * np.asarray(bound, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)


@dataclasses.dataclass
class Job:
    """One planted (l,d) instance set: `seqs` is an (n, t) uint8 array of b'ACGT'."""
    n: int
    t: int
    l: int
    d: int
    seed: int
    gc: float
    seqs: np.ndarray
    consensus: str
    offsets: np.ndarray          # planted offset per sequence (-1 if t < l)
    mutated: np.ndarray          # (n, d) mutated consensus positions per sequence
    arrival_s: float = 0.0       # serving workloads: arrival time

    def rows(self) -> list[str]:
        return [r.tobytes().decode() for r in self.seqs]


def background(n: int, t: int, seed: int, gc: float = 0.5, stream: int = 0) -> np.ndarray:
    """(n, t) i.i.d. bases with GC fraction gc."""
    u = _unit(draws(seed, stream, n * t))
    pa = (1.0 - gc) / 2.0
    pc = gc / 2.0
    idx = (u >= pa).astype(np.uint8) + (u >= pa + pc) + (u >= pa + 2 * pc)
    return _ALPHA[idx].reshape(n, t)


def fm_job(n: int, t: int, l: int, d: int, seed: int, gc: float = 0.5) -> Job:
    """Background plus one FM-planted instance per sequence (exactly d mutations)."""
    if n < 1 or t < 1 or l < 1 or d < 0:
        raise ValueError("need n, t, l >= 1 and d >= 0")
    seqs = background(n, t, seed, gc, stream=0)
    cons_idx = (draws(seed, 1, l) >> np.uint64(62)).astype(np.int64)
    consensus = _ALPHA[cons_idx].tobytes().decode()
    dd = min(d, l)
    offsets = np.full(n, -1, dtype=np.int64)
    mutated = np.zeros((n, dd), dtype=np.int64)
    if t >= l:
        z = draws(seed, 2, n * (1 + 2 * dd))
        zi = 0
        for s in range(n):
            # d distinct positions: partial Fisher-Yates shuffle of 0..l-1.
            perm = list(range(l))
            for i in range(dd):
                j = i + int(_below(z[zi:zi + 1], l - i)[0]); zi += 1
                perm[i], perm[j] = perm[j], perm[i]
            inst = cons_idx.copy()
            for i in range(dd):
                pos = perm[i]
                shift = 1 + int(_below(z[zi:zi + 1], 3)[0]); zi += 1
                inst[pos] = (inst[pos] + shift) % 4      # a uniformly chosen different base
            mutated[s] = perm[:dd]
            off = int(_below(draws(seed, 3 + s, 1), t - l + 1)[0])
            offsets[s] = off
            seqs[s, off:off + l] = _ALPHA[inst]
    return Job(n, t, l, d, seed, gc, seqs, consensus, offsets, mutated)


# ---- the benchmark workloads ------------------------------------------------------------------

# Single jobs: (l, d, n, t, seed).
SINGLE_CONFIGS = {
    "l9d2": (9, 2, 20, 600, 1),
    "l15d4": (15, 4, 20, 600, 2),
    "l17d5": (17, 5, 20, 600, 3),
    "l11d4": (11, 4, 28, 859, 7),
}


def single(name: str) -> Job:
    l, d, n, t, seed = SINGLE_CONFIGS[name]
    return fm_job(n, t, l, d, seed)


def batched_jobs(seed: int = 4, count: int = 64) -> list[Job]:
    """Uneven batch: l ~ U{9..15}, d ~ U{1..4}, n ~ U{5..40}, t ~ U{200..1000}, FM-planted."""
    z = draws(seed, 100, 4 * count)
    jobs = []
    for j in range(count):
        l = 9 + int(_below(z[4 * j:4 * j + 1], 7)[0])
        d = 1 + int(_below(z[4 * j + 1:4 * j + 2], 4)[0])
        n = 5 + int(_below(z[4 * j + 2:4 * j + 3], 36)[0])
        t = 200 + int(_below(z[4 * j + 3:4 * j + 4], 801)[0])
        jobs.append(fm_job(n, t, l, d, seed * 1000003 + j))
    return jobs


def serving_jobs(rate: float, count: int, seed: int = 5) -> list[Job]:
    """Poisson arrivals at `rate` jobs/s: l ~ U{11..15}, d ~ U{2..4}, n ~ U{10..30},
    t ~ U{300..800}, GC fraction from {0.4, 0.5, 0.6}; FM-planted."""
    z = draws(seed, 200 + int(rate * 1000), 6 * count)
    now = 0.0
    jobs = []
    for j in range(count):
        u = float(_unit(z[6 * j:6 * j + 1])[0])
        now += -math.log(1.0 - u) / rate
        l = 11 + int(_below(z[6 * j + 1:6 * j + 2], 5)[0])
        d = 2 + int(_below(z[6 * j + 2:6 * j + 3], 3)[0])
        n = 10 + int(_below(z[6 * j + 3:6 * j + 4], 21)[0])
        t = 300 + int(_below(z[6 * j + 4:6 * j + 5], 501)[0])
        gc = (0.4, 0.5, 0.6)[int(_below(z[6 * j + 5:6 * j + 6], 3)[0])]
        job = fm_job(n, t, l, d, seed * 7919 + j * 31 + int(rate), gc)
        job.arrival_s = now
        jobs.append(job)
    return jobs


def random_text(n: int, t: int, seed: int, gc: float = 0.5) -> list[str]:
    """n unplanted sequences of t bases (list of str)."""
    return [r.tobytes().decode() for r in background(n, t, seed, gc, stream=7)]
