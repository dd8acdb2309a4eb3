"""Writes the stored expected results under tests/golden/ from the CPU oracle alone.

Usage: python tests/golden/make_golden.py [l9d2] [l15d4] [l17d5] [--threads N]
                                           [--chunks K --partial-dir DIR]
(default: l9d2).  Each file records the generator's input digest, the accepted codes and the
canonical compare tally of one workload, computed by oracle/ (never by the CUDA path).  The whole
(15,4) space takes about 25 minutes on 8 cores; (17,5), 16 times as many candidates, about seven
hours.  With --chunks the candidate space is searched as K equal index ranges, one after another;
each range's result is kept in DIR as it finishes, and a later run with the same arguments
searches only the ranges that are not there yet, so a long run can be stopped and resumed.
Ranges are disjoint and ascending, so their codes concatenate in order and their tallies add.
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle  # noqa: E402
from paper_1403_1313_gb300 import fmgen  # noqa: E402


def search_chunked(name, job, threads, chunks, partial_dir):
    """The whole space as `chunks` equal ranges, each kept in `partial_dir` once searched."""
    os.makedirs(partial_dir, exist_ok=True)
    total = 4 ** job.l
    digest = hashlib.sha256(job.seqs.tobytes()).hexdigest()
    codes, compares = [], 0
    for k in range(chunks):
        lo, hi = total * k // chunks, total * (k + 1) // chunks
        part = os.path.join(partial_dir, "%s.part%04d-of-%04d.json" % (name, k, chunks))
        rec = None
        if os.path.exists(part):
            with open(part) as f:
                rec = json.load(f)
            if (rec.get("seqs_sha256"), rec.get("lo"), rec.get("hi")) != (digest, lo, hi):
                rec = None
        if rec is None:
            c, m = oracle.search(job.rows(), job.l, job.d, lo=lo, hi=hi, threads=threads)
            rec = {"seqs_sha256": digest, "lo": lo, "hi": hi, "codes": [int(x) for x in c],
                   "compares": int(m)}
            with open(part + ".tmp", "w") as f:
                json.dump(rec, f)
            os.replace(part + ".tmp", part)
            print("%s range %d/%d [%d, %d): %d codes, %d compares" %
                  (name, k + 1, chunks, lo, hi, len(c), m), flush=True)
        codes.extend(rec["codes"])
        compares += rec["compares"]
    return codes, compares


def write(name, job, threads=8, chunks=0, partial_dir=None):
    if chunks:
        codes, compares = search_chunked(name, job, threads, chunks, partial_dir)
    else:
        codes, compares = oracle.search(job.rows(), job.l, job.d, threads=threads)
    rec = {
        "workload": name, "n": job.n, "t": job.t, "l": job.l, "d": job.d, "seed": job.seed,
        "seqs_sha256": hashlib.sha256(job.seqs.tobytes()).hexdigest(),
        "consensus": job.consensus, "codes": [int(c) for c in codes], "compares": int(compares),
        "written_by": "tests/golden/make_golden.py (oracle/ only)",
    }
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(name, len(codes), compares)


NAMES = {"l9d2": "l9d2_n20_t600_seed1", "l15d4": "l15d4_n20_t600_seed2",
         "l17d5": "l17d5_n20_t600_seed3"}

if __name__ == "__main__":
    args = sys.argv[1:]
    threads = os.cpu_count() or 8
    if "--threads" in args:
        i = args.index("--threads")
        threads = int(args[i + 1])
        del args[i:i + 2]
    chunks, partial_dir = 0, None
    if "--chunks" in args:
        i = args.index("--chunks")
        chunks = int(args[i + 1])
        del args[i:i + 2]
        i = args.index("--partial-dir")
        partial_dir = args[i + 1]
        del args[i:i + 2]
    for key in args or ["l9d2"]:
        write(NAMES[key], fmgen.single(key), threads=threads, chunks=chunks,
              partial_dir=partial_dir)
