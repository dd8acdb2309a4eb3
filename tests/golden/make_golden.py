"""Writes the stored expected results under tests/golden/ from the CPU oracle alone.

Usage: python tests/golden/make_golden.py [l9d2] [l15d4] [l17d5] [--threads N]
(default: l9d2).  Each file records the generator's input digest, the accepted codes and the
canonical compare tally of one workload, computed by oracle/ (never by the CUDA path).  The whole
(15,4) space takes a few minutes on 8 cores; (17,5), 16 times as many candidates, about an hour
or two.
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle  # noqa: E402
from paper_1403_1313_gb300 import fmgen  # noqa: E402


def write(name, job, threads=8):
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
    for key in args or ["l9d2"]:
        write(NAMES[key], fmgen.single(key), threads=threads)
