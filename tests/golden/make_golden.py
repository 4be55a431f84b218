"""Write the oracle's expected values for the named workloads.

Calls only the CPU oracle (``oracle``) and the shared input generators
(``graphgen``).  Each output file records, per workload: vertex and edge
counts, the SHA-256 of the int32 core-number array (little endian), the
maximum core number, the maximum clique size omega with one witness, and
the oracle's run statistics.  Usage:

    python tests/golden/make_golden.py [--out DIR] [--cores-only] [--threads N] chung-lu-20k rmat-s22 ...

(--out: write the files to DIR instead of this folder; --cores-only: record
the core numbers only, with omega and its witness null; --threads N: find
omega with the oracle's threaded search, N workers sharing the incumbent,
for workloads whose single-threaded search takes too long.)
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from graphgen import workloads as W  # noqa: E402

SLUGS = {
    "chung-lu-20k": (W.CHUNG_LU_20K, W.chung_lu_20k),
    "rmat-s22": (W.RMAT_S22, W.rmat_s22),
    "rmat-s24": (W.RMAT_S24, W.rmat_s24),
    "chung-lu-100m": (W.CHUNG_LU_100M, W.chung_lu_100m),
}


def core_hash(core: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(core, dtype="<i4").tobytes()).hexdigest()


OUT = HERE


def batch_golden(count):
    """Oracle omega of every graph of the Erdos-Renyi batch."""
    b = W.er_batch_4096(count)
    t0 = time.time()
    omegas = []
    for g in b.graphs:
        om, wit, _ = oracle.max_clique(g)
        assert oracle.is_clique(g, wit) and len(wit) == om
        omegas.append(int(om))
    out = {"workload": b.name, "graphs": b.count, "n": b.n, "m": b.m, "omegas": omegas,
           "oracle_s": round(time.time() - t0, 1)}
    with open(os.path.join(OUT, "er-batch-%d.json" % count), "w") as f:
        json.dump(out, f)
    print("er-batch", count, "max omega", max(omegas), round(time.time() - t0, 1), flush=True)


def main(slugs, cores_only=False, threads=0):
    for slug in slugs:
        if slug.startswith("er-batch-"):
            batch_golden(int(slug.split("-")[-1]))
            continue
        name, fn = SLUGS[slug]
        g = fn()
        t0 = time.time()
        core = oracle.core_numbers(g)
        t1 = time.time()
        out = {"workload": name, "n": g.n, "m": g.m, "core_sha256": core_hash(core),
               "max_core": int(core.max()), "omega": None, "witness": None, "oracle_stats": None,
               "oracle_core_s": round(t1 - t0, 3), "oracle_max_clique_s": None}
        if not cores_only:
            if threads > 0:
                om, wit, st = oracle.max_clique_threads(g, threads)
            else:
                om, wit, st = oracle.max_clique(g)
            t2 = time.time()
            assert oracle.is_clique(g, wit) and len(wit) == om
            out.update({"omega": int(om), "witness": [int(x) for x in wit], "oracle_stats": st,
                        "oracle_max_clique_s": round(t2 - t1, 3),
                        "oracle_search": ("threaded, %d workers" % threads) if threads > 0 else "single thread"})
        with open(os.path.join(OUT, slug + ".json"), "w") as f:
            json.dump(out, f, indent=1)
        print(slug, out["max_core"], out["omega"], round(time.time() - t0, 1), flush=True)


if __name__ == "__main__":
    args = sys.argv[1:]
    if len(args) >= 2 and args[0] == "--out":
        OUT = args[1]
        args = args[2:]
    only = "--cores-only" in args
    args = [a for a in args if a != "--cores-only"]
    nthreads = 0
    if "--threads" in args:
        i = args.index("--threads")
        nthreads = int(args[i + 1])
        args = args[:i] + args[i + 2:]
    main(args or ["chung-lu-20k"], cores_only=only, threads=nthreads)
