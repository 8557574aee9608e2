"""Write tests/golden/long_pair_1mbp.json: the oracle's result on the single long
pair workload (1,000,000-base uniform ACGT reference, query at 1% divergence
plus one inserted 5,000-base random segment, global affine DNA +2/-4, open 4,
extend 2, X-drop 1000, traceback).

Only the oracle computes the stored values (plain C, int64, every evaluated
cell kept: about 40 bytes per cell, some 35 GB of host memory for this pair);
the inputs come from the seeded generator in `synth`.  The GPU test of the
long-pair path compares its score, end cell, status, cell count and CIGAR
(length and SHA-256 of the little-endian uint32 BAM ops) with this file.

Run from the repository root:  python tests/golden/make_long_pair_golden.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "long_pair_1mbp.json")


def cigar_digest(ops: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(ops, dtype="<u4").tobytes()).hexdigest()


def main():
    b = synth.long_pair()  # seed 5, X-drop 1000
    q, r = b.pair(0)
    t0 = time.time()
    o = oracle.align(q, r, b.subst, **b.scoring)
    dt = time.time() - t0
    ops = o["cigar"]
    rec = {
        "_about": ("Oracle result (oracle/oracle.c, run by this script) for the single long "
                   "pair of synth.long_pair(): global affine DNA (+2/-4, open 4, extend 2), "
                   "X-drop 1000 on the previous antidiagonal's best (Sec. 5.2), traceback on."),
        "generator": {"function": "synth.long_pair", "length": 1_000_000, "div": 0.01,
                      "seg": 5000, "seed": 5, "xdrop": 1000},
        "M": int(q.shape[0]),
        "N": int(r.shape[0]),
        "score": int(o["score"]),
        "q_end": int(o["q_end"]),
        "r_end": int(o["r_end"]),
        "status": int(o["status"]),
        "cells": int(o["cells"]),
        "n_ops": int(ops.shape[0]),
        "cigar_sha256": cigar_digest(ops),
        "cigar_head": [int(x) for x in ops[:8]],
        "cigar_tail": [int(x) for x in ops[-8:]],
        "oracle_seconds": round(dt, 1),
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
