"""Writes oracle_small.json: fixed-input outputs of the FP64 oracle, kept as regression
anchors (the paper prints no worked example of the transform, so no value here is the
paper's).  Every value is computed by oracle/ from the inputs named beside it; inputs come
from paper_1606_05732_gb300.synth (seeded numpy, no method arithmetic).

    python tests/golden/make_golden.py        # rewrites tests/golden/oracle_small.json
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1606_05732_gb300 import synth  # noqa: E402

SMALL = dict(n=1000, d=8, m=4, B=64, seed=3, p=0.1, input_seed=3)


def small_input():
    return synth.csr_bernoulli(SMALL["n"], SMALL["d"], SMALL["p"], seed=SMALL["input_seed"])


def build():
    out = {"about": "outputs of the FP64 oracle on fixed inputs; written by tests/golden/make_golden.py"}
    words = []
    for seed in (0, 1, 2**64 - 1):
        for tag in (0, 1, 2):
            for idx in (0, 2**32 + 5):
                words.append({"seed": seed, "tag": tag, "idx": idx,
                              "words": [int(w) for w in oracle.philox_words(seed, tag, idx, 1).ravel()]})
    out["philox_words"] = {"cite": "Philox4x32-10 (Salmon et al., SC'11); key (lo32, hi32 of seed), "
                                   "counter (lo32 idx, hi32 idx, tag, 0)", "cases": words}
    h, s = oracle.hash_sign(1, 4096, 0, 16)
    out["hash_sign"] = {"cite": "Section 1.1 / Section 7: w = word i mod 4 of the tag-0 call at floor(i/4); "
                                   "h(i) = floor(w B / 2^32), sigma(i) from the lowest bit of w",
                        "seed": 1, "B": 4096, "row0": 0, "h": [int(x) for x in h], "sigma": [int(x) for x in s]}
    g = oracle.gaussian_block(5, 1, 8, 0, 8, 0, 4)
    out["gaussian"] = {"cite": "Theorem 1 (unit-variance Gaussians): Box-Muller of the tag-1 stream, "
                               "entry (r, c) = lane r%4 of call c*ceil(R/4) + r/4",
                       "seed": 5, "tag": 1, "R": 8, "rows": [0, 8], "cols": [0, 4], "values": g.tolist()}
    X = small_input()
    Y = oracle.apply_csr(SMALL["seed"], X.n, X.d, SMALL["m"], SMALL["B"], X.row_ptr, X.col_idx, X.vals)
    Yp = oracle.plain_csr(SMALL["seed"], X.n, X.d, SMALL["m"], X.row_ptr, X.col_idx, X.vals)
    out["apply_csr"] = {"cite": "Section 1.1: T.X = G.(S.X)", **SMALL, "nnz": int(X.nnz), "Y": Y.tolist()}
    out["plain_csr"] = {"cite": "Abstract / Section 4: the plain G~.X", **SMALL, "nnz": int(X.nnz), "Y": Yp.tolist()}
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(build(), f, indent=1)
        f.write("\n")
