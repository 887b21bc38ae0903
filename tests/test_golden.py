"""Regression anchors: tests/golden/oracle_small.json holds outputs of the FP64 oracle on
fixed inputs (written by tests/golden/make_golden.py, which calls only the oracle).  The
CPU test catches any later change to the oracle's arithmetic; the GPU test checks the
CUDA path against the same stored values (integers bit-exact, floats at the parity bars)."""
import json
import os
import sys

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_golden  # noqa: E402

with open(os.path.join(HERE, "golden", "oracle_small.json")) as f:
    GOLDEN = json.load(f)


def test_oracle_reproduces_golden():
    now = make_golden.build()
    for case_now, case in zip(now["philox_words"]["cases"], GOLDEN["philox_words"]["cases"]):
        assert case_now == case
    assert now["hash_sign"] == GOLDEN["hash_sign"]
    # FP64 libm may differ by an ulp between machines: floats to 1e-13 relative
    for key in ("gaussian",):
        np.testing.assert_allclose(now[key]["values"], GOLDEN[key]["values"], rtol=1e-13, atol=1e-13)
    for key in ("apply_csr", "plain_csr"):
        np.testing.assert_allclose(now[key]["Y"], GOLDEN[key]["Y"], rtol=1e-12, atol=1e-12)


@pytest.mark.gpu
def test_cuda_path_matches_golden():
    torch = pytest.importorskip("torch")
    from paper_1606_05732_gb300 import countgauss
    for case in GOLDEN["philox_words"]["cases"]:
        got = countgauss.generate_words(case["seed"], case["tag"], case["idx"], 1).cpu().numpy().view(np.uint32)
        assert [int(w) for w in got.ravel()] == case["words"]
    hs = GOLDEN["hash_sign"]
    h, s = countgauss.generate_hash_sign(hs["seed"], hs["B"], hs["row0"], len(hs["h"]))
    assert h.cpu().numpy().tolist() == hs["h"] and s.cpu().numpy().tolist() == hs["sigma"]
    g = GOLDEN["gaussian"]
    got = countgauss.generate_gaussian(g["seed"], g["tag"], g["R"], *g["rows"], *g["cols"]).cpu().numpy()
    np.testing.assert_allclose(got, np.asarray(g["values"]), rtol=0, atol=4e-6 * 6)
    X = make_golden.small_input()
    dev = torch.device("cuda", 0)
    rp = torch.from_numpy(X.row_ptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(X.col_idx).to(dev)
    v = torch.from_numpy(X.vals).to(dev)
    a = GOLDEN["apply_csr"]
    plan = countgauss.CountGauss(a["n"], a["d"], a["m"], a["B"], a["seed"])
    for key, Y in (("apply_csr", plan.apply_csr(rp, ci, v)), ("plain_csr", plan.plain_csr(rp, ci, v))):
        want = np.asarray(GOLDEN[key]["Y"])
        got = Y.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-5, key
    plan.check()
