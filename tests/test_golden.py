"""The oracle reproduces its stored regression record (tests/golden), so the
x86 and Arm builds of the same C source agree."""
import json
import os

import numpy as np

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "tiny_sweep.json")


def test_oracle_matches_golden_record(ora):
    g = json.load(open(GOLD))
    t = synth.make_tensor((12, 10, 9), 400, (3, 3, 2), sigma=0.1, seed=21, n_test=40)
    m = synth.init_model(t.dims, (3, 2, 2), seed=21)
    F1, _ = ora.sweep(t.dims, m.core, m.factors, t.idx, t.vals, 0.01)
    F2, _ = ora.sweep(t.dims, m.core, F1, t.idx, t.vals, 0.01)
    for a, b in zip(F2, g["factors_after_2"]):
        np.testing.assert_allclose(a, np.array(b), rtol=1e-11, atol=1e-13)
    assert abs(ora.sse(m.core, F2, t.idx, t.vals) - g["sse_after_2"]) <= 1e-10 * g["sse_after_2"]
    R = ora.partial_error(m.core, F2, t.idx, t.vals).reshape(-1)
    np.testing.assert_allclose(R, np.array(g["R_after_2"]), rtol=1e-9, atol=1e-11)
