"""Writes tests/golden/tiny_sweep.json by calling only the oracle (and the
seeded input generator).  The fixture is a cross-machine regression record of
the oracle (x86 build vs the Arm build of the same C source), not a pin: the
pins live in tests/test_oracle_pins.py.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    t = synth.make_tensor((12, 10, 9), 400, (3, 3, 2), sigma=0.1, seed=21, n_test=40)
    m = synth.init_model(t.dims, (3, 2, 2), seed=21)
    F1, _ = oracle.sweep(t.dims, m.core, m.factors, t.idx, t.vals, 0.01)
    F2, _ = oracle.sweep(t.dims, m.core, F1, t.idx, t.vals, 0.01)
    R = oracle.partial_error(m.core, F2, t.idx, t.vals)
    out = dict(
        recipe="synth.make_tensor((12,10,9), 400, (3,3,2), sigma=0.1, seed=21, n_test=40); "
               "synth.init_model(dims, (3,2,2), seed=21); two plain sweeps, lambda=0.01",
        factors_after_2=[f.tolist() for f in F2],
        sse_after_2=oracle.sse(m.core, F2, t.idx, t.vals),
        test_sse_after_2=oracle.sse(m.core, F2, t.test_idx, t.test_vals),
        R_after_2=R.reshape(-1).tolist(),
    )
    with open(os.path.join(ROOT, "tests", "golden", "tiny_sweep.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
