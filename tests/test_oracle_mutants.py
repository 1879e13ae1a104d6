"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a dropped
factor, a wrong index, a flipped sign, a missing term, an unstable order),
builds that copy into its own library on the CPU, and runs the pin that
guards the step: the pin must fail.  The unmodified copy must pass the same
pins, so a failure is the planted mistake's doing.  The committed oracle is
never modified.
"""
import importlib.util
import os

import numpy as np
import pytest

from tests import test_oracle_pins as pins

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

# (name, text in ptk_oracle.c, replacement, the pin that must catch it, its arguments)
MUTANTS = [
    ("delta_drops_last_factor",
     "            if (k == mode) continue;\n            p *= A[k][(int64_t)coord[k] * J[k] + j[k]];\n        }\n"
     "        delta[j[mode]] += p;",
     "            if (k == mode || k == N - 1) continue;\n            p *= A[k][(int64_t)coord[k] * J[k] + j[k]];\n"
     "        }\n        delta[j[mode]] += p;",
     pins.test_delta_equals_dense_linearity, dict(J=(2, 3, 2))),
    ("gram_wrong_index", "B[p * Jn + q] += d[p] * d[q];", "B[p * Jn + q] += d[p] * d[p];",
     pins.test_row_update_is_ridge_regression, dict(lam=0.01)),
    ("c_sign_flipped", "c[p] += vals[e] * d[p];", "c[p] -= vals[e] * d[p];",
     pins.test_row_update_is_ridge_regression, dict(lam=1.0)),
    ("lambda_dropped", "double s = B[i * n + j] + (i == j ? lambda : 0.0);", "double s = B[i * n + j];",
     pins.test_spd_solve_matches_numpy, {}),
    ("cholesky_transposed", "s -= L[i * n + k] * L[j * n + k];", "s -= L[i * n + k] * L[k * n + j];",
     pins.test_spd_solve_matches_numpy, {}),
    ("sse_absolute", "s += r * r;", "s += fabs(r);",
     pins.test_error_matches_dense, {}),
    ("slices_unstable", "for (int64_t e = 0; e < E; ++e) perm[cursor[idx[e * N + mode]]++] = e;",
     "for (int64_t e = E - 1; e >= 0; --e) perm[cursor[idx[e * N + mode]]++] = e;",
     pins.test_slices_match_stable_sort, dict(E=200, dims=(7, 3, 9))),
    ("r_beta_sign", "R[b] += p[b] * (-2.0 * x + p[b] + 2.0 * others);",
     "R[b] += p[b] * (2.0 * x + p[b] + 2.0 * others);",
     pins.test_partial_error_forms_and_brute_force, {}),
    ("qr_sign_not_fixed", "        if (R[r * n + r] < 0) {", "        if (0) {",
     pins.test_qr_finalize, {}),
    ("cache_rescale_inverted", "d[j[n]] += pres[e * Gs + b] / a;", "d[j[n]] += pres[e * Gs + b] * a;",
     pins.test_cache_equals_plain, {}),
]


def _oracle_copy(tmp_path, name, old=None, new=None):
    """A separate instance of the oracle module, built from a (mutated) copy of its source."""
    src = open(os.path.join(ORACLE_DIR, "ptk_oracle.c")).read()
    if old is not None:
        assert src.count(old) >= 1, f"mutation site of {name} not found"
        src = src.replace(old, new, 1)
    d = tmp_path / name
    d.mkdir()
    (d / "ptk_oracle.c").write_text(src)
    spec = importlib.util.spec_from_file_location(f"oracle_copy_{name}", os.path.join(ORACLE_DIR, "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC = str(d / "ptk_oracle.c")
    mod._LIB = str(d / "libptk_oracle.so")
    mod._lib = None
    mod.build()
    return mod


def test_unmodified_copy_passes_the_pins(tmp_path):
    ora = _oracle_copy(tmp_path, "identity")
    seen = set()
    for _, _, _, pin, kw in MUTANTS:
        key = (pin.__name__, tuple(sorted(kw.items())))
        if key in seen:
            continue
        seen.add(key)
        pin(ora, **kw)


@pytest.mark.parametrize("name,old,new,pin,kw", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, pin, kw):
    ora = _oracle_copy(tmp_path, name, old, new)
    with np.errstate(all="ignore"), pytest.raises((AssertionError, ValueError, RuntimeError)):
        pin(ora, **kw)
