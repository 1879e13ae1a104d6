"""Brute-force dense helpers used to pin the oracle (tests only).

Everything here works on tiny tensors by materialising the full dense
reconstruction with the n-mode products of Sec. 2.1 (numpy einsum), which is a
different computation from the oracle's per-entry loops.
"""
import string

import numpy as np


def dense_reconstruction(core, factors):
    """X_hat = G x_1 A^(1) x_2 ... x_N A^(N) as a dense array [I_1..I_N]."""
    N = core.ndim
    js = string.ascii_lowercase[:N]
    iss = string.ascii_uppercase[:N]
    spec = js + "," + ",".join(iss[k] + js[k] for k in range(N)) + "->" + iss
    return np.einsum(spec, core, *factors, optimize=True)


def dense_delta(core, factors, coord, mode):
    """delta_j = X_hat(coord) with row coord[mode] of A^(mode) replaced by e_j
    (X_hat is linear in that row)."""
    Jn = core.shape[mode]
    out = np.empty(Jn)
    for j in range(Jn):
        f = [a.copy() for a in factors]
        f[mode][coord[mode], :] = 0.0
        f[mode][coord[mode], j] = 1.0
        out[j] = dense_reconstruction(core, f)[tuple(coord)]
    return out


def dense_sse(core, factors, idx, vals):
    X = dense_reconstruction(core, factors)
    r = np.asarray(vals) - X[tuple(np.asarray(idx).T)]
    return float(np.sum(r * r))


def ridge_lstsq(D, x, lam):
    """argmin_a ||D a - x||^2 + lam ||a||^2 by least squares on the stacked
    system [D; sqrt(lam) I] a = [x; 0] (numpy's SVD-based lstsq)."""
    J = D.shape[1]
    M = np.vstack([D, np.sqrt(lam) * np.eye(J)])
    y = np.concatenate([x, np.zeros(J)])
    return np.linalg.lstsq(M, y, rcond=None)[0]


def tiny_problem(dims=(4, 5, 3), J=(2, 3, 2), E=40, seed=1, core_scale=1.0):
    rng = np.random.default_rng(seed)
    core = rng.standard_normal(J) * core_scale
    factors = [rng.random((I, j)) for I, j in zip(dims, J)]
    idx = np.stack([rng.integers(0, I, size=E) for I in dims], axis=1).astype(np.int32)
    vals = rng.standard_normal(E)
    return core, factors, idx, vals
