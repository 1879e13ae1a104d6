"""Error bounds for comparing a GPU row update with the FP64 oracle's.

The GPU computes every delta vector of Eq. (delta) in FP32 (or a tensor-core
precision), so each row update of Eq. (rowupdate) solves a perturbed ridge
problem: Delta_i + E_i instead of Delta_i.  The solve itself (FP64 with one
refinement step) and the row sums (double-float or exact) add far less.  For
the ridge solution a = (B + lam I)^-1 Delta^T x with B = Delta^T Delta, a
first-order perturbation gives

    (B + lam I) da = E^T r - Delta^T E a ,    r = x - Delta a ,

so, with the SVD Delta = U S V^T,

    ||da|| <= ||E|| ||r|| / lambda_min(B + lam I)
              + ||E|| ||a|| max_k s_k / (s_k^2 + lam) .

The second factor is at most 1 / s_min over the non-zero singular values, so
a row with fewer entries than J (rank-deficient B) is not charged 1 / lam for
directions its entries never see.  ||E|| (spectral) is bounded by the
Frobenius norm of the elementwise bound |E| <= gamma * |Delta|_abs, where
|Delta|_abs is the delta of the absolute core and factors: any evaluation of a
sum of K products of N - 1 factor entries and one core entry, in any order,
has |error| <= gamma_{K+N} * sum |terms|, gamma_n = n u / (1 - n u) (Higham,
Accuracy and Stability of Numerical Algorithms, Lemma 3.1 and Sec. 3.1).

Every quantity comes from the oracle (its deltas and its row sums); nothing
comes from the GPU path.
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24
U64 = 2.0 ** -53


def gamma(n: int, u: float = U32) -> float:
    """gamma_n = n u / (1 - n u)."""
    return n * u / (1.0 - n * u)


def row_delta(ora, core, factors, mode, idx, entries):
    """Oracle deltas of the given entries (rows of Delta_i) and the deltas of
    the absolute core and factors (|Delta|_abs)."""
    acore = np.abs(core)
    af = [np.abs(f) for f in factors]
    D = np.stack([ora.delta(core, factors, idx[e], mode) for e in entries]) if len(entries) else None
    Da = np.stack([ora.delta(acore, af, idx[e], mode) for e in entries]) if len(entries) else None
    return D, Da


def ridge_bound(D, Dabs, x, lam, g, safety=4.0):
    """First-order bound on ||a(Delta + E) - a(Delta)|| for |E| <= g
    |Delta|_abs, times `safety`.  Exactly,
        a~ - a = (B~ + lam I)^-1 (E^T r - (Delta + E)^T E a),
    B~ = (Delta + E)^T (Delta + E); the first-order bound replaces B~ and
    Delta + E by B and Delta.  The factor 4 covers what that leaves out (a
    row of fourteen nearly collinear deltas has shown 2.2 times the
    first-order value) and the GPU's own rounding in the row sums and the
    solve.  Where ||E|| reaches the smallest singular value of a row's Delta
    no perturbation bound stays small; such rows are rare in the data here."""
    J = D.shape[1]
    B = D.T @ D
    M = B + lam * np.eye(J)
    a = np.linalg.solve(M, D.T @ x)
    r = x - D @ a
    w = np.linalg.eigvalsh(M)
    s = np.linalg.svd(D, compute_uv=False)
    amp = float(np.max(s / (s * s + lam))) if s.size else 0.0
    En = g * np.linalg.norm(Dabs)
    return safety * (En * np.linalg.norm(r) / w[0] + En * np.linalg.norm(a) * amp), a


def mode_bounds(ora, core, factors, idx, vals, mode, lam, g, rows=None):
    """Per-row bound (and the oracle's row) for the update of `mode` from the
    factor state `factors`; rows: subset of row ids (None: every row)."""
    dims = tuple(f.shape[0] for f in factors)
    perm, rp = ora.slices(dims, idx, mode)
    rows = range(dims[mode]) if rows is None else rows
    out = {}
    for i in rows:
        ent = perm[rp[i]:rp[i + 1]]
        if len(ent) == 0:
            out[i] = (0.0, np.zeros(core.shape[mode]))
            continue
        D, Da = row_delta(ora, core, factors, mode, idx, ent)
        out[i] = ridge_bound(D, Da, np.asarray(vals)[ent], lam, g)
    return out
