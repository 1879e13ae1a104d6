"""Pins of the FP64 oracle against facts fixed by the paper and the mathematics.

None of these checks re-types the oracle's loops: each compares against a
different computation (dense reconstruction via n-mode products, numpy's
least-squares / QR / stable sort) or against an invariant the paper proves.
"""
import math

import numpy as np
import pytest

from tests.dense_ref import (dense_delta, dense_reconstruction, dense_sse, ridge_lstsq,
                             tiny_problem)

LAM = 0.01


# ---- P1: Omega^(n)_{i_n} grouping (Table 1; Alg. 3 slice loop) -------------
@pytest.mark.parametrize("E,dims", [(0, (3, 4)), (1, (5, 2)), (200, (7, 3, 9)), (1000, (1, 50, 2))])
def test_slices_match_stable_sort(ora, E, dims):
    rng = np.random.default_rng(E)
    idx = np.stack([rng.integers(0, I, size=E) for I in dims], axis=1).astype(np.int32).reshape(E, len(dims))
    for mode in range(len(dims)):
        perm, rp = ora.slices(dims, idx, mode)
        ref = np.argsort(idx[:, mode], kind="stable")
        assert np.array_equal(perm, ref)
        counts = np.bincount(idx[:, mode], minlength=dims[mode])
        assert np.array_equal(np.diff(rp), counts)
        assert rp[0] == 0 and rp[-1] == E


def test_slices_reject_out_of_range(ora):
    idx = np.array([[0, 5]], dtype=np.int32)
    with pytest.raises(ValueError):
        ora.slices((2, 3), idx, 1)


# ---- P2: delta, Eq. (delta) --------------------------------------------------
@pytest.mark.parametrize("J", [(2, 3, 2), (1, 1, 1), (3, 1, 4)])
def test_delta_equals_dense_linearity(ora, J):
    core, factors, idx, _ = tiny_problem(J=J)
    for e in range(6):
        for mode in range(3):
            d = ora.delta(core, factors, idx[e], mode)
            ref = dense_delta(core, factors, idx[e], mode)
            np.testing.assert_allclose(d, ref, rtol=1e-12, atol=1e-12)


def test_delta_order4_dense(ora):
    core, factors, idx, _ = tiny_problem(dims=(3, 4, 2, 3), J=(2, 2, 3, 2), E=10)
    for e in range(4):
        for mode in range(4):
            np.testing.assert_allclose(ora.delta(core, factors, idx[e], mode),
                                       dense_delta(core, factors, idx[e], mode), rtol=1e-12, atol=1e-12)


def test_delta_matrix_case(ora):
    """N = 2: the row update is matrix-completion ALS; delta = G a2^T / G^T a1^T."""
    rng = np.random.default_rng(3)
    G = rng.standard_normal((3, 4))
    A1, A2 = rng.random((5, 3)), rng.random((6, 4))
    coord = np.array([2, 5], dtype=np.int32)
    np.testing.assert_allclose(ora.delta(G, [A1, A2], coord, 0), G @ A2[5], rtol=1e-13)
    np.testing.assert_allclose(ora.delta(G, [A1, A2], coord, 1), G.T @ A1[2], rtol=1e-13)


def test_delta_superdiagonal_is_cp(ora):
    """Superdiagonal core (CP model): delta_j = g_j * prod_{k != n} a^(k)_{i_k j}."""
    rng = np.random.default_rng(4)
    R = 3
    g = rng.standard_normal(R)
    G = np.zeros((R, R, R))
    for r in range(R):
        G[r, r, r] = g[r]
    F = [rng.random((4, R)) for _ in range(3)]
    coord = np.array([1, 3, 2], dtype=np.int32)
    for mode in range(3):
        ref = g.copy()
        for k in range(3):
            if k != mode:
                ref = ref * F[k][coord[k]]
        np.testing.assert_allclose(ora.delta(G, F, coord, mode), ref, rtol=1e-13)


# ---- P3: row update, Eqs. (rowupdate)-(rowC), Theorem 1 ---------------------
@pytest.mark.parametrize("lam", [0.01, 1.0, 1e-6])
def test_row_update_is_ridge_regression(ora, lam):
    core, factors, idx, vals = tiny_problem(E=60)
    mode = 1
    ent = np.nonzero(idx[:, mode] == 2)[0]
    D = np.stack([dense_delta(core, factors, idx[e], mode) for e in ent])
    row, B, c, rc = ora.row_update(core, factors, mode, idx, vals, lam, entries=ent)
    assert rc == 0
    np.testing.assert_allclose(B, D.T @ D, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(c, D.T @ vals[ent], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(row, ridge_lstsq(D, vals[ent], lam), rtol=1e-9, atol=1e-10)
    # Theorem 1: gradient of the loss w.r.t. the row vanishes at the update
    grad = -2 * D.T @ (vals[ent] - D @ row) + 2 * lam * row
    assert np.max(np.abs(grad)) < 1e-9 * max(1.0, np.max(np.abs(D.T @ vals[ent])))


def test_spd_solve_matches_numpy(ora):
    rng = np.random.default_rng(5)
    for n in (1, 2, 5, 10, 16):
        M = rng.standard_normal((n + 3, n))
        B = M.T @ M
        c = rng.standard_normal(n)
        a, rc = ora.spd_solve(B, c, 0.01)
        assert rc == 0
        np.testing.assert_allclose(a, np.linalg.solve(B + 0.01 * np.eye(n), c), rtol=1e-9, atol=1e-12)


def test_empty_slice_gives_zero_row(ora):
    """B = 0, c = 0 with lambda > 0: the minimiser of lambda ||a||^2 is a = 0."""
    core, factors, idx, vals = tiny_problem(dims=(6, 5, 3), E=20)
    idx[:, 0] = np.minimum(idx[:, 0], 4)        # row 5 of mode 0 has no entries
    F, rc = ora.update_mode((6, 5, 3), core, factors, idx, vals, 0, LAM)
    assert rc == 0
    assert np.all(F[0][5] == 0.0)


# ---- P4: sweep, Theorem 2 -------------------------------------------------
def test_loss_monotone_every_mode(ora):
    dims = (8, 7, 6)
    core, factors, idx, vals = tiny_problem(dims=dims, J=(3, 2, 3), E=150, seed=7)
    F = [f.copy() for f in factors]
    prev = ora.loss(dims, core, F, idx, vals, LAM)
    for _ in range(4):
        for mode in range(3):
            F, rc = ora.update_mode(dims, core, F, idx, vals, mode, LAM)
            cur = ora.loss(dims, core, F, idx, vals, LAM)
            assert cur <= prev * (1 + 1e-12) + 1e-12
            prev = cur


def test_loss_matches_dense(ora):
    dims = (4, 5, 3)
    core, factors, idx, vals = tiny_problem(dims=dims)
    reg = sum(float(np.sum(a * a)) for a in factors)
    assert ora.loss(dims, core, factors, idx, vals, 0.3) == pytest.approx(
        dense_sse(core, factors, idx, vals) + 0.3 * reg, rel=1e-12)


def test_sweep_invariant_to_entry_order_and_threads(ora):
    dims = (9, 8, 7)
    core, factors, idx, vals = tiny_problem(dims=dims, J=(2, 3, 2), E=300, seed=11)
    F1, _ = ora.sweep(dims, core, factors, idx, vals, LAM, nthreads=1)
    F4, _ = ora.sweep(dims, core, factors, idx, vals, LAM, nthreads=4)
    for a, b in zip(F1, F4):
        assert np.array_equal(a, b)
    p = np.random.default_rng(0).permutation(len(vals))
    Fp, _ = ora.sweep(dims, core, factors, idx[p], vals[p], LAM)
    for a, b in zip(F1, Fp):
        np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12)


def test_sweep_equals_row_by_row_ridge(ora):
    """One mode update equals per-row ridge regressions built from dense deltas."""
    dims = (5, 4, 3)
    core, factors, idx, vals = tiny_problem(dims=dims, E=50, seed=2)
    F, _ = ora.update_mode(dims, core, factors, idx, vals, 0, LAM)
    for i in range(dims[0]):
        ent = np.nonzero(idx[:, 0] == i)[0]
        if len(ent) == 0:
            assert np.all(F[0][i] == 0)
            continue
        D = np.stack([dense_delta(core, factors, idx[e], 0) for e in ent])
        np.testing.assert_allclose(F[0][i], ridge_lstsq(D, vals[ent], LAM), rtol=1e-8, atol=1e-10)


# ---- P5: planted recovery ---------------------------------------------------
def _centered_planted(t):
    """Planted factors mapped to U(-1,1): all-positive U(0,1) columns are so
    collinear that ALS needs thousands of sweeps; centred ones converge in a
    few hundred, which keeps the pin quick."""
    import synth
    PF = [2.0 * f - 1.0 for f in t.planted_factors]
    return PF, synth.planted_values(t.planted_core, PF, t.idx), synth.planted_values(t.planted_core, PF, t.test_idx)


def test_planted_recovery_noise_free(ora):
    import synth
    t = synth.make_tensor((30, 30, 30), 5000, (3, 3, 3), sigma=0.0, seed=3, n_test=500)
    PF, vals, _ = _centered_planted(t)
    rng = np.random.default_rng(0)
    F = [f + 0.01 * rng.standard_normal(f.shape) for f in PF]
    G, F, errs = ora.fit(t.dims, t.planted_core, F, t.idx, vals, 1e-12, sweeps=250)
    rmse = ora.error_stats(G, F, t.idx, vals)["rmse"]
    assert rmse <= 1e-6 * np.std(vals)
    assert np.all(np.diff(errs) <= 1e-12 * errs[0])


def test_planted_recovery_noise_floor(ora):
    import synth
    sigma = 0.1
    t = synth.make_tensor((30, 30, 30), 8000, (3, 3, 3), sigma=0.0, seed=5, n_test=2000)
    PF, vals, tvals = _centered_planted(t)
    rng = np.random.default_rng(1)
    vals = vals + sigma * rng.standard_normal(len(vals))
    tvals = tvals + sigma * rng.standard_normal(len(tvals))
    F = [f + 0.05 * rng.standard_normal(f.shape) for f in PF]
    G, F, _ = ora.fit(t.dims, t.planted_core, F, t.idx, vals, 0.01, sweeps=60)
    tr = ora.error_stats(G, F, t.idx, vals)["rmse"]
    te = ora.error_stats(G, F, t.test_idx, tvals)["rmse"]
    assert 0.9 * sigma <= tr <= 1.1 * sigma
    assert abs(te - sigma) <= 0.05 * sigma
    # least squares with p free parameters (the factor entries; the core is
    # fixed) leaves E[train SSE] = sigma^2 (n - p): tr^2 / sigma^2 near 1 - p/n,
    # within a few standard deviations sqrt(2/n) of a chi-square mean
    n, p = len(vals), sum(d * j for d, j in zip(t.dims, (3, 3, 3)))
    assert abs(tr ** 2 / sigma ** 2 - (1 - p / n)) <= 4 * np.sqrt(2.0 / n)


# ---- P6: P-Tucker-Cache reaches the plain result ----------------------------
def test_cache_equals_plain(ora):
    dims = (7, 6, 5)
    core, factors, idx, vals = tiny_problem(dims=dims, J=(2, 3, 2), E=120, seed=9)
    Fp, _ = ora.sweep(dims, core, factors, idx, vals, LAM)
    Fc, _ = ora.sweep(dims, core, factors, idx, vals, LAM, variant="cache")
    for a, b in zip(Fp, Fc):
        np.testing.assert_allclose(b, a, rtol=1e-10, atol=1e-12)


def test_cache_zero_fallback(ora):
    """Exact zeros in factors exercise the plain-product fallback of Sec. 3.3."""
    dims = (6, 5, 4)
    core, factors, idx, vals = tiny_problem(dims=dims, J=(2, 2, 2), E=80, seed=10)
    for f in factors:
        f[::2, 0] = 0.0
    Fp, _ = ora.sweep(dims, core, factors, idx, vals, LAM)
    Fc, _ = ora.sweep(dims, core, factors, idx, vals, LAM, variant="cache")
    for a, b in zip(Fp, Fc):
        assert np.all(np.isfinite(b))
        np.testing.assert_allclose(b, a, rtol=1e-10, atol=1e-12)


# ---- P7: error, Eq. (reconfull) ---------------------------------------------
def test_error_matches_dense(ora):
    core, factors, idx, vals = tiny_problem()
    s = ora.sse(core, factors, idx, vals)
    assert s == pytest.approx(dense_sse(core, factors, idx, vals), rel=1e-12)
    st = ora.error_stats(core, factors, idx, vals)
    assert st["error"] == pytest.approx(np.sqrt(s))
    assert st["rmse"] == pytest.approx(np.sqrt(s / len(vals)))


# ---- P8: P-Tucker-Approx, Eq. (recon_partial), Alg. 4 -----------------------
def test_partial_error_forms_and_brute_force(ora):
    core, factors, idx, vals = tiny_problem(dims=(4, 3, 3), J=(2, 2, 2), E=25, seed=12)
    Rl = ora.partial_error(core, factors, idx, vals, literal=True)
    Rs = ora.partial_error(core, factors, idx, vals, literal=False)
    np.testing.assert_allclose(Rs, Rl, rtol=1e-9, atol=1e-9)
    base = dense_sse(core, factors, idx, vals)
    for b in range(core.size):
        G0 = core.copy().reshape(-1)
        G0[b] = 0.0
        ref = base - dense_sse(G0.reshape(core.shape), factors, idx, vals)
        assert Rs.reshape(-1)[b] == pytest.approx(ref, rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("rule", ["r_beta", "magnitude"])
def test_truncation_selection(ora, rule):
    rng = np.random.default_rng(13)
    G = rng.standard_normal((4, 5))
    G[0, 0] = 0.0                         # already removed: not counted
    R = rng.standard_normal((4, 5))
    R[1, 1] = R[2, 2]                     # a tie
    G2, removed = ora.truncate(G, R, 0.2, rule)
    nz = np.flatnonzero(G.reshape(-1))
    k = int(np.floor(0.2 * len(nz)))
    key = -R.reshape(-1)[nz] if rule == "r_beta" else np.abs(G.reshape(-1)[nz])
    order = nz[np.lexsort((nz, key))]
    assert list(removed) == list(order[:k])
    assert np.count_nonzero(G2) == len(nz) - k
    assert np.all(G2.reshape(-1)[order[k:]] == G.reshape(-1)[order[k:]])


def test_approx_fit_reduces_core(ora):
    dims = (8, 8, 8)
    core, factors, idx, vals = tiny_problem(dims=dims, J=(3, 3, 3), E=300, seed=14)
    G, F, errs = ora.fit(dims, core, factors, idx, vals, LAM, variant="approx", sweeps=3)
    nnz = 27
    for _ in range(3):
        nnz -= int(np.floor(0.2 * nnz))
    assert np.count_nonzero(G) == nnz
    # Approx deltas skip zeros: same as dense deltas with the truncated core
    e = 0
    for mode in range(3):
        np.testing.assert_allclose(ora.delta(G, F, idx[e], mode), dense_delta(G, F, idx[e], mode), rtol=1e-12,
                                   atol=1e-12)


# ---- P9: QR finalisation (Alg. 2, last loop) --------------------------------
def test_qr_finalize(ora):
    dims = (9, 7, 6)
    core, factors, _, _ = tiny_problem(dims=dims, J=(3, 2, 4))
    G, F = ora.qr_finalize(dims, core, factors)
    np.testing.assert_allclose(dense_reconstruction(G, F), dense_reconstruction(core, factors), rtol=1e-12,
                               atol=1e-12)
    for n, (q, a) in enumerate(zip(F, factors)):
        np.testing.assert_allclose(q.T @ q, np.eye(q.shape[1]), atol=1e-12)
        Q2, R2 = np.linalg.qr(a)
        s = np.sign(np.diag(R2))
        np.testing.assert_allclose(q, Q2 * s, atol=1e-12)


def test_qr_finalize_needs_tall(ora):
    with pytest.raises(ValueError):
        ora.qr_finalize((2, 5), np.ones((3, 2)), [np.ones((2, 3)), np.ones((5, 2))])


# ---- P10: predict and fold-in -------------------------------------------------
def test_predict_matches_dense(ora):
    core, factors, idx, _ = tiny_problem(dims=(3, 4, 2, 3)[:3], J=(2, 3, 2))
    X = dense_reconstruction(core, factors)
    np.testing.assert_allclose(ora.predict(core, factors, idx), X[tuple(idx.T)], rtol=1e-12, atol=1e-12)


def test_foldin_existing_row_reproduces_update(ora):
    dims = (6, 5, 4)
    core, factors, idx, vals = tiny_problem(dims=dims, E=90, seed=15)
    F, _ = ora.update_mode(dims, core, factors, idx, vals, 0, LAM)
    i = 3
    ent = np.nonzero(idx[:, 0] == i)[0]
    row, rc = ora.foldin(core, factors, 0, idx[ent][:, 1:], vals[ent], LAM)
    assert rc == 0
    assert np.array_equal(row, F[0][i])


# ---- c-9: the stopping rule of the Alg. 2 driver ------------------------------
def _rank1_als_errors(g, a, b, c, idx, x, lam, sweeps):
    """J = (1, 1, 1): each row update is the scalar ridge regression
    a_i = sum delta x / (sum delta^2 + lambda), delta = g * (other two
    entries); error = sqrt(sum (x - g a b c)^2).  Hand-computed per sweep."""
    a, b, c = list(a), list(b), list(c)
    errs = []
    for _ in range(sweeps):
        for mode, vec in ((0, a), (1, b), (2, c)):
            num = [0.0] * len(vec)
            den = [0.0] * len(vec)
            for (i, j, k), xv in zip(idx, x):
                row, d = ((i, g * b[j] * c[k]), (j, g * a[i] * c[k]), (k, g * a[i] * b[j]))[mode]
                num[row] += d * xv
                den[row] += d * d
            for r in range(len(vec)):
                vec[r] = num[r] / (den[r] + lam)
        errs.append(math.sqrt(sum((xv - g * a[i] * b[j] * c[k]) ** 2 for (i, j, k), xv in zip(idx, x))))
    return errs


def test_fit_stopping_rule_against_hand_computed_errors(ora):
    """The driver stops after sweep t, the first with |err_t - err_{t-1}| /
    err_{t-1} < tol (reading c-9), and reports err_1..err_t."""
    rng = np.random.default_rng(21)
    dims = (4, 3, 2)
    idx = np.array([(i, j, k) for i in range(4) for j in range(3) for k in range(2)][:20], dtype=np.int32)
    x = rng.random(len(idx)) + 0.5
    g, lam = 1.3, 0.01
    a0, b0, c0 = rng.random(4), rng.random(3), rng.random(2)
    ref = _rank1_als_errors(g, a0, b0, c0, [tuple(r) for r in idx], x, lam, 12)
    rel = [abs(ref[t] - ref[t - 1]) / ref[t - 1] for t in range(1, len(ref))]
    # stop after 0-based sweep t >= 4 whose change is below every earlier change:
    # a tol between them stops the driver exactly there
    stop = next(t for t in range(4, len(ref)) if rel[t - 1] < min(rel[:t - 1]))
    tol = math.sqrt(rel[stop - 1] * min(rel[:stop - 1]))
    assert all(r > tol for r in rel[:stop - 1]) and rel[stop - 1] < tol
    core = np.full((1, 1, 1), g)
    F = [a0[:, None], b0[:, None], c0[:, None]]
    _, _, errs = ora.fit(dims, core, F, idx, x, lam, sweeps=12, tol=tol)
    assert len(errs) == stop + 1                     # sweeps 1..stop+1 run (0-based error stop)
    np.testing.assert_allclose(errs, ref[:stop + 1], rtol=1e-12)
    _, _, errs_all = ora.fit(dims, core, F, idx, x, lam, sweeps=12, tol=0.0)
    np.testing.assert_allclose(errs_all, ref, rtol=1e-12)
