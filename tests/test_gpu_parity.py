"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Sizes span several kernel tiles with ragged tails; the FP64 path is compared
element by element at rtol 1e-9 (the same arithmetic, different summation
order), the FP32 path against the oracle run on the FP32-rounded inputs with a
bound derived from each row's condition number (see test_sweep_fp32).
"""
import numpy as np
import pytest

import bounds
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1710_02261_gb300 as P  # noqa: E402

LAM = 0.01


@pytest.fixture(scope="module")
def ctx():
    c = P.Context(0)
    yield c
    c.close()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def to_gpu(t, dtype):
    return P.SparseObs.from_numpy(t.idx, t.vals, t.dims, dtype=dtype)


# ---- a1: slice layout ---------------------------------------------------------
@pytest.mark.parametrize("dims,E,dist", [
    ((7, 5, 3), 0, "uniform"),
    ((7, 5, 3), 1, "uniform"),
    ((300, 1, 40), 5000, "uniform"),
    ((100000, 50000, 30, 24), 300000, [("zipf", 1.1), ("zipf", 1.1), "uniform", "uniform"]),
    ((1 << 20, 3, 70000), 200000, "uniform"),
    ((2000, 2000), 4097, "uniform"),
])
def test_slices_bit_exact(ctx, ora, dims, E, dist):
    t = synth.make_tensor(dims, E, (1,) * len(dims), dist=dist, sigma=0.0, seed=3, n_test=0)
    x = to_gpu(t, torch.float32)
    for mode in range(len(dims)):
        s = P.build_mode_slices(ctx, x, mode)
        perm, rp = s.perm_and_rowptr()
        torch.cuda.synchronize()
        operm, orp = ora.slices(dims, t.idx, mode)
        assert np.array_equal(perm.cpu().numpy().astype(np.int64), operm)
        assert np.array_equal(rp.cpu().numpy(), orp)
        s.close()


def test_slices_reject_bad_index(ctx):
    idx = torch.tensor([[0, 1], [5, 0]], dtype=torch.int32, device="cuda")
    x = P.SparseObs(idx, torch.ones(2, device="cuda"), (3, 2))
    with pytest.raises(P.PtkError) as e:
        P.build_mode_slices(ctx, x, 0)
    assert e.value.status == 1


# ---- a2 + a9: delta through prediction (Eq. recon2) ---------------------------
@pytest.mark.parametrize("dims,J", [
    ((40, 30), (3, 5)),
    ((20, 30, 25), (5, 5, 5)),
    ((20, 30, 25), (2, 7, 4)),          # non-uniform ranks: generic kernel
    ((9, 8, 7, 6), (10, 10, 10, 10)),
    ((6, 5, 4, 3, 5), (3, 3, 3, 3, 3)),
    ((50, 40, 30), (16, 16, 16)),
])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_predict_matches_oracle(ctx, ora, dims, J, dtype):
    t = synth.make_tensor(dims, 777, J, sigma=0.1, seed=5, n_test=0)
    m0 = synth.init_model(dims, J, seed=5)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    core, facs = (m0.core, m0.factors) if dtype == "f64" else (f32(m0.core), [f32(a) for a in m0.factors])
    model = P.Model.from_numpy(core, facs, dtype=tdt)
    got = P.predict(ctx, model, torch.tensor(t.idx, device="cuda")).double().cpu().numpy()
    ref = ora.predict(core, facs, t.idx)
    tol = 1e-12 if dtype == "f64" else 2e-6
    np.testing.assert_allclose(got, ref, rtol=tol, atol=tol * np.max(np.abs(ref)))


# ---- a2..a6: FP64 sweep is the oracle's arithmetic ------------------------------
def _fp64_case(dims, E, J, dist="uniform", seed=0):
    t = synth.make_tensor(dims, E, J, dist=dist, sigma=0.1, seed=seed, n_test=0)
    m0 = synth.init_model(dims, J, seed=seed)
    return t, m0


@pytest.mark.parametrize("dims,E,J,dist", [
    ((200, 150, 100), 20000, (5, 5, 5), "uniform"),
    ((3, 400, 50), 9000, (3, 4, 2), "uniform"),                 # rows far longer than a tile
    ((2000, 1500, 7), 3000, (4, 4, 4), "uniform"),              # mostly 1-2 entries per row, empty rows
    ((500, 300, 20, 10), 12000, (3, 3, 3, 3), [("zipf", 1.1), ("zipf", 1.1), "uniform", "uniform"]),
    ((60, 50), 4000, (6, 5), "uniform"),
])
def test_sweep_fp64_matches_oracle(ctx, ora, dims, E, J, dist):
    t, m0 = _fp64_case(dims, E, J, dist)
    x = to_gpu(t, torch.float64)
    sl = P.build_all_slices(ctx, x, dtype=torch.float64)
    model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float64)
    F = [a.copy() for a in m0.factors]
    for sweep in range(2):
        st = P.als_sweep(ctx, x, sl, model, precision="fp64", lam=LAM)
        F, rc = ora.sweep(dims, m0.core, F, t.idx, t.vals, LAM)
        _, Fg = model.to_numpy()
        for a, b in zip(Fg, F):
            np.testing.assert_allclose(a, b, rtol=1e-8, atol=1e-10)
        ref = ora.error_stats(m0.core, F, t.idx, t.vals)
        assert st["rmse"] == pytest.approx(ref["rmse"], rel=1e-9)
        assert st["loss"] == pytest.approx(ora.loss(dims, m0.core, F, t.idx, t.vals, LAM), rel=1e-9)
    for s in sl:
        s.close()


@pytest.mark.parametrize("dims,E,J", [((80, 60, 40), 9000, (10, 10, 10)), ((70, 50, 40), 6000, (16, 12, 13)),
                                      ((40, 30, 20, 10), 5000, (8, 9, 7, 8))])
def test_sweep_fp64_large_ranks(ctx, ora, dims, E, J):
    """Ranks whose Gram sums are split over several threads per run."""
    t, m0 = _fp64_case(dims, E, J, seed=6)
    x = to_gpu(t, torch.float64)
    sl = P.build_all_slices(ctx, x, dtype=torch.float64)
    model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float64)
    P.als_sweep(ctx, x, sl, model, precision="fp64", lam=LAM)
    F, _ = ora.sweep(dims, m0.core, m0.factors, t.idx, t.vals, LAM)
    _, Fg = model.to_numpy()
    for a, b in zip(Fg, F):
        np.testing.assert_allclose(a, b, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("schedule", ["rows_static", "rows_dynamic"])
@pytest.mark.parametrize("dims,E,J,dist", [
    ((3, 400, 50), 9000, (3, 4, 2), "uniform"),                 # rows far longer than a tile
    ((2000, 1500, 7), 3000, (4, 4, 4), "uniform"),              # empty rows, more rows than warps' first pass
    ((500, 300, 20, 10), 12000, (3, 3, 3, 3), [("zipf", 1.1), ("zipf", 1.1), "uniform", "uniform"]),
    ((40, 30, 20), 4000, (16, 12, 13), "uniform"),              # 5 outputs per lane at J = 16
])
def test_row_schedules_fp64_match_oracle(ctx, ora, schedule, dims, E, J, dist):
    """Sec. 3.4's row-per-thread mapping (one warp per row, static or dynamic
    dealing) computes the same B_i, c_i as the entry split."""
    t, m0 = _fp64_case(dims, E, J, dist, seed=4)
    x = to_gpu(t, torch.float64)
    sl = P.build_all_slices(ctx, x, dtype=torch.float64)
    model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float64)
    st = P.als_sweep(ctx, x, sl, model, precision="fp64", lam=LAM, schedule=schedule)
    F, _ = ora.sweep(dims, m0.core, m0.factors, t.idx, t.vals, LAM)
    _, Fg = model.to_numpy()
    for a, b in zip(Fg, F):
        np.testing.assert_allclose(a, b, rtol=1e-8, atol=1e-10)
    assert st["rmse"] == pytest.approx(ora.error_stats(m0.core, F, t.idx, t.vals)["rmse"], rel=1e-9)
    for s in sl:
        s.close()


def test_row_schedule_rejects_unknown_value(ctx):
    t, m0 = _fp64_case((20, 10, 5), 100, (2, 2, 2))
    x = to_gpu(t, torch.float64)
    sl = P.build_all_slices(ctx, x, dtype=torch.float64)
    model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float64)
    o = P._opts("plain", "fp64", LAM)
    o.schedule = 5
    coo, m = x.cstruct(), model.cstruct()
    arr = (P.C.c_void_p * P.F.MAX_ORDER)(*[s._h for s in sl])
    rc = P._lib().ptk_als_sweep(ctx.handle, P.C.byref(coo), P.C.cast(arr, P.C.POINTER(P.C.c_void_p)), P.C.byref(m),
                                P.C.byref(o), None, None)
    assert rc == 1
    for s in sl:
        s.close()


def _sweep_bits_and_launches(ctx, t, m0, schedule):
    x = to_gpu(t, torch.float32)
    sl = P.build_all_slices(ctx, x)
    model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float32)
    torch.cuda.synchronize()
    l0 = P.launch_count()
    P.als_sweep(ctx, x, sl, model, precision="fp32", lam=LAM, schedule=schedule)
    launches = P.launch_count() - l0
    _, F = model.to_numpy()
    for s in sl:
        s.close()
    return [a.copy() for a in F], launches


@pytest.mark.parametrize("dims,E,dist,expect", [
    ((100000, 100000, 100000), 4_000_000, "uniform", "rows_static"),   # ~40 entries per row, longest ~70
    ((500, 300, 20, 10), 12000, [("zipf", 1.1), ("zipf", 1.1), "uniform", "uniform"], "tensor"),
])
def test_auto_schedule_choice(ctx, dims, E, dist, expect):
    """The default schedule takes whole rows per warp for short, even rows and
    the tensor-core chunks where most entries sit in rows of 64 or more (every
    mode of the skewed case): bit-identical to the schedule it picks."""
    J = (4,) * len(dims)
    t = synth.make_tensor(dims, E, J, dist=dist, sigma=0.1, seed=9, n_test=0)
    m0 = synth.init_model(dims, J, seed=9)
    Fa, la = _sweep_bits_and_launches(ctx, t, m0, "auto")
    Fe, le = _sweep_bits_and_launches(ctx, t, m0, expect)
    assert la == le
    for a, b in zip(Fa, Fe):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.mark.parametrize("schedule", ["auto", "entries", "rows_static", "rows_dynamic"])
@pytest.mark.parametrize("J", [(10, 10, 10), (5, 5, 5), (14, 14, 14)])
def test_gram_compensated_rank_deficient(ctx, ora, J, schedule):
    """Rows with fewer entries than J and |delta| ~ 1e3: B_i is rank deficient
    and lambda = 0.01 is far below eps_fp32 * ||B_i||, so only compensated sums
    keep B_i + lambda I positive definite and the rows equal to the oracle's
    (run on the same FP32-rounded inputs)."""
    dims = (600, 40, 30)
    rng = np.random.default_rng(17)
    idx = np.stack([rng.integers(0, d, size=900) for d in dims], axis=1).astype(np.int32)
    vals = f32(100.0 * rng.standard_normal(900))
    core = f32(rng.random(J))
    F0 = [f32(20.0 * rng.random((d, j))) for d, j in zip(dims, J)]
    x = P.SparseObs.from_numpy(idx, vals, dims, dtype=torch.float32)
    s0 = P.build_mode_slices(ctx, x, 0)
    sl = [s0] + [P.build_mode_slices(ctx, x, n) for n in (1, 2)]
    model = P.Model.from_numpy(core, F0, dtype=torch.float32)
    st = P.als_sweep(ctx, x, sl, model, precision="fp32", lam=LAM, schedule=schedule)
    assert st["bad_rows"] == 0
    _, Fg = model.to_numpy()
    # what is left is the FP32 delta itself: |E| <= gamma_{K+N} |Delta|_abs,
    # carried to each row by the first-order ridge perturbation bound
    # (tests/bounds.py), which charges a rank-deficient row only 1 / s_min of
    # the directions its entries span
    K = J[1] * J[2]
    rows = bounds.mode_bounds(ora, core, F0, idx, vals, 0, LAM, bounds.gamma(K + 3))
    for i, (bd, aref) in rows.items():
        assert np.linalg.norm(Fg[0][i] - aref) <= bd + 1e-12, i


@pytest.mark.parametrize("E", [1, 1919, 1920, 1921, 3840, 5000])
def test_gram_tile_boundaries_fp64(ctx, ora, E):
    """One giant row plus scattered short rows around every tile boundary."""
    rng = np.random.default_rng(E)
    dims = (50, 30, 20)
    idx = np.stack([rng.integers(0, d, size=E) for d in dims], axis=1).astype(np.int32)
    idx[: E // 2, 0] = 7                          # half of all entries in row 7 of mode 0
    vals = rng.standard_normal(E)
    m0 = synth.init_model(dims, (4, 3, 5), seed=1)
    x = P.SparseObs.from_numpy(idx, vals, dims, dtype=torch.float64)
    sl = P.build_all_slices(ctx, x, dtype=torch.float64)
    model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float64)
    P.als_sweep(ctx, x, sl, model, precision="fp64", lam=LAM)
    F, _ = ora.sweep(dims, m0.core, m0.factors, idx, vals, LAM)
    _, Fg = model.to_numpy()
    for a, b in zip(Fg, F):
        np.testing.assert_allclose(a, b, rtol=1e-8, atol=1e-10)


# ---- FP32 path ------------------------------------------------------------------
def _row_conditions(ora, core, F_before, idx, vals, mode, lam):
    """kappa(B_i + lam I) of every row of `mode` from the oracle's B_i."""
    perm, rp = ora.slices(tuple(f.shape[0] for f in F_before), idx, mode)
    kap = np.ones(F_before[mode].shape[0])
    for i in range(len(rp) - 1):
        if rp[i + 1] == rp[i]:
            continue
        _, B, _, _ = ora.row_update(core, F_before, mode, idx, vals, lam, entries=perm[rp[i]:rp[i + 1]])
        w = np.linalg.eigvalsh(B + lam * np.eye(B.shape[0]))
        kap[i] = w[-1] / w[0]
    return kap


def test_sweep_fp32_matches_oracle(ctx, ora):
    """FP32 sweep vs the oracle on the FP32-rounded inputs, mode 0 (no earlier
    mode's rounding feeds it): ||a_gpu - a_ref|| <= 64 kappa_i 2^-24 ||a_ref||,
    and rows with kappa_i <= 100 within 1e-5 relative."""
    dims, J = (400, 300, 200), (5, 5, 5)
    t = synth.make_tensor(dims, 40000, J, sigma=0.1, seed=2, n_test=0)
    m0 = synth.init_model(dims, J, seed=2)
    core, F0, vals = f32(m0.core), [f32(a) for a in m0.factors], f32(t.vals)
    x = P.SparseObs.from_numpy(t.idx, vals, dims, dtype=torch.float32)
    sl = P.build_all_slices(ctx, x)
    model = P.Model.from_numpy(core, F0, dtype=torch.float32)
    P.als_sweep(ctx, x, sl, model, precision="fp32", lam=LAM)
    _, Fg = model.to_numpy()
    Fref, _ = ora.update_mode(dims, core, F0, t.idx, vals, 0, LAM)
    kap = _row_conditions(ora, core, F0, t.idx, vals, 0, LAM)
    a, b = Fg[0], Fref[0]
    err = np.linalg.norm(a - b, axis=1)
    nrm = np.linalg.norm(b, axis=1)
    assert np.all(err <= 64 * kap * 2.0 ** -24 * nrm + 1e-30)
    good = kap <= 100
    assert np.all(err[good] <= 1e-5 * nrm[good])


def test_sweep_fp32_all_modes_close(ctx, ora):
    dims, J = (300, 200, 100), (5, 4, 3)
    t = synth.make_tensor(dims, 30000, J, sigma=0.1, seed=4, n_test=3000)
    m0 = synth.init_model(dims, J, seed=4)
    core, F0, vals = f32(m0.core), [f32(a) for a in m0.factors], f32(t.vals)
    x = P.SparseObs.from_numpy(t.idx, vals, dims, dtype=torch.float32)
    sl = P.build_all_slices(ctx, x)
    model = P.Model.from_numpy(core, F0, dtype=torch.float32)
    st = P.als_sweep(ctx, x, sl, model, precision="fp32", lam=LAM)
    Fref, _ = ora.sweep(dims, core, F0, t.idx, vals, LAM)
    ref = ora.error_stats(core, Fref, t.idx, vals)
    assert st["rmse"] == pytest.approx(ref["rmse"], rel=1e-4)
    xt = P.SparseObs.from_numpy(t.test_idx, t.test_vals, dims, dtype=torch.float32)
    te = P.error(ctx, xt, model, LAM)
    rte = ora.error_stats(core, Fref, t.test_idx, t.test_vals)
    assert te["rmse"] == pytest.approx(rte["rmse"], rel=1e-4)


# ---- a9: fold-in ------------------------------------------------------------------
def test_foldin_matches_oracle(ctx, ora):
    dims, J = (100, 80, 60), (6, 5, 4)
    m0 = synth.init_model(dims, J, seed=9)
    rng = np.random.default_rng(9)
    counts = [1, 5, 37, 300, 2500, 0, 7]
    obs_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    tot = int(obs_ptr[-1])
    obs = np.stack([np.zeros(tot, int), rng.integers(0, 80, tot), rng.integers(0, 60, tot)], 1).astype(np.int32)
    vals = rng.standard_normal(tot)
    qn = [3, 0, 100, 1, 2, 4, 5]
    q_ptr = np.concatenate([[0], np.cumsum(qn)]).astype(np.int64)
    qt = int(q_ptr[-1])
    q = np.stack([np.zeros(qt, int), rng.integers(0, 80, qt), rng.integers(0, 60, qt)], 1).astype(np.int32)
    model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float64)
    rows, preds = P.foldin(ctx, model, 0, torch.tensor(obs_ptr, device="cuda"), torch.tensor(obs, device="cuda"),
                           torch.tensor(vals, device="cuda"), torch.tensor(q_ptr, device="cuda"),
                           torch.tensor(q, device="cuda"), lam=LAM)
    rows, preds = rows.cpu().numpy(), preds.cpu().numpy()
    for r in range(len(counts)):
        a, b = obs_ptr[r], obs_ptr[r + 1]
        ref, _ = ora.foldin(m0.core, m0.factors, 0, obs[a:b][:, 1:], vals[a:b], LAM)
        np.testing.assert_allclose(rows[r], ref, rtol=1e-9, atol=1e-12)
        F = [np.array(ref)[None, :]] + m0.factors[1:]
        qq = q[q_ptr[r]:q_ptr[r + 1]].copy()
        qq[:, 0] = 0
        np.testing.assert_allclose(preds[q_ptr[r]:q_ptr[r + 1]], ora.predict(m0.core, F, qq), rtol=1e-9, atol=1e-12)


# ---- a8: QR finalisation ---------------------------------------------------------
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_qr_finalize_matches_oracle(ctx, ora, dtype):
    dims, J = (500, 40, 30), (5, 4, 6)
    m0 = synth.init_model(dims, J, seed=11)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    core, facs = (m0.core, m0.factors) if dtype == "f64" else (f32(m0.core), [f32(a) for a in m0.factors])
    model = P.Model.from_numpy(core, facs, dtype=tdt)
    P.qr_finalize(ctx, model)
    Gg, Fg = model.to_numpy()
    Gr, Fr = ora.qr_finalize(dims, core, facs)
    tol = 1e-9 if dtype == "f64" else 2e-4
    np.testing.assert_allclose(Gg, Gr, rtol=tol, atol=tol * np.max(np.abs(Gr)))
    for a, b in zip(Fg, Fr):
        np.testing.assert_allclose(a, b, rtol=tol, atol=tol)


# ---- a5: P-Tucker-Cache ------------------------------------------------------------
def _stepwise_check(ora, core, F0, Fg, idx, vals, g_of_mode, lam=LAM):
    """Mode n of a GPU sweep against the oracle's update of mode n from the
    state the GPU had before it (its own modes < n, the initial modes >= n),
    within the ridge bound for delta errors |E| <= g_of_mode(n) |Delta|_abs:
    each mode's own rounding, not the drift of the earlier modes."""
    N = len(F0)
    for n in range(N):
        state = [Fg[k] if k < n else F0[k] for k in range(N)]
        for i, (bd, aref) in bounds.mode_bounds(ora, core, state, idx, vals, n, lam, g_of_mode(n)).items():
            assert np.linalg.norm(Fg[n][i] - aref) <= bd + 1e-12, (n, i)


def _cache_gamma(J):
    """Rounding steps in one Cache delta of mode n: building Pres (N products),
    two per earlier mode's rescale (the ratio a_new / a_old and the product),
    the K - 1 additions of the delta sum and its one division."""
    N, K = len(J), int(np.prod(J))
    return lambda n: bounds.gamma(N + 2 * n + K // J[n] + 1)


@pytest.mark.parametrize("dims,J", [((60, 50, 40), (3, 4, 3)), ((20, 15, 10, 8), (3, 4, 2, 5)),
                                    ((8, 7, 6, 5, 4), (2, 3, 2, 3, 2)), ((40, 30, 20, 10), (6, 5, 7, 4))])
def test_cache_sweep_matches_oracle(ctx, ora, dims, J):
    """Cache sweep (Pres built, read and rescaled in FP32) against the
    oracle's Cache sweep for the totals and against the oracle's row update,
    mode by mode, within the derived bound."""
    t = synth.make_tensor(dims, 6000, J, sigma=0.1, seed=12, n_test=0)
    m0 = synth.init_model(dims, J, seed=12)
    core, F0, vals = f32(m0.core), [f32(a) for a in m0.factors], f32(t.vals)
    F0[1][::3, 1] = 0.0                               # exact zeros: plain-product fallback
    x = P.SparseObs.from_numpy(t.idx, vals, dims, dtype=torch.float32)
    sl = P.build_all_slices(ctx, x)
    mc = P.Model.from_numpy(core, F0, dtype=torch.float32)
    mp = P.Model.from_numpy(core, F0, dtype=torch.float32)
    sc = P.als_sweep(ctx, x, sl, mc, variant="cache", precision="fp32", lam=LAM)
    sp = P.als_sweep(ctx, x, sl, mp, variant="plain", precision="fp32", lam=LAM)
    _, Fc = mc.to_numpy()
    _stepwise_check(ora, core, F0, Fc, t.idx, vals, _cache_gamma(J))
    assert sc["rmse"] == pytest.approx(sp["rmse"], rel=1e-4)
    for s_ in sl:
        s_.close()


@pytest.mark.parametrize("order", [6, 8, 10])
def test_cache_high_order_matches_oracle(ctx, ora, order):
    """The order experiment's shape (Sec. 5: I_n = 100, 1000 entries, J = 3)
    at orders 6, 8 and 10, where Pres holds 3^N values per entry: the Cache
    sweep against the oracle's, mode by mode, and its error pass against the
    oracle's Cache sweep."""
    dims, J = (100,) * order, (3,) * order
    t = synth.make_tensor(dims, 1000, J, sigma=0.1, seed=order, n_test=0)
    m0 = synth.init_model(dims, J, seed=order)
    core, F0, vals = f32(m0.core), [f32(a) for a in m0.factors], f32(t.vals)
    x = P.SparseObs.from_numpy(t.idx, vals, dims, dtype=torch.float32)
    sl = P.build_all_slices(ctx, x)
    mc = P.Model.from_numpy(core, F0, dtype=torch.float32)
    sc = P.als_sweep(ctx, x, sl, mc, variant="cache", precision="fp32", lam=LAM)
    _, Fc = mc.to_numpy()
    _stepwise_check(ora, core, F0, Fc, t.idx, vals, _cache_gamma(J))
    # error pass: predictions from the last mode's Cache deltas dotted with the
    # new row (J more roundings); |x_hat error| <= g |x_hat|_abs moves the SSE
    # by at most sum(2 |r| e + e^2)
    g = _cache_gamma(J)(order - 1) + bounds.gamma(J[-1] + 1)
    pred = ora.predict(core, Fc, t.idx)
    e = g * ora.predict(np.abs(core), [np.abs(f) for f in Fc], t.idx)
    r = vals - pred
    ref = ora.error_stats(core, Fc, t.idx, vals)["rmse"]
    d_sse = float(np.sum(2 * np.abs(r) * e + e * e))
    assert abs(sc["rmse"] - ref) <= 2 * d_sse / (len(vals) * ref) + 1e-7 * ref
    for s_ in sl:
        s_.close()


# ---- a7: P-Tucker-Approx -----------------------------------------------------------
@pytest.mark.parametrize("dims,J", [((40, 30, 20), (3, 4, 2)), ((30, 25, 20), (10, 10, 10)),
                                    ((12, 10, 9, 8), (8, 8, 8, 8))])
def test_partial_error_matches_oracle(ctx, ora, dims, J):
    """u, v sums in registers (few core prefixes) and in shared memory (many)."""
    t = synth.make_tensor(dims, 3000, J, sigma=0.1, seed=13, n_test=0)
    m0 = synth.init_model(dims, J, seed=13)
    core, F0, vals = f32(m0.core), [f32(a) for a in m0.factors], f32(t.vals)
    core.reshape(-1)[5] = 0.0
    x = P.SparseObs.from_numpy(t.idx, vals, dims, dtype=torch.float32)
    model = P.Model.from_numpy(core, F0, dtype=torch.float32)
    R = P.partial_error(ctx, x, model).cpu().numpy()
    Rr = ora.partial_error(core, F0, t.idx, vals)
    np.testing.assert_allclose(R, Rr, rtol=1e-3, atol=1e-4 * np.max(np.abs(Rr)))
    assert R.reshape(-1)[5] == 0.0


@pytest.mark.parametrize("rule", ["r_beta", "magnitude"])
def test_approx_sweep_selection(ctx, ora, rule):
    """Alg. 4 inside the sweep: floor(p * nnz) entries removed; for the
    magnitude rule exactly the oracle's choice; for the R(beta) rule the
    removed entries are the largest of the oracle's FP64 scores (taken with
    the GPU's post-sweep factors and the pre-truncation core), up to swaps
    among scores within 1e-4 max|R| of the cut (the GPU sums u, v in FP32)."""
    dims, J = (50, 40, 30), (4, 3, 5)
    t = synth.make_tensor(dims, 5000, J, sigma=0.1, seed=14, n_test=0)
    m0 = synth.init_model(dims, J, seed=14)
    core, F0, vals = f32(m0.core), [f32(a) for a in m0.factors], f32(t.vals)
    x = P.SparseObs.from_numpy(t.idx, vals, dims, dtype=torch.float32)
    sl = P.build_all_slices(ctx, x)
    model = P.Model.from_numpy(core, F0, dtype=torch.float32)
    nnz = core.size
    for sweep in range(3):
        G_before = model.core.double().cpu().numpy()
        st = P.als_sweep(ctx, x, sl, model, variant="approx", precision="fp32", lam=LAM, trunc_rate=0.2,
                         trunc_rule=rule)
        Gg = model.core.double().cpu().numpy()
        k = int(np.floor(0.2 * nnz))
        nnz -= k
        assert np.count_nonzero(Gg) == nnz == st["core_nnz"]
        removed = (G_before != 0) & (Gg == 0)
        assert removed.sum() == k
        if rule == "magnitude":
            Gsel, _ = ora.truncate(G_before, None, 0.2, rule)
            assert np.array_equal(Gg != 0, Gsel != 0)
        else:
            _, F = model.to_numpy()
            Rr = ora.partial_error(G_before, F, t.idx, vals)
            live = G_before != 0
            cut = np.sort(Rr[live])[::-1][k - 1]
            tol = 1e-4 * np.max(np.abs(Rr[live]))
            assert np.all(Rr[removed] >= cut - tol)
            assert np.all(Rr[live & ~removed] <= cut + tol)

# ---- failure detection -------------------------------------------------------------
def test_bounded_wait_times_out_and_context_survives(ctx, ora):
    """A device wait that nothing completes gives up, the call reports
    PTK_ERR_TIMEOUT, and the same context then computes correctly."""
    from paper_1710_02261_gb300 import _ffi
    assert P.selftest_wait(ctx, 4096) == _ffi.ERR_TIMEOUT
    dims, J = (20, 15, 10), (3, 4, 2)
    t = synth.make_tensor(dims, 500, J, sigma=0.1, seed=21, n_test=0)
    m0 = synth.init_model(dims, J, seed=21)
    core, F0 = f32(m0.core), [f32(a) for a in m0.factors]
    model = P.Model.from_numpy(core, F0, dtype=torch.float32)
    got = P.predict(ctx, model, torch.tensor(t.idx, device="cuda")).double().cpu().numpy()
    np.testing.assert_allclose(got, ora.predict(core, F0, t.idx), rtol=1e-5, atol=1e-5)
