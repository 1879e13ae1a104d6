"""Fold-in server with the request loop on the GPU (ptk_dserver_*).

Each request is a new slice of one mode (Theorem 1: the row update of
Eq. rowupdate with G and the other factors fixed) plus predictions of its
query coordinates (Eq. recon2).  Persistent CTAs take the requests from a ring
in mapped host memory; one CTA computes a whole request, so a request's
result bits are the same alone and in any mix.
"""
import time

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
DIMS = (1000, 1000, 1000)
J = (10, 10, 10)


def _model(dtype, J=J, dims=DIMS, seed=5):
    m0 = synth.init_model(dims, J, seed=seed)
    core = np.asarray(m0.core, dtype=np.float64)
    F = [np.asarray(a, dtype=np.float64) for a in m0.factors]
    if dtype == torch.float32:
        core = core.astype(np.float32).astype(np.float64)
        F = [a.astype(np.float32).astype(np.float64) for a in F]
    return core, F, P.Model.from_numpy(core, F, dtype=dtype)


def _requests(count, seed, lo=5, hi=5000, nq=100, dims=DIMS):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        oi = np.stack([rng.integers(0, d, size=m) for d in dims], axis=1).astype(np.int32)
        ov = rng.standard_normal(m)
        qi = np.stack([rng.integers(0, d, size=nq) for d in dims], axis=1).astype(np.int32)
        out.append((oi, ov, qi))
    return out


def _serve(srv, reqs):
    tickets = [srv.submit(*r) for r in reqs]
    return [srv.wait(t, nq) for t, nq in tickets]


def test_rows_and_predictions_match_oracle(ora):
    core, F, model = _model(torch.float64)
    reqs = _requests(12, seed=21)
    srv = P.DeviceServer(model, 0, lam=LAM, workers=8)
    try:
        res = _serve(srv, reqs)
    finally:
        srv.close()
    for (oi, ov, qi), (row, preds, lat) in zip(reqs, res):
        ref_row, rc = ora.foldin(core, F, 0, oi, ov, LAM)
        assert rc == 0
        np.testing.assert_allclose(row, ref_row, rtol=1e-9, atol=1e-11)
        Fq = list(F)
        Fq[0] = ref_row[None, :]
        q = qi.copy()
        q[:, 0] = 0
        ref_pred = ora.predict(core, Fq, q)
        np.testing.assert_allclose(preds, ref_pred, rtol=1e-9, atol=1e-9 * np.max(np.abs(ref_pred)))
        assert lat >= 0.0


def test_other_mode_and_order_match_oracle(ora):
    """A 4-order model with uneven ranks, requests for mode 2."""
    dims, Jm = (50, 40, 30, 20), (4, 6, 3, 5)
    core, F, model = _model(torch.float64, J=Jm, dims=dims, seed=6)
    reqs = _requests(6, seed=22, hi=800, nq=17, dims=dims)
    srv = P.DeviceServer(model, 2, lam=LAM, workers=3, max_queries=32)
    try:
        res = _serve(srv, reqs)
    finally:
        srv.close()
    for (oi, ov, qi), (row, preds, _) in zip(reqs, res):
        ref_row, rc = ora.foldin(core, F, 2, oi, ov, LAM)
        np.testing.assert_allclose(row, ref_row, rtol=1e-9, atol=1e-11)
        Fq = list(F)
        Fq[2] = ref_row[None, :]
        q = qi.copy()
        q[:, 2] = 0
        np.testing.assert_allclose(preds, ora.predict(core, Fq, q), rtol=1e-9, atol=1e-11)


def test_alone_equals_mixed_bitwise():
    _, _, model = _model(torch.float32)
    reqs = _requests(24, seed=23)
    srv = P.DeviceServer(model, 0, lam=LAM)
    try:
        alone = [_serve(srv, [r])[0] for r in reqs]     # one at a time
        mixed = _serve(srv, reqs)                        # all at once, on many CTAs
        st = srv.stats()
    finally:
        srv.close()
    assert st["completed"] == 2 * len(reqs) and st["bad_rows"] == 0
    for (ra, pa, _), (rm, pm, _) in zip(alone, mixed):
        assert np.array_equal(ra.view(np.uint8), rm.view(np.uint8))
        assert np.array_equal(pa.view(np.uint8), pm.view(np.uint8))


def test_fp32_rows_within_conditioning_bound(ora):
    core, F, model = _model(torch.float32)
    reqs = _requests(8, seed=24, lo=5, hi=2000)
    srv = P.DeviceServer(model, 0, lam=LAM)
    try:
        res = _serve(srv, reqs)
    finally:
        srv.close()
    g = bounds.gamma(J[1] * J[2] + len(J))
    for (oi, ov, qi), (row, preds, _) in zip(reqs, res):
        x = ov.astype(np.float32).astype(np.float64)
        ref_row, _ = ora.foldin(core, F, 0, oi, x, LAM)
        D, Da = bounds.row_delta(ora, core, F, 0, oi, range(len(oi)))
        bd, _ = bounds.ridge_bound(D, Da, x, LAM, g)
        assert np.linalg.norm(row - ref_row) <= bd + 1e-12, (len(oi), np.linalg.norm(row - ref_row), bd)


def test_idle_loop_leaves_and_comes_back():
    """With no work for idle_ms every CTA leaves (a bounded wait, counted);
    the next request relaunches the loop and is served."""
    _, _, model = _model(torch.float32)
    reqs = _requests(2, seed=25, hi=300)
    srv = P.DeviceServer(model, 0, lam=LAM, workers=4, idle_ms=10.0)
    try:
        first = _serve(srv, reqs[:1])[0]
        t0 = time.perf_counter()
        while srv.stats()["running"] and time.perf_counter() - t0 < 10.0:
            time.sleep(0.01)
        st = srv.stats()
        assert st["running"] == 0 and st["idle_exits"] == 4 and st["launches"] == 1
        second = _serve(srv, reqs[1:])[0]
        st = srv.stats()
        assert st["launches"] == 2 and st["completed"] == 2
    finally:
        srv.close()
    assert first[0].shape == (10,) and second[0].shape == (10,)


def test_arena_admission_and_oversized_request():
    """A 256 KiB arena holds a few requests at a time: thirty are admitted in
    turn as earlier ones finish; one larger than the arena is refused."""
    _, _, model = _model(torch.float32)
    reqs = _requests(30, seed=26, lo=1000, hi=3000, nq=20)
    srv = P.DeviceServer(model, 0, lam=LAM, arena_bytes=256 << 10, ring=8, max_queries=32)
    try:
        res = _serve(srv, reqs)
        assert all(r[0].shape == (10,) for r in res)
        big = _requests(1, seed=27, lo=30000, hi=30001, nq=1)[0]
        with pytest.raises(P.PtkError) as e:
            srv.submit(*big)
        assert e.value.status == P.F.ERR_BUSY
        assert srv.stats()["completed"] == 30
    finally:
        srv.close()


def test_empty_request_gives_zero_row():
    _, _, model = _model(torch.float32)
    srv = P.DeviceServer(model, 0, lam=LAM, workers=2)
    try:
        qi = np.zeros((3, 3), dtype=np.int32)
        row, preds, _ = _serve(srv, [(np.zeros((0, 3), np.int32), np.zeros(0), qi)])[0]
    finally:
        srv.close()
    assert np.all(row == 0) and np.all(preds == 0)
