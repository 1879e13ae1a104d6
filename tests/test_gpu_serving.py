"""Continuous-batching fold-in server (ptk_server_*) through the C ABI.

A request is a new slice of one mode: its row is the row update of
Eq. (rowupdate) with G and the other factors fixed, and its query
coordinates are predicted by Eq. (recon2).  The server batches requests as
they arrive; each request's arithmetic does not depend on its batch, so its
row and predictions are bit-identical alone and in any mix.
"""
import threading
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


def _model(dtype):
    m0 = synth.init_model(DIMS, J, seed=5)
    core = np.asarray(m0.core, dtype=np.float64)
    F = [np.asarray(a, dtype=np.float64) for a in m0.factors]
    if dtype == torch.float32:
        core = core.astype(np.float32).astype(np.float64)
        F = [a.astype(np.float32).astype(np.float64) for a in F]
    return core, F, P.Model.from_numpy(core, F, dtype=dtype)


def _requests(count, seed, lo=5, hi=5000, nq=100):
    """log-uniform observed-entry counts in [lo, hi]; values N(0, 1)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        oi = np.stack([rng.integers(0, d, size=m) for d in DIMS], axis=1).astype(np.int32)
        ov = rng.standard_normal(m)
        qi = np.stack([rng.integers(0, d, size=nq) for d in DIMS], axis=1).astype(np.int32)
        out.append((oi, ov, qi))
    return out


def _serve(server, reqs, *, stagger_s=0.0):
    tickets = []
    for oi, ov, qi in reqs:
        tickets.append(server.submit(oi, ov, qi))
        if stagger_s:
            time.sleep(stagger_s)
    return [server.wait(t, nq) for t, nq in tickets]


@pytest.mark.parametrize("dtype,prec", [(torch.float64, "fp64"), (torch.float32, "fp32"), (torch.float32, "bf16")])
def test_alone_equals_mixed_bitwise(dtype, prec):
    core, F, model = _model(dtype)
    reqs = _requests(24, seed=11)
    with_alone = P.Server(model, 0, lam=LAM, precision=prec, max_batch_requests=1, slots=1)
    try:
        alone = [_serve(with_alone, [r])[0] for r in reqs]
    finally:
        with_alone.close()
    mixed_srv = P.Server(model, 0, lam=LAM, precision=prec, max_batch_requests=16, max_batch_entries=20000,
                         slots=3)
    try:
        mixed = _serve(mixed_srv, reqs)
        st = mixed_srv.stats()
    finally:
        mixed_srv.close()
    assert st["completed"] == len(reqs)
    assert st["batches"] < len(reqs)  # requests did share batches
    for (ra, pa, _), (rm, pm, _) in zip(alone, mixed):
        assert np.array_equal(ra.view(np.uint8), rm.view(np.uint8))
        assert np.array_equal(pa.view(np.uint8), pm.view(np.uint8))


def test_rows_and_predictions_match_oracle(ora):
    """FP64 server against the oracle's fold-in row and prediction."""
    core, F, model = _model(torch.float64)
    reqs = _requests(12, seed=12)
    srv = P.Server(model, 0, lam=LAM, precision="fp64", max_batch_requests=8, slots=2)
    try:
        res = _serve(srv, reqs)
    finally:
        srv.close()
    for (oi, ov, qi), (row, preds, lat) in zip(reqs, res):
        ref_row, rc = ora.foldin(core, F, 0, oi, ov, LAM)
        assert rc == 0
        assert np.allclose(row, ref_row, rtol=1e-9, atol=1e-11), np.max(np.abs(row - ref_row))
        Fq = list(F)
        Fq[0] = ref_row[None, :]
        q = qi.copy()
        q[:, 0] = 0
        ref_pred = ora.predict(core, Fq, q)
        assert np.allclose(preds, ref_pred, rtol=1e-9, atol=1e-9 * np.max(np.abs(ref_pred)))
        assert lat >= 0.0


def test_fp32_rows_within_conditioning_bound(ora):
    """FP32 fold-in rows against the oracle's, within the first-order ridge
    perturbation bound of an FP32 delta (|E| <= gamma_{K+N} |Delta|_abs,
    tests/bounds.py), short requests (rank-deficient rows) included."""
    core, F, model = _model(torch.float32)
    reqs = _requests(8, seed=13, lo=5, hi=2000)
    srv = P.Server(model, 0, lam=LAM, precision="fp32", slots=2)
    try:
        res = _serve(srv, reqs)
    finally:
        srv.close()
    g = bounds.gamma(J[1] * J[2] + len(J))
    for (oi, ov, qi), (row, preds, _) in zip(reqs, res):
        x = ov.astype(np.float32).astype(np.float64)
        ref_row, _ = ora.foldin(core, F, 0, oi, x, LAM)
        D, Da = bounds.row_delta(ora, core, F, 0, oi, range(len(oi)))
        bd, a = bounds.ridge_bound(D, Da, x, LAM, g)
        # the bound's own FP64 row is the oracle's (up to FP64 rounding of a rank-deficient system)
        assert np.linalg.norm(a - ref_row) <= 1e-6 * np.linalg.norm(ref_row)
        assert np.linalg.norm(row - ref_row) <= bd + 1e-12, (len(oi), np.linalg.norm(row - ref_row), bd)


def test_requests_arriving_during_flight_are_served():
    """Submissions from another thread while batches are on the GPU; every
    ticket completes and later batches hold more than one request."""
    _, _, model = _model(torch.float32)
    reqs = _requests(64, seed=14)
    srv = P.Server(model, 0, lam=LAM, precision="fp32", max_batch_requests=32, slots=2)
    out = {}
    try:
        def producer():
            for i, r in enumerate(reqs):
                out[i] = srv.submit(*r)
                time.sleep(0.0002)
        th = threading.Thread(target=producer)
        th.start()
        th.join()
        res = [srv.wait(*out[i]) for i in range(len(reqs))]
        st = srv.stats()
    finally:
        srv.close()
    assert len(res) == len(reqs) and st["completed"] == len(reqs)
    assert st["max_inflight_bytes"] > 0


def test_admission_refuses_over_cap_and_full_queue():
    _, _, model = _model(torch.float32)
    (oi, ov, qi), = _requests(1, seed=15, lo=4000, hi=4001)
    srv = P.Server(model, 0, lam=LAM, precision="fp32", memory_cap_bytes=4096, slots=1)
    try:
        with pytest.raises(P.PtkError) as e:
            srv.submit(oi, ov, qi)
        assert "BUSY" in str(e.value) or "cap" in str(e.value)
        assert srv.stats()["rejected"] == 1
    finally:
        srv.close()
    srv = P.Server(model, 0, lam=LAM, precision="fp32", slots=1)
    try:
        with pytest.raises(P.PtkError):
            bad = oi.copy()
            bad[0, 1] = DIMS[1]
            srv.submit(bad, ov, qi)
        t = srv.submit(oi[:0], ov[:0], qi)  # an empty slice: the zero row (lambda > 0)
        row, preds, _ = srv.wait(*t)
        assert np.all(row == 0) and np.all(preds == 0)
    finally:
        srv.close()
