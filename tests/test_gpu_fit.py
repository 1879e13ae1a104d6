"""Alg. 2's driver (ptk_fit) on one and on many independent problems.

Each problem's arithmetic does not depend on the lane it runs on or on
whether sweeps 2.. run inside a CUDA graph with a device-side loop, so a
batched fit must reproduce, bit for bit, the same problem fitted alone and
eagerly; FP64 fits follow the oracle's Alg. 2 (errors per sweep, the
stopping rule, the QR finalisation) to rounding.
"""
import numpy as np
import pytest

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


# uneven orders, sizes, ranks and entry counts (the batched workload's ranges, scaled down)
SHAPES = [((60, 50, 40), 3000, 4), ((30, 20, 10, 12), 5000, 3), ((9, 8, 7, 6, 5), 2000, 2), ((200, 150, 30), 20000, 5),
          ((40, 30, 20, 10), 8000, 6), ((500, 400, 300), 1500, 3)]


def _problem(ctx, dims, E, J, seed, dtype):
    t = synth.make_tensor(dims, E, (J,) * len(dims), seed=seed, n_test=0)
    m0 = synth.init_model(dims, (J,) * len(dims), seed=seed)
    if dtype == torch.float32:
        core = m0.core.astype(np.float32).astype(np.float64)
        F = [a.astype(np.float32).astype(np.float64) for a in m0.factors]
        vals = t.vals.astype(np.float32).astype(np.float64)
    else:
        core, F, vals = m0.core, m0.factors, t.vals
    x = P.SparseObs.from_numpy(t.idx, vals, dims, dtype=dtype)
    sl = P.build_all_slices(ctx, x, dtype=dtype)
    model = P.Model.from_numpy(core, F, dtype=dtype)
    return dict(t=t, core=core, F=F, vals=vals, x=x, sl=sl, model=model)


def _bits(model):
    core, F = model.to_numpy()
    return [core.copy()] + [a.copy() for a in F]


def _same_bits(a, b):
    return all(np.array_equal(u.view(np.uint64), v.view(np.uint64)) for u, v in zip(a, b))


@pytest.mark.parametrize("dtype,prec", [(torch.float64, "fp64"), (torch.float32, "fp32"), (torch.float32, "bf16")])
def test_batched_equals_alone_bitwise(ctx, dtype, prec):
    alone = []
    for i, (dims, E, J) in enumerate(SHAPES):
        pr = _problem(ctx, dims, E, J, 40 + i, dtype)
        errs = P.fit(ctx, pr["x"], pr["sl"], pr["model"], precision=prec, lam=LAM, max_sweeps=4, graphs=False)
        alone.append((errs, _bits(pr["model"])))
    probs = [_problem(ctx, dims, E, J, 40 + i, dtype) for i, (dims, E, J) in enumerate(SHAPES)]
    errs = P.fit_many(ctx, [(p["x"], p["sl"], p["model"]) for p in probs], precision=prec, lam=LAM, max_sweeps=4,
                      lanes=4, graphs=True)
    for (ea, ba), eb, p in zip(alone, errs, probs):
        assert len(eb) == 4
        assert np.array_equal(np.array(ea), np.array(eb))
        assert _same_bits(ba, _bits(p["model"]))


def test_fp64_fit_follows_oracle(ctx, ora):
    dims, E, J = (60, 50, 40), 3000, 4
    pr = _problem(ctx, dims, E, J, 7, torch.float64)
    errs = P.fit(ctx, pr["x"], pr["sl"], pr["model"], precision="fp64", lam=LAM, max_sweeps=5, finalize_qr=True)
    G, Fo, eo = ora.fit(dims, pr["core"], pr["F"], pr["t"].idx, pr["vals"], LAM, sweeps=5, finalize=True)
    assert np.allclose(errs, eo, rtol=1e-9)
    core, F = pr["model"].to_numpy()
    assert np.allclose(core, G, rtol=1e-7, atol=1e-9 * np.abs(G).max())
    for a, b in zip(F, Fo):
        assert np.allclose(a, b, rtol=1e-7, atol=1e-9)


def test_tolerance_stops_on_device_like_the_oracle(ctx, ora):
    dims, E, J = (30, 20, 10, 12), 5000, 3
    tol = 1e-3
    pr = _problem(ctx, dims, E, J, 9, torch.float64)
    errs = P.fit(ctx, pr["x"], pr["sl"], pr["model"], precision="fp64", lam=LAM, max_sweeps=40, tol=tol)
    _, _, eo = ora.fit(dims, pr["core"], pr["F"], pr["t"].idx, pr["vals"], LAM, sweeps=40, tol=tol)
    assert len(errs) == len(eo) < 40
    assert np.allclose(errs, eo, rtol=1e-9)
    # the eager driver applies the same rule on the host
    pr2 = _problem(ctx, dims, E, J, 9, torch.float64)
    errs2 = P.fit(ctx, pr2["x"], pr2["sl"], pr2["model"], precision="fp64", lam=LAM, max_sweeps=40, tol=tol,
                  graphs=False)
    assert np.array_equal(np.array(errs), np.array(errs2))


def test_batched_launch_count_covers_graph_replays(ctx):
    probs = [_problem(ctx, dims, E, J, 60 + i, torch.float32) for i, (dims, E, J) in enumerate(SHAPES[:3])]
    l0 = P.launch_count()
    P.fit_many(ctx, [(p["x"], p["sl"], p["model"]) for p in probs], lam=LAM, max_sweeps=1, lanes=2)
    one = P.launch_count() - l0
    probs = [_problem(ctx, dims, E, J, 60 + i, torch.float32) for i, (dims, E, J) in enumerate(SHAPES[:3])]
    l0 = P.launch_count()
    P.fit_many(ctx, [(p["x"], p["sl"], p["model"]) for p in probs], lam=LAM, max_sweeps=3, lanes=2)
    three = P.launch_count() - l0
    # sweeps 2 and 3 add two loop bodies and one arm kernel per problem
    assert three > 2 * one


def test_autotuned_batch_equals_alone_bitwise(ctx):
    """FP32: the tuned launch shapes (chunk, blocks per SM) leave every
    problem's arithmetic unchanged."""
    shapes = SHAPES[:3] + [((12, 10, 9, 8), 3000, 16), ((6, 5, 4, 5, 6), 2000, 8)]
    alone = []
    P.autotune_clear(ctx)
    for i, (dims, E, J) in enumerate(shapes):
        pr = _problem(ctx, dims, E, J, 80 + i, torch.float32)
        P.fit(ctx, pr["x"], pr["sl"], pr["model"], lam=LAM, max_sweeps=2, graphs=False)
        alone.append(_bits(pr["model"]))
    probs = [_problem(ctx, dims, E, J, 80 + i, torch.float32) for i, (dims, E, J) in enumerate(shapes)]
    P.fit_many(ctx, [(p["x"], p["sl"], p["model"]) for p in probs], lam=LAM, max_sweeps=2, lanes=3, autotune=True)
    for a, p in zip(alone, probs):
        assert _same_bits(a, _bits(p["model"]))
    P.autotune_clear(ctx)
