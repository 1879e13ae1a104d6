"""The local step of a row-sharded sweep on the GPU (ptk_als_mode).

A rank updates its own rows of one mode from its own entries.  With every
rank run in turn on one GPU (no rank waits on another: the rows of a mode are
disjoint and none of them is read by that mode's update), the result is the
unsharded sweep's: compared with ptk_als_sweep on the same data and with the
FP64 oracle.  The exchange between processes is
covered on CPU ranks (tests/test_shard.py); a single-rank RowShardedSweep
with the CUDA backend reproduces ptk_als_sweep bit for bit.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1710_02261_gb300 as P  # noqa: E402
from paper_1710_02261_gb300.shard import CudaRows, RowShardedSweep, ShardPlan  # noqa: E402

LAM = 0.01


@pytest.fixture(scope="module")
def ctx():
    c = P.Context(0)
    yield c
    c.close()


def _case(dims, J, E, seed):
    t = synth.make_tensor(dims, E, J, dist=[("zipf", 1.1)] + ["uniform"] * (len(dims) - 1), sigma=0.1, seed=seed,
                          n_test=0)
    return t, synth.init_model(dims, J, seed=seed)


@pytest.mark.parametrize("world", [2, 3, 5])
def test_ranks_in_turn_equal_the_unsharded_sweep(ctx, ora, world):
    dims, J = (60, 40, 3), (4, 3, 2)          # mode 3 has fewer rows than some worlds have ranks
    t, m0 = _case(dims, J, 4000, 7)
    plans = [ShardPlan(dims, t.idx, r, world) for r in range(world)]
    sharded = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float64)
    locals_ = []
    for r in range(world):
        xs, ss = [], []
        for n in range(len(dims)):
            ent = plans[r].entries[n]
            x = P.SparseObs.from_numpy(t.idx[ent], t.vals[ent], dims, dtype=torch.float64)
            xs.append(x)
            ss.append(P.build_mode_slices(ctx, x, n, dtype=torch.float64))
        locals_.append((xs, ss))
    for _ in range(2):
        for n in range(len(dims)):
            for r in range(world):
                lo, hi = plans[r].own(n)
                xs, ss = locals_[r]
                P.als_mode(ctx, xs[n], ss[n], sharded, n, lo, hi, precision="fp64", lam=LAM)
    x = P.SparseObs.from_numpy(t.idx, t.vals, dims, dtype=torch.float64)
    sl = P.build_all_slices(ctx, x, dtype=torch.float64)
    whole = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float64)
    for _ in range(2):
        P.als_sweep(ctx, x, sl, whole, precision="fp64", lam=LAM)
    _, Fs = sharded.to_numpy()
    _, Fw = whole.to_numpy()
    F = m0.factors
    for _ in range(2):
        F, _ = ora.sweep(dims, m0.core, F, t.idx, t.vals, LAM)
    # FP64: the sharded and whole sweeps sum some rows in other orders (the row
    # sums' schedule is chosen per layout), so they agree to rounding, and both
    # agree with the oracle as the FP64 parity tests require
    for a, b, c in zip(Fs, Fw, F):
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-11)
        np.testing.assert_allclose(a, c, rtol=1e-8, atol=1e-10)
    for xs, ss in locals_:
        for s in ss:
            s.close()
    for s in sl:
        s.close()


def test_single_rank_cuda_backend_is_the_sweep(ctx):
    dims, J = (500, 300, 30, 24), (6, 6, 6, 6)
    t, m0 = _case(dims, J, 60000, 9)
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)  # noqa: E731
    core, F0, vals = f32(m0.core), [f32(a) for a in m0.factors], f32(t.vals)
    plan = ShardPlan(dims, t.idx, 0, 1)
    model = P.Model.from_numpy(core, F0, dtype=torch.float32)
    be = CudaRows(ctx, plan, t.idx, vals, model, precision="tf32", lam=LAM)
    sse = RowShardedSweep(plan, be).sweep()
    x = P.SparseObs.from_numpy(t.idx, vals, dims, dtype=torch.float32)
    sl = P.build_all_slices(ctx, x)
    whole = P.Model.from_numpy(core, F0, dtype=torch.float32)
    st = P.als_sweep(ctx, x, sl, whole, precision="tf32", lam=LAM)
    for a, b in zip(model.factors, whole.factors):
        assert torch.equal(a, b)
    # the sharded error is ptk_error over the entries (its own FP32 deltas);
    # the sweep's error pass reuses the last mode's TF32 deltas
    assert sse == pytest.approx(P.error(ctx, x, whole, LAM)["sse"], rel=1e-9)
    assert sse == pytest.approx(st["sse"], rel=1e-3)
    be.close()
    for s in sl:
        s.close()
