"""Delta of Eq. (delta) from a truncated core (P-Tucker-Approx, Sec. 3.3).

After truncation most core entries are zero, and an Approx sweep has the
CUDA-core delta walk only the non-zeros (compacted per mode into records
ordered by j_n) when that is cheaper than the dense contraction (below about
15 % of the core at order 3, 10 % at order 4, 8 % at order 5).  The factor
update of a sweep
uses the core as it stands, truncation follows after it, so the factors after
one Approx sweep are those of a plain sweep with the same core: every row is
compared with the FP64 oracle's row update (on the FP32-rounded inputs)
within the first-order ridge bound of an FP32 delta (tests/bounds.py).  The
launch counts show which path ran.  (Approx runs on FP32 models.)
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


def _case(dims, J, E, density, seed):
    t = synth.make_tensor(dims, E, J, dist="uniform", sigma=0.1, seed=seed, n_test=0)
    m0 = synth.init_model(dims, J, seed=seed)
    rng = np.random.default_rng(seed + 100)
    core = np.array(m0.core, dtype=np.float64)
    core[rng.random(core.shape) >= density] = 0.0
    return t, core, [np.asarray(a, dtype=np.float64) for a in m0.factors]


def _approx_sweep(ctx, t, core, F, dtype, precision):
    x = P.SparseObs.from_numpy(t.idx, t.vals, t.dims, dtype=dtype)
    sl = P.build_all_slices(ctx, x, dtype=dtype)
    model = P.Model.from_numpy(core, F, dtype=dtype)
    torch.cuda.synchronize()
    l0 = P.launch_count()
    P.als_sweep(ctx, x, sl, model, variant="approx", precision=precision, lam=LAM, trunc_rate=0.01,
                trunc_rule="magnitude")
    launches = P.launch_count() - l0
    _, Fg = model.to_numpy()
    for s in sl:
        s.close()
    return Fg, launches


def _f32_case(dims, J, E, density, seed):
    t, core, F = _case(dims, J, E, density, seed)
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)  # noqa: E731
    t.vals = f32(t.vals)
    return t, f32(core), [f32(a) for a in F]


def _check_rows(ora, t, core, F, Fg, J):
    """Mode by mode (the sweep is Gauss-Seidel over modes): every row of the
    GPU's factor against the oracle's update from the same state."""
    K = int(np.prod(J))
    N = len(J)
    for n in range(N):
        state = [Fg[k] if k < n else F[k] for k in range(N)]
        g = bounds.gamma(K // J[n] + N)
        for i, (bd, aref) in bounds.mode_bounds(ora, core, state, t.idx, t.vals, n, LAM, g).items():
            assert np.linalg.norm(Fg[n][i] - aref) <= bd + 1e-12, (n, i)


@pytest.mark.parametrize("dims,J,E", [
    ((40, 30, 20), (6, 5, 4), 3001),              # order 3, unequal ranks, ragged tail
    ((25, 20, 15, 12), (5, 4, 6, 3), 4999),       # order 4
    ((12, 10, 9, 8, 7), (3, 4, 2, 5, 3), 2500),   # order 5: two outer middle modes
    ((30, 20, 10), (16, 12, 10), 1500),           # the widest rank the kernel takes
])
@pytest.mark.parametrize("density", [0.04, 0.0])
def test_sparse_core_sweep_matches_oracle(ctx, ora, dims, J, E, density):
    t, core, F = _f32_case(dims, J, E, density, seed=11)
    Fg, _ = _approx_sweep(ctx, t, core, F, torch.float32, "fp32")
    if density == 0.0:  # no core entries: every delta, and so every row, is zero
        assert all(np.all(a == 0.0) for a in Fg)
    _check_rows(ora, t, core, F, Fg, J)


def test_sparse_path_taken_below_the_density_threshold(ctx, ora):
    """One more launch per mode (the compaction) when the core is sparse
    enough, the dense kernel otherwise; both within the oracle's bound."""
    dims, J, E = (40, 30, 20), (6, 5, 4), 3001
    t, sparse_core, F = _f32_case(dims, J, E, 0.1, seed=12)
    _, dense_core, _ = _f32_case(dims, J, E, 0.9, seed=12)
    Fs, ls = _approx_sweep(ctx, t, sparse_core, F, torch.float32, "fp32")
    Fd, ld = _approx_sweep(ctx, t, dense_core, F, torch.float32, "fp32")
    assert ls - ld == len(dims), (ls, ld)
    _check_rows(ora, t, sparse_core, F, Fs, J)
    _check_rows(ora, t, dense_core, F, Fd, J)


@pytest.mark.parametrize("dims,J,E", [
    ((50, 40, 30), (10, 8, 6), 6000),             # order 3
    ((30, 25, 20, 15), (6, 5, 4, 6), 8000),       # order 4
    ((14, 12, 10, 9, 8), (4, 3, 5, 3, 4), 5000),  # order 5
])
def test_sparse_r_beta_selection(ctx, ora, dims, J, E):
    """Alg. 4 with the R(beta) rule on a core at 10 % density: u, v are summed
    over the non-zero core entries only (one more launch, the compaction,
    than with the dense pass; the sparse delta walk adds one per mode).  The
    removed entries are floor(p nnz) of the largest oracle FP64 scores (the
    GPU's post-sweep factors, the pre-truncation core), up to swaps among
    scores within 1e-4 max|R| of the cut (the GPU sums u, v in FP32)."""
    t, core, F = _f32_case(dims, J, E, 0.1, seed=15)
    x = P.SparseObs.from_numpy(t.idx, t.vals, dims, dtype=torch.float32)
    sl = P.build_all_slices(ctx, x)
    model = P.Model.from_numpy(core, F, dtype=torch.float32)
    nnz = int(np.count_nonzero(core))
    G_before = model.core.double().cpu().numpy()
    st = P.als_sweep(ctx, x, sl, model, variant="approx", precision="fp32", lam=LAM, trunc_rate=0.2,
                     trunc_rule="r_beta")
    Gg = model.core.double().cpu().numpy()
    k = int(np.floor(0.2 * nnz))
    assert np.count_nonzero(Gg) == nnz - k == st["core_nnz"]
    removed = (G_before != 0) & (Gg == 0)
    assert removed.sum() == k
    _, Fg = model.to_numpy()
    Rr = ora.partial_error(G_before, Fg, t.idx, t.vals)
    live = G_before != 0
    cut = np.sort(Rr[live])[::-1][k - 1]
    tol = 1e-4 * np.max(np.abs(Rr[live]))
    assert np.all(Rr[removed] >= cut - tol)
    assert np.all(Rr[live & ~removed] <= cut + tol)
    for s in sl:
        s.close()
