"""The delta contraction (Eq. delta) on CUDA cores and on tcgen05 tensor cores
against the FP64 oracle, through the C ABI (ptk_delta, ptk_als_sweep).

Tensor-core bound: with operands rounded to a format of unit roundoff u
(BF16 2^-9, TF32 2^-11, both rounded to nearest) and FP32 accumulation,
|delta_tc - delta| <= 2u * sum_beta |G_beta| prod |a| + FP32 terms, i.e. the
oracle's delta of |G| and |A^(k)| scaled by 2u (tested with a 1.25 margin).
BF16x3 splits each operand into BF16 high and low parts (a = hi + lo within
2^-18 |a|) and keeps hi*hi + hi*lo + lo*hi, so u = 2^-16 covers it.
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
U = {"bf16": 2.0 ** -9, "tf32": 2.0 ** -11, "bf16x3": 2.0 ** -16, "fp32": 2.0 ** -24}


@pytest.fixture(scope="module")
def ctx():
    c = P.Context(0)
    yield c
    c.close()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _case(dims, J, n, seed):
    rng = np.random.default_rng(seed)
    core = f32(rng.standard_normal(J))
    F = [f32(rng.random((d, j))) for d, j in zip(dims, J)]
    idx = np.stack([rng.integers(0, d, size=n) for d in dims], axis=1).astype(np.int32)
    return core, F, idx


SHAPES = [((50, 40, 30), (10, 10, 10)), ((30, 20, 10, 12), (10, 10, 10, 10)), ((20, 20, 20), (5, 5, 5)),
          ((9, 8, 7, 6, 5), (4, 4, 4, 4, 4)), ((40, 30, 20, 10), (11, 11, 11, 11)), ((30, 30, 30), (3, 3, 3)),
          ((10, 11, 12, 13), (6, 6, 6, 6)), ((8, 9, 10, 11, 12), (5, 5, 5, 5, 5))]


@pytest.mark.parametrize("dims,J", SHAPES)
@pytest.mark.parametrize("prec", ["bf16", "tf32", "bf16x3", "fp32"])
def test_delta_matches_oracle(ctx, ora, dims, J, prec):
    n = 300                                     # 2 full tiles of 128 and a ragged one
    core, F, idx = _case(dims, J, n, 7)
    model = P.Model.from_numpy(core, F, dtype=torch.float32)
    coords = torch.tensor(idx, device="cuda")
    for mode in range(len(dims)):
        got = P.delta(ctx, model, mode, coords, precision=prec).double().cpu().numpy()
        ref = np.stack([ora.delta(core, F, idx[e], mode) for e in range(n)])
        mag = np.stack([ora.delta(np.abs(core), F, idx[e], mode) for e in range(n)])
        u = U[prec] if (prec == "fp32" or P.tc_available(model, prec)) else U["fp32"]
        bound = 2.5 * u * mag + 64 * 2.0 ** -24 * mag
        assert np.all(np.abs(got - ref) <= bound + 1e-30), (mode, np.max(np.abs(got - ref) / (mag + 1e-30)))


def test_tc_path_is_taken_for_the_benchmark_shape(ctx):
    core = np.ones((10, 10, 10, 10))
    F = [np.ones((5, 10)) for _ in range(4)]
    model = P.Model.from_numpy(core, F, dtype=torch.float32)
    assert P.tc_available(model, "bf16") and P.tc_available(model, "tf32") and P.tc_available(model, "bf16x3")


@pytest.mark.parametrize("prec", ["bf16", "tf32", "bf16x3"])
def test_tc_delta_large_n_against_fp32(ctx, prec):
    """Many tiles across many CTAs: the tensor-core delta stays within its
    bound of the CUDA-core FP32 delta (which the oracle pins above)."""
    dims, J = (3000, 2000, 30, 24), (10, 10, 10, 10)
    core, F, idx = _case(dims, J, 200_000, 3)
    model = P.Model.from_numpy(core, F, dtype=torch.float32)
    absm = P.Model.from_numpy(np.abs(core), F, dtype=torch.float32)
    coords = torch.tensor(idx, device="cuda")
    for mode in range(4):
        a = P.delta(ctx, model, mode, coords, precision=prec).double()
        b = P.delta(ctx, model, mode, coords, precision="fp32").double()
        mag = P.delta(ctx, absm, mode, coords, precision="fp32").double()
        assert bool(torch.all((a - b).abs() <= 2.5 * U[prec] * mag + 1e-6 * mag))


def _rmse_case(dims, E, dist, seed, sweeps, prec, ctx, ora):
    J = (10, 10, 10, 10)
    t = synth.make_tensor(dims, E, J, dist=dist, seed=seed, n_test=E // 10)
    m0 = synth.init_model(dims, J, seed=seed)
    core, F0, vals = f32(m0.core), [f32(a) for a in m0.factors], f32(t.vals)
    x = P.SparseObs.from_numpy(t.idx, vals, dims, dtype=torch.float32)
    sl = P.build_all_slices(ctx, x)
    model = P.Model.from_numpy(core, F0, dtype=torch.float32)
    assert P.tc_available(model, prec)
    Fr = F0
    for _ in range(sweeps):
        P.als_sweep(ctx, x, sl, model, precision=prec, lam=LAM)
        Fr, _ = ora.sweep(dims, core, Fr, t.idx, vals, LAM, nthreads=ora.max_threads())
    xt = P.SparseObs.from_numpy(t.test_idx, t.test_vals, dims, dtype=torch.float32)
    got = P.error(ctx, xt, model, LAM)["rmse"]
    ref = ora.error_stats(core, Fr, t.test_idx, t.test_vals)["rmse"]
    for s_ in sl:
        s_.close()
    return got, ref


@pytest.mark.parametrize("prec", ["bf16", "tf32", "bf16x3"])
def test_sweep_tc_test_rmse_within_half_percent(ctx, ora, prec):
    """Two sweeps with tensor-core deltas on a well-posed 4-order tensor (at
    least 200 entries per row in every mode): test RMSE within 0.5 % of the
    FP64 oracle's on held-out coordinates."""
    got, ref = _rmse_case((200, 150, 30, 24), 40000, "uniform", 8, 2, prec, ctx, ora)
    assert abs(got - ref) <= 0.005 * ref, (got, ref)


@pytest.mark.parametrize("prec,tol", [("bf16", 0.10), ("tf32", 0.02), ("bf16x3", 0.005)])
def test_sweep_tc_test_rmse_zipf_tail(ctx, ora, prec, tol):
    """Zipf(1.1) rows: the tail rows hold one or two entries, their systems are
    ill-conditioned, and a BF16 delta moves their solutions (and the held-out
    predictions that hit them) by a few percent (measured 2.8 % after one
    sweep), a TF32 delta by up to 0.6 % depending on the seed (measured
    -0.3 % .. +0.57 % over three seeds); the bounds here record that.  BF16x3,
    the precision the benchmark times, keeps the 0.5 % bound of held-out RMSE
    against the FP64 oracle on these rows (measured within 0.013 %)."""
    got, ref = _rmse_case((600, 400, 30, 24), 40000, [("zipf", 1.1), ("zipf", 1.1), "uniform", "uniform"], 8, 1,
                          prec, ctx, ora)
    assert abs(got - ref) <= tol * ref, (got, ref)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bench_heldout_rmse_check_passes(seed):
    """The benchmark line's own held-out RMSE check (the timed BF16x3 delta
    against the FP64 oracle, zipf4 recipe scaled down) is within 0.5 %, for
    three seeds of the data."""
    import bench
    r = bench.heldout_rmse_vs_oracle(P, torch, "bf16x3", seed=seed)
    assert r["within_tolerance"], r


# cores larger than shared memory: streamed through it in chunks
BIG = [((12, 10, 9, 8), (16, 16, 16, 16), torch.float32), ((6, 5, 4, 5, 6), (8, 8, 8, 8, 8), torch.float32),
       ((10, 9, 8, 7), (12, 12, 12, 12), torch.float64), ((5, 4, 6, 5, 4), (7, 9, 8, 6, 9), torch.float32)]


@pytest.mark.parametrize("dims,J,dtype", BIG)
def test_streamed_core_delta_matches_oracle(ctx, ora, dims, J, dtype):
    n = 700                                     # two blocks of 256 entries and a ragged one
    core, F, idx = _case(dims, J, n, 5)
    model = P.Model.from_numpy(core, F, dtype=dtype)
    coords = torch.tensor(idx, device="cuda")
    prec = "fp64" if dtype == torch.float64 else "fp32"
    u = 2.0 ** -53 if dtype == torch.float64 else 2.0 ** -24
    for mode in range(len(dims)):
        got = P.delta(ctx, model, mode, coords, precision=prec).double().cpu().numpy()
        ref = np.stack([ora.delta(core, F, idx[e], mode) for e in range(n)])
        mag = np.stack([ora.delta(np.abs(core), F, idx[e], mode) for e in range(n)])
        assert np.all(np.abs(got - ref) <= 64 * u * mag + 1e-300), mode


@pytest.mark.parametrize("dims,J,dtype", BIG[:3])
def test_autotuned_shapes_give_identical_bits(ctx, dims, J, dtype):
    """Chunk size and blocks per SM change the schedule, not any entry's
    arithmetic: the tuned launch reproduces the default one bit for bit."""
    core, F, idx = _case(dims, J, 5000, 6)
    model = P.Model.from_numpy(core, F, dtype=dtype)
    prec = "fp64" if dtype == torch.float64 else "fp32"
    x = P.SparseObs.from_numpy(idx, np.ones(len(idx)), dims, dtype=dtype)
    s0 = P.build_mode_slices(ctx, x, 0, dtype=dtype)
    coords = torch.tensor(idx, device="cuda")
    P.autotune_clear(ctx)
    base = [P.delta(ctx, model, m, coords, precision=prec).clone() for m in range(len(dims))]
    cands, best = P.autotune_delta(ctx, s0, model, precision=prec, max_entries=4096, reps=1)
    assert len(cands) >= 8 and 0 <= best < len(cands)
    assert all(c[0] == "cuda_cores" and c[3] > 0 for c in cands)
    for m in range(len(dims)):
        got = P.delta(ctx, model, m, coords, precision=prec)
        assert torch.equal(got.view(torch.int8), base[m].view(torch.int8)), m
    P.autotune_clear(ctx)
    s0.close()


def test_autotuner_offers_tensor_cores_for_bf16(ctx):
    dims, J = (300, 200, 30, 24), (10, 10, 10, 10)
    core, F, idx = _case(dims, J, 20000, 2)
    model = P.Model.from_numpy(core, F, dtype=torch.float32)
    x = P.SparseObs.from_numpy(idx, np.ones(len(idx)), dims, dtype=torch.float32)
    s0 = P.build_mode_slices(ctx, x, 0)
    cands, best = P.autotune_delta(ctx, s0, model, precision="bf16", max_entries=20000, reps=2)
    assert cands[0][0] == "tensor_cores" and any(c[0] == "cuda_cores" for c in cands)
    P.autotune_clear(ctx)
    s0.close()
