"""Row sums of Eqs. (rowB), (rowC) on the tensor cores (PTK_SCHED_TENSOR).

Rows of at least 64 entries are cut into chunks of at most 512; every Delta
value is written as four (or three) signed 7-bit digits scaled by a power of
two per chunk and column, so BF16 tensor-core products and the chunk's FP32
sums are exact and the sums differ from those of the FP32 Delta values only
by the last digit's rounding (2^-29, or 2^-22, of the chunk's column maximum,
at most) and the double-float combination (~2^-46 of sum |z_j z_k|).  Rows split between CTAs are merged in
CTA order.  The checks call ptk_row_sums through the C ABI on Delta arrays
built here, against FP64 sums of the same values computed with numpy.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1710_02261_gb300 as P  # noqa: E402

CH, TLONG = 512, 64


@pytest.fixture(scope="module")
def ctx():
    c = P.Context(0)
    yield c
    c.close()
# row lengths around every boundary: empty, short, the tensor-core threshold,
# the chunk size, and rows long enough to be split between many CTAs
LENGTHS = [0, 1, 5, 63, 64, 65, 100, 511, 512, 513, 1024, 1025, 3000, 20000, 7, 0, 64, 2, 9000, 129]


def _ld(J):
    return J + 1 if (J + 1) % 2 else J + 2


def _layout(lengths):
    rp = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    rid = np.repeat(np.arange(len(lengths)), lengths).astype(np.int32)
    return rp, rid


def _ref(Z, rp, J):
    """FP64 B (upper, row-major) and c per row, and sum |z_j z_k| per output."""
    rows = len(rp) - 1
    iu = np.triu_indices(J)
    out = np.zeros((rows, J * (J + 1) // 2 + J))
    mag = np.zeros_like(out)
    for r in range(rows):
        z = Z[rp[r]:rp[r + 1], :J + 1].astype(np.float64)
        G, A = z.T @ z, np.abs(z).T @ np.abs(z)
        out[r] = np.concatenate([G[:J, :J][iu], G[J, :J]])
        mag[r] = np.concatenate([A[:J, :J][iu], A[J, :J]])
    return out, mag


def _chunks(b, e):
    """A row of m >= 64 entries: ceil(m / 512) chunks of equal size (+-1)."""
    m = e - b
    nc = -(-m // CH)
    return [(b + q * m // nc, b + (q + 1) * m // nc) for q in range(nc)]


def _digit_bound(Z, rp, J, digits=4):
    """|tensor-core sum - exact sum| per output: each value of chunk c, column
    j, moves by at most eps_jc = 2^{e_jc - 8 - 7 (digits - 1)} (2^{e_jc - 1} <=
    max |z_j| < 2^{e_jc}; the last digit's rounding), so a product moves by
    |z_j| eps_k + |z_k| eps_j + eps_j eps_k."""
    rows = len(rp) - 1
    iu = np.triu_indices(J)
    out = np.zeros((rows, J * (J + 1) // 2 + J))
    for r in range(rows):
        b, e = rp[r], rp[r + 1]
        if e - b < TLONG:
            continue
        acc = np.zeros((J + 1, J + 1))
        for c0, c1 in _chunks(b, e):
            z = np.abs(Z[c0:c1, :J + 1].astype(np.float64))
            mx = z.max(axis=0)
            expo = np.floor(np.log2(np.where(mx > 0, mx, 1))) + 1
            eps = np.where(mx > 0, 2.0 ** (expo - 8 - 7 * (digits - 1)), 0.0)
            s = z.sum(axis=0)
            acc += np.outer(s, eps) + np.outer(eps, s) + len(z) * np.outer(eps, eps)
        out[r] = np.concatenate([acc[:J, :J][iu], acc[J, :J]])
    return out


def _call(ctx, Z, rp, rid, J, schedule, digits=4):
    d = torch.tensor(Z, device="cuda")
    return P.row_sums(ctx, d, torch.tensor(rp, device="cuda"), torch.tensor(rid, device="cuda"), J,
                      schedule=schedule, digits=digits).cpu().numpy()


@pytest.mark.parametrize("J", [1, 3, 10, 15])
def test_small_integers_exact(ctx, J):
    """Integer values |z| <= 127: one digit each, so the tensor-core sums are
    exact, equal to numpy's integer sums bit for bit (and so are the
    double-float CUDA-core schedules')."""
    rng = np.random.default_rng(J)
    rp, rid = _layout(LENGTHS)
    Z = np.zeros((rp[-1], _ld(J)), dtype=np.float32)
    Z[:, :J + 1] = rng.integers(-127, 128, size=(rp[-1], J + 1))
    ref, _ = _ref(Z, rp, J)
    for sched, digits in [("tensor", 4), ("tensor", 3), ("entries", 4), ("rows_static", 4)]:
        got = _call(ctx, Z, rp, rid, J, sched, digits)
        assert np.array_equal(got, ref), (sched, digits)


@pytest.mark.parametrize("digits", [4, 3])
@pytest.mark.parametrize("J", [2, 10, 15])
def test_fp32_values_within_digit_bound(ctx, J, digits):
    """FP32 values of mixed signs and magnitudes (columns 10^-3..10^4, a few
    values 10^3 larger in one row): the tensor-core sums within the digit
    bound plus 2^-44 sum |z_j z_k|; rows below 64 entries (double-float, one
    warp per row) within 2^-44 sum |z_j z_k|."""
    rng = np.random.default_rng(100 + J)
    rp, rid = _layout(LENGTHS)
    n = rp[-1]
    Z = np.zeros((n, _ld(J)), dtype=np.float32)
    scale = 10.0 ** rng.uniform(-3, 4, size=J + 1)
    Z[:, :J + 1] = (rng.standard_normal((n, J + 1)) * scale).astype(np.float32)
    Z[rp[13] + 7, :J + 1] *= 1000.0                       # an outlier inside the 20000-entry row
    ref, mag = _ref(Z, rp, J)
    bound = _digit_bound(Z, rp, J, digits) + 2.0 ** -44 * mag
    got = _call(ctx, Z, rp, rid, J, "tensor", digits)
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / np.maximum(bound, 1e-300))
    auto = _call(ctx, Z, rp, rid, J, "auto", digits)
    assert np.array_equal(auto, got)                       # auto takes the tensor cores here


def test_tensor_schedule_deterministic_and_zero_columns(ctx):
    """Two calls give the same bits; an all-zero column (and x = 0) gives
    exact zeros in its sums."""
    J = 10
    rng = np.random.default_rng(7)
    rp, rid = _layout(LENGTHS)
    Z = np.zeros((rp[-1], _ld(J)), dtype=np.float32)
    Z[:, :J + 1] = rng.random((rp[-1], J + 1)).astype(np.float32)
    Z[:, 4] = 0.0
    Z[:, J] = 0.0
    a = _call(ctx, Z, rp, rid, J, "tensor")
    b = _call(ctx, Z, rp, rid, J, "tensor")
    assert np.array_equal(a, b)
    ref, mag = _ref(Z, rp, J)
    assert np.all(a[:, J * (J + 1) // 2:] == 0.0)
    iu = np.triu_indices(J)
    zero_col = (iu[0] == 4) | (iu[1] == 4)
    assert np.all(a[:, :J * (J + 1) // 2][:, zero_col] == 0.0)
    assert np.all(np.abs(a - ref) <= _digit_bound(Z, rp, J) + 2.0 ** -44 * mag)


def test_tensor_schedule_unsupported_cases(ctx):
    rp, rid = _layout([3, 5, 10])                          # no row of 64 entries
    Z = np.ones((18, _ld(4)), dtype=np.float32)
    with pytest.raises(P.PtkError):
        _call(ctx, Z, rp, rid, 4, "tensor")
    got = _call(ctx, Z, rp, rid, 4, "auto")                # auto falls back to the CUDA cores
    ref, _ = _ref(Z, rp, 4)
    assert np.array_equal(got, ref)


def test_sweep_tensor_schedule_matches_oracle(ctx, ora):
    """A full FP32 sweep with the tensor-core row sums on Zipf-skewed modes
    (rows of thousands of entries, split between CTAs, next to rows of a few),
    mode by mode against the oracle's row update from the same state, within
    the first-order ridge bound of the FP32 delta (tests/bounds.py)."""
    import bounds
    import synth
    dims, J = (60, 45, 30), (6, 5, 4)
    t = synth.make_tensor(dims, 120_000, J, dist=[("zipf", 1.1), ("zipf", 1.1), "uniform"], sigma=0.1, seed=31,
                          n_test=0)
    m0 = synth.init_model(dims, J, seed=31)
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)  # noqa: E731
    core, F0, vals = f32(m0.core), [f32(a) for a in m0.factors], f32(t.vals)
    x = P.SparseObs.from_numpy(t.idx, vals, dims, dtype=torch.float32)
    sl = P.build_all_slices(ctx, x)
    model = P.Model.from_numpy(core, F0, dtype=torch.float32)
    st = P.als_sweep(ctx, x, sl, model, precision="fp32", lam=0.01, schedule="tensor")
    assert st["bad_rows"] == 0
    _, Fg = model.to_numpy()
    K = int(np.prod(J))
    for n in range(len(dims)):
        state = [Fg[k] if k < n else F0[k] for k in range(len(dims))]
        g = bounds.gamma(K // J[n] + len(dims))
        for i, (bd, aref) in bounds.mode_bounds(ora, core, state, t.idx, vals, n, 0.01, g).items():
            assert np.linalg.norm(Fg[n][i] - aref) <= bd + 1e-12, (n, i)
    for s_ in sl:
        s_.close()
