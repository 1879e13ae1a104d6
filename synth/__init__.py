"""Seeded synthetic workloads for sparse Tucker factorization.

This module only draws inputs: observed coordinates, planted models, noise and
model initialisations.  It is shared by the FP64 oracle tests and the CUDA path
so that both sides see byte-identical inputs.  It contains none of the row-wise
update (delta, Gram, solve), none of the error / truncation logic and none of
the CUDA code.  The one piece of tensor arithmetic here is the evaluation of the
*planted* model that defines what the synthetic observations are (value = planted
Tucker value + Gaussian noise, the recipe of the paper's synthetic tensors,
Sec. 5.2 "Synthetic Data" and Table 3); it is a chain of dense mode contractions
in float64 and is not used to produce any expected result.

Random streams: every component draws from its own child of
``numpy.random.SeedSequence(seed)`` with a Philox bit generator, in this fixed
order of children: planted core, planted factors, training coordinates, noise,
test coordinates, test noise, model initialisation.  Changing a size therefore
never shifts another component's draws.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_STREAMS = ("core", "factors", "coords", "noise", "test_coords", "test_noise", "init")


def _rng(seed: int, stream: str) -> np.random.Generator:
    child = np.random.SeedSequence(seed).spawn(len(_STREAMS))[_STREAMS.index(stream)]
    return np.random.Generator(np.random.Philox(child))


@dataclass
class SparseTensor:
    """Observed entries Omega of an N-order tensor (0-based coordinates)."""
    dims: tuple
    idx: np.ndarray            # int32 [E][N]
    vals: np.ndarray           # float64 [E]
    test_idx: np.ndarray       # int32 [E_test][N]
    test_vals: np.ndarray      # float64 [E_test]
    planted_core: np.ndarray | None = None
    planted_factors: list | None = None
    meta: dict = field(default_factory=dict)

    @property
    def order(self) -> int:
        return len(self.dims)

    @property
    def nnz(self) -> int:
        return int(self.idx.shape[0])


@dataclass
class Model:
    """Core tensor G (dense, C-order over j_1..j_N) and factors A^(n) [I_n][J_n]."""
    core: np.ndarray
    factors: list

    @property
    def J(self) -> tuple:
        return tuple(self.core.shape)

    def copy(self) -> "Model":
        return Model(self.core.copy(), [a.copy() for a in self.factors])


def zipf_indices(rng: np.random.Generator, n: int, size: int, s: float) -> np.ndarray:
    """Indices r-1 with P(r) proportional to r^-s over ranks r = 1..size."""
    w = np.arange(1, size + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(n)
    out = np.searchsorted(cdf, u, side="right")
    return np.minimum(out, size - 1).astype(np.int32)


def draw_coords(rng: np.random.Generator, dims, n: int, dist) -> np.ndarray:
    idx = np.empty((n, len(dims)), dtype=np.int32)
    for k, I in enumerate(dims):
        kind = dist[k] if isinstance(dist, (list, tuple)) else dist
        if kind == "uniform":
            idx[:, k] = rng.integers(0, I, size=n, dtype=np.int64).astype(np.int32)
        elif isinstance(kind, tuple) and kind[0] == "zipf":
            idx[:, k] = zipf_indices(rng, n, I, kind[1])
        else:
            raise ValueError(f"unknown coordinate distribution {kind!r}")
    return idx


def planted_values(core: np.ndarray, factors, idx: np.ndarray, chunk: int = 1 << 15) -> np.ndarray:
    """Planted Tucker value at each coordinate (data synthesis, float64).

    Contracts the dense core with the gathered factor rows one mode at a time,
    last mode first.
    """
    N = core.ndim
    E = idx.shape[0]
    out = np.empty(E, dtype=np.float64)
    Jl = core.shape[-1]
    g_last = core.reshape(-1, Jl)                       # [prod J_<N][J_N]
    for s in range(0, E, chunk):
        e = min(E, s + chunk)
        t = factors[N - 1][idx[s:e, N - 1]] @ g_last.T  # [c][prod J_<N]
        for k in range(N - 2, -1, -1):
            Jk = core.shape[k]
            t = t.reshape(e - s, -1, Jk)
            t = np.einsum("cpj,cj->cp", t, factors[k][idx[s:e, k]])
        out[s:e] = t.reshape(e - s)
    return out


def make_tensor(dims, nnz: int, J, *, dist="uniform", sigma: float = 0.1, seed: int = 0,
                n_test: int | None = None, core_dist: str = "normal") -> SparseTensor:
    """Planted-model tensor: core ~ N(0,1) (or U(0,1)), factors ~ U(0,1), i.i.d.
    coordinates (duplicates kept), value = planted value + N(0, sigma^2)."""
    dims = tuple(int(d) for d in dims)
    J = tuple(int(j) for j in J)
    N = len(dims)
    rc = _rng(seed, "core")
    core = rc.standard_normal(J) if core_dist == "normal" else rc.random(J)
    rf = _rng(seed, "factors")
    factors = [rf.random((dims[k], J[k])) for k in range(N)]
    idx = draw_coords(_rng(seed, "coords"), dims, nnz, dist)
    vals = planted_values(core, factors, idx)
    if sigma > 0:
        vals += sigma * _rng(seed, "noise").standard_normal(nnz)
    if n_test is None:
        n_test = int(math.ceil(nnz / 10))
    tidx = draw_coords(_rng(seed, "test_coords"), dims, n_test, dist)
    tvals = planted_values(core, factors, tidx) if n_test else np.zeros(0)
    if sigma > 0 and n_test:
        tvals += sigma * _rng(seed, "test_noise").standard_normal(n_test)
    return SparseTensor(dims, idx, vals, tidx, tvals, core, factors,
                        meta=dict(J_planted=J, sigma=sigma, seed=seed, dist=dist))


def init_model(dims, J, seed: int = 0) -> Model:
    """Model initialisation with U(0,1) entries (Alg. 2, first step): core first,
    then A^(1..N), each row-major."""
    rng = _rng(seed, "init")
    J = tuple(int(j) for j in J)
    core = rng.random(J)
    factors = [rng.random((int(dims[k]), J[k])) for k in range(len(dims))]
    return Model(core, factors)


# ---------------------------------------------------------------------------
# The paper-shaped workloads (sizes of the paper's experiments, Sec. 5, as synthetic stand-ins).
# ``scale`` shrinks entry counts and mode sizes proportionally for quick tests.

def workload_plain_fp64(seed: int = 0, scale: float = 1.0) -> SparseTensor:
    """3-order 1000^3, 1e5 uniform entries, planted J=(5,5,5), sigma 0.1."""
    I = max(8, int(1000 * scale))
    return make_tensor((I, I, I), max(64, int(100_000 * scale)), (5, 5, 5), seed=seed)


def workload_zipf4(seed: int = 0, scale: float = 1.0, nnz: int | None = None) -> SparseTensor:
    """4-order 100000 x 50000 x 30 x 24, Zipf(1.1) on modes 1-2, uniform on 3-4,
    1e7 entries, planted J=(10,10,10,10), sigma 0.1."""
    dims = (max(16, int(100_000 * scale)), max(16, int(50_000 * scale)), 30, 24)
    E = nnz if nnz is not None else max(256, int(10_000_000 * scale))
    return make_tensor(dims, E, (10, 10, 10, 10), dist=[("zipf", 1.1), ("zipf", 1.1), "uniform", "uniform"],
                       seed=seed)


def workload_scal3(seed: int = 0, scale: float = 1.0) -> SparseTensor:
    """3-order 1e7^3 with 1e8 uniform entries, planted J=(10,10,10), sigma 0.1."""
    I = max(16, int(10_000_000 * scale))
    return make_tensor((I, I, I), max(256, int(100_000_000 * scale)), (10, 10, 10), seed=seed)


def batched_shapes(count: int = 512, seed: int = 0):
    """Shapes of the batched workload: order U{3,4,5}, each I_n log-uniform in
    [1e2, 1e5], nnz log-uniform in [1e4, 5e6], J uniform in {3..16} (same for all modes)."""
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 4242])))
    shapes = []
    for t in range(count):
        N = int(rng.integers(3, 6))
        dims = tuple(int(round(math.exp(rng.uniform(math.log(1e2), math.log(1e5))))) for _ in range(N))
        nnz = int(round(math.exp(rng.uniform(math.log(1e4), math.log(5e6)))))
        J = int(rng.integers(3, 17))
        shapes.append(dict(dims=dims, nnz=nnz, J=(J,) * N, seed=t))
    return shapes


def foldin_requests(model_dims, count: int, seed: int = 0, m_min: int = 5, m_max: int = 5000,
                    n_query: int = 100, planted=None, sigma: float = 0.1, dtype=np.float32):
    """New mode-1 slices: each request draws m ~ round(exp U(ln m_min, ln m_max))
    observed (i_2..i_N) coordinates uniformly plus n_query held-out coordinates.

    Coordinate arrays are [m][N] int32 with the mode-1 column 0.  With
    ``planted = (core, factors)`` each request also gets a new planted row
    ~ U(0,1)^J_1 and values = planted value + N(0, sigma^2) (``obs_vals``, and
    the noise-free ``query_vals``)."""
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 777])))
    reqs = []
    N = len(model_dims)
    for r in range(count):
        m = int(round(math.exp(rng.uniform(math.log(m_min), math.log(m_max)))))
        oidx = np.zeros((m, N), dtype=np.int32)
        qidx = np.zeros((n_query, N), dtype=np.int32)
        for k in range(1, N):
            oidx[:, k] = rng.integers(0, model_dims[k], size=m)
        for k in range(1, N):
            qidx[:, k] = rng.integers(0, model_dims[k], size=n_query)
        req = dict(obs_idx=oidx, query_idx=qidx)
        if planted is not None:
            core, factors = planted
            row = rng.random((1, core.shape[0]))
            fac = [row] + list(factors[1:])
            req["obs_vals"] = (planted_values(core, fac, oidx) + sigma * rng.standard_normal(m)).astype(dtype)
            req["query_vals"] = planted_values(core, fac, qidx).astype(dtype)
        reqs.append(req)
    return reqs
