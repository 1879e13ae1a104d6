"""Seeded synthetic workloads drawn on the GPU with PyTorch, for inputs too
large to draw in numpy in a benchmark's time (10^8 entries, or cores of
10^6 elements): the same recipe as ``synth.make_tensor`` (planted core
N(0,1), planted factors U(0,1), i.i.d. uniform coordinates, value = planted
Tucker value + N(0, sigma^2), model initialised U(0,1)), drawn from torch's
CUDA Philox generator with one seed per component derived from
``numpy.random.SeedSequence(seed)``.  The draws differ from the numpy
generator's; they are reproducible for a given seed and GPU.

The planted value is a chain of dense mode contractions (last mode first) in
float32 matmuls; like ``synth.planted_values`` it defines the observations and
is never used as an expected result.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

_STREAMS = ("core", "factors", "coords", "noise", "init")


def _gen(seed: int, stream: str, device) -> torch.Generator:
    child = np.random.SeedSequence(seed).spawn(len(_STREAMS))[_STREAMS.index(stream)]
    g = torch.Generator(device=device)
    g.manual_seed(int(child.generate_state(1, dtype=np.uint64)[0] >> np.uint64(1)))
    return g


@dataclass
class DeviceTensor:
    dims: tuple
    J: tuple
    idx: torch.Tensor       # int32 [E][N] on the device
    vals: torch.Tensor      # float32 [E]
    core: torch.Tensor      # planted core, float32
    factors: list           # planted factors, float32 [I_n][J_n]


def planted_values(core: torch.Tensor, factors, idx: torch.Tensor, max_elems: int = 1 << 27) -> torch.Tensor:
    N = core.dim()
    E = idx.shape[0]
    out = torch.empty(E, dtype=torch.float32, device=idx.device)
    Jl = core.shape[-1]
    g_last = core.reshape(-1, Jl)                         # [prod J_<N][J_N]
    chunk = max(1, min(E, max_elems // max(1, g_last.shape[0])))
    for s in range(0, E, chunk):
        e = min(E, s + chunk)
        c = e - s
        t = factors[N - 1][idx[s:e, N - 1].long()] @ g_last.T   # [c][prod J_<N]
        for k in range(N - 2, -1, -1):
            Jk = core.shape[k]
            a = factors[k][idx[s:e, k].long()]                   # [c][J_k]
            t = torch.bmm(t.reshape(c, -1, Jk), a.reshape(c, Jk, 1)).reshape(c, -1)
        out[s:e] = t.reshape(c)
    return out


def make_tensor(dims, nnz: int, J, *, sigma: float = 0.1, seed: int = 0, device="cuda") -> DeviceTensor:
    dims = tuple(int(d) for d in dims)
    J = tuple(int(j) for j in J)
    N = len(dims)
    gc = _gen(seed, "core", device)
    core = torch.randn(J, generator=gc, device=device, dtype=torch.float32)
    gf = _gen(seed, "factors", device)
    factors = [torch.rand((dims[k], J[k]), generator=gf, device=device, dtype=torch.float32) for k in range(N)]
    gx = _gen(seed, "coords", device)
    idx = torch.empty((nnz, N), dtype=torch.int32, device=device)
    for k in range(N):
        idx[:, k] = torch.randint(0, dims[k], (nnz,), generator=gx, device=device, dtype=torch.int32)
    vals = planted_values(core, factors, idx)
    if sigma > 0:
        gn = _gen(seed, "noise", device)
        vals += sigma * torch.randn(nnz, generator=gn, device=device, dtype=torch.float32)
    return DeviceTensor(dims, J, idx, vals, core, factors)


def init_model(dims, J, seed: int = 0, device="cuda"):
    """Core and factors with U(0,1) entries (Alg. 2's initialisation), float32."""
    g = _gen(seed, "init", device)
    core = torch.rand(tuple(J), generator=g, device=device, dtype=torch.float32)
    factors = [torch.rand((int(d), int(j)), generator=g, device=device, dtype=torch.float32) for d, j in zip(dims, J)]
    return core, factors
