"""Row-sharded ALS sweeps over several processes, one GPU each.

Rows of A^(n) are independent once the other factors are fixed (Sec. 3.2,
Theorem 1), so a sweep shards by rows: for every mode n each process (rank)
owns a contiguous range of rows holding an equal share of the observed entries
(the entry-balanced split of Sec. 3.4, by entries rather than rows because
slices are uneven), keeps the observed entries of those rows (so Omega is
split N times, once per mode) and full copies of the core and every factor.
One sweep (Alg. 2, one iteration of Alg. 3 over the modes in order):

    for n = 1..N:
        update the owned rows of A^(n) from the owned entries  (local)
        all-gather the updated rows: every rank holds the new A^(n)
    error: each rank sums the squared residuals of its entries of the last
    mode (a partition of Omega) and the sums are all-reduced.

The local step is a backend's ``update_rows``; ``CudaRows`` runs it through
the C ABI (``ptk_als_mode`` on the rank's own entries and rows) with the
factors on the rank's GPU, and the exchange uses torch.distributed (NCCL for
GPU tensors, gloo for CPU tensors).  Collectives are issued only between the
modes' local steps, never inside a kernel.
"""
from __future__ import annotations

import numpy as np


def row_partition(counts, world: int):
    """Contiguous row ranges [lo, hi) per rank with about equal entry counts:
    rank k starts at the first row r whose earlier rows hold at least
    k * E / world entries.  Every row belongs to exactly one rank."""
    counts = np.asarray(counts, dtype=np.int64)
    R = counts.shape[0]
    prefix = np.concatenate([[0], np.cumsum(counts)])  # entries in rows [0, r)
    E = int(prefix[-1])
    bounds = [0]
    for k in range(1, world):
        target = -(-E * k // world)  # ceil(E k / world)
        bounds.append(int(np.searchsorted(prefix, target, side="left")))
    bounds.append(R)
    for k in range(1, world + 1):  # keep the ranges ordered
        bounds[k] = max(bounds[k], bounds[k - 1])
    bounds[world] = R
    return [(bounds[k], bounds[k + 1]) for k in range(world)]


class ShardPlan:
    """Per mode: every rank's row range and this rank's entries (their ids,
    in input order, which keeps each row's entries in the slice order the
    unsharded sweep uses)."""

    def __init__(self, dims, idx, rank: int, world: int):
        idx = np.asarray(idx)
        self.dims = tuple(int(d) for d in dims)
        self.rank, self.world = rank, world
        self.ranges, self.entries = [], []
        for n, d in enumerate(self.dims):
            counts = np.bincount(idx[:, n], minlength=d)
            ranges = row_partition(counts, world)
            lo, hi = ranges[rank]
            self.ranges.append(ranges)
            self.entries.append(np.nonzero((idx[:, n] >= lo) & (idx[:, n] < hi))[0])

    def own(self, mode: int):
        return self.ranges[mode][self.rank]

    def max_rows(self, mode: int) -> int:
        return max(hi - lo for lo, hi in self.ranges[mode])


class RowShardedSweep:
    """Drives the sharded sweep: ``backend.update_rows(mode, lo, hi)`` updates
    this rank's rows of the backend's model in place and returns them as a
    tensor [hi - lo][J]; ``backend.set_rows(mode, lo, rows)`` writes gathered
    rows; ``backend.local_sse()`` returns the squared residuals of this
    rank's entries of the last mode; ``backend.zeros(rows, J)`` makes a
    buffer on the backend's device."""

    def __init__(self, plan: ShardPlan, backend, dist=None, group=None):
        self.plan, self.backend, self.dist, self.group = plan, backend, dist, group

    def _all_gather_rows(self, mode: int, mine):
        plan = self.plan
        if plan.world == 1:
            return
        width = int(mine.shape[1])
        mr = plan.max_rows(mode)
        send = self.backend.zeros(mr, width)
        send[: mine.shape[0]] = mine
        recv = [self.backend.zeros(mr, width) for _ in range(plan.world)]
        self.dist.all_gather(recv, send, group=self.group)
        for k, (lo, hi) in enumerate(plan.ranges[mode]):
            if k != plan.rank and hi > lo:
                self.backend.set_rows(mode, lo, recv[k][: hi - lo])

    def sweep(self, error_pass: bool = True):
        """One sharded sweep; returns the sum of squared residuals over all
        of Omega (None without error_pass)."""
        for n in range(len(self.plan.dims)):
            lo, hi = self.plan.own(n)
            mine = self.backend.update_rows(n, lo, hi)
            self._all_gather_rows(n, mine)
        if not error_pass:
            return None
        sse = float(self.backend.local_sse())
        if self.plan.world > 1:
            t = self.backend.zeros(1, 1).double()
            t.fill_(sse)
            self.dist.all_reduce(t, group=self.group)
            sse = float(t.reshape(-1)[0].item())
        return sse


class CudaRows:
    """The local step on this rank's GPU through the C ABI: per mode, the
    rank's own entries (a SparseObs and its slice layout of that mode) and
    ``ptk_als_mode`` on its rows; the model lives on the GPU."""

    def __init__(self, ctx, plan: ShardPlan, idx, vals, model, *, precision="fp32", lam=0.01, schedule="auto",
                 dtype=None):
        import torch

        from . import SparseObs, build_mode_slices
        self.ctx, self.plan, self.model = ctx, plan, model
        self.precision, self.lam, self.schedule = precision, lam, schedule
        dtype = dtype or model.core.dtype
        idx = np.asarray(idx)
        vals = np.asarray(vals)
        self.x, self.slices = [], []
        for n in range(len(plan.dims)):
            ent = plan.entries[n]
            x = SparseObs.from_numpy(idx[ent], vals[ent], plan.dims, dtype=dtype)
            self.x.append(x)
            self.slices.append(build_mode_slices(ctx, x, n, dtype=dtype))
        self.torch = torch

    def zeros(self, rows, width):
        return self.torch.zeros((rows, width), dtype=self.model.core.dtype, device="cuda")

    def update_rows(self, mode, lo, hi):
        from . import als_mode
        als_mode(self.ctx, self.x[mode], self.slices[mode], self.model, mode, lo, hi, precision=self.precision,
                 lam=self.lam, schedule=self.schedule)
        J = self.model.J[mode]
        return self.model.factors[mode][lo:hi, :J]

    def set_rows(self, mode, lo, rows):
        J = self.model.J[mode]
        self.model.factors[mode][lo:lo + rows.shape[0], :J] = rows

    def local_sse(self):
        from . import error
        n = len(self.plan.dims) - 1
        return error(self.ctx, self.x[n], self.model, self.lam)["sse"]

    def close(self):
        for s in self.slices:
            s.close()
