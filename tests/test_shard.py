"""Row-sharded sweeps (paper_1710_02261_gb300.shard) on CPU ranks.

The partition of every mode's rows into contiguous, entry-balanced ranges and
the sweep's exchange (an all-gather of the updated rows per mode, an
all-reduce of the error) run on world_size-2 and 3 gloo process groups.  The
local step of each rank is the FP64 oracle's row update on the rank's own
entries (the role ptk_als_mode plays on a GPU), so the sharded factors must
equal the single-process oracle sweep's bit for bit: each row's sums take the
same entries in the same order.
"""
import os
import socket

import numpy as np
import pytest

import synth
from paper_1710_02261_gb300.shard import RowShardedSweep, ShardPlan, row_partition

LAM = 0.01


def test_row_partition_properties():
    rng = np.random.default_rng(3)
    for R, world in [(1, 1), (5, 3), (1000, 2), (1000, 7), (37, 8), (4, 6)]:
        counts = rng.zipf(1.3, size=R).astype(np.int64)
        counts[rng.random(R) < 0.2] = 0
        parts = row_partition(counts, world)
        assert len(parts) == world and parts[0][0] == 0 and parts[-1][1] == R
        assert all(parts[k][1] == parts[k + 1][0] for k in range(world - 1))
        assert all(lo <= hi for lo, hi in parts)
        E = counts.sum()
        share = [counts[lo:hi].sum() for lo, hi in parts]
        assert sum(share) == E
        # each range ends within one row of its entry target
        for k, (lo, hi) in enumerate(parts[:-1]):
            assert abs(int(np.sum(counts[:hi])) - E * (k + 1) / world) <= counts.max()


class _OracleRows:
    """Local step of a rank with the oracle: the update of one mode from this
    rank's entries (rows without entries there are not this rank's)."""

    def __init__(self, plan, core, factors, idx, vals):
        import torch
        self.torch = torch
        self.plan, self.core = plan, core
        self.F = [np.array(f, dtype=np.float64) for f in factors]
        self.idx, self.vals = np.asarray(idx), np.asarray(vals)

    def zeros(self, rows, width):
        return self.torch.zeros((rows, width), dtype=self.torch.float64)

    def update_rows(self, mode, lo, hi):
        import oracle
        ent = self.plan.entries[mode]
        Fn, _ = oracle.update_mode(self.plan.dims, self.core, self.F, self.idx[ent], self.vals[ent], mode, LAM)
        self.F[mode][lo:hi] = Fn[mode][lo:hi]
        return self.torch.from_numpy(self.F[mode][lo:hi].copy())

    def set_rows(self, mode, lo, rows):
        self.F[mode][lo:lo + rows.shape[0]] = rows.numpy()

    def local_sse(self):
        import oracle
        n = len(self.plan.dims) - 1
        ent = self.plan.entries[n]
        return oracle.sse(self.core, self.F, self.idx[ent], self.vals[ent])


def _case():
    dims, J = (40, 30, 25), (3, 4, 2)
    t = synth.make_tensor(dims, 3000, J, dist=[("zipf", 1.1), "uniform", ("zipf", 1.3)], sigma=0.1, seed=5,
                          n_test=0)
    m0 = synth.init_model(dims, J, seed=5)
    return t, m0


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t, m0 = _case()
        plan = ShardPlan(t.dims, t.idx, rank, world)
        be = _OracleRows(plan, m0.core, m0.factors, t.idx, t.vals)
        sw = RowShardedSweep(plan, be, dist=dist)
        sses = [sw.sweep() for _ in range(2)]
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), *be.F, sse=np.array(sses))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sweeps_match_single_process_oracle(tmp_path, world, ora):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    t, m0 = _case()
    F = m0.factors
    ref_sse = []
    for _ in range(2):
        F, _ = ora.sweep(t.dims, m0.core, F, t.idx, t.vals, LAM)
        ref_sse.append(ora.sse(m0.core, F, t.idx, t.vals))
    for rank in range(world):
        got = np.load(tmp_path / f"rank{rank}.npz")
        for n in range(len(t.dims)):
            assert np.array_equal(got[f"arr_{n}"], F[n]), (rank, n)     # every rank holds every full factor
        np.testing.assert_allclose(got["sse"], ref_sse, rtol=1e-12)      # partial sums in another order
