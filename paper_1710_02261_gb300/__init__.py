"""GB300 (sm_103a) row-wise ALS for sparse Tucker factorisation (P-Tucker,
arXiv 1710.02261) -- Python binding of libptk.

Thin wrappers with the C ABI's names: they marshal torch CUDA tensors (device
memory and the current stream) into the ``include/ptk.h`` structs and check the
returned status.  All arithmetic runs in libptk's kernels; there is no CPU or
eager-PyTorch fallback.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _ffi as F
from ._ffi import PtkError  # noqa: F401

__all__ = ["Context", "SparseObs", "Model", "Slices", "build_mode_slices", "als_sweep", "error", "partial_error",
           "fit", "fit_many", "autotune_delta", "autotune_clear", "qr_finalize", "predict", "foldin", "delta", "Server",
           "DeviceServer", "als_mode", "row_sums", "PtkError", "padded_ld"]


def _lib():
    return F.load()


def tc_available(model, precision: str = "bf16") -> bool:
    """Whether the tcgen05 delta kernel covers this model's shape."""
    fn = _lib().ptk_delta_tc_supported
    m = model.cstruct()
    return all(fn(C.byref(m), n, F.PREC[precision]) == 1 for n in range(model.core.dim()))


def launch_count() -> int:
    """Kernel launches issued through libptk in this process."""
    return int(_lib().ptk_launch_count())


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F.F32
    if t.dtype == torch.float64:
        return F.F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def padded_ld(J: int, dtype=torch.float32) -> int:
    """Row length used for factor storage: J rounded up to 16 bytes."""
    w = 4 if dtype == torch.float32 else 2
    return (J + w - 1) // w * w


class Context:
    """A libptk context on one CUDA device (scratch buffers, status words)."""

    def __init__(self, device: int = 0):
        self._h = C.c_void_p()
        F.check(_lib().ptk_create(C.byref(self._h), device), "ptk_create")
        self.device = device

    @property
    def handle(self):
        return self._h

    def set_timing(self, on: bool = True):
        F.check(_lib().ptk_set_timing(self._h, 1 if on else 0), "ptk_set_timing")

    def read_timers(self):
        """{group: (device ms, kernel launches, timed instances)} since the last read."""
        n = len(F.TIMERS)
        ms, la, gr = (C.c_double * n)(), (C.c_int64 * n)(), (C.c_int64 * n)()
        F.check(_lib().ptk_read_timers(self._h, ms, la, gr), "ptk_read_timers")
        return {name: (ms[i], la[i], gr[i]) for i, name in enumerate(F.TIMERS)}

    def close(self):
        if self._h:
            _lib().ptk_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class SparseObs:
    """Observed entries: idx int32 [E][N] and vals [E] on the GPU."""
    idx: torch.Tensor
    vals: torch.Tensor
    dims: tuple

    def __post_init__(self):
        assert self.idx.is_cuda and self.idx.dtype == torch.int32 and self.idx.is_contiguous()
        assert self.vals.is_cuda and self.vals.is_contiguous()
        self.dims = tuple(int(d) for d in self.dims)

    @property
    def nnz(self):
        return int(self.idx.shape[0])

    def cstruct(self) -> F.Coo:
        c = F.Coo()
        c.order = len(self.dims)
        for k, d in enumerate(self.dims):
            c.dims[k] = d
        c.nnz = self.nnz
        c.idx = self.idx.data_ptr() if self.nnz else None
        c.vals = self.vals.data_ptr() if self.nnz else None
        c.dtype = _dt(self.vals)
        return c

    @staticmethod
    def from_numpy(idx, vals, dims, dtype=torch.float32, device="cuda"):
        return SparseObs(torch.as_tensor(idx, dtype=torch.int32).contiguous().to(device),
                         torch.as_tensor(vals).to(dtype).contiguous().to(device), dims)


@dataclass
class Model:
    """Core G (dense, C order) and factors A^(n) stored [I_n][ld_n] (ld_n >= J_n)."""
    core: torch.Tensor
    factors: list

    @property
    def J(self):
        return tuple(int(j) for j in self.core.shape)

    @property
    def dims(self):
        return tuple(int(f.shape[0]) for f in self.factors)

    def cstruct(self) -> F.Model:
        m = F.Model()
        m.order = self.core.dim()
        for k in range(self.core.dim()):
            m.J[k] = self.core.shape[k]
            m.dims[k] = self.factors[k].shape[0]
            m.factors[k] = self.factors[k].data_ptr()
            m.ld[k] = self.factors[k].stride(0)
        m.core = self.core.data_ptr()
        m.dtype = _dt(self.core)
        return m

    def factor_views(self):
        """Factors without the padding columns, [I_n][J_n]."""
        return [f[:, :j] for f, j in zip(self.factors, self.J)]

    @staticmethod
    def from_numpy(core, factors, dtype=torch.float32, device="cuda"):
        G = torch.as_tensor(core).to(dtype).contiguous().to(device)
        fs = []
        for a in factors:
            a = torch.as_tensor(a).to(dtype)
            I, J = a.shape
            buf = torch.zeros((I, padded_ld(J, dtype)), dtype=dtype, device=a.device)
            buf[:, :J] = a
            fs.append(buf.contiguous().to(device))
        return Model(G, fs)

    def to_numpy(self):
        return self.core.detach().double().cpu().numpy(), [f.double().cpu().numpy() for f in self.factor_views()]


class Slices:
    """Slice layout of one mode (owned by libptk)."""

    def __init__(self, handle, mode: int):
        self._h = handle
        self.mode = mode

    def view(self):
        perm, rp, rid = C.c_void_p(), C.c_void_p(), C.c_void_p()
        nnz, rows = C.c_int64(), C.c_int64()
        F.check(_lib().ptk_slices_view(self._h, C.byref(perm), C.byref(rp), C.byref(rid), C.byref(nnz),
                                       C.byref(rows)), "ptk_slices_view")
        return perm.value, rp.value, rid.value, nnz.value, rows.value

    def perm_and_rowptr(self, stream=None):
        """Copies of perm (int32 [nnz]) and row_ptr (int64 [rows+1]) as CUDA tensors."""
        _, _, _, nnz, rows = self.view()
        perm = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        rp = torch.empty(rows + 1, dtype=torch.int64, device="cuda")
        F.check(_lib().ptk_slices_export(self._h, perm.data_ptr(), rp.data_ptr(), _stream(stream)),
                "ptk_slices_export")
        return perm[:nnz], rp

    def close(self):
        if self._h:
            _lib().ptk_slices_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
def build_mode_slices(ctx: Context, x: SparseObs, mode: int, dtype=torch.float32, stream=None) -> Slices:
    h = C.c_void_p()
    coo = x.cstruct()
    F.check(_lib().ptk_build_mode_slices(ctx.handle, C.byref(coo), mode, F.F64 if dtype == torch.float64 else F.F32,
                                         C.byref(h), _stream(stream)), "ptk_build_mode_slices")
    return Slices(h, mode)


def build_all_slices(ctx: Context, x: SparseObs, dtype=torch.float32, stream=None):
    return [build_mode_slices(ctx, x, n, dtype, stream) for n in range(len(x.dims))]


def _opts(variant="plain", precision="fp32", lam=0.01, trunc_rate=0.2, trunc_rule="r_beta", error_pass=True,
          schedule="auto"):
    o = F.AlsOpts()
    o.variant = F.VARIANT[variant]
    o.precision = F.PREC[precision]
    o.lam = lam
    o.trunc_rate = trunc_rate
    o.trunc_rule = F.TRUNC[trunc_rule]
    o.error_pass = 1 if error_pass else 0
    o.schedule = F.SCHEDULE[schedule]
    return o


def _stats_dict(s: F.SweepStats):
    return dict(sse=s.sse, error=s.error, rmse=s.rmse, loss=s.loss, core_nnz=s.core_nnz, bad_rows=s.bad_rows)


def als_sweep(ctx: Context, x: SparseObs, slices, model: Model, *, variant="plain", precision="fp32", lam=0.01,
              trunc_rate=0.2, trunc_rule="r_beta", error_pass=True, sync_stats=True, stream=None, schedule="auto",
              _coo=None, _model=None, _slices=None):
    """One iteration of Alg. 2 (Alg. 3 over all modes, error, Approx truncation).

    ``schedule`` picks how the row sums are spread over the GPU: "entries"
    (equal entry tiles), "rows_static" or "rows_dynamic" (one warp per row,
    dealt in turn or from a shared counter; Sec. 3.4's choice), "tensor" (FP32,
    J <= 15: rows of 64 entries or more on the tensor cores, the rest one per
    warp), or "auto" (the default: tensor where it applies, else rows_static
    for modes whose longest row is short next to a warp's share of the
    entries, entries otherwise)."""
    coo = _coo if _coo is not None else x.cstruct()
    m = _model if _model is not None else model.cstruct()
    sl = _slices if _slices is not None else (C.c_void_p * F.MAX_ORDER)(*[s._h for s in slices])
    o = _opts(variant, precision, lam, trunc_rate, trunc_rule, error_pass, schedule)
    st = F.SweepStats()
    want = error_pass and sync_stats
    rc = _lib().ptk_als_sweep(ctx.handle, C.byref(coo), C.cast(sl, C.POINTER(C.c_void_p)), C.byref(m), C.byref(o),
                              C.byref(st) if want else None, _stream(stream))
    F.check(rc, "ptk_als_sweep")
    return _stats_dict(st) if want else None


def als_mode(ctx: Context, x: SparseObs, slices_mode, model: Model, mode: int, row_lo: int, row_hi: int, *,
             precision="fp32", lam=0.01, schedule="auto", stream=None):
    """Alg. 3 for one mode on rows [row_lo, row_hi) from the entries of x
    (``slices_mode``: x's slice layout of that mode); other rows untouched."""
    coo, m = x.cstruct(), model.cstruct()
    o = _opts("plain", precision, lam, 0.2, "r_beta", False, schedule)
    F.check(_lib().ptk_als_mode(ctx.handle, C.byref(coo), slices_mode._h, C.byref(m), mode, row_lo, row_hi,
                                C.byref(o), _stream(stream)), "ptk_als_mode")


def sweep_stats_read(ctx: Context, stream=None):
    """Statistics of the last sweep run with error_pass (waits for the stream)."""
    st = F.SweepStats()
    F.check(_lib().ptk_sweep_stats_read(ctx.handle, C.byref(st), _stream(stream)), "ptk_sweep_stats_read")
    return _stats_dict(st)


def error(ctx: Context, x: SparseObs, model: Model, lam=0.01, stream=None):
    st = F.SweepStats()
    coo, m = x.cstruct(), model.cstruct()
    F.check(_lib().ptk_error(ctx.handle, C.byref(coo), C.byref(m), lam, C.byref(st), _stream(stream)), "ptk_error")
    return _stats_dict(st)


def partial_error(ctx: Context, x: SparseObs, model: Model, stream=None) -> torch.Tensor:
    R = torch.empty(model.core.numel(), dtype=torch.float64, device="cuda")
    coo, m = x.cstruct(), model.cstruct()
    F.check(_lib().ptk_partial_error(ctx.handle, C.byref(coo), C.byref(m), R.data_ptr(), _stream(stream)),
            "ptk_partial_error")
    return R.view(model.core.shape)


def qr_finalize(ctx: Context, model: Model, stream=None):
    m = model.cstruct()
    F.check(_lib().ptk_qr_finalize(ctx.handle, C.byref(m), _stream(stream)), "ptk_qr_finalize")


def predict(ctx: Context, model: Model, coords: torch.Tensor, stream=None) -> torch.Tensor:
    coords = coords.to(torch.int32).contiguous()
    out = torch.empty(coords.shape[0], dtype=model.core.dtype, device="cuda")
    m = model.cstruct()
    F.check(_lib().ptk_predict(ctx.handle, C.byref(m), coords.data_ptr() if coords.numel() else None,
                               coords.shape[0], out.data_ptr() if out.numel() else None, _stream(stream)),
            "ptk_predict")
    return out


def delta(ctx: Context, model: Model, mode: int, coords: torch.Tensor, precision="fp32", stream=None):
    """delta vectors of Eq. (delta) for the given coordinates: [n][J_mode]."""
    coords = coords.to(torch.int32).contiguous()
    n = coords.shape[0]
    out = torch.empty((n, model.J[mode]), dtype=model.core.dtype, device="cuda")
    m = model.cstruct()
    F.check(_lib().ptk_delta(ctx.handle, C.byref(m), mode, coords.data_ptr() if n else None, n, F.PREC[precision],
                             out.data_ptr() if n else None, _stream(stream)), "ptk_delta")
    return out


def row_sums(ctx: Context, delta: torch.Tensor, row_ptr: torch.Tensor, rid: torch.Tensor, J: int, schedule="auto",
             digits=4, stream=None):
    """B_i (upper triangle, row-major) and c_i of Eqs. (rowB), (rowC) for
    slice-ordered Delta rows [delta_0..delta_{J-1}, x] (``delta`` [nnz][ld],
    ld = J + 1 rounded up to an odd number): FP64 [rows][J(J+1)/2 + J]."""
    delta = delta.contiguous()
    row_ptr = row_ptr.to(torch.int64).contiguous()
    rid = rid.to(torch.int32).contiguous()
    rows = row_ptr.shape[0] - 1
    nnz = delta.shape[0]
    out = torch.empty((rows, J * (J + 1) // 2 + J), dtype=torch.float64, device="cuda")
    F.check(_lib().ptk_row_sums(ctx.handle, delta.data_ptr() if nnz else None, _dt(delta), delta.shape[1], J,
                                row_ptr.data_ptr(), rid.data_ptr() if nnz else None, rows, nnz,
                                F.SCHEDULE[schedule], digits, out.data_ptr(), _stream(stream)), "ptk_row_sums")
    return out


def fit(ctx: Context, x: SparseObs, slices, model: Model, *, variant="plain", precision="fp32", lam=0.01,
        trunc_rate=0.2, trunc_rule="r_beta", max_sweeps=5, tol=0.0, finalize_qr=False, graphs=True, stream=None):
    """Alg. 2 on one problem; returns the per-sweep errors."""
    return fit_many(ctx, [(x, slices, model)], variant=variant, precision=precision, lam=lam, trunc_rate=trunc_rate,
                    trunc_rule=trunc_rule, max_sweeps=max_sweeps, tol=tol, finalize_qr=finalize_qr, lanes=1,
                    graphs=graphs, stream=stream)[0]


def fit_many(ctx: Context, problems, *, variant="plain", precision="fp32", lam=0.01, trunc_rate=0.2,
             trunc_rule="r_beta", max_sweeps=5, tol=0.0, finalize_qr=False, lanes=0, graphs=True, autotune=False,
             stream=None):
    """Alg. 2 on independent problems [(x, slices, model), ...] batched over
    `lanes` streams; returns each problem's per-sweep errors."""
    count = len(problems)
    p = (F.Problem * max(count, 1))()
    for i, (x, slices, model) in enumerate(problems):
        p[i].x = x.cstruct()
        for k, s in enumerate(slices):
            p[i].slices[k] = s._h
        p[i].model = model.cstruct()
    o = F.FitOpts()
    o.als = _opts(variant, precision, lam, trunc_rate, trunc_rule, True)
    o.max_sweeps = max_sweeps
    o.tol = tol
    o.finalize_qr = 1 if finalize_qr else 0
    o.lanes = lanes
    o.graphs = 1 if graphs else 0
    o.autotune = 1 if autotune else 0
    errs = (C.c_double * max(1, count * max_sweeps))()
    sw = (C.c_int32 * max(1, count))()
    F.check(_lib().ptk_fit(ctx.handle, p, count, C.byref(o), errs, sw, _stream(stream)), "ptk_fit")
    return [[errs[i * max_sweeps + s] for s in range(sw[i])] for i in range(count)]


def autotune_delta(ctx: Context, slices: "Slices", model: Model, precision="fp32", max_entries=1 << 18, reps=2,
                   stream=None):
    """Times the delta launch shapes for the model's class on the first
    `max_entries` entries of `slices` and keeps the fastest in the context.
    Returns the candidates [(backend, chunk_kb, ctas_per_sm, ms, entries_per_thread)] and the index chosen."""
    r = F.TuneReport()
    m = model.cstruct()
    F.check(_lib().ptk_autotune_delta(ctx.handle, slices._h, C.byref(m), F.PREC[precision], max_entries, reps,
                                      C.byref(r), _stream(stream)), "ptk_autotune_delta")
    names = {1: "cuda_cores", 2: "tensor_cores"}
    cands = [(names[r.backend[i]], r.chunk_kb[i], r.ctas_per_sm[i], r.ms[i], r.entries_per_thread[i])
             for i in range(r.candidates)]
    return cands, r.best


def selftest_wait(ctx: Context, limit=4096, stream=None):
    """Runs the bounded-wait self-test; returns the status code (PTK_ERR_TIMEOUT expected)."""
    return _lib().ptk_selftest_wait(ctx.handle, limit, _stream(stream))


def autotune_clear(ctx: Context):
    _lib().ptk_autotune_clear(ctx.handle)


def foldin(ctx: Context, model: Model, mode: int, obs_ptr, obs_idx, obs_vals, query_ptr, query_idx, lam=0.01,
           precision="fp32", stream=None):
    """Rows for new mode-``mode`` slices and predictions of their query coordinates.

    obs_ptr / query_ptr: int64 [count+1] offsets; obs_idx / query_idx: int32 [*][N]
    (mode column ignored); obs_vals: model dtype.  Returns (rows [count][J], preds)."""
    count = int(obs_ptr.shape[0]) - 1
    Jn = model.J[mode]
    dt = model.core.dtype
    rows = torch.empty((max(count, 0), Jn), dtype=dt, device="cuda")
    nq = int(query_idx.shape[0]) if query_idx is not None else 0
    preds = torch.empty(max(nq, 1), dtype=dt, device="cuda")
    b = F.FoldinBatch()
    b.count = count
    b.obs_ptr = obs_ptr.data_ptr()
    b.obs_idx = obs_idx.data_ptr() if obs_idx.numel() else None
    b.obs_vals = obs_vals.data_ptr() if obs_vals.numel() else None
    b.query_ptr = query_ptr.data_ptr() if query_ptr is not None else None
    b.query_idx = query_idx.data_ptr() if nq else None
    b.rows_out = rows.data_ptr() if rows.numel() else None
    b.preds_out = preds.data_ptr()
    b.total_obs = int(obs_idx.shape[0])
    b.total_query = nq
    m = model.cstruct()
    F.check(_lib().ptk_foldin(ctx.handle, C.byref(m), mode, C.byref(b), lam, F.PREC[precision], _stream(stream)),
            "ptk_foldin")
    return rows, preds[:nq]


class DeviceServer:
    """Fold-in server whose request loop runs on the GPU (ptk_dserver_*):
    persistent CTAs take requests from a ring in mapped host memory; each
    request is computed by one CTA, so results are the same alone and in any
    mix."""

    def __init__(self, model: Model, mode: int, *, lam=0.01, ring=1024, arena_bytes=64 << 20, max_queries=1024,
                 max_pending=1 << 16, workers=0, idle_ms=50.0, device=0):
        self.model = model  # keeps the device arrays alive
        self.mode = mode
        self.J = model.J[mode]
        self.np_dtype = np.float64 if model.core.dtype == torch.float64 else np.float32
        o = F.DServerOpts()
        o.mode, o.lam, o.ring, o.arena_bytes = mode, lam, ring, arena_bytes
        o.max_queries, o.max_pending, o.workers, o.idle_ms = max_queries, max_pending, workers, idle_ms
        self._m = model.cstruct()
        self._h = C.c_void_p()
        F.check(_lib().ptk_dserver_create(C.byref(self._m), device, C.byref(o), C.byref(self._h)),
                "ptk_dserver_create")

    @staticmethod
    def clock():
        """Seconds on the clock arrival times and latencies use."""
        return _lib().ptk_clock_seconds()

    def submit(self, obs_idx, obs_vals, query_idx, arrival_s=0.0):
        oi = np.ascontiguousarray(obs_idx, dtype=np.int32)
        ov = np.ascontiguousarray(obs_vals, dtype=self.np_dtype)
        qi = np.ascontiguousarray(query_idx, dtype=np.int32)
        t = C.c_uint64()
        F.check(_lib().ptk_dserver_submit(self._h, oi.ctypes.data if oi.size else None,
                                          ov.ctypes.data if ov.size else None, oi.shape[0],
                                          qi.ctypes.data if qi.size else None, qi.shape[0], float(arrival_s),
                                          C.byref(t)), "ptk_dserver_submit")
        return t.value, qi.shape[0]

    def poll(self, ticket, nq):
        row = np.empty(self.J, dtype=self.np_dtype)
        preds = np.empty(max(nq, 1), dtype=self.np_dtype)
        done = C.c_int32()
        lat = C.c_double()
        F.check(_lib().ptk_dserver_poll(self._h, ticket, row.ctypes.data, preds.ctypes.data, C.byref(done),
                                        C.byref(lat)), "ptk_dserver_poll")
        return (row, preds[:nq], lat.value) if done.value else None

    def wait(self, ticket, nq, timeout_s=60.0):
        import time
        t0 = time.perf_counter()
        while True:
            r = self.poll(ticket, nq)
            if r is not None:
                return r
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError(f"request {ticket} not done after {timeout_s} s")
            time.sleep(20e-6)

    def stats(self):
        st = F.DServerStats()
        F.check(_lib().ptk_dserver_read_stats(self._h, C.byref(st)), "ptk_dserver_read_stats")
        return {k: getattr(st, k) for k, _ in F.DServerStats._fields_}

    def close(self):
        if self._h:
            _lib().ptk_dserver_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching fold-in server (ptk_server_*): requests are new
    slices of `mode`; results are bit-identical alone and in any mix."""

    def __init__(self, model: Model, mode: int, *, lam=0.01, precision="fp32", max_batch_requests=256,
                 max_batch_entries=1 << 20, max_batch_queries=1 << 16, memory_cap_bytes=1 << 30, slots=3,
                 max_queue=1 << 16, device=0):
        self.model = model  # keeps the device arrays alive
        self.mode = mode
        self.J = model.J[mode]
        self.np_dtype = np.float64 if model.core.dtype == torch.float64 else np.float32
        o = F.ServerOpts()
        o.mode, o.lam, o.precision = mode, lam, F.PREC[precision]
        o.max_batch_requests, o.max_batch_entries, o.max_batch_queries = max_batch_requests, max_batch_entries, \
            max_batch_queries
        o.memory_cap_bytes, o.slots, o.max_queue = memory_cap_bytes, slots, max_queue
        self._m = model.cstruct()
        self._h = C.c_void_p()
        F.check(_lib().ptk_server_create(C.byref(self._m), device, C.byref(o), C.byref(self._h)), "ptk_server_create")

    def submit(self, obs_idx, obs_vals, query_idx):
        """Queue a request (host arrays).  Returns its ticket; raises PtkError
        (status BUSY) when admission refuses it."""
        oi = np.ascontiguousarray(obs_idx, dtype=np.int32)
        ov = np.ascontiguousarray(obs_vals, dtype=self.np_dtype)
        qi = np.ascontiguousarray(query_idx, dtype=np.int32)
        t = C.c_uint64()
        F.check(_lib().ptk_server_submit(self._h, oi.ctypes.data if oi.size else None,
                                         ov.ctypes.data if ov.size else None, oi.shape[0],
                                         qi.ctypes.data if qi.size else None, qi.shape[0], C.byref(t)),
                "ptk_server_submit")
        return t.value, qi.shape[0]

    def poll(self, ticket, nq):
        """(row, predictions, latency_ms) when done, else None."""
        row = np.empty(self.J, dtype=self.np_dtype)
        preds = np.empty(max(nq, 1), dtype=self.np_dtype)
        done = C.c_int32()
        lat = C.c_double()
        F.check(_lib().ptk_server_poll(self._h, ticket, row.ctypes.data, preds.ctypes.data, C.byref(done),
                                       C.byref(lat)), "ptk_server_poll")
        return (row, preds[:nq], lat.value) if done.value else None

    def wait(self, ticket, nq, timeout_s=60.0):
        import time
        t0 = time.perf_counter()
        while True:
            r = self.poll(ticket, nq)
            if r is not None:
                return r
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError(f"request {ticket} not done after {timeout_s} s")
            time.sleep(50e-6)

    def stats(self):
        st = F.ServerStats()
        F.check(_lib().ptk_server_read_stats(self._h, C.byref(st)), "ptk_server_read_stats")
        return {k: getattr(st, k) for k, _ in F.ServerStats._fields_}

    def close(self):
        if self._h:
            _lib().ptk_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
