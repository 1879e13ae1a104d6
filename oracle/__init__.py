"""FP64 CPU oracle for P-Tucker (arXiv 1710.02261) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the timed CPU baseline of
``bench.py`` may import this package.  The product (``paper_1710_02261_gb300``)
never does, and the two share no code.  The arithmetic lives in plain C
(``ptk_oracle.c``, double precision, literal loops in the paper's order); this
module compiles it with gcc and marshals numpy arrays through ctypes.

Parity status: every function is pinned by ``tests/test_oracle_pins.py``
against brute force, closed forms or the paper's theorems.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ptk_oracle.c")
_LIB = os.path.join(_HERE, "libptk_oracle.so")
_lock = threading.Lock()
_lib = None

_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_pp = C.POINTER(C.c_void_p)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FMA contraction so x86 and Arm agree)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB)
    lib.ora_slices.argtypes = [C.c_int, _i64p, C.c_int64, _i32p, C.c_int, _i64p, _i64p]
    lib.ora_slices.restype = C.c_int
    lib.ora_delta.argtypes = [C.c_int, _i32p, _f64p, _pp, _i32p, C.c_int, _f64p]
    lib.ora_delta.restype = None
    lib.ora_predict.argtypes = [C.c_int, _i32p, _f64p, _pp, C.c_int64, _i32p, _f64p]
    lib.ora_predict.restype = None
    lib.ora_sse.argtypes = [C.c_int, _i32p, _f64p, _pp, C.c_int64, _i32p, _f64p]
    lib.ora_sse.restype = C.c_double
    lib.ora_loss.argtypes = [C.c_int, _i64p, _i32p, _f64p, _pp, C.c_int64, _i32p, _f64p, C.c_double]
    lib.ora_loss.restype = C.c_double
    lib.ora_spd_solve.argtypes = [C.c_int, _f64p, _f64p, C.c_double, _f64p]
    lib.ora_spd_solve.restype = C.c_int
    lib.ora_row_update.argtypes = [C.c_int, _i32p, _f64p, _pp, C.c_int, C.c_int64, C.c_void_p, _i32p, _f64p,
                                   C.c_double, _f64p, C.c_void_p, C.c_void_p]
    lib.ora_row_update.restype = C.c_int
    lib.ora_update_mode.argtypes = [C.c_int, _i64p, _i32p, C.c_int64, _i32p, _f64p, _f64p, _pp, C.c_int,
                                    C.c_double, C.c_int]
    lib.ora_update_mode.restype = C.c_int
    lib.ora_sweep.argtypes = [C.c_int, _i64p, _i32p, C.c_int64, _i32p, _f64p, _f64p, _pp, C.c_double, C.c_int]
    lib.ora_sweep.restype = C.c_int
    lib.ora_sweep_cache.argtypes = lib.ora_sweep.argtypes
    lib.ora_sweep_cache.restype = C.c_int
    lib.ora_partial_error.argtypes = [C.c_int, _i32p, _f64p, _pp, C.c_int64, _i32p, _f64p, C.c_int, _f64p]
    lib.ora_partial_error.restype = None
    lib.ora_truncate.argtypes = [C.c_int, _i32p, _f64p, _f64p, C.c_double, C.c_int, C.c_void_p]
    lib.ora_truncate.restype = C.c_int64
    lib.ora_qr_finalize.argtypes = [C.c_int, _i64p, _i32p, _f64p, _pp]
    lib.ora_qr_finalize.restype = C.c_int
    lib.ora_fit.argtypes = [C.c_int, _i64p, _i32p, C.c_int64, _i32p, _f64p, _f64p, _pp, C.c_double, C.c_int,
                            C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, _f64p]
    lib.ora_fit.restype = C.c_int
    lib.ora_max_threads.argtypes = []
    lib.ora_max_threads.restype = C.c_int
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
def _dims(d):
    return np.ascontiguousarray(d, dtype=np.int64)


def _J(core):
    return np.ascontiguousarray(core.shape, dtype=np.int32)


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _idx(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class _Factors:
    """Keeps float64 C-contiguous factor arrays alive and exposes double**."""

    def __init__(self, factors, copy=False):
        self.arrays = [np.array(a, dtype=np.float64, order="C", copy=True) if copy else _f(a) for a in factors]
        self.ptrs = (C.c_void_p * len(self.arrays))(*[a.ctypes.data for a in self.arrays])

    @property
    def pp(self):
        return C.cast(self.ptrs, _pp)


def max_threads() -> int:
    return int(_load().ora_max_threads())


def slices(dims, idx, mode):
    """Stable grouping of entries by their mode-``mode`` index: (perm, row_ptr)."""
    idx = _idx(idx)
    E, N = idx.shape
    perm = np.empty(E, dtype=np.int64)
    rp = np.empty(int(dims[mode]) + 1, dtype=np.int64)
    rc = _load().ora_slices(N, _dims(dims), E, idx, mode, perm, rp)
    if rc:
        raise ValueError(f"ora_slices failed ({rc})")
    return perm, rp


def delta(core, factors, coord, mode):
    core = _f(core)
    F = _Factors(factors)
    out = np.empty(core.shape[mode], dtype=np.float64)
    _load().ora_delta(core.ndim, _J(core), core, F.pp, np.ascontiguousarray(coord, dtype=np.int32), mode, out)
    return out


def predict(core, factors, coords):
    core = _f(core)
    coords = _idx(coords)
    F = _Factors(factors)
    out = np.empty(coords.shape[0], dtype=np.float64)
    _load().ora_predict(core.ndim, _J(core), core, F.pp, coords.shape[0], coords, out)
    return out


def sse(core, factors, idx, vals):
    core = _f(core)
    idx = _idx(idx)
    F = _Factors(factors)
    return float(_load().ora_sse(core.ndim, _J(core), core, F.pp, idx.shape[0], idx, _f(vals)))


def error_stats(core, factors, idx, vals):
    """Eq. (reconfull) error, RMSE over the given set, and relative error."""
    s = sse(core, factors, idx, vals)
    n = max(1, len(vals))
    xs = float(np.sum(np.asarray(vals, dtype=np.float64) ** 2))
    return dict(sse=s, error=s ** 0.5, rmse=(s / n) ** 0.5, rel=(s ** 0.5) / (xs ** 0.5 if xs > 0 else 1.0))


def loss(dims, core, factors, idx, vals, lam):
    core = _f(core)
    idx = _idx(idx)
    F = _Factors(factors)
    return float(_load().ora_loss(core.ndim, _dims(dims), _J(core), core, F.pp, idx.shape[0], idx, _f(vals), lam))


def spd_solve(B, c, lam):
    B = _f(B)
    n = B.shape[0]
    a = np.empty(n, dtype=np.float64)
    rc = _load().ora_spd_solve(n, B, _f(c), lam, a)
    return a, rc


def row_update(core, factors, mode, idx, vals, lam, entries=None):
    """Row update from the given entries: returns (row, B, c)."""
    core = _f(core)
    idx = _idx(idx)
    vals = _f(vals)
    F = _Factors(factors)
    Jn = core.shape[mode]
    row = np.empty(Jn, dtype=np.float64)
    B = np.empty((Jn, Jn), dtype=np.float64)
    c = np.empty(Jn, dtype=np.float64)
    if entries is None:
        m, ep = idx.shape[0], None
    else:
        entries = np.ascontiguousarray(entries, dtype=np.int64)
        m, ep = entries.shape[0], entries.ctypes.data
    rc = _load().ora_row_update(core.ndim, _J(core), core, F.pp, mode, m, ep, idx, vals, lam, row,
                                B.ctypes.data, c.ctypes.data)
    return row, B, c, rc


def update_mode(dims, core, factors, idx, vals, mode, lam, nthreads=1):
    """Alg. 3 for a single mode; returns new factor list (inputs untouched)."""
    core = _f(core)
    idx = _idx(idx)
    F = _Factors(factors, copy=True)
    rc = _load().ora_update_mode(core.ndim, _dims(dims), _J(core), idx.shape[0], idx, _f(vals), core, F.pp,
                                 mode, lam, nthreads)
    return F.arrays, rc


def sweep(dims, core, factors, idx, vals, lam, variant="plain", nthreads=1):
    """One ALS sweep (Alg. 3, modes 1..N); returns new factors and status."""
    core = _f(core)
    idx = _idx(idx)
    F = _Factors(factors, copy=True)
    fn = _load().ora_sweep_cache if variant == "cache" else _load().ora_sweep
    rc = fn(core.ndim, _dims(dims), _J(core), idx.shape[0], idx, _f(vals), core, F.pp, lam, nthreads)
    return F.arrays, rc


def partial_error(core, factors, idx, vals, literal=False):
    core = _f(core)
    idx = _idx(idx)
    F = _Factors(factors)
    R = np.empty(core.size, dtype=np.float64)
    _load().ora_partial_error(core.ndim, _J(core), core, F.pp, idx.shape[0], idx, _f(vals), int(bool(literal)), R)
    return R.reshape(core.shape)


def truncate(core, R, p, rule="r_beta"):
    """Alg. 4 selection; returns (new core, removed linear indices)."""
    G = np.array(core, dtype=np.float64, order="C", copy=True)
    Rf = _f(R).reshape(-1) if R is not None else np.zeros(G.size)
    removed = np.empty(G.size, dtype=np.int64)
    k = _load().ora_truncate(G.ndim, _J(G), G, Rf, p, 0 if rule == "r_beta" else 1, removed.ctypes.data)
    return G, removed[:k].copy()


def qr_finalize(dims, core, factors):
    G = np.array(core, dtype=np.float64, order="C", copy=True)
    F = _Factors(factors, copy=True)
    rc = _load().ora_qr_finalize(G.ndim, _dims(dims), _J(G), G, F.pp)
    if rc:
        raise ValueError("QR finalisation needs I_n >= J_n")
    return G, F.arrays


def fit(dims, core, factors, idx, vals, lam, variant="plain", sweeps=5, tol=0.0, trunc_p=0.2,
        trunc_rule="r_beta", finalize=False, nthreads=1):
    G = np.array(core, dtype=np.float64, order="C", copy=True)
    idx = _idx(idx)
    F = _Factors(factors, copy=True)
    errs = np.zeros(max(1, sweeps), dtype=np.float64)
    v = {"plain": 0, "cache": 1, "approx": 2}[variant]
    s = _load().ora_fit(G.ndim, _dims(dims), _J(G), idx.shape[0], idx, _f(vals), G, F.pp, lam, v, sweeps, tol,
                        trunc_p, 0 if trunc_rule == "r_beta" else 1, int(bool(finalize)), nthreads, errs)
    if s < 0:
        raise RuntimeError(f"ora_fit failed ({s})")
    return G, F.arrays, errs[:s]


def foldin(core, factors, mode, obs_idx, obs_vals, lam):
    """Row for a new slice of mode ``mode`` from its observed entries
    (coordinates of the other modes in ``obs_idx`` columns, mode column ignored)."""
    core = _f(core)
    N = core.ndim
    idx = _idx(obs_idx)
    if idx.shape[1] == N - 1:
        full = np.zeros((idx.shape[0], N), dtype=np.int32)
        full[:, [k for k in range(N) if k != mode]] = idx
        idx = full
    facs = list(factors)
    facs[mode] = np.zeros((1, core.shape[mode]))
    idx = idx.copy()
    idx[:, mode] = 0
    row, B, c, rc = row_update(core, facs, mode, idx, obs_vals, lam)
    return row, rc
