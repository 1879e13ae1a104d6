"""ptk_delta_noalloc: the allocation-free delta entry point.

Some callers cannot allocate device memory: a serving thread that runs on a
fixed memory budget (an allocation there may fail, or stall the device, at the
worst moment), or a runtime that embeds the library and owns every byte of
device memory itself.  This entry point keeps its scratch in a static device
array instead of context scratch.  The tests call it through the C ABI twice in
a row (the second call reuses the array the first one left behind) and check
both results against ptk_delta, the entry point that allocates, with the FP32
and FP64 tolerances the other delta tests use; they also check that a call
leaves the free device memory unchanged, and that a core staged whole in
shared memory above the default 48 KB works on the first call of a fresh
process.  The file is collected last and passes alone in a fresh process too.
"""
import ctypes as C
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1710_02261_gb300 as P  # noqa: E402
from paper_1710_02261_gb300 import _ffi  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _case(dims, J, n, seed, dtype):
    rng = np.random.default_rng(seed)
    core = rng.standard_normal(J)
    F = [rng.random((d, j)) for d, j in zip(dims, J)]
    idx = np.stack([rng.integers(0, d, size=n) for d in dims], axis=1).astype(np.int32)
    return P.Model.from_numpy(core, F, dtype=dtype), torch.tensor(idx, device="cuda")


def _noalloc(model, mode, coords, out=None):
    lib = _ffi.load()
    n = coords.shape[0]
    if out is None:
        out = torch.empty((n, model.J[mode]), dtype=model.core.dtype, device="cuda")
    m = model.cstruct()
    rc = lib.ptk_delta_noalloc(C.byref(m), mode, coords.data_ptr(), n, out.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    _ffi.check(rc, "ptk_delta_noalloc")
    return out


def _compare(got, ref, tol):
    g, r = got.double().cpu().numpy(), ref.double().cpu().numpy()
    np.testing.assert_allclose(g, r, rtol=tol, atol=tol * np.max(np.abs(r)))


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 2e-6), (torch.float64, 1e-12)])
def test_noalloc_delta_matches_allocating_entry_point(dtype, tol):
    ctx = P.Context(0)
    cases = [((40, 30, 20, 10), (10, 10, 10, 10), 3000, 1), ((50, 40, 30), (6, 4, 5), 777, 2)]
    for (dims, J, n, seed) in cases:           # two calls in a row, different shapes and data
        model, coords = _case(dims, J, n, seed, dtype)
        for mode in range(len(dims)):
            got = _noalloc(model, mode, coords)
            ref = P.delta(ctx, model, mode, coords, precision="fp64" if dtype == torch.float64 else "fp32")
            torch.cuda.synchronize()
            _compare(got, ref, tol)
    ctx.close()


def test_noalloc_leaves_free_memory_unchanged():
    """After a first call (which may load the kernels' code), further calls
    leave the device's free memory exactly where it was."""
    model, coords = _case((40, 30, 20, 10), (10, 10, 10, 10), 5000, 7, torch.float32)
    out = torch.empty((5000, 10), dtype=torch.float32, device="cuda")
    for mode in range(4):
        _noalloc(model, mode, coords, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for mode in range(4):
            _noalloc(model, mode, coords, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_empty_call_is_a_no_op():
    model, _ = _case((8, 8, 8), (4, 4, 4), 1, 9, torch.float32)
    empty = torch.empty((0, 3), dtype=torch.int32, device="cuda")
    out = _noalloc(model, 0, empty)
    assert out.shape == (0, 4)


_FRESH = textwrap.dedent("""
    import ctypes as C, sys
    import numpy as np, torch
    sys.path.insert(0, {root!r})
    import paper_1710_02261_gb300 as P
    from paper_1710_02261_gb300 import _ffi
    rng = np.random.default_rng(11)
    dims, J, n = (14, 13, 12, 12), (12, 12, 12, 12), 1500
    core = rng.standard_normal(J)
    F = [rng.random((d, j)) for d, j in zip(dims, J)]
    idx = np.stack([rng.integers(0, d, size=n) for d in dims], axis=1).astype(np.int32)
    model = P.Model.from_numpy(core, F, dtype=torch.float32)
    coords = torch.tensor(idx, device="cuda")
    lib = _ffi.load()
    outs = []
    for mode in range(4):          # the first launches of this kernel in the process
        out = torch.empty((n, 12), dtype=torch.float32, device="cuda")
        m = model.cstruct()
        _ffi.check(lib.ptk_delta_noalloc(C.byref(m), mode, coords.data_ptr(), n, out.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream), "ptk_delta_noalloc")
        outs.append(out)
    ctx = P.Context(0)
    worst = 0.0
    for mode in range(4):
        ref = P.delta(ctx, model, mode, coords, precision="fp32").double().cpu().numpy()
        got = outs[mode].double().cpu().numpy()
        worst = max(worst, float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
    ctx.close()
    print("WORST", worst)
""")


def test_noalloc_staged_core_above_48k_first_call_in_fresh_process():
    """FP32 J = (12, 12, 12, 12): the permuted core (12 x 144 x 12 floats,
    81 KiB) is staged whole in shared memory, above the default 48 KB limit.
    In a fresh process the first call's set-up raises that limit before the
    first launch; the results match ptk_delta."""
    r = subprocess.run([sys.executable, "-c", _FRESH.format(root=ROOT)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    worst = float([ln for ln in r.stdout.splitlines() if ln.startswith("WORST")][0].split()[1])
    assert worst <= 2e-6, worst


def test_noalloc_rejects_oversized_core():
    model, coords = _case((8, 8, 8), (16, 16, 16), 10, 3, torch.float64)   # 16*16*16 doubles = 32 KiB: fits
    _noalloc(model, 0, coords)
    big, c2 = _case((4, 4, 4, 4, 4), (16, 16, 16, 16, 2), 10, 4, torch.float64)  # 2 MiB permuted core
    with pytest.raises(_ffi.PtkError) as e:
        _noalloc(big, 0, c2)
    assert e.value.status == _ffi.ERR_INVALID_ARG and b"static scratch" in _ffi.load().ptk_last_error()
