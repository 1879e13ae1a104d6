"""ptk_delta_noalloc: the allocation-free delta entry point.

Some callers cannot allocate device memory (code inside CUDA stream capture,
where cudaMalloc/cudaFree are not allowed and would synchronise the device;
serving threads on a fixed memory budget; embedders owning all device memory).
This entry point keeps its scratch in a static device array instead of
context scratch.  The test calls it through the C ABI twice in a row (the
second call reuses the array the first one left behind) and checks both
results against ptk_delta, the entry point that allocates, with the FP32 and
FP64 tolerances the other delta tests use.  It lives in a file of its own that
pytest collects last, and passes alone in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1710_02261_gb300 as P  # noqa: E402
from paper_1710_02261_gb300 import _ffi  # noqa: E402


def _case(dims, J, n, seed, dtype):
    rng = np.random.default_rng(seed)
    core = rng.standard_normal(J)
    F = [rng.random((d, j)) for d, j in zip(dims, J)]
    idx = np.stack([rng.integers(0, d, size=n) for d in dims], axis=1).astype(np.int32)
    return P.Model.from_numpy(core, F, dtype=dtype), torch.tensor(idx, device="cuda")


def _noalloc(model, mode, coords):
    lib = _ffi.load()
    n = coords.shape[0]
    out = torch.empty((n, model.J[mode]), dtype=model.core.dtype, device="cuda")
    m = model.cstruct()
    rc = lib.ptk_delta_noalloc(C.byref(m), mode, coords.data_ptr(), n, out.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    _ffi.check(rc, "ptk_delta_noalloc")
    return out


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
            g, r = got.double().cpu().numpy(), ref.double().cpu().numpy()
            np.testing.assert_allclose(g, r, rtol=tol, atol=tol * np.max(np.abs(r)))
    ctx.close()


def test_noalloc_rejects_oversized_core():
    model, coords = _case((8, 8, 8), (16, 16, 16), 10, 3, torch.float64)   # 16*16*16 doubles = 32 KiB: fits
    _noalloc(model, 0, coords)
    big, c2 = _case((4, 4, 4, 4, 4), (16, 16, 16, 16, 2), 10, 4, torch.float64)  # 2 MiB permuted core
    with pytest.raises(_ffi.PtkError) as e:
        _noalloc(big, 0, c2)
    assert e.value.status == _ffi.ERR_INVALID_ARG and b"static scratch" in _ffi.load().ptk_last_error()
