"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every function include/ptk.h declares, and the ctypes structs have the
C layout."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ptk.h")


def _lib():
    from paper_1710_02261_gb300 import _ffi
    if not os.path.exists(_ffi.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("libptk.so not built and nvcc unavailable")
        from paper_1710_02261_gb300 import build
        build.build()
    return _ffi, _ffi.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:ptk_status|void|int64_t|int|double|const char\s*\*)\s*(ptk_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported():
    ffi, lib = _lib()
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"
        assert n in ffi.SIGNATURES, f"{n} has no ctypes signature"
    assert set(ffi.SIGNATURES) == set(names)


def test_struct_layout_matches_c():
    ffi, _ = _lib()
    if shutil.which("gcc") is None:
        pytest.skip("gcc unavailable")
    structs = {"ptk_coo": ffi.Coo, "ptk_model": ffi.Model, "ptk_als_opts": ffi.AlsOpts,
               "ptk_sweep_stats": ffi.SweepStats, "ptk_problem": ffi.Problem, "ptk_fit_opts": ffi.FitOpts,
               "ptk_foldin_batch": ffi.FoldinBatch, "ptk_server_opts": ffi.ServerOpts,
               "ptk_server_stats": ffi.ServerStats}
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "ptk.h"', "int main(void){"]
    for cname in structs:
        src.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
    src += ['printf("ptk_model.core %zu\\n", offsetof(ptk_model, core));',
            'printf("ptk_model.ld %zu\\n", offsetof(ptk_model, ld));',
            'printf("ptk_foldin_batch.total_obs %zu\\n", offsetof(ptk_foldin_batch, total_obs));',
            'printf("ptk_problem.model %zu\\n", offsetof(ptk_problem, model));',
            'printf("ptk_server_opts.max_queue %zu\\n", offsetof(ptk_server_opts, max_queue));', "return 0;}"]
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        open(c, "w").write("\n".join(src))
        exe = os.path.join(d, "l")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = dict(line.split() for line in out.strip().splitlines())
    import ctypes as C
    for cname, cls in structs.items():
        assert int(got[cname]) == C.sizeof(cls), cname
    assert int(got["ptk_model.core"]) == ffi.Model.core.offset
    assert int(got["ptk_model.ld"]) == ffi.Model.ld.offset
    assert int(got["ptk_foldin_batch.total_obs"]) == ffi.FoldinBatch.total_obs.offset
    assert int(got["ptk_problem.model"]) == ffi.Problem.model.offset
    assert int(got["ptk_server_opts.max_queue"]) == ffi.ServerOpts.max_queue.offset


def test_version_and_error_string():
    _, lib = _lib()
    assert lib.ptk_version().startswith(b"ptk")
    assert isinstance(lib.ptk_last_error(), bytes)


def test_null_arguments_are_rejected_without_a_device():
    ffi, lib = _lib()
    # argument checks run before any CUDA call
    assert lib.ptk_create(None, 0) == ffi.ERR_INVALID_ARG
    assert lib.ptk_build_mode_slices(None, None, 0, 0, None, None) == ffi.ERR_INVALID_ARG
    assert lib.ptk_als_sweep(None, None, None, None, None, None, None) == ffi.ERR_INVALID_ARG
    assert lib.ptk_predict(None, None, None, 0, None, None) == ffi.ERR_INVALID_ARG
    assert b"null" in lib.ptk_last_error()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1710_02261_gb300 import _ffi
    saved = _ffi._lib
    try:
        _ffi._lib = None
        with pytest.raises(ImportError):
            _ffi.load(str(tmp_path / "missing.so"))
    finally:
        _ffi._lib = saved
