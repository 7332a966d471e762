"""The C ABI on the CPU: the library loads, exports every symbol include/shine.h declares, and
rejects bad arguments on the host before touching a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "shine.h")).read()
    return sorted(set(re.findall(r"SHINE_API\s+[\w\s\*]+?\b(shine_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2201_03611_b300 import _lib
    return _lib.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("shine_pipeline_fwd", "shine_pipeline_bwd", "shine_pipeline_bwd_workspace",
              "shine_pipeline_fwd_bwd", "shine_plan_create", "shine_pipeline_batched", "shine_plan_destroy",
              "shine_status_string", "shine_output_shape"):
        assert n in names


def test_every_declared_symbol_is_exported(L):
    for name in _declared():
        assert hasattr(L, name), name


def _exported(path):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    return {ln.split()[-1] for ln in out.splitlines() if " T " in ln}


def test_only_the_abi_is_exported():
    from paper_2201_03611_b300._lib import LIB_PATH
    assert _exported(LIB_PATH) == set(_declared())


def test_status_strings(L):
    from paper_2201_03611_b300 import _lib
    assert _lib.status_string(0) == "ok"
    for s in range(1, 6):
        assert _lib.status_string(s) not in ("ok", "unknown status")
    assert _lib.status_string(99) == "unknown status"


def test_output_shape(L):
    from paper_2201_03611_b300.ops import output_shape
    from paper_2201_03611_b300._lib import ShineError
    assert output_shape(256, 256, "valid") == (252, 252)
    assert output_shape(1, 1, "clamp") == (1, 1)
    assert output_shape(8192, 8192, "clamp") == (8192, 8192)
    with pytest.raises(ShineError):
        output_shape(4, 9, "valid")
    with pytest.raises(ShineError):
        output_shape(0, 9, "clamp")
    with pytest.raises(ShineError):
        output_shape(2 ** 31, 9, "clamp")


def _fwd(L, img=1 << 12, H=8, W=8, pitch=24, dt=0, border=1, kappa=1 << 12, wx=1 << 12, wy=1 << 12,
         out=1 << 12, out_pitch=8, out_dt=0):
    v = ctypes.c_void_p
    return L.shine_pipeline_fwd(v(img), H, W, pitch, dt, border, v(kappa), v(wx), v(wy), v(out), out_pitch,
                                out_dt, None)


def test_fwd_rejects_bad_arguments_on_the_host(L):
    # every one of these returns before any CUDA call (the pointers are never dereferenced)
    assert _fwd(L, img=0) == 1
    assert _fwd(L, out=0) == 1
    assert _fwd(L, kappa=0) == 1
    assert _fwd(L, dt=7) == 1
    assert _fwd(L, border=3) == 1
    assert _fwd(L, H=0) == 1
    assert _fwd(L, H=4, border=0) == 1
    assert _fwd(L, pitch=23) == 1            # pitch < 3W
    assert _fwd(L, out_pitch=7) == 1         # pitch < W_out
    assert _fwd(L, out_dt=1) == 4            # f32 image -> bf16 output is not offered
    assert _fwd(L, img=(1 << 12) + 1) == 2   # misaligned element pointer
    assert _fwd(L, wx=(1 << 12) + 2) == 2


def test_bwd_workspace_and_errors(L):
    n = ctypes.c_size_t()
    assert L.shine_pipeline_bwd_workspace(64, 64, 1, ctypes.byref(n)) == 0 and n.value > 0
    assert n.value % 8 == 0
    assert L.shine_pipeline_bwd_workspace(4, 64, 0, ctypes.byref(n)) == 1
    v = ctypes.c_void_p
    p = v(1 << 12)
    # workspace missing -> SHINE_ERR_WORKSPACE, checked before anything is launched
    rc = L.shine_pipeline_bwd(p, 64, 64, 192, 0, 1, p, p, p, p, 64, 0, p, 192, p, p, p, None, 0, None)
    assert rc == 3
    rc = L.shine_pipeline_bwd(p, 64, 64, 192, 0, 1, p, p, p, None, 64, 0, p, 192, p, p, p, p, 1 << 20, None)
    assert rc == 1
    rc = L.shine_pipeline_fwd_bwd(p, 64, 64, 192, 0, 1, p, p, p, p, 64, p, 64, p, 192, p, p, p, None, 0, None)
    assert rc == 3


def test_plan_rejects_bad_arguments(L):
    handle = ctypes.c_void_p()
    hw = (ctypes.c_int64 * 4)(8, 8, 3, 9)
    assert L.shine_plan_create(hw, 2, 0, 0, 3, None, ctypes.byref(handle)) == 1   # 3x9 is too small for VALID
    assert L.shine_plan_create(hw, 0, 0, 1, 3, None, ctypes.byref(handle)) == 1
    assert L.shine_plan_create(hw, 2, 0, 1, 2, None, ctypes.byref(handle)) == 1   # mode 2 is not a mode
    L.shine_plan_destroy(None)


def test_package_import_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib
    from paper_2201_03611_b300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.lib()
    importlib.reload(_lib)


def test_debug_build_exports_the_same_symbols():
    """libshine_debug.so (index checks compiled in) offers exactly the release library's ABI."""
    import os
    from paper_2201_03611_b300 import _lib
    if not os.path.exists(_lib.DEBUG_LIB_PATH):
        pytest.skip("libshine_debug.so not built")
    assert _exported(_lib.DEBUG_LIB_PATH) == _exported(_lib.LIB_PATH)
