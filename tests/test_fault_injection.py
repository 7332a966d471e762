"""The host-side fault injector of the C ABI (SHINE_FAULT_INJECT="<call>=<status>[,...]", "*" for
every call): a named entry point returns the injected status before reading its arguments or
touching a GPU, and the Python binding turns it into ShineError. Runs on the CPU; no compute
call ever reaches a kernel here (every call below returns on the host)."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def L():
    from paper_2201_03611_b300 import _lib
    return _lib.lib()


@pytest.fixture
def inject(monkeypatch):
    def set_spec(spec):
        monkeypatch.setenv("SHINE_FAULT_INJECT", spec)
    yield set_spec
    monkeypatch.delenv("SHINE_FAULT_INJECT", raising=False)


def _fwd_null(L):
    # a NULL image: an argument error (1) unless a fault is injected first
    v = ctypes.c_void_p
    return L.shine_pipeline_fwd(None, 8, 8, 24, 0, 1, v(4096), v(4096), v(4096), v(4096), 8, 0, None)


def _mv_null(L):
    return L.shine_mv(None, 4, 4, 4, 0, None, None, None)


def _its_null(L):
    return L.shine_iterate_stencil(None, 4, 4, 4, None, 1, None, 4, None)


def test_no_injection_by_default(L, monkeypatch):
    monkeypatch.delenv("SHINE_FAULT_INJECT", raising=False)
    assert _fwd_null(L) == 1 and _mv_null(L) == 1 and _its_null(L) == 1


def test_named_call_returns_the_injected_status(L, inject):
    inject("shine_pipeline_fwd=5")
    assert _fwd_null(L) == 5          # before the argument check
    assert _mv_null(L) == 1           # other calls are untouched
    inject("shine_mv=4,shine_iterate_stencil=3")
    assert _fwd_null(L) == 1 and _mv_null(L) == 4 and _its_null(L) == 3


def test_wildcard_and_malformed_specs(L, inject):
    inject("*=2")
    assert _fwd_null(L) == 2 and _mv_null(L) == 2 and _its_null(L) == 2
    for bad in ("shine_pipeline_fwd=9", "shine_pipeline_fwd=0", "shine_pipeline_fwd", "=5", "shine_pipeline_fw=5",
                "shine_pipeline_fwd_extra=5"):
        inject(bad)
        assert _fwd_null(L) == 1, bad


def _noalloc_null(L):
    v = ctypes.c_void_p
    return L.shine_pipeline_bwd_noalloc(None, 8, 8, 24, 0, 1, v(4096), v(4096), v(4096), v(4096), 8, 0, None, 24,
                                        None, None, None, None)


def test_noalloc_is_targeted_on_its_own(L, inject):
    # the no-allocation backward consults the injector once, under its own name: injecting into
    # shine_pipeline_bwd leaves it alone, and injecting into it leaves shine_pipeline_bwd alone
    v = ctypes.c_void_p
    bwd_null = lambda: L.shine_pipeline_bwd(None, 8, 8, 24, 0, 1, v(4096), v(4096), v(4096), v(4096), 8, 0, None, 24,
                                            None, None, None, None, 0, None)
    inject("shine_pipeline_bwd=5")
    assert bwd_null() == 5 and _noalloc_null(L) == 1
    inject("shine_pipeline_bwd_noalloc=4")
    assert bwd_null() == 1 and _noalloc_null(L) == 4


def test_binding_raises_shine_error(L, inject):
    from paper_2201_03611_b300 import _lib
    inject("shine_mv=5")
    with pytest.raises(_lib.ShineError, match="CUDA error"):
        _lib.check(_mv_null(L), "shine_mv")
