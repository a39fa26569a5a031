"""Host-side tests of the C ABI (no GPU needed): the library builds, loads and
exports every function include/sadi.h declares; argument validation happens
before any device call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "sadi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(sadi_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2312_06206_gb300 import build
    build.build()
    from paper_2312_06206_gb300 import sadi
    return sadi.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ["sadi_create", "sadi_set_initial", "sadi_step", "sadi_get", "sadi_destroy",
              "sadi_set_options", "sadi_set_stream", "sadi_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared_functions():
        assert hasattr(lib, n), n
    from paper_2312_06206_gb300 import sadi
    assert set(sadi._SIGS) == set(_declared_functions())


@pytest.mark.parametrize("args,frag", [
    ((0, 1.5, 1.0, 0.01, (-1.0, 1.0)), "N must be"),
    ((8193, 1.5, 1.0, 0.01, (-1.0, 1.0)), "N must be"),
    ((15, 1.0, 1.0, 0.01, (-1.0, 1.0)), "alpha"),
    ((15, 2.5, 1.0, 0.01, (-1.0, 1.0)), "alpha"),
    ((15, float("nan"), 1.0, 0.01, (-1.0, 1.0)), "alpha"),
    ((15, 1.5, 0.0, 0.01, (-1.0, 1.0)), "kappa"),
    ((15, 1.5, 1.0, -0.01, (-1.0, 1.0)), "tau"),
    ((15, 1.5, 1.0, 0.01, (1.0, -1.0)), "domain"),
])
def test_create_rejects_invalid_arguments_without_a_gpu(lib, args, frag):
    from paper_2312_06206_gb300 import sadi
    with pytest.raises(sadi.SadiError) as ei:
        sadi.Sadi(*args)
    assert ei.value.status == sadi.SADI_EINVAL
    assert frag in str(ei.value)


def test_null_out_pointer_rejected(lib):
    dom = (ctypes.c_double * 2)(-1.0, 1.0)
    assert lib.sadi_create(15, 1.5, 1.0, 0.01, dom, None) == 1
    assert lib.sadi_create(15, 1.5, 1.0, 0.01, None, ctypes.byref(ctypes.c_void_p())) == 1
    assert b"NULL" in lib.sadi_last_error(None)
    lib.sadi_destroy(None)  # no-op


def test_noalloc_step_rejects_null_context_without_a_gpu(lib):
    assert lib.sadi_step_noalloc(None, None, None, None, 1) == 1


def test_batch_create_validates_before_any_device_call(lib):
    out = ctypes.c_void_p()
    n = (ctypes.c_int * 1)(63)
    d = (ctypes.c_double * 1)(1.5)
    assert lib.sadi_batch_create(0, n, d, d, d, None, 0, 1, ctypes.byref(out)) == 1      # count < 1
    assert out.value is None
    assert lib.sadi_batch_create(1, n, d, d, d, None, 0, 7, ctypes.byref(out)) == 1      # prec
    assert lib.sadi_batch_create(1, None, d, d, d, None, 0, 1, ctypes.byref(out)) == 1   # arrays
    assert b"prec" in lib.sadi_batch_last_error(None) or b"arrays" in lib.sadi_batch_last_error(None)
