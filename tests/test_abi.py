"""The C-ABI library builds for sm_103a, loads, exports every declared entry point and
rejects bad arguments on the host (no GPU needed)."""
import ctypes as C

import numpy as np
import pytest

from paper_2606_04206_gb300 import build, dlo


@pytest.fixture(scope="module")
def lib():
    build.build()
    return dlo.load()


def test_every_declared_function_is_exported(lib):
    names = dlo.header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    assert lib.dlo_status_string(0) == b"ok"
    assert lib.dlo_status_string(1) == b"invalid argument"
    assert lib.dlo_status_string(8) == b"index out of bounds (debug build)"
    assert lib.dlo_status_string(99) == b"unknown status"
    assert lib.dlo_build_flags() == 0          # the release library has no bounds checks
    assert lib.dlo_last_error(None) == b"null context"


def _create(lib, nv, mat=None, opt=None, x=None):
    B = len(nv)
    mats = (dlo.Material * B)()
    for b in range(B):
        mats[b] = mat or dlo.Material(1000, 0.002, 1e5, 1e4, 1e3, 0, 0, 0, 0, 1, 1, 0)
    o = opt or dlo.Options(1e-3, 10, 5, 9.81, 0.3, 0.5, 0.0, 0.5, 2.0, 0, 0, 0, 0)
    nva = np.asarray(nv, np.int32)
    xs = np.zeros((max(int(np.sum(nv)), 1), 3), np.float32)
    xs[:, 0] = np.arange(len(xs)) * 0.01
    ctx = C.c_void_p()
    st = lib.dlo_create(C.byref(ctx), B, nva.ctypes.data_as(C.POINTER(C.c_int)), mats,
                        x if x is not None else xs.ctypes.data_as(C.POINTER(C.c_float)), None, C.byref(o), None,
                        None)
    return st, ctx


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    assert _create(lib, [1])[0] == 1                     # too few vertices
    assert _create(lib, [])[0] == 1                      # an empty batch
    assert _create(lib, [300])[0] == 1                   # above the 256-vertex limit
    bad = dlo.Material(-1, 0.002, 1e5, 1e4, 1e3, 0, 0, 0, 0, 1, 1, 0)
    assert _create(lib, [10], mat=bad)[0] == 1           # negative density
    closed2 = dlo.Material(1000, 0.002, 1e5, 1e4, 1e3, 0, 0, 0, 0, 1, 1, 1)
    assert _create(lib, [2], mat=closed2)[0] == 1        # a loop needs three vertices
    o = dlo.Options(0.0, 10, 5, 9.81, 0.3, 0.5, 0.0, 0.5, 2.0, 0, 0, 0, 0)
    assert _create(lib, [10], opt=o)[0] == 1             # dt must be positive
    st = lib.dlo_create(None, 1, None, None, None, None, None, None, None)
    assert st == 1
    assert lib.dlo_set_state(None, None, None, None) == 1
    assert lib.dlo_step(None, None, 1, 0, None) == 1
    assert lib.dlo_backward(None, None, None, None, None, None, None, None, None) == 1
    lib.dlo_destroy(None)
