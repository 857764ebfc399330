"""The C-ABI library builds, loads and exports every entry point that
include/cncpd.h declares; argument errors are reported without a GPU."""

import ctypes
import os
import re

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib(root):
    from paper_2302_05119_gb300 import build
    build.build()
    from paper_2302_05119_gb300 import _lib
    return _lib.lib()


def _declared(root):
    src = open(os.path.join(root, "include", "cncpd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cncpd_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib, root):
    names = _declared(root)
    assert "cncpd_create" in names and "cncpd_step" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header(root):
    from paper_2302_05119_gb300 import _lib
    assert set(_declared(root)) == set(_lib.SIGNATURES)


def test_struct_layouts():
    from paper_2302_05119_gb300 import _lib
    o = _lib.cncpd_opts()
    _lib.cncpd_default_opts(ctypes.byref(o))
    assert (o.eps, o.max_it, o.lra_eps, o.lra_max_it) == (1e-8, 1000, 1e-4, 200)
    assert o.delta_w == 0.9999 and o.reupdate == 1 and o.storage == -1 and o.use_core == 0
    assert ctypes.sizeof(_lib.cncpd_opts) == 8 + 8 + 8 + 8 + 8 + 4 * 6 + 4 * 6
    assert o.autotune == 1


def test_argument_errors_without_gpu(lib):
    import paper_2302_05119_gb300 as P
    X = np.ones((3, 4, 5))
    with pytest.raises(P.CncpdError, match="EINVAL"):
        P.CoupledNCP([X], 2, [3, 0, 0])          # L_n > min R (Section II-C)
    with pytest.raises(P.CncpdError, match="EINVAL"):
        P.CoupledNCP([X, np.ones((3, 5, 5))], 2, [0, 1, 0])   # coupled mode sizes differ
    with pytest.raises(P.CncpdError, match="EINVAL"):
        P.CoupledNCP([X], 65, [0, 0, 0])         # rank above 64
    with pytest.raises(P.CncpdError, match="EINVAL"):
        P.CoupledNCP([np.ones((3, 4))], 2, [0, 0])   # order 2


def test_null_handle_is_rejected(lib):
    from paper_2302_05119_gb300 import _lib
    s = _lib.cncpd_stats()
    assert _lib.cncpd_step(None, 1, ctypes.byref(s)) == -1
    assert b"null handle" in _lib.cncpd_last_error()
    _lib.cncpd_destroy(None)
