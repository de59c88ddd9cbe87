"""The C-ABI library builds, loads and exports every symbol include/qxd.h
declares; argument checks that need no GPU reject bad geometries."""
import ctypes
import os
import re

import pytest

from paper_1908_11673_gb300 import build, qxd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "qxd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qxd_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return qxd.load_library()


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(qxd.EXPORTS)


@pytest.mark.parametrize("L,cstar,theta", [
    ((4, 4, 4, 5), 0, (0, 0, 0, 0)),      # odd extent
    ((4, 4, 4, 0), 0, (0, 0, 0, 0)),      # empty
    ((4, 4, 4, 4), 4, (0, 0, 0, 0)),      # cstar out of range
    ((4, 4, 4, 4), 1, (3.14, 0.1, 0, 0)),  # spatial phase with C*
])
def test_create_rejects_bad_geometry(lib, L, cstar, theta):
    g = qxd.Geom()
    g.L[:] = L
    g.cstar = cstar
    g.theta[:] = theta
    h = ctypes.c_void_p()
    assert lib.qxd_create(ctypes.byref(g), 0, ctypes.byref(h)) == 1
    assert not h.value


def test_null_context_is_safe(lib):
    assert lib.qxd_volume(None) == 0
    assert lib.qxd_last_error(None) == b"NULL context"
    lib.qxd_destroy(None)


def declared_arities():
    """Number of parameters of every function prototype in include/qxd.h."""
    src = open(os.path.join(ROOT, "include", "qxd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(?:int|void|long long|const char\*)\s+\**(qxd_[A-Za-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src,
                         flags=re.S):
        params = " ".join(m.group(2).split())
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_arity_matches_header(lib):
    arity = declared_arities()
    assert set(arity) == set(qxd.EXPORTS)
    for name, n in arity.items():
        assert len(getattr(lib, name).argtypes) == n, name
