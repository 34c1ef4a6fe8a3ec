"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/cl.h, and rejects bad arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cl():
    from paper_2607_24978_gb300 import build_ext, cl as clmod
    build_ext.build()
    clmod.lib()
    return clmod


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cl_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(cl):
    names = [n for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h") for n in _declared(h)]
    assert "cl_step" in names and "cl_init_lattice" in names
    for n in names:
        assert hasattr(cl.lib(), n), n
    assert sorted(set(names)) == sorted(set(names) & set(dir(cl.lib()) + names))


def test_binding_covers_the_header(cl):
    declared = set(_declared("cl.h"))
    assert declared == set(cl.EXPORTS)


def _params(cl, **kw):
    p = cl.cl_lattice_params()
    p.N, p.nfields, p.precision, p.integrator, p.gauge, p.expansion = 8, 1, 0, 0, 0, 1
    p.L, p.alpha, p.kappa, p.dt, p.a0 = 1.0, 1.0, 0.1, 0.01, 1.0
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("kw", [dict(N=1), dict(N=100000), dict(nfields=3), dict(precision=7), dict(integrator=9),
                                dict(L=0.0), dict(dt=-1.0), dict(a0=0.0), dict(dims=4), dict(dims=-1),
                                dict(gauge=5)])
def test_init_rejects_bad_params(cl, kw):
    h = C.c_void_p(123)
    s = cl.lib().cl_init_lattice(C.byref(h), C.byref(_params(cl, **kw)))
    assert s == cl.CL_EINVAL
    assert not h.value


@pytest.mark.parametrize("kw", [dict(dims=2, gauge=1, integrator=2), dict(dims=1, gauge=1, integrator=3)])
def test_reduced_lattices_refuse_gauge_fields(cl, kw):
    """The (1+1) / (2+1)-dimensional lattices carry scalar fields only."""
    h = C.c_void_p(123)
    s = cl.lib().cl_init_lattice(C.byref(h), C.byref(_params(cl, **kw)))
    assert s == cl.CL_EUNSUPPORTED
    assert not h.value


def test_null_arguments(cl):
    L = cl.lib()
    assert L.cl_init_lattice(None, None) == cl.CL_EINVAL
    assert L.cl_step(None, 1) == cl.CL_EINVAL
    assert L.cl_energies(None, None, 1) == cl.CL_EINVAL
    assert L.cl_sync(None) == cl.CL_EINVAL
    L.cl_free(None)
    assert L.cl_strerror(cl.CL_ENAN) == b"non-finite energy"
