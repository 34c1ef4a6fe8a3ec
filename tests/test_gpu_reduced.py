"""GPU parity of the reduced (1+1) and (2+1)-dimensional scalar lattices (section "Scalar
dynamics in 1+1 and 2+1 dimensions") against the oracle: N^d sites, the Laplacian and the
gradient energy over the d directions, leapfrog compositions and 2N-RK stages.

Tolerances as for the 3-D lattices: 1e-10 relative L2 in FP64, 1e-4 in FP32 (+ Kahan).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cl():
    from paper_2607_24978_gb300 import build_ext, cl as clmod
    build_ext.build()
    clmod.lib()
    return clmod


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_pair(cl, dims, N, nf, prec, integ, scheme, nsteps, dt=0.01, seed=3, graph=1, variant=None, oracle=True):
    L = 0.8 * N
    pot = [0.6, 1.0, 0.3, 0.5 if nf == 2 else 0.0, 2.5 if nf == 2 else 0.0]
    if nf == 1:
        pot[2] = 0.0
    m = O.make_model(N, L, nf=nf, alpha=0.5, kappa=0.4, expansion=True, m2=(pot[0], pot[2]),
                     lam=(pot[1], pot[3]), g2=pot[4], dims=dims)
    st = O.new_state(m)
    rng = np.random.default_rng(seed)
    st.phi[:] = np.array([0.9, 0.1])[:nf, None, None, None] + 0.05 * rng.standard_normal(st.phi.shape)
    st.pi[:] = 0.05 * rng.standard_normal(st.pi.shape)
    st.abt[:] = (1.0, 0.0, 0.0)
    st.abt[1] = math.sqrt(0.4 * O.energies(m, st)["rho"] / 3.0)
    dtype = np.float64 if prec == 0 else np.float32
    with cl.Lattice(N, L, nf, prec, integ, expansion=True, alpha=0.5, kappa=0.4, dt=dt, dims=dims) as g:
        g.cl_set_potential(cl.CL_POT_POLY, pot)
        g.cl_set_option(cl.CL_OPT_GRAPH, graph)
        if variant is not None:
            g.cl_set_option(cl.CL_OPT_PASS_VARIANT, variant)
        for f in range(nf):
            g.cl_set_state(cl.CL_FIELD_PHI0 + f, st.phi[f].astype(dtype))
            g.cl_set_state(cl.CL_FIELD_PI0 + f, st.pi[f].astype(dtype))
        g.cl_set_scalars(st.abt[0], st.abt[1], 0.0)
        e0 = g.cl_energies()
        eo0 = O.energies(m, st)
        g.cl_step(nsteps)
        launches = g.cl_last_launch_count()
        gphi = np.stack([g.cl_get_state(cl.CL_FIELD_PHI0 + f) for f in range(nf)])
        gpi = np.stack([g.cl_get_state(cl.CL_FIELD_PI0 + f) for f in range(nf)])
        e = g.cl_energies()
    if not oracle:
        return gphi, gpi, e0, None, e, None, None, launches
    O.step(m, st, scheme, dt, nsteps)
    return gphi, gpi, e0, eo0, e, st, O.energies(m, st), launches


SCHEMES = [(0, O.VV2, 1), (1, O.YOSHIDA4, 3), (2, O.RK3_3, 3), (3, O.RK4_5, 5)]


@pytest.mark.parametrize("dims,N", [(1, 64), (2, 32)])
@pytest.mark.parametrize("integ,scheme,passes", SCHEMES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4)])
@pytest.mark.parametrize("nf", [1, 2])
def test_reduced_parity(cl, dims, N, integ, scheme, passes, prec, tol, nf):
    n = 12
    gphi, gpi, e0, eo0, e, st, eo, launches = run_pair(cl, dims, N, nf, prec, integ, scheme, n)
    assert gphi.shape[1:] == st.phi.shape[1:]
    assert rel_l2(gphi, st.phi) < tol
    assert rel_l2(gpi, st.pi) < tol
    assert e["a"] == pytest.approx(st.abt[0], rel=tol)
    assert e["adot"] == pytest.approx(st.abt[1], rel=max(tol, 1e-9))
    for k in ("rho", "p", "V"):
        assert e[k] == pytest.approx(eo[k], rel=max(tol, 1e-9)), k
        assert e0[k] == pytest.approx(eo0[k], rel=max(tol, 1e-9)), k
    assert e0["G0"] == pytest.approx(eo0["G0"], rel=max(tol, 1e-9))
    leapfrog = integ in (0, 1)
    assert launches == n * passes + (1 if leapfrog else 0)  # the leapfrog opens with one half-kick pass


def test_reduced_large_plane(cl):
    """A 512^2 (2+1) lattice: several grid-stride sweeps per block."""
    gphi, gpi, e0, eo0, e, st, eo, _ = run_pair(cl, 2, 512, 2, 0, cl.CL_INT_YOSHIDA4, O.YOSHIDA4, 3)
    assert rel_l2(gphi, st.phi) < 1e-10 and rel_l2(gpi, st.pi) < 1e-10
    assert e["rho"] == pytest.approx(eo["rho"], rel=1e-9)


def test_reduced_graph_equals_plain(cl):
    a = run_pair(cl, 2, 32, 2, 2, cl.CL_INT_YOSHIDA4, O.YOSHIDA4, 5, graph=1)
    b = run_pair(cl, 2, 32, 2, 2, cl.CL_INT_YOSHIDA4, O.YOSHIDA4, 5, graph=0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_reduced_lattice_refusals(cl):
    with cl.Lattice(16, 8.0, 1, 0, cl.CL_INT_RK4_5, dims=2) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [0.6, 1.0, 0.0, 0.0, 0.0])
        with pytest.raises(cl.CLError):
            g.cl_init_vacuum(1, 1e30, 1e-4, (1.0,))
        with pytest.raises(cl.CLError):
            g.cl_set_nonminimal(0.3)
        with pytest.raises(cl.CLError):
            g.cl_spectrum(cl.CL_FIELD_PHI0)
    with cl.Lattice(16, 8.0, 1, 0, cl.CL_INT_VV2, dims=1) as g:
        with pytest.raises(cl.CLError):
            g.cl_enable_gw()
        with pytest.raises(cl.CLError):
            g.cl_autotune()


@pytest.mark.parametrize("N", [128, 256])
@pytest.mark.parametrize("integ,scheme,passes", SCHEMES[:2])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4)])
@pytest.mark.parametrize("nf", [1, 2])
def test_plane_pass_parity(cl, N, integ, scheme, passes, prec, tol, nf):
    """The row-marching (2+1) pass (the library's choice where N is a multiple of 128 (FP32)
    or 64 (FP64); N = 128 is one strip of columns in FP32) against the oracle."""
    gphi, gpi, e0, eo0, e, st, eo, launches = run_pair(cl, 2, N, nf, prec, integ, scheme, 6)
    assert rel_l2(gphi, st.phi) < tol
    assert rel_l2(gpi, st.pi) < tol
    assert e["a"] == pytest.approx(st.abt[0], rel=tol)
    for k in ("rho", "p", "V", "G0", "K0"):
        assert e[k] == pytest.approx(eo[k], rel=max(tol, 1e-9)), k
    assert launches == 6 * passes + 1


@pytest.mark.parametrize("N,prec,tol", [(4096, 2, 2e-6), (1024, 0, 1e-13), (640, 2, 2e-6)])
def test_plane_pass_matches_the_site_kernel(cl, N, prec, tol):
    """Row marching (variant 1, chunks of 18 rows at 4096^2: a ragged last chunk) against one
    thread per site (variant 0) on the same state: the same compensated operations, so the
    fields agree to rounding of the contracted multiply-adds."""
    a = run_pair(cl, 2, N, 2, prec, cl.CL_INT_YOSHIDA4, O.YOSHIDA4, 2, variant=1, oracle=False)
    b = run_pair(cl, 2, N, 2, prec, cl.CL_INT_YOSHIDA4, O.YOSHIDA4, 2, variant=0, oracle=False)
    assert rel_l2(a[0], b[0]) < tol and rel_l2(a[1], b[1]) < tol
    assert a[4]["rho"] == pytest.approx(b[4]["rho"], rel=1e-9)
    with cl.Lattice(N, 0.8 * N, 2, prec, cl.CL_INT_YOSHIDA4, dims=2) as g:
        assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == 1
        g.cl_set_option(cl.CL_OPT_PASS_VARIANT, 0)
        assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == 0
