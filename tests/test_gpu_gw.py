"""GPU parity of the gravitational-wave auxiliaries (section "New algorithm for GWs") and
their TT energy spectrum against the oracle: the five v_ij and their momenta after leapfrog
steps alongside the scalars (FP64 1e-10, FP32 1e-4 relative L2) and the binned
d rho_GW / d log k."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs

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


SCHEMES = {0: O.VV2, 1: O.YOSHIDA4}


@pytest.mark.parametrize("integ", [0, 1])
@pytest.mark.parametrize("prec,tol,nf,N", [(0, 1e-10, 2, 12), (2, 1e-4, 1, 16), (1, 1e-4, 2, 12), (0, 1e-10, 1, 10),
                                           (1, 1e-4, 2, 64), (2, 1e-4, 1, 64), (1, 1e-4, 2, 128)])
def test_gw_evolution_and_spectrum_parity(cl, integ, prec, tol, nf, N):
    """Sizes 10 to 128 (several tiles and z chunks at 64 and 128)."""
    L, dt, n = 0.8 * N, 0.02, (15 if N <= 16 else (4 if N <= 64 else 2))
    phi, pi = inputs.scalar_state(N, nf, seed=51, fbar=(0.9, 0.1), amp=0.1, pamp=0.1)
    m = O.make_model(N, L, nf=nf, alpha=1.0, kappa=0.6, expansion=True, m2=(0.5, 0.2), lam=(1.0, 0.0),
                     g2=1.5 if nf == 2 else 0.0)
    dtype = np.float64 if prec == 0 else np.float32
    rg = inputs.rng(52)
    gv = (1e-3 * rg.standard_normal((5, N, N, N))).astype(dtype).astype(np.float64)
    gp = (1e-3 * rg.standard_normal((5, N, N, N))).astype(dtype).astype(np.float64)
    st = O.State(phi.astype(dtype).astype(np.float64), pi.astype(dtype).astype(np.float64), np.array([1.0, 0.3, 0.0]))
    pot = [0.5, 1.0, 0.2, 0.0, 1.5] if nf == 2 else [0.5, 1.0, 0.0, 0.0, 0.0]
    with cl.Lattice(N, L, nf, prec, integ, expansion=True, alpha=1.0, kappa=0.6, dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_POLY, pot)
        for f in range(nf):
            g.cl_set_state(cl.CL_FIELD_PHI0 + f, st.phi[f].astype(dtype))
            g.cl_set_state(cl.CL_FIELD_PI0 + f, st.pi[f].astype(dtype))
        g.cl_set_scalars(1.0, 0.3, 0.0)
        g.cl_enable_gw()
        for c in range(5):
            g.cl_set_state(cl.CL_FIELD_GW_V11 + c, gv[c].astype(dtype))
            g.cl_set_state(cl.CL_FIELD_GW_P11 + c, gp[c].astype(dtype))
        g.cl_step(n)
        launches = g.cl_last_launch_count()
        v = np.stack([g.cl_get_state(cl.CL_FIELD_GW_V11 + c) for c in range(5)])
        p = np.stack([g.cl_get_state(cl.CL_FIELD_GW_P11 + c) for c in range(5)])
        phi0 = g.cl_get_state(cl.CL_FIELD_PHI0)
        spec = [g.cl_gw_spectrum(dn, t) for dn, t in ((1.0, 1), (0.5, 2))]
    gvo, gpo = gv.copy(), gp.copy()
    O.step_gw(m, st, gvo, gpo, SCHEMES[integ], dt, n)
    assert rel_l2(phi0, st.phi[0]) < tol
    assert rel_l2(v, gvo) < tol
    assert rel_l2(p, gpo) < tol
    passes = 1 if integ == 0 else 3
    assert launches == 2 * passes * n + 2  # GW + scalar pass per pass, and the opening pair
    for (dn, t), (k, d, c) in zip(((1.0, 1), (0.5, 2)), spec):
        ko, do, co = O.gw_spectrum(m, gpo, st.abt, dn, t)
        assert np.array_equal(c, co)
        np.testing.assert_allclose(k, ko, rtol=1e-14)
        np.testing.assert_allclose(d, do, rtol=max(2 * tol, 1e-9), atol=1e-12 * do.max())


def test_gw_needs_a_leapfrog_scalar_lattice(cl):
    with cl.Lattice(8, 6.0, 1, 0, cl.CL_INT_RK3_3) as g:
        with pytest.raises(cl.CLError):
            g.cl_enable_gw()
    with cl.Lattice(8, 6.0, 1, 0, cl.CL_INT_VV2) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
        with pytest.raises(cl.CLError):
            g.cl_gw_spectrum()  # not enabled
        with pytest.raises(cl.CLError):
            g.cl_get_state(cl.CL_FIELD_GW_V11)
