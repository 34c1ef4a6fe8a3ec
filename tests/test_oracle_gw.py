"""Pins of the oracle's gravitational waves (section "New algorithm for GWs"): five traceless
auxiliaries v_ij (v33 = -v11 - v22) evolved with the leapfrog alongside the scalars, and the
energy spectrum of their TT projection.

* Without a source each v_ij is a free lattice wave: the exact discrete velocity-Verlet map.
* A scalar field that depends on x alone has a source diagonal in (x; y, z) with equal y and z
  entries; every mode it excites points along x, where the TT projector removes it: the GW
  spectrum stays zero.
* A pure TT plane wave (plus and cross polarisations along z) puts all its energy in one bin
  and the binned spectrum sums to rho_GW = <h'_ij h'_ij> / (4 kappa a^(2 alpha)) (Parseval);
  a trace / longitudinal configuration has none.
* The coupled scalar + GW system converges at second order under VV-2.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs


def _vv_matrix(h, w2):
    return np.array([[1 - 0.5 * h * h * w2, h], [-h * w2 * (1 - 0.25 * h * h * w2), 1 - 0.5 * h * h * w2]])


def _sum_spectrum(d, dn=1.0):
    l = np.arange(len(d))
    return float(np.sum(d[1:] * dn / (l[1:] * dn)))


def test_free_gw_auxiliary_is_a_lattice_wave():
    N, L, h, n = 8, 6.0, 0.05, 60
    dx = L / N
    m = O.make_model(N, L, nf=1, alpha=0.0, kappa=0.3)
    st = O.new_state(m)
    st.phi[:] = 0.7  # homogeneous, massless, no potential: no source
    s = np.array([1, 2, 1])
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    shape = np.cos(2 * np.pi / N * (s[0] * x + s[1] * y + s[2] * z))
    gv = np.zeros((5, N, N, N))
    gp = np.zeros((5, N, N, N))
    gv[1] = shape
    O.step_gw(m, st, gv, gp, O.VV2, h, n)
    w2 = np.sum(4.0 / dx ** 2 * np.sin(np.pi * s / N) ** 2)
    amp = np.linalg.matrix_power(_vv_matrix(h, w2), n) @ np.array([1.0, 0.0])
    np.testing.assert_allclose(gv[1], amp[0] * shape, atol=1e-12)
    np.testing.assert_allclose(gp[1], amp[1] * shape, atol=1e-12)
    assert np.abs(gv[[0, 2, 3, 4]]).max() == 0.0 and np.abs(gp[[0, 2, 3, 4]]).max() == 0.0


def test_planar_scalar_field_sources_no_tt_power():
    N, L = 8, 6.0
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    res = []
    for planar in (True, False):
        m = O.make_model(N, L, nf=1, alpha=1.0, kappa=0.5, expansion=True, m2=(0.5, 0.0), lam=(1.0, 0.0))
        st = O.new_state(m)
        f = 0.8 + 0.3 * np.sin(2 * np.pi * x / N) + (0.0 if planar else 0.2 * np.cos(2 * np.pi * (y + z) / N))
        st.phi[0] = f
        st.abt[1] = 0.2
        gv = np.zeros((5, N, N, N))
        gp = np.zeros((5, N, N, N))
        O.step_gw(m, st, gv, gp, O.VV2, 0.02, 30)
        _, d, _ = O.gw_spectrum(m, gp, st.abt)
        res.append(d)
        if planar:
            assert np.abs(gv).max() > 1e-6  # the diagonal auxiliaries are sourced
    assert res[1].max() > 0
    assert res[0].max() < 1e-22 * res[1].max()


@pytest.mark.parametrize("alpha,a", [(0.0, 1.0), (1.0, 1.7)])
def test_tt_plane_wave_parseval(alpha, a):
    N, L, kappa = 8, 6.0, 0.4
    m = O.make_model(N, L, nf=1, alpha=alpha, kappa=kappa)
    z = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")[0]
    c = np.cos(2 * np.pi * 2 * z / N)
    gp = np.zeros((5, N, N, N))
    gp[0], gp[3], gp[1] = 0.3 * c, -0.3 * c, 0.5 * c  # plus (11 = -22) and cross (12) along z
    abt = np.array([a, 0.0, 0.0])
    _, d, cnt = O.gw_spectrum(m, gp, abt)
    hp = a ** (alpha - 3) * np.stack([gp[0], gp[1], gp[2], gp[3], gp[4], -gp[0] - gp[3]])
    # sum over the six components of h'_ij h'_ij: off-diagonal ones twice
    hh = hp[0] ** 2 + hp[3] ** 2 + hp[5] ** 2 + 2 * (hp[1] ** 2 + hp[2] ** 2 + hp[4] ** 2)
    rho = float(np.mean(hh)) / (4 * kappa * a ** (2 * alpha))
    assert _sum_spectrum(d) == pytest.approx(rho, rel=1e-12)
    assert np.count_nonzero(d > 1e-14 * d.max()) == 1 and d[2] > 0


def test_trace_and_longitudinal_configurations_have_no_gw_energy():
    N, L = 8, 6.0
    m = O.make_model(N, L, nf=1, alpha=0.0, kappa=0.4)
    z = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")[0]
    c = np.cos(2 * np.pi * z / N)
    gp = np.zeros((5, N, N, N))
    gp[0], gp[3] = 0.3 * c, 0.3 * c  # h = c diag(1, 1, -2) with k along z
    _, d, _ = O.gw_spectrum(m, gp, np.array([1.0, 0.0, 0.0]))
    assert np.abs(d).max() < 1e-28
    gp = np.zeros((5, N, N, N))
    gp[2] = 0.4 * c  # h_13 with k along z: longitudinal
    _, d, _ = O.gw_spectrum(m, gp, np.array([1.0, 0.0, 0.0]))
    assert np.abs(d).max() < 1e-28


def test_coupled_system_converges_at_second_order():
    N, L, T = 4, 4.0, 0.6
    m = O.make_model(N, L, nf=2, alpha=1.0, kappa=0.6, expansion=True, m2=(0.5, 0.2), lam=(1.0, 0.0), g2=1.5)
    out = []
    for h in (0.04, 0.02, 0.01):
        phi, pi = inputs.scalar_state(N, 2, seed=12, fbar=(0.9, 0.1), amp=0.1, pamp=0.1)
        st = O.State(phi, pi, np.array([1.0, 0.3, 0.0]))
        gv = np.zeros((5, N, N, N))
        gp = np.zeros((5, N, N, N))
        O.step_gw(m, st, gv, gp, O.VV2, h, int(round(T / h)))
        out.append(np.concatenate([gv.ravel(), gp.ravel()]))
    e1, e2 = np.abs(out[0] - out[1]).max(), np.abs(out[1] - out[2]).max()
    assert math.log2(e1 / e2) == pytest.approx(2.0, abs=0.1)
