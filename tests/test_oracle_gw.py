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


# ---------------------------------------------------------------- source amplitude
def _cd(f, axis_xyz, dx):
    """Central difference (f(n + e) - f(n - e)) / (2 dx) along x, y or z of an array [z, y, x]."""
    ax = 2 - axis_xyz
    return (np.roll(f, -1, axis=ax) - np.roll(f, 1, axis=ax)) / (2.0 * dx)


def _lap(f, dx):
    return sum(np.roll(f, -1, axis=ax) + np.roll(f, 1, axis=ax) - 2.0 * f for ax in range(3)) / dx ** 2


@pytest.mark.parametrize("alpha,a,kappa", [(0.0, 1.0, 0.5), (0.5, 1.7, 0.37), (1.0, 0.6, 2.0)])
def test_gw_source_of_plane_waves_in_closed_form(alpha, a, kappa):
    """With v = v' = 0 the printed equation gives v'' = (2 / m_p^2) a^(-2(1-alpha)) [Pi_ij - delta_ij Pi / 3]
    (m_p^-2 -> kappa in program units), so pi_v' = a^(3-alpha) v'' at that instant.  For plane waves
    phi_0 = A sin(k1 x) + B sin(k2 y), phi_1 = C sin(k3 z) + D cos(k4 x) the central differences
    are closed forms (d/dx sin(k x) -> cos(k x) sin(k dx) / dx), so Pi_ij is written out by hand
    here.  A factor kappa instead of 2 kappa, a power a^alpha instead of a^(1+alpha), a dropped
    trace term or a swapped component fails this."""
    N, L = 8, 6.0
    dx = L / N
    m = O.make_model(N, L, nf=2, alpha=alpha, kappa=kappa)
    z, y, x = np.meshgrid(np.arange(N) * dx, np.arange(N) * dx, np.arange(N) * dx, indexing="ij")
    k = lambda n: 2 * np.pi * n / L
    A, B, Cc, D = 0.3, -0.7, 0.5, 0.9
    k1, k2, k3, k4 = k(1), k(2), k(3), k(1)
    phi = np.stack([A * np.sin(k1 * x) + B * np.sin(k2 * y), Cc * np.sin(k3 * z) + D * np.cos(k4 * x)])
    s = lambda kk: np.sin(kk * dx) / dx
    grads = [  # per field: (d_x, d_y, d_z) in closed form
        (A * s(k1) * np.cos(k1 * x), B * s(k2) * np.cos(k2 * y), np.zeros_like(x)),
        (-D * s(k4) * np.sin(k4 * x), np.zeros_like(x), Cc * s(k3) * np.cos(k3 * z)),
    ]
    Pi = np.zeros((3, 3) + x.shape)
    for g in grads:
        for i in range(3):
            for j in range(3):
                Pi[i, j] += g[i] * g[j]
    tr = Pi[0, 0] + Pi[1, 1] + Pi[2, 2]
    vpp = lambda i, j: 2.0 * kappa * a ** (-2.0 * (1.0 - alpha)) * (Pi[i, j] - (tr / 3.0 if i == j else 0.0))
    want = np.stack([a ** (3.0 - alpha) * vpp(i, j) for i, j in ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2))])
    got = O.gw_force(m, phi, np.zeros((5, N, N, N)), a)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    assert np.abs(want).max() > 0.1


def test_gw_trajectory_satisfies_the_printed_equation():
    """The oracle's leapfrog of (v, pi_v) and the scalars, with expansion, satisfies the paper's
    second-order equation
        v'' + (3 - alpha)(a'/a) v' - a^(-2(1-alpha)) Lap v = 2 kappa a^(-2(1-alpha)) [Pi_ij - delta_ij Pi / 3]
    up to the scheme's O(h^2): v'' from the second difference of the trajectory, v' = a^(alpha-3) pi_v
    at the integer time, Lap and the central-difference Pi_ij evaluated here with numpy.  The
    residual relative to the source term must be small and fall by ~4 when h halves; a wrong source
    factor leaves an O(1) residual."""
    N, L, alpha, kappa = 6, 5.0, 0.5, 0.8
    dx = L / N
    m = O.make_model(N, L, nf=1, alpha=alpha, kappa=kappa, expansion=True, m2=(0.7, 0.0), lam=(0.5, 0.0))
    res = []
    for h in (0.004, 0.002):
        phi, pi = inputs.scalar_state(N, 1, seed=40, fbar=(0.8,), amp=0.3, pamp=0.2)
        st = O.State(phi, pi, np.array([1.2, 0.25, 0.0]))
        g = inputs.rng(41)
        gv = 1e-3 * g.standard_normal((5, N, N, N))
        gp = 1e-3 * g.standard_normal((5, N, N, N))
        O.step_gw(m, st, gv, gp, O.VV2, h, int(round(0.05 / h)))  # leave the initial conditions behind
        traj = []
        for _ in range(3):
            traj.append((gv.copy(), gp.copy(), st.phi.copy(), st.abt.copy()))
            O.step_gw(m, st, gv, gp, O.VV2, h, 1)
        (v0, _, _, _), (v1, p1, f1, abt1), (v2, _, _, _) = traj
        a, b = abt1[0], abt1[1]
        vpp = (v2 - 2.0 * v1 + v0) / h ** 2
        vp = a ** (alpha - 3.0) * p1
        d = [_cd(f1[0], i, dx) for i in range(3)]
        tr = d[0] ** 2 + d[1] ** 2 + d[2] ** 2
        src, lhs = [], []
        for c, (i, j) in enumerate(((0, 0), (0, 1), (0, 2), (1, 1), (1, 2))):
            S = d[i] * d[j] - (tr / 3.0 if i == j else 0.0)
            src.append(2.0 * kappa * a ** (-2.0 * (1.0 - alpha)) * S)
            lhs.append(vpp[c] + (3.0 - alpha) * (b / a) * vp[c] - a ** (-2.0 * (1.0 - alpha)) * _lap(v1[c], dx))
        src, lhs = np.stack(src), np.stack(lhs)
        res.append(np.abs(lhs - src).max() / np.abs(src).max())
    assert res[1] < 1e-3
    assert math.log2(res[0] / res[1]) == pytest.approx(2.0, abs=0.3)
