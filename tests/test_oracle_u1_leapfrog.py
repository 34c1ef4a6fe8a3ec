"""Pins of the oracle's axion-U(1) leapfrog (oracle/u1.c: orc_u1_leapfrog; section "ALP-gauge
interactions" with the kick at fixed positions implicit in the momenta, as in the generalized
Stoermer-Verlet method of Hairer, Lubich and Wanner, Geometric Numerical Integration VI.3).

  * with the gauge fields zero the coupling vanishes, the kick is explicit and the step is
    the scalar velocity-Verlet step of lattice.c, expansion included (an independent code
    path of the oracle);
  * without the coupling a small transverse wave follows the exact velocity-Verlet map of a
    harmonic oscillator at the lattice frequency: theta_n = A cos(n Theta) with
    cos Theta = 1 - (h w)^2 / 2, w = 2 sin(k dx/2)/dx (not the continuum phase w n h);
  * with the coupling and expansion the step converges at order 2 to a fine RK4-5 solution;
  * iterated to convergence the step is time-reversible (the implicit half-kick is the
    adjoint of the explicit one), and three evaluations are converged far below the
    scheme's own error;
  * without the coupling the lattice Gauss law holds to rounding; with it the violation
    is O(h^2);
  * without expansion the energy error is bounded and O(h^2).
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs


def coupled_model(N=4, expansion=True, alpha=0.5, alphaL=1.5):
    return O.make_model(N, 3.0, nf=1, alpha=alpha, kappa=0.8, expansion=expansion, gauge=1, alphaL=alphaL,
                        ws2=0.5, m2=(1.0, 0.0), lam=(0.4, 0.0))


def random_state(model, seed, th_amp=0.3, e_amp=0.3):
    st = O.new_state(model)
    g = inputs.rng(seed)
    st.phi[:] = 0.8 + 0.2 * g.standard_normal(st.phi.shape)
    st.pi[:] = 0.2 * g.standard_normal(st.pi.shape)
    st.links, st.efield = inputs.gauge_state(model.N, seed=seed + 1, theta_amp=th_amp, e_amp=e_amp)
    return st


def hubble_start(model, st):
    e = O.energies(model, st)
    st.abt[:] = [1.0, np.sqrt(model.kappa * e["rho"] / 3.0), 0.0]


def flat(st):
    return np.concatenate([st.phi.ravel(), st.pi.ravel(), st.links.ravel(), st.efield.ravel(), st.abt[:2]])


def test_without_gauge_fields_it_is_the_scalar_velocity_verlet():
    N = 6
    mg = O.make_model(N, 5.0, nf=1, alpha=0.5, kappa=0.4, expansion=True, gauge=1, alphaL=3.0, ws2=0.7,
                      m2=(1.0, 0.0), lam=(0.5, 0.0))
    ms = O.make_model(N, 5.0, nf=1, alpha=0.5, kappa=0.4, expansion=True, m2=(1.0, 0.0), lam=(0.5, 0.0))
    g = inputs.rng(21)
    sg = O.new_state(mg)
    sg.phi[:] = 1.0 + 0.1 * g.standard_normal(sg.phi.shape)
    sg.pi[:] = 0.1 * g.standard_normal(sg.pi.shape)
    hubble_start(mg, sg)
    ss = O.new_state(ms)
    ss.phi[:], ss.pi[:], ss.abt[:] = sg.phi, sg.pi, sg.abt
    O.step(mg, sg, O.VV2, 0.05, 40)
    O.step(ms, ss, O.VV2, 0.05, 40)
    assert sg.abt[0] > 1.05
    assert np.array_equal(sg.links, np.zeros_like(sg.links)) and np.array_equal(sg.efield, np.zeros_like(sg.efield))
    for a, b in ((sg.phi, ss.phi), (sg.pi, ss.pi), (sg.abt, ss.abt)):
        assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(b))


def test_free_wave_follows_the_velocity_verlet_map():
    N, L = 8, 8.0
    model = O.make_model(N, L, nf=1, alpha=0.0, kappa=1.0, gauge=1, alphaL=0.0, ws2=1.0)
    st = O.new_state(model)
    z = np.arange(N)[:, None, None] * np.ones((N, N, N))
    k, dx, amp = 2 * np.pi / L, L / N, 1e-6
    st.links[0] = amp * np.cos(k * z * dx)
    w = 2 * np.sin(k * dx / 2) / dx
    h, n = 0.05, 300
    O.step(model, st, O.VV2, h, n)
    theta = np.arccos(1.0 - 0.5 * (h * w) ** 2)
    expect = amp * np.cos(n * theta) * np.cos(k * z[:, 0, 0] * dx)
    assert np.max(np.abs(st.links[0, :, 0, 0] - expect)) < 1e-15
    # the continuum phase is measurably different at this step size
    assert abs(amp * np.cos(w * n * h) - expect[0]) > 1e-10
    assert np.max(np.abs(st.links[1:])) == 0.0


def test_coupled_step_is_second_order():
    model = coupled_model()
    base = random_state(model, 31)
    hubble_start(model, base)
    T = 0.8
    ref = base.copy()
    O.step(model, ref, O.RK4_5, 0.005, int(round(T / 0.005)))
    errs = []
    for h in (0.04, 0.02, 0.01):
        st = base.copy()
        O.step(model, st, O.VV2, h, int(round(T / h)))
        errs.append(np.max(np.abs(flat(st) - flat(ref))))
    assert errs[0] > 1e-6
    for e0, e1 in zip(errs, errs[1:]):
        assert np.log2(e0 / e1) == pytest.approx(2.0, abs=0.1)


def test_converged_step_is_time_reversible_and_three_evaluations_suffice():
    model = coupled_model()
    base = random_state(model, 41)
    hubble_start(model, base)
    h, n = 0.02, 25
    st = base.copy()
    O.u1_leapfrog(model, st, h, n, iters=40)
    fwd = st.copy()
    O.u1_leapfrog(model, st, -h, n, iters=40)
    assert np.max(np.abs(flat(st) - flat(base))) < 1e-12
    # three evaluations against the converged kick, and against the scheme's own error
    st3 = base.copy()
    O.u1_leapfrog(model, st3, h, n, iters=3)
    half = base.copy()
    O.u1_leapfrog(model, half, h / 2, 2 * n, iters=40)
    trunc = np.max(np.abs(flat(st3) - flat(fwd)))
    scheme = np.max(np.abs(flat(half) - flat(fwd)))
    assert trunc < 1e-3 * scheme
    # step(VV2) is the three-evaluation form
    st_s = base.copy()
    O.step(model, st_s, O.VV2, h, n)
    assert np.array_equal(flat(st_s), flat(st3))


def curl_field(N, dx, U):
    E = np.zeros_like(U)
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        E[i] = (U[k] - np.roll(U[k], 1, axis=2 - j)) / dx - (U[j] - np.roll(U[j], 1, axis=2 - k)) / dx
    return E


def test_gauss_law_exact_without_coupling_and_second_order_with_it():
    N, L = 6, 4.0
    m0 = O.make_model(N, L, nf=1, alpha=0.0, kappa=0.5, expansion=True, gauge=1, alphaL=0.0, ws2=0.4, m2=(1.0, 0.0))
    st = random_state(m0, 7, th_amp=0.4)
    st.efield = curl_field(N, L / N, 0.3 * inputs.rng(8).standard_normal((3, N, N, N)))
    st.abt[:] = [1.0, 0.3, 0.0]
    O.step(m0, st, O.VV2, 0.02, 40)
    assert st.abt[0] > 1.0
    assert np.max(np.abs(O.u1_gauss(m0, st))) < 1e-12 * np.max(np.abs(st.efield)) * N / L
    # with the coupling: a state that satisfies the Gauss law, then the violation after a
    # fixed time shrinks as h^2
    model = coupled_model(N=4)
    viol = []
    for h in (0.04, 0.02):
        s = random_state(model, 51, th_amp=0.3)
        s.efield = curl_field(4, 3.0 / 4, 0.3 * inputs.rng(52).standard_normal((3, 4, 4, 4)))
        # remove the g W part of the charge: start from E with div(a^(1-alpha) E + g W) = 0
        g0 = O.u1_gauss(model, s)
        assert np.max(np.abs(g0)) > 1e-3  # W contributes
        s.efield = s.efield - _gradient_solve(g0, 3.0 / 4)
        hubble_start(model, s)
        assert np.max(np.abs(O.u1_gauss(model, s))) < 1e-12
        O.step(model, s, O.VV2, h, int(round(0.8 / h)))
        viol.append(np.max(np.abs(O.u1_gauss(model, s))))
    assert viol[0] > 1e-8
    assert np.log2(viol[0] / viol[1]) == pytest.approx(2.0, abs=0.3)


def _gradient_solve(rho, dx):
    """E = grad+ chi with div- E = rho (periodic; rho has zero mean): chi from the lattice
    Poisson equation in Fourier space.  At a = 1 a^(1-alpha) = 1, so subtracting E removes rho."""
    N = rho.shape[0]
    s = np.fft.fftfreq(N) * 2 * np.pi
    kz, ky, kx = np.meshgrid(s, s, s, indexing="ij")
    lap = -(2 - 2 * np.cos(kx) + 2 - 2 * np.cos(ky) + 2 - 2 * np.cos(kz)) / dx ** 2
    rk = np.fft.fftn(rho)
    lap[0, 0, 0] = 1.0
    ck = rk / lap
    ck[0, 0, 0] = 0.0
    chi = np.real(np.fft.ifftn(ck))
    E = np.zeros((3,) + rho.shape)
    for d in range(3):
        E[d] = (np.roll(chi, -1, axis=2 - d) - chi) / dx
    return E


def test_energy_error_is_bounded_and_second_order():
    model = coupled_model(expansion=False, alpha=0.0)
    errs = []
    for h in (0.04, 0.02):
        st = random_state(model, 61, th_amp=0.2, e_amp=0.2)
        e0 = O.energies(model, st)["rho"]
        dev = []
        for _ in range(int(round(4.0 / h)) // 10):
            O.step(model, st, O.VV2, h, 10)
            dev.append(abs(O.energies(model, st)["rho"] / e0 - 1.0))
        errs.append(max(dev))
        half = len(dev) // 2
        assert max(dev[half:]) < 2.0 * max(dev[:half])  # no secular drift
    assert errs[0] > 1e-7
    assert np.log2(errs[0] / errs[1]) == pytest.approx(2.0, abs=0.3)
