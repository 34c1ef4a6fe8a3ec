"""Pins of the oracle's time integrators and self-consistent expansion.

  * exact discrete dispersion of a free plane wave (velocity Verlet, Yoshida-4,
    RK3-3) -- pins Laplacian, kick, drift, ordering and the RK3-3 coefficients;
  * the cn-elliptic closed form of homogeneous lambda phi^4 oscillation -- pins
    the nonlinear kick and the convergence order of every integrator;
  * bounded O(dt^2) energy error without expansion;
  * time reversibility with self-consistent expansion;
  * radiation-era a ~ t^(1/2) and matter-era a ~ t^(2/3) -- pins Eq. Friedmann1's
    (2 alpha - 1) rho - 3 p bracket;
  * O(dt^2) convergence of the Eq. Friedmann2 violation -- pins the Friedmann1
    prefactor against the energies of Eq. rhoLocal.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.special

from oracle import oracle as O
from tests import inputs


def _free_wave(N=8, L=4.0, m2=0.7, mode=(1, 2, 3)):
    model = O.make_model(N, L=L, nf=1, alpha=1.0, m2=(m2, 0.0))
    st = O.new_state(model)
    st.phi[0] = inputs.plane_wave(N, mode, amp=1.0, phase=0.2)
    dx = L / N
    w2 = m2 + sum(4.0 / dx**2 * np.sin(np.pi * mi / N) ** 2 for mi in mode)
    return model, st, w2


def _vv_matrix(h, w2):
    """Velocity-Verlet transfer matrix of one oscillator mode: (phi, pi) -> (phi, pi)."""
    c = 1.0 - 0.5 * h * h * w2
    return np.array([[c, h], [-h * w2 * (1.0 - 0.25 * h * h * w2), c]])


def test_vv_exact_discrete_dispersion():
    model, st, w2 = _free_wave()
    h, n = 0.05, 120
    shape = st.phi[0].copy()
    O.step(model, st, O.VV2, h, n)
    amp = np.linalg.matrix_power(_vv_matrix(h, w2), n) @ np.array([1.0, 0.0])
    np.testing.assert_allclose(st.phi[0], amp[0] * shape, atol=1e-12)
    np.testing.assert_allclose(st.pi[0], amp[1] * shape, atol=1e-12)
    # the same amplitude through the phase of the discrete map: cos(theta) = 1 - h^2 w^2 / 2
    theta = np.arccos(1.0 - 0.5 * h * h * w2)
    assert amp[0] == pytest.approx(np.cos(n * theta), abs=1e-12)


def test_yoshida4_exact_composition():
    model, st, w2 = _free_wave()
    h, n = 0.05, 40
    c = 2.0 ** (1.0 / 3.0)
    w1, w0 = 1.0 / (2.0 - c), -c / (2.0 - c)
    shape = st.phi[0].copy()
    O.step(model, st, O.YOSHIDA4, h, n)
    M = _vv_matrix(w1 * h, w2) @ _vv_matrix(w0 * h, w2) @ _vv_matrix(w1 * h, w2)
    amp = np.linalg.matrix_power(M, n) @ np.array([1.0, 0.0])
    np.testing.assert_allclose(st.phi[0], amp[0] * shape, atol=1e-12)
    np.testing.assert_allclose(st.pi[0], amp[1] * shape, atol=1e-12)


def test_rk33_stability_polynomial():
    """Any 3-stage third-order explicit RK maps y' = A y by R(hA) = I + hA + (hA)^2/2 + (hA)^3/6."""
    model, st, w2 = _free_wave()
    h, n = 0.05, 30
    shape = st.phi[0].copy()
    O.step(model, st, O.RK3_3, h, n)
    Z = h * np.array([[0.0, 1.0], [-w2, 0.0]])
    R = np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6
    amp = np.linalg.matrix_power(R, n) @ np.array([1.0, 0.0])
    np.testing.assert_allclose(st.phi[0], amp[0] * shape, atol=1e-12)
    np.testing.assert_allclose(st.pi[0], amp[1] * shape, atol=1e-12)


def test_rk34_stability_polynomial():
    """RK3-4 is built so that its stability function is the degree-4 Taylor polynomial of e^z:
    on y' = A y one step is I + hA + (hA)^2/2 + (hA)^3/6 + (hA)^4/24 (third order, with the z^4
    coefficient b A^3 1 = 1/24 fixed as the scheme's last condition)."""
    model, st, w2 = _free_wave()
    h, n = 0.05, 30
    shape = st.phi[0].copy()
    O.step(model, st, O.RK3_4, h, n)
    Z = h * np.array([[0.0, 1.0], [-w2, 0.0]])
    R = np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    amp = np.linalg.matrix_power(R, n) @ np.array([1.0, 0.0])
    np.testing.assert_allclose(st.phi[0], amp[0] * shape, atol=1e-12)
    np.testing.assert_allclose(st.pi[0], amp[1] * shape, atol=1e-12)


def _butcher_2n(A, B):
    """Butcher matrix and weights of a 2N-storage scheme k <- A_s k + h F, y <- y + B_s k."""
    s = len(B)
    a = np.zeros((s + 1, s))
    for i in range(1, s + 1):
        for j in range(1, i + 1):
            a[i, j - 1] = sum(B[m - 1] * np.prod([A[q - 1] for q in range(j + 1, m + 1)]) for m in range(j, i + 1))
    return a[:s], a[s]


def test_rk34_embedded_estimate_is_second_order():
    """The state after RK3-4's third stage is a second-order solution at t + h, so the estimate
    |y_4 - y_3| of a step falls as h^3 (homogeneous lambda phi^4, against cn)."""
    model = O.make_model(2, L=1.0, nf=1, alpha=1.0, lam=(1.0, 0.0))
    eps = []
    for h in (0.04, 0.02, 0.01):
        st = O.new_state(model)
        st.phi[:] = 1.0
        st.pi[:] = 0.3
        _, hu, ep = O.step_adaptive(model, st, h, 1e-6, 1, hmin=h, hmax=h)  # one step of fixed size
        assert hu[0] == h
        eps.append(ep[0])
    assert np.log2(eps[0] / eps[1]) == pytest.approx(3.0, abs=0.1)
    assert np.log2(eps[1] / eps[2]) == pytest.approx(3.0, abs=0.1)


def test_rk34_adaptive_controller():
    """The adaptive driver takes every step and sets the next one from its estimate,
    h <- h min(2, max(1/5, 0.9 (tol/eps)^(1/3))) within [hmin, hmax]: the estimates settle near
    tol, a tighter tolerance takes smaller steps (h ~ tol^(1/3)), and the end state converges
    to the cn-elliptic solution as tol falls."""
    model = O.make_model(2, L=1.0, nf=1, alpha=1.0, lam=(1.0, 0.0))
    res = {}
    for tol in (1e-6, 1e-8):
        st = O.new_state(model)
        st.phi[:] = 1.0
        h, hu, ep = O.step_adaptive(model, st, 0.01, tol, 200)
        for i in range(199):
            f = min(2.0, max(0.2, 0.9 * (tol / ep[i]) ** (1.0 / 3.0)))
            assert hu[i + 1] == pytest.approx(hu[i] * f, rel=1e-14)
        assert np.all(ep[20:] < 10 * tol) and 0.2 * tol < np.median(ep[20:]) < 2 * tol
        T = st.abt[2]
        sn, cn, dn, ph = scipy.special.ellipj(T, 0.5)
        res[tol] = (hu[2], abs(st.phi.flat[0] - cn))
    # from the same state near t = 0 the estimate is C h^3, so h settles at 0.9 (tol / C)^(1/3)
    assert res[1e-6][0] / res[1e-8][0] == pytest.approx(100.0 ** (1.0 / 3.0), rel=0.02)
    assert res[1e-8][1] < res[1e-6][1]


def test_rk34_coefficients_satisfy_their_conditions():
    """The 2N table meets the conditions that define it: third order, c_4 = 1 with
    sum_j a_4j c_j = 1/2 (the embedded second-order state), and b A^3 1 = 1/24."""
    A = [0.0, -0.7825460361923582986318837, -2.042914325731224687686953, -1.799337253940777102361562]
    B = [0.06688758201974096587947945, 2.876554598956718963241208, 0.553465736134398241034173,
         0.3912730180961791493159418]
    a, b = _butcher_2n(A, B)
    c = a.sum(1)
    for got, want in [(b.sum(), 1.0), (b @ c, 0.5), (b @ c ** 2, 1 / 3), (b @ a @ c, 1 / 6), (c[3], 1.0),
                      (a[3] @ c, 0.5), (b @ a @ a @ c, 1 / 24)]:
        assert got == pytest.approx(want, abs=1e-14)
    # the oracle steps with exactly this table: one step of y' = lambda y against the Butcher form
    model, st, w2 = _free_wave()
    h = 0.07
    shape = st.phi[0].copy()
    O.step(model, st, O.RK3_4, h, 1)
    Z = h * np.array([[0.0, 1.0], [-w2, 0.0]])
    K = np.zeros((4, 2))
    y0 = np.array([1.0, 0.0])
    for i in range(4):
        K[i] = Z @ (y0 + sum(a[i, j] * K[j] for j in range(i)))
    y1 = y0 + b @ K
    np.testing.assert_allclose(st.phi[0], y1[0] * shape, atol=1e-13)
    np.testing.assert_allclose(st.pi[0], y1[1] * shape, atol=1e-13)


def test_rk45_one_step_order():
    """RK4-5 one-step error against the exact matrix exponential scales as h^5."""
    model, st0, w2 = _free_wave()
    A = np.array([[0.0, 1.0], [-w2, 0.0]])
    errs = []
    for h in (0.08, 0.04):
        st = st0.copy()
        O.step(model, st, O.RK4_5, h, 1)
        ex = scipy.linalg.expm(h * A) @ np.array([1.0, 0.0])
        idx = np.unravel_index(np.argmax(np.abs(st0.phi[0])), st0.phi[0].shape)
        s = st0.phi[0][idx]
        errs.append(abs(st.phi[0][idx] / s - ex[0]) + abs(st.pi[0][idx] / s - ex[1]))
    assert np.log2(errs[0] / errs[1]) == pytest.approx(5.0, abs=0.15)


def _cn_error(scheme, h, T=2.0):
    """|phi(T) - cn(T; 1/2)| for homogeneous phi'' = -phi^3, phi(0) = 1, phi'(0) = 0."""
    model = O.make_model(2, L=1.0, nf=1, alpha=1.0, lam=(1.0, 0.0))
    st = O.new_state(model)
    st.phi[:] = 1.0
    n = int(round(T / h))
    O.step(model, st, scheme, h, n)
    sn, cn, dn, ph = scipy.special.ellipj(n * h, 0.5)
    assert np.ptp(st.phi) == 0.0  # stays homogeneous
    return abs(st.phi.flat[0] - cn)


@pytest.mark.parametrize("scheme,order,h,tol", [(O.VV2, 2, 0.02, 0.05), (O.YOSHIDA4, 4, 0.1, 0.1),
                                                (O.RK3_3, 3, 0.05, 0.1), (O.RK4_5, 4, 0.025, 0.1),
                                                (O.RK3_4, 3, 0.05, 0.1),
                                                (O.YOSHIDA6, 6, 0.1, 0.1), (O.YOSHIDA8, 8, 0.0625, 0.1),
                                                (O.YOSHIDA10, 10, 0.1, 0.2)])
def test_cn_elliptic_convergence_order(scheme, order, h, tol):
    """The higher Yoshida compositions are pinned by their order alone: a wrong weight, sign or
    recursion depth leaves a lower-order error term.  h is chosen so that the errors stay well
    above rounding (orders 8 and 10 reach 1e-12 quickly).  Bounds: order 2.00 +- 0.05 for velocity
    Verlet and +- 0.1 for the others; order 10 keeps +- 0.2, its finer error meets rounding."""
    e1, e2 = _cn_error(scheme, h), _cn_error(scheme, h / 2)
    assert e1 < 1e-2
    assert np.log2(e1 / e2) == pytest.approx(order, abs=tol)


def test_energy_bounded_and_second_order():
    """No expansion: total lattice energy oscillates with amplitude ~ dt^2 and no drift."""
    N = 4
    model = O.make_model(N, L=6.0, nf=2, alpha=1.0, m2=(0.5, 0.2), lam=(1.0, 0.0), g2=3.0)
    phi, pi = inputs.scalar_state(N, 2, seed=1, fbar=(1.0, 0.1), amp=0.05, pamp=0.05)
    devs = []
    for h in (0.04, 0.02):
        st = O.State(phi.copy(), pi.copy(), np.array([1.0, 0.0, 0.0]))
        rho0 = O.energies(model, st)["rho"]
        n = int(round(40.0 / h))
        d = []
        for _ in range(8):
            O.step(model, st, O.VV2, h, n // 8)
            d.append(abs(O.energies(model, st)["rho"] / rho0 - 1.0))
        devs.append(d)
    # second order: halving dt divides the energy error by ~4
    assert max(devs[0]) / max(devs[1]) == pytest.approx(4.0, rel=0.15)
    # no secular drift: the late error is not larger than the early error envelope
    assert max(devs[1][4:]) < 2.0 * max(devs[1][:4]) + 1e-12


@pytest.mark.parametrize("scheme", [O.VV2, O.YOSHIDA4, O.YOSHIDA6])
def test_time_reversibility_with_expansion(scheme):
    N = 4
    model = O.make_model(N, L=5.0, nf=2, alpha=1.0, kappa=0.5, expansion=True, m2=(0.0, 0.0),
                         lam=(1.0, 0.0), g2=2.0)
    phi, pi = inputs.scalar_state(N, 2, seed=2, fbar=(1.0, 0.05), amp=0.05, pamp=0.05)
    st = O.State(phi.copy(), pi.copy(), np.array([1.0, 0.4, 0.0]))
    ref = st.copy()
    O.step(model, st, scheme, 0.02, 60)
    assert st.abt[0] > 1.2  # the universe did expand
    st.pi *= -1.0
    st.abt[1] *= -1.0
    O.step(model, st, scheme, 0.02, 60)
    st.pi *= -1.0
    st.abt[1] *= -1.0
    np.testing.assert_allclose(st.phi, ref.phi, atol=1e-12)
    np.testing.assert_allclose(st.pi, ref.pi, atol=1e-12)
    assert st.abt[0] == pytest.approx(ref.abt[0], abs=1e-12)
    assert st.abt[1] == pytest.approx(ref.abt[1], abs=1e-12)


def _era_slope(model, phi0, h, n_chunks, chunk):
    """Run a homogeneous field, return the late-time slope d ln a / d ln t (t cosmic)."""
    st = O.new_state(model)
    st.phi[:] = phi0
    e = O.energies(model, st)
    st.abt[1] = st.abt[0] * np.sqrt(st.abt[0] ** (2 * model.alpha) * model.kappa * e["rho"] / 3.0)
    t_cos = 0.0
    ts, as_ = [], []
    for _ in range(n_chunks):
        for _ in range(chunk):
            a_old = st.abt[0]
            O.step(model, st, O.VV2, h, 1)
            t_cos += 0.5 * h * (a_old ** model.alpha + st.abt[0] ** model.alpha)  # dt = a^alpha d eta
        ts.append(t_cos)
        as_.append(st.abt[0])
    ts, as_ = np.log(np.array(ts)), np.log(np.array(as_))
    k = len(ts) // 2
    return np.polyfit(ts[k:], as_[k:], 1)[0]


def test_radiation_era_lambda_phi4():
    """Homogeneous lambda phi^4 averages to w = 1/3, hence a ~ t^(1/2) (Eq. Friedmann1, alpha = 1)."""
    model = O.make_model(2, L=1.0, nf=1, alpha=1.0, kappa=1.0, expansion=True, lam=(1.0, 0.0))
    slope = _era_slope(model, 1.0, 0.05, 200, 100)
    assert slope == pytest.approx(0.5, abs=0.01)


def test_matter_era_m2phi2():
    """Homogeneous m^2 phi^2 averages to w = 0, hence a ~ t^(2/3) (Eq. Friedmann1, alpha = 0)."""
    model = O.make_model(2, L=1.0, nf=1, alpha=0.0, kappa=1.0, expansion=True, m2=(1.0, 0.0))
    slope = _era_slope(model, 1.0, 0.05, 200, 100)
    assert slope == pytest.approx(2.0 / 3.0, abs=0.01)


@pytest.mark.parametrize("scheme,order", [(O.VV2, 2), (O.RK3_3, 3)])
def test_hubble_constraint_converges(scheme, order):
    """Starting on the Eq. Friedmann2 surface, evolving with Eq. Friedmann1 keeps the violation
    at O(dt^p): only the right prefactor of a'' is consistent with the energies."""
    N = 4
    model = O.make_model(N, L=5.0, nf=2, alpha=0.5, kappa=0.8, expansion=True, m2=(1.0, 0.3),
                         lam=(0.5, 0.0), g2=2.0)
    phi, pi = inputs.scalar_state(N, 2, seed=4, fbar=(1.0, 0.1), amp=0.1, pamp=0.1)
    viol = []
    for h in (0.02, 0.01):
        st = O.State(phi.copy(), pi.copy(), np.array([1.0, 0.0, 0.0]))
        e = O.energies(model, st)
        st.abt[1] = np.sqrt(model.kappa * e["rho"] / 3.0)  # a = 1
        O.step(model, st, scheme, h, int(round(3.0 / h)))
        viol.append(O.energies(model, st)["hubble_violation"])
    assert st.abt[0] > 1.5
    assert viol[0] < 1e-3
    assert np.log2(viol[0] / viol[1]) == pytest.approx(order, abs=0.25)
