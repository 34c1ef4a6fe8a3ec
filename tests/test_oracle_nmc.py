"""Pins of the oracle's non-minimally coupled scalar (section "Scalar fields non-minimally
coupled to gravity": Eq. eomNMC, Eq. cosmic_R, Eq. eomR, Eq. piadot), run with the 2N
Runge-Kutta schemes as that section prescribes.

* Conformal coupling xi = 1/6 with a massless quartic potential: (1 - 6 xi) = 0 and
  4 V - 6 xi phi V' = lambda phi^4 - lambda phi^4 = 0, so R = 0, a'' = 0 in conformal time
  (alpha = 1): a(eta) = a0 + a0' eta exactly, for any field configuration.
* xi = 0: the trace equation a''/a + (1 - alpha) H^2 = a^(2 alpha) kappa (rho - 3p) / 6 and the
  minimally coupled Eq. Friedmann1 agree on the constraint surface H^2 = a^(2 alpha) kappa rho/3,
  which both flows preserve; from such a state the two integrations differ only by
  truncation error, which falls at the scheme's order.
* The coupled system converges at the order of the Runge-Kutta scheme.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs


def _state(model, seed, fbar=0.9, amp=0.05):
    phi, pi = inputs.scalar_state(model.N, 1, seed=seed, fbar=(fbar,), amp=amp, pamp=amp)
    return O.State(phi.copy(), pi.copy(), np.array([1.0, 0.0, 0.0]))


def _on_constraint(model, st):
    st.abt[1] = st.abt[0] * math.sqrt(st.abt[0] ** (2 * model.alpha) * model.kappa * O.energies(model, st)["rho"] / 3.0)
    return st


@pytest.mark.parametrize("scheme", [O.RK3_3, O.RK4_5])
def test_conformal_coupling_with_quartic_potential_keeps_a_linear(scheme):
    N, L = 6, 5.0
    m = O.make_model(N, L, nf=1, alpha=1.0, kappa=0.8, expansion=True, lam=(1.0, 0.0), xi=1.0 / 6.0)
    st = _state(m, 3, fbar=1.2, amp=0.2)
    st.abt[1] = 0.3
    assert abs(O.nmc_ricci(m, st)) < 1e-14
    h, n = 0.02, 40
    O.step(m, st, scheme, h, n)
    assert st.abt[0] == pytest.approx(1.0 + 0.3 * h * n, rel=1e-13)
    assert st.abt[1] == pytest.approx(0.3, rel=1e-13)


@pytest.mark.parametrize("scheme,order", [(O.RK3_3, 3), (O.RK4_5, 4)])
def test_zero_coupling_reduces_to_the_minimal_scalar(scheme, order):
    N, L, T = 6, 5.0, 0.8
    diffs = []
    for h in (0.04, 0.02):
        mn = O.make_model(N, L, nf=1, alpha=0.0, kappa=0.5, expansion=True, m2=(0.6, 0.0), lam=(1.0, 0.0), xi=0.0)
        mm = O.make_model(N, L, nf=1, alpha=0.0, kappa=0.5, expansion=True, m2=(0.6, 0.0), lam=(1.0, 0.0))
        a = _on_constraint(mm, _state(mm, 4))
        b = a.copy()
        n = int(round(T / h))
        O.step(mn, a, scheme, h, n)
        O.step(mm, b, scheme, h, n)
        diffs.append(abs(a.abt[0] - b.abt[0]) + np.abs(a.phi - b.phi).max())
    assert diffs[1] < 1e-6
    assert math.log2(diffs[0] / diffs[1]) == pytest.approx(order, abs=0.5)


@pytest.mark.parametrize("scheme,order", [(O.RK3_3, 3), (O.RK4_5, 4)])
def test_coupled_system_converges_at_the_scheme_order(scheme, order):
    N, L, T = 4, 4.0, 0.8
    m = O.make_model(N, L, nf=1, alpha=1.0, kappa=0.7, expansion=True, m2=(0.5, 0.0), lam=(1.0, 0.0), xi=-0.4)
    res = []
    for h in (0.04, 0.02, 0.01):
        st = _state(m, 5, fbar=1.0, amp=0.1)
        st.abt[1] = 0.4
        O.step(m, st, scheme, h, int(round(T / h)))
        res.append(np.concatenate([st.phi.ravel(), st.pi.ravel(), st.abt[:2]]))
    e1, e2 = np.abs(res[0] - res[1]).max(), np.abs(res[1] - res[2]).max()
    assert math.log2(e1 / e2) == pytest.approx(order, abs=0.2)


def test_ricci_of_a_homogeneous_minimally_coupled_field_is_the_trace():
    """xi = 0, homogeneous field: R = kappa (rho - 3 p) = kappa (4 V - 2 K) (the trace of the
    energy-momentum tensor), with K = pi^2 / (2 a^6)."""
    m = O.make_model(4, 3.0, nf=1, alpha=0.0, kappa=0.9, m2=(0.7, 0.0), lam=(0.5, 0.0), xi=0.0)
    st = O.new_state(m, a=1.3)
    st.phi[:] = 0.8
    st.pi[:] = 0.6
    V = 0.5 * 0.7 * 0.8 ** 2 + 0.25 * 0.5 * 0.8 ** 4
    K = 0.6 ** 2 / (2 * 1.3 ** 6)
    assert O.nmc_ricci(m, st) == pytest.approx(0.9 * (4 * V - 2 * K), rel=1e-14)
