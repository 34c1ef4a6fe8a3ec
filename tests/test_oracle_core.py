"""Pins of the oracle's lattice operators, energies and random numbers.

Each check compares the oracle with something other than itself: a matrix
built a different way, a closed-form eigenvalue, a library FFT, published
known-answer vectors, or finite differences of the oracle's own Hamiltonian.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    """Philox-4x32-10 against the published known-answer vectors (Salmon et al., SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert O.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def _kron_laplacian(N, dx):
    """3-D periodic Laplacian as a Kronecker sum of 1-D circulant second differences.
    Index order (z, y, x) with x fastest, so the x operator is the last factor."""
    I = np.eye(N)
    L1 = -2.0 * np.eye(N) + np.roll(np.eye(N), 1, axis=1) + np.roll(np.eye(N), -1, axis=1)
    return (np.kron(np.kron(L1, I), I) + np.kron(np.kron(I, L1), I) + np.kron(np.kron(I, I), L1)) / dx**2


@pytest.mark.parametrize("N", [3, 4, 5])
def test_laplacian_explicit_matrix(N):
    dx = 0.37
    f = inputs.rng(N).standard_normal((N, N, N))
    ref = (_kron_laplacian(N, dx) @ f.ravel()).reshape(N, N, N)
    np.testing.assert_allclose(O.laplacian(N, dx, f), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_laplacian_plane_wave_eigenvalue():
    """Lap e^{i k.n dx} = -sum_i (4/dx^2) sin^2(k_i dx / 2) e^{i k.n dx} (the lattice dispersion)."""
    N, dx = 8, 0.5
    m = (1, 3, 2)
    f = inputs.plane_wave(N, m, phase=0.3)
    lam = -sum(4.0 / dx**2 * np.sin(np.pi * mi / N) ** 2 for mi in m)
    np.testing.assert_allclose(O.laplacian(N, dx, f), lam * f, atol=1e-12)


def test_summation_by_parts():
    """sum (grad+ f)^2 = - sum f Lap f dx^2: the forward-difference gradient energy and the
    7-point Laplacian are the same quadratic form."""
    N, dx = 6, 0.8
    f = inputs.rng(11).standard_normal((N, N, N))
    g2 = O.grad2_sum(N, f)
    assert g2 == pytest.approx(-np.sum(f * O.laplacian(N, dx, f)) * dx**2, rel=1e-13)


@pytest.mark.parametrize("N", [4, 6])
def test_dft_matches_library_fft(N):
    g = inputs.rng(3)
    re, im = g.standard_normal((N, N, N)), g.standard_normal((N, N, N))
    fwd = O.dft3(re, im, sign=-1)
    np.testing.assert_allclose(fwd, np.fft.fftn(re + 1j * im), atol=1e-11)
    inv = O.dft3(re, im, sign=+1)
    np.testing.assert_allclose(inv, np.fft.ifftn(re + 1j * im), atol=1e-13)


def _hamiltonian(model, phi, pi, a):
    """H = a^(3+alpha) N^3 rho, assembled from the oracle's volume-averaged energies."""
    st = O.State(phi, pi, np.array([a, 0.0, 0.0]))
    e = O.energies(model, st)
    return a ** (3.0 + model.alpha) * model.N**3 * e["rho"]


@pytest.mark.parametrize("nf", [1, 2])
def test_kick_and_drift_are_hamiltonian_derivatives(nf):
    """Brute force on 4^3: pi' = -dH/dphi(n) and phi' = dH/dpi(n) = a^(alpha-3) pi(n), by
    central finite differences of the oracle's own lattice energy.  Ties the energies of
    Eq. energy-contrib (all powers of a) to the kick of Eq. singletEOM."""
    N, a = 4, 1.7
    model = O.make_model(N, L=3.1, nf=nf, alpha=0.5, m2=(0.8, 1.3), lam=(1.1, 0.4), g2=2.5)
    phi, pi = inputs.scalar_state(N, nf, seed=5, fbar=(0.7, -0.4), amp=0.2, pamp=0.3)
    h = 1e-5
    rng = inputs.rng(9)
    for f in range(nf):
        kick = O.kick_force(model, phi, f, a)
        for _ in range(6):
            z, y, x = rng.integers(0, N, 3)
            pp, pm = phi.copy(), phi.copy()
            pp[f, z, y, x] += h
            pm[f, z, y, x] -= h
            dH = (_hamiltonian(model, pp, pi, a) - _hamiltonian(model, pm, pi, a)) / (2 * h)
            assert -dH == pytest.approx(kick[z, y, x], rel=1e-7, abs=1e-8)
            # H is quadratic in pi, so a large step is exact up to roundoff
            hp = 1e-2
            qp, qm = pi.copy(), pi.copy()
            qp[f, z, y, x] += hp
            qm[f, z, y, x] -= hp
            dHp = (_hamiltonian(model, phi, qp, a) - _hamiltonian(model, phi, qm, a)) / (2 * hp)
            assert dHp == pytest.approx(a ** (model.alpha - 3.0) * pi[f, z, y, x], rel=1e-7, abs=1e-9)


def test_energies_homogeneous_closed_form():
    """Homogeneous state: K = pi^2/(2 a^6), G = 0, V = V(phi); rho and p per Eq. rhoLocal."""
    N, a = 3, 1.3
    model = O.make_model(N, L=1.0, nf=2, alpha=1.0, m2=(1.0, 0.5), lam=(0.3, 0.0), g2=4.0)
    phi = np.stack([np.full((N, N, N), 0.9), np.full((N, N, N), 0.2)])
    pi = np.stack([np.full((N, N, N), 0.4), np.full((N, N, N), -0.1)])
    e = O.energies(model, O.State(phi, pi, np.array([a, 0.0, 0.0])))
    K = (0.4**2 + 0.1**2) / (2 * a**6)
    V = 0.5 * 0.9**2 + 0.25 * 0.3 * 0.9**4 + 0.5 * 0.5 * 0.2**2 + 0.5 * 4.0 * 0.9**2 * 0.2**2
    assert e["K0"] + e["K1"] == pytest.approx(K, rel=1e-14)
    assert e["G0"] == pytest.approx(0.0, abs=1e-30)
    assert e["V"] == pytest.approx(V, rel=1e-14)
    assert e["rho"] == pytest.approx(K + V, rel=1e-14)
    assert e["p"] == pytest.approx(K - V, rel=1e-14)
