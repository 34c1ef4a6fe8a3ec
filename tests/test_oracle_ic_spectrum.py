"""Pins of the oracle's vacuum initial conditions and binned spectra.

  * Parseval: sum_l Delta_l dlog k = <f^2> - fbar^2, the lattice form of
    <df^2> = int dlog k Delta(k) (Eq. SpectrumContinuum with Eq. discretePSaux);
  * a single plane wave lands in one bin with a closed-form amplitude;
  * Type I / Type II differ by exactly Upsilon = #/(4 pi n^2 dn) (Eq. UpsilonII);
  * the vacuum state has the mode variances of Eq. QuantumFlucts, the momentum
    variance omega^2 + H^2 and the cross-correlation -H of Eq. fpr_influct2
    (checked with numpy's FFT over an ensemble of seeds), and its Type-II
    spectrum equals k^3 P(k) / (2 pi^2);
  * the zero mode and |k| > k_cut are empty; a' satisfies Eq. Friedmann2.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs


@pytest.mark.parametrize("dn", [1.0, 0.5, 2.0])
def test_spectrum_parseval(dn):
    N, L = 8, 5.0
    f = 0.3 + inputs.rng(1).standard_normal((N, N, N))
    k, D, c = O.spectrum(N, L, f, dn, 1)
    nl = np.arange(len(D)) * dn
    total = np.sum(D[1:] * dn / nl[1:])
    assert total == pytest.approx(np.mean(f**2) - np.mean(f) ** 2, rel=1e-12)
    assert np.sum(c) == N**3
    np.testing.assert_allclose(k, 2 * np.pi / L * nl, rtol=1e-15)


def test_spectrum_plane_wave_single_bin():
    N, L, A = 8, 3.0, 0.7
    f = inputs.plane_wave(N, (1, 2, 2), amp=A, phase=0.4)  # |m| = 3
    k, D, c = O.spectrum(N, L, f, 1.0, 1)
    assert D[3] == pytest.approx(3.0 * A**2 / 2.0, rel=1e-12)
    assert np.sum(np.abs(np.delete(D, 3))) < 1e-12 * D[3]


def test_type_one_over_type_two_is_upsilon():
    N, L, dn = 8, 2.0, 1.0
    f = inputs.rng(2).standard_normal((N, N, N))
    k, D1, c = O.spectrum(N, L, f, dn, 1)
    _, D2, _ = O.spectrum(N, L, f, dn, 2)
    l = np.arange(1, len(D1))
    ok = c[1:] > 0
    ups = c[1:] / (4 * np.pi * (l * dn) ** 2 * dn)
    np.testing.assert_allclose(D1[1:][ok] / D2[1:][ok], ups[ok], rtol=1e-12)


def _vacuum_ensemble(model, nseeds, kcut, amp2, fbar, dfbar):
    sts = [O.vacuum(model, 1000 + s, kcut, amp2, fbar, dfbar) for s in range(nseeds)]
    return sts


def _mode_grid(N, L):
    n = np.fft.fftfreq(N, 1.0 / N)
    nz, ny, nx = np.meshgrid(n, n, n, indexing="ij")
    kmod = 2 * np.pi / L * np.sqrt(nx**2 + ny**2 + nz**2)
    selfconj = ((nx == 0) | (nx == -N // 2)) & ((ny == 0) | (ny == -N // 2)) & ((nz == 0) | (nz == -N // 2))
    return kmod, selfconj


def test_vacuum_mode_statistics():
    N, L = 16, 10.0
    dx = L / N
    model = O.make_model(N, L=L, nf=2, alpha=1.0, kappa=0.4, expansion=True, m2=(1.0, 0.0),
                         lam=(0.0, 0.0), g2=5.0)
    fbar, dfbar, amp2, kcut = (1.0, 0.0), (0.3, 0.0), 1e-4, 2 * np.pi / L * 6.5
    sts = _vacuum_ensemble(model, 6, kcut, amp2, fbar, dfbar)
    kmod, selfconj = _mode_grid(N, L)
    rho_h = 0.5 * 1.0 + 0.5 * 0.3**2
    H = np.sqrt(0.4 * rho_h / 3.0)
    inside = (kmod > 0) & (kmod <= kcut) & ~selfconj
    for f, m2eff in ((0, 1.0), (1, 5.0 * 1.0)):
        w = np.sqrt(kmod**2 + m2eff)
        var = (N / dx) ** 3 * amp2 / (2 * w)  # (N/dx)^3 P(k), a = 1
        F = np.array([np.fft.fftn(st.phi[f] - np.mean(st.phi[f])) for st in sts])
        P = np.array([np.fft.fftn(st.pi[f] - np.mean(st.pi[f])) for st in sts])
        r_ff = np.mean(np.abs(F) ** 2, axis=0)[inside] / var[inside]
        r_pp = np.mean(np.abs(P) ** 2, axis=0)[inside] / ((w**2 + H**2) * var)[inside]
        r_fp = np.mean(np.real(np.conj(F) * P), axis=0)[inside] / (-H * var[inside])
        nmodes = r_ff.size * len(sts)
        assert np.mean(r_ff) == pytest.approx(1.0, abs=4.0 / np.sqrt(nmodes))
        assert np.mean(r_pp) == pytest.approx(1.0, abs=4.0 / np.sqrt(nmodes))
        # cross term: E[Re(F* Pi)] = -H (N/dx)^3 P; its scatter is ~ omega/H times larger
        assert np.mean(r_fp) == pytest.approx(1.0, abs=4.0 * np.mean(w[inside]) / H / np.sqrt(nmodes))
        # empty outside the sphere and at the zero mode (the homogeneous value is separate)
        assert np.max(np.abs(F[:, (kmod > kcut)])) < 1e-9 * np.sqrt(var[inside].max())
        assert np.mean(sts[0].phi[f]) == pytest.approx(fbar[f], abs=1e-13)
        assert np.mean(sts[0].pi[f]) == pytest.approx(dfbar[f], abs=1e-13)  # a = 1
    # a' from Eq. Friedmann2 with the lattice energy
    for st in sts:
        assert O.energies(model, st)["hubble_violation"] < 1e-13


def test_vacuum_type_two_spectrum_is_k3P_over_2pi2():
    """Ensemble-averaged Type-II spectrum of the vacuum state against the continuum
    definition Delta(k) = k^3 P(k) / (2 pi^2) of Eq. SpectrumContinuum."""
    N, L = 16, 8.0
    model = O.make_model(N, L=L, nf=1, alpha=1.0, lam=(1.0, 0.0))
    amp2 = 1e-4
    sts = [O.vacuum(model, 7 + s, 1e9, amp2, (1.0,), (0.0,)) for s in range(8)]
    spec = np.array([O.spectrum(N, L, st.phi[0], 1.0, 2)[1] for st in sts])
    k, _, cnt = O.spectrum(N, L, sts[0].phi[0], 1.0, 2)
    m2 = 3.0  # V'' of phi^4/4 at phi = 1
    for l in range(2, 8):
        P = amp2 / (2 * np.sqrt(k[l] ** 2 + m2))
        expect = k[l] ** 3 * P / (2 * np.pi**2)
        stat = 1.0 / np.sqrt(cnt[l] / 2 * len(sts))  # independent modes: half of the shell
        assert np.mean(spec[:, l]) / expect == pytest.approx(1.0, abs=4 * stat + 0.06)


def test_vacuum_is_deterministic_in_seed_and_member():
    model = O.make_model(8, L=4.0, nf=1, alpha=1.0, lam=(1.0, 0.0))
    a = O.vacuum(model, 5, 1e9, 1e-4, (1.0,), (0.0,))
    b = O.vacuum(model, 5, 1e9, 1e-4, (1.0,), (0.0,))
    c = O.vacuum(model, 5, 1e9, 1e-4, (1.0,), (0.0,), member=1)
    assert np.array_equal(a.phi, b.phi)
    assert not np.allclose(a.phi, c.phi)
