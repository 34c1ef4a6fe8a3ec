"""Pins of the oracle's axion-U(1) sector (section "ALP-gauge interactions").

  * the energy a^(3+alpha) N^3 rho (field, electric and magnetic parts) is constant
    along the flow without expansion: the force terms, the Chern-Simons coupling (which
    must do no net work) and the energies agree;
  * the lattice Gauss charge is constant along the flow, with the coupling and with
    expansion: gauge invariance of the discretisation;
  * with the coupling off, a divergence-free electric field stays divergence-free
    under Runge-Kutta to machine precision;
  * free transverse waves oscillate at the lattice frequency 2 sin(k dx/2)/dx;
  * chiral instability: with phi' = v fixed, a transverse wave of the unstable helicity
    grows at Gamma^2 = g v sin(k dx)/dx - (2 sin(k dx/2)/dx)^2, the lattice form of
    Gamma^2 = g v k - k^2 of Eq. AxionInfEOM;
  * the Friedmann2 violation with electromagnetic energy converges at the scheme's order.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs


def random_state(model, seed, th_amp=0.3, e_amp=0.3):
    st = O.new_state(model)
    g = inputs.rng(seed)
    st.phi[:] = 0.8 + 0.2 * g.standard_normal(st.phi.shape)
    st.pi[:] = 0.2 * g.standard_normal(st.pi.shape)
    st.links, st.efield = inputs.gauge_state(model.N, seed=seed + 1, theta_amp=th_amp, e_amp=e_amp)
    return st


def advance(st, F, eps):
    s = st.copy()
    s.phi = st.phi + eps * F[0]
    s.pi = st.pi + eps * F[1]
    s.links = st.links + eps * F[2]
    s.efield = st.efield + eps * F[3]
    return s


def hamiltonian(model, st):
    e = O.energies(model, st)
    a = st.abt[0]
    return a ** (3.0 + model.alpha) * model.N ** 3 * e["rho"], a ** (3.0 + model.alpha) * model.N ** 3 * (e["KEM"] + e["GEM"])


@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_energy_is_constant_along_the_flow(alpha):
    model = O.make_model(4, 3.0, nf=1, alpha=alpha, kappa=0.7, gauge=1, alphaL=2.0, ws2=0.6, m2=(0.8, 0.0),
                         lam=(0.3, 0.0))
    st = random_state(model, 3)
    st.abt[0] = 1.3  # fixed scale factor (no expansion)
    F = O.u1_rhs(model, st)
    eps = 1e-4  # central differences: truncation O(eps^2), roundoff ~ 1e-16 H / eps
    Hp, EMp = hamiltonian(model, advance(st, F, eps))
    Hm, EMm = hamiltonian(model, advance(st, F, -eps))
    dH, dEM = (Hp - Hm) / (2 * eps), (EMp - EMm) / (2 * eps)
    assert abs(dEM) > 1e-2          # energy does flow between the sectors
    assert abs(dH) < 1e-6 * abs(dEM)


@pytest.mark.parametrize("expansion", [False, True])
def test_gauss_charge_is_constant_along_the_flow(expansion):
    model = O.make_model(4, 3.0, nf=1, alpha=0.5, kappa=0.7, expansion=expansion, gauge=1, alphaL=2.0, ws2=0.6,
                         m2=(0.8, 0.0))
    st = random_state(model, 5)
    st.abt[:] = [1.2, 0.4, 0.0]
    F = O.u1_rhs(model, st)
    eps = 1e-4
    Fa = (0.0, st.abt[1]) if expansion else (0.0, 0.0)
    sp, sm = advance(st, F, eps), advance(st, F, -eps)
    sp.abt[0] += eps * Fa[1]
    sm.abt[0] -= eps * Fa[1]
    dG = (O.u1_gauss(model, sp) - O.u1_gauss(model, sm)) / (2 * eps)
    # scale: the rate of the electric divergence alone
    m0 = O.make_model(4, 3.0, nf=1, alpha=0.5, kappa=0.7, gauge=1, alphaL=0.0, ws2=0.6)
    dE_div = (O.u1_gauss(m0, sp) - O.u1_gauss(m0, sm)) / (2 * eps)
    assert np.max(np.abs(dE_div)) > 1e-2
    assert np.max(np.abs(dG)) < 1e-6 * np.max(np.abs(dE_div))


def curl_field(N, dx, U):
    """E_i(n) = sum_jk eps_ijk (U_k(n) - U_k(n - j)) / dx, the backward curl (the form of the
    magnetic force): its backward divergence vanishes identically."""
    E = np.zeros_like(U)
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        # arrays are [z, y, x]: direction d -> numpy axis 2 - d; roll(+1) gives f(n - d)
        E[i] = (U[k] - np.roll(U[k], 1, axis=2 - j)) / dx - (U[j] - np.roll(U[j], 1, axis=2 - k)) / dx
    return E


def test_gauss_exact_without_coupling():
    N, L = 6, 4.0
    model = O.make_model(N, L, nf=1, alpha=0.0, kappa=0.5, expansion=True, gauge=1, alphaL=0.0, ws2=0.4,
                         m2=(1.0, 0.0))
    st = random_state(model, 7, th_amp=0.4)
    st.efield = curl_field(N, L / N, 0.3 * inputs.rng(8).standard_normal((3, N, N, N)))
    st.abt[:] = [1.0, 0.3, 0.0]
    assert np.max(np.abs(O.u1_gauss(model, st))) < 1e-13
    O.step(model, st, O.RK4_5, 0.02, 20)
    assert st.abt[0] > 1.0
    assert np.max(np.abs(O.u1_gauss(model, st))) < 1e-12 * np.max(np.abs(st.efield)) * N / L


def _z_wave(N, L, th_amp):
    st_links = np.zeros((3, N, N, N))
    z = np.arange(N)[:, None, None] * np.ones((N, N, N))
    k = 2 * np.pi / L
    dx = L / N
    st_links[0] = th_amp * np.cos(k * z * dx)  # theta_x(z), linear polarisation
    return st_links, k, dx


def _mode_amplitude(links, N, L):
    """Amplitude of the k = 2 pi / L mode along z of theta_x and theta_y."""
    z = np.arange(N) * L / N
    k = 2 * np.pi / L
    out = 0.0
    for c in (0, 1):
        prof = links[c, :, 0, 0]
        out += abs(np.sum(prof * np.exp(-1j * k * z))) ** 2
    return np.sqrt(out) * 2 / N


def test_free_wave_lattice_frequency():
    N, L = 8, 8.0
    model = O.make_model(N, L, nf=1, alpha=0.0, kappa=1.0, gauge=1, alphaL=0.0, ws2=1.0)
    st = O.new_state(model)
    st.links, k, dx = _z_wave(N, L, 1e-6)
    w = 2 * np.sin(k * dx / 2) / dx
    h, n = 0.02, 300
    O.step(model, st, O.RK4_5, h, n)
    # theta_x(t) = A cos(w t): compare the phase at t = n h
    expect = 1e-6 * np.cos(w * n * h)
    assert st.links[0, 0, 0, 0] == pytest.approx(expect, abs=1e-12)


@pytest.mark.parametrize("kappa", [1.0, 0.3])
def test_chiral_instability_growth_rate(kappa):
    """Rolling axion, no expansion, no back-reaction: the E equation of the paper's
    ALP-gauge system reads, in cosmic time and physical units,
        A'' = curl curl A - (alpha_L / m_p) phi_dot curl A,
    so a helical mode of wavenumber k grows at Gamma^2 = (alpha_L / m_p) phi_dot k - k^2.
    In program units phi = f_star phi~ and x = x~ / omega_star, phi_dot = f_star omega_star v,
    hence Gamma~^2 = alpha_L (f_star / m_p) v k~ - k~^2 with f_star / m_p = sqrt(kappa).  On the
    lattice k -> sin(k dx)/dx in the clover curl and k^2 -> (2 sin(k dx/2)/dx)^2.  Run at
    kappa = 0.3 too, where alpha_L kappa, alpha_L sqrt(kappa) and alpha_L differ."""
    N, L = 8, 8.0
    kB_fn = lambda k, dx: np.sin(k * dx) / dx
    kL_fn = lambda k, dx: 2 * np.sin(k * dx / 2) / dx
    k, dx = 2 * np.pi / L, L / N
    kB, kL = kB_fn(k, dx), kL_fn(k, dx)
    g_phys = 2 * kL ** 2 / kB  # alpha_L f_star / m_p, chosen so that Gamma = kL at v = 1
    alphaL = g_phys / np.sqrt(kappa)
    model = O.make_model(N, L, nf=1, alpha=0.0, kappa=kappa, gauge=1, alphaL=alphaL, ws2=0.0)
    st = O.new_state(model)
    v = 1.0
    st.pi[:] = v  # phi' = v (a = 1, alpha = 0), V = 0, no back-reaction
    st.links, _, _ = _z_wave(N, L, 1e-9)
    gamma = np.sqrt(alphaL * np.sqrt(kappa) * v * kB - kL ** 2)
    h, ts, amps = 0.05, [], []
    for _ in range(12):
        O.step(model, st, O.RK4_5, h, 20)
        ts.append(st.abt[2])
        amps.append(_mode_amplitude(st.links, N, L))
    assert np.allclose(st.pi, 1.0)  # the axion velocity is untouched
    slope = np.polyfit(ts[6:], np.log(amps[6:]), 1)[0]
    assert slope == pytest.approx(gamma, rel=2e-3)
    assert amps[-1] < 1e-4  # linear regime
    # and the continuum rate within the lattice corrections
    assert slope == pytest.approx(np.sqrt(g_phys * k - k * k), rel=0.1)


@pytest.mark.parametrize("scheme,order", [(O.RK3_3, 3)])
def test_hubble_constraint_with_gauge_fields_converges(scheme, order):
    N = 4
    model = O.make_model(N, 3.0, nf=1, alpha=0.5, kappa=0.8, expansion=True, gauge=1, alphaL=1.5, ws2=0.5,
                         m2=(1.0, 0.0))
    viol = []
    for h in (0.02, 0.01):
        st = random_state(model, 11, th_amp=0.3, e_amp=0.3)
        e = O.energies(model, st)
        st.abt[:] = [1.0, np.sqrt(model.kappa * e["rho"] / 3.0), 0.0]
        O.step(model, st, scheme, h, int(round(2.0 / h)))
        viol.append(O.energies(model, st)["hubble_violation"])
    assert viol[0] < 1e-3
    assert np.log2(viol[0] / viol[1]) == pytest.approx(order, abs=0.3)


# ---------------------------------------------------------------- gauge spectra
def _bins_from_power(N, power, dn=1.0):
    """Type-I binning of a per-mode power array (numpy FFT index order), as the oracle bins."""
    s = np.fft.fftfreq(N, 1.0 / N)
    s = np.where(s == -N // 2, N // 2, s)  # Nyquist counted positive, as the oracle does
    sz, sy, sx = np.meshgrid(s, s, s, indexing="ij")
    nm = np.sqrt(sx ** 2 + sy ** 2 + sz ** 2)
    lbin = np.floor(nm / dn + 0.5).astype(int)
    nb = int(np.floor(np.sqrt(3.0) * (N // 2) / dn + 0.5)) + 1
    S = np.bincount(lbin.ravel(), weights=power.ravel(), minlength=nb)[:nb]
    l = np.arange(nb)
    d = np.zeros(nb)
    d[1:] = l[1:] * dn * S[1:] / (float(N) ** 6 * dn)
    return d, (sx, sy, sz)


def _gauge_model(N, L=6.0):
    return O.make_model(N, L, nf=1, gauge=1, alphaL=2.0, ws2=0.6)


def test_gauge_spectra_parseval_electric():
    """Sum over all modes of the electric spectrum = N^3 sum_n E^2 (unnormalised DFT)."""
    N = 8
    m = _gauge_model(N)
    st = O.new_state(m)
    st.links, st.efield = inputs.gauge_state(N, seed=4, theta_amp=0.3, e_amp=0.3)
    k, d, c = O.gauge_spectrum(m, st, 0)
    l = np.arange(len(d))
    S = np.zeros(len(d))
    S[1:] = d[1:] * float(N) ** 6 / l[1:]
    zero = sum(float(np.sum(st.efield[i])) ** 2 for i in range(3))
    assert S.sum() + zero == pytest.approx(N ** 3 * float(np.sum(st.efield ** 2)), rel=1e-12)
    assert c.sum() == N ** 3


def test_gauge_chiralities_sum_to_the_transverse_power():
    """A+ and A- together carry the transverse part of A (numpy FFT with the half-link phase
    and the lattice momentum), bin by bin."""
    N, L = 8, 6.0
    dx = L / N
    m = _gauge_model(N, L)
    st = O.new_state(m)
    st.links, st.efield = inputs.gauge_state(N, seed=5, theta_amp=0.4, e_amp=0.1)
    _, dp, _ = O.gauge_spectrum(m, st, 2)
    _, dm, _ = O.gauge_spectrum(m, st, 3)
    Ah = [np.fft.fftn(st.links[i] / dx) for i in range(3)]  # axes (z, y, x)
    _, (sx, sy, sz) = _bins_from_power(N, np.zeros((N, N, N)))
    kt = [2.0 / dx * np.sin(np.pi * s / N) for s in (sx, sy, sz)]
    Ah = [np.exp(-1j * np.pi * s / N) * a for s, a in zip((sx, sy, sz), Ah)]
    k2 = kt[0] ** 2 + kt[1] ** 2 + kt[2] ** 2
    kdotA = kt[0] * Ah[0] + kt[1] * Ah[1] + kt[2] * Ah[2]
    tot = sum(np.abs(a) ** 2 for a in Ah)
    with np.errstate(invalid="ignore", divide="ignore"):
        trans = np.where(k2 > 0, tot - np.abs(kdotA) ** 2 / k2, 0.0)
    dt, _ = _bins_from_power(N, trans)
    np.testing.assert_allclose(dp + dm, dt, rtol=1e-11, atol=1e-14 * dt.max())
    assert 0.2 < dp[1:].sum() / dm[1:].sum() < 5.0  # a random field populates both


def test_gauge_chiralities_vanish_for_a_gradient():
    """A = grad+ chi (theta_i = chi(n + e_i) - chi(n)) is longitudinal: no chirality."""
    N = 8
    m = _gauge_model(N)
    st = O.new_state(m)
    chi = inputs.rng(6).standard_normal((N, N, N))
    st.links = np.stack([np.roll(chi, -1, axis=2 - i) - chi for i in range(3)])
    st.efield = np.zeros_like(st.links)
    for w in (2, 3):
        _, d, _ = O.gauge_spectrum(m, st, w)
        assert np.abs(d).max() < 1e-26


@pytest.mark.parametrize("sign", [1, -1])
def test_helical_wave_lands_in_its_chirality(sign):
    """A circularly polarised plane wave built from numpy's eigenvector of i kh x with
    eigenvalue `sign` puts all of its power into that chirality's bin; its magnetic
    spectrum is |kt|^2 times it at small amplitude (B = curl A)."""
    N, L = 8, 6.0
    dx = L / N
    s = np.array([1, 2, 0])
    kt = 2.0 / dx * np.sin(np.pi * s / N)
    kh = kt / np.linalg.norm(kt)
    cross = np.array([[0, -kh[2], kh[1]], [kh[2], 0, -kh[0]], [-kh[1], kh[0], 0]])
    w, vec = np.linalg.eig(1j * cross)
    e = vec[:, int(np.argmin(np.abs(w - sign)))]
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    amp = 1e-5
    links = []
    for c in range(3):
        pos = [x + 0.5 * (c == 0), y + 0.5 * (c == 1), z + 0.5 * (c == 2)]
        phase = 2 * np.pi / N * (s[0] * pos[0] + s[1] * pos[1] + s[2] * pos[2])
        links.append(dx * np.real(amp * e[c] * np.exp(1j * phase)))
    m = _gauge_model(N, L)
    st = O.new_state(m)
    st.links = np.stack(links)
    st.efield = np.zeros_like(st.links)
    _, dp, _ = O.gauge_spectrum(m, st, 2)
    _, dm, _ = O.gauge_spectrum(m, st, 3)
    _, dB, _ = O.gauge_spectrum(m, st, 1)
    mine, other = (dp, dm) if sign > 0 else (dm, dp)
    lb = int(np.floor(np.linalg.norm(s) + 0.5))
    assert mine[lb] > 0 and other.max() < 1e-24 * mine[lb]
    assert np.count_nonzero(mine > 1e-20 * mine[lb]) == 1
    assert dB[lb] == pytest.approx(np.dot(kt, kt) * mine[lb], rel=1e-8)
