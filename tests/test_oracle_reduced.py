"""Pins of the oracle's reduced (d+1)-dimensional lattices (section "Scalar dynamics in 1+1
and 2+1 dimensions": N^d sites, the Laplacian and the gradient energy summed over the d
directions, everything else as in 3+1).

  * exact discrete dispersion of a free plane wave on N and N^2 sites: the VV transfer
    matrix with omega^2 = m^2 + sum over the d directions of (4/dx^2) sin^2(k_i dx / 2)
    only -- a term of a missing direction would shift the frequency;
  * embedding: a reduced state continued constantly along the missing directions of an
    N^3 lattice evolves, under the (separately pinned) 3-D oracle, into the continued
    reduced result, with the same a, a' and energies -- for the leapfrog, Yoshida-4 and
    RK4-5 with self-consistent expansion and two interacting fields.
"""
import numpy as np
import pytest

from oracle import oracle as O


def _vv_matrix(h, w2):
    c = 1.0 - 0.5 * h * h * w2
    return np.array([[c, h], [-h * w2 * (1.0 - 0.25 * h * h * w2), c]])


@pytest.mark.parametrize("dims,mode", [(1, (3,)), (2, (1, 2))])
def test_reduced_exact_discrete_dispersion(dims, mode):
    N, L, m2 = 8, 4.0, 0.7
    model = O.make_model(N, L=L, nf=1, alpha=1.0, m2=(m2, 0.0), dims=dims)
    st = O.new_state(model)
    x = np.arange(N)
    if dims == 1:
        shape = np.cos(2 * np.pi * mode[0] * x / N + 0.2)[None, None, :]
    else:
        shape = np.cos(2 * np.pi * (mode[0] * x[None, :] + mode[1] * x[:, None]) / N + 0.2)[None, :, :]
    st.phi[0] = shape
    dx = L / N
    w2 = m2 + sum(4.0 / dx**2 * np.sin(np.pi * mi / N) ** 2 for mi in mode)
    h, n = 0.05, 120
    O.step(model, st, O.VV2, h, n)
    amp = np.linalg.matrix_power(_vv_matrix(h, w2), n) @ np.array([1.0, 0.0])
    np.testing.assert_allclose(st.phi[0], amp[0] * shape, atol=1e-12)
    np.testing.assert_allclose(st.pi[0], amp[1] * shape, atol=1e-12)
    e = O.energies(model, st)
    # gradient energy of the wave over the d directions: <(grad+ phi)^2> / (2 a^2)
    g2 = sum(((np.roll(st.phi[0], -1, axis=2 - i) - st.phi[0]) ** 2).mean() for i in range(dims))
    assert e["G0"] == pytest.approx(g2 / dx**2 / 2.0, rel=1e-12)


@pytest.mark.parametrize("dims", [1, 2])
@pytest.mark.parametrize("scheme,h,n", [(O.VV2, 0.02, 15), (O.YOSHIDA4, 0.02, 6), (O.RK4_5, 0.02, 6)])
def test_reduced_lattice_embeds_in_three_dimensions(dims, scheme, h, n):
    N, L = 8, 6.0
    kw = dict(nf=2, alpha=0.5, kappa=0.4, expansion=True, m2=(0.6, 0.3), lam=(1.0, 0.5), g2=2.5)
    red = O.make_model(N, L, dims=dims, **kw)
    full = O.make_model(N, L, **kw)
    rng = np.random.default_rng(7 + dims)
    sr = O.new_state(red)
    sr.phi[:] = np.array([0.9, 0.1])[:, None, None, None] + 0.05 * rng.standard_normal(sr.phi.shape)
    sr.pi[:] = 0.05 * rng.standard_normal(sr.pi.shape)
    sr.abt[:] = (1.0, 0.0, 0.0)
    sr.abt[1] = np.sqrt(0.4 * O.energies(red, sr)["rho"] / 3.0)
    sf = O.new_state(full)
    sf.phi[:] = np.broadcast_to(sr.phi, sf.phi.shape)
    sf.pi[:] = np.broadcast_to(sr.pi, sf.pi.shape)
    sf.abt[:] = sr.abt
    e_r0, e_f0 = O.energies(red, sr), O.energies(full, sf)
    for k in ("K0", "K1", "G0", "G1", "V", "rho", "p"):
        assert e_r0[k] == pytest.approx(e_f0[k], rel=1e-13, abs=1e-15), k
    O.step(red, sr, scheme, h, n)
    O.step(full, sf, scheme, h, n)
    np.testing.assert_allclose(sf.phi, np.broadcast_to(sr.phi, sf.phi.shape), rtol=0, atol=1e-12)
    np.testing.assert_allclose(sf.pi, np.broadcast_to(sr.pi, sf.pi.shape), rtol=0, atol=1e-12)
    np.testing.assert_allclose(sr.abt, sf.abt, rtol=1e-13)
    e_r, e_f = O.energies(red, sr), O.energies(full, sf)
    for k in ("K0", "K1", "G0", "G1", "V", "rho", "p"):
        assert e_r[k] == pytest.approx(e_f[k], rel=1e-12, abs=1e-15), k
