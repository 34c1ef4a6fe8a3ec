"""GPU parity of the axion-U(1) Runge-Kutta stages against the oracle.

Section "ALP-gauge interactions", Eq. AxionInfEOM, integrated with the low-storage
RK3-3 / RK4-5 schemes.  Tolerances: 1e-10 relative L2 in FP64, 1e-4 in FP32, for the
axion, its momentum, the link angles and the electric fields; the Gauss diagnostic is
compared with the oracle's lattice Gauss charge.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs

pytestmark = pytest.mark.gpu

KAPPA, ALPHAL, WS2, M2, LAM = 0.7, 2.0, 0.6, 0.8, 0.3


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


def random_state(model, seed, th_amp=0.3, e_amp=0.3):
    st = O.new_state(model)
    g = inputs.rng(seed)
    st.phi[:] = 0.8 + 0.2 * g.standard_normal(st.phi.shape)
    st.pi[:] = 0.2 * g.standard_normal(st.pi.shape)
    st.links, st.efield = inputs.gauge_state(model.N, seed=seed + 1, theta_amp=th_amp, e_amp=e_amp)
    return st


def up(f, d):
    """f(n + e_d) for direction d (d = 0 is the fastest index)."""
    return np.roll(f, -1, axis=2 - d)


def down(f, d):
    return np.roll(f, 1, axis=2 - d)


def clover_B(th, dx):
    """Clover average of sin(plaquette) / dx^2 in the plane normal to each direction."""
    out = np.zeros_like(th)
    for k in range(3):
        i, j = (k + 1) % 3, (k + 2) % 3
        s = np.sin(th[i] + up(th[j], i) - up(th[i], j) - th[j])
        out[k] = (s + down(s, i) + down(s, j) + down(down(s, i), j)) / (4 * dx * dx)
    return out


def gauss_scale(model, st, g):
    """max_n sum_i (|P_i(n)| + |P_i(n - i)|) / dx with P = a^(1-alpha) E + g W."""
    dx = model.L / model.N
    B = clover_B(st.links, dx)
    phi = st.phi[0]
    sc = np.zeros_like(phi)
    for i in range(3):
        P = st.abt[0] ** (1 - model.alpha) * st.efield[i] + g * 0.5 * (phi * B[i] + up(phi * B[i], i))
        sc += np.abs(P) + np.abs(down(P, i))
    return float(sc.max() / dx)


def run_pair(cl, N, prec, integ, scheme, nsteps, dt=0.01, alpha=0.0, expansion=True, alphaL=ALPHAL, graph=1,
             seed=5, L=None, th_amp=0.3, variant=None):
    L = 0.75 * N if L is None else L
    m = O.make_model(N, L, nf=1, alpha=alpha, kappa=KAPPA, expansion=expansion, gauge=1, alphaL=alphaL, ws2=WS2,
                     m2=(M2, 0.0), lam=(LAM, 0.0))
    st = random_state(m, seed, th_amp=th_amp)
    st.abt[:] = (1.0, 0.0, 0.0)
    if expansion:
        st.abt[1] = math.sqrt(KAPPA * O.energies(m, st)["rho"] / 3.0)  # a = 1
    st0 = st.copy()
    dtype = np.float64 if prec == 0 else np.float32
    with cl.Lattice(N, L, 1, prec, integ, gauge=cl.CL_GAUGE_U1_AXION, expansion=expansion, alpha=alpha,
                    kappa=KAPPA, dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [M2, LAM, 0.0, 0.0, 0.0])
        g.cl_set_gauge_coupling(alphaL, WS2)
        g.cl_set_option(cl.CL_OPT_GRAPH, graph)
        if variant is not None:
            g.cl_set_option(cl.CL_OPT_PASS_VARIANT, variant)
        g.cl_set_state(cl.CL_FIELD_PHI0, st.phi[0].astype(dtype))
        g.cl_set_state(cl.CL_FIELD_PI0, st.pi[0].astype(dtype))
        for i in range(3):
            g.cl_set_state(cl.CL_FIELD_THETA1 + i, st.links[i].astype(dtype))
            g.cl_set_state(cl.CL_FIELD_E1 + i, st.efield[i].astype(dtype))
        g.cl_set_scalars(st.abt[0], st.abt[1], 0.0)
        e0 = g.cl_energies()
        g.cl_step(nsteps)
        launches = g.cl_last_launch_count()
        out = {
            "phi": g.cl_get_state(cl.CL_FIELD_PHI0),
            "pi": g.cl_get_state(cl.CL_FIELD_PI0),
            "th": np.stack([g.cl_get_state(cl.CL_FIELD_THETA1 + i) for i in range(3)]),
            "E": np.stack([g.cl_get_state(cl.CL_FIELD_E1 + i) for i in range(3)]),
        }
        e = g.cl_energies()
    O.step(m, st, scheme, dt, nsteps)
    return out, e0, e, st0, st, m, launches


CASES = [(2, O.RK3_3, 3), (3, O.RK4_5, 5), (7, O.RK3_4, 4)]


@pytest.mark.parametrize("integ,scheme,stages", CASES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4)])
@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_u1_parity(cl, integ, scheme, stages, prec, tol, alpha):
    out, e0, e, st0, st, m, launches = run_pair(cl, 8, prec, integ, scheme, 20, alpha=alpha)
    assert rel_l2(out["phi"], st.phi[0]) < tol
    assert rel_l2(out["pi"], st.pi[0]) < tol
    assert rel_l2(out["th"], st.links) < tol
    assert rel_l2(out["E"], st.efield) < tol
    eo = O.energies(m, st)
    assert e["a"] == pytest.approx(st.abt[0], rel=tol)
    assert e["adot"] == pytest.approx(st.abt[1], rel=tol)
    assert e["t"] == pytest.approx(st.abt[2], rel=1e-12)
    for k_gpu, k_orc in [("KE", "KEM"), ("GB", "GEM"), ("rho", "rho"), ("p", "p"), ("V", "V"), ("K0", "K0"),
                         ("G0", "G0")]:
        assert e[k_gpu] == pytest.approx(eo[k_orc], rel=max(tol, 1e-9), abs=1e-14), k_gpu
    assert e["step"] == 20
    # helper fields + stage kernel, and one Gauss-tracking reduction per step (gather form)
    assert launches == 20 * stages * 2 + 20


@pytest.mark.parametrize("integ,scheme,stages", CASES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4)])
@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_u1_fused_stage_parity(cl, integ, scheme, stages, prec, tol, alpha):
    """The fused stage (CL_OPT_PASS_VARIANT 1: plaquettes in shared memory, one launch per
    stage) at N = 32 and 64 against the oracle, including the energies and the magnetic
    energy each block counts for the plaquettes whose lower corner it owns."""
    for N, n in ((32, 6), (64, 2)):
        out, e0, e, st0, st, m, launches = run_pair(cl, N, prec, integ, scheme, n, alpha=alpha, th_amp=0.5,
                                                    variant=1)
        assert rel_l2(out["phi"], st.phi[0]) < tol
        assert rel_l2(out["pi"], st.pi[0]) < tol
        assert rel_l2(out["th"], st.links) < tol
        assert rel_l2(out["E"], st.efield) < tol
        eo = O.energies(m, st)
        e0o = O.energies(m, st0)
        assert e["a"] == pytest.approx(st.abt[0], rel=tol)
        assert e["adot"] == pytest.approx(st.abt[1], rel=tol)
        for k_gpu, k_orc in [("KE", "KEM"), ("GB", "GEM"), ("rho", "rho"), ("p", "p")]:
            assert e[k_gpu] == pytest.approx(eo[k_orc], rel=max(tol, 1e-9)), k_gpu
            assert e0[k_gpu] == pytest.approx(e0o[k_orc], rel=max(tol, 1e-9)), k_gpu
        # one fused launch per stage; per step the plaquette fields and the Gauss-tracking reduction
        assert launches == n * stages + 2 * n


def test_u1_fused_and_two_launch_forms_agree(cl):
    """The fused stage and the plaquette + stage launches on the same 32^3 state."""
    res = []
    for variant in (1, 0):
        out, e0, e, st0, st, m, launches = run_pair(cl, 32, 0, cl.CL_INT_RK3_3, O.RK3_3, 4, alpha=0.5,
                                                    variant=variant)
        res.append((out, e, launches))
    for k in ("phi", "pi", "th", "E"):
        assert rel_l2(res[0][0][k], res[1][0][k]) < 1e-13, k
    assert res[0][1]["rho"] == pytest.approx(res[1][1]["rho"], rel=1e-12)
    assert res[0][2] == 4 * 3 + 4 * 2 and res[1][2] == 4 * 3 * 2 + 4


@pytest.mark.parametrize("integ,scheme,stages", CASES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4)])
@pytest.mark.parametrize("alpha", [0.0, 1.0])
@pytest.mark.parametrize("form", [2, 3])
def test_u1_staged_parity(cl, integ, scheme, stages, prec, tol, alpha, form):
    """The staged launches (CL_OPT_PASS_VARIANT 2, the default where N % 32 == 0: every
    plane's neighbourhood in shared memory; 3: the same in one launch per stage with the
    plaquette fields in shared memory) at N = 32 and 64 against the oracle, with the energies
    of the initial and final states."""
    for N, n in ((32, 6), (64, 2)):
        out, e0, e, st0, st, m, launches = run_pair(cl, N, prec, integ, scheme, n, alpha=alpha, th_amp=0.5,
                                                    variant=form if (N == 32 or form == 3) else None)
        assert rel_l2(out["phi"], st.phi[0]) < tol
        assert rel_l2(out["pi"], st.pi[0]) < tol
        assert rel_l2(out["th"], st.links) < tol
        assert rel_l2(out["E"], st.efield) < tol
        eo = O.energies(m, st)
        e0o = O.energies(m, st0)
        assert e["a"] == pytest.approx(st.abt[0], rel=tol)
        assert e["adot"] == pytest.approx(st.abt[1], rel=tol)
        for k_gpu, k_orc in [("KE", "KEM"), ("GB", "GEM"), ("rho", "rho"), ("p", "p"), ("V", "V"), ("K0", "K0"),
                             ("G0", "G0")]:
            assert e[k_gpu] == pytest.approx(eo[k_orc], rel=max(tol, 1e-9)), k_gpu
            assert e0[k_gpu] == pytest.approx(e0o[k_orc], rel=max(tol, 1e-9)), k_gpu
        assert launches == n * stages * (2 if form == 2 else 1)


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (2, 2e-6)])
@pytest.mark.parametrize("dz", [0, 1, 5, 31])
@pytest.mark.parametrize("form", [2, 3])
def test_u1_staged_and_gather_forms_agree(cl, prec, tol, dz, form):
    """Staged and gather launches on the same 32^3 state, with the library's z chunk and
    with chunks of 1, 5 (ragged last chunk) and 31 planes (a last chunk of one plane)."""
    res = []
    for variant in (form, 0):
        L = 24.0
        m = O.make_model(32, L, nf=1, alpha=0.5, kappa=KAPPA, expansion=True, gauge=1, alphaL=ALPHAL, ws2=WS2,
                         m2=(M2, 0.0), lam=(LAM, 0.0))
        st = random_state(m, 11, th_amp=0.5)
        dtype = np.float64 if prec == 0 else np.float32
        with cl.Lattice(32, L, 1, prec, cl.CL_INT_RK3_3, gauge=cl.CL_GAUGE_U1_AXION, expansion=True, alpha=0.5,
                        kappa=KAPPA, dt=0.01) as g:
            g.cl_set_potential(cl.CL_POT_POLY, [M2, LAM, 0.0, 0.0, 0.0])
            g.cl_set_gauge_coupling(ALPHAL, WS2)
            g.cl_set_option(cl.CL_OPT_PASS_VARIANT, variant)
            if dz:
                g.cl_set_option(cl.CL_OPT_TILE_DZ, dz)
            assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == variant
            g.cl_set_state(cl.CL_FIELD_PHI0, st.phi[0].astype(dtype))
            g.cl_set_state(cl.CL_FIELD_PI0, st.pi[0].astype(dtype))
            for i in range(3):
                g.cl_set_state(cl.CL_FIELD_THETA1 + i, st.links[i].astype(dtype))
                g.cl_set_state(cl.CL_FIELD_E1 + i, st.efield[i].astype(dtype))
            g.cl_set_scalars(1.0, 0.3, 0.0)
            g.cl_step(4)
            out = {k: g.cl_get_state(f) for k, f in (("phi", cl.CL_FIELD_PHI0), ("pi", cl.CL_FIELD_PI0),
                                                       ("E1", cl.CL_FIELD_E1), ("E3", cl.CL_FIELD_E3),
                                                       ("th2", cl.CL_FIELD_THETA2))}
            res.append((out, g.cl_energies()))
    for k in res[0][0]:
        assert rel_l2(res[0][0][k], res[1][0][k]) < tol, k
    for k in ("rho", "KE", "GB", "a", "adot"):
        assert res[0][1][k] == pytest.approx(res[1][1][k], rel=max(tol, 1e-12)), k


def test_u1_variant_defaults(cl):
    """The library picks the staged launches where N % 32 == 0 and the gather launches
    elsewhere; variant 2 is accepted only on an axion-U(1) lattice."""
    for N, want in ((32, 2), (24, 0)):
        with cl.Lattice(N, 10.0, 1, 2, cl.CL_INT_RK3_3, gauge=cl.CL_GAUGE_U1_AXION, kappa=KAPPA, dt=0.01) as g:
            assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == want
    with cl.Lattice(32, 10.0, 1, 2, cl.CL_INT_VV2) as g:
        with pytest.raises(cl.CLError):
            g.cl_set_option(cl.CL_OPT_PASS_VARIANT, 2)


@pytest.mark.parametrize("N", [5, 7, 12])
def test_u1_ragged_sizes(cl, N):
    out, *_, st, m, _ = run_pair(cl, N, 0, cl.CL_INT_RK4_5, O.RK4_5, 6, alpha=0.5)
    assert rel_l2(out["phi"], st.phi[0]) < 1e-12
    assert rel_l2(out["pi"], st.pi[0]) < 1e-12
    assert rel_l2(out["th"], st.links) < 1e-12
    assert rel_l2(out["E"], st.efield) < 1e-12


def test_u1_frozen_background(cl):
    """Without expansion a and a' stay at their initial values (no Hubble friction)."""
    out, e0, e, st0, st, m, _ = run_pair(cl, 8, 0, cl.CL_INT_RK3_3, O.RK3_3, 10, expansion=False)
    assert rel_l2(out["E"], st.efield) < 1e-10
    assert e["a"] == 1.0 and e["adot"] == 0.0


def test_u1_graph_equals_plain(cl):
    a = run_pair(cl, 8, 2, cl.CL_INT_RK4_5, O.RK4_5, 7, graph=1)[0]
    b = run_pair(cl, 8, 2, cl.CL_INT_RK4_5, O.RK4_5, 7, graph=0)[0]
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_u1_energies_of_initial_state(cl):
    out, e0, e, st0, st, m, _ = run_pair(cl, 8, 0, cl.CL_INT_RK3_3, O.RK3_3, 1, alpha=1.0)
    eo = O.energies(m, st0)
    assert e0["KE"] == pytest.approx(eo["KEM"], rel=1e-12)
    assert e0["GB"] == pytest.approx(eo["GEM"], rel=1e-12)
    assert e0["rho"] == pytest.approx(eo["rho"], rel=1e-12)
    assert e0["hubble_violation"] == pytest.approx(eo["hubble_violation"], abs=1e-12)


@pytest.mark.parametrize("alphaL", [0.0, ALPHAL])
def test_u1_gauss_diagnostic_matches_oracle(cl, alphaL):
    """cl_energies reports max|G| / max sum|P| of the current state; compare with the
    oracle's Gauss charge of the same state (random links and fields: G is O(1))."""
    out, e0, e, st0, st, m, _ = run_pair(cl, 8, 0, cl.CL_INT_RK3_3, O.RK3_3, 4, alphaL=alphaL, alpha=0.5)
    g = alphaL * math.sqrt(KAPPA)
    for est, s in [(e0, st0), (e, st)]:
        ref = np.abs(O.u1_gauss(m, s)).max() / gauss_scale(m, s, g)
        assert est["gauss_violation"] == pytest.approx(ref, rel=1e-8)


def test_u1_gauss_conserved(cl):
    """A divergence-free electric field with the coupling off: the lattice Gauss law holds to
    roundoff through Runge-Kutta (each stage adds a divergence-free increment)."""
    N, L = 8, 6.0
    m = O.make_model(N, L, nf=1, alpha=0.0, kappa=KAPPA, expansion=True, gauge=1, alphaL=0.0, ws2=WS2,
                     m2=(M2, 0.0), lam=(LAM, 0.0))
    st = random_state(m, 11)
    # E = backward curl of a random vector field: div- E = 0 identically
    v = inputs.rng(12).standard_normal((3, N, N, N)) * 0.3
    dx = L / N
    st.efield = np.stack([((v[(i + 2) % 3] - down(v[(i + 2) % 3], (i + 1) % 3))
                           - (v[(i + 1) % 3] - down(v[(i + 1) % 3], (i + 2) % 3))) / dx for i in range(3)])
    assert np.abs(O.u1_gauss(m, st)).max() < 1e-12
    with cl.Lattice(N, L, 1, cl.CL_PREC_FP64, cl.CL_INT_RK4_5, gauge=cl.CL_GAUGE_U1_AXION, alpha=0.0,
                    kappa=KAPPA, dt=0.01) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [M2, LAM, 0.0, 0.0, 0.0])
        g.cl_set_gauge_coupling(0.0, WS2)
        g.cl_set_state(cl.CL_FIELD_PHI0, st.phi[0])
        g.cl_set_state(cl.CL_FIELD_PI0, st.pi[0])
        for i in range(3):
            g.cl_set_state(cl.CL_FIELD_THETA1 + i, st.links[i])
            g.cl_set_state(cl.CL_FIELD_E1 + i, st.efield[i])
        g.cl_set_scalars(1.0)  # a' from Eq. Friedmann2 with the electromagnetic energy
        assert g.cl_energies()["gauss_violation"] < 1e-14
        g.cl_step(40)
        e = g.cl_energies()
        assert e["gauss_violation"] < 1e-13
        assert e["hubble_violation"] < 1e-3


def test_u1_hubble_init_includes_em_energy(cl):
    """cl_set_scalars(a, NaN) solves Eq. Friedmann2 with rho including E^2 and B^2."""
    N, L = 8, 6.0
    m = O.make_model(N, L, nf=1, alpha=1.0, kappa=KAPPA, expansion=True, gauge=1, alphaL=ALPHAL, ws2=WS2,
                     m2=(M2, 0.0), lam=(LAM, 0.0))
    st = random_state(m, 21)
    st.abt[:] = (1.2, 0.0, 0.0)
    rho = O.energies(m, st)["rho"]
    with cl.Lattice(N, L, 1, cl.CL_PREC_FP64, cl.CL_INT_RK3_3, gauge=cl.CL_GAUGE_U1_AXION, alpha=1.0,
                    kappa=KAPPA, dt=0.01) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [M2, LAM, 0.0, 0.0, 0.0])
        g.cl_set_gauge_coupling(ALPHAL, WS2)
        g.cl_set_state(cl.CL_FIELD_PHI0, st.phi[0])
        g.cl_set_state(cl.CL_FIELD_PI0, st.pi[0])
        for i in range(3):
            g.cl_set_state(cl.CL_FIELD_THETA1 + i, st.links[i])
            g.cl_set_state(cl.CL_FIELD_E1 + i, st.efield[i])
        g.cl_set_scalars(1.2)
        e = g.cl_energies()
    assert e["rho"] == pytest.approx(rho, rel=1e-12)
    assert e["adot"] == pytest.approx(1.2 ** 2 * math.sqrt(KAPPA * rho / 3.0), rel=1e-12)
    assert e["hubble_violation"] < 1e-12


def test_u1_invalid_configurations(cl):
    with pytest.raises(cl.CLError):  # the leapfrog of a gauge lattice is order 2 only
        cl.Lattice(8, 6.0, 1, cl.CL_PREC_FP64, cl.CL_INT_YOSHIDA4, gauge=cl.CL_GAUGE_U1_AXION)
    with pytest.raises(cl.CLError):
        cl.Lattice(8, 6.0, 2, cl.CL_PREC_FP64, cl.CL_INT_RK3_3, gauge=cl.CL_GAUGE_U1_AXION)
    with pytest.raises(cl.CLError):
        cl.Lattice(8, 6.0, 1, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_RK3_3, gauge=cl.CL_GAUGE_U1_AXION)
    with cl.Lattice(8, 6.0, 1, cl.CL_PREC_FP64, cl.CL_INT_RK3_3) as g:
        with pytest.raises(cl.CLError):
            g.cl_set_gauge_coupling(1.0, 1.0)
        with pytest.raises(cl.CLError):
            g.cl_set_state(cl.CL_FIELD_THETA1, np.zeros((8, 8, 8)))
    with cl.Lattice(8, 6.0, 1, cl.CL_PREC_FP64, cl.CL_INT_RK3_3, gauge=cl.CL_GAUGE_U1_AXION) as g:
        with pytest.raises(cl.CLError):
            g.cl_set_gauge_coupling(1.0, -1.0)


@pytest.mark.parametrize("N,prec", [(8, 0), (12, 2), (32, 0), (16, 2)])
def test_gauge_spectra_match_oracle(cl, N, prec):
    """Electric, magnetic and the two chirality spectra (cl_gauge_spectrum) against the
    oracle on the same state (FP32 states are handed to the oracle as stored), both
    binnings and types, N = 8 .. 32 (Nyquist planes and the conjugate partners of the half
    spectrum)."""
    L = 0.75 * N
    m = O.make_model(N, L, nf=1, alpha=0.0, kappa=KAPPA, gauge=1, alphaL=ALPHAL, ws2=WS2, m2=(M2, 0.0),
                     lam=(LAM, 0.0))
    st = random_state(m, 9, th_amp=0.4, e_amp=0.3)
    dtype = np.float64 if prec == 0 else np.float32
    st.links = st.links.astype(dtype).astype(np.float64)
    st.efield = st.efield.astype(dtype).astype(np.float64)
    with cl.Lattice(N, L, 1, prec, cl.CL_INT_RK3_3, gauge=cl.CL_GAUGE_U1_AXION, alpha=0.0, kappa=KAPPA,
                    dt=0.01) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [M2, LAM, 0.0, 0.0, 0.0])
        g.cl_set_gauge_coupling(ALPHAL, WS2)
        g.cl_set_state(cl.CL_FIELD_PHI0, st.phi[0].astype(dtype))
        g.cl_set_state(cl.CL_FIELD_PI0, st.pi[0].astype(dtype))
        for i in range(3):
            g.cl_set_state(cl.CL_FIELD_THETA1 + i, st.links[i].astype(dtype))
            g.cl_set_state(cl.CL_FIELD_E1 + i, st.efield[i].astype(dtype))
        g.cl_set_scalars(1.0)
        for which in (cl.CL_GSPEC_E, cl.CL_GSPEC_B, cl.CL_GSPEC_APLUS, cl.CL_GSPEC_AMINUS):
            for dn, type_ in ((1.0, 1), (0.5, 2)):
                k, d, c = g.cl_gauge_spectrum(which, dn, type_)
                ko, do, co = O.gauge_spectrum(m, st, which, dn, type_)
                assert np.array_equal(c, co), (which, dn)
                np.testing.assert_allclose(k, ko, rtol=1e-14)
                np.testing.assert_allclose(d, do, rtol=1e-10, atol=1e-12 * do.max()), (which, dn)
    with cl.Lattice(8, 6.0, 1, 0, cl.CL_INT_VV2) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
        with pytest.raises(cl.CLError):
            g.cl_gauge_spectrum(cl.CL_GSPEC_E)  # no gauge field


@pytest.mark.parametrize("variant,N", [(2, 32), (0, 32), (1, 32), (3, 32), (None, 12)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4)])
def test_u1_gauss_tracked_each_step(cl, variant, N, prec, tol):
    """cl_step tracks the Gauss law every step (config "Gauss constraint tracked each step"):
    after each step, gauss_rms_step is the rms lattice Gauss charge of that step's starting
    state, r = dx sqrt(sum_n G(n)^2) / (a^(1-alpha) sqrt(sum_n E(n)^2)) with G the oracle's
    Gauss charge, and gauss_rms_max the largest value so far.  The staged launch form (2)
    sums it in its first stage; the gather (0) and fused (1) forms, and N = 12 (gather by
    default), launch a reduction for it.  Random links and fields: G is O(1)."""
    L, dt, alpha = 0.75 * N, 0.01, 0.5
    m = O.make_model(N, L, nf=1, alpha=alpha, kappa=KAPPA, expansion=True, gauge=1, alphaL=ALPHAL, ws2=WS2,
                     m2=(M2, 0.0), lam=(LAM, 0.0))
    st = random_state(m, 31)
    st.abt[:] = (1.1, 0.0, 0.0)
    st.abt[1] = 1.1 * math.sqrt(KAPPA * 1.1 ** (2 * alpha) * O.energies(m, st)["rho"] / 3.0)
    dtype = np.float64 if prec == 0 else np.float32
    dx = L / N
    with cl.Lattice(N, L, 1, prec, cl.CL_INT_RK3_3, gauge=cl.CL_GAUGE_U1_AXION, expansion=True, alpha=alpha,
                    kappa=KAPPA, dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [M2, LAM, 0.0, 0.0, 0.0])
        g.cl_set_gauge_coupling(ALPHAL, WS2)
        if variant is not None:
            g.cl_set_option(cl.CL_OPT_PASS_VARIANT, variant)
        g.cl_set_state(cl.CL_FIELD_PHI0, st.phi[0].astype(dtype))
        g.cl_set_state(cl.CL_FIELD_PI0, st.pi[0].astype(dtype))
        for i in range(3):
            g.cl_set_state(cl.CL_FIELD_THETA1 + i, st.links[i].astype(dtype))
            g.cl_set_state(cl.CL_FIELD_E1 + i, st.efield[i].astype(dtype))
        g.cl_set_scalars(st.abt[0], st.abt[1], 0.0)
        assert g.cl_energies()["gauss_rms_max"] == 0.0
        want = {2: 2, 0: 0, 1: 1, 3: 3}.get(variant, 0)
        assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == want
        rmax = 0.0
        for _ in range(3):
            G = O.u1_gauss(m, st)
            r = dx * math.sqrt(float(np.sum(G * G))) / (st.abt[0] ** (1 - alpha) *
                                                        math.sqrt(float(np.sum(st.efield ** 2))))
            rmax = max(rmax, r)
            g.cl_step(1)
            e = g.cl_energies()
            assert r > 0.1
            assert e["gauss_rms_step"] == pytest.approx(r, rel=tol)
            assert e["gauss_rms_max"] == pytest.approx(rmax, rel=tol)
            O.step(m, st, O.RK3_3, dt, 1)


@pytest.mark.parametrize("prec,bound", [(0, 1e-13), (2, 1e-5)])
def test_u1_gauss_tracking_of_a_gauss_state(cl, prec, bound):
    """With the coupling off and a divergence-free E the tracked violation stays at rounding
    level over many steps (staged form, N = 32)."""
    N, L = 32, 24.0
    m = O.make_model(N, L, nf=1, alpha=0.0, kappa=KAPPA, expansion=True, gauge=1, alphaL=0.0, ws2=WS2,
                     m2=(M2, 0.0), lam=(LAM, 0.0))
    st = random_state(m, 13, th_amp=0.2)
    dtype = np.float64 if prec == 0 else np.float32
    E = inputs.solenoidal_field(N, seed=14, amp=0.3)
    with cl.Lattice(N, L, 1, prec, cl.CL_INT_RK3_3, gauge=cl.CL_GAUGE_U1_AXION, alpha=0.0, kappa=KAPPA,
                    dt=0.01, expansion=True) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [M2, LAM, 0.0, 0.0, 0.0])
        g.cl_set_gauge_coupling(0.0, WS2)
        g.cl_set_state(cl.CL_FIELD_PHI0, st.phi[0].astype(dtype))
        g.cl_set_state(cl.CL_FIELD_PI0, st.pi[0].astype(dtype))
        for i in range(3):
            g.cl_set_state(cl.CL_FIELD_THETA1 + i, st.links[i].astype(dtype))
            g.cl_set_state(cl.CL_FIELD_E1 + i, E[i].astype(dtype))
        g.cl_set_scalars(1.0)
        g.cl_step(30)
        e = g.cl_energies()
        assert 0.0 <= e["gauss_rms_max"] < bound
        assert e["gauss_rms_step"] <= e["gauss_rms_max"]


@pytest.mark.parametrize("form", ["rk33", "leapfrog"])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4)])
def test_u1_staged_96_cubed_from_a_periodic_state(cl, form, prec, tol):
    """The staged launches at 96^3, where the stage tiles (32 x 16, 32 x 8 in FP64) and the
    plaquette launches' taller tiles over half z chunks cut the lattice into 3 x 6 and 3 x 3
    tiles (3 x 12 and 3 x 6 in FP64) and the library's z chunks: a state that repeats every 16
    sites evolves as the 16^3 oracle lattice tiled (translation invariance), RK3-3 and the
    leapfrog, FP64 and FP32."""
    integ, scheme = (cl.CL_INT_RK3_3, O.RK3_3) if form == "rk33" else (cl.CL_INT_VV2, O.VV2)
    N, P, n = 96, 16, 4
    reps = N // P
    L = 0.75 * N
    m = O.make_model(P, L * P / N, nf=1, alpha=0.5, kappa=KAPPA, expansion=True, gauge=1, alphaL=ALPHAL, ws2=WS2,
                     m2=(M2, 0.0), lam=(LAM, 0.0))
    st = random_state(m, 13, th_amp=0.5)
    dtype = np.float64 if prec == 0 else np.float32
    for arr in (st.phi, st.pi, st.links, st.efield):
        arr[:] = arr.astype(dtype)
    st.abt[:] = (1.0, math.sqrt(KAPPA * O.energies(m, st)["rho"] / 3.0), 0.0)
    with cl.Lattice(N, L, 1, prec, integ, gauge=cl.CL_GAUGE_U1_AXION, expansion=True, alpha=0.5, kappa=KAPPA,
                    dt=0.01) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [M2, LAM, 0.0, 0.0, 0.0])
        g.cl_set_gauge_coupling(ALPHAL, WS2)
        assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == 2
        g.cl_set_state(cl.CL_FIELD_PHI0, np.tile(st.phi[0], (reps,) * 3).astype(dtype))
        g.cl_set_state(cl.CL_FIELD_PI0, np.tile(st.pi[0], (reps,) * 3).astype(dtype))
        for i in range(3):
            g.cl_set_state(cl.CL_FIELD_THETA1 + i, np.tile(st.links[i], (reps,) * 3).astype(dtype))
            g.cl_set_state(cl.CL_FIELD_E1 + i, np.tile(st.efield[i], (reps,) * 3).astype(dtype))
        g.cl_set_scalars(st.abt[0], st.abt[1], 0.0)
        g.cl_step(n)
        out = {"phi": g.cl_get_state(cl.CL_FIELD_PHI0), "pi": g.cl_get_state(cl.CL_FIELD_PI0),
               "th": np.stack([g.cl_get_state(cl.CL_FIELD_THETA1 + i) for i in range(3)]),
               "E": np.stack([g.cl_get_state(cl.CL_FIELD_E1 + i) for i in range(3)])}
        e = g.cl_energies()
    O.step(m, st, scheme, 0.01, n)
    assert rel_l2(out["phi"], np.tile(st.phi[0], (reps,) * 3)) < tol
    assert rel_l2(out["pi"], np.tile(st.pi[0], (reps,) * 3)) < tol
    for i in range(3):
        assert rel_l2(out["th"][i], np.tile(st.links[i], (reps,) * 3)) < tol
        assert rel_l2(out["E"][i], np.tile(st.efield[i], (reps,) * 3)) < tol
    eo = O.energies(m, st)
    for k_gpu, k_orc in [("KE", "KEM"), ("GB", "GEM"), ("rho", "rho"), ("V", "V")]:
        assert e[k_gpu] == pytest.approx(eo[k_orc], rel=max(tol, 1e-9)), k_gpu
    assert e["a"] == pytest.approx(st.abt[0], rel=max(tol, 1e-10))
