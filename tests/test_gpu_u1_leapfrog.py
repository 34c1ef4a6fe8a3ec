"""GPU parity of the axion-U(1) leapfrog against the oracle (oracle/u1.c: orc_u1_leapfrog).

Section "ALP-gauge interactions" with positions (phi, theta, a) at integer steps and the kick
of the momenta (pi, E, a') implicit at fixed positions, solved with three fixed-point
evaluations of the momentum force (generalized Stoermer-Verlet).  The library runs a step as
three passes -- the second and third evaluations (the third with the drift), then the closing
half-kick merged with the first evaluation of the next step -- and the oracle as the same
arithmetic step by step; tolerances as for the Runge-Kutta schemes: 1e-10 relative L2 in
FP64, 1e-4 in FP32.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests.test_gpu_u1 import ALPHAL, KAPPA, LAM, M2, WS2, gauss_scale, random_state, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cl():
    from paper_2607_24978_gb300 import build_ext, cl as clmod
    build_ext.build()
    clmod.lib()
    return clmod


def start(m, seed, th_amp=0.3, a=1.0):
    st = random_state(m, seed, th_amp=th_amp)
    st.abt[:] = (a, 0.0, 0.0)
    if m.expansion:
        st.abt[1] = a * math.sqrt(KAPPA * a ** (2 * m.alpha) * O.energies(m, st)["rho"] / 3.0)
    return st


def upload(cl, g, st, dtype):
    g.cl_set_state(cl.CL_FIELD_PHI0, st.phi[0].astype(dtype))
    g.cl_set_state(cl.CL_FIELD_PI0, st.pi[0].astype(dtype))
    for i in range(3):
        g.cl_set_state(cl.CL_FIELD_THETA1 + i, st.links[i].astype(dtype))
        g.cl_set_state(cl.CL_FIELD_E1 + i, st.efield[i].astype(dtype))
    g.cl_set_scalars(st.abt[0], st.abt[1], st.abt[2])


def download(cl, g):
    return {"phi": g.cl_get_state(cl.CL_FIELD_PHI0), "pi": g.cl_get_state(cl.CL_FIELD_PI0),
            "th": np.stack([g.cl_get_state(cl.CL_FIELD_THETA1 + i) for i in range(3)]),
            "E": np.stack([g.cl_get_state(cl.CL_FIELD_E1 + i) for i in range(3)])}


def lattice(cl, N, L, prec, alpha, expansion=True, dt=0.01, alphaL=ALPHAL, variant=None, graph=1):
    g = cl.Lattice(N, L, 1, prec, cl.CL_INT_VV2, gauge=cl.CL_GAUGE_U1_AXION, expansion=expansion, alpha=alpha,
                   kappa=KAPPA, dt=dt)
    g.cl_set_potential(cl.CL_POT_POLY, [M2, LAM, 0.0, 0.0, 0.0])
    g.cl_set_gauge_coupling(alphaL, WS2)
    g.cl_set_option(cl.CL_OPT_GRAPH, graph)
    if variant is not None:
        g.cl_set_option(cl.CL_OPT_PASS_VARIANT, variant)
    return g


def check_state(out, st, tol):
    assert rel_l2(out["phi"], st.phi[0]) < tol
    assert rel_l2(out["pi"], st.pi[0]) < tol
    assert rel_l2(out["th"], st.links) < tol
    assert rel_l2(out["E"], st.efield) < tol


def check_energies(e, m, st, tol):
    eo = O.energies(m, st)
    assert e["a"] == pytest.approx(st.abt[0], rel=tol)
    assert e["adot"] == pytest.approx(st.abt[1], rel=tol)
    assert e["t"] == pytest.approx(st.abt[2], rel=1e-12)
    for k_gpu, k_orc in [("KE", "KEM"), ("GB", "GEM"), ("rho", "rho"), ("p", "p"), ("V", "V"), ("K0", "K0"),
                         ("G0", "G0")]:
        assert e[k_gpu] == pytest.approx(eo[k_orc], rel=max(tol, 1e-9), abs=1e-13), k_gpu
    # a relative quantity, small where the constraint holds: compared absolutely
    assert e["hubble_violation"] == pytest.approx(eo["hubble_violation"], abs=tol)


@pytest.mark.parametrize("N,variant", [(8, None), (12, None), (32, None), (32, 0), (64, None), (32, 3), (64, 3)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4)])
@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.0])
def test_leapfrog_parity(cl, N, variant, prec, tol, alpha):
    """Gather launches (N = 8, 12, and 32 on request) and staged launches (N = 32, 64, the
    default where N % 32 == 0), with self-consistent expansion: fields, a, a', the energies of
    the integer-time state and the launch count (the opening pass, then per step three
    plaquette + stage launch pairs, and with the gather form one Gauss reduction)."""
    n = 20 if N <= 32 else 4
    L = 0.75 * N
    m = O.make_model(N, L, nf=1, alpha=alpha, kappa=KAPPA, expansion=True, gauge=1, alphaL=ALPHAL, ws2=WS2,
                     m2=(M2, 0.0), lam=(LAM, 0.0))
    st = start(m, 5, th_amp=0.5)
    dtype = np.float64 if prec == 0 else np.float32
    with lattice(cl, N, L, prec, alpha, variant=variant) as g:
        assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == (2 if N % 32 == 0 and variant is None else (variant or 0))
        upload(cl, g, st, dtype)
        g.cl_step(n)
        launches = g.cl_last_launch_count()
        out = download(cl, g)
        e = g.cl_energies()
    O.step(m, st, O.VV2, 0.01, n)
    check_state(out, st, tol)
    check_energies(e, m, st, tol)
    assert e["step"] == n
    per_step = {None: 6 if N % 32 == 0 else 7, 0: 7, 3: 3}[variant]
    assert launches == (1 if variant == 3 else 2) + per_step * n


@pytest.mark.parametrize("prec,tol,ftol", [(0, 1e-10, 1e-12), (2, 1e-4, 1e-5)])
@pytest.mark.parametrize("first", [0, 3])
def test_switching_to_the_staged_form_with_the_leapfrog_open(cl, prec, tol, ftol, first):
    """Passes 2 and 3 of the staged form reuse the sin P and cos P that its pass 1 saved.
    After steps in the gather (0) or single-launch (3) form, whose pass 1 saves nothing, the
    first staged step saves them with one plaquette launch of its own: 3 + 4 steps across the
    switch follow the oracle and agree with 7 staged steps to rounding (the forms differ only
    in the order of their roundings)."""
    N, L, alpha = 32, 24.0, 0.5
    m = O.make_model(N, L, nf=1, alpha=alpha, kappa=KAPPA, expansion=True, gauge=1, alphaL=ALPHAL, ws2=WS2,
                     m2=(M2, 0.0), lam=(LAM, 0.0))
    st = start(m, 9, th_amp=0.5)
    dtype = np.float64 if prec == 0 else np.float32
    with lattice(cl, N, L, prec, alpha, variant=first) as g:
        upload(cl, g, st, dtype)
        g.cl_step(3)
        g.cl_set_option(cl.CL_OPT_PASS_VARIANT, 2)
        g.cl_step(4)
        launches = g.cl_last_launch_count()
        out = download(cl, g)
    with lattice(cl, N, L, prec, alpha) as g:
        upload(cl, g, st, dtype)
        g.cl_step(7)
        ref = download(cl, g)
    O.step(m, st, O.VV2, 0.01, 7)
    check_state(out, st, tol)
    for k in ref:
        assert rel_l2(out[k], ref[k]) < ftol, k
    assert launches == 1 + 6 * 4


@pytest.mark.parametrize("prec", [0, 2])
def test_reads_leave_the_trajectory_alone_and_graphs_match_plain_launches(cl, prec):
    """Reading states, energies and spectra between steps keeps the leapfrog open (the
    integer-time momenta are kept beside the staggered ones), so 5 + 5 steps equal 10 steps
    bit for bit; graph replays equal plain launches."""
    N, L, alpha = 32, 24.0, 0.5
    m = O.make_model(N, L, nf=1, alpha=alpha, kappa=KAPPA, expansion=True, gauge=1, alphaL=ALPHAL, ws2=WS2,
                     m2=(M2, 0.0), lam=(LAM, 0.0))
    st = start(m, 7)
    dtype = np.float64 if prec == 0 else np.float32
    res = []
    for split, graph in ((True, 1), (False, 1), (False, 0)):
        with lattice(cl, N, L, prec, alpha, graph=graph) as g:
            upload(cl, g, st, dtype)
            if split:
                g.cl_step(5)
                download(cl, g)
                g.cl_energies()
                g.cl_spectrum(cl.CL_FIELD_PI0)
                g.cl_gauge_spectrum(cl.CL_GSPEC_E)
                g.cl_get_scalars()
                g.cl_step(5)
            else:
                g.cl_step(10)
            res.append((download(cl, g), g.cl_energies()))
    for r in res[1:]:
        for k in res[0][0]:
            assert np.array_equal(r[0][k], res[0][0][k]), k
        for k in ("rho", "a", "adot", "gauss_rms_step"):
            assert r[1][k] == res[0][1][k], k


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4)])
def test_writing_the_state_closes_the_leapfrog(cl, prec, tol):
    """cl_set_state commits the integer-time momenta and a'; the next cl_step opens again
    with the force of that state, like a new oracle call."""
    N, L, alpha = 32, 24.0, 0.0
    m = O.make_model(N, L, nf=1, alpha=alpha, kappa=KAPPA, expansion=True, gauge=1, alphaL=ALPHAL, ws2=WS2,
                     m2=(M2, 0.0), lam=(LAM, 0.0))
    st = start(m, 9)
    dtype = np.float64 if prec == 0 else np.float32
    with lattice(cl, N, L, prec, alpha) as g:
        upload(cl, g, st, dtype)
        g.cl_step(6)
        phi = g.cl_get_state(cl.CL_FIELD_PHI0)
        g.cl_set_state(cl.CL_FIELD_PHI0, phi)  # same values: closes the leapfrog
        g.cl_step(6)
        out = download(cl, g)
        e = g.cl_energies()
    O.step(m, st, O.VV2, 0.01, 6)
    st.phi[0] = st.phi[0].astype(dtype)  # what was written back
    O.step(m, st, O.VV2, 0.01, 6)
    check_state(out, st, tol)
    check_energies(e, m, st, tol)


@pytest.mark.parametrize("N", [12, 32])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4)])
def test_gauss_tracked_each_step_and_the_diagnostic(cl, N, prec, tol):
    """gauss_rms_step after cl_step is the rms lattice Gauss charge of the latest step's
    integer-time starting state, r = dx sqrt(sum G^2) / (a^(1-alpha) sqrt(sum E^2)),
    gauss_rms_max the largest over the steps' starting states; gauss_violation is
    max|G| / max sum|P| of the current state."""
    L, alpha, dt = 0.75 * N, 0.5, 0.01
    m = O.make_model(N, L, nf=1, alpha=alpha, kappa=KAPPA, expansion=True, gauge=1, alphaL=ALPHAL, ws2=WS2,
                     m2=(M2, 0.0), lam=(LAM, 0.0))
    st = start(m, 31, a=1.1)
    dtype = np.float64 if prec == 0 else np.float32
    dx = L / N

    def rms(s):
        G = O.u1_gauss(m, s)
        return dx * math.sqrt(float(np.sum(G * G))) / (s.abt[0] ** (1 - alpha) * math.sqrt(float(np.sum(s.efield ** 2))))

    st0 = st.copy()
    with lattice(cl, N, L, prec, alpha, dt=dt) as g:
        upload(cl, g, st0, dtype)
        # the oracle's state after n steps, each from one call (the library stays open between calls)
        states = [st0] + [O.step(m, st0.copy(), O.VV2, dt, n) for n in range(1, 7)]
        rs = [rms(x) for x in states]
        assert min(rs) > 0.1
        for k in range(1, 4):
            g.cl_step(2)
            st = states[2 * k]
            e = g.cl_energies()
            assert e["gauss_rms_step"] == pytest.approx(rs[2 * k - 1], rel=tol)
            assert e["gauss_rms_max"] == pytest.approx(max(rs[:2 * k]), rel=tol)
            gv = np.abs(O.u1_gauss(m, st)).max() / gauss_scale(m, st, ALPHAL * math.sqrt(KAPPA))
            assert e["gauss_violation"] == pytest.approx(gv, rel=max(tol, 1e-8))


def test_gauss_law_without_coupling_and_spectra_of_the_open_state(cl):
    """Coupling off, divergence-free E: the tracked violation stays at rounding level; the
    electric and magnetic spectra of the open state are those of its integer-time fields."""
    from tests import inputs
    N, L = 32, 24.0
    m = O.make_model(N, L, nf=1, alpha=0.0, kappa=KAPPA, expansion=True, gauge=1, alphaL=0.0, ws2=WS2,
                     m2=(M2, 0.0), lam=(LAM, 0.0))
    st = random_state(m, 13, th_amp=0.2)
    st.efield = inputs.solenoidal_field(N, seed=14, amp=0.3)
    st.abt[:] = (1.0, 0.0, 0.0)
    st.abt[1] = math.sqrt(KAPPA * O.energies(m, st)["rho"] / 3.0)
    with lattice(cl, N, L, 0, 0.0, alphaL=0.0) as g:
        upload(cl, g, st, np.float64)
        g.cl_step(30)
        e = g.cl_energies()
        assert 0.0 <= e["gauss_rms_max"] < 1e-13
        spec = {w: g.cl_gauge_spectrum(w, 1.0, 1) for w in (cl.CL_GSPEC_E, cl.CL_GSPEC_B)}
    O.step(m, st, O.VV2, 0.01, 30)
    for w, (k, d, c) in spec.items():
        ko, do, co = O.gauge_spectrum(m, st, w, 1.0, 1)
        np.testing.assert_allclose(d, do, rtol=1e-10, atol=1e-12 * do.max())


def test_leapfrog_options(cl):
    """The fused single-launch form serves only the Runge-Kutta stages."""
    with lattice(cl, 32, 24.0, 2, 0.0) as g:
        with pytest.raises(cl.CLError):
            g.cl_set_option(cl.CL_OPT_PASS_VARIANT, 1)
        g.cl_set_option(cl.CL_OPT_PASS_VARIANT, 0)
        assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == 0
