"""GPU parity of the low-storage Runge-Kutta stages (RK3-3, RK4-5) against the oracle.

Tolerances as for the leapfrog path: 1e-10 relative L2 in FP64, 1e-4 in FP32.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs

pytestmark = pytest.mark.gpu


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


def run_pair(cl, N, nf, prec, integ, scheme, nsteps, dt=0.01, graph=1, seed=31, expansion=True, opts=(),
             effective=None):
    L = 0.8 * N
    pot = [0.6, 1.0, 0.3, 0.0, 2.5 if nf == 2 else 0.0]
    if nf == 1:
        pot[2] = 0.0
    phi, pi = inputs.scalar_state(N, nf, seed=seed, fbar=(0.9, 0.1), amp=0.05, pamp=0.05)
    m = O.make_model(N, L, nf=nf, alpha=0.5, kappa=0.4, expansion=expansion, m2=(pot[0], pot[2]),
                     lam=(pot[1], pot[3]), g2=pot[4])
    st = O.State(phi.copy(), pi.copy(), np.array([1.0, 0.0, 0.0]))
    if expansion:
        st.abt[1] = math.sqrt(0.4 * O.energies(m, st)["rho"] / 3.0)  # a = 1, alpha-time
    dtype = np.float64 if prec == 0 else np.float32
    with cl.Lattice(N, L, nf, prec, integ, expansion=expansion, alpha=0.5, kappa=0.4, dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_POLY, pot)
        g.cl_set_option(cl.CL_OPT_GRAPH, graph)
        for opt, val in opts:
            g.cl_set_option(opt, val)
        if effective is not None:
            effective.update({k: g.cl_get_option(k) for k in (cl.CL_OPT_STAGES, cl.CL_OPT_TILE_BY, cl.CL_OPT_TILE_DZ)})
        for f in range(nf):
            g.cl_set_state(cl.CL_FIELD_PHI0 + f, st.phi[f].astype(dtype))
            g.cl_set_state(cl.CL_FIELD_PI0 + f, st.pi[f].astype(dtype))
        g.cl_set_scalars(st.abt[0], st.abt[1], 0.0)
        g.cl_step(nsteps)
        gphi = np.stack([g.cl_get_state(cl.CL_FIELD_PHI0 + f) for f in range(nf)])
        gpi = np.stack([g.cl_get_state(cl.CL_FIELD_PI0 + f) for f in range(nf)])
        e = g.cl_energies()
        launches = g.cl_last_launch_count()
    O.step(m, st, scheme, dt, nsteps)
    return gphi, gpi, e, st, O.energies(m, st), launches


@pytest.mark.parametrize("integ,scheme,stages", [(2, O.RK3_3, 3), (3, O.RK4_5, 5), (7, O.RK3_4, 4)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4), (2, 1e-4)])
def test_rk_parity(cl, integ, scheme, stages, prec, tol):
    gphi, gpi, e, st, eo, launches = run_pair(cl, 16, 2, prec, integ, scheme, 30)
    assert rel_l2(gphi, st.phi) < tol
    assert rel_l2(gpi, st.pi) < tol
    assert e["a"] == pytest.approx(st.abt[0], rel=tol)
    assert e["adot"] == pytest.approx(st.abt[1], rel=tol)
    assert e["t"] == pytest.approx(st.abt[2], rel=1e-12)
    assert e["rho"] == pytest.approx(eo["rho"], rel=max(tol, 1e-9))
    assert e["step"] == 30
    assert launches == 30 * stages  # no opening pass for Runge-Kutta


@pytest.mark.parametrize("N,nf", [(32, 1), (32, 2), (48, 2)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-6), (2, 2e-6)])
def test_rk_tma_matches_direct_kernel(cl, N, nf, prec, tol):
    """The TMA-staged stage kernel (the default for 16-byte vectors) and the direct-load
    kernel (CL_OPT_STAGES -1) on the same state: same arithmetic per site, so the fields
    agree to the rounding of a and a' (reduction order)."""
    eff_t, eff_d = {}, {}
    t = run_pair(cl, N, nf, prec, cl.CL_INT_RK4_5, O.RK4_5, 6, effective=eff_t)
    d = run_pair(cl, N, nf, prec, cl.CL_INT_RK4_5, O.RK4_5, 6, opts=((cl.CL_OPT_STAGES, -1),), effective=eff_d)
    assert eff_t[cl.CL_OPT_STAGES] >= 3 and eff_d[cl.CL_OPT_STAGES] == -1
    assert rel_l2(t[0], d[0]) < tol
    assert rel_l2(t[1], d[1]) < tol
    assert t[2]["rho"] == pytest.approx(d[2]["rho"], rel=max(tol, 1e-12))
    assert t[2]["a"] == pytest.approx(d[2]["a"], rel=max(tol, 1e-13))


@pytest.mark.parametrize("by,stages,dz", [(1, 3, 0), (5, 4, 0), (7, 0, 0), (3, 6, 5), (0, 3, 31), (32, 0, 0),
                                          (5, 4, -1), (1, 0, -1)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4)])
def test_rk_tma_tilings(cl, by, stages, dz, prec, tol):
    """TMA-staged stages against the oracle at 32^3 over tilings: one-row tiles, a ragged last
    tile (5 and 7 rows), the whole box in one tile, 3 to 6 stages, the library's z chunks,
    fixed chunks (5 planes; 31, leaving a chunk of one plane) and balanced persistent ranges
    (-1)."""
    opts = [(cl.CL_OPT_TILE_BY, by)] if by else []
    opts += [(cl.CL_OPT_STAGES, stages)] if stages else []
    opts += [(cl.CL_OPT_TILE_DZ, dz)] if dz else []
    eff = {}
    gphi, gpi, e, st, eo, launches = run_pair(cl, 32, 2, prec, cl.CL_INT_RK4_5, O.RK4_5, 4, opts=tuple(opts),
                                              effective=eff)
    assert eff[cl.CL_OPT_STAGES] >= 3
    if by:
        assert eff[cl.CL_OPT_TILE_BY] == min(by, 448 // (32 // (4 if prec else 2)))
    assert rel_l2(gphi, st.phi) < tol
    assert rel_l2(gpi, st.pi) < tol
    assert e["a"] == pytest.approx(st.abt[0], rel=tol)
    assert e["rho"] == pytest.approx(eo["rho"], rel=max(tol, 1e-9))
    assert launches == 4 * 5


@pytest.mark.parametrize("N", [7, 10, 24])
def test_rk_ragged_sizes(cl, N):
    gphi, gpi, e, st, eo, _ = run_pair(cl, N, 2, 0, cl.CL_INT_RK4_5, O.RK4_5, 12)
    assert rel_l2(gphi, st.phi) < 1e-12
    assert rel_l2(gpi, st.pi) < 1e-12


def test_rk_graph_equals_plain(cl):
    a = run_pair(cl, 16, 1, 1, cl.CL_INT_RK3_3, O.RK3_3, 11, graph=1)
    b = run_pair(cl, 16, 1, 1, cl.CL_INT_RK3_3, O.RK3_3, 11, graph=0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_rk_without_expansion(cl):
    gphi, gpi, e, st, eo, _ = run_pair(cl, 12, 1, 0, cl.CL_INT_RK4_5, O.RK4_5, 20, expansion=False)
    assert rel_l2(gphi, st.phi) < 1e-12
    assert e["a"] == 1.0


def run_nmc(cl, N, prec, integ, scheme, nsteps, xi, alpha, dt=0.01, pot=(0.6, 1.0), seed=37, adot=0.3, fbar=0.9,
            amp=0.05, opts=(), effective=None, energies_first=True):
    L = 0.8 * N
    phi, pi = inputs.scalar_state(N, 1, seed=seed, fbar=(fbar,), amp=amp, pamp=amp)
    m = O.make_model(N, L, nf=1, alpha=alpha, kappa=0.6, expansion=True, m2=(pot[0], 0.0), lam=(pot[1], 0.0),
                     xi=xi)
    st = O.State(phi.copy(), pi.copy(), np.array([1.0, adot, 0.0]))
    dtype = np.float64 if prec == 0 else np.float32
    with cl.Lattice(N, L, 1, prec, integ, expansion=True, alpha=alpha, kappa=0.6, dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [pot[0], pot[1], 0.0, 0.0, 0.0])
        g.cl_set_nonminimal(xi)
        for opt, val in opts:
            g.cl_set_option(opt, val)
        if effective is not None:
            effective["stages"] = g.cl_get_option(cl.CL_OPT_STAGES)
        g.cl_set_state(cl.CL_FIELD_PHI0, st.phi[0].astype(dtype))
        g.cl_set_state(cl.CL_FIELD_PI0, st.pi[0].astype(dtype))
        g.cl_set_scalars(st.abt[0], st.abt[1], 0.0)
        e0 = g.cl_energies() if energies_first else None
        r0 = O.nmc_ricci(m, st)
        g.cl_step(nsteps)
        launches = g.cl_last_launch_count()
        gphi, gpi = g.cl_get_state(cl.CL_FIELD_PHI0), g.cl_get_state(cl.CL_FIELD_PI0)
        e = g.cl_energies()
    O.step(m, st, scheme, dt, nsteps)
    return gphi, gpi, e0, r0, e, st, m, launches


@pytest.mark.parametrize("integ,scheme,stages", [(2, O.RK3_3, 3), (3, O.RK4_5, 5)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4), (2, 1e-4)])
@pytest.mark.parametrize("xi,alpha", [(0.25, 1.0), (-0.4, 0.0)])
def test_nmc_parity(cl, integ, scheme, stages, prec, tol, xi, alpha):
    """Non-minimally coupled field (cl_set_nonminimal): fields, a, a' and the background
    Ricci scalar against the oracle; two launches per stage (Ricci reduction + stage)."""
    N, n = 12, 20
    eff = {}
    gphi, gpi, e0, r0, e, st, m, launches = run_nmc(cl, N, prec, integ, scheme, n, xi, alpha, effective=eff)
    assert rel_l2(gphi, st.phi[0]) < tol
    assert rel_l2(gpi, st.pi[0]) < tol
    assert e["a"] == pytest.approx(st.abt[0], rel=tol)
    assert e["adot"] == pytest.approx(st.abt[1], rel=max(tol, 1e-9))
    assert e0["ricci"] == pytest.approx(r0, rel=max(tol, 1e-9))
    assert e["ricci"] == pytest.approx(O.nmc_ricci(m, st), rel=max(tol, 1e-9))
    # TMA-staged stages carry the Ricci scalar of their output (the energies computed it for
    # the initial state); the direct-load kernel needs a reduction launch per stage
    assert launches == (n * stages if eff["stages"] > 0 else 2 * n * stages)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (2, 1e-5)])
@pytest.mark.parametrize("N", [32, 48])
def test_nmc_fused_ricci_matches_separate_reduction(cl, prec, tol, N):
    """The Ricci scalar summed by the stage kernel for its output state (the default with the
    TMA-staged kernel) against a reduction launch before every stage (CL_OPT_STAGES -1), with
    no energies before the first step (so the first step starts with one reduction launch)."""
    res = []
    for opts in ((), ((cl.CL_OPT_STAGES, -1),)):
        eff = {}
        gphi, gpi, e0, r0, e, st, m, launches = run_nmc(cl, N, prec, cl.CL_INT_RK4_5, O.RK4_5, 6, 0.3, 1.0,
                                                        opts=opts, effective=eff, energies_first=False)
        res.append((gphi, gpi, e, launches, eff["stages"]))
    (fa, pa, ea, la, sa), (fb, pb, eb, lb, sb) = res
    assert sa > 0 and sb == -1
    assert la == 6 * 5 + 1 and lb == 2 * 6 * 5
    assert rel_l2(fa, fb) < tol and rel_l2(pa, pb) < tol
    for k in ("ricci", "a", "adot", "rho"):
        assert ea[k] == pytest.approx(eb[k], rel=max(tol, 1e-12)), k


def test_nmc_conformal_quartic_keeps_a_linear(cl):
    """xi = 1/6 with a massless quartic potential: R = 0 and, in conformal time, a'' = 0."""
    gphi, gpi, e0, r0, e, st, m, _ = run_nmc(cl, 16, 0, cl.CL_INT_RK4_5, O.RK4_5, 30, 1.0 / 6.0, 1.0, pot=(0.0, 1.0),
                                             adot=0.3, fbar=1.2, amp=0.2)
    assert abs(e["ricci"]) < 1e-13 and abs(e0["ricci"]) < 1e-13
    assert e["a"] == pytest.approx(1.0 + 0.3 * 0.01 * 30, rel=1e-13)
    assert e["adot"] == pytest.approx(0.3, rel=1e-13)


def test_nmc_needs_one_field_and_runge_kutta(cl):
    with cl.Lattice(8, 6.0, 1, 0, cl.CL_INT_VV2) as g:
        with pytest.raises(cl.CLError):
            g.cl_set_nonminimal(0.1)
    with cl.Lattice(8, 6.0, 2, 0, cl.CL_INT_RK3_3) as g:
        with pytest.raises(cl.CLError):
            g.cl_set_nonminimal(0.1)
    with cl.Lattice(8, 6.0, 1, 0, cl.CL_INT_RK3_3) as g:
        with pytest.raises(cl.CLError):
            g.cl_set_nonminimal(float("nan"))


@pytest.mark.parametrize("N,nf,stages_opt", [(16, 2, 0), (32, 1, 0), (32, 2, -1), (15, 1, 0)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_rk34_adaptive_matches_oracle(cl, N, nf, stages_opt, prec, tol):
    """Adaptive RK3-4 (cl_set_adaptive): every step is taken and its last stage sets the next
    step size on the device from the embedded estimate |y_4 - y_3| / |y_4|.  The GPU's step
    sizes, estimates, fields and scale factor follow the oracle's adaptive driver step by step
    (the TMA-staged stage kernel, the direct-load one with CL_OPT_STAGES -1, and odd N)."""
    L, tol_rk, nsteps = 0.8 * N, 1e-5, 12
    pot = [0.6, 1.0, 0.3 if nf == 2 else 0.0, 0.0, 2.5 if nf == 2 else 0.0]
    phi, pi = inputs.scalar_state(N, nf, seed=41, fbar=(0.9, 0.1), amp=0.05, pamp=0.05)
    m = O.make_model(N, L, nf=nf, alpha=0.5, kappa=0.4, expansion=True, m2=(pot[0], pot[2]), lam=(pot[1], pot[3]),
                     g2=pot[4])
    st = O.State(phi.copy(), pi.copy(), np.array([1.0, 0.0, 0.0]))
    st.abt[1] = math.sqrt(0.4 * O.energies(m, st)["rho"] / 3.0)
    dtype = np.float64 if prec == 0 else np.float32
    with cl.Lattice(N, L, nf, prec, cl.CL_INT_RK3_4, expansion=True, alpha=0.5, kappa=0.4, dt=0.02) as g:
        g.cl_set_potential(cl.CL_POT_POLY, pot)
        if stages_opt:
            g.cl_set_option(cl.CL_OPT_STAGES, stages_opt)
        for f in range(nf):
            g.cl_set_state(cl.CL_FIELD_PHI0 + f, st.phi[f].astype(dtype))
            g.cl_set_state(cl.CL_FIELD_PI0 + f, st.pi[f].astype(dtype))
        g.cl_set_scalars(st.abt[0], st.abt[1], 0.0)
        g.cl_set_adaptive(tol_rk, 1e-4, 0.05)
        assert g.cl_energies()["dt"] == 0.02
        h = 0.02
        ts = []
        for k in range(nsteps):
            g.cl_step(1)
            e = g.cl_energies()
            h_next, hu, ep = O.step_adaptive(m, st, h, tol_rk, 1, hmin=1e-4, hmax=0.05)
            # the estimate is a norm of small increments: in FP32 it carries ~1e-4 of rounding,
            # of which the next step size takes a third (h ~ eps^(-1/3))
            assert e["rk_error"] == pytest.approx(ep[0], rel=1e-8 if prec == 0 else 1e-3), k
            assert e["dt"] == pytest.approx(h_next, rel=max(tol, 1e-8)), k
            assert e["t"] == pytest.approx(st.abt[2], rel=1e-8 if prec == 0 else tol)  # t sums the h taken
            h = h_next
            ts.append(h)
        gphi = np.stack([g.cl_get_state(cl.CL_FIELD_PHI0 + f) for f in range(nf)])
        gpi = np.stack([g.cl_get_state(cl.CL_FIELD_PI0 + f) for f in range(nf)])
        e = g.cl_energies()
        assert e["step"] == nsteps
    assert len(set(np.round(ts, 12))) > 3  # the step size really changes
    assert rel_l2(gphi, st.phi) < tol and rel_l2(gpi, st.pi) < tol
    assert e["a"] == pytest.approx(st.abt[0], rel=tol)


def test_rk34_adaptive_graph_replay_and_switch_off(cl):
    """Adaptive steps replay from the captured graph (cl_step(n) in one call equals n calls),
    and cl_set_adaptive(0) returns to the fixed dt."""
    N = 16
    phi, pi = inputs.scalar_state(N, 1, seed=43, fbar=(0.9,), amp=0.05, pamp=0.05)
    res = []
    for chunks in ((8,), (1,) * 8):
        with cl.Lattice(N, 12.0, 1, cl.CL_PREC_FP64, cl.CL_INT_RK3_4, expansion=True, alpha=1.0, kappa=0.3,
                        dt=0.01) as g:
            g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
            g.cl_set_state(cl.CL_FIELD_PHI0, phi[0])
            g.cl_set_state(cl.CL_FIELD_PI0, pi[0])
            g.cl_set_scalars(1.0)
            g.cl_set_adaptive(1e-6, 0.0, 1.0)
            for c in chunks:
                g.cl_step(c)
            e = g.cl_energies()
            res.append((g.cl_get_state(cl.CL_FIELD_PHI0), e["dt"], e["t"]))
            g.cl_set_adaptive(0.0)
            g.cl_step(2)
            e2 = g.cl_energies()
            assert e2["dt"] == 0.01 and e2["t"] == pytest.approx(e["t"] + 0.02, rel=1e-12)
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1] and res[0][2] == res[1][2]


def test_rk34_adaptive_rejects_unsupported(cl):
    with cl.Lattice(8, 6.0, 1, cl.CL_PREC_FP64, cl.CL_INT_RK3_3, dt=0.01) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
        with pytest.raises(cl.CLError) as ei:
            g.cl_set_adaptive(1e-6)
        assert ei.value.status == cl.CL_EUNSUPPORTED
    with cl.Lattice(8, 6.0, 1, cl.CL_PREC_FP64, cl.CL_INT_RK3_4, dt=0.01) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
        with pytest.raises(cl.CLError) as ei:
            g.cl_set_adaptive(1e-6, 0.5, 0.1)
        assert ei.value.status == cl.CL_EINVAL
