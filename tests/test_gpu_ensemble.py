"""GPU parity of the batched ensemble (many independent lattices in one launch per pass)
against independent oracle runs of every member.

Each member has its own size, box, couplings, scale factor and initial state; the
ensemble must advance each exactly as a lone lattice would.  Tolerances as for the single
lattice: 1e-10 relative L2 in FP64, 1e-4 in FP32 (+ Kahan).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs

pytestmark = pytest.mark.gpu

ALPHA, KAPPA = 1.0, 0.3


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


def member_params(sizes, nf, seed=7):
    """Per-member box, couplings (POLY order), scale factor and initial state."""
    g = inputs.rng(seed)
    out = []
    for m, N in enumerate(sizes):
        L = float(0.6 * N * (1.0 + 0.5 * g.random()))
        lam0 = float(10 ** g.uniform(-1.0, 0.5))
        m20 = float(g.uniform(0.0, 1.0))
        pot = [m20, lam0, 0.0, 0.0, 0.0]
        if nf == 2:
            pot[2], pot[3], pot[4] = float(g.uniform(0.1, 1.0)), 0.0, float(g.uniform(0.5, 3.0))
        phi, pi = inputs.scalar_state(N, nf, seed=seed * 100 + m, fbar=(0.9, 0.1), amp=0.05, pamp=0.05)
        a0 = float(1.0 + 0.5 * g.random())
        out.append(dict(N=N, L=L, pot=pot, phi=phi, pi=pi, a0=a0))
    return out


def oracle_member(P, nf, scheme, dt, nsteps, expansion=True):
    m = O.make_model(P["N"], P["L"], nf=nf, alpha=ALPHA, kappa=KAPPA, expansion=expansion,
                     m2=(P["pot"][0], P["pot"][2]), lam=(P["pot"][1], P["pot"][3]), g2=P["pot"][4])
    st = O.State(P["phi"].copy(), P["pi"].copy(), np.array([P["a0"], 0.0, 0.0]))
    if expansion:  # a' from Eq. Friedmann2 at the initial state
        rho = O.energies(m, st)["rho"]
        st.abt[1] = P["a0"] * math.sqrt(P["a0"] ** (2 * ALPHA) * KAPPA * rho / 3.0)
    O.step(m, st, scheme, dt, nsteps)
    return m, st


def run_ensemble(cl, params, nf, prec, integ, dt, nsteps, graph=1, expansion=True, opts=()):
    sizes = [P["N"] for P in params]
    with cl.Lattice(sizes[0], 1.0, nf, prec, integ, expansion=expansion, alpha=ALPHA, kappa=KAPPA, dt=dt,
                    member_N=sizes, member_L=[P["L"] for P in params]) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [x for P in params for x in P["pot"]])
        g.cl_set_option(cl.CL_OPT_GRAPH, graph)
        for k, v in opts:
            g.cl_set_option(k, v)
        for m, P in enumerate(params):
            for f in range(nf):
                g.cl_set_state(cl.CL_FIELD_PHI0 + f, P["phi"][f].astype(g.dtype), member=m)
                g.cl_set_state(cl.CL_FIELD_PI0 + f, P["pi"][f].astype(g.dtype), member=m)
            g.cl_set_scalars(P["a0"], math.nan if expansion else 0.0, 0.0, member=m)
        g.cl_step(nsteps)
        launches = g.cl_last_launch_count()
        phis = [np.stack([g.cl_get_state(cl.CL_FIELD_PHI0 + f, member=m) for f in range(nf)])
                for m in range(len(params))]
        pis = [np.stack([g.cl_get_state(cl.CL_FIELD_PI0 + f, member=m) for f in range(nf)])
               for m in range(len(params))]
        es = g.cl_energies(len(params))
    return phis, pis, es, launches


SCHEMES = {0: O.VV2, 1: O.YOSHIDA4}


@pytest.mark.parametrize("integ", [0, 1])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4), (2, 1e-4)])
@pytest.mark.parametrize("nf", [1, 2])
def test_ensemble_parity(cl, integ, prec, tol, nf):
    sizes = [8, 12, 16, 8, 20, 12]
    params = member_params(sizes, nf)
    nsteps, dt = 25, 0.02
    phis, pis, es, launches = run_ensemble(cl, params, nf, prec, integ, dt, nsteps)
    for m, P in enumerate(params):
        model, st = oracle_member(P, nf, SCHEMES[integ], dt, nsteps)
        assert rel_l2(phis[m], st.phi) < tol, m
        assert rel_l2(pis[m], st.pi) < tol, m
        eo = O.energies(model, st)
        assert es[m]["a"] == pytest.approx(st.abt[0], rel=tol)
        assert es[m]["adot"] == pytest.approx(st.abt[1], rel=max(tol, 1e-9))
        assert es[m]["t"] == pytest.approx(st.abt[2], rel=1e-12)
        assert es[m]["rho"] == pytest.approx(eo["rho"], rel=max(tol, 1e-9))
        assert es[m]["step"] == nsteps
    passes = 1 if integ == 0 else 3
    assert launches == 1 + nsteps * passes  # opening half-kick, then one launch per pass for all members


@pytest.mark.parametrize("sizes", [[7, 5, 9], [6, 10, 14, 2], [32, 48, 64]])
def test_ensemble_ragged_sizes(cl, sizes):
    """Odd sizes force scalar vectors; N = 2 is the smallest lattice; 32/48/64 are the sizes
    of the production ensemble (several work items per member)."""
    params = member_params(sizes, 1, seed=11)
    nsteps = 6 if max(sizes) > 20 else 15
    phis, pis, es, _ = run_ensemble(cl, params, 1, 0, 0, 0.02, nsteps)
    for m, P in enumerate(params):
        _, st = oracle_member(P, 1, O.VV2, 0.02, nsteps)
        assert rel_l2(phis[m], st.phi) < 1e-11, m
        assert rel_l2(pis[m], st.pi) < 1e-11, m


def test_ensemble_tile_options_do_not_change_results(cl):
    """Different work-item shapes reorder only the FP64 reductions of a and a'."""
    sizes = [16, 24, 12]
    params = member_params(sizes, 1, seed=3)
    a = run_ensemble(cl, params, 1, 0, 1, 0.02, 10)
    b = run_ensemble(cl, params, 1, 0, 1, 0.02, 10, opts=((cl.CL_OPT_TILE_BY, 3), (cl.CL_OPT_TILE_DZ, 5)))
    for m in range(len(sizes)):
        assert rel_l2(a[0][m], b[0][m]) < 1e-13
        assert rel_l2(a[1][m], b[1][m]) < 1e-13
        assert a[2][m]["a"] == pytest.approx(b[2][m]["a"], rel=1e-14)


def test_ensemble_graph_equals_plain(cl):
    params = member_params([8, 16, 12], 2, seed=5)
    a = run_ensemble(cl, params, 2, 1, 1, 0.02, 9, graph=1)
    b = run_ensemble(cl, params, 2, 1, 1, 0.02, 9, graph=0)
    for m in range(3):
        assert np.array_equal(a[0][m], b[0][m])
        assert np.array_equal(a[1][m], b[1][m])
        assert a[2][m]["a"] == b[2][m]["a"]


def test_ensemble_members_are_independent(cl):
    """Changing one member's state changes no other member's result."""
    params = member_params([8, 12, 10], 1, seed=9)
    a = run_ensemble(cl, params, 1, 0, 0, 0.02, 12)
    params[1]["phi"] = params[1]["phi"] * 1.1
    b = run_ensemble(cl, params, 1, 0, 0, 0.02, 12)
    for m in (0, 2):
        assert np.array_equal(a[0][m], b[0][m])
        assert a[2][m]["rho"] == b[2][m]["rho"]
    assert not np.array_equal(a[0][1], b[0][1])


def test_ensemble_frozen_background(cl):
    params = member_params([8, 12], 1, seed=13)
    phis, pis, es, _ = run_ensemble(cl, params, 1, 0, 0, 0.02, 10, expansion=False)
    for m, P in enumerate(params):
        _, st = oracle_member(P, 1, O.VV2, 0.02, 10, expansion=False)
        assert rel_l2(phis[m], st.phi) < 1e-11
        assert es[m]["a"] == P["a0"]


def test_ensemble_vacuum_members_follow_their_philox_streams(cl):
    """cl_init_vacuum(member = -1) seeds member m with counter (mode, field, m, 0), as the
    oracle's vacuum generator does for that member."""
    sizes = [8, 12, 10]
    Ls = [6.0, 9.0, 7.0]
    lam = 0.7
    with cl.Lattice(8, 1.0, 1, cl.CL_PREC_FP64, cl.CL_INT_VV2, alpha=ALPHA, kappa=KAPPA, dt=0.01,
                    member_N=sizes, member_L=Ls) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [lam])
        g.cl_init_vacuum(99, 1e9, 1e-3, (1.0,), (0.0,))
        got = [g.cl_get_state(cl.CL_FIELD_PHI0, member=m) for m in range(3)]
        gpi = [g.cl_get_state(cl.CL_FIELD_PI0, member=m) for m in range(3)]
        es = g.cl_energies(3)
    for m in range(3):
        model = O.make_model(sizes[m], Ls[m], nf=1, alpha=ALPHA, kappa=KAPPA, expansion=True, lam=(lam, 0.0))
        st = O.vacuum(model, 99, 1e9, 1e-3, (1.0,), (0.0,), member=m)
        assert rel_l2(got[m] - 1.0, st.phi[0] - 1.0) < 1e-10
        assert rel_l2(gpi[m], st.pi[0]) < 1e-10
        assert es[m]["adot"] == pytest.approx(st.abt[1], rel=1e-10)


def test_ensemble_per_member_calls(cl):
    params = member_params([8, 12], 1, seed=17)
    with cl.Lattice(8, 1.0, 1, cl.CL_PREC_FP64, cl.CL_INT_VV2, alpha=ALPHA, kappa=KAPPA, dt=0.01,
                    member_N=[8, 12]) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [0.5])
        g.cl_set_scalars(1.5, 0.25, 2.0, member=1)
        assert g.cl_get_scalars(1) == (1.5, 0.25, 2.0)
        assert g.cl_get_scalars(0)[0] == 1.0
        with pytest.raises(cl.CLError):
            g.cl_set_state(cl.CL_FIELD_PHI0, np.zeros(8 ** 3), member=2)
        with pytest.raises(cl.CLError):
            g.cl_set_state(cl.CL_FIELD_PHI0, np.zeros(8 ** 3), member=-1)
        with pytest.raises(ValueError):
            g.cl_set_state(cl.CL_FIELD_PHI0, np.zeros(8 ** 3), member=1)  # member 1 holds 12^3
        with pytest.raises(cl.CLError):
            g.cl_set_potential(cl.CL_POT_LPHI4, [0.5, 0.6, 0.7])  # neither shared nor one per member
        g.cl_set_potential(cl.CL_POT_LPHI4, [0.5, 0.6])
        k, d, c = g.cl_spectrum(cl.CL_FIELD_PHI0, member=1)
        assert len(k) == int(math.floor(math.sqrt(3.0) * 6 + 0.5)) + 1
        with pytest.raises(cl.CLError):
            g.cl_set_option(cl.CL_OPT_STAGES, 7)  # at most 6 TMA stages
    with pytest.raises(cl.CLError):
        cl.Lattice(8, 1.0, 1, cl.CL_PREC_FP64, cl.CL_INT_RK3_3, member_N=[8, 8])
    with pytest.raises(cl.CLError):
        cl.Lattice(8, 1.0, 1, cl.CL_PREC_FP64, cl.CL_INT_VV2, member_N=[8, 1024])


@pytest.mark.parametrize("prec", [0, 1])
def test_ensemble_tma_and_direct_loaders_agree(cl, prec):
    """The TMA-staged ensemble kernel (16-byte rows) and the direct loader do the same
    per-site arithmetic on the same work items."""
    params = member_params([16, 24, 12, 32], 1, seed=23)
    a = run_ensemble(cl, params, 1, prec, 1, 0.02, 8)
    b = run_ensemble(cl, params, 1, prec, 1, 0.02, 8, opts=((cl.CL_OPT_STAGES, -1),))
    c = run_ensemble(cl, params, 1, prec, 1, 0.02, 8, opts=((cl.CL_OPT_STAGES, 2),))
    for m in range(4):
        for other in (b, c):
            assert rel_l2(a[0][m], other[0][m]) < 1e-14
            assert rel_l2(a[1][m], other[1][m]) < 1e-14
            assert a[2][m]["rho"] == pytest.approx(other[2][m]["rho"], rel=1e-13)


@pytest.mark.parametrize("prec,nf", [(1, 1), (1, 2), (0, 1), (2, 2)])
def test_ensemble_ringless_and_ring_kernels_identical(cl, prec, nf):
    """The ringless TMA ensemble kernel re-drifts the y-neighbour rows from the stage instead
    of sharing them through a ring: on the same items the fields, energies and scale factors
    agree bit for bit with the ring kernel, for every stage count."""
    params = member_params([16, 24, 12, 32, 8], nf, seed=41)
    ref = run_ensemble(cl, params, nf, prec, 1, 0.02, 6,
                       opts=((cl.CL_OPT_PASS_VARIANT, 0), (cl.CL_OPT_STAGES, 3)))
    for stages in (3, 4, 6):
        got = run_ensemble(cl, params, nf, prec, 1, 0.02, 6,
                           opts=((cl.CL_OPT_PASS_VARIANT, 1), (cl.CL_OPT_STAGES, stages)))
        for m in range(len(params)):
            assert np.array_equal(got[0][m], ref[0][m]), (stages, m)
            assert np.array_equal(got[1][m], ref[1][m]), (stages, m)
            assert got[2][m]["rho"] == ref[2][m]["rho"]
            assert got[2][m]["a"] == ref[2][m]["a"]


def test_autotune_keeps_the_state_and_caches_its_choice(cl, tmp_path):
    sizes = [16, 24, 32, 16]
    params = member_params(sizes, 1, seed=29)
    cache = str(tmp_path / "tune.jsonl")
    with cl.Lattice(16, 1.0, 1, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_VV2, alpha=ALPHA, kappa=KAPPA, dt=0.02,
                    member_N=sizes, member_L=[P["L"] for P in params]) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [x for P in params for x in P["pot"]])
        for m, P in enumerate(params):
            g.cl_set_state(cl.CL_FIELD_PHI0, P["phi"][0].astype(np.float32), member=m)
            g.cl_set_state(cl.CL_FIELD_PI0, P["pi"][0].astype(np.float32), member=m)
            g.cl_set_scalars(P["a0"], math.nan, 0.0, member=m)
        g.cl_step(3)
        before = [(g.cl_get_state(cl.CL_FIELD_PHI0, member=m), g.cl_get_state(cl.CL_FIELD_PI0, member=m),
                   g.cl_get_scalars(m)) for m in range(4)]
        stages, by, dz, us, variant = g.cl_autotune(cache)
        # the tiling in effect, as cl_get_option reports it (0: the loader without TMA staging)
        assert us > 0 and stages in (0, 2, 3, 4, 5, 6) and variant in (0, 1)
        assert (stages, by, dz, variant) == tuple(g.cl_get_option(o) for o in (
            cl.CL_OPT_STAGES, cl.CL_OPT_TILE_BY, cl.CL_OPT_TILE_DZ, cl.CL_OPT_PASS_VARIANT))
        for m in range(4):
            assert np.array_equal(g.cl_get_state(cl.CL_FIELD_PHI0, member=m), before[m][0])
            assert np.array_equal(g.cl_get_state(cl.CL_FIELD_PI0, member=m), before[m][1])
            # a' at the integer time is re-synchronised through a pass whose FP64 reduction order
            # depends on the tiling: equal to rounding
            assert g.cl_get_scalars(m) == pytest.approx(before[m][2], rel=1e-12)
        again = g.cl_autotune(cache)  # cache hit: the same choice without trials
        assert again == (stages, by, dz, pytest.approx(us, rel=1e-3), variant)
        g.cl_step(4)
        phis = [g.cl_get_state(cl.CL_FIELD_PHI0, member=m) for m in range(4)]
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and '"key": "ensemble B=4' in lines[0]
    # the tuned run follows the same trajectory as the default tiling
    ref = run_ensemble(cl, params, 1, 1, 0, 0.02, 7)
    for m in range(4):
        assert rel_l2(phis[m], ref[0][m][0]) < 1e-6


def test_autotune_single_lattice(cl):
    N = 64
    phi, pi = inputs.scalar_state(N, 2, seed=31, fbar=(1.0, 0.0), amp=1e-3, pamp=1e-3)
    with cl.Lattice(N, 20.0, 2, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_YOSHIDA4, alpha=0.0, kappa=0.1, dt=0.005) as g:
        g.cl_set_potential(cl.CL_POT_M2_G2, [1.0, 100.0])
        for f in range(2):
            g.cl_set_state(cl.CL_FIELD_PHI0 + f, phi[f].astype(np.float32))
            g.cl_set_state(cl.CL_FIELD_PI0 + f, pi[f].astype(np.float32))
        g.cl_set_scalars(1.0)
        e0 = g.cl_energies()
        stages, by, dz, us, variant = g.cl_autotune()
        assert us > 0 and variant in (0, 1)
        assert variant == 0 or 2 <= stages <= 5
        assert (stages, by, dz, variant) == tuple(g.cl_get_option(o) for o in (
            cl.CL_OPT_STAGES, cl.CL_OPT_TILE_BY, cl.CL_OPT_TILE_DZ, cl.CL_OPT_PASS_VARIANT))
        # the energies of the unchanged state, summed over another tiling (per-thread FP32 sums
        # of other sites): equal to their rounding
        assert g.cl_energies()["rho"] == pytest.approx(e0["rho"], rel=1e-9)
        assert np.array_equal(g.cl_get_state(cl.CL_FIELD_PHI1), phi[1].astype(np.float32))
    with cl.Lattice(8, 6.0, 1, cl.CL_PREC_FP64, cl.CL_INT_RK3_3) as g:
        g.cl_set_potential(cl.CL_POT_M2, [1.0])
        with pytest.raises(cl.CLError):
            g.cl_autotune()
