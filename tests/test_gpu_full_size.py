"""Parity at the benchmark workloads' full sizes, in the launch configurations bench.py times.

The oracle cannot step 192^3 or 256^3 lattices in seconds, so these tests use a property that
holds at any size: the equations are translation invariant, so a state that repeats with
period P in every direction stays periodic, and the full-size lattice evolves exactly as the
P-periodic lattice does, tiled.  The GPU runs the full-size lattice (every tile, z chunk, stage
buffer and reduction of the benchmark's launch configuration) from a P-periodic random state;
the oracle runs the small lattice; the fields must agree everywhere and the volume averages
(which the tiling leaves unchanged) must agree.  The ensemble is checked member by member on a
sample of the 1024 members, each against its own oracle run.
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


def tile3(a, reps):
    return np.tile(a, (reps, reps, reps))


# the axion-U(1) workload of bench.py --workload u1 / u1lf (192^3, FP32), with a state that
# repeats every 16 sites; couplings and spacing as the benchmark's
U1N, U1P = 192, 16
U1 = dict(L=2 * math.pi / 0.1, dt=0.01, alphaL=30.0, ws2=1e-4, kappa=1.0, alpha=0.0, m2=1.0)


@pytest.mark.parametrize("integ,scheme", [("rk33", O.RK3_3), ("leapfrog", O.VV2)])
def test_u1_192_cubed(cl, integ, scheme):
    c = U1
    Ls = c["L"] * U1P / U1N  # the small lattice with the same spacing
    m = O.make_model(U1P, Ls, nf=1, alpha=c["alpha"], kappa=c["kappa"], expansion=True, gauge=1, alphaL=c["alphaL"],
                     ws2=c["ws2"], m2=(c["m2"], 0.0))
    g0 = inputs.rng(71)
    st = O.new_state(m)
    st.phi[:] = 1.0 + 0.05 * g0.standard_normal(st.phi.shape)
    st.pi[:] = -0.5 + 0.05 * g0.standard_normal(st.pi.shape)
    st.links, st.efield = inputs.gauge_state(U1P, seed=72, theta_amp=0.3, e_amp=0.05)
    # FP32 inputs, as the GPU holds them
    for arr in (st.phi, st.pi, st.links, st.efield):
        arr[:] = arr.astype(np.float32)
    st.abt[:] = (1.0, math.sqrt(c["kappa"] * O.energies(m, st)["rho"] / 3.0), 0.0)
    n = 3
    with cl.Lattice(U1N, c["L"], 1, cl.CL_PREC_FP32, cl.CL_INT_RK3_3 if integ == "rk33" else cl.CL_INT_VV2,
                    gauge=cl.CL_GAUGE_U1_AXION, expansion=True, alpha=c["alpha"], kappa=c["kappa"], dt=c["dt"]) as g:
        g.cl_set_potential(cl.CL_POT_M2, [c["m2"]])
        g.cl_set_gauge_coupling(c["alphaL"], c["ws2"])
        assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == 2  # the staged launches bench.py times
        reps = U1N // U1P
        g.cl_set_state(cl.CL_FIELD_PHI0, tile3(st.phi[0], reps).astype(np.float32))
        g.cl_set_state(cl.CL_FIELD_PI0, tile3(st.pi[0], reps).astype(np.float32))
        for i in range(3):
            g.cl_set_state(cl.CL_FIELD_THETA1 + i, tile3(st.links[i], reps).astype(np.float32))
            g.cl_set_state(cl.CL_FIELD_E1 + i, tile3(st.efield[i], reps).astype(np.float32))
        g.cl_set_scalars(st.abt[0], st.abt[1], 0.0)
        g.cl_step(n)
        out = {"phi": g.cl_get_state(cl.CL_FIELD_PHI0),
               "pi": g.cl_get_state(cl.CL_FIELD_PI0),
               "th": np.stack([g.cl_get_state(cl.CL_FIELD_THETA1 + i) for i in range(3)]),
               "E": np.stack([g.cl_get_state(cl.CL_FIELD_E1 + i) for i in range(3)])}
        e = g.cl_energies()
    O.step(m, st, scheme, c["dt"], n)
    reps = U1N // U1P
    assert rel_l2(out["phi"], tile3(st.phi[0], reps)) < 1e-4
    assert rel_l2(out["pi"], tile3(st.pi[0], reps)) < 1e-4
    for i in range(3):
        assert rel_l2(out["th"][i], tile3(st.links[i], reps)) < 1e-4
        assert rel_l2(out["E"][i], tile3(st.efield[i], reps)) < 1e-4
    eo = O.energies(m, st)
    for k_gpu, k_orc in [("KE", "KEM"), ("GB", "GEM"), ("rho", "rho"), ("V", "V"), ("K0", "K0")]:
        assert e[k_gpu] == pytest.approx(eo[k_orc], rel=1e-4), k_gpu
    assert e["a"] == pytest.approx(st.abt[0], rel=1e-6)


def test_gw_256_cubed(cl):
    """bench.py --workload gw: the headline's two fields at 256^3, Yoshida-4, FP32 + Kahan,
    with the five GW auxiliaries; state periodic with period 16."""
    N, P, L, dt = 256, 16, 8.0 * math.pi, 0.005
    Ls = L * P / N
    m = O.make_model(P, Ls, nf=2, alpha=0.0, kappa=0.1, expansion=True, m2=(1.0, 0.0), g2=4e4)
    phi, pi = inputs.scalar_state(P, 2, seed=81, fbar=(1.0, 0.0), amp=1e-3, pamp=1e-3)
    rg = inputs.rng(82)
    gv = (1e-4 * rg.standard_normal((5, P, P, P))).astype(np.float32).astype(np.float64)
    gp = (1e-4 * rg.standard_normal((5, P, P, P))).astype(np.float32).astype(np.float64)
    st = O.State(phi.astype(np.float32).astype(np.float64), pi.astype(np.float32).astype(np.float64),
                 np.array([1.0, 0.0, 0.0]))
    st.abt[1] = math.sqrt(0.1 * O.energies(m, st)["rho"] / 3.0)
    reps = N // P
    n = 2
    with cl.Lattice(N, L, 2, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_YOSHIDA4, expansion=True, alpha=0.0, kappa=0.1,
                    dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_M2_G2, [1.0, 4e4])
        for f in range(2):
            g.cl_set_state(cl.CL_FIELD_PHI0 + f, tile3(st.phi[f], reps).astype(np.float32))
            g.cl_set_state(cl.CL_FIELD_PI0 + f, tile3(st.pi[f], reps).astype(np.float32))
        g.cl_set_scalars(st.abt[0], st.abt[1], 0.0)
        g.cl_enable_gw()
        for c in range(5):
            g.cl_set_state(cl.CL_FIELD_GW_V11 + c, tile3(gv[c], reps).astype(np.float32))
            g.cl_set_state(cl.CL_FIELD_GW_P11 + c, tile3(gp[c], reps).astype(np.float32))
        g.cl_step(n)
        v = [g.cl_get_state(cl.CL_FIELD_GW_V11 + c) for c in range(5)]
        p = [g.cl_get_state(cl.CL_FIELD_GW_P11 + c) for c in range(5)]
        phi0 = g.cl_get_state(cl.CL_FIELD_PHI0)
        e = g.cl_energies()
    O.step_gw(m, st, gv, gp, O.YOSHIDA4, dt, n)
    assert rel_l2(phi0, tile3(st.phi[0], reps)) < 1e-6
    for c in range(5):
        assert rel_l2(v[c], tile3(gv[c], reps)) < 1e-4, c
        assert rel_l2(p[c], tile3(gp[c], reps)) < 1e-4, c
    assert e["rho"] == pytest.approx(O.energies(m, st)["rho"], rel=1e-5)


def test_reduced_4096_squared(cl):
    """bench.py --workload reduced: the (2+1)-dimensional 4096^2 lattice, two fields,
    Yoshida-4, FP32 + Kahan, the row-marching pass with its ragged last chunk of rows;
    state periodic with period 64."""
    N, P, dt = 4096, 64, 0.005
    L = 2048.0 * math.pi
    Ls = L * P / N
    m = O.make_model(P, Ls, nf=2, alpha=0.0, kappa=0.1, expansion=True, m2=(1.0, 0.0), g2=4e4, dims=2)
    rng = np.random.default_rng(91)
    st = O.new_state(m)
    st.phi[:] = (np.array([1.0, 0.0])[:, None, None, None] + 1e-3 * rng.standard_normal(st.phi.shape))
    st.pi[:] = 1e-3 * rng.standard_normal(st.pi.shape)
    st.phi[:] = st.phi.astype(np.float32)
    st.pi[:] = st.pi.astype(np.float32)
    st.abt[:] = (1.0, math.sqrt(0.1 * O.energies(m, st)["rho"] / 3.0), 0.0)
    reps = N // P
    n = 3
    with cl.Lattice(N, L, 2, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_YOSHIDA4, expansion=True, alpha=0.0, kappa=0.1,
                    dt=dt, dims=2) as g:
        g.cl_set_potential(cl.CL_POT_M2_G2, [1.0, 4e4])
        assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == 1
        assert N % g.cl_get_option(cl.CL_OPT_TILE_DZ) != 0  # a ragged last chunk of rows
        for f in range(2):
            g.cl_set_state(cl.CL_FIELD_PHI0 + f, np.tile(st.phi[f], (1, reps, reps)).astype(np.float32))
            g.cl_set_state(cl.CL_FIELD_PI0 + f, np.tile(st.pi[f], (1, reps, reps)).astype(np.float32))
        g.cl_set_scalars(st.abt[0], st.abt[1], 0.0)
        g.cl_step(n)
        gphi = [g.cl_get_state(cl.CL_FIELD_PHI0 + f) for f in range(2)]
        gpi = [g.cl_get_state(cl.CL_FIELD_PI0 + f) for f in range(2)]
        e = g.cl_energies()
    O.step(m, st, O.YOSHIDA4, dt, n)
    for f in range(2):
        assert rel_l2(gphi[f], np.tile(st.phi[f], (1, reps, reps))) < 1e-6
        assert rel_l2(gpi[f], np.tile(st.pi[f], (1, reps, reps))) < 1e-4
    eo = O.energies(m, st)
    assert e["rho"] == pytest.approx(eo["rho"], rel=1e-5)
    assert e["a"] == pytest.approx(st.abt[0], rel=1e-7)


def test_ensemble_1024_members_sampled(cl):
    """bench.py --workload ensemble: 1024 lambda phi^4 lattices of sizes drawn from
    {32, 48, 64}^3 with the benchmark's seeds, vacuum states, autotuned launch; after 4
    steps twelve members (the first, the last and ten drawn) against their own oracle runs
    from the states the library holds."""
    members, sizes_set, L, dt, alpha, kappa, seed = 1024, (32, 48, 64), 8.0 * math.pi, 0.01, 1.0, 0.1, 1234
    rg = np.random.default_rng(seed)
    sizes = [int(x) for x in rg.choice(sizes_set, members)]
    lam = 10.0 ** rg.uniform(math.log10(1e-6), math.log10(1e-3), members)
    sample = sorted({0, members - 1} | set(int(x) for x in np.random.default_rng(5).choice(members, 10, replace=False)))
    n = 4
    with cl.Lattice(sizes[0], L, 1, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_VV2, expansion=True, alpha=alpha, kappa=kappa,
                    dt=dt, member_N=sizes) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
        kcut = 16 * 2 * math.pi / L
        for mm in range(members):
            g.cl_init_vacuum(seed, kcut, float(lam[mm]), (1.0,), (0.0,), member=mm)
        g.cl_autotune()
        start = {}
        for mm in sample:
            e0 = g.cl_energies(members)[mm]
            start[mm] = (g.cl_get_state(cl.CL_FIELD_PHI0, member=mm), g.cl_get_state(cl.CL_FIELD_PI0, member=mm),
                         e0["a"], e0["adot"])
        g.cl_step(n)
        es = g.cl_energies(members)
        end = {mm: (g.cl_get_state(cl.CL_FIELD_PHI0, member=mm), g.cl_get_state(cl.CL_FIELD_PI0, member=mm))
               for mm in sample}
    for mm in sample:
        Nm = sizes[mm]
        model = O.make_model(Nm, L, nf=1, alpha=alpha, kappa=kappa, expansion=True, lam=(1.0, 0.0))
        phi0, pi0, a0, b0 = start[mm]
        st = O.State(phi0.reshape(1, Nm, Nm, Nm).astype(np.float64), pi0.reshape(1, Nm, Nm, Nm).astype(np.float64),
                     np.array([a0, b0, 0.0]))
        O.step(model, st, O.VV2, dt, n)
        assert rel_l2(end[mm][0], st.phi[0]) < 1e-6, mm
        assert rel_l2(end[mm][1], st.pi[0]) < 1e-4, mm
        assert es[mm]["a"] == pytest.approx(st.abt[0], rel=1e-7), mm


def test_headline_512_cubed(cl):
    """The headline model at 512^3 (the roofline size of the two-field workload; two-row
    tiles), Yoshida-4, FP32 + Kahan; state periodic with period 32."""
    N, P, dt = 512, 32, 0.005
    L = 8.0 * math.pi * N / 256  # the headline's spacing
    Ls = L * P / N
    m = O.make_model(P, Ls, nf=2, alpha=0.0, kappa=0.1, expansion=True, m2=(1.0, 0.0), g2=4e4)
    phi, pi = inputs.scalar_state(P, 2, seed=101, fbar=(1.0, 0.0), amp=1e-3, pamp=1e-3)
    st = O.State(phi.astype(np.float32).astype(np.float64), pi.astype(np.float32).astype(np.float64),
                 np.array([1.0, 0.0, 0.0]))
    st.abt[1] = math.sqrt(0.1 * O.energies(m, st)["rho"] / 3.0)
    reps = N // P
    n = 2
    with cl.Lattice(N, L, 2, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_YOSHIDA4, expansion=True, alpha=0.0, kappa=0.1,
                    dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_M2_G2, [1.0, 4e4])
        for f in range(2):
            g.cl_set_state(cl.CL_FIELD_PHI0 + f, tile3(st.phi[f], reps).astype(np.float32))
            g.cl_set_state(cl.CL_FIELD_PI0 + f, tile3(st.pi[f], reps).astype(np.float32))
        g.cl_set_scalars(st.abt[0], st.abt[1], 0.0)
        g.cl_step(n)
        out = [(g.cl_get_state(cl.CL_FIELD_PHI0 + f), g.cl_get_state(cl.CL_FIELD_PI0 + f)) for f in range(2)]
        e = g.cl_energies()
    O.step(m, st, O.YOSHIDA4, dt, n)
    for f in range(2):
        assert rel_l2(out[f][0], tile3(st.phi[f], reps)) < 1e-6
        assert rel_l2(out[f][1], tile3(st.pi[f], reps)) < 1e-4
    assert e["rho"] == pytest.approx(O.energies(m, st)["rho"], rel=1e-5)
    assert e["a"] == pytest.approx(st.abt[0], rel=1e-7)


def test_nonminimal_256_cubed(cl):
    """bench.py --workload nmc: one lambda phi^4 field non-minimally coupled (xi = 0.3) at
    256^3, RK4-5, FP32 + Kahan, the TMA-staged stage that carries the Ricci scalar; state
    periodic with period 16."""
    N, P, dt, xi = 256, 16, 0.005, 0.3
    L = 8.0 * math.pi
    Ls = L * P / N
    m = O.make_model(P, Ls, nf=1, alpha=1.0, kappa=0.1, expansion=True, lam=(1.0, 0.0), xi=xi)
    phi, pi = inputs.scalar_state(P, 1, seed=111, fbar=(1.0,), amp=1e-2, pamp=1e-2)
    st = O.State(phi.astype(np.float32).astype(np.float64), pi.astype(np.float32).astype(np.float64),
                 np.array([1.0, 0.0, 0.0]))
    reps = N // P
    n = 3
    with cl.Lattice(N, L, 1, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_RK4_5, expansion=True, alpha=1.0, kappa=0.1,
                    dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
        g.cl_set_nonminimal(xi)
        g.cl_set_state(cl.CL_FIELD_PHI0, tile3(st.phi[0], reps).astype(np.float32))
        g.cl_set_state(cl.CL_FIELD_PI0, tile3(st.pi[0], reps).astype(np.float32))
        g.cl_set_scalars(1.0)  # a' from the constraint of the non-minimally coupled system
        e0 = g.cl_energies()
        st.abt[:] = (e0["a"], e0["adot"], 0.0)
        g.cl_step(n)
        gphi, gpi = g.cl_get_state(cl.CL_FIELD_PHI0), g.cl_get_state(cl.CL_FIELD_PI0)
        e = g.cl_energies()
    O.step(m, st, O.RK4_5, dt, n)
    assert rel_l2(gphi, tile3(st.phi[0], reps)) < 1e-6
    assert rel_l2(gpi, tile3(st.pi[0], reps)) < 1e-4
    assert e["a"] == pytest.approx(st.abt[0], rel=1e-7)
    assert e["adot"] == pytest.approx(st.abt[1], rel=1e-5)
