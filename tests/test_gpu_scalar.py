"""GPU parity of the fused scalar pass (through the C ABI) against the FP64 oracle.

Tolerances: FP64 fields within 1e-10 relative L2 of the oracle after 200 steps in
the linear phase; FP32 + Kahan within 1e-4 (the paper's single-precision round-off
is O(1e-7) per operation; 1e-4 leaves room for its growth over the run).
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


def gpu_lattice(cl, N, L, nf, prec, integ, **kw):
    return cl.Lattice(N, L, nf, prec, integ, **kw)


def upload(g, cl, st, nf):
    for f in range(nf):
        g.cl_set_state(cl.CL_FIELD_PHI0 + f, st.phi[f].astype(g.dtype))
        g.cl_set_state(cl.CL_FIELD_PI0 + f, st.pi[f].astype(g.dtype))
    g.cl_set_scalars(st.abt[0], st.abt[1], st.abt[2])


def download(g, cl, nf):
    phi = np.stack([g.cl_get_state(cl.CL_FIELD_PHI0 + f) for f in range(nf)])
    pi = np.stack([g.cl_get_state(cl.CL_FIELD_PI0 + f) for f in range(nf)])
    return phi, pi


# ---------------------------------------------------------------- config 1
CFG1 = dict(N=32, L=8 * math.pi, lam=1.0, alpha=1.0, kappa=0.1, dt=0.01, steps=200, seed=1234, amp2=1e-4)


def _config1_oracle():
    c = CFG1
    kcut = 16 * 2 * math.pi / c["L"]
    m = O.make_model(c["N"], c["L"], nf=1, alpha=c["alpha"], kappa=c["kappa"], expansion=True,
                     lam=(c["lam"], 0.0))
    st = O.vacuum(m, c["seed"], kcut, c["amp2"], (1.0,), (0.0,))
    st0 = st.copy()
    O.step(m, st, O.VV2, c["dt"], c["steps"])
    return m, st0, st, kcut


@pytest.fixture(scope="module")
def config1_oracle():
    return _config1_oracle()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_config1_lphi4_vv2_parity(cl, config1_oracle, prec, tol):
    """32^3 lambda phi^4, vacuum state from each side's own Philox stream, VV-2,
    dt = 0.01, 200 steps, self-consistent expansion."""
    m, st0, st, kcut = config1_oracle
    c = CFG1
    with gpu_lattice(cl, c["N"], c["L"], 1, prec, cl.CL_INT_VV2, expansion=True, alpha=c["alpha"],
                     kappa=c["kappa"], dt=c["dt"]) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [c["lam"]])
        g.cl_init_vacuum(c["seed"], kcut, c["amp2"], (1.0,), (0.0,))
        e0 = g.cl_energies()
        g.cl_step(c["steps"])
        phi, pi = download(g, cl, 1)
        e = g.cl_energies()
    eo0 = O.energies(m, st0)
    eo = O.energies(m, st)
    assert rel_l2(phi, st.phi) < tol
    assert rel_l2(pi, st.pi) < tol
    assert e["step"] == c["steps"]
    assert e["t"] == pytest.approx(st.abt[2], rel=1e-12)
    assert e["a"] == pytest.approx(st.abt[0], rel=tol)
    assert e["adot"] == pytest.approx(st.abt[1], rel=tol)
    for k in ("rho", "p", "V"):
        assert e0[k] == pytest.approx(eo0[k], rel=max(tol, 1e-12))
        assert e[k] == pytest.approx(eo[k], rel=max(tol, 1e-9))
    assert e["a"] > 1.01  # expansion happened


@pytest.mark.parametrize("N,nf,prec", [(16, 1, 0), (16, 2, 0), (10, 2, 0), (16, 2, 1)])
def test_vacuum_state_parity(cl, N, nf, prec):
    L = 7.0
    m = O.make_model(N, L, nf=nf, alpha=1.0, kappa=0.3, expansion=True, m2=(1.0, 0.0), lam=(0.5, 0.0),
                     g2=50.0 if nf == 2 else 0.0)
    kcut = 2 * math.pi / L * 5.5
    fbar, dfbar = (1.0, 0.2), (0.3, 0.0)
    st = O.vacuum(m, 77, kcut, 1e-3, fbar[:nf], dfbar[:nf])
    with gpu_lattice(cl, N, L, nf, prec, cl.CL_INT_VV2, expansion=True, alpha=1.0, kappa=0.3, dt=0.01) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [1.0, 0.5, 0.0, 0.0, 50.0 if nf == 2 else 0.0])
        g.cl_init_vacuum(77, kcut, 1e-3, fbar[:nf], dfbar[:nf])
        phi, pi = download(g, cl, nf)
        a, adot, t = g.cl_get_scalars()
        e = g.cl_energies()
    for f in range(nf):
        if prec == 0:  # FP64: the fluctuations themselves agree to 1e-12
            assert np.max(np.abs(phi[f] - st.phi[f])) < 1e-12 * np.max(np.abs(st.phi[f] - fbar[f]))
            assert np.max(np.abs(pi[f] - st.pi[f])) < 1e-12 * np.max(np.abs(st.pi[f]))
        else:  # FP32 storage: one rounding of each value (half an ulp, 6e-8 relative)
            assert np.max(np.abs(phi[f] - st.phi[f]) / np.maximum(np.abs(st.phi[f]), 1e-30)) < 6.5e-8
            assert np.max(np.abs(pi[f] - st.pi[f]) / np.maximum(np.abs(st.pi[f]), 1e-30)) < 6.5e-8
    tol = 1e-12 if prec == 0 else 1e-6
    assert adot == pytest.approx(st.abt[1], rel=max(tol, 1e-12))
    assert e["hubble_violation"] < (1e-12 if prec == 0 else 1e-6)


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4), (2, 1e-4)])
def test_two_field_yoshida4_parity(cl, prec, tol):
    """m^2 phi^2 + g^2 phi^2 chi^2 (q = 100 -> g2 = 4q), Yoshida-4, seeded white-noise input."""
    N, L, dt, n = 24, 8 * math.pi, 0.005, 60
    phi, pi = inputs.scalar_state(N, 2, seed=3, fbar=(1.0, 0.0), amp=1e-3, pamp=1e-3)
    m = O.make_model(N, L, nf=2, alpha=0.0, kappa=0.1, expansion=True, m2=(1.0, 0.0), g2=400.0)
    st = O.State(phi.copy(), pi.copy(), np.array([1.0, 0.0, 0.0]))
    e0 = O.energies(m, st)
    st.abt[1] = math.sqrt(0.1 * e0["rho"] / 3.0)
    with gpu_lattice(cl, N, L, 2, prec, cl.CL_INT_YOSHIDA4, expansion=True, alpha=0.0, kappa=0.1, dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_M2_G2, [1.0, 400.0])
        upload(g, cl, st, 2)
        g.cl_step(n)
        gphi, gpi = download(g, cl, 2)
        e = g.cl_energies()
    O.step(m, st, O.YOSHIDA4, dt, n)
    assert rel_l2(gphi, st.phi) < tol
    assert rel_l2(gpi, st.pi) < tol
    assert e["a"] == pytest.approx(st.abt[0], rel=tol)


@pytest.mark.parametrize("scheme,prec,n", [(4, 0, 6), (5, 0, 3), (6, 0, 1), (4, 1, 6), (5, 2, 3)])
def test_higher_yoshida_parity(cl, scheme, prec, n):
    """Yoshida-6/8/10 (9, 27, 81 fused passes per step) against the FP64 oracle, two fields,
    self-consistent expansion."""
    N, L, dt = 16, 6.0, 0.02
    phi, pi = inputs.scalar_state(N, 2, seed=23, fbar=(0.8, 0.1), amp=0.05, pamp=0.05)
    m = O.make_model(N, L, nf=2, alpha=1.0, kappa=0.5, expansion=True, m2=(0.3, 0.2), lam=(1.0, 0.5), g2=2.0)
    st = O.State(phi.copy(), pi.copy(), np.array([1.0, 0.2, 0.0]))
    with gpu_lattice(cl, N, L, 2, prec, scheme, expansion=True, alpha=1.0, kappa=0.5, dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [0.3, 1.0, 0.2, 0.5, 2.0])
        upload(g, cl, st, 2)
        g.cl_step(n)
        gphi, gpi = download(g, cl, 2)
        e = g.cl_energies()
        assert g.cl_last_launch_count() == {4: 9, 5: 27, 6: 81}[scheme] * n + 1  # + the opening half-kick
    O.step(m, st, {4: O.YOSHIDA6, 5: O.YOSHIDA8, 6: O.YOSHIDA10}[scheme], dt, n)
    tol = 1e-10 if prec == 0 else 1e-4
    assert rel_l2(gphi, st.phi) < tol
    assert rel_l2(gpi, st.pi) < tol
    assert e["a"] == pytest.approx(st.abt[0], rel=tol)
    assert e["t"] == pytest.approx(n * dt, rel=1e-12)


@pytest.mark.parametrize("N,by,dz", [(6, 4, 4), (10, 3, 4), (34, 5, 7), (7, 2, 3), (5, 1, 2), (48, 0, 0)])
@pytest.mark.parametrize("prec", [0, 1])
def test_ragged_sizes_and_tiles(cl, N, by, dz, prec):
    """Odd sizes and tiles that do not divide N exercise the ragged rows/planes and the
    scalar (VW = 1) and paired (VW = 2) vector paths."""
    L, dt, n = 0.9 * N, 0.02, 25
    phi, pi = inputs.scalar_state(N, 2, seed=N, fbar=(0.8, 0.1), amp=0.05, pamp=0.05)
    m = O.make_model(N, L, nf=2, alpha=1.0, kappa=0.5, expansion=True, m2=(0.3, 0.2), lam=(1.0, 0.5), g2=2.0)
    st = O.State(phi.copy(), pi.copy(), np.array([1.0, 0.2, 0.0]))
    with gpu_lattice(cl, N, L, 2, prec, cl.CL_INT_VV2, expansion=True, alpha=1.0, kappa=0.5, dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [0.3, 1.0, 0.2, 0.5, 2.0])
        if by:
            g.cl_set_option(cl.CL_OPT_TILE_BY, by)
            g.cl_set_option(cl.CL_OPT_TILE_DZ, dz)
        upload(g, cl, st, 2)
        g.cl_step(n)
        gphi, gpi = download(g, cl, 2)
    O.step(m, st, O.VV2, dt, n)
    tol = 1e-12 if prec == 0 else 1e-5
    assert rel_l2(gphi, st.phi) < tol
    assert rel_l2(gpi, st.pi) < tol


def test_graph_and_plain_launches_identical(cl):
    N = 16
    phi, pi = inputs.scalar_state(N, 1, seed=8, fbar=(1.0,), amp=0.1, pamp=0.1)
    outs = []
    for graph in (1, 0):
        with gpu_lattice(cl, N, 5.0, 1, 1, cl.CL_INT_YOSHIDA4, expansion=True, alpha=1.0, kappa=0.2, dt=0.01) as g:
            g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
            g.cl_set_option(cl.CL_OPT_GRAPH, graph)
            g.cl_set_state(cl.CL_FIELD_PHI0, phi[0].astype(np.float32))
            g.cl_set_state(cl.CL_FIELD_PI0, pi[0].astype(np.float32))
            g.cl_set_scalars(1.0)
            g.cl_step(7)
            g.cl_step(6)
            outs.append(download(g, cl, 1) + (g.cl_energies()["a"],))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


@pytest.mark.parametrize("N,nf,prec", [(64, 2, 1), (32, 1, 0), (48, 2, 2), (40, 2, 0)])
def test_tma_and_direct_loaders_identical(cl, N, nf, prec):
    """The TMA-staged loader only changes how rows reach shared memory: FP32 fields must be
    bit-identical to the direct loader with the same tiles.  In FP64 the direct loader sums
    the gradient energy by parts and evaluates the potential in Horner form (fewer FP64
    operations; the TMA loaders keep the forward differences), so a(t) and the fields agree
    to rounding instead."""
    phi, pi = inputs.scalar_state(N, nf, seed=13, fbar=(1.0, 0.1), amp=0.05, pamp=0.05)
    dt = np.float64 if prec == 0 else np.float32
    outs = []
    for stages in (-1, 2, 3, 4):
        with gpu_lattice(cl, N, 9.0, nf, prec, cl.CL_INT_YOSHIDA4, expansion=True, alpha=1.0, kappa=0.2,
                         dt=0.01) as g:
            g.cl_set_potential(cl.CL_POT_POLY, [0.5, 1.0, 0.2 if nf == 2 else 0.0, 0.0, 3.0 if nf == 2 else 0.0])
            g.cl_set_option(cl.CL_OPT_TILE_BY, 3)
            g.cl_set_option(cl.CL_OPT_TILE_DZ, 5)
            g.cl_set_option(cl.CL_OPT_STAGES, stages)
            for f in range(nf):
                g.cl_set_state(cl.CL_FIELD_PHI0 + f, phi[f].astype(dt))
                g.cl_set_state(cl.CL_FIELD_PI0 + f, pi[f].astype(dt))
            g.cl_set_scalars(1.0)
            g.cl_step(9)
            outs.append(download(g, cl, nf))
    for o in outs[1:]:
        if prec == 0:
            assert rel_l2(o[0], outs[0][0]) < 1e-13 and rel_l2(o[1], outs[0][1]) < 1e-13
        else:
            assert np.array_equal(o[0], outs[0][0])
            assert np.array_equal(o[1], outs[0][1])


@pytest.mark.parametrize("N,nf,prec,by,dz,stages",
                         [(64, 2, 2, 3, 5, 4), (64, 1, 1, 0, 0, 0), (40, 2, 1, 7, 9, 2), (32, 1, 0, 3, 5, 3),
                          (48, 2, 2, 16, 1, 5), (128, 2, 2, 0, 0, 0), (256, 2, 2, 0, 0, 0)])
def test_ringless_and_ring_passes_identical(cl, N, nf, prec, by, dz, stages):
    """The ringless TMA pass re-drifts the y-neighbour rows from the stage instead of sharing
    drifted rows through a ring: the same arithmetic, so fields must agree bit for bit with the
    ring pass, and energies and the scale factor too when both run the same tiles."""
    phi, pi = inputs.scalar_state(N, nf, seed=17, fbar=(1.0, 0.1), amp=0.05, pamp=0.05)
    dt = np.float64 if prec == 0 else np.float32
    outs = []
    for variant in (0, 1):
        with gpu_lattice(cl, N, 9.0, nf, prec, cl.CL_INT_YOSHIDA4, expansion=True, alpha=1.0, kappa=0.2,
                         dt=0.01) as g:
            g.cl_set_potential(cl.CL_POT_POLY, [0.5, 1.0, 0.2 if nf == 2 else 0.0, 0.0, 3.0 if nf == 2 else 0.0])
            if by:
                g.cl_set_option(cl.CL_OPT_TILE_BY, by)
                g.cl_set_option(cl.CL_OPT_TILE_DZ, dz)
            if stages:
                g.cl_set_option(cl.CL_OPT_STAGES, stages)
            g.cl_set_option(cl.CL_OPT_PASS_VARIANT, variant)
            for f in range(nf):
                g.cl_set_state(cl.CL_FIELD_PHI0 + f, phi[f].astype(dt))
                g.cl_set_state(cl.CL_FIELD_PI0 + f, pi[f].astype(dt))
            g.cl_set_scalars(1.0)
            g.cl_step(7)
            e = g.cl_energies()
            outs.append(download(g, cl, nf) + (e["a"], e["rho"], g.cl_get_scalars()))
    for k in range(2):
        assert np.array_equal(outs[1][k], outs[0][k])
    if by:
        assert outs[1][2:] == outs[0][2:]
    else:  # default tiles differ (448 vs 480 consumer threads): the per-thread compensated FP32
        # energy sums cover other sites, so energies agree to their rounding only
        assert outs[1][2] == pytest.approx(outs[0][2], rel=1e-10)
        assert outs[1][3] == pytest.approx(outs[0][3], rel=1e-10)
        for u, v in zip(outs[1][4], outs[0][4]):
            assert u == pytest.approx(v, rel=1e-10)


def test_effective_options_reported(cl):
    """cl_get_option reports the tiling the library chose: the ringless TMA pass where rows are
    16-byte vectors, the ring variant otherwise; overrides are reflected."""
    with gpu_lattice(cl, 256, 9.0, 2, 1, cl.CL_INT_YOSHIDA4, expansion=True, alpha=0.0, kappa=0.1, dt=0.005) as g:
        # the headline tiling: two fields with Kahan compensation, six arrays a row, four stages
        assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == 1
        assert g.cl_get_option(cl.CL_OPT_STAGES) == 4
        assert g.cl_get_option(cl.CL_OPT_TILE_BY) == 7
    with gpu_lattice(cl, 256, 9.0, 2, 2, cl.CL_INT_YOSHIDA4, expansion=True, alpha=0.0, kappa=0.1, dt=0.005) as g:
        # plain FP32: four arrays a row leave room for a fifth stage beside the same tile
        assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == 1
        assert g.cl_get_option(cl.CL_OPT_STAGES) == 5
        assert g.cl_get_option(cl.CL_OPT_TILE_BY) == 7
        assert g.cl_get_option(cl.CL_OPT_TILE_DZ) == 64
        assert g.cl_get_option(cl.CL_OPT_GRAPH) == 1
        g.cl_set_option(cl.CL_OPT_PASS_VARIANT, 0)
        assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == 0
        assert g.cl_get_option(cl.CL_OPT_STAGES) == 3
        g.cl_set_option(cl.CL_OPT_STAGES, -1)
        assert g.cl_get_option(cl.CL_OPT_STAGES) == 0
        with pytest.raises(cl.CLError):
            g.cl_get_option(99)
    with gpu_lattice(cl, 34, 9.0, 1, 1, cl.CL_INT_VV2, expansion=True, alpha=0.0, kappa=0.1, dt=0.005) as g:
        assert g.cl_get_option(cl.CL_OPT_PASS_VARIANT) == 0  # 8-byte vectors: no ringless kernel


def test_ringless_pass_matches_oracle(cl):
    """Yoshida-4 with Kahan drifts through the ringless pass against the FP64 oracle."""
    N, L, dt, n = 40, 0.9 * 40, 0.02, 12
    phi, pi = inputs.scalar_state(N, 2, seed=21, fbar=(0.8, 0.1), amp=0.05, pamp=0.05)
    m = O.make_model(N, L, nf=2, alpha=1.0, kappa=0.5, expansion=True, m2=(0.3, 0.2), lam=(1.0, 0.5), g2=2.0)
    st = O.State(phi.copy(), pi.copy(), np.array([1.0, 0.2, 0.0]))
    with gpu_lattice(cl, N, L, 2, 2, cl.CL_INT_YOSHIDA4, expansion=True, alpha=1.0, kappa=0.5, dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_POLY, [0.3, 1.0, 0.2, 0.5, 2.0])
        g.cl_set_option(cl.CL_OPT_PASS_VARIANT, 1)
        upload(g, cl, st, 2)
        g.cl_step(n)
        gphi, gpi = download(g, cl, 2)
    O.step(m, st, O.YOSHIDA4, dt, n)
    assert rel_l2(gphi, st.phi) < 1e-5
    assert rel_l2(gpi, st.pi) < 1e-5


def test_tiles_do_not_change_results(cl):
    N = 32
    phi, pi = inputs.scalar_state(N, 1, seed=9, fbar=(1.0,), amp=0.1, pamp=0.1)
    res = []
    for by, dz in ((0, 0), (1, 32), (3, 5), (32, 1)):
        with gpu_lattice(cl, N, 9.0, 1, 0, cl.CL_INT_VV2, expansion=True, alpha=1.0, kappa=0.2, dt=0.01) as g:
            g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
            g.cl_set_option(cl.CL_OPT_TILE_BY, by)
            g.cl_set_option(cl.CL_OPT_TILE_DZ, dz)
            g.cl_set_state(cl.CL_FIELD_PHI0, phi[0])
            g.cl_set_state(cl.CL_FIELD_PI0, pi[0])
            g.cl_set_scalars(1.0)
            g.cl_step(20)
            res.append(download(g, cl, 1))
    for r in res[1:]:
        assert rel_l2(r[0], res[0][0]) < 1e-14
        assert rel_l2(r[1], res[0][1]) < 1e-13


def test_checkpoint_resume(cl):
    """get_state / set_state round trip: resuming from the integer-time state continues the run."""
    N = 16
    phi, pi = inputs.scalar_state(N, 1, seed=10, fbar=(1.0,), amp=0.1, pamp=0.1)
    kw = dict(expansion=True, alpha=1.0, kappa=0.2, dt=0.01)
    with gpu_lattice(cl, N, 5.0, 1, 0, cl.CL_INT_VV2, **kw) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
        g.cl_set_state(cl.CL_FIELD_PHI0, phi[0])
        g.cl_set_state(cl.CL_FIELD_PI0, pi[0])
        g.cl_set_scalars(1.0)
        g.cl_step(10)
        cp = download(g, cl, 1) + (g.cl_get_scalars(),)
        g.cl_step(10)
        ref = download(g, cl, 1)
    with gpu_lattice(cl, N, 5.0, 1, 0, cl.CL_INT_VV2, **kw) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
        g.cl_set_state(cl.CL_FIELD_PHI0, cp[0][0])
        g.cl_set_state(cl.CL_FIELD_PI0, cp[1][0])
        g.cl_set_scalars(*cp[2])
        g.cl_step(10)
        got = download(g, cl, 1)
    assert rel_l2(got[0], ref[0]) < 1e-13
    assert rel_l2(got[1], ref[1]) < 1e-12


def test_nan_is_reported(cl):
    N = 8
    phi, pi = inputs.scalar_state(N, 1, seed=11, fbar=(1.0,))
    phi[0, 3, 2, 1] = np.nan  # fault injected on the host
    with gpu_lattice(cl, N, 5.0, 1, 0, cl.CL_INT_VV2, expansion=True, dt=0.01) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
        g.cl_set_state(cl.CL_FIELD_PHI0, phi[0])
        g.cl_set_state(cl.CL_FIELD_PI0, pi[0])
        g.cl_set_scalars(1.0, 0.1)
        g.cl_step(2)
        with pytest.raises(cl.CLError) as ei:
            g.cl_sync()
        assert ei.value.status == cl.CL_ENAN
        g.cl_sync()  # the status is reported once


def test_hubble_limit_is_reported(cl):
    N = 8
    phi, pi = inputs.scalar_state(N, 1, seed=12, fbar=(1.0,), amp=0.2, pamp=0.2)
    with gpu_lattice(cl, N, 5.0, 1, 0, cl.CL_INT_VV2, expansion=True, kappa=0.5, dt=0.05) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
        g.cl_set_state(cl.CL_FIELD_PHI0, phi[0])
        g.cl_set_state(cl.CL_FIELD_PI0, pi[0])
        g.cl_set_scalars(1.0)  # a' from Eq. Friedmann2
        assert g.cl_energies()["hubble_violation"] < 1e-13
        g.cl_set_hubble_limit(1e-14)
        g.cl_step(5)
        with pytest.raises(cl.CLError) as ei:
            g.cl_energies()
        assert ei.value.status == cl.CL_ECONSTRAINT


def test_spectrum_parity(cl):
    N, L = 16, 6.0
    f = 0.5 + inputs.rng(21).standard_normal((N, N, N))
    with gpu_lattice(cl, N, L, 1, 0, cl.CL_INT_VV2) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
        g.cl_set_state(cl.CL_FIELD_PHI0, f)
        for dn, t in ((1.0, 1), (1.0, 2), (0.5, 1), (2.5, 2)):
            k, d, c = g.cl_spectrum(cl.CL_FIELD_PHI0, dn, t)
            ko, do, co = O.spectrum(N, L, f, dn, t)
            np.testing.assert_array_equal(c, co)
            np.testing.assert_allclose(k, ko, rtol=1e-14)
            np.testing.assert_allclose(d, do, rtol=1e-11, atol=1e-14 * do.max())


def test_launch_count_and_step_counter(cl):
    with gpu_lattice(cl, 8, 4.0, 1, 1, cl.CL_INT_YOSHIDA4, dt=0.01) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
        g.cl_set_state(cl.CL_FIELD_PHI0, np.ones((8, 8, 8), np.float32))
        g.cl_step(4)
        assert g.cl_last_launch_count() == 1 + 4 * 3  # opening half kick + 3 passes per step
        g.cl_step(2)
        assert g.cl_last_launch_count() == 2 * 3
        assert g.cl_energies()["step"] == 6


def test_full_size_yoshida4_fp32_kahan_one_step(cl):
    """The bench workload (256^3, two fields, q = 1e4, Yoshida-4, FP32 + Kahan) for two
    steps from a seeded input, against the FP64 oracle over the whole lattice."""
    N, L, dt = 256, 8 * math.pi, 0.005
    phi, pi = inputs.scalar_state(N, 2, seed=5, fbar=(1.0, 0.0), amp=1e-4, pamp=1e-4)
    m = O.make_model(N, L, nf=2, alpha=0.0, kappa=0.1, expansion=True, m2=(1.0, 0.0), g2=4e4)
    st = O.State(phi, pi, np.array([1.0, 0.0, 0.0]))
    st.abt[1] = math.sqrt(0.1 * O.energies(m, st)["rho"] / 3.0)
    with gpu_lattice(cl, N, L, 2, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_YOSHIDA4, expansion=True, alpha=0.0,
                     kappa=0.1, dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_M2_G2, [1.0, 4e4])
        upload(g, cl, st, 2)
        g.cl_step(2)
        gphi, gpi = download(g, cl, 2)
        e = g.cl_energies()
    O.step(m, st, O.YOSHIDA4, dt, 2)
    assert rel_l2(gphi, st.phi) < 1e-6
    assert rel_l2(gpi[0], st.pi[0]) < 1e-4
    assert rel_l2(gpi[1], st.pi[1]) < 1e-4
    assert e["a"] == pytest.approx(st.abt[0], rel=1e-7)


def test_largest_lattice_homogeneous(cl):
    """N = 1536 (the largest size the tiling accepts), FP32 + Kahan, homogeneous phi^4:
    every site must stay identical and follow the oracle's homogeneous run."""
    import torch
    N, dt, n = 1536, 0.02, 50
    with gpu_lattice(cl, N, 100.0, 1, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_VV2, expansion=False, dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
        buf = torch.ones(N ** 3, dtype=torch.float32, device="cuda")
        g.cl_set_state(cl.CL_FIELD_PHI0, buf)
        g.cl_step(n)
        g.cl_get_state(cl.CL_FIELD_PHI0, buf)
        torch.cuda.synchronize()
        lo, hi = float(buf.min()), float(buf.max())
        del buf
    m = O.make_model(2, 1.0, nf=1, alpha=1.0, lam=(1.0, 0.0))
    st = O.new_state(m)
    st.phi[:] = 1.0
    O.step(m, st, O.VV2, dt, n)
    assert lo == hi
    assert lo == pytest.approx(st.phi.flat[0], abs=2e-6)
