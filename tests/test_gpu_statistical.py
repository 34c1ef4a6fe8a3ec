"""Statistical parity past the linear phase: the GPU path against an FP64 oracle trajectory.

Two-field preheating (V = m^2 phi^2/2 + g^2 phi^2 chi^2/2, q = 1e4) on a 64^3 lattice with the
benchmark's box and time step, Yoshida-4, self-consistent expansion (kappa = 0.01), from the
vacuum state of seed 1234, run for 10^4 steps.  The chi modes of the resonance band grow
until, near t = 30 (step 6000), they carry a sizeable fraction of the energy and rescatter
into phi; from there on the dynamics is nonlinear and chaotic.  The oracle's trajectory is
stored in tests/golden/statistical_64_q1e4.json (written by make_statistical_goldens.py,
oracle only).  The GPU runs the same initial state from its own Philox + cuFFT vacuum
generator (equal to the oracle's to rounding).

Chaos amplifies the rounding differences of two correct runs.  Once the dynamics is
nonlinear, the largest per-bin spectrum difference between two runs grows about tenfold every
100-200 steps: FP32 + Kahan and FP64 runs part at the 1 % level near step 7200, and even two
FP64 runs (the GPU's reductions and the oracle's loops sum in different orders) near step
8800.  So agreement is required as follows (1 % throughout, the bound the statistical parity
calls for):
  * pointwise while the runs are still correlated -- up to step 8500 in FP64, up to step 7000
    in FP32 + Kahan (the onset of the nonlinear phase: the rescattered phi gradient energy has
    grown 40-fold since step 6000): every recorded volume average (K, G of each field, V,
    rho; the pressure, which changes sign, relative to rho) and every bin (k > 0) of the
    binned Type-I spectra of phi and chi at every snapshot;
  * in the chaotic phase, statistics that one 64^3 realisation determines to 1 %: rho at every
    record, 2000-step window means of each energy and of the Hubble-constraint violation, and
    the spectra averaged over the 21 snapshots of steps 8000-10000, compared as the field
    variance in five k-bands of equal mode count, the total variance and the peak bin.  (A
    single bin of one snapshot scatters by 2-50 % between two chaotic runs: its mode count
    is 7 to 12,000.  The choice of statistics was calibrated on independent, equally valid
    FP64 runs -- the oracle with its sums in another order and with 1e-13 perturbations of
    the initial field -- and on GPU runs: across them the window means stay within 0.3 %, the
    total variances within 0.3 % and the equal-mode bands within 0.5 % of the stored run, while
    five bands of equal width in k reach 1.1 %, since the lowest of them holds few modes.)
The Hubble-constraint violation (Eq. Friedmann2) stays below 1e-3 everywhere.
"""
import json
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "statistical_64_q1e4.json")
POINTWISE_END = {"fp64": 8500, "fp32k": 7000}
KEYS_GPU = {"K0": "K0", "K1": "K1", "G0": "G0", "G1": "G1", "V": "V", "rho": "rho", "p": "p",
            "hubble_violation": "hubble_violation", "a": "a", "b": "adot"}


@pytest.fixture(scope="module")
def golden():
    return json.load(open(GOLDEN))


def run_gpu(prec, gold):
    """The GPU trajectory in the golden's format: energies every 50 steps, spectra at the
    golden's snapshot steps."""
    from paper_2607_24978_gb300 import build_ext, cl
    build_ext.build()
    m, v = gold["model"], gold["vacuum"]
    cols = gold["energy_columns"]
    every = int(gold["energies"][1][0] - gold["energies"][0][0])
    steps_total = int(gold["energies"][-1][0])
    snaps = set(int(s) for s in gold["spectrum_steps"])
    out = {"energies": [], "spectra": {}}
    with cl.Lattice(m["N"], m["L"], 2, prec, cl.CL_INT_YOSHIDA4, expansion=True, alpha=m["alpha"],
                    kappa=m["kappa"], dt=m["dt"]) as g:
        g.cl_set_potential(cl.CL_POT_M2_G2, [m["m2"], m["g2"]])
        g.cl_init_vacuum(v["seed"], v["kcut"], v["amp2"], tuple(v["fbar"]), tuple(v["dfbar"]))

        def record(step):
            e = g.cl_energies()
            out["energies"].append([step, e["t"]] + [e[KEYS_GPU[k]] for k in cols[2:]])

        record(0)
        for s in range(every, steps_total + 1, every):
            g.cl_step(every)
            record(s)
            if s in snaps:
                out["spectra"][str(s)] = {nm: g.cl_spectrum(f)[1] for f, nm in ((cl.CL_FIELD_PHI0, "phi"),
                                                                                 (cl.CL_FIELD_PHI1, "chi"))}
    out["energies"] = np.array(out["energies"])
    return out


@pytest.fixture(scope="module")
def gpu64(golden):
    from paper_2607_24978_gb300 import cl
    return run_gpu(cl.CL_PREC_FP64, golden)


@pytest.fixture(scope="module")
def gpu32(golden):
    from paper_2607_24978_gb300 import cl
    return run_gpu(cl.CL_PREC_FP32_KAHAN, golden)


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))


@pytest.mark.parametrize("which", ["fp64", "fp32k"])
def test_energies(golden, gpu64, gpu32, which):
    gpu = gpu64 if which == "fp64" else gpu32
    G = np.array(golden["energies"])
    c = golden["energy_columns"]
    assert gpu["energies"].shape == G.shape
    assert np.array_equal(gpu["energies"][:, 0], G[:, 0])
    ix = {k: c.index(k) for k in c}
    steps = G[:, 0]
    pointwise = steps <= POINTWISE_END[which]
    for k in ("K0", "K1", "G0", "G1", "V", "rho", "a", "b"):
        r = rel(gpu["energies"][pointwise, ix[k]], G[pointwise, ix[k]])
        assert r.max() < 1e-2, (k, float(r.max()), float(steps[pointwise][np.argmax(r)]))
    dp = np.abs(gpu["energies"][pointwise, ix["p"]] - G[pointwise, ix["p"]]) / G[pointwise, ix["rho"]]
    assert dp.max() < 1e-2
    # rho at every record
    assert rel(gpu["energies"][:, ix["rho"]], G[:, ix["rho"]]).max() < 1e-2
    assert np.all(gpu["energies"][:, ix["hubble_violation"]] < 1e-3)
    # 2000-step window means in the nonlinear phase
    for lo, hi in ((6000, 8000), (7000, 9000), (8000, 10000)):
        w = (steps >= lo) & (steps <= hi)
        for k in ("K0", "K1", "G0", "G1", "V", "rho", "hubble_violation"):
            r = abs(gpu["energies"][w, ix[k]].mean() - G[w, ix[k]].mean()) / abs(G[w, ix[k]].mean())
            assert r < 1e-2, (k, lo, hi, r)
        assert abs(gpu["energies"][w, ix["p"]].mean() - G[w, ix["p"]].mean()) < 1e-2 * G[w, ix["rho"]].mean()


def _snap(rec, s, f):
    d = rec["spectra"][str(s)][f]
    return np.asarray(d, dtype=np.float64)


@pytest.mark.parametrize("which", ["fp64", "fp32k"])
def test_spectra_per_bin(golden, gpu64, gpu32, which):
    """Every bin (k > 0) of the phi and chi spectra within 1 % at the snapshots where the runs
    are still correlated: up to step 8500 in FP64, up to step 7000 in FP32 + Kahan."""
    gpu = gpu64 if which == "fp64" else gpu32
    last = POINTWISE_END[which]
    for s in golden["spectrum_steps"]:
        if s > last:
            continue
        for f in ("phi", "chi"):
            a, b = _snap(gpu, s, f), _snap(golden, s, f)
            assert a.shape == b.shape
            r = rel(a[1:], b[1:])
            assert r.max() < 1e-2, (s, f, float(r.max()), int(np.argmax(r)) + 1)


@pytest.mark.parametrize("which", ["fp64", "fp32k"])
def test_spectra_in_the_chaotic_phase(golden, gpu64, gpu32, which):
    """Spectra averaged over the 21 snapshots of steps 8000-10000: field variance per k-band
    (five bands holding a fifth of the k > 0 modes each), the total variance and the peak bin."""
    gpu = gpu64 if which == "fp64" else gpu32
    steps = [s for s in golden["spectrum_steps"] if 8000 <= s <= 10000]
    assert len(steps) == 21
    for f in ("phi", "chi"):
        a = np.mean([_snap(gpu, s, f) for s in steps], axis=0)
        b = np.mean([_snap(golden, s, f) for s in steps], axis=0)
        lidx = np.arange(len(b))
        # Type I: Delta_l = n_l S_l / N^6 (bin width 1), so Delta_l / l is the bin's share of <f^2>
        va, vb = a[1:] / lidx[1:], b[1:] / lidx[1:]
        assert abs(va.sum() - vb.sum()) / vb.sum() < 1e-2
        cum = np.cumsum(np.asarray(golden["spectrum_counts"][f][1:], dtype=np.float64))
        cum /= cum[-1]
        edges = [0] + [int(np.searchsorted(cum, q / 5.0)) + 1 for q in range(1, 5)] + [len(vb)]
        for i in range(5):
            sa, sb = va[edges[i]:edges[i + 1]].sum(), vb[edges[i]:edges[i + 1]].sum()
            assert abs(sa - sb) / sb < 1e-2, (f, i, abs(sa - sb) / sb)
        assert np.argmax(a[1:]) == np.argmax(b[1:])
