"""Writes statistical_64_q1e4.json: an FP64 oracle trajectory of two-field preheating
past its linear phase, for the statistical parity test (tests/test_gpu_statistical.py).

The run is the two-field model of the benchmark (V = m^2 phi^2/2 + g^2 phi^2 chi^2/2,
q = g^2 phi0^2 / (4 m^2) = 1e4, program units m = 1, f_star = phi0, alpha = 0), on a 64^3
lattice with the benchmark's box L = 8 pi, dt = 0.005, Yoshida-4, self-consistent
expansion with kappa = (phi0 / m_p)^2 = 0.01, from the oracle's own vacuum state
(Philox seed 1234, amplitude (omega_star / f_star)^2 = 1e-9, no momentum cut-off;
sections "Initial conditions" and "Inherited capabilities" of the paper).  With
kappa = 0.01 the chi modes of the broad resonance band grow until their energy is a
fraction of the total near t = 30, after which the fields rescatter: 10^4 steps
(t = 50) reach well into the nonlinear regime.  (With kappa = 0.1 expansion dilutes the
resonance so that 10^4 steps stay linear.)

Recorded, as plain JSON:
  * every 50 steps: t, a, a', K_phi, K_chi, G_phi, G_chi, V, rho, p and the
    Hubble-constraint violation (Eq. Friedmann2), the volume averages the paper defines
    (Eq. energy-contrib, Eq. rhoLocal);
  * the binned Type-I spectra (Eq. discretePST2, bin width 1) of phi and chi at steps
    2000, 4000, 6000, 6500 and every 100 steps from 7000 to 10000 (in the chaotic phase
    a single snapshot of a 64^3 lattice is one noisy realisation; the test compares
    spectra averaged over these snapshots), with the mode count of every bin.

Only the oracle is called (its serial build, whose sums run in a fixed order, so the
file is reproducible bit for bit on any host).  About 25 minutes on one core.
"""
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402

N, L, DT, Q, KAPPA, AMP2, SEED = 64, 8.0 * math.pi, 0.005, 1.0e4, 0.01, 1.0e-9, 1234
STEPS, EVERY = 10000, 50
CHECKPOINTS = [2000, 4000, 6000, 6500] + list(range(7000, 10001, 100))
OUT = os.path.join(HERE, "statistical_64_q1e4.json")
KEYS = ["K0", "K1", "G0", "G1", "V", "rho", "p", "hubble_violation", "a", "b"]


def model():
    return O.make_model(N, L, nf=2, alpha=0.0, kappa=KAPPA, expansion=True, m2=(1.0, 0.0), g2=4.0 * Q)


def main():
    m = model()
    st = O.vacuum(m, SEED, 1e30, AMP2, (1.0, 0.0), (0.0, 0.0))
    rec = {"about": "FP64 oracle trajectory for the statistical parity test; written by "
                    "tests/golden/make_statistical_goldens.py (oracle only)",
           "model": {"N": N, "L": L, "dt": DT, "q": Q, "g2": 4.0 * Q, "m2": 1.0, "kappa": KAPPA, "alpha": 0.0,
                     "integrator": "yoshida4", "expansion": True},
           "vacuum": {"seed": SEED, "kcut": 1e30, "amp2": AMP2, "fbar": [1.0, 0.0], "dfbar": [0.0, 0.0]},
           "energies": [], "spectra": {}, "spectrum_counts": {}}
    t0 = time.time()

    def record(step):
        e = O.energies(m, st)
        rec["energies"].append([step, float(st.abt[2])] + [float("%.15g" % e[k]) for k in KEYS])

    record(0)
    for s in range(EVERY, STEPS + 1, EVERY):
        O.step(m, st, O.YOSHIDA4, DT, EVERY)
        record(s)
        if s in CHECKPOINTS:
            spec = {}
            for f, name in ((0, "phi"), (1, "chi")):
                k, d, c = O.spectrum(N, L, st.phi[f], 1.0, 1)
                spec[name] = [float("%.12g" % x) for x in d]
                rec["spectrum_counts"][name] = [int(x) for x in c]
                rec["spectrum_k"] = [float(x) for x in k]
            rec["spectra"][str(s)] = spec
            print("step %d t=%.3f rho=%.6e  (%.0f s)" % (s, st.abt[2], rec["energies"][-1][2 + KEYS.index("rho")],
                                                         time.time() - t0), flush=True)
    rec["spectrum_steps"] = CHECKPOINTS
    rec["energy_columns"] = ["step", "t"] + KEYS
    with open(OUT + ".tmp", "w") as fh:
        json.dump(rec, fh, separators=(",", ":"))
    os.replace(OUT + ".tmp", OUT)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
