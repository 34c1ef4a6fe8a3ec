"""The stored FP64 oracle trajectory of the statistical parity test (tests/golden/
statistical_64_q1e4.json, written by make_statistical_goldens.py from the oracle alone).

  * provenance: the oracle as committed reproduces the file's first records (its vacuum state,
    energies and spectrum definitions), so the file belongs to this oracle;
  * the run does what the test needs it to: the chi modes of the resonance band grow by orders
    of magnitude, then carry a sizeable fraction of the energy, and phi fluctuations sourced by
    rescattering grow by orders of magnitude after them (the nonlinear phase), with the
    Hubble-constraint violation (Eq. Friedmann2) below 1e-3 throughout.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "statistical_64_q1e4.json")


@pytest.fixture(scope="module")
def golden():
    return json.load(open(GOLDEN))


def test_oracle_reproduces_the_first_records(golden):
    m, v = golden["model"], golden["vacuum"]
    model = O.make_model(m["N"], m["L"], nf=2, alpha=m["alpha"], kappa=m["kappa"], expansion=True,
                         m2=(m["m2"], 0.0), g2=m["g2"])
    st = O.vacuum(model, v["seed"], v["kcut"], v["amp2"], tuple(v["fbar"]), tuple(v["dfbar"]))
    cols = golden["energy_columns"]
    E = np.array(golden["energies"])
    every = int(E[1, 0] - E[0, 0])
    for i in range(2):
        if i:
            O.step(model, st, O.YOSHIDA4, m["dt"], every)
        e = O.energies(model, st)
        for k in cols[2:]:
            assert e[k] == pytest.approx(E[i, cols.index(k)], rel=1e-12, abs=1e-300), (i, k)
        assert st.abt[2] == pytest.approx(E[i, 1], rel=1e-12, abs=1e-15)


def test_golden_trajectory_goes_nonlinear(golden):
    E = np.array(golden["energies"])
    c = golden["energy_columns"]
    col = lambda k: E[:, c.index(k)]
    rho, K1, G1, G0 = col("rho"), col("K1"), col("G1"), col("G0")
    st = E[:, 0]
    chi_frac = (K1 + G1) / rho
    assert chi_frac[st == 2000][0] < 1e-3
    assert chi_frac[(st >= 8000)].mean() > 0.05
    assert G0[st == 10000][0] / G0[st == 6000][0] > 100
    assert np.all(col("hubble_violation") < 1e-3)
    assert len(golden["spectra"]) == len(golden["spectrum_steps"]) == 35
