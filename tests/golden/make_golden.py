"""Write the stored expected values of tests/golden/ from the CPU oracle only.

    python tests/golden/make_golden.py

tiny4_spectrum.json: the 4-atom synthetic workload (seeded generator of
paper_1005_5340_gb300/synth.py) at five frequencies of its grid:
  * P_ik(omega) of eq. eqpolarizability by the oracle's dense LU solve of eq. sle;
  * the ten strongest exact poles Omega_n of the model (transition-space
    eigen-decomposition) with their trace residues g_n = tr g_n,ik / 3.
The paper prints no worked numerical example, so these are oracle values:
they pin the generator and the oracle against silent drift.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle.spectrum_oracle as SO  # noqa: E402
import oracle.tddft_oracle as O  # noqa: E402
from paper_1005_5340_gb300 import synth  # noqa: E402

OMEGA_INDEX = [0, 13, 27, 40, 63]


def tiny4_values():
    s, w = synth.workload("tiny4")
    M = O.transition_vertex(s)
    om = np.asarray(w["omega"])[OMEGA_INDEX]
    P = np.stack([O.polarizability_lu(s, x, w["eps"], M)[0] for x in om])
    Om, g = SO.casida_poles(s, M)
    tr = np.einsum("nii->n", g) / 3.0
    top = np.argsort(-tr)[:10]
    return dict(
        source="oracle/tddft_oracle.py polarizability_lu and oracle/spectrum_oracle.py "
               "casida_poles on synth.workload('tiny4')",
        eps=float(w["eps"]), omega=[float(x) for x in om],
        P_re=P.real.tolist(), P_im=P.imag.tolist(),
        poles_omega=[float(Om[i]) for i in sorted(top)],
        poles_g_trace=[float(tr[i]) for i in sorted(top)])


if __name__ == "__main__":
    with open(os.path.join(HERE, "tiny4_spectrum.json"), "w") as f:
        json.dump(tiny4_values(), f, indent=1)
