"""The stored oracle values of tests/golden/ (written by
tests/golden/make_golden.py from the oracle alone) against a fresh run of the
seeded generator and the oracle: the synthetic workload and the oracle's
spectrum and poles do not drift."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tiny4_spectrum_and_poles_match_the_stored_values():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(HERE, "golden", "tiny4_spectrum.json")) as f:
        stored = json.load(f)
    now = mg.tiny4_values()
    assert now["omega"] == stored["omega"] and now["eps"] == stored["eps"]
    P_s = np.array(stored["P_re"]) + 1j * np.array(stored["P_im"])
    P_n = np.array(now["P_re"]) + 1j * np.array(now["P_im"])
    assert np.max(np.abs(P_n - P_s)) <= 1e-9 * np.max(np.abs(P_s))
    assert np.allclose(now["poles_omega"], stored["poles_omega"], rtol=1e-10, atol=0)
    assert np.allclose(now["poles_g_trace"], stored["poles_g_trace"], rtol=1e-8, atol=0)
    # the golden spectrum itself satisfies the physics: P symmetric, P(0) real
    assert np.max(np.abs(P_s - np.swapaxes(P_s, 1, 2))) <= 1e-9 * np.max(np.abs(P_s))
    assert np.max(np.abs(P_s[0].imag)) <= 1e-9 * np.max(np.abs(P_s[0]))
