"""Adaptive frequency grid and pole extraction (tddft_spectrum_adaptive) on the
GPU against the oracle's rule driven by dense LU solves, and against the
exact poles of the model."""
import numpy as np
import pytest

import oracle.spectrum_oracle as SO
import oracle.tddft_oracle as O
from paper_1005_5340_gb300 import synth
from tests.libutil import ensure_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_library()


def T():
    from paper_1005_5340_gb300 import tddft
    return tddft


ARGS = dict(n_initial=33, max_points=300, rel_tol=0.02, peak_floor=0.02)


@pytest.fixture(scope="module")
def tiny4_reference():
    s, w = synth.workload("tiny4")
    eps = w["eps"]
    M = O.transition_vertex(s)
    solve = lambda ws: np.array([O.polarizability_lu(s, x, eps, M)[0] for x in ws])
    om, P = SO.adaptive_grid(solve, 0.0, 1.0, ARGS["n_initial"], ARGS["max_points"],
                             ARGS["rel_tol"], eps / 8)
    poles = SO.extract_poles(om, P, eps, ARGS["peak_floor"])
    return s, w, M, om, P, poles


def test_grid_and_poles_match_the_oracle(tiny4_reference):
    """float64 solves to 1e-11: the same refinement decisions, hence the same
    grid; P, the peaks and their fits agree with the dense-LU run."""
    s, w, M, om_o, P_o, poles_o = tiny4_reference
    eps = w["eps"]
    with T().Context(s, batch=96, restart=w["restart"], tol=1e-11, max_restarts=100) as ctx:
        om, P, poles = ctx.spectrum_adaptive(0.0, 1.0, eps, **ARGS)
    assert om.size == om_o.size
    assert np.max(np.abs(om - om_o)) < 1e-12
    assert np.max(np.abs(P - P_o)) <= 1e-8 * np.max(np.abs(P_o))
    assert len(poles) == len(poles_o)
    for p, (Om, g, pk, w_pk) in zip(poles, poles_o):
        assert abs(p["omega_peak"] - w_pk) < 1e-12
        assert abs(p["omega"] - Om) < 1e-6 * eps
        assert abs(p["g"] - g) <= 1e-5 * abs(g) + 1e-12
        assert abs(p["peak"] - pk) <= 1e-8 * abs(pk)


def test_every_fitted_pole_lies_at_an_exact_pole(tiny4_reference):
    """The fitted positions sit within eps of an eigenvalue Omega_n of the
    model's transition-space matrix (exact poles from the oracle)."""
    s, w, M, _, _, _ = tiny4_reference
    Om_exact, _ = SO.casida_poles(s, M)
    with T().Context(s, batch=96, restart=w["restart"], tol=1e-8) as ctx:
        _, _, poles = ctx.spectrum_adaptive(0.0, 1.0, w["eps"], **ARGS)
    assert len(poles) >= 5
    for p in poles:
        assert np.min(np.abs(Om_exact - p["omega"])) < w["eps"]


def test_refinement_form_finds_the_strong_peaks(tiny4_reference):
    """The chosen production form (split bf16 with emulated float64 residuals,
    tol 1e-6) places the five strongest peaks where the float64 run does."""
    s, w, M, om_o, P_o, poles_o = tiny4_reference
    with T().Context(s, batch=96, restart=w["restart"], tol=1e-6, prec="bf16x3emu") as ctx:
        _, _, poles = ctx.spectrum_adaptive(0.0, 1.0, w["eps"], **ARGS)
    strong = sorted(poles_o, key=lambda t: -t[2])[:5]
    found = np.array([p["omega"] for p in poles])
    for Om, _, _, _ in strong:
        assert np.min(np.abs(found - Om)) < 0.05 * w["eps"]


def test_bad_arguments_are_rejected(tiny4_reference):
    s, w = tiny4_reference[0], tiny4_reference[1]
    with T().Context(s, batch=8) as ctx:
        for bad in (dict(w_lo=1.0, w_hi=0.5), dict(eps=0.0), dict(n_initial=1),
                    dict(max_points=4, n_initial=8), dict(rel_tol=0.0), dict(peak_floor=1.0)):
            kw = dict(w_lo=0.0, w_hi=1.0, eps=w["eps"], n_initial=9, max_points=20)
            kw.update(bad)
            with pytest.raises(T().TddftError) as e:
                ctx.spectrum_adaptive(kw.pop("w_lo"), kw.pop("w_hi"), kw.pop("eps"), **kw)
            assert e.value.status == T().ERR_INVALID_ARG
        # still usable, and a budget smaller than the rule wants is respected
        om, P, _ = ctx.spectrum_adaptive(0.0, 1.0, w["eps"], n_initial=9, max_points=20)
    assert om.size == 20 and np.all(np.diff(om) > 0)
