"""The refinement form (TDDFT_PREC_BF16X3_IR) through the C boundary:
the split-bf16 tensor-core GEMM against float64, the reduced-precision
operator against the oracle (relative error <= 1e-4, the split-bf16
products being good to ~1e-5), and spectra that, thanks to the float64
residual that closes every cycle, reach the same tolerance as the float64
path and agree with the oracle's dense LU."""
import numpy as np
import pytest

import oracle.tddft_oracle as O
from paper_1005_5340_gb300 import synth
from tests.libutil import ensure_library
from tests.test_gpu_parity import ragged_system, rel

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


@pytest.mark.parametrize("shape", [(128, 128, 64), (300, 200, 100), (704, 1024, 832),
                                   (1000, 384, 1664)])
def test_tensor_core_gemm_selftest(shape):
    M, N, K = shape
    err = T().selftest_gemm(M, N, K, seed=7)
    assert err < 2e-5, err


@pytest.mark.parametrize("sysname", ["tiny4", "ragged"])
def test_lowprec_operators_match_oracle(sysname):
    if sysname == "tiny4":
        s, w = synth.workload("tiny4")
        eps = w["eps"]
    else:
        s, eps = ragged_system(), 0.02
    M = O.transition_vertex(s)
    omegas = np.array([0.0, 0.13, 0.5, 0.77, 1.0])
    z = synth.random_complex_vectors(omegas.size, s.n_prod, 9)
    with T().Context(s, batch=8, prec="bf16x3") as ctx:
        chi = ctx.chi0_apply(z, omegas, eps)
        Az = ctx.apply_A(z, omegas, eps)
    for r, om in enumerate(omegas):
        c = O.chi0_explicit(s, om, eps, M)
        assert rel(chi[r], c @ z[r]) < 1e-4
        ref = z[r] - c @ (s.K @ z[r])
        assert rel(Az[r] - z[r], ref - z[r]) < 1e-4


def test_lowprec_spectrum_reaches_float64_accuracy():
    s, w = synth.workload("tiny4")
    M = O.transition_vertex(s)
    om = w["omega"][::3]
    with T().Context(s, batch=66, restart=w["restart"], tol=1e-11, max_restarts=60,
                     prec="bf16x3", inner_tol=1e-4) as ctx:
        P, info = ctx.polarizability(om, w["eps"])
    assert info["converged"].all() and np.all(info["resid"] <= 1e-11)
    P_lu = np.stack([O.polarizability_lu(s, x, w["eps"], M)[0] for x in om])
    assert rel(P, P_lu) < 1e-9
    # each cycle gains at least three digits: a handful of float64 residuals
    assert info["cycles"].max() <= 6


def test_lowprec_spectrum_at_workload_tolerance():
    s, w = synth.workload("tiny4")
    M = O.transition_vertex(s)
    om = w["omega"]
    with T().Context(s, batch=192, restart=w["restart"], tol=w["tol"], prec="bf16x3") as ctx:
        P, info = ctx.polarizability(om, w["eps"])
    assert info["converged"].all() and np.all(info["resid"] <= w["tol"])
    P_lu = np.stack([O.polarizability_lu(s, x, w["eps"], M)[0] for x in om])
    alpha, alpha_lu = -P, -P_lu
    im = np.einsum("wii->wi", alpha).imag
    im_lu = np.einsum("wii->wi", alpha_lu).imag
    assert np.max(np.abs(im - im_lu)) / np.max(np.abs(im_lu)) < 1e-4


@pytest.mark.slow
def test_medium64_lowprec_operator_and_spectrum_samples():
    s, w = synth.workload("medium64")
    op = O.StepOperator(s)
    omegas = np.array([0.0, 0.75, 1.5])
    z = synth.random_complex_vectors(omegas.size, s.n_prod, 11)
    om = w["omega"][[5, 128, 250]]
    with T().Context(s, batch=9, restart=w["restart"], tol=w["tol"], prec="bf16x3") as ctx:
        chi = ctx.chi0_apply(z, omegas, w["eps"])
        P_lp, info_lp = ctx.polarizability(om, w["eps"])
    for r, x in enumerate(omegas):
        assert rel(chi[r], op.apply(z[r], x, w["eps"])) < 1e-4
    with T().Context(s, batch=9, restart=w["restart"], tol=w["tol"]) as ctx:
        P_64, info_64 = ctx.polarizability(om, w["eps"])
    assert info_lp["converged"].all() and info_64["converged"].all()
    # both solutions satisfy the same float64 residual bound
    assert rel(P_lp, P_64) < 1e-4
