"""The TF32 refinement forms (TDDFT_PREC_TF32_IR, _EMU) through the C
boundary: the tcgen05 kind::tf32 GEMM against float64 (operands rounded to
10 mantissa bits: about 2^-11 relative per entry), the TF32 operator against
the oracle's chi0 (relative error stated below), and spectra that the
float64 residual closing every cycle brings to the same tolerance as the
float64 path, checked against the oracle's dense LU (eq. sle)."""
import numpy as np
import pytest

import oracle.tddft_oracle as O
from paper_1005_5340_gb300 import synth
from tests.libutil import ensure_library
from tests.test_gpu_parity import ragged_system, rel

pytestmark = pytest.mark.gpu

# the TF32 operator: four chained tf32 products (step 2, both transforms,
# step 5) and, in A, the K product; each rounds its operands to 2^-11
OP_TOL = 2e-3


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
def test_tf32_gemm_selftest(shape):
    M, N, K = shape
    err = T().selftest_gemm(M, N, K, seed=7, tf32=True)
    print(f"tf32 GEMM {shape}: max error / max |C| = {err:.2e}")
    assert 1e-6 < err < 2e-3, err   # tf32 rounding is visible, and bounded


@pytest.mark.parametrize("sysname", ["tiny4", "ragged"])
def test_tf32_operators_match_oracle(sysname):
    if sysname == "tiny4":
        s, w = synth.workload("tiny4")
        eps = w["eps"]
    else:
        s, eps = ragged_system(), 0.02
    M = O.transition_vertex(s)
    omegas = np.array([0.0, 0.13, 0.5, 0.77, 1.0])
    z = synth.random_complex_vectors(omegas.size, s.n_prod, 9)
    errs = []
    for n_tile in (64, 128, 256):
        with T().Context(s, batch=8, prec="tf32", n_tile=n_tile) as ctx:
            chi = ctx.chi0_apply(z, omegas, eps)
            Az = ctx.apply_A(z, omegas, eps)
        for r, om in enumerate(omegas):
            c = O.chi0_explicit(s, om, eps, M)
            e1 = rel(chi[r], c @ z[r])
            e2 = rel(Az[r] - z[r], -(c @ (s.K @ z[r])))
            errs.append(max(e1, e2))
    print(f"{sysname}: TF32 operator max relative error {max(errs):.2e}")
    assert max(errs) < OP_TOL


def test_tf32_spectrum_reaches_float64_accuracy():
    s, w = synth.workload("tiny4")
    M = O.transition_vertex(s)
    om = w["omega"][::3]
    with T().Context(s, batch=66, restart=w["restart"], tol=1e-11, max_restarts=60,
                     prec="tf32", inner_tol=1e-4) as ctx:
        P, info = ctx.polarizability(om, w["eps"])
    assert info["converged"].all() and np.all(info["resid"] <= 1e-11)
    P_lu = np.stack([O.polarizability_lu(s, x, w["eps"], M)[0] for x in om])
    err = rel(P, P_lu)
    print(f"tf32 spectrum at 1e-11 vs LU: {err:.2e}, cycles max {info['cycles'].max()}")
    assert err < 1e-8
    assert info["cycles"].max() <= 12


@pytest.mark.parametrize("prec", ["tf32", "tf32emu"])
def test_tf32_spectrum_at_workload_tolerance(prec):
    s, w = synth.workload("tiny4")
    M = O.transition_vertex(s)
    om = w["omega"]
    with T().Context(s, batch=192, restart=w["restart"], tol=w["tol"], prec=prec) as ctx:
        P, info = ctx.polarizability(om, w["eps"])
    assert info["converged"].all() and np.all(info["resid"] <= w["tol"])
    P_lu = np.stack([O.polarizability_lu(s, x, w["eps"], M)[0] for x in om])
    im = np.einsum("wii->wi", -P).imag
    im_lu = np.einsum("wii->wi", -P_lu).imag
    assert np.max(np.abs(im - im_lu)) / np.max(np.abs(im_lu)) < 1e-4


@pytest.mark.slow
def test_medium64_tf32emu_against_the_float64_path():
    from tests.test_gpu_emulated import native_residuals
    s, w = synth.workload("medium64")
    om = w["omega"][[5, 128, 250]]
    with T().Context(s, batch=9, restart=w["restart"], tol=w["tol"], prec="tf32emu") as ctx:
        P_t, X, info_t = ctx.polarizability_guess(om, w["eps"])
    P_t, X = P_t.cpu().numpy(), X.cpu().numpy()
    with T().Context(s, batch=9, restart=w["restart"], tol=w["tol"]) as ctx:
        P_64, info_64 = ctx.polarizability(om, w["eps"])
    assert info_t["converged"].all() and info_64["converged"].all()
    r = native_residuals(s, om, w["eps"], X)
    print(f"medium64 tf32emu: native float64 residuals {r}, cycles {info_t['cycles'].mean():.2f}, "
          f"products/RHS {info_t['matvecs'].mean():.1f}")
    assert np.all(r <= 1.01 * w["tol"])
    im_t = np.einsum("wii->wi", -P_t).imag
    im_64 = np.einsum("wii->wi", -P_64).imag
    assert np.max(np.abs(im_t - im_64)) / np.max(np.abs(im_64)) < 1e-4
