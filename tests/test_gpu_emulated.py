"""Float64 products emulated on the tensor cores (integer slices, the
TDDFT_PREC_*_EMU forms) through the C boundary: the standalone GEMM against
float64 products (inside its stated error bound, improving with the number
of slices, exact on integer operands over many K chunks), the emulated
float64 operator against the oracle, spectra against the oracle's dense LU,
and the refinement form with emulated residuals against the native float64
path, its final residuals re-checked with native float64 products."""
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


def gemm(A, B, s=6, lda_pad=0):
    import torch
    Ad = torch.zeros((A.shape[0], A.shape[1] + lda_pad), dtype=torch.float64, device="cuda")
    Ad[:, :A.shape[1]] = torch.from_numpy(A)
    Ad = Ad[:, :A.shape[1]]
    C = T().gemm_f64_emulated(Ad, torch.from_numpy(np.ascontiguousarray(B)).cuda(), s)
    return C.cpu().numpy()


def scale(A, B):
    """2^eA_m 2^eB_n K with |A_mk| < 2^eA_m over row m, |B_kn| < 2^eB_n over column n."""
    eA = np.frexp(np.max(np.abs(A), axis=1))[1]
    eB = np.frexp(np.max(np.abs(B), axis=0))[1]
    return np.ldexp(1.0, eA)[:, None] * np.ldexp(1.0, eB)[None, :] * A.shape[1]


def operands(M, N, K, seed, spread=3.0):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(M, K)) * 10.0 ** rng.uniform(-spread, spread, size=(M, 1))
    B = rng.normal(size=(K, N)) * 10.0 ** rng.uniform(-spread, spread, size=(1, N))
    return A, B


@pytest.mark.parametrize("shape", [(128, 64, 64), (300, 70, 1000), (704, 1030, 832),
                                   (1000, 129, 9080)])
def test_emulated_gemm_within_its_bound(shape):
    M, N, K = shape
    A, B = operands(M, N, K, sum(shape))
    ref = A @ B
    C = gemm(A, B, 6, lda_pad=3)
    # stated bound plus the float64 reference's own rounding
    bound = (1 + 7 / 4) * 2.0 ** -42 * scale(A, B) + K * 2.0 ** -52 * (np.abs(A) @ np.abs(B))
    err = np.abs(C - ref)
    print(f"{shape}: max error / scale {np.max(err / scale(A, B)):.2e}")
    assert np.all(err <= bound)


def test_emulated_gemm_improves_with_the_number_of_slices():
    A, B = operands(256, 96, 2000, 3, spread=1.0)
    ref = A @ B
    e = {}
    for s in range(3, 9):
        C = gemm(A, B, s)
        e[s] = float(np.max(np.abs(C - ref) / scale(A, B)))
        assert e[s] <= (1 + (s + 1) / 4) * 2.0 ** (-7 * s) + 2000 * 2.0 ** -52
    print("max error / scale by slices:", {k: f"{v:.1e}" for k, v in e.items()})
    for s in range(3, 6):
        assert e[s + 1] < e[s] / 16


def test_emulated_gemm_is_exact_on_integer_operands():
    """Every slice product is summed exactly: integer operands of 10 bits over
    4160 = 8.1 chunks of K, and operands whose slices all sit at the largest
    values (x = 2^e (1 - 2^-8) gives q_1 = 128, q_2 = -64)."""
    rng = np.random.default_rng(5)
    A = rng.integers(-1023, 1024, size=(257, 4160)).astype(float)
    B = rng.integers(-1023, 1024, size=(4160, 100)).astype(float)
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(float)
    assert np.array_equal(gemm(A, B, 6), exact)
    assert np.array_equal(gemm(A, B, 3), exact)
    x = 1.0 - 2.0 ** -8
    A = np.full((130, 4096), x)
    B = np.full((4096, 70), -x)
    assert np.array_equal(gemm(A, B, 6), np.full((130, 70), -4096 * x * x))


def test_emulated_gemm_zero_rows_and_columns():
    A, B = operands(200, 80, 300, 9, spread=0.5)
    A[17] = 0.0
    B[:, 5] = 0.0
    C = gemm(A, B)
    assert np.all(C[17] == 0.0) and np.all(C[:, 5] == 0.0)
    assert rel(C, A @ B) < 1e-11


@pytest.mark.parametrize("sysname", ["tiny4", "ragged"])
def test_emulated_operators_match_oracle(sysname):
    if sysname == "tiny4":
        s, w = synth.workload("tiny4")
        eps = w["eps"]
    else:
        s, eps = ragged_system(), 0.02
    M = O.transition_vertex(s)
    omegas = np.array([0.0, 0.13, 0.5, 0.77, 1.0])
    z = synth.random_complex_vectors(omegas.size, s.n_prod, 9)
    with T().Context(s, batch=8, prec="fp64emu") as ctx:
        chi = ctx.chi0_apply(z, omegas, eps)
        Az = ctx.apply_A(z, omegas, eps)
        Kz = ctx.kernel_apply(z)
    assert rel(Kz, (s.K @ z.T).T) < 1e-11
    for r, om in enumerate(omegas):
        c = O.chi0_explicit(s, om, eps, M)
        assert rel(chi[r], c @ z[r]) < 1e-11
        ref = z[r] - c @ (s.K @ z[r])
        assert rel(Az[r] - z[r], ref - z[r]) < 1e-11


def test_emulated_float64_spectrum_matches_dense_lu():
    s, w = synth.workload("tiny4")
    M = O.transition_vertex(s)
    om = w["omega"][::4]
    with T().Context(s, batch=48, restart=w["restart"], tol=1e-12, max_restarts=40,
                     prec="fp64emu") as ctx:
        P, info = ctx.polarizability(om, w["eps"])
    assert info["converged"].all()
    P_lu = np.stack([O.polarizability_lu(s, x, w["eps"], M)[0] for x in om])
    err = rel(P, P_lu)
    print(f"fp64emu spectrum vs LU: {err:.2e}")
    assert err < 1e-9


def test_refinement_with_emulated_residuals_reaches_float64_accuracy():
    s, w = synth.workload("tiny4")
    M = O.transition_vertex(s)
    om = w["omega"][::3]
    with T().Context(s, batch=66, restart=w["restart"], tol=1e-11, max_restarts=60,
                     prec="bf16x3emu", inner_tol=1e-4) as ctx:
        P, info = ctx.polarizability(om, w["eps"])
    assert info["converged"].all() and np.all(info["resid"] <= 1e-11)
    P_lu = np.stack([O.polarizability_lu(s, x, w["eps"], M)[0] for x in om])
    assert rel(P, P_lu) < 1e-8
    assert info["cycles"].max() <= 6


def native_residuals(s, om, eps, X):
    """||b - A x|| / ||b|| per (omega, direction) with native float64 products."""
    n = om.size
    rows = np.repeat(om, 3)
    D = np.tile(s.dipole.astype(complex), (n, 1))
    with T().Context(s, batch=3 * n) as ctx:
        b = ctx.chi0_apply(D, rows, eps)
        Ax = ctx.apply_A(X, rows, eps)
    return np.linalg.norm(b - Ax, axis=1) / np.linalg.norm(b, axis=1)


@pytest.mark.slow
def test_medium64_refinement_with_emulated_residuals():
    s, w = synth.workload("medium64")
    om = w["omega"][[5, 128, 250]]
    with T().Context(s, batch=9, restart=w["restart"], tol=w["tol"], prec="bf16x3emu") as ctx:
        P_e, X, info_e = ctx.polarizability_guess(om, w["eps"])
    P_e, X = P_e.cpu().numpy(), X.cpu().numpy()
    with T().Context(s, batch=9, restart=w["restart"], tol=w["tol"]) as ctx:
        P_64, info_64 = ctx.polarizability(om, w["eps"])
    assert info_e["converged"].all() and info_64["converged"].all()
    r = native_residuals(s, om, w["eps"], X)
    print(f"medium64: native float64 residuals of the emulated-residual solutions {r}")
    assert np.all(r <= 1.01 * w["tol"])
    im_e = np.einsum("wii->wi", -P_e).imag
    im_64 = np.einsum("wii->wi", -P_64).imag
    assert np.max(np.abs(im_e - im_64)) / np.max(np.abs(im_64)) < 1e-4
