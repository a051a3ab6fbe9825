"""Pins for the CPU oracle: each test ties it to something other than
itself -- a literal term-by-term sum, a closed form derived by hand, an
identity from linear algebra, an invariant of the physics, or an
independent library routine -- so that a dropped term, a wrong sign, a wrong
index or a transposed operand in the oracle fails at least one of them."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle.tddft_oracle as O
from paper_1005_5340_gb300 import synth


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b))


TINY_SEEDS = [3, 5, 8]


@pytest.mark.parametrize("seed", TINY_SEEDS)
@pytest.mark.parametrize("omega", [0.0, 0.37, 1.2])
def test_chi0_explicit_matches_term_by_term_sum(seed, omega):
    """eq. response-mat summed over every ordered (E, F) with pure loops
    pins the merged pair factor D and the transition vertex M."""
    s = synth.tiny_system(seed)
    brute = O.chi0_brute(s, omega, 0.03)
    assert rel(O.chi0_explicit(s, omega, 0.03), brute) < 1e-12


def test_chi0_brute_with_fractional_step_occupations():
    """Same check with occupations 1 on occupied states (open-shell-like
    step profile): the (n_o - n_u) factor must follow."""
    s = synth.tiny_system(4, n_atoms=2, orb_per_atom=3, occ_per_atom=1)
    s.occupations = np.where(s.occupations > 0, 1.0, 0.0)
    assert rel(O.chi0_explicit(s, 0.4, 0.02), O.chi0_brute(s, 0.4, 0.02)) < 1e-12


@pytest.mark.parametrize("seed", TINY_SEEDS)
def test_five_step_apply_matches_explicit(seed):
    s = synth.tiny_system(seed, n_atoms=3, orb_per_atom=3, occ_per_atom=1, density=0.02)
    z = synth.random_complex_vectors(1, s.n_prod, seed)[0]
    for omega in (0.0, 0.25, 0.9):
        ref = O.chi0_explicit(s, omega, 0.02) @ z
        assert rel(O.chi0_apply_steps(s, z, omega, 0.02), ref) < 1e-12


def test_five_step_apply_matches_explicit_tiny4():
    s, w = synth.workload("tiny4")
    M = O.transition_vertex(s)
    op = O.StepOperator(s)
    z = synth.random_complex_vectors(2, s.n_prod, 17)
    for omega in (0.0, 0.5, 1.0):
        chi = O.chi0_explicit(s, omega, w["eps"], M)
        for k in range(2):
            assert rel(op.apply(z[k], omega, w["eps"]), chi @ z[k]) < 1e-12


def _brute_oscillator_strength(s):
    """s_k^{ou} = sum_mu d_k^mu X_a^o V_mu^{ab} X_b^u with explicit loops."""
    V = O.dense_vertex(s)
    occ, emp = O.occupied_empty(s)
    S = np.zeros((3, occ.size, emp.size))
    for k in range(3):
        for i, o in enumerate(occ):
            for j, u in enumerate(emp):
                acc = 0.0
                for mu in range(s.n_prod):
                    for a in range(s.n_orb):
                        for b in range(s.n_orb):
                            acc += s.dipole[k, mu] * s.X[a, o] * V[mu, a, b] * s.X[b, u]
                S[k, i, j] = acc
    return S


@pytest.mark.parametrize("omega", [0.0, 0.3, 0.8])
def test_zero_kernel_is_a_sum_of_lorentzians(omega):
    """K = 0: alpha_ik = -P_ik = sum_ou f^{ik}_ou / (Delta_ou^2 - (omega + i eps)^2),
    f^{ik}_ou = 2 n_o Delta_ou s_i^{ou} s_k^{ou}."""
    s = synth.tiny_system(6)
    s.K = np.zeros_like(s.K)
    eps = 0.02
    S = _brute_oscillator_strength(s)
    occ, emp = O.occupied_empty(s)
    delta = s.eigenvalues[emp][None, :] - s.eigenvalues[occ][:, None]
    n = s.occupations[occ][:, None]
    w = complex(omega, eps)
    alpha = np.zeros((3, 3), dtype=complex)
    for i in range(3):
        for k in range(3):
            alpha[i, k] = np.sum(2 * n * delta * S[i] * S[k] / (delta ** 2 - w ** 2))
    P_lu, _ = O.polarizability_lu(s, omega, eps)
    assert rel(-P_lu, alpha) < 1e-12
    P_g, infos = O.polarizability_gmres(s, [omega], eps, restart=10, tol=1e-14)
    assert all(i["converged"] for i in infos)
    assert rel(-P_g[0], alpha) < 1e-12


def _two_level_system(theta, v, k, d, n_occ_val=2.0):
    """One atom, two orbitals, one product: X a rotation, V a symmetric 2x2."""
    c, sn = math.cos(theta), math.sin(theta)
    return synth.System(
        n_atoms=1, atom_orb_offset=np.array([0, 2], dtype=np.int32),
        eigenvalues=np.array([-0.3, 0.2]), occupations=np.array([n_occ_val, 0.0]),
        X=np.array([[c, -sn], [sn, c]]), prod_atoms=np.array([[0, 0]], dtype=np.int32),
        vertex_offset=np.array([0, 4], dtype=np.int64), vertex=np.asarray(v, float).ravel(),
        K=np.array([[k]]), dipole=np.array([[d], [0.5 * d], [-d]]))


@pytest.mark.parametrize("omega", [0.0, 0.41, 0.5, 0.55, 1.3])
def test_two_level_single_pole_closed_form(omega):
    """Single transition, single product: P = d_i d_k c0 / (1 - k c0) with
    c0 = 2 n Delta s^2 / ((omega + i eps)^2 - Delta^2), i.e. one pole at
    Omega^2 = Delta^2 + 2 n Delta k s^2 (the single-pole approximation).
    Evaluated in exact rational arithmetic."""
    theta, v, k, d, eps = 0.3, [[0.7, -0.4], [-0.4, 1.1]], 0.8, 1.5, 0.01
    s = _two_level_system(theta, v, k, d)
    c, sn = math.cos(theta), math.sin(theta)
    x0 = np.array([c, sn])
    x1 = np.array([-sn, c])
    svert = float(x0 @ np.array(v) @ x1)
    delta, n = 0.5, 2.0
    # exact evaluation of the closed form in rationals (re, im pairs)
    F = Fraction
    wr, wi = F(omega), F(eps)
    den_r = wr * wr - wi * wi - F(delta) ** 2 - F(2 * n * delta * k) * F(svert) ** 2
    den_i = 2 * wr * wi
    num = F(2 * n * delta) * F(svert) ** 2
    mag = den_r * den_r + den_i * den_i
    p_unit = complex(float(num * den_r / mag), float(-num * den_i / mag))
    dvec = s.dipole[:, 0]
    P_exact = p_unit * np.outer(dvec, dvec)
    P_lu, _ = O.polarizability_lu(s, omega, eps)
    assert rel(P_lu, P_exact) < 1e-12
    P_t = O.polarizability_transition(s, omega, eps)
    assert rel(P_t, P_exact) < 1e-12


def test_two_level_peak_sits_at_the_shifted_pole():
    theta, v, k, d, eps = 0.3, [[0.7, -0.4], [-0.4, 1.1]], 0.8, 1.5, 1e-3
    s = _two_level_system(theta, v, k, d)
    c, sn = math.cos(theta), math.sin(theta)
    svert = float(np.array([c, sn]) @ np.array(v) @ np.array([-sn, c]))
    Omega = math.sqrt(0.25 + 2 * 2.0 * 0.5 * k * svert ** 2)
    grid = np.linspace(0.3, 1.2, 9001)
    im = [-(O.polarizability_lu(s, w, eps)[0][0, 0]).imag for w in grid]
    assert abs(grid[int(np.argmax(im))] - Omega) < 2e-4


def test_invariants_symmetry_static_limit_and_absorption_sign():
    """chi0 = chi0^T; P_ik = P_ki; P(0) real; Im alpha_ii >= 0 for omega > 0
    for any real symmetric kernel, here an indefinite random one."""
    s = synth.make_system(3, 21, orb_per_atom=4, occ_per_atom=1, n_local=5, n_bilocal=3,
                          density=0.02)
    rng = synth.CounterRNG(99, 1)
    G = rng.normal(s.n_prod ** 2).reshape(s.n_prod, s.n_prod)
    M = O.transition_vertex(s)
    for K in (s.K, 0.3 * (G + G.T)):
        s.K = K
        for omega in (0.0, 0.2, 0.45, 0.9):
            chi = O.chi0_explicit(s, omega, 0.02, M)
            assert rel(chi, chi.T) < 1e-13
            P, _ = O.polarizability_lu(s, omega, 0.02, M)
            assert rel(P, P.T) < 1e-10
            if omega == 0.0:
                assert np.max(np.abs(P.imag)) <= 1e-12 * np.max(np.abs(P))
            else:
                assert np.all(-np.diag(P).imag >= -1e-12 * np.max(np.abs(P)))


@pytest.mark.parametrize("omega", [0.0, 0.33, 0.71])
def test_transition_space_identity_matches_product_space_lu(omega):
    s, w = synth.workload("tiny4")
    M = O.transition_vertex(s)
    P, X = O.polarizability_lu(s, omega, w["eps"], M)
    assert rel(O.polarizability_transition(s, omega, w["eps"], M), P) < 1e-10
    chi = O.chi0_explicit(s, omega, w["eps"], M)
    A = np.eye(s.n_prod) - chi @ s.K
    for k in range(3):
        b = chi @ s.dipole[k]
        assert np.linalg.norm(A @ X[k] - b) / np.linalg.norm(b) < 1e-13


def test_gmres_terminates_exactly_with_full_krylov_space():
    s = synth.tiny_system(9, n_atoms=2, orb_per_atom=4, occ_per_atom=1, n_local=4, n_bilocal=3)
    P_lu, X_lu = O.polarizability_lu(s, 0.37, 0.02)
    op = O.StepOperator(s)
    for k in range(3):
        b = op.apply(s.dipole[k].astype(complex), 0.37, 0.02)
        x, info = O.gmres(lambda z: O.apply_A(s, op, z, 0.37, 0.02), b,
                          restart=s.n_prod, tol=0.0, max_restarts=1)
        assert info["matvecs"] <= s.n_prod + 1
        assert rel(x, X_lu[k]) < 1e-10


def test_gmres_against_scipy_on_a_nonnormal_matrix():
    sp = pytest.importorskip("scipy.sparse.linalg")
    n = 60
    rng = synth.CounterRNG(5, 2)
    A = np.eye(n) * 3 + (rng.normal(n * n).reshape(n, n) + 1j * rng.normal(n * n).reshape(n, n)) / math.sqrt(n)
    b = rng.normal(n) + 1j * rng.normal(n)
    x, info = O.gmres(lambda z: A @ z, b, restart=8, tol=1e-12)
    assert info["converged"]
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 1e-12
    xs, flag = sp.gmres(A, b, restart=8, rtol=1e-12, maxiter=500)
    assert flag == 0
    assert rel(x, xs) < 1e-9
    assert rel(x, np.linalg.solve(A, b)) < 1e-10


def test_gmres_reports_non_convergence():
    n = 40
    A = np.diag(np.linspace(1, 1e4, n)).astype(complex)
    b = np.ones(n, dtype=complex)
    x, info = O.gmres(lambda z: A @ z, b, restart=2, tol=1e-14, max_restarts=3)
    assert not info["converged"] and info["resid"] > 1e-14


def test_gmres_spectrum_matches_lu_on_tiny4():
    s, w = synth.workload("tiny4")
    M = O.transition_vertex(s)
    om = w["omega"][[0, 17, 40, 63]]
    P_g, infos = O.polarizability_gmres(s, om, w["eps"], w["restart"], 1e-13)
    assert all(i["converged"] for i in infos)
    for t, omega in enumerate(om):
        P_lu, _ = O.polarizability_lu(s, omega, w["eps"], M)
        assert rel(P_g[t], P_lu) < 1e-10


def test_planted_mistakes_are_caught(monkeypatch):
    """Each planted error in the oracle breaks at least one pin above."""
    s = synth.tiny_system(3)
    brute = O.chi0_brute(s, 0.37, 0.03)
    good = O.pair_factor

    def wrong_sign(sysm, omega, eps):           # second term with + instead of -
        occ, emp = O.occupied_empty(sysm)
        E, n = sysm.eigenvalues, sysm.occupations
        dn = n[occ][:, None] - n[emp][None, :]
        d = E[emp][None, :] - E[occ][:, None]
        wc = omega + 1j * eps
        return dn * (1.0 / (wc - d) + 1.0 / (wc + d))

    def dropped_term(sysm, omega, eps):
        occ, emp = O.occupied_empty(sysm)
        E, n = sysm.eigenvalues, sysm.occupations
        d = E[emp][None, :] - E[occ][:, None]
        return (n[occ][:, None] - n[emp][None, :]) / (omega + 1j * eps - d)

    for bad in (wrong_sign, dropped_term):
        monkeypatch.setattr(O, "pair_factor", bad)
        assert rel(O.chi0_explicit(s, 0.37, 0.03), brute) > 1e-3
    monkeypatch.setattr(O, "pair_factor", good)

    # transposed X inside the transition vertex
    real_tv = O.transition_vertex
    Xt = s.X.T.copy()
    s2 = synth.tiny_system(3)
    s2.X = Xt
    assert rel(O.chi0_explicit(s, 0.37, 0.03, real_tv(s2)), brute) > 1e-3
