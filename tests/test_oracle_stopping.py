"""Pins for the oracle's implementation of the paper's stopping criterion
(Sec. 4.1: eps_P = |A^-1| |<d|r>| / |P|, eps_X = |A^-1| |r| / |X| with |A^-1|
the Frobenius norm of the inverse of the Krylov representation of A).

Each test ties the oracle to something outside it: the first GMRES step of a
2 x 2 diagonal system worked out by hand, the Frobenius norm of A^-1 itself
once the Krylov space is the whole space, and the ordering of the two rules
that follows from their definitions."""
import math

import numpy as np
import pytest

import oracle.tddft_oracle as O
from paper_1005_5340_gb300 import synth


def test_first_step_of_a_diagonal_two_by_two_by_hand():
    """A = diag(l1, l2), b = (b1, b2), d = (d1, d2).  After one Arnoldi step
    the Krylov representation of A is the 1 x 1 matrix h = <v0|A|v0>, so
    |A^-1| ~ 1/|h| (not 1/sqrt(|h|^2 + h_10^2), the rotated diagonal); the
    iterate is x = y v0 with y the least-squares solution of
    [h; h_10] y = [beta; 0]."""
    l1, l2 = 0.7 + 0.2j, -1.9 + 0.05j
    b1, b2 = 0.6 - 0.3j, 1.1 + 0.4j
    d = np.array([0.8, -1.3])
    beta = math.sqrt(abs(b1) ** 2 + abs(b2) ** 2)
    h = (abs(b1) ** 2 * l1 + abs(b2) ** 2 * l2) / beta ** 2
    # A v0 - h v0, componentwise
    w1, w2 = (l1 - h) * b1 / beta, (l2 - h) * b2 / beta
    h10 = math.sqrt(abs(w1) ** 2 + abs(w2) ** 2)
    y = beta * np.conj(h) / (abs(h) ** 2 + h10 ** 2)
    x1, x2 = y * b1 / beta, y * b2 / beta
    r1, r2 = b1 - l1 * x1, b2 - l2 * x2
    F = 1.0 / abs(h)
    eps_p = F * abs(d[0] * r1 + d[1] * r2) / abs(d[0] * x1 + d[1] * x2)
    eps_x = F * math.sqrt(abs(r1) ** 2 + abs(r2) ** 2) / math.sqrt(abs(x1) ** 2 + abs(x2) ** 2)

    A = np.diag([l1, l2])
    _, info = O.gmres(lambda z: A @ z, np.array([b1, b2]), restart=2, tol=1e-300,
                      max_restarts=1, stop="eps_px", d=d, trace=True)
    cycle, j, F_o, ep_o, ex_o = info["trace"][0]
    assert (cycle, j) == (0, 0)
    assert abs(F_o - F) <= 1e-13 * F
    assert abs(ep_o - eps_p) <= 1e-12 * eps_p
    assert abs(ex_o - eps_x) <= 1e-12 * eps_x


def test_full_krylov_space_gives_the_frobenius_norm_of_the_inverse():
    """With restart = n the last step's Krylov representation is V^H A V for a
    unitary V, so its inverse has the Frobenius norm of A^-1 (numpy's inverse
    of A itself); the iterate is then exact and both estimates vanish."""
    rng = np.random.default_rng(11)
    n = 6
    A = np.eye(n) + 0.35 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    d = rng.standard_normal(n)
    _, info = O.gmres(lambda z: A @ z, b, restart=n, tol=0.0, max_restarts=1,
                      stop="eps_px", d=d, trace=True)
    last = info["trace"][n - 1]
    assert last[1] == n - 1
    ref = np.linalg.norm(np.linalg.inv(A), "fro")
    assert abs(last[2] - ref) <= 1e-10 * ref
    assert last[3] < 1e-11 and last[4] < 1e-11


def test_estimates_reduce_to_the_ratio_definitions():
    """error_estimates is the paper's pair of ratios, including the reading
    0 / 0 = 0 and num / 0 = infinity."""
    d = np.array([1.0, 2.0])
    r = np.array([0.3j, -0.1])
    x = np.array([1.0 + 1j, 0.5])
    ep, ex = O.error_estimates(2.0, r, x, d)
    assert ep == pytest.approx(2.0 * abs(0.3j - 0.2) / abs(1.0 + 1j + 1.0))
    assert ex == pytest.approx(2.0 * math.sqrt(0.09 + 0.01) / math.sqrt(2.0 + 0.25))
    assert O.error_estimates(5.0, np.zeros(2), x, d) == (0.0, 0.0)
    assert O.error_estimates(5.0, r, np.zeros(2), d) == (math.inf, math.inf)


def test_combined_rule_never_stops_before_the_eps_p_rule():
    """eps_px requires eps_P <= tol and eps_X <= tol, so on the same Krylov
    path it ends no earlier than eps_p, and both converge."""
    s = synth.workload_system("tiny4")
    op = O.StepOperator(s)
    for w in (0.0, 0.31, 0.77):
        _, i_p = O.polarizability_gmres(s, [w], 0.01, 30, 1e-2, stop="eps_p", op=op)
        _, i_px = O.polarizability_gmres(s, [w], 0.01, 30, 1e-2, stop="eps_px", op=op)
        for a, c in zip(i_p, i_px):
            assert a["converged"] and c["converged"]
            assert a["matvecs"] <= c["matvecs"]
            assert a["eps_p"] <= 1e-2 and c["eps_p"] <= 1e-2 and c["eps_x"] <= 1e-2


def test_combined_rule_bounds_the_error_of_p_on_tiny4():
    """The paper's claim for the combined rule: P is reliable at the
    tolerance.  On the 4-atom system at 1% the relative error of every
    diagonal P_kk against the dense LU solve stays below the tolerance."""
    s = synth.workload_system("tiny4")
    op = O.StepOperator(s)
    for w in np.linspace(0.0, 1.0, 6):
        P_lu = O.polarizability_lu(s, w, 0.01)[0]
        P, infos = O.polarizability_gmres(s, [w], 0.01, 30, 1e-2, stop="eps_px", op=op)
        for k in range(3):
            assert abs(P[0, k, k] - P_lu[k, k]) <= 1e-2 * abs(P_lu[k, k])


def test_unknown_rule_is_rejected():
    with pytest.raises(ValueError):
        O.gmres(lambda z: z, np.ones(2), 2, 1e-6, stop="eps")
