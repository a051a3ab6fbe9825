"""Pins for the oracle's poles, adaptive grid and pole fit
(oracle/spectrum_oracle.py): the Casida-form poles against the dense LU solve
and against the K = 0 closed form, the fit against exact one-pole data, and
the grid plus fit against the single-pole closed form of a two-level system
and against a spectrum of known Lorentzians."""
import math

import numpy as np
import pytest

import oracle.spectrum_oracle as SO
import oracle.tddft_oracle as O
from paper_1005_5340_gb300 import synth


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


@pytest.mark.parametrize("omega", [0.0, 0.37, 1.1])
def test_poles_reproduce_the_dense_solve(omega):
    """sum_n g_n / (Omega_n^2 - z^2) from the eigen-decomposition equals -P from
    the dense LU solve of eq. sle: two independent routes."""
    s = synth.tiny_system(5)
    M = O.transition_vertex(s)
    Om, g = SO.casida_poles(s, M)
    a = SO.alpha_from_poles(Om, g, omega, 0.02)[0]
    assert rel(a, -O.polarizability_lu(s, omega, 0.02, M)[0]) < 1e-10
    assert np.all(np.diff(Om) >= 0.0)


def test_zero_kernel_poles_are_the_transition_energies():
    """K = 0: Omega = Delta_ou and g_ii = 2 (n_o - n_u) Delta_ou (d_i . M^ou)^2."""
    s = synth.tiny_system(8)
    s.K = np.zeros_like(s.K)
    M = O.transition_vertex(s)
    Om, g = SO.casida_poles(s, M)
    occ, emp = O.occupied_empty(s)
    E, n = s.eigenvalues, s.occupations
    ref = []
    for a, o in enumerate(occ):
        for b, u in enumerate(emp):
            sd = s.dipole @ M[:, a, b]
            ref.append((E[u] - E[o], 2.0 * (n[o] - n[u]) * (E[u] - E[o]) * sd ** 2))
    ref.sort(key=lambda t: t[0])
    assert np.allclose(Om, [t[0] for t in ref], rtol=0, atol=1e-12)
    gd = np.einsum("nii->ni", g)
    assert np.allclose(gd, np.array([t[1] for t in ref]), rtol=1e-10, atol=1e-14)


def test_fit_is_exact_on_one_pole_and_a_background():
    Omega, g, b, eps = 0.53, 0.21 + 0.0j, 0.04 - 0.013j, 0.01
    w = np.array([0.51, 0.52, 0.53, 0.535, 0.55])
    a = g / (Omega ** 2 - (w + 1j * eps) ** 2) + b
    Om_f, g_f, b_f = SO.fit_pole(w, a, eps)
    assert abs(Om_f - Omega) < 1e-12 and abs(g_f - g) < 1e-12 and abs(b_f - b) < 1e-12


def test_two_level_system_pole_from_the_adaptive_grid():
    """One transition: the only pole is Omega^2 = Delta^2 + 2 n Delta k s^2
    (derived by hand), and alpha is exactly one Lorentzian pair, so the grid
    finds one peak and the fit returns Omega and g = 2 n Delta s^2 d_i^2."""
    theta, v, k, d, eps = 0.3, [[0.7, -0.4], [-0.4, 1.1]], 0.8, 1.5, 0.01
    c, sn = math.cos(theta), math.sin(theta)
    s = synth.System(
        n_atoms=1, atom_orb_offset=np.array([0, 2], dtype=np.int32),
        eigenvalues=np.array([-0.3, 0.2]), occupations=np.array([2.0, 0.0]),
        X=np.array([[c, -sn], [sn, c]]), prod_atoms=np.array([[0, 0]], dtype=np.int32),
        vertex_offset=np.array([0, 4], dtype=np.int64), vertex=np.asarray(v, float).ravel(),
        K=np.array([[k]]), dipole=np.array([[d], [0.5 * d], [-d]]))
    svert = float(np.array([c, sn]) @ np.array(v) @ np.array([-sn, c]))
    Omega = math.sqrt(0.25 + 2 * 2.0 * 0.5 * k * svert ** 2)
    g_tr = 2 * 2.0 * 0.5 * svert ** 2 * (d ** 2 + (0.5 * d) ** 2 + d ** 2) / 3.0
    solve = lambda ws: np.array([O.polarizability_lu(s, x, eps)[0] for x in ws])
    om, P = SO.adaptive_grid(solve, 0.3, 1.2, 10, 200, 0.01, eps / 8)
    poles = SO.extract_poles(om, P, eps, 0.01)
    assert len(poles) == 1
    Om_f, g_f, _, w_pk = poles[0]
    assert abs(Om_f - Omega) < 1e-9 and abs(g_f - g_tr) < 1e-9 * g_tr
    assert abs(w_pk - Omega) < eps
    # refinement concentrates on the peak
    near = om[np.abs(om - Omega) < 2 * eps]
    assert np.min(np.diff(near)) <= eps / 4 and np.max(np.diff(om)) >= 0.045


def test_known_lorentzians_are_recovered():
    Om = np.array([0.31, 0.62, 0.97])
    gk = np.array([0.2, 0.5, 0.1])
    G = gk[:, None, None] * np.eye(3)[None]
    eps = 0.01
    solve = lambda w: -SO.alpha_from_poles(Om, G, w, eps)
    om, P = SO.adaptive_grid(solve, 0.0, 1.2, 25, 400, 0.01, eps / 8)
    poles = SO.extract_poles(om, P, eps, 0.01)
    assert len(poles) == 3
    for (Om_f, g_f, _, _), Om_t, g_t in zip(poles, Om, gk):
        # the other peaks' tails are only approximately the fit's constant background
        assert abs(Om_f - Om_t) < 5e-3 * eps
        assert abs(g_f - g_t) < 0.05 * g_t
    assert len(om) < 200


def test_grid_respects_its_point_budget():
    Om = np.array([0.31, 0.62, 0.97])
    G = np.array([0.2, 0.5, 0.1])[:, None, None] * np.eye(3)[None]
    solve = lambda w: -SO.alpha_from_poles(Om, G, w, 0.01)
    om, _ = SO.adaptive_grid(solve, 0.0, 1.2, 25, 60, 1e-4, 1e-4)
    assert len(om) == 60 and np.all(np.diff(om) > 0)


def test_refinement_stops_at_the_floating_point_resolution():
    """With no tolerance to stop it, the rule still ends: an interval whose
    midpoint rounds onto one of its ends is not split again."""
    Om = np.array([0.31])
    G = np.array([0.2])[:, None, None] * np.eye(3)[None]
    solve = lambda w: -SO.alpha_from_poles(Om, G, w, 0.01)
    om, _ = SO.adaptive_grid(solve, 0.30, 0.30 + 4e-15, 3, 10 ** 6, 1e-300, 0.0)
    assert len(om) < 100 and np.all(np.diff(om) > 0)
