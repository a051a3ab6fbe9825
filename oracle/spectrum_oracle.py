"""CPU oracle for the adaptive frequency grid and pole extraction (test
infrastructure).

THIS MODULE IS TEST INFRASTRUCTURE.  Only the tests, the package's smoke check
and the CPU legs of the benchmark may import it; the product path never calls
it and it shares no code with the library.

The paper names an adaptive frequency grid and the positions and residues of
the poles of the spectrum as its next step (Sec. 8, conclusions).  What is
computed here:

* ``casida_poles``     -- the exact poles and residues of the synthetic model.
  With z = omega + i eps the merged pair factor of eq. response-mat is
  D_ou(z) = w_ou / (z^2 - Delta_ou^2), w_ou = 2 (n_o - n_u) Delta_ou, so the
  transition-space form of eq. eqpolarizability,
      P(z) = s^T (D^-1 - M^T K M)^-1 s,   s_i = M^T d_i,
  equals s^T W^1/2 (z^2 - C)^-1 W^1/2 s with the symmetric matrix
  C = Delta^2 + W^1/2 M^T K M W^1/2.  With C = U Omega^2 U^T,
      alpha_ik(omega) = -P_ik = sum_n g_n,ik / (Omega_n^2 - z^2),
      g_n,ik = (u_n . W^1/2 s_i) (u_n . W^1/2 s_k).
* ``alpha_from_poles`` -- that sum at given frequencies.
* ``fit_pole``         -- one pole and a constant background,
  a(z) = g / (p - z^2) + b, fitted to complex samples by linear least squares
  in (p, b, q = g + b p): a p + z^2 b - q = a z^2.
* ``adaptive_grid``    -- the refinement rule: a uniform start, then rounds that
  solve the midpoints of the flagged intervals and flag both halves again
  where the midpoint's absorption departs from the linear interpolation of
  its ends by more than rel_tol times the largest absorption seen.
* ``extract_poles``    -- local maxima of the absorption on the final grid,
  each fitted on its five nearest grid points.

The absorption is S(omega) = Im alpha_tr(omega), alpha_tr = -tr P / 3.
"""
from __future__ import annotations

import numpy as np

from oracle.tddft_oracle import occupied_empty, transition_vertex


def casida_poles(sysm, M=None):
    """Exact poles Omega_n (ascending) and residues g [n, 3, 3] of alpha = -P."""
    M = transition_vertex(sysm) if M is None else M
    occ, emp = occupied_empty(sysm)
    E, n = sysm.eigenvalues, sysm.occupations
    pairs = [(o, u) for o in occ for u in emp]
    delta = np.array([E[u] - E[o] for o, u in pairs])
    w = np.array([2.0 * (n[o] - n[u]) * (E[u] - E[o]) for o, u in pairs])
    Mf = M.reshape(sysm.n_prod, len(pairs))
    sw = np.sqrt(w)
    C = np.diag(delta ** 2) + (sw[:, None] * (Mf.T @ sysm.K @ Mf)) * sw[None, :]
    lam, U = np.linalg.eigh(C)
    S = Mf.T @ sysm.dipole.T                  # [n_trans, 3]
    amp = U.T @ (sw[:, None] * S)             # u_n . W^1/2 s_i
    g = amp[:, :, None] * amp[:, None, :]
    return np.sqrt(lam), g


def alpha_from_poles(Omega, g, omegas, eps):
    """alpha_ik(omega) = sum_n g_n,ik / (Omega_n^2 - (omega + i eps)^2)."""
    z2 = (np.atleast_1d(omegas) + 1j * eps) ** 2
    den = Omega[None, :] ** 2 - z2[:, None]
    return np.einsum("wn,nik->wik", 1.0 / den, g)


def fit_pole(omegas, a, eps):
    """Least-squares (Omega, g, b) of a(z) = g / (Omega^2 - z^2) + b.
    Returns (Omega, g, b) with Omega = sqrt(Re p) and g = q - b p."""
    z2 = (np.asarray(omegas) + 1j * eps) ** 2
    a = np.asarray(a, dtype=complex)
    A = np.stack([a, z2, -np.ones_like(a)], axis=1)
    p, b, q = np.linalg.lstsq(A, a * z2, rcond=None)[0]
    return float(np.sqrt(max(p.real, 0.0))), q - b * p, b


def absorption(P):
    """S(omega) = Im alpha_tr = Im(-tr P / 3) for P [n, 3, 3]."""
    return -np.einsum("wii->w", P).imag / 3.0


def adaptive_grid(solve, w_lo, w_hi, n_initial, max_points, rel_tol, min_step):
    """The refinement rule; solve(omegas) -> P [n, 3, 3].  Returns (omega
    ascending, P).  A round solves the midpoints of all flagged intervals
    (longer than 2 min_step) in one call, in ascending order, while the grid
    has room; an interval is flagged again, both halves, when
    |S(mid) - (S(left) + S(right)) / 2| > rel_tol max|S|."""
    om = list(np.linspace(w_lo, w_hi, n_initial))
    Ps = list(solve(np.array(om)))
    S = {w: s for w, s in zip(om, absorption(np.array(Ps)))}
    Pd = {w: p for w, p in zip(om, Ps)}
    flagged = list(zip(om[:-1], om[1:]))
    while flagged and len(S) < max_points:
        flagged = [iv for iv in flagged if iv[1] - iv[0] > 2.0 * min_step]
        # an interval whose midpoint rounds onto a grid point cannot be split
        flagged = [iv for iv in flagged if 0.5 * (iv[0] + iv[1]) not in S]
        flagged = flagged[:max_points - len(S)]
        if not flagged:
            break
        mids = np.array([0.5 * (l + r) for l, r in flagged])
        Pm = solve(mids)
        Sm = absorption(Pm)
        for w, s, p in zip(mids, Sm, Pm):
            S[w] = s
            Pd[w] = p
        scale = max(abs(v) for v in S.values())
        nxt = []
        for (l, r), w, s in zip(flagged, mids, Sm):
            if abs(s - 0.5 * (S[l] + S[r])) > rel_tol * scale:
                nxt += [(l, w), (w, r)]
        flagged = nxt
    keys = sorted(S)
    return np.array(keys), np.array([Pd[w] for w in keys])


def extract_poles(omegas, P, eps, peak_floor):
    """(Omega, g, peak, omega_peak) for each local maximum of S above
    peak_floor max S, fitted on the five nearest grid points of alpha_tr."""
    S = absorption(P)
    a_tr = -np.einsum("wii->w", P) / 3.0
    top = S.max()
    out = []
    n = len(omegas)
    for i in range(n):
        left = S[i - 1] if i > 0 else -np.inf
        right = S[i + 1] if i + 1 < n else -np.inf
        if S[i] > left and S[i] >= right and S[i] > peak_floor * top:
            lo = min(max(0, i - 2), max(0, n - 5))
            sl = slice(lo, min(n, lo + 5))
            Om, g, _ = fit_pole(omegas[sl], a_tr[sl], eps)
            out.append((Om, g, S[i], omegas[i]))
    return out
