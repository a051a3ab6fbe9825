"""CPU oracle for the iterative polarizability solve (test infrastructure).

THIS MODULE IS TEST INFRASTRUCTURE.  Only the tests, the package's smoke
check and the CPU-baseline leg of the benchmark may import it.  The product
path never calls it and it shares no code with the CUDA path: it reads a
synthetic ``System`` (plain numpy arrays) and computes everything in float64
/ complex128 with plain numpy.

What it computes (paper: Koval, Foerster, Coulaud, arXiv:1005.5340):

* ``dense_vertex``       -- V_mu^{ab} as dense symmetric matrices (Sec. 3,
                            eq. vertex-ansatz; the B x A mirror of a bilocal
                            block is implied by the symmetry of f^a f^b).
* ``transition_vertex``  -- M_mu^{EF} = X_a^E V_mu^{ab} X_b^F, the factor of
                            eq. response-mat, for E occupied and F empty.
* ``pair_factor``        -- D_EF(omega): the two terms of eq. response-mat for
                            the ordered pairs (E,F) and (F,E), merged.
* ``chi0_brute``         -- eq. response-mat summed literally over all E, F
                            with pure-Python loops (tiny inputs only).
* ``chi0_explicit``      -- chi0 = M diag(D) M^T.
* ``chi0_apply_steps``   -- the five-step chi0 . z of Sec. 4.2 (Fig. f:flops,
                            Table t:flops) with the stored alpha object.
* ``polarizability_lu``  -- eq. eqpolarizability via eq. sle solved by a dense
                            LU (numpy.linalg.solve).
* ``polarizability_transition`` -- the same P from the transition-space
                            (push-through) identity, an independent route.
* ``gmres``              -- restarted GMRES (Saad and Schultz) with modified
                            Gram-Schmidt Arnoldi (eq. orthogonal-krylov-basis)
                            and Givens rotations, zero initial guess.
* ``polarizability_gmres`` -- the matrix-free solve of eq. sle at each
                            frequency with A z = z - chi0 (K z) (Sec. 4.1).

Conventions (readings of the paper):
* occupied states are those with n_E > 0 and empty ones those with n_E = 0;
  pairs with n_E = n_F drop out of eq. response-mat by its (n_F - n_E) factor,
  which is the paper's "E.F < 0 after the Fermi shift" condition.
* P is the paper's P_ik = d_i . X_k (eq. eqpolarizability); the physical
  polarizability is alpha = -P, whose imaginary part is >= 0 for omega > 0.
* GMRES stops by default when the true residual ||b - A x|| / ||b|| <= tol
  (recomputed at each restart and at exit).  ``stop="eps_p"`` and
  ``stop="eps_px"`` take the paper's criterion of Sec. 4.1 instead: the
  error estimates eps_P = |A^-1| |<d|r>| / |<d|X>| and eps_X = |A^-1| |r| / |X|
  with |A^-1| the Frobenius norm of the inverse of the square Krylov
  representation of A (``error_estimates``); "eps_p" stops on eps_P <= tol,
  "eps_px" on eps_P <= tol and eps_X <= tol (the paper's combined rule).
"""
from __future__ import annotations

import math
import os

import numpy as np


# --------------------------------------------------------------------------
# Vertex and transition quantities (Sec. 3)
# --------------------------------------------------------------------------

def _atom_slices(sysm):
    off = sysm.atom_orb_offset
    return [slice(int(off[i]), int(off[i + 1])) for i in range(sysm.n_atoms)]


def dense_vertex(sysm) -> np.ndarray:
    """V[mu] as dense n_orb x n_orb symmetric matrices (eq. vertex-ansatz).

    A local product (A == A) holds its symmetric block on A x A.  A bilocal
    product on (A, B) holds its block on A x B and the transpose on B x A,
    because f^a f^b = f^b f^a.
    """
    sl = _atom_slices(sysm)
    n = sysm.n_orb
    V = np.zeros((sysm.n_prod, n, n))
    for mu in range(sysm.n_prod):
        A, B = sysm.prod_atoms[mu]
        blk = sysm.vertex_block(mu)
        V[mu, sl[A], sl[B]] += blk
        if A != B:
            V[mu, sl[B], sl[A]] += blk.T
    return V


def occupied_empty(sysm):
    occ = np.flatnonzero(sysm.occupations > 0)
    emp = np.flatnonzero(sysm.occupations == 0)
    return occ, emp


def transition_vertex(sysm, V=None) -> np.ndarray:
    """M[mu, o, u] = sum_ab X_a^o V_mu^{ab} X_b^u for o occupied, u empty
    (the bracketed factors of eq. response-mat)."""
    if V is None:
        V = dense_vertex(sysm)
    occ, emp = occupied_empty(sysm)
    Xo = sysm.X[:, occ]
    Xu = sysm.X[:, emp]
    return np.einsum("ao,mab,bu->mou", Xo, V, Xu, optimize=True)


def pair_factor(sysm, omega: float, eps: float) -> np.ndarray:
    """D[o, u](omega) for o occupied, u empty.

    eq. response-mat has one term for (E, F) = (u, o) and one for (o, u):
      (n_o - n_u) / (omega - (E_u - E_o) + i eps)
    + (n_u - n_o) / (omega - (E_o - E_u) + i eps),
    and both multiply the same (M_mu^{ou})(M_nu^{ou}) since V is symmetric.
    """
    occ, emp = occupied_empty(sysm)
    E = sysm.eigenvalues
    n = sysm.occupations
    dn = n[occ][:, None] - n[emp][None, :]
    delta = E[emp][None, :] - E[occ][:, None]
    w = omega + 1j * eps
    return dn * (1.0 / (w - delta) - 1.0 / (w + delta))


def chi0_brute(sysm, omega: float, eps: float) -> np.ndarray:
    """eq. response-mat written out term by term: every ordered pair (E, F)
    of states, every a, b, c, d.  Pure Python; only for tiny systems."""
    V = dense_vertex(sysm)
    X = sysm.X
    E = sysm.eigenvalues
    nE = sysm.occupations
    norb, nprod = sysm.n_orb, sysm.n_prod
    w = complex(omega, eps)
    chi = np.zeros((nprod, nprod), dtype=complex)
    for e in range(norb):
        for f in range(norb):
            weight = (nE[f] - nE[e]) / (w - (E[e] - E[f]))
            if nE[f] == nE[e]:
                continue
            left = np.zeros(nprod)
            right = np.zeros(nprod)
            for mu in range(nprod):
                s_l = 0.0
                s_r = 0.0
                for a in range(norb):
                    for b in range(norb):
                        s_l += X[a, e] * V[mu, a, b] * X[b, f]
                        s_r += X[a, f] * V[mu, a, b] * X[b, e]
                left[mu] = s_l
                right[mu] = s_r
            chi += weight * np.outer(left, right)
    return chi


def chi0_explicit(sysm, omega: float, eps: float, M=None) -> np.ndarray:
    """chi0_{mu nu}(omega) = sum_{o,u} M_mu^{ou} D_ou M_nu^{ou}
    (eq. response-mat with the two orderings merged)."""
    if M is None:
        M = transition_vertex(sysm)
    D = pair_factor(sysm, omega, eps)
    Mf = M.reshape(M.shape[0], -1)
    return (Mf * D.reshape(1, -1)) @ Mf.T


# --------------------------------------------------------------------------
# The five-step chi0 . z of Sec. 4.2 (Fig. f:flops, Table t:flops)
# --------------------------------------------------------------------------

class StepOperator:
    """chi0(omega) . z without forming chi0, in the paper's order.

    Step 1 (once):  alpha_nu^{cE} = V_nu^{cd} X_d^E  (E occupied), stored per
                    product on the rows c of its one or two atoms.
    Step 2:         beta^{cE} = alpha_nu^{cE} z^nu
    Step 3:         a^{FE} = X_c^F beta^{cE}  (F empty), then a^{FE} *= D_EF
                    (the denominator omitted from Fig. f:flops)
    Step 4:         gamma_b^E = sum_F X_b^F a^{FE}
    Step 5:         n_mu = sum_E alpha_mu^{bE} gamma_b^E
    """

    def __init__(self, sysm):
        self.sysm = sysm
        occ, emp = occupied_empty(sysm)
        self.Xo = sysm.X[:, occ]
        self.Xu = sysm.X[:, emp]
        sl = _atom_slices(sysm)
        groups = {}
        for mu in range(sysm.n_prod):
            A, B = (int(t) for t in sysm.prod_atoms[mu])
            groups.setdefault((A, B), []).append(mu)
        self.groups = []
        for (A, B), prods in groups.items():
            if A == B:
                rows = np.arange(sl[A].start, sl[A].stop)
                alpha = np.stack([sysm.vertex_block(mu) @ self.Xo[sl[A]] for mu in prods])
            else:
                rows = np.concatenate([np.arange(sl[A].start, sl[A].stop),
                                       np.arange(sl[B].start, sl[B].stop)])
                alpha = np.stack([
                    np.vstack([sysm.vertex_block(mu) @ self.Xo[sl[B]],
                               sysm.vertex_block(mu).T @ self.Xo[sl[A]]])
                    for mu in prods])
            self.groups.append((np.asarray(prods), rows, alpha))

    def apply(self, z: np.ndarray, omega: float, eps: float) -> np.ndarray:
        sysm = self.sysm
        beta = np.zeros(self.Xo.shape, dtype=complex)
        for prods, rows, alpha in self.groups:                       # step 2
            beta[rows] += np.einsum("prE,p->rE", alpha, z[prods])
        a = self.Xu.T @ beta                                         # step 3
        a *= pair_factor(sysm, omega, eps).T
        gamma = self.Xu @ a                                          # step 4
        n = np.zeros(sysm.n_prod, dtype=complex)
        for prods, rows, alpha in self.groups:                       # step 5
            n[prods] = np.einsum("prE,rE->p", alpha, gamma[rows])
        return n


def chi0_apply_steps(sysm, z, omega, eps, op: StepOperator | None = None):
    return (op or StepOperator(sysm)).apply(np.asarray(z, dtype=complex), omega, eps)


def apply_A(sysm, op: StepOperator, z, omega, eps):
    """A z = z - chi0(omega) (K z)  (Sec. 4.1, matrix-free)."""
    return z - op.apply(sysm.K @ z, omega, eps)


# --------------------------------------------------------------------------
# Direct solves (eqs. sle and eqpolarizability)
# --------------------------------------------------------------------------

def polarizability_lu(sysm, omega: float, eps: float, M=None):
    """P_ik(omega) = d_i . X_k with (1 - chi0 K) X_k = chi0 d_k, dense LU.

    Returns (P [3, 3] complex, X [3, n_prod] complex)."""
    chi = chi0_explicit(sysm, omega, eps, M)
    A = np.eye(sysm.n_prod) - chi @ sysm.K
    b = chi @ sysm.dipole.T.astype(complex)
    Xs = np.linalg.solve(A, b)
    return sysm.dipole @ Xs, Xs.T


def polarizability_transition(sysm, omega: float, eps: float, M=None):
    """Same P from the transition space.  With chi0 = M D M^T and s_k = M^T d_k,
    (1 - M D M^T K)^{-1} M D M^T = M (D^{-1} - M^T K M)^{-1} M^T (push-through),
    so P_ik = s_i^T (D^{-1} - M^T K M)^{-1} s_k."""
    if M is None:
        M = transition_vertex(sysm)
    Mf = M.reshape(M.shape[0], -1)
    D = pair_factor(sysm, omega, eps).ravel()
    S = Mf.T @ sysm.dipole.T
    Z = np.diag(1.0 / D) - Mf.T @ sysm.K @ Mf
    return S.T @ np.linalg.solve(Z, S.astype(complex))


# --------------------------------------------------------------------------
# Restarted GMRES (Sec. 4.1)
# --------------------------------------------------------------------------

def _givens(a: complex, b: float):
    """Rotation [[c, s], [-conj(s), c]] with real c that maps (a, b) to (r, 0)."""
    if b == 0.0:
        return 1.0, 0.0
    if a == 0.0:
        return 0.0, 1.0
    r = math.hypot(abs(a), b)
    c = abs(a) / r
    s = (a / abs(a)) * b / r
    return c, s


STOP_RULES = ("residual", "eps_p", "eps_px")


def _ratio(F: float, num: float, den: float) -> float:
    """F num / den, read as 0 when num = 0 and as infinity when only den = 0."""
    if num == 0.0:
        return 0.0
    if den == 0.0:
        return math.inf
    return F * num / den


def error_estimates(Finv: float, r, x, d):
    """The paper's error estimates of Sec. 4.1 for the iterate x with residual
    r = b - A x: Delta X = A^-1 r and Delta P = <d|A^-1|r> are estimated with
    a matrix norm of A^-1, |A^-1| ~ Finv, so that
        eps_P = Finv |<d|r>| / |<d|x>|,   eps_X = Finv ||r|| / ||x||.
    d is real, so <d|r> = d . r.  Returns (eps_P, eps_X)."""
    r = np.asarray(r, dtype=complex)
    x = np.asarray(x, dtype=complex)
    return (_ratio(Finv, abs(d @ r), abs(d @ x)),
            _ratio(Finv, np.linalg.norm(r), np.linalg.norm(x)))


def krylov_inverse_norm(Hsq) -> float:
    """|A^-1| ~ sqrt(sum_ij |<i|A^-1|j>|^2) (Sec. 4.1): the Frobenius norm of
    the inverse of the square Krylov representation H_ij = <i|A|j> of A on
    the current basis (infinity when it is singular)."""
    try:
        return float(np.linalg.norm(np.linalg.inv(Hsq), "fro"))
    except np.linalg.LinAlgError:
        return math.inf


def _stop_met(stop: str, ep: float, ex: float, tol: float) -> bool:
    if stop == "eps_p":
        return ep <= tol
    return ep <= tol and ex <= tol


def gmres(matvec, b, restart: int, tol: float, max_restarts: int = 200, x0=None,
          stop: str = "residual", d=None, trace: bool = False):
    """Restarted GMRES(m): Arnoldi with modified Gram-Schmidt, Givens QR of the
    Hessenberg matrix, minimal residual in each Krylov space.  The first
    basis vector is the (normalised) residual, which for a zero initial guess
    is b itself.

    stop = "residual": a cycle ends once the Givens residual estimate
    |g_{j+1}| / ||b|| <= tol, and the solve ends when ||b - A x|| / ||b|| <= tol,
    that residual being recomputed from scratch after every cycle.
    stop = "eps_p" / "eps_px" (the paper's criterion, needs the real vector d
    of P = <d|X>): after every Arnoldi step j the iterate x_j = x + V y_j
    (y_j the least-squares solution on the unrotated Hessenberg matrix), its
    residual r_j = r_0 - sum_i y_i A v_i and |A^-1| ~ ||H_j^-1||_F of the
    square (j+1) x (j+1) Hessenberg block give eps_P and eps_X
    (``error_estimates``); the cycle ends once the rule holds, and the solve
    ends when it holds for the recomputed residual with the |A^-1| of the
    cycle's last step (before any cycle, |A^-1| is unknown: infinity).

    Returns (x, info) with info = dict(converged, matvecs, cycles, resid,
    eps_p, eps_x) and, with trace, info["trace"] = [(cycle, j, Finv, eps_p,
    eps_x), ...] of every step."""
    if stop not in STOP_RULES:
        raise ValueError(f"stop must be one of {STOP_RULES}")
    b = np.asarray(b, dtype=complex)
    bnorm = np.linalg.norm(b)
    n = b.shape[0]
    x = np.zeros(n, dtype=complex) if x0 is None else np.array(x0, dtype=complex)
    info = dict(converged=False, matvecs=0, cycles=0, resid=1.0, eps_p=math.nan,
                eps_x=math.nan)
    if trace:
        info["trace"] = []
    if stop != "residual":
        d = np.asarray(d, dtype=float)
    if bnorm == 0.0:
        info.update(converged=True, resid=0.0)
        return x, info
    m = restart
    Flast = math.inf
    for cycle in range(max_restarts + 1):
        if cycle == 0 and x0 is None:
            r = b.copy()
        else:
            r = b - matvec(x)
            info["matvecs"] += 1
        beta = np.linalg.norm(r)
        info["resid"] = beta / bnorm
        if stop == "residual":
            done = beta / bnorm <= tol
        else:
            ep, ex = error_estimates(Flast, r, x, d)
            info.update(eps_p=ep, eps_x=ex)
            done = beta == 0.0 or _stop_met(stop, ep, ex, tol)
        if done:
            info["converged"] = True
            return x, info
        if cycle == max_restarts:
            break
        info["cycles"] += 1
        V = np.zeros((m + 1, n), dtype=complex)
        AV = np.zeros((m, n), dtype=complex)
        H = np.zeros((m + 1, m), dtype=complex)
        Hraw = np.zeros((m + 1, m), dtype=complex)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=complex)
        g = np.zeros(m + 1, dtype=complex)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = matvec(V[j])
            AV[j] = w
            info["matvecs"] += 1
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            hnext = np.linalg.norm(w)
            H[j + 1, j] = hnext
            Hraw[:, j] = H[:, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            c, s = _givens(H[j, j], hnext)
            cs[j], sn[j] = c, s
            H[j, j] = c * H[j, j] + s * hnext
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            k = j + 1
            if stop == "residual":
                hit = abs(g[j + 1]) / bnorm <= tol
            else:
                Flast = krylov_inverse_norm(Hraw[:k, :k])
                rhs = np.zeros(k + 1, dtype=complex)
                rhs[0] = beta
                yj = np.linalg.lstsq(Hraw[:k + 1, :k], rhs, rcond=None)[0]
                ep, ex = error_estimates(Flast, r - yj @ AV[:k], x + yj @ V[:k], d)
                if trace:
                    info["trace"].append((cycle, j, Flast, ep, ex))
                hit = _stop_met(stop, ep, ex, tol)
            if hnext == 0.0 or hit:
                break
            V[j + 1] = w / hnext
        y = np.zeros(k, dtype=complex)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + y @ V[:k]
    return x, info


def polarizability_gmres(sysm, omegas, eps: float, restart: int, tol: float,
                         max_restarts: int = 200, dirs=(0, 1, 2), op=None,
                         stop: str = "residual"):
    """Matrix-free P(omega) for each omega: b_k = chi0 d_k, GMRES on
    (1 - chi0 K) X_k = b_k, P_ik = d_i . X_k.  ``stop`` is the GMRES stopping
    rule (``gmres``), with d = d_k for the right-hand side of direction k.

    Returns (P [n_omega, 3, len(dirs)] complex, infos list)."""
    op = op or StepOperator(sysm)
    omegas = np.atleast_1d(np.asarray(omegas, dtype=float))
    P = np.zeros((omegas.size, 3, len(dirs)), dtype=complex)
    infos = []
    for iw, w in enumerate(omegas):
        for jk, k in enumerate(dirs):
            b = op.apply(sysm.dipole[k].astype(complex), w, eps)
            x, info = gmres(lambda z: apply_A(sysm, op, z, w, eps), b, restart, tol,
                            max_restarts, stop=stop, d=sysm.dipole[k])
            info.update(omega=float(w), dir=int(k))
            infos.append(info)
            P[iw, :, jk] = sysm.dipole @ x
    return P, infos


# --------------------------------------------------------------------------
# Parallel driver over (omega, direction) tasks, as in Sec. 6.1.3
# --------------------------------------------------------------------------

_W = {}


def _worker_init(source, eps, restart, tol, max_restarts):
    sysm = source[0](*source[1]) if isinstance(source, tuple) else source
    _W.update(sysm=sysm, eps=eps, restart=restart, tol=tol, max_restarts=max_restarts,
              op=StepOperator(sysm))


def _worker_task(task):
    w, k = task
    P, infos = polarizability_gmres(_W["sysm"], [w], _W["eps"], _W["restart"], _W["tol"],
                                    _W["max_restarts"], dirs=(k,), op=_W["op"])
    return P[0, :, 0], infos[0]


def polarizability_gmres_parallel(source, omegas, eps, restart, tol, workers: int,
                                  max_restarts: int = 200, dirs=(0, 1, 2)):
    """One (omega, direction) task per process with a dynamic schedule, the
    paper's scheme for this phase.  Workers are spawned with one BLAS thread
    each.  ``source`` is a System or a picklable (factory, args) pair that each
    worker calls to rebuild it.  Returns (P [n_omega, 3, len(dirs)], infos)."""
    import multiprocessing as mp
    omegas = np.atleast_1d(np.asarray(omegas, dtype=float))
    tasks = [(float(w), int(k)) for w in omegas for k in dirs]
    env = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                          "MKL_NUM_THREADS")}
    for v in env:
        os.environ[v] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers, initializer=_worker_init,
                      initargs=(source, eps, restart, tol, max_restarts)) as pool:
            out = pool.map(_worker_task, tasks, chunksize=1)
    finally:
        for v, val in env.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val
    P = np.zeros((omegas.size, 3, len(dirs)), dtype=complex)
    infos = []
    for t, (p, info) in enumerate(out):
        P[t // len(dirs), :, t % len(dirs)] = p
        infos.append(info)
    return P, infos
