"""Frequency sweep with a learned initial guess (host-side driver).

The spectrum is solved in three passes over the uniform grid:
  pass 0: every 4th frequency and the last one, from a zero guess;
  pass 1: the remaining frequencies with index = 2 mod 4, each from its two
          solved neighbours at distance 2;
  pass 2: the rest (odd indices), from their neighbours at distance 1.
In passes 1 and 2 the guess is the linear interpolation of the neighbours'
solutions (mode "interp") or that interpolation corrected per product by the
network of tddft_mlp_* (mode "learned"); mode "zero" solves every pass from
zero.  Each guess first costs one float64 product and is dropped in favour
of zero when it is worse (tddft_polarizability_guess), so converged results
meet the same float64 residual tolerance in every mode.

Everything runs in the library's kernels; this module only orders the
frequencies, gathers the neighbour indices and drives training.
"""
from __future__ import annotations

import numpy as np

from . import synth


def sweep_passes(n_omega: int):
    """(indices, left neighbour, right neighbour) per pass; pass 0 has none."""
    p0 = sorted(set(range(0, n_omega, 4)) | {n_omega - 1})
    solved = set(p0)
    passes = [(np.array(p0), None, None)]
    for cond in (lambda i: i % 4 == 2, lambda i: True):
        idx = [i for i in range(n_omega) if i not in solved and cond(i)]
        srt = sorted(solved)
        left = [max(j for j in srt if j < i) for i in idx]
        right = [min(j for j in srt if j > i) for i in idx]
        passes.append((np.array(idx, dtype=int), np.array(left), np.array(right)))
        solved |= set(idx)
    return passes


def _targets(omega, idx, left, right):
    """Per (frequency, direction) target: neighbour rows, weight t, spacing."""
    k = np.tile(np.arange(3), idx.size)
    ii = np.repeat(idx, 3)
    ll = np.repeat(left, 3)
    rr = np.repeat(right, 3)
    nb = np.stack([ll * 3 + k, rr * 3 + k], axis=1).astype(np.int32)
    t = (omega[ii] - omega[ll]) / (omega[rr] - omega[ll])
    return nb, t, omega[ii], k.astype(np.int32), omega[rr] - omega[ll]


def solve_sweep(ctx, omega, eps, mode="zero", mlp=None, bf16=True):
    """Solve the spectrum pass by pass.  Returns (P [n,3,3] complex numpy,
    stats dict with per-(omega, dir) matvecs/cycles/resid/converged/
    guess_rejected, X [3n, n_prod] complex CUDA tensor)."""
    import torch
    omega = np.asarray(omega, dtype=float)
    n = omega.size
    dev = torch.device("cuda", torch.cuda.current_device())
    X = torch.zeros((3 * n, ctx.n_prod), dtype=torch.complex128, device=dev)
    P = np.zeros((n, 3, 3), dtype=complex)
    stats = {k: np.zeros((n, 3), dtype=dt) for k, dt in
             (("matvecs", int), ("cycles", int), ("resid", float), ("converged", bool),
              ("guess_rejected", bool))}
    for pi, (idx, left, right) in enumerate(sweep_passes(n)):
        if idx.size == 0:
            continue
        x0 = None
        if pi > 0 and mode != "zero":
            nb, t, om_t, k, h = _targets(omega, idx, left, right)
            F, lin, scale = ctx.guess_features(nb, t, om_t, k, float(np.mean(h)) / eps, X)
            if mode == "learned":
                Y = mlp.forward(F, bf16=bf16)
                x0 = mlp.combine(Y, lin, scale)
            else:
                x0 = lin
        Pp, Xp, st = ctx.polarizability_guess(omega[idx], eps, x0)
        rows = (np.repeat(idx, 3) * 3 + np.tile(np.arange(3), idx.size))
        X[torch.as_tensor(rows, device=dev)] = Xp
        P[idx] = Pp.cpu().numpy()
        for key in stats:
            stats[key][idx] = st[key]
    return P, stats, X


def training_targets(ctx, omega, eps, X):
    """Features, interpolation, scale and exact solutions of every pass-1 and
    pass-2 target of one solved spectrum X (CUDA tensors)."""
    import torch
    omega = np.asarray(omega, dtype=float)
    out = []
    for pi, (idx, left, right) in enumerate(sweep_passes(omega.size)):
        if pi == 0 or idx.size == 0:
            continue
        nb, t, om_t, k, h = _targets(omega, idx, left, right)
        F, lin, scale = ctx.guess_features(nb, t, om_t, k, float(np.mean(h)) / eps, X)
        rows = torch.as_tensor(np.repeat(idx, 3) * 3 + np.tile(np.arange(3), idx.size),
                               device=X.device)
        out.append((F, lin, scale, X[rows].contiguous()))
    return out


def train(mlp, datasets, steps: int, targets_per_step: int, lr: float = 1e-3, seed: int = 0,
          log_every: int = 0):
    """Adam on random groups of targets drawn from the datasets (lists of
    (F, lin, scale, xstar) per molecule and pass).  Returns the mean loss
    history (one value per step)."""
    import torch
    rng = np.random.default_rng(seed)
    hist = []
    for it in range(steps):
        F, lin, scale, xs = datasets[rng.integers(len(datasets))]
        nt, n_prod = lin.shape
        m = min(targets_per_step, nt)
        pick = np.sort(rng.choice(nt, m, replace=False))
        pt = torch.as_tensor(pick, device=lin.device)
        rows = (pt[:, None] * n_prod + torch.arange(n_prod, device=lin.device)[None, :]).reshape(-1)
        loss = mlp.train_step(F[rows], lin[pt], xs[pt], scale[pt], lr)
        hist.append(float(loss.mean()))
        if log_every and it % log_every == 0:
            print(f"step {it}: loss {hist[-1]:.4e}", flush=True)
    return np.array(hist)


def guess_error(mlp, datasets, bf16=True):
    """Mean relative squared error of interpolation and of the learned guess."""
    import torch
    e_lin, e_mlp = [], []
    for F, lin, scale, xs in datasets:
        nrm = torch.sum(torch.abs(xs) ** 2, dim=1)
        e_lin.append((torch.sum(torch.abs(lin - xs) ** 2, dim=1) / nrm).cpu().numpy())
        x0 = mlp.combine(mlp.forward(F, bf16=bf16), lin, scale)
        e_mlp.append((torch.sum(torch.abs(x0 - xs) ** 2, dim=1) / nrm).cpu().numpy())
    return float(np.mean(np.concatenate(e_lin))), float(np.mean(np.concatenate(e_mlp)))


def molecule(n_atoms: int, seed: int):
    """A synthetic molecule of the learned-guess study (same generator)."""
    return synth.make_system(n_atoms, seed, density=0.0094)
