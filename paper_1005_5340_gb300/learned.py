"""Learned initial guess: training of the guess network (host-side driver).

The warm-started frequency sweep itself (three passes over the grid, guesses
from the two nearest solved neighbours, interpolated or corrected by the
network, each arbitrated against the zero guess) runs inside the library:
tddft_polarizability with a context whose guess mode is "interp" or
"learned" (tddft_set_guess, tddft_guess_load).  This module gathers training
targets from solved spectra (the sweep's pass plan comes from
tddft_sweep_plan) and drives the library's training kernels.
"""
from __future__ import annotations

import os
import tempfile

import numpy as np

from . import synth


def sweep_passes(n_omega: int):
    """(indices, left neighbour, right neighbour) per pass of the library's
    sweep (tddft_sweep_plan); pass 0 has no neighbours."""
    from .tddft import sweep_plan
    pas, left, right = sweep_plan(n_omega)
    out = []
    for p in range(3):
        idx = np.flatnonzero(pas == p)
        out.append((idx, None, None) if p == 0 else (idx, left[idx], right[idx]))
    return out


def _targets(omega, idx, left, right):
    """Per (frequency, direction) target: neighbour rows, weight t, spacing."""
    k = np.tile(np.arange(3), idx.size)
    ii = np.repeat(idx, 3)
    ll = np.repeat(left, 3)
    rr = np.repeat(right, 3)
    nb = np.stack([ll * 3 + k, rr * 3 + k], axis=1).astype(np.int32)
    t = (omega[ii] - omega[ll]) / (omega[rr] - omega[ll])
    return nb, t, omega[ii], k.astype(np.int32), omega[rr] - omega[ll]


def solve_sweep(ctx, omega, eps, mode="zero", mlp=None):
    """The library's sweep on ctx in the given mode ("zero", "interp",
    "learned", "interp_subspace" or "learned_subspace"; mlp is loaded into
    the context for the learned modes).  Returns
    (P [n,3,3] complex numpy, stats dict, X [3n, n_prod] complex CUDA tensor)."""
    if mode.startswith("learned"):
        fd, path = tempfile.mkstemp(suffix=".net")
        os.close(fd)
        try:
            mlp.save(path)
            ctx.guess_load(path)
        finally:
            os.remove(path)
    ctx.set_guess(mode)
    try:
        P, X, st = ctx.polarizability_guess(np.asarray(omega, dtype=float), eps)
    finally:
        ctx.set_guess("zero")
    return P.cpu().numpy(), st, X


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
