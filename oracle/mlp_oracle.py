"""CPU oracle of the learned-guess network (test infrastructure only).

Float64 numpy restatement of what the library's training and inference
kernels compute: the per-product network n_in -> width -> width -> n_out
with tanh hidden layers and the packed parameter layout
[W1 (width x n_in), b1, W2 (width x width), b2, W3 (n_out x width), b3];
the guess x0 = lin + s * y; the loss mean_r |x0_r - x*_r|^2 / |x*_r|^2 and
its gradient; and the per-product features built from two solved
neighbouring frequencies.  Pinned by a hand-built 2 -> 3 -> 3 -> 2 network
whose outputs are worked out by hand from literal weights (activation,
packing order and orientation of every block), by a hand-built three-product
feature case with every column written out from its definition, by finite
differences and by the exact reduction of an untrained network to linear
interpolation.
"""
from __future__ import annotations

import numpy as np


def unpack(p, n_in, width, n_out):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + width * n_in].reshape(width, n_in); o += width * n_in
    b1 = p[o:o + width]; o += width
    W2 = p[o:o + width * width].reshape(width, width); o += width * width
    b2 = p[o:o + width]; o += width
    W3 = p[o:o + n_out * width].reshape(n_out, width); o += n_out * width
    b3 = p[o:o + n_out]; o += n_out
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def forward(p, F, dims):
    W1, b1, W2, b2, W3, b3 = unpack(p, *dims)
    H1 = np.tanh(F @ W1.T + b1)
    H2 = np.tanh(H1 @ W2.T + b2)
    return H2 @ W3.T + b3, (H1, H2)


def backward(p, F, dY, dims):
    """Gradient of sum(dY * Y) with respect to the packed parameters."""
    W1, b1, W2, b2, W3, b3 = unpack(p, *dims)
    Y, (H1, H2) = forward(p, F, dims)
    gW3 = dY.T @ H2
    gb3 = dY.sum(axis=0)
    dH2 = (dY @ W3) * (1.0 - H2 ** 2)
    gW2 = dH2.T @ H1
    gb2 = dH2.sum(axis=0)
    dH1 = (dH2 @ W2) * (1.0 - H1 ** 2)
    gW1 = dH1.T @ F
    gb1 = dH1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def guess_loss(Y, lin, xstar, scale):
    """Mean over targets of |lin + s y - x*|^2 / |x*|^2 and d/dY.
    Y [n_target*n_prod, 2] real; lin, xstar [n_target, n_prod] complex."""
    nt, n_prod = lin.shape
    y = (Y[:, 0] + 1j * Y[:, 1]).reshape(nt, n_prod)
    r = lin + scale[:, None] * y - xstar
    nrm = np.sum(np.abs(xstar) ** 2, axis=1)
    per = np.sum(np.abs(r) ** 2, axis=1) / nrm
    g = 2.0 * scale[:, None] * r / nrm[:, None] / nt
    dY = np.stack([g.real.ravel(), g.imag.ravel()], axis=1)
    return per, dY


def features(Xm, Xp, t, omega, h_over_eps, bilocal, d_k, vnorm_rel):
    """Ten features per product for one target (see the C boundary)."""
    n = Xm.size
    s = np.sqrt((np.sum(np.abs(Xm) ** 2) + np.sum(np.abs(Xp) ** 2)) / (2 * n))
    dr = np.sqrt(np.mean(d_k ** 2))
    F = np.stack([Xm.real / s, Xm.imag / s, Xp.real / s, Xp.imag / s,
                  np.full(n, t), np.full(n, omega), np.full(n, h_over_eps),
                  bilocal.astype(float), d_k / dr, vnorm_rel], axis=1)
    lin = (1 - t) * Xm + t * Xp
    return F, lin, s
