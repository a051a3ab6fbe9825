"""Pins for the learned-guess oracle: finite-difference gradients, the
untrained network reducing to interpolation, the loss gradient."""
import numpy as np

import oracle.mlp_oracle as M

DIMS = (10, 16, 2)


def _params(seed=0, zero_last=False):
    rng = np.random.default_rng(seed)
    n = 16 * 10 + 16 + 16 * 16 + 16 + 2 * 16 + 2
    p = rng.normal(size=n) * 0.3
    if zero_last:
        p[-(2 * 16 + 2):] = 0.0
    return p


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    F = rng.normal(size=(7, 10))
    dY = rng.normal(size=(7, 2))
    p = _params(2)
    g = M.backward(p, F, dY, DIMS)
    h = 1e-6
    for i in rng.choice(p.size, 40, replace=False):
        e = np.zeros_like(p); e[i] = h
        fp = np.sum(dY * M.forward(p + e, F, DIMS)[0])
        fm = np.sum(dY * M.forward(p - e, F, DIMS)[0])
        assert abs((fp - fm) / (2 * h) - g[i]) <= 1e-7 * max(1.0, abs(g[i]))


def test_untrained_network_is_linear_interpolation():
    rng = np.random.default_rng(3)
    Xm = rng.normal(size=50) + 1j * rng.normal(size=50)
    Xp = rng.normal(size=50) + 1j * rng.normal(size=50)
    F, lin, s = M.features(Xm, Xp, 0.25, 0.4, 2.0, rng.integers(0, 2, 50), rng.normal(size=50),
                           np.abs(rng.normal(size=50)))
    Y, _ = M.forward(_params(4, zero_last=True), F, DIMS)
    assert np.all(Y == 0.0)
    assert np.allclose(lin, 0.75 * Xm + 0.25 * Xp)
    assert np.isclose(s, np.sqrt((np.sum(abs(Xm) ** 2) + np.sum(abs(Xp) ** 2)) / 100))


def test_guess_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    nt, n = 3, 6
    lin = rng.normal(size=(nt, n)) + 1j * rng.normal(size=(nt, n))
    xs = rng.normal(size=(nt, n)) + 1j * rng.normal(size=(nt, n))
    scale = rng.uniform(0.5, 2.0, nt)
    Y = rng.normal(size=(nt * n, 2))
    per, dY = M.guess_loss(Y, lin, xs, scale)
    h = 1e-6
    for i in range(nt * n):
        for c in range(2):
            e = np.zeros_like(Y); e[i, c] = h
            lp = M.guess_loss(Y + e, lin, xs, scale)[0].mean()
            lm = M.guess_loss(Y - e, lin, xs, scale)[0].mean()
            assert abs((lp - lm) / (2 * h) - dY[i, c]) <= 1e-7
    # zero error at the exact solution
    y_exact = (xs - lin) / scale[:, None]
    Y0 = np.stack([y_exact.real.ravel(), y_exact.imag.ravel()], axis=1)
    assert np.max(M.guess_loss(Y0, lin, xs, scale)[0]) < 1e-28
