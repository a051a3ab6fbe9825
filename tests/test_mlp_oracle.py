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


def test_forward_of_a_hand_built_network():
    """A 2 -> 3 -> 3 -> 2 network with literal weights, packed in the order the
    C boundary states ([W1 (width x n_in) row-major, b1, W2, b2, W3, b3]).
    Each output is written out by hand as a chain of tanh calls, so a wrong
    activation, a swapped or transposed weight block or a dropped bias fails.
    Row 1 (F = (0.5, 0.25)):
        z1 = (0.5, 0.25 + 0.5, 0.5 - 0.25) = (0.5, 0.75, 0.25),  h1 = tanh z1
        z2 = (h1_0, 2 h1_2, 0.1 - h1_1),                        h2 = tanh z2
        y  = (h2_0 + h2_1 + 0.2, -3 h2_2)
    Row 2 (F = (-1, 2)): z1 = (-1, 2.5, -3), the rest as above."""
    import math
    th = math.tanh
    W1 = [1.0, 0.0,
          0.0, 1.0,
          1.0, -1.0]
    b1 = [0.0, 0.5, 0.0]
    W2 = [1.0, 0.0, 0.0,
          0.0, 0.0, 2.0,
          0.0, -1.0, 0.0]
    b2 = [0.0, 0.0, 0.1]
    W3 = [1.0, 1.0, 0.0,
          0.0, 0.0, -3.0]
    b3 = [0.2, 0.0]
    p = np.array(W1 + b1 + W2 + b2 + W3 + b3)
    F = np.array([[0.5, 0.25], [-1.0, 2.0]])
    Y, (H1, H2) = M.forward(p, F, (2, 3, 2))
    exp = []
    for z1 in ([0.5, 0.75, 0.25], [-1.0, 2.5, -3.0]):
        h1 = [th(z) for z in z1]
        h2 = [th(h1[0]), th(2.0 * h1[2]), th(0.1 - h1[1])]
        exp.append([h2[0] + h2[1] + 0.2, -3.0 * h2[2]])
    # the same numbers as decimals (tanh evaluated once, by hand, to 16 digits)
    lit = [[1.0858954904817475, 1.4679213896995118], [-1.4053370971315398, 2.1291523152862215]]
    assert np.max(np.abs(Y - np.array(exp))) < 1e-12
    assert np.max(np.abs(Y - np.array(lit))) < 1e-12
    assert np.allclose(H1[0], [0.46211715726000974, 0.6351489523872873, 0.24491866240370913],
                       rtol=0, atol=1e-14)


def test_backward_of_the_hand_built_network_at_the_output_layer():
    """For the network above with dY = e_0 on one row, the gradient with respect
    to b3 is (1, 0) and with respect to W3 row 0 is h2 (by hand: d y0 / d W3_0j
    = h2_j); those entries sit at the end of the packed vector."""
    import math
    th = math.tanh
    p = np.array([1.0, 0.0, 0.0, 1.0, 1.0, -1.0, 0.0, 0.5, 0.0,
                  1.0, 0.0, 0.0, 0.0, 0.0, 2.0, 0.0, -1.0, 0.0, 0.0, 0.0, 0.1,
                  1.0, 1.0, 0.0, 0.0, 0.0, -3.0, 0.2, 0.0])
    F = np.array([[0.5, 0.25]])
    g = M.backward(p, F, np.array([[1.0, 0.0]]), (2, 3, 2))
    h1 = [th(0.5), th(0.75), th(0.25)]
    h2 = [th(h1[0]), th(2.0 * h1[2]), th(0.1 - h1[1])]
    assert np.allclose(g[-2:], [1.0, 0.0], rtol=0, atol=1e-15)
    assert np.allclose(g[-8:-5], h2, rtol=0, atol=1e-15)     # W3 row 0
    assert np.allclose(g[-5:-2], 0.0, rtol=0, atol=1e-15)    # W3 row 1 (dY_1 = 0)
    # b2: d y0 / d b2_j = W3_0j (1 - h2_j^2)
    assert np.allclose(g[-11:-8], [1.0 - h2[0] ** 2, 1.0 - h2[1] ** 2, 0.0], rtol=0, atol=1e-15)


def test_features_of_a_hand_built_three_product_case():
    """Every column of the ten features written out from its definition:
    s = sqrt((sum |X-|^2 + sum |X+|^2) / (2 n)) = sqrt((3 + 3) / 6) = 1 here;
    Re/Im X-/s, Re/Im X+/s, t, omega, (omega+ - omega-)/eps, the bilocal
    flag, d_k / rms(d_k) with rms((3, 0, -4)) = 5/sqrt(3), ||V|| / mean ||V||;
    lin = (1 - t) X- + t X+."""
    Xm = np.array([1.0, 1j, -1.0])
    Xp = np.array([1.0, -1.0, 1j])
    d = np.array([3.0, 0.0, -4.0])
    vn = np.array([0.5, 1.5, 1.0])
    F, lin, s = M.features(Xm, Xp, 0.25, 0.4, 2.0, np.array([0, 1, 1]), d, vn)
    r3 = np.sqrt(3.0)
    expect = np.array([
        # ReX-  ImX-  ReX+  ImX+  t     omega h/eps  bil  d/rms          vnorm
        [1.0,  0.0,  1.0,  0.0,  0.25, 0.4,  2.0,  0.0, 3.0 * r3 / 5,  0.5],
        [0.0,  1.0, -1.0,  0.0,  0.25, 0.4,  2.0,  1.0, 0.0,           1.5],
        [-1.0, 0.0,  0.0,  1.0,  0.25, 0.4,  2.0,  1.0, -4.0 * r3 / 5, 1.0]])
    assert s == 1.0
    assert F.shape == (3, 10)
    assert np.max(np.abs(F - expect)) < 1e-15
    assert np.allclose(lin, [1.0, 0.75j - 0.25, -0.75 + 0.25j], rtol=0, atol=1e-15)
