"""The learned initial guess on the GPU: the network's kernels against the
CPU oracle (forward, backward, bf16 inference), the features against their
definition, warm-started sweeps reaching the same float64 tolerance, and
what a trained network gains over interpolation and over zero guesses."""
import numpy as np
import pytest

import oracle.mlp_oracle as M
import oracle.tddft_oracle as O
from paper_1005_5340_gb300 import synth
from tests.libutil import ensure_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_library()


def T():
    from paper_1005_5340_gb300 import tddft
    return tddft


def L():
    from paper_1005_5340_gb300 import learned
    return learned


@pytest.mark.parametrize("width,rows", [(16, 37), (256, 300)])
def test_network_kernels_match_oracle(width, rows):
    import torch
    dims = (10, width, 2)
    net = T().Mlp(10, width, 2, max_rows=1024, seed=3)
    rng = np.random.default_rng(width)
    p = (rng.normal(size=net.n_params) * 0.2).astype(np.float32)
    net.set_params(p)
    assert np.array_equal(net.get_params(), p)
    F = rng.normal(size=(rows, 10)).astype(np.float32)
    dY = rng.normal(size=(rows, 2)).astype(np.float32)
    Fd, dYd = torch.from_numpy(F).cuda(), torch.from_numpy(dY).cuda()
    Y_ref, _ = M.forward(p.astype(float), F.astype(float), dims)
    Y = net.forward(Fd).cpu().numpy()
    assert np.max(np.abs(Y - Y_ref)) <= 1e-4 * np.max(np.abs(Y_ref))
    Yb = net.forward(Fd, bf16=True).cpu().numpy()
    assert np.max(np.abs(Yb - Y_ref)) <= 3e-2 * np.max(np.abs(Y_ref))
    g_ref = M.backward(p.astype(float), F.astype(float), dY.astype(float), dims)
    g = net.backward(Fd, dYd)
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * np.max(np.abs(g_ref))
    net.close()


def test_parameters_survive_a_file_round_trip(tmp_path):
    """tddft_mlp_save / tddft_mlp_load: the same parameters and the same
    forward pass after a round trip; a network of another shape is refused."""
    import torch
    net = T().Mlp(10, 64, 2, max_rows=256, seed=7)
    rng = np.random.default_rng(4)
    p = (rng.standard_normal(net.n_params) * 0.2).astype(np.float32)
    net.set_params(p)
    path = tmp_path / "guess.net"
    net.save(path)
    other = T().Mlp(10, 64, 2, max_rows=256, seed=8)
    other.load(path)
    assert np.array_equal(other.get_params(), p)
    F = torch.from_numpy(rng.standard_normal((100, 10)).astype(np.float32)).cuda()
    assert np.array_equal(other.forward(F).cpu().numpy(), net.forward(F).cpu().numpy())
    wrong = T().Mlp(10, 32, 2, max_rows=16, seed=9)
    with pytest.raises(T().TddftError) as e:
        wrong.load(path)
    assert e.value.status == T().ERR_SHAPE
    with pytest.raises(T().TddftError) as e:
        other.load(tmp_path / "missing.net")
    assert e.value.status == T().ERR_INVALID_ARG
    for net_ in (net, other, wrong):
        net_.close()


def test_untrained_network_starts_at_zero_output():
    import torch
    net = T().Mlp(10, 256, 2, max_rows=64, seed=1)
    F = torch.randn(64, 10, dtype=torch.float32, device="cuda")
    assert float(torch.max(torch.abs(net.forward(F)))) == 0.0
    net.close()


def test_features_and_interpolation_match_definition():
    import torch
    s, w = synth.workload("tiny4")
    om = w["omega"][:9]
    with T().Context(s, batch=27, restart=w["restart"], tol=1e-10) as ctx:
        P, X, st = ctx.polarizability_guess(om, w["eps"])
        nb = np.array([[0 * 3 + 1, 4 * 3 + 1], [4 * 3 + 2, 8 * 3 + 2]], dtype=np.int32)
        t = np.array([0.5, 0.25])
        F, lin, scale = ctx.guess_features(nb, t, om[[2, 5]], [1, 2],
                                           (om[4] - om[0]) / w["eps"], X)
    Xh = X.cpu().numpy()
    bil = s.prod_atoms[:, 0] != s.prod_atoms[:, 1]
    vn = np.array([np.linalg.norm(s.vertex_block(m)) for m in range(s.n_prod)])
    for r, (a, b) in enumerate(nb):
        Fr, linr, sr = M.features(Xh[a], Xh[b], t[r], [om[2], om[5]][r],
                                  (om[4] - om[0]) / w["eps"], bil, s.dipole[[1, 2][r]],
                                  vn / vn.mean())
        got = F.cpu().numpy()[r * s.n_prod:(r + 1) * s.n_prod]
        assert np.allclose(got, Fr, rtol=1e-5, atol=1e-6)
        assert np.allclose(lin.cpu().numpy()[r], linr, rtol=1e-12, atol=0)
        assert np.isclose(scale.cpu().numpy()[r], sr, rtol=1e-12)


def test_warm_started_sweeps_reach_the_same_answer():
    """Dense grid (spacing 0.1 eps): every mode converges to the LU answer,
    an untrained network reproduces the interpolation exactly, and warm
    starts do not cost more operator products than zero guesses."""
    s, w = synth.workload("tiny4")
    om = np.linspace(0.40, 0.47, 64)
    M_ = O.transition_vertex(s)
    P_lu = np.stack([O.polarizability_lu(s, x, w["eps"], M_)[0] for x in om])
    net = T().Mlp(10, 256, 2, max_rows=64 * s.n_prod * 3, seed=2)
    res = {}
    for prec in ("fp64", "bf16x3"):
        with T().Context(s, batch=96, restart=w["restart"], tol=1e-10, prec=prec) as ctx:
            for mode in ("zero", "interp", "learned", "interp_subspace", "learned_subspace"):
                P, st, X = L().solve_sweep(ctx, om, w["eps"], mode=mode, mlp=net)
                assert st["converged"].all() and np.all(st["resid"] <= 1e-10)
                assert np.max(np.abs(P - P_lu)) <= 1e-8 * np.max(np.abs(P_lu))
                res[prec, mode] = int(st["matvecs"].sum())
    print("products per sweep:", res)
    for prec in ("fp64", "bf16x3"):
        assert res[prec, "learned"] == res[prec, "interp"]
    assert res["fp64", "interp"] <= res["fp64", "zero"]
    # the minimum-residual point of a span holding the guess is never worse
    assert res["fp64", "interp_subspace"] <= res["fp64", "interp"]
    net.close()


@pytest.mark.slow
def test_trained_network_gains_over_interpolation():
    """Train on spectra of six 8-12 atom molecules solved by the method
    itself (128 frequencies in [0.3, 0.5] Ha, spacing 0.3 eps, as in the
    1024-point workload); on a held-out 16-atom molecule the learned guess
    must be closer to the solution than the interpolation.  The products of
    zero-guess, interpolated and learned sweeps are reported."""
    eps, tol, restart = 0.005, 1e-6, 40
    om = np.linspace(0.3, 0.5, 128)
    net = T().Mlp(10, 256, 2, max_rows=1 << 20, seed=5)
    data = []
    for i, n_at in enumerate((8, 9, 10, 11, 12, 10)):
        s = L().molecule(n_at, 5000 + i)
        with T().Context(s, batch=384, restart=restart, tol=1e-9, prec="bf16x3") as ctx:
            P, X, st = ctx.polarizability_guess(om, eps)
            data += L().training_targets(ctx, om, eps, X)
    hist = L().train(net, data, steps=800, targets_per_step=64, lr=1e-3, seed=1)
    assert hist[-50:].mean() < hist[:50].mean()
    s = L().molecule(16, 6000)
    mv = {}
    with T().Context(s, batch=384, restart=restart, tol=1e-9, prec="bf16x3") as ctx:
        P, X, st = ctx.polarizability_guess(om, eps)
        held = L().training_targets(ctx, om, eps, X)
        e_lin, e_mlp = L().guess_error(net, held)
    with T().Context(s, batch=384, restart=restart, tol=tol, prec="fp64") as ctx:
        for mode in ("zero", "interp", "learned", "interp_subspace", "learned_subspace"):
            P, st, _ = L().solve_sweep(ctx, om, eps, mode=mode, mlp=net)
            assert st["converged"].all() and np.all(st["resid"] <= tol)
            mv[mode] = int(st["matvecs"].sum())
    print(f"held-out guess error: interpolation {e_lin:.3e}, learned {e_mlp:.3e}; "
          f"products {mv} (the subspace modes add 3 products in the context's precision "
          f"per guessed right-hand side, not counted here)")
    assert e_mlp < e_lin
    assert mv["learned"] <= mv["zero"]
    net.close()


def test_learned_sweep_through_the_c_boundary(tmp_path):
    """tddft_options.guess and tddft_guess_load: a learned-guess spectrum from
    tddft_polarizability alone (host pointers, no Python arithmetic), every
    frequency at the float64 tolerance and equal to the zero-guess spectrum
    within it; the interpolating mode likewise; the errors of a missing or
    misshapen network."""
    s, w = synth.workload("tiny4")
    om = np.linspace(0.40, 0.47, 33)
    net = T().Mlp(10, 64, 2, max_rows=1024, seed=11)
    rng = np.random.default_rng(2)
    p = net.get_params()
    p[-(2 * 64 + 2):] = rng.normal(size=2 * 64 + 2).astype(np.float32) * 1e-3
    net.set_params(p)
    path = tmp_path / "g.net"
    net.save(path)
    res = {}
    for mode in ("zero", "interp", "learned"):
        with T().Context(s, batch=48, restart=w["restart"], tol=1e-10, guess=mode) as ctx:
            if mode == "learned":
                ctx.guess_load(path)
            P, st = ctx.polarizability(om, w["eps"])
        assert st["converged"].all() and np.all(st["resid"] <= 1e-10)
        res[mode] = (P, int(st["matvecs"].sum()))
    for mode in ("interp", "learned"):
        assert np.max(np.abs(res[mode][0] - res["zero"][0])) <= 1e-8 * np.max(np.abs(res["zero"][0]))
    print("products:", {k: v[1] for k, v in res.items()})
    with T().Context(s, batch=48, restart=w["restart"], tol=1e-10, guess="learned") as ctx:
        with pytest.raises(T().TddftError) as e:
            ctx.polarizability(om, w["eps"])
        assert e.value.status == T().ERR_INVALID_ARG
        wrong = T().Mlp(12, 16, 2, max_rows=16, seed=1)
        wpath = tmp_path / "w.net"
        wrong.save(wpath)
        with pytest.raises(T().TddftError) as e:
            ctx.guess_load(wpath)
        assert e.value.status == T().ERR_SHAPE
        wrong.close()
    net.close()
