"""Parity of the CUDA path (through the C boundary) with the CPU oracle.

Operators (chi0 . z, K . z, A . z) must match to <= 1e-12 relative in
float64; spectra solved to tol 1e-12 must match the oracle's dense-LU P to
<= 1e-10 relative (normwise over the spectrum).  Sizes span several tiles of
every kernel and ragged tails (orbitals per atom 5..16, odd n_occ, odd
numbers of right-hand sides)."""
import numpy as np
import pytest

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


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


def ragged_system(seed=12):
    """Atoms with 5, 13, 16, 9 and 13 orbitals, n_occ = 11, varied products."""
    base = synth.make_system(5, seed, orb_per_atom=16, occ_per_atom=2, n_local=7, n_bilocal=5,
                             density=0.02)
    sizes = np.array([5, 13, 16, 9, 13])
    aoff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    n_orb = int(aoff[-1])
    rng = synth.CounterRNG(seed, 50)
    blocks, pairs = [], []
    for mu in range(base.n_prod):
        A, B = base.prod_atoms[mu]
        g = rng.normal(sizes[A] * sizes[B]).reshape(sizes[A], sizes[B]) * 0.05
        if A == B:
            g = (g + g.T) / np.sqrt(2.0)
        blocks.append(g)
        pairs.append((A, B))
    voff = np.concatenate([[0], np.cumsum([b.size for b in blocks])]).astype(np.int64)
    E = np.sort(-1.0 + 1.5 * synth.CounterRNG(seed, 51).uniform(n_orb))
    occ = np.zeros(n_orb)
    occ[:11] = 2.0
    X = synth.haar_orthogonal(n_orb, synth.CounterRNG(seed, 52))
    return synth.System(n_atoms=5, atom_orb_offset=aoff, eigenvalues=E, occupations=occ, X=X,
                        prod_atoms=np.array(pairs, dtype=np.int32),
                        vertex_offset=voff, vertex=np.concatenate([b.ravel() for b in blocks]),
                        K=base.K, dipole=base.dipole)


@pytest.fixture(scope="module")
def tiny4():
    s, w = synth.workload("tiny4")
    return s, w


def test_kernel_apply_matches(tiny4):
    s, w = tiny4
    z = synth.random_complex_vectors(7, s.n_prod, 1)
    with T().Context(s, batch=8) as ctx:
        out = ctx.kernel_apply(z)
    assert rel(out, (s.K @ z.T).T) < 1e-13


@pytest.mark.parametrize("sysname", ["tiny4", "ragged"])
def test_chi0_apply_matches_explicit_chi0(sysname, tiny4):
    if sysname == "tiny4":
        s, w = tiny4
        eps = w["eps"]
    else:
        s, eps = ragged_system(), 0.02
    M = O.transition_vertex(s)
    omegas = np.array([0.0, 0.13, 0.5, 0.77, 1.0, 0.31, 0.9])
    z = synth.random_complex_vectors(omegas.size, s.n_prod, 2)
    with T().Context(s, batch=omegas.size) as ctx:
        out = ctx.chi0_apply(z, omegas, eps)
        outA = ctx.apply_A(z, omegas, eps)
    for r, om in enumerate(omegas):
        chi = O.chi0_explicit(s, om, eps, M)
        assert rel(out[r], chi @ z[r]) < 1e-12
        assert rel(outA[r], z[r] - chi @ (s.K @ z[r])) < 1e-12


def test_single_rhs_and_device_pointers(tiny4):
    import torch
    s, w = tiny4
    z = synth.random_complex_vectors(1, s.n_prod, 3)
    op = O.StepOperator(s)
    with T().Context(s, batch=3) as ctx:
        host = ctx.chi0_apply(z, [0.4], w["eps"])
        dev = ctx.chi0_apply(torch.from_numpy(z).cuda(),
                             torch.tensor([0.4], dtype=torch.float64).cuda(), w["eps"])
        torch.cuda.synchronize()
    ref = op.apply(z[0], 0.4, w["eps"])
    assert rel(host[0], ref) < 1e-12
    assert rel(dev.cpu().numpy()[0], ref) < 1e-12


def test_spectrum_matches_dense_lu(tiny4):
    s, w = tiny4
    M = O.transition_vertex(s)
    om = w["omega"]
    with T().Context(s, batch=64, restart=w["restart"], tol=1e-12, max_restarts=100) as ctx:
        P, info = ctx.polarizability(om, w["eps"])
    assert info["converged"].all()
    P_lu = np.stack([O.polarizability_lu(s, x, w["eps"], M)[0] for x in om])
    assert rel(P, P_lu) < 1e-10
    # invariants of the spectrum
    assert rel(P, np.swapaxes(P, 1, 2)) < 1e-9
    assert np.max(np.abs(P[0].imag)) < 1e-9 * np.max(np.abs(P[0]))
    alpha = -P
    diag = np.einsum("wii->wi", alpha)[1:]
    assert np.all(diag.imag >= -1e-9 * np.max(np.abs(alpha)))


def test_spectrum_at_workload_tolerance_and_iteration_counts(tiny4):
    """At tol 1e-8 the GPU and the oracle's GMRES both stop early; each is
    within the conditioning bound of the LU answer and their Krylov
    dimensions agree to within one restart check."""
    s, w = tiny4
    om = w["omega"][::9]
    with T().Context(s, batch=32, restart=w["restart"], tol=w["tol"]) as ctx:
        P, info = ctx.polarizability(om, w["eps"])
    P_o, infos = O.polarizability_gmres(s, om, w["eps"], w["restart"], w["tol"])
    mv_o = np.array([i["matvecs"] for i in infos]).reshape(om.size, 3)
    assert np.all(np.abs(info["matvecs"] - mv_o) <= 2)
    assert info["converged"].all() and np.all(info["resid"] <= w["tol"])
    M = O.transition_vertex(s)
    P_lu = np.stack([O.polarizability_lu(s, x, w["eps"], M)[0] for x in om])
    assert rel(P, P_lu) < 1e-5
    assert rel(P, P_o) < 1e-5


def test_batches_smaller_than_the_spectrum(tiny4):
    """7 right-hand sides per group over 5 frequencies (15 solves): ragged groups."""
    s, w = tiny4
    om = np.array([0.05, 0.35, 0.6, 0.85, 0.95])
    with T().Context(s, batch=7, restart=12, tol=1e-12, max_restarts=200) as ctx:
        P, info = ctx.polarizability(om, w["eps"])
    M = O.transition_vertex(s)
    P_lu = np.stack([O.polarizability_lu(s, x, w["eps"], M)[0] for x in om])
    assert info["converged"].all()
    assert rel(P, P_lu) < 1e-10


def test_ragged_system_spectrum(tiny4):
    s = ragged_system()
    om = np.array([0.0, 0.21, 0.47, 0.8])
    M = O.transition_vertex(s)
    with T().Context(s, batch=5, restart=9, tol=1e-12, max_restarts=400) as ctx:
        P, info = ctx.polarizability(om, 0.02)
    P_lu = np.stack([O.polarizability_lu(s, x, 0.02, M)[0] for x in om])
    assert info["converged"].all()
    assert rel(P, P_lu) < 1e-10


def test_non_convergence_is_reported(tiny4):
    s, w = tiny4
    with T().Context(s, batch=3, restart=2, tol=1e-14, max_restarts=1) as ctx:
        with pytest.raises(T().TddftError) as e:
            ctx.polarizability([0.5], w["eps"])
        assert e.value.status == T().ERR_NOT_CONVERGED
        P, info = ctx.polarizability([0.5], w["eps"], raise_on_nonconvergence=False)
    assert not info["converged"].any() and np.all(info["matvecs"] == 3)
    assert np.all(np.isfinite(P))


def test_bad_call_arguments(tiny4):
    s, w = tiny4
    z = synth.random_complex_vectors(4, s.n_prod, 4)
    with T().Context(s, batch=3) as ctx:
        with pytest.raises(T().TddftError) as e:
            ctx.chi0_apply(z, np.zeros(4), w["eps"])
        assert e.value.status == T().ERR_SHAPE
        with pytest.raises(T().TddftError) as e:
            ctx.chi0_apply(z[:2], np.zeros(2), 0.0)
        assert e.value.status == T().ERR_INVALID_ARG
        with pytest.raises(T().TddftError) as e:
            ctx.polarizability([np.nan], w["eps"])
        assert e.value.status == T().ERR_INVALID_ARG
        # the context still works after rejected calls
        out = ctx.chi0_apply(z[:2], np.array([0.2, 0.3]), w["eps"])
    op = O.StepOperator(s)
    assert rel(out[1], op.apply(z[1], 0.3, w["eps"])) < 1e-12


@pytest.mark.slow
def test_medium64_operator_samples():
    """Full-size 64-atom molecule (9080 products): chi0 . z and A . z on a
    batch of 6 vectors against the oracle's five-step operator."""
    s, w = synth.workload("medium64")
    op = O.StepOperator(s)
    omegas = np.array([0.0, 0.3, 0.75, 1.1, 1.4, 1.5])
    z = synth.random_complex_vectors(omegas.size, s.n_prod, 5)
    with T().Context(s, batch=omegas.size) as ctx:
        out = ctx.apply_A(z, omegas, w["eps"])
    for r, om in enumerate(omegas):
        ref = z[r] - op.apply(s.K @ z[r], om, w["eps"])
        assert rel(out[r], ref) < 1e-12


@pytest.mark.slow
def test_medium64_spectrum_samples():
    """Full-size 64-atom molecule, restart 40, two frequencies x 3
    directions solved to 1e-10 on both sides."""
    s, w = synth.workload("medium64")
    om = w["omega"][[0, 160]]
    with T().Context(s, batch=12, restart=w["restart"], tol=1e-10) as ctx:
        P, info = ctx.polarizability(om, w["eps"])
    assert info["converged"].all()
    P_o, infos = O.polarizability_gmres(s, om, w["eps"], w["restart"], 1e-10)
    assert rel(P, P_o) < 1e-7
