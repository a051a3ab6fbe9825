"""The split-bf16 K product in the launch modes the 64-atom workload's full
batches take: two K halves added into a zeroed output (split K) and clusters
of 2-3 CTAs, one per N tile of an M row block, at each N tile width (64, 128,
256).  apply_A of a refinement-form context (every product in split bf16,
relative error ~1e-5) is compared with the float64 context for every vector
and with the oracle's operator z - chi0 (K z) (Sec. 4.1, the five steps of
Table t:flops) for vectors sampled from every N tile, at <= 1e-4."""
import numpy as np
import pytest

import oracle.tddft_oracle as O
from paper_1005_5340_gb300 import synth
from tests.libutil import ensure_library

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

# (right-hand sides, N tile): 2 n_rhs real columns in 1-6 N tiles of 71 M tiles
CASES = [(96, 64), (96, 128), (96, 256), (192, 64), (192, 128), (192, 256)]
PLANS = {}


@pytest.fixture(scope="module")
def medium():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_library()
    from paper_1005_5340_gb300 import tddft
    s, w = synth.workload("medium64")
    op = O.StepOperator(s)
    z = synth.random_complex_vectors(192, s.n_prod, 77)
    om = np.linspace(0.0, 1.5, 192)[np.random.default_rng(3).permutation(192)]
    with tddft.Context(s, batch=192) as ctx:
        ref = ctx.apply_A(z, om, w["eps"])
    return s, w, op, z, om, ref


def vrel(a, b):
    return np.max(np.abs(a - b), axis=-1) / np.max(np.abs(b), axis=-1)


@pytest.mark.parametrize("n_rhs,bn", CASES)
def test_k_product_launch_modes_match_the_oracle(medium, n_rhs, bn):
    from paper_1005_5340_gb300 import tddft
    s, w, op, z, om, ref = medium
    with tddft.Context(s, batch=n_rhs, prec="bf16x3", n_tile=bn) as ctx:
        assert ctx.tuning() == (bn, bn, bn)
        plan = ctx.kproduct_plan(n_rhs)
        Az = ctx.apply_A(z[:n_rhs], om[:n_rhs], w["eps"])
    PLANS[(n_rhs, bn)] = plan
    print(f"n_rhs {n_rhs}, N tile {bn}: clusters of {plan[0]}, {plan[1]} K slice(s)")
    # every vector against the float64 path: the chi0 K z part, per vector
    e = vrel(Az - z[:n_rhs], ref[:n_rhs] - z[:n_rhs])
    assert np.all(e < 1e-4), (np.argmax(e), e.max())
    # vectors from every N tile (real columns 2r, 2r+1; tiles of <= bn columns)
    ntiles = -(-2 * n_rhs // bn)
    tn = min(bn, (-(-2 * n_rhs // ntiles) + 15) // 16 * 16)
    picks = sorted({min(n_rhs - 1, (t * tn + tn // 2) // 2) for t in range(ntiles)} | {n_rhs - 1})
    for r in picks[:4]:
        oref = z[r] - op.apply(s.K @ z[r], om[r], w["eps"])
        assert vrel(Az[r] - z[r], oref - z[r]) < 1e-4, r


def test_the_launch_modes_were_taken():
    """The cases above cover clusters (2 and 3 CTAs) and the split K."""
    if len(PLANS) < len(CASES):
        pytest.skip("the parametrised cases did not all run")
    ncl = {p[0] for p in PLANS.values()}
    ks = {p[1] for p in PLANS.values()}
    assert {2, 3} <= ncl and 2 in ks, PLANS
    assert any(p[0] > 1 and p[1] == 2 for p in PLANS.values()), PLANS
