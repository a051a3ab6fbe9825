"""Several molecules of uneven size in one batch (one graph per round with a
branch per molecule) against each molecule solved alone."""
import numpy as np
import pytest

from paper_1005_5340_gb300 import synth
from tests.libutil import ensure_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_library()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_batch_matches_molecules_alone(prec):
    from paper_1005_5340_gb300 import tddft
    mols = [synth.make_system(n, 4000 + i, density=0.0094) for i, n in enumerate((4, 9, 16, 6))]
    om = np.linspace(0.0, 1.5, 24)
    eps, tol = 0.005, 1e-8
    with tddft.Batch(mols, batch=30, restart=40, tol=tol, prec=prec) as b:
        P, st = b.polarizability(om, eps)
    assert st["converged"].all() and np.all(st["resid"] <= tol)
    for i, s in enumerate(mols):
        with tddft.Context(s, batch=30, restart=40, tol=tol, prec=prec) as ctx:
            Pi, info = ctx.polarizability(om, eps)
        assert np.array_equal(info["matvecs"], st["matvecs"][i])
        assert np.max(np.abs(P[i] - Pi)) <= 1e-13 * np.max(np.abs(Pi))
