"""Graph-captured GMRES iterations against the host-driven launch sequence:
replays of one captured iteration polled by the host (options.graph = 1)
and the whole loop on the device, one launch of a conditional WHILE node per
group (options.graph = 2).  Both give the same spectra and the same operator
counts as the host loop, for every precision and for groups smaller than
the spectrum."""
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


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "bf16x3emu", "tf32emu"])
@pytest.mark.parametrize("batch", [192, 50])
def test_graph_replays_match_host_driven_iterations(prec, batch):
    from paper_1005_5340_gb300 import tddft
    s, w = synth.workload("tiny4")
    om = w["omega"]
    out = {}
    for graph in (0, 1, 2):
        with tddft.Context(s, batch=batch, restart=w["restart"], tol=w["tol"], prec=prec,
                           graph=graph) as ctx:
            P, info = ctx.polarizability(om, w["eps"])
        assert info["converged"].all()
        out[graph] = (P, info)
    P0, i0 = out[0]
    for graph in (1, 2):
        P1, i1 = out[graph]
        assert np.array_equal(i0["matvecs"], i1["matvecs"]), graph
        assert np.max(np.abs(P1 - P0)) <= 1e-13 * np.max(np.abs(P0)), graph


def test_graph_mode_on_the_medium_molecule():
    from paper_1005_5340_gb300 import tddft
    s, w = synth.workload("medium64")
    om = w["omega"][::32]
    res = {}
    for graph in (0, 1, 2):
        with tddft.Context(s, batch=3 * om.size, restart=w["restart"], tol=w["tol"],
                           prec="bf16x3", graph=graph) as ctx:
            P, info = ctx.polarizability(om, w["eps"])
        assert info["converged"].all()
        res[graph] = P
    for graph in (1, 2):
        assert np.max(np.abs(res[graph] - res[0])) <= 1e-12 * np.max(np.abs(res[0]))
