"""Checkpoint and resume of a spectrum (tddft_polarizability_resume): every
(omega, direction) is independent (Sec. 6.2.3), so a spectrum computed in
pieces, with a record appended per finished frequency, equals the spectrum
computed at once; a later call solves only what the file lacks; a record cut
short by an interruption is solved again; another problem's file is refused."""
import os

import numpy as np
import pytest

from paper_1005_5340_gb300 import synth
from tests.libutil import ensure_library

pytestmark = pytest.mark.gpu

RECORD, HEADER = 280, 64


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_library()


def test_resume_solves_only_missing_frequencies(tmp_path):
    from paper_1005_5340_gb300 import tddft
    s, w = synth.workload("tiny4")
    om = w["omega"][:20]
    path = str(tmp_path / "spectrum.ckp")
    with tddft.Context(s, batch=12, restart=w["restart"], tol=1e-11) as ctx:
        P_all, st_all = ctx.polarizability(om, w["eps"])
        P1, st1, n1 = ctx.polarizability_resume(om[:8], w["eps"], path)
        assert n1 == 8 and os.path.getsize(path) == HEADER + 8 * RECORD
        P2, st2, n2 = ctx.polarizability_resume(om, w["eps"], path)
        assert n2 == 12 and os.path.getsize(path) == HEADER + 20 * RECORD
        P3, st3, n3 = ctx.polarizability_resume(om, w["eps"], path)
        assert n3 == 0
        assert np.array_equal(P3, P2) and np.array_equal(st3["matvecs"], st2["matvecs"])
        # an interruption in the middle of the last record: that frequency is solved again
        with open(path, "r+b") as f:
            f.truncate(HEADER + 19 * RECORD + 100)
        P4, st4, n4 = ctx.polarizability_resume(om, w["eps"], path)
        assert n4 == 1 and os.path.getsize(path) == HEADER + 20 * RECORD
    ref = np.max(np.abs(P_all))
    for P in (P1, P2[:8]):
        assert np.max(np.abs(P - P_all[:8])) <= 1e-10 * ref
    assert np.max(np.abs(P2 - P_all)) <= 1e-10 * ref
    assert np.max(np.abs(P4 - P_all)) <= 1e-10 * ref
    assert st2["converged"].all()


def test_checkpoint_of_another_problem_is_refused(tmp_path):
    from paper_1005_5340_gb300 import tddft
    s, w = synth.workload("tiny4")
    path = str(tmp_path / "a.ckp")
    with tddft.Context(s, batch=6, restart=w["restart"], tol=1e-8) as ctx:
        ctx.polarizability_resume(w["omega"][:2], w["eps"], path)
    with tddft.Context(s, batch=6, restart=w["restart"], tol=1e-9) as ctx:
        with pytest.raises(tddft.TddftError) as e:
            ctx.polarizability_resume(w["omega"][:2], w["eps"], path)
        assert e.value.status == tddft.ERR_INVALID_ARG and "another problem" in str(e.value)
    bad = tmp_path / "b.ckp"
    bad.write_bytes(b"x" * 100)
    with tddft.Context(s, batch=6, restart=w["restart"], tol=1e-8) as ctx:
        with pytest.raises(tddft.TddftError) as e:
            ctx.polarizability_resume(w["omega"][:2], w["eps"], str(bad))
        assert e.value.status == tddft.ERR_INVALID_ARG
