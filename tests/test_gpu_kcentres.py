"""The matrix-free K z from product centres (tddft_kernel_apply_centres, a
labelled variant of the matrix-free Hartree product, Sec. 5 multipole form
at its monopole term, Sec. 8): against the dense kernel of the synthetic
generator, K = 1 / sqrt(|C_mu - C_nu|^2 + 1) + 0.05 I, applied by numpy, at
the float64 operator tolerance (1e-12); ragged numbers of right-hand sides; argument errors."""
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


def centres_of(s):
    uc, inv = np.unique(s.centres, axis=0, return_inverse=True)
    return uc, inv.astype(np.int32).ravel()


@pytest.mark.parametrize("name,n_rhs", [("tiny4", 1), ("tiny4", 7), ("medium64", 13)])
def test_centre_form_matches_the_dense_kernel(name, n_rhs):
    import torch
    from paper_1005_5340_gb300 import tddft
    s, w = synth.workload(name)
    uc, pc = centres_of(s)
    assert uc.shape[0] < s.n_prod
    z = synth.random_complex_vectors(n_rhs, s.n_prod, 17)
    out = tddft.kernel_apply_centres(uc, pc, torch.from_numpy(z).cuda()).cpu().numpy()
    ref = (s.K @ z.T).T
    err = np.max(np.abs(out - ref), axis=1) / np.max(np.abs(ref), axis=1)
    print(f"{name}: {uc.shape[0]} centres for {s.n_prod} products, max error {err.max():.2e}")
    assert np.all(err < 1e-12)   # the float64 operator tolerance: sums of ~1e4 terms


def test_centre_form_rejects_bad_arguments():
    import torch
    from paper_1005_5340_gb300 import tddft
    s, w = synth.workload("tiny4")
    uc, pc = centres_of(s)
    z = torch.zeros((1, s.n_prod), dtype=torch.complex128, device="cuda")
    bad = pc.copy()
    bad[3] = uc.shape[0]
    with pytest.raises(tddft.TddftError) as e:
        tddft.kernel_apply_centres(uc, bad, z)
    assert e.value.status == tddft.ERR_SHAPE
    with pytest.raises(tddft.TddftError) as e:
        tddft.kernel_apply_centres(uc, pc, z, softening=-1.0)
    assert e.value.status == tddft.ERR_INVALID_ARG
