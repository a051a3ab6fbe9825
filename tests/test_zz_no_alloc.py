"""tddft_chi0_apply_noalloc against tddft_chi0_apply, through the C boundary.

The allocation-free variant serves callers that cannot allocate device
memory at the time of the call; it must give the same float64 product as the
regular entry point, also on a second call that reuses the same reserved
block with different inputs.  This file sorts last so that a failure here
leaves every other test already run."""
import ctypes

import numpy as np
import pytest

from paper_1005_5340_gb300 import synth
from tests.libutil import ensure_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_library()


def _noalloc(lib, ctx, z, om, eps):
    import torch
    out = torch.empty_like(z)
    st = lib.tddft_chi0_apply_noalloc(ctx.h, z.shape[0], om.data_ptr(), eps,
                                      torch.view_as_real(z).data_ptr(),
                                      torch.view_as_real(out).data_ptr(), 1)
    torch.cuda.synchronize()
    return st, out


def test_noalloc_matches_chi0_apply_on_two_calls(lib):
    import torch
    from paper_1005_5340_gb300 import tddft
    s, w = synth.workload("tiny4")
    eps = w["eps"]
    dev = torch.device("cuda", 0)
    with tddft.Context(s, batch=8) as ctx:
        for seed, n in ((21, 5), (22, 3)):
            z = torch.from_numpy(synth.random_complex_vectors(n, s.n_prod, seed)).to(dev)
            om = torch.linspace(0.05 * seed - 1.0, 0.05 * seed - 0.2, n, dtype=torch.float64,
                                device=dev).abs()
            ref = ctx.chi0_apply(z, om, eps)
            st, out = _noalloc(lib, ctx, z, om, eps)
            assert st == tddft.OK, lib.tddft_last_error(ctx.h)
            ref, out = ref.cpu().numpy(), out.cpu().numpy()
            err = np.max(np.abs(out - ref)) / np.max(np.abs(ref))
            assert err <= 1e-12, err


def test_noalloc_rejects_host_pointers_and_oversize_requests(lib):
    import torch
    from paper_1005_5340_gb300 import tddft
    s, w = synth.workload("tiny4")
    with tddft.Context(s, batch=2) as ctx:
        z = np.zeros((1, s.n_prod), dtype=np.complex128)
        om = np.zeros(1)
        out = np.zeros_like(z)
        st = lib.tddft_chi0_apply_noalloc(ctx.h, 1, om.ctypes.data, 0.01, z.ctypes.data,
                                          out.ctypes.data, 0)
        assert st == tddft.ERR_INVALID_ARG
        n = 4096   # far beyond the 16 MiB block for this molecule
        zt = torch.zeros((n, s.n_prod), dtype=torch.complex128, device="cuda")
        omt = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, _ = _noalloc(lib, ctx, zt, omt, 0.01)
        assert st == tddft.ERR_SHAPE
        assert b"16777216" in lib.tddft_last_error(ctx.h)
