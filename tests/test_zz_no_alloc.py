"""tddft_chi0_apply_noalloc against tddft_chi0_apply and the oracle, through
the C boundary.

The allocation-free variant serves callers that cannot allocate device
memory at the time of the call; it must give the same float64 product as the
regular entry point of a float64 context (and as the oracle's explicit
chi0), whatever the precision of the context it is called on, also on a
second call that reuses the same reserved block with different inputs, and
at a size that fills most of the block.  This file sorts last so that a
failure here leaves every other test already run."""
import numpy as np
import pytest

import oracle.tddft_oracle as O
from paper_1005_5340_gb300 import synth
from tests.libutil import ensure_library

pytestmark = pytest.mark.gpu

BLOCK_DOUBLES = 2 * 1024 * 1024   # the 16 MiB block stated in include/tddft.h


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


def scratch_doubles(n, ctx):
    """Scratch of n right-hand sides by the header's formula (each term
    rounded up to a multiple of 32 doubles)."""
    up = lambda x: (x + 31) // 32 * 32   # noqa: E731
    n_virt = ctx.n_orb - ctx.n_occ
    return (2 * up(2 * n * ctx.n_prod) + up(2 * n * ctx.n_blocks * 256)
            + 2 * up(ctx.n_orb * 2 * n * ctx.n_occ) + up(n_virt * 2 * n * ctx.n_occ) + up(n))


def largest_fit(ctx):
    n = 1
    while scratch_doubles(n + 1, ctx) <= BLOCK_DOUBLES:
        n += 1
    return n


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "bf16x3emu"])
def test_noalloc_matches_chi0_apply_on_two_calls(lib, prec):
    import torch
    from paper_1005_5340_gb300 import tddft
    s, w = synth.workload("tiny4")
    eps = w["eps"]
    dev = torch.device("cuda", 0)
    Mv = O.transition_vertex(s)
    with tddft.Context(s, batch=8, prec=prec) as ctx, tddft.Context(s, batch=8) as ref_ctx:
        for seed, n in ((21, 5), (22, 3)):
            z = torch.from_numpy(synth.random_complex_vectors(n, s.n_prod, seed)).to(dev)
            om = torch.linspace(0.05 * seed - 1.0, 0.05 * seed - 0.2, n, dtype=torch.float64,
                                device=dev).abs()
            ref = ref_ctx.chi0_apply(z, om, eps)
            st, out = _noalloc(lib, ctx, z, om, eps)
            assert st == tddft.OK, lib.tddft_last_error(ctx.h)
            assert lib.tddft_last_error(ctx.h) == b""
            ref, out, zn, omn = ref.cpu().numpy(), out.cpu().numpy(), z.cpu().numpy(), om.cpu().numpy()
            err = np.max(np.abs(out - ref)) / np.max(np.abs(ref))
            assert err <= 1e-12, err
            for r in range(n):
                c = O.chi0_explicit(s, omn[r], eps, Mv) @ zn[r]
                assert np.max(np.abs(out[r] - c)) / np.max(np.abs(c)) <= 1e-12


def test_noalloc_at_the_largest_size_that_fits(lib):
    """The largest n_rhs whose scratch fits the block works (twice, with
    different inputs); one more is rejected with SHAPE before any work."""
    import torch
    from paper_1005_5340_gb300 import tddft
    s, w = synth.workload("tiny4")
    eps = w["eps"]
    with tddft.Context(s, batch=2) as probe:
        n = largest_fit(probe)
    assert n > 100
    with tddft.Context(s, batch=n) as ctx:
        for seed in (31, 32):
            z = torch.from_numpy(synth.random_complex_vectors(n, s.n_prod, seed)).cuda()
            om = torch.linspace(0.0, 1.0, n, dtype=torch.float64, device="cuda") * (seed - 30)
            ref = ctx.chi0_apply(z, om, eps).cpu().numpy()
            st, out = _noalloc(lib, ctx, z, om, eps)
            assert st == tddft.OK, lib.tddft_last_error(ctx.h)
            out = out.cpu().numpy()
            assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) <= 1e-12
        zt = torch.zeros((n + 1, s.n_prod), dtype=torch.complex128, device="cuda")
        omt = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
        st, _ = _noalloc(lib, ctx, zt, omt, eps)
        assert st == tddft.ERR_SHAPE


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
