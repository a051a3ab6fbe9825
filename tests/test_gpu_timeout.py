"""The bounded waits of the tensor-core kernels (include/tddft.h,
wait_timeout_ns): with a limit too short for any real wait (1 ns), every
pipeline wait of the split-bf16 GEMM and of the emulated float64 GEMM gives
up; the kernels stop issuing work, let their own copies and MMAs finish,
free their tensor memory and return, so the call returns TIMEOUT instead of
hanging.  The same context then works again with the default limit, and its
results match the float64 path."""
import numpy as np
import pytest

from paper_1005_5340_gb300 import synth
from tests.libutil import ensure_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def medium():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_library()
    return synth.workload("medium64")


@pytest.mark.parametrize("prec,call", [("bf16x3", "apply_A"), ("fp64emu", "kernel_apply")])
def test_short_wait_limit_returns_timeout_and_the_context_recovers(medium, prec, call):
    from paper_1005_5340_gb300 import tddft
    s, w = medium
    z = synth.random_complex_vectors(24, s.n_prod, 5)
    om = np.linspace(0.1, 1.4, 24)
    args = (z, om, w["eps"]) if call == "apply_A" else (z,)
    with tddft.Context(s, batch=24) as ref_ctx:
        ref = getattr(ref_ctx, call)(*args)
    with tddft.Context(s, batch=24, prec=prec, wait_timeout_ns=1) as ctx:
        with pytest.raises(tddft.TddftError) as ei:
            getattr(ctx, call)(*args)
        assert ei.value.status == tddft.ERR_TIMEOUT
        assert "gave up" in str(ei.value)
        ctx.set_wait_timeout(0)
        out = getattr(ctx, call)(*args)
    tol = 1e-4 if prec == "bf16x3" else 1e-11
    d = (out - z, ref - z) if call == "apply_A" else (out, ref)
    err = np.max(np.abs(d[0] - d[1])) / np.max(np.abs(d[1]))
    assert err < tol, err
