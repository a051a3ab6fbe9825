"""The C boundary without a GPU: the library builds, loads, exports every
function include/tddft.h declares, and rejects bad input on the host before
any device work."""
import ctypes

import numpy as np
import pytest

from paper_1005_5340_gb300 import synth, tddft
from tests.libutil import ensure_library, header_functions


@pytest.fixture(scope="module")
def lib():
    return ensure_library()


def test_every_declared_function_is_exported_and_bound(lib):
    names = header_functions()
    assert "tddft_create" in names and "tddft_polarizability" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in tddft.SIGNATURES, n
    assert set(tddft.SIGNATURES) <= set(names)


def test_struct_layouts_match_the_header(tmp_path):
    """Sizes and field offsets of the structs the binding passes by pointer,
    as a C compiler lays them out from include/tddft.h."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"tddft_system": tddft._System, "tddft_options": tddft._Options,
               "tddft_solve_stats": tddft.SolveStats,
               "tddft_adaptive_options": tddft.AdaptiveOptions, "tddft_pole": tddft.Pole}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "tddft.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                         text=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(out[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(out[f"{cname}.{f}"]) == getattr(py, f).offset, f"{cname}.{f}"


def _create(sysm, **opt):
    lib = tddft.load_library()
    keep = dict(
        aoff=np.ascontiguousarray(sysm.atom_orb_offset, np.int32),
        E=np.ascontiguousarray(sysm.eigenvalues, np.float64),
        occ=np.ascontiguousarray(sysm.occupations, np.float64),
        X=np.asfortranarray(sysm.X, np.float64),
        pa=np.ascontiguousarray(sysm.prod_atoms, np.int32),
        voff=np.ascontiguousarray(sysm.vertex_offset, np.int64),
        v=np.ascontiguousarray(sysm.vertex, np.float64),
        K=np.ascontiguousarray(sysm.K, np.float64),
        d=np.ascontiguousarray(sysm.dipole, np.float64))
    s = tddft._System(sysm.n_atoms, keep["aoff"].ctypes.data, keep["E"].size, keep["E"].ctypes.data,
                      keep["occ"].ctypes.data, keep["X"].ctypes.data, keep["pa"].shape[0],
                      keep["pa"].ctypes.data, keep["voff"].ctypes.data, keep["v"].ctypes.data,
                      keep["K"].ctypes.data, keep["d"].ctypes.data)
    o = tddft._Options(opt.get("prec", 0), opt.get("restart", 10), opt.get("max_restarts", 5),
                       opt.get("tol", 1e-8), opt.get("batch", 4), None, opt.get("inner_tol", 1e-4),
                       opt.get("graph", 0), opt.get("stop", 0), opt.get("emu_slices", 0),
                       opt.get("n_tile", 0), opt.get("guess", 0), opt.get("wait_timeout_ns", 0))
    h = ctypes.c_void_p()
    st = lib.tddft_create(ctypes.byref(s), ctypes.byref(o), ctypes.byref(h))
    return st, lib.tddft_last_error(None).decode(), h


def _bad(mutate, **opt):
    s = synth.tiny_system(3)
    mutate(s)
    return _create(s, **opt)


def test_validation_rejects_bad_input_before_device_work(lib):
    def nan_k(s):
        s.K = s.K.copy(); s.K[0, 1] = np.nan
    st, msg, h = _bad(nan_k)
    assert st == tddft.ERR_INVALID_ARG and "NaN" in msg and not h.value

    def asym_k(s):
        s.K = s.K.copy(); s.K[0, 1] += 1e-3
    st, msg, _ = _bad(asym_k)
    assert st == tddft.ERR_UNSUPPORTED and "symmetric" in msg

    def unsorted(s):
        s.eigenvalues = s.eigenvalues[::-1].copy()
    assert _bad(unsorted)[0] == tddft.ERR_INVALID_ARG

    def fractional(s):
        s.occupations = s.occupations.copy(); s.occupations[0] = 1.0
    assert _bad(fractional)[0] == tddft.ERR_UNSUPPORTED

    def no_empty(s):
        s.occupations = np.full_like(s.occupations, 2.0)
    assert _bad(no_empty)[0] == tddft.ERR_UNSUPPORTED

    def bad_pair(s):
        s.prod_atoms = s.prod_atoms.copy(); s.prod_atoms[-1] = (1, 0)
    assert _bad(bad_pair)[0] == tddft.ERR_SHAPE

    def bad_offset(s):
        s.vertex_offset = s.vertex_offset.copy(); s.vertex_offset[1] += 1
    assert _bad(bad_offset)[0] == tddft.ERR_SHAPE

    def asym_local(s):
        s.vertex = s.vertex.copy(); s.vertex[1] += 0.5
    assert _bad(asym_local)[0] == tddft.ERR_INVALID_ARG

    assert _bad(lambda s: None, restart=0)[0] == tddft.ERR_INVALID_ARG
    assert _bad(lambda s: None, tol=-1.0)[0] == tddft.ERR_INVALID_ARG
    assert _bad(lambda s: None, batch=0)[0] == tddft.ERR_INVALID_ARG
    assert _bad(lambda s: None, prec=9)[0] == tddft.ERR_UNSUPPORTED
    assert _bad(lambda s: None, prec=2, inner_tol=0.0)[0] == tddft.ERR_INVALID_ARG
    assert _bad(lambda s: None, prec=2, inner_tol=1.5)[0] == tddft.ERR_INVALID_ARG
    assert _bad(lambda s: None, prec=3, inner_tol=0.0)[0] == tddft.ERR_INVALID_ARG
    assert _bad(lambda s: None, prec=-1)[0] == tddft.ERR_UNSUPPORTED
    assert _bad(lambda s: None, stop=3)[0] == tddft.ERR_INVALID_ARG
    assert _bad(lambda s: None, stop=-1)[0] == tddft.ERR_INVALID_ARG
    assert _bad(lambda s: None, prec=1, emu_slices=2)[0] == tddft.ERR_INVALID_ARG
    assert _bad(lambda s: None, prec=1, emu_slices=9)[0] == tddft.ERR_INVALID_ARG
    assert _bad(lambda s: None, prec=2, n_tile=96)[0] == tddft.ERR_INVALID_ARG
    assert _bad(lambda s: None, prec=2, n_tile=-64)[0] == tddft.ERR_INVALID_ARG
    assert _bad(lambda s: None, wait_timeout_ns=-1)[0] == tddft.ERR_INVALID_ARG
    assert _bad(lambda s: None, guess=3)[0] != tddft.OK


def test_emulated_gemm_rejects_bad_arguments_on_the_host(lib):
    f = lib.tddft_gemm_f64_emulated
    buf = ctypes.c_void_p(16)   # never dereferenced: every call fails validation
    assert f(4, 4, 4, None, 4, buf, 4, buf, 4, 6, None) == tddft.ERR_INVALID_ARG
    assert f(0, 4, 4, buf, 4, buf, 4, buf, 4, 6, None) == tddft.ERR_INVALID_ARG
    assert f(4, 4, 4, buf, 4, buf, 4, buf, 4, 2, None) == tddft.ERR_INVALID_ARG
    assert f(4, 4, 4, buf, 4, buf, 4, buf, 4, 9, None) == tddft.ERR_INVALID_ARG
    assert f(4, 4, 8, buf, 4, buf, 4, buf, 4, 6, None) == tddft.ERR_SHAPE
    assert f(4, 8, 4, buf, 4, buf, 4, buf, 8, 6, None) == tddft.ERR_SHAPE
    assert f(4, 8, 4, buf, 4, buf, 8, buf, 4, 6, None) == tddft.ERR_SHAPE


def test_more_than_16_orbitals_per_atom_is_unsupported(lib):
    s = synth.make_system(2, 4, orb_per_atom=17, occ_per_atom=1, n_local=2, n_bilocal=1,
                          density=0.02)
    st, msg, _ = _create(s)
    assert st == tddft.ERR_UNSUPPORTED and "16" in msg


def test_calls_on_a_null_context_fail_cleanly(lib):
    assert lib.tddft_chi0_apply(None, 1, None, 0.1, None, None, 0) == tddft.ERR_INVALID_ARG
    assert lib.tddft_polarizability(None, 1, None, 0.1, None, None, 0) == tddft.ERR_INVALID_ARG
    assert lib.tddft_spectrum_adaptive(None, 0.0, 1.0, 0.01, None, None, None, None, None, 0,
                                       None) == tddft.ERR_INVALID_ARG
    assert lib.tddft_mlp_save(None, b"x") == tddft.ERR_INVALID_ARG
    assert lib.tddft_mlp_load(None, b"x") == tddft.ERR_INVALID_ARG
    lib.tddft_destroy(None)
    assert isinstance(lib.tddft_last_error(None), bytes)


def test_create_without_a_gpu_reports_a_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, msg, h = _create(synth.tiny_system(3))
    assert st in (tddft.ERR_CUDA, tddft.ERR_NOMEM) and msg and not h.value


def test_sweep_plan_follows_its_definition(lib):
    """tddft_sweep_plan (host only): pass 0 = every 4th frequency and the last;
    pass 1 = the other indices 2 mod 4; pass 2 = the rest; every guessed
    frequency's neighbours are the nearest frequencies solved in earlier
    passes, one on each side."""
    for n in list(range(1, 14)) + [64, 257, 512]:
        pas, left, right = tddft.sweep_plan(n)
        for i in range(n):
            if i % 4 == 0 or i == n - 1:
                assert pas[i] == 0 and left[i] == -1 and right[i] == -1
            else:
                assert pas[i] == (1 if i % 4 == 2 else 2)
                before = [j for j in range(n) if pas[j] < pas[i]]
                assert left[i] == max(j for j in before if j < i)
                assert right[i] == min(j for j in before if j > i)
    assert lib.tddft_sweep_plan(0, None, None, None) == tddft.ERR_INVALID_ARG
