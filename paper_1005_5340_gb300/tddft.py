"""Python binding of libtddft (include/tddft.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels.  Host numpy
arrays or CUDA torch tensors are accepted; torch supplies device memory and
the stream.  If the shared library is missing the import fails loudly: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtddft.so")

OK, ERR_INVALID_ARG, ERR_SHAPE, ERR_NOMEM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_TIMEOUT, \
    ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ["OK", "INVALID_ARG", "SHAPE", "NOMEM", "CUDA", "NOT_CONVERGED", "TIMEOUT",
                "UNSUPPORTED"]
DEVICE_PTRS = 1
PREC = {"fp64": 0, "fp64emu": 1, "bf16x3": 2, "bf16x3emu": 3, "tf32": 4, "tf32emu": 5}
# initial guesses of tddft_polarizability
GUESS = {"zero": 0, "interp": 1, "learned": 2, "interp_subspace": 3, "learned_subspace": 4}
# GMRES stopping rules (Sec. 4.1): relative residual, eps_P, eps_P and eps_X
STOP = {"residual": 0, "eps_p": 1, "eps_px": 2}


class TddftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class _System(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("atom_orb_offset", ctypes.c_void_p),
                ("n_orb", ctypes.c_int32), ("eigenvalues", ctypes.c_void_p),
                ("occupations", ctypes.c_void_p), ("X", ctypes.c_void_p),
                ("n_prod", ctypes.c_int32), ("prod_atoms", ctypes.c_void_p),
                ("vertex_offset", ctypes.c_void_p), ("vertex", ctypes.c_void_p),
                ("K", ctypes.c_void_p), ("dipole", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("max_restarts", ctypes.c_int32), ("tol", ctypes.c_double),
                ("batch", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("inner_tol", ctypes.c_double), ("graph", ctypes.c_int32),
                ("stop", ctypes.c_int32), ("emu_slices", ctypes.c_int32),
                ("n_tile", ctypes.c_int32), ("guess", ctypes.c_int32),
                ("wait_timeout_ns", ctypes.c_int64)]


class SolveStats(ctypes.Structure):
    _fields_ = [("matvecs", ctypes.c_int32), ("cycles", ctypes.c_int32),
                ("resid", ctypes.c_double), ("converged", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("eps_p", ctypes.c_double),
                ("eps_x", ctypes.c_double)]


class AdaptiveOptions(ctypes.Structure):
    _fields_ = [("n_initial", ctypes.c_int32), ("max_points", ctypes.c_int32),
                ("rel_tol", ctypes.c_double), ("min_step", ctypes.c_double),
                ("peak_floor", ctypes.c_double)]


class Pole(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("g_re", ctypes.c_double), ("g_im", ctypes.c_double),
                ("peak", ctypes.c_double), ("omega_peak", ctypes.c_double)]


# Every exported symbol with its ctypes signature (checked by the tests
# against include/tddft.h).
_P = ctypes.c_void_p
SIGNATURES = {
    "tddft_create": (ctypes.c_int, [ctypes.POINTER(_System), ctypes.POINTER(_Options),
                                    ctypes.POINTER(ctypes.c_void_p)]),
    "tddft_chi0_apply": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_double, _P, _P,
                                        ctypes.c_int32]),
    "tddft_chi0_apply_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_double, _P, _P,
                                                ctypes.c_int32]),
    "tddft_kernel_apply": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int32]),
    "tddft_kernel_apply_centres": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, _P,
                                                  ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                                  _P, _P, _P]),
    "tddft_apply_A": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_double, _P, _P,
                                     ctypes.c_int32]),
    "tddft_polarizability": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_double, _P, _P,
                                            ctypes.c_int32]),
    "tddft_polarizability_guess": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_double, _P,
                                                  _P, _P, _P, ctypes.c_int32]),
    "tddft_polarizability_resume": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_double, _P, _P,
                                                   ctypes.c_char_p, _P]),
    "tddft_sizes": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "tddft_spectrum_adaptive": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, _P, _P, _P, _P, _P,
                                               ctypes.c_int32, _P]),
    "tddft_tuning": (ctypes.c_int, [_P, _P]),
    "tddft_set_wait_timeout": (ctypes.c_int, [_P, ctypes.c_int64]),
    "tddft_kproduct_plan": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "tddft_batch_create": (ctypes.c_int, [ctypes.c_int32, _P, _P, ctypes.POINTER(ctypes.c_void_p)]),
    "tddft_batch_polarizability": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_double, _P, _P]),
    "tddft_batch_context": (ctypes.c_void_p, [_P, ctypes.c_int32]),
    "tddft_batch_last_error": (ctypes.c_char_p, [_P]),
    "tddft_batch_destroy": (None, [_P]),
    "tddft_mlp_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int64, ctypes.c_uint64, _P,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "tddft_mlp_destroy": (None, [_P]),
    "tddft_mlp_last_error": (ctypes.c_char_p, [_P]),
    "tddft_mlp_num_params": (ctypes.c_int64, [_P]),
    "tddft_mlp_params": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32]),
    "tddft_mlp_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "tddft_mlp_load": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "tddft_mlp_forward": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, ctypes.c_int32]),
    "tddft_mlp_backward": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P]),
    "tddft_mlp_train_step": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P,
                                            _P, ctypes.c_float]),
    "tddft_guess_features": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_double,
                                            _P, _P, _P, _P]),
    "tddft_guess_combine": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, _P, _P, _P, _P, _P]),
    "tddft_sweep_plan": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P]),
    "tddft_set_guess": (ctypes.c_int, [_P, ctypes.c_int32]),
    "tddft_guess_load": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "tddft_timing_enable": (ctypes.c_int, [_P, ctypes.c_int32]),
    "tddft_timing_count": (ctypes.c_int32, [_P]),
    "tddft_timing_get": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_char_p),
                                        _P, _P, _P]),
    "tddft_timing_bytes": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "tddft_selftest_gemm": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
    "tddft_selftest_gemm_tf32": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
    "tddft_gemm_f64_emulated": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                               _P, ctypes.c_int64, _P, ctypes.c_int64, _P,
                                               ctypes.c_int64, ctypes.c_int32, _P]),
    "tddft_last_error": (ctypes.c_char_p, [_P]),
    "tddft_destroy": (None, [_P]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtddft.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_1005_5340_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _marshal(system):
    """A _System pointing into contiguous copies (returned too, to keep them alive)."""
    keep = dict(
        aoff=_c(system.atom_orb_offset, np.int32), E=_c(system.eigenvalues, np.float64),
        occ=_c(system.occupations, np.float64),
        X=np.asfortranarray(system.X, dtype=np.float64),
        pa=_c(system.prod_atoms, np.int32), voff=_c(system.vertex_offset, np.int64),
        v=_c(system.vertex, np.float64), K=_c(system.K, np.float64),
        d=_c(system.dipole, np.float64))
    s = _System(int(system.n_atoms), keep["aoff"].ctypes.data, int(keep["E"].size),
                keep["E"].ctypes.data, keep["occ"].ctypes.data, keep["X"].ctypes.data,
                int(keep["pa"].shape[0]), keep["pa"].ctypes.data, keep["voff"].ctypes.data,
                keep["v"].ctypes.data, keep["K"].ctypes.data, keep["d"].ctypes.data)
    return s, keep


class Context:
    """One molecule resident on the GPU (tddft_create .. tddft_destroy)."""

    def __init__(self, system, *, restart: int = 40, max_restarts: int = 200, tol: float = 1e-6,
                 batch: int = 64, prec: str = "fp64", inner_tol: float = 1e-4, stream=None,
                 graph: int = 0, stop: str = "residual", emu_slices: int = 0,
                 n_tile: int = 0, guess: str = "zero", wait_timeout_ns: int = 0):
        lib = load_library()
        self._lib = lib
        s, keep = _marshal(system)
        if stream is None:
            stream = _current_stream()
        self.stream_handle = stream
        o = _Options(PREC[prec], restart, max_restarts, tol, batch, stream or 0, inner_tol,
                     int(graph), STOP[stop], emu_slices, n_tile, GUESS[guess],
                     wait_timeout_ns)
        self.prec = prec
        h = ctypes.c_void_p()
        st = lib.tddft_create(ctypes.byref(s), ctypes.byref(o), ctypes.byref(h))
        if st != OK:
            raise TddftError(st, lib.tddft_last_error(None).decode())
        self.h = h
        self.batch = batch
        self.n_prod = int(system.n_prod)
        n_orb, n_occ, n_prod, nb = (ctypes.c_int32() for _ in range(4))
        lib.tddft_sizes(h, ctypes.byref(n_orb), ctypes.byref(n_occ), ctypes.byref(n_prod),
                        ctypes.byref(nb))
        self.n_orb, self.n_occ, self.n_blocks = n_orb.value, n_occ.value, nb.value

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self._lib.tddft_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st):
        if st != OK:
            raise TddftError(st, self._lib.tddft_last_error(self.h).decode())

    # -- operators -----------------------------------------------------------
    def _apply(self, fn, z, omega, eps, with_omega: bool):
        if _is_torch(z) and z.is_cuda:
            import torch
            z = z.to(torch.complex128).contiguous()
            n = z.shape[0]
            out = torch.empty_like(z)
            args = [self.h, n]
            if with_omega:
                om = torch.as_tensor(omega, dtype=torch.float64, device=z.device).reshape(-1)
                om = om.expand(n).contiguous() if om.numel() == 1 else om.contiguous()
                args += [om.data_ptr(), float(eps)]
            args += [torch.view_as_real(z).data_ptr(), torch.view_as_real(out).data_ptr(),
                     DEVICE_PTRS]
            self._check(fn(*args))
            return out
        z = np.ascontiguousarray(np.atleast_2d(z), dtype=np.complex128)
        n = z.shape[0]
        out = np.empty_like(z)
        args = [self.h, n]
        if with_omega:
            om = np.broadcast_to(np.asarray(omega, dtype=np.float64), (n,)).copy()
            args += [om.ctypes.data, float(eps)]
        args += [z.ctypes.data, out.ctypes.data, 0]
        self._check(fn(*args))
        return out

    def chi0_apply(self, z, omega, eps):
        """chi0(omega_r) z_r for each row r of z (n_rhs x n_prod complex)."""
        return self._apply(self._lib.tddft_chi0_apply, z, omega, eps, True)

    def chi0_apply_noalloc(self, z, omega, eps):
        """chi0(omega_r) z_r in float64 using only the library's reserved
        device block (no allocation); z and omega must be CUDA tensors."""
        import torch
        z = z.to(torch.complex128).contiguous()
        n = z.shape[0]
        om = torch.as_tensor(omega, dtype=torch.float64, device=z.device).reshape(-1).contiguous()
        out = torch.empty_like(z)
        self._check(self._lib.tddft_chi0_apply_noalloc(
            self.h, n, om.data_ptr(), float(eps), torch.view_as_real(z).data_ptr(),
            torch.view_as_real(out).data_ptr(), DEVICE_PTRS))
        return out

    def kernel_apply(self, z):
        """K z_r for each row r of z."""
        return self._apply(self._lib.tddft_kernel_apply, z, None, None, False)

    def apply_A(self, z, omega, eps):
        """z_r - chi0(omega_r) K z_r for each row r of z."""
        return self._apply(self._lib.tddft_apply_A, z, omega, eps, True)

    def polarizability_guess(self, omega, eps, x0=None, want_x: bool = True, *,
                             raise_on_nonconvergence: bool = True):
        """Like polarizability, on CUDA tensors, with optional initial guesses
        x0 (n_omega*3 x n_prod complex, row w*3+k) and the solutions returned
        (same layout) when want_x.  Returns (P, X or None, stats)."""
        import torch
        om = torch.as_tensor(omega, dtype=torch.float64).cuda().contiguous()
        n = om.numel()
        P = torch.empty((n, 3, 3), dtype=torch.complex128, device=om.device)
        X = torch.empty((3 * n, self.n_prod), dtype=torch.complex128, device=om.device) \
            if want_x else None
        if x0 is not None:
            x0 = x0.to(torch.complex128).contiguous()
            assert x0.shape == (3 * n, self.n_prod)
        stats = (SolveStats * (3 * n))()
        st = self._lib.tddft_polarizability_guess(
            self.h, n, om.data_ptr(), float(eps),
            torch.view_as_real(x0).data_ptr() if x0 is not None else None,
            torch.view_as_real(X).data_ptr() if X is not None else None,
            torch.view_as_real(P).data_ptr(), stats, DEVICE_PTRS)
        if st != OK and not (st == ERR_NOT_CONVERGED and not raise_on_nonconvergence):
            self._check(st)
        return P, X, _stats_dict(stats, n)

    def guess_features(self, nb, t, omega, direction, h_over_eps, X):
        """Features F, interpolation lin and scale of the targets (CUDA tensors)."""
        import torch
        dev = X.device
        nb = torch.as_tensor(nb, dtype=torch.int32, device=dev).contiguous()
        t = torch.as_tensor(t, dtype=torch.float64, device=dev).contiguous()
        om = torch.as_tensor(omega, dtype=torch.float64, device=dev).contiguous()
        dr = torch.as_tensor(direction, dtype=torch.int32, device=dev).contiguous()
        nt = t.numel()
        F = torch.empty((nt * self.n_prod, 10), dtype=torch.float32, device=dev)
        lin = torch.empty((nt, self.n_prod), dtype=torch.complex128, device=dev)
        scale = torch.empty(nt, dtype=torch.float64, device=dev)
        self._check(self._lib.tddft_guess_features(
            self.h, nt, nb.data_ptr(), t.data_ptr(), om.data_ptr(), dr.data_ptr(),
            float(h_over_eps), torch.view_as_real(X.contiguous()).data_ptr(), F.data_ptr(),
            torch.view_as_real(lin).data_ptr(), scale.data_ptr()))
        return F, lin, scale

    def spectrum_adaptive(self, w_lo, w_hi, eps, *, n_initial: int = 33, max_points: int = 512,
                          rel_tol: float = 0.02, min_step: float | None = None,
                          peak_floor: float = 0.02, max_poles: int = 256):
        """tddft_spectrum_adaptive: (omega [n], P [n, 3, 3] complex, poles) with
        poles a list of dicts (omega, g, peak, omega_peak)."""
        o = AdaptiveOptions(n_initial, max_points, rel_tol,
                            eps / 8.0 if min_step is None else min_step, peak_floor)
        om = np.empty(max_points, dtype=np.float64)
        P = np.empty((max_points, 3, 3), dtype=np.complex128)
        poles = (Pole * max(1, max_poles))()
        n_pts, n_pol = ctypes.c_int32(), ctypes.c_int32()
        st = self._lib.tddft_spectrum_adaptive(self.h, float(w_lo), float(w_hi), float(eps),
                                               ctypes.byref(o), om.ctypes.data, P.ctypes.data,
                                               ctypes.byref(n_pts), poles, max_poles,
                                               ctypes.byref(n_pol))
        self._check(st)
        n = n_pts.value
        out = [dict(omega=p.omega, g=complex(p.g_re, p.g_im), peak=p.peak,
                    omega_peak=p.omega_peak) for p in poles[:min(n_pol.value, max_poles)]]
        return om[:n].copy(), P[:n].copy(), out

    def polarizability(self, omega, eps, *, raise_on_nonconvergence: bool = True):
        """P[w, i, k] (complex, n_omega x 3 x 3) and per-(w, k) stats."""
        if _is_torch(omega) and omega.is_cuda:
            import torch
            om = omega.to(torch.float64).contiguous()
            n = om.numel()
            P = torch.empty((n, 3, 3), dtype=torch.complex128, device=om.device)
            stats = (SolveStats * (3 * n))()
            st = self._lib.tddft_polarizability(self.h, n, om.data_ptr(), float(eps),
                                                torch.view_as_real(P).data_ptr(), stats,
                                                DEVICE_PTRS)
        elif _is_torch(omega):
            # host tensors (pinned ones are copied without staging); P in pinned memory
            import torch
            om = omega.to(torch.float64).contiguous()
            n = om.numel()
            P = torch.empty((n, 3, 3), dtype=torch.complex128,
                            pin_memory=torch.cuda.is_available())
            stats = (SolveStats * (3 * n))()
            st = self._lib.tddft_polarizability(self.h, n, om.data_ptr(), float(eps),
                                                torch.view_as_real(P).data_ptr(), stats, 0)
        else:
            om = np.ascontiguousarray(np.atleast_1d(omega), dtype=np.float64)
            n = om.size
            P = np.empty((n, 3, 3), dtype=np.complex128)
            stats = (SolveStats * (3 * n))()
            st = self._lib.tddft_polarizability(self.h, n, om.ctypes.data, float(eps),
                                                P.ctypes.data, stats, 0)
        if st != OK and not (st == ERR_NOT_CONVERGED and not raise_on_nonconvergence):
            self._check(st)
        return P, _stats_dict(stats, n)

    def set_guess(self, mode: str):
        """tddft_set_guess: 'zero', 'interp' or 'learned' for the later solves."""
        self._check(self._lib.tddft_set_guess(self.h, GUESS[mode]))

    def guess_load(self, path):
        """tddft_guess_load: the learned guess's network from a tddft_mlp_save file."""
        self._check(self._lib.tddft_guess_load(self.h, os.fsencode(path)))

    def set_wait_timeout(self, ns: int):
        """tddft_set_wait_timeout: the limit of the tensor-core kernels' waits (0 = 2 s)."""
        self._check(self._lib.tddft_set_wait_timeout(self.h, int(ns)))

    def kproduct_plan(self, n_rhs: int):
        """(cluster size, K slices) of the split-bf16 K product for n_rhs vectors."""
        ncl, ks = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.tddft_kproduct_plan(self.h, n_rhs, ctypes.byref(ncl),
                                                  ctypes.byref(ks)))
        return ncl.value, ks.value

    def polarizability_resume(self, omega, eps, path, *, raise_on_nonconvergence: bool = True):
        """tddft_polarizability_resume: (P [n,3,3], stats, frequencies solved by this call),
        finished frequencies appended to and read back from the checkpoint at path."""
        om = np.ascontiguousarray(np.atleast_1d(omega), dtype=np.float64)
        n = om.size
        P = np.empty((n, 3, 3), dtype=np.complex128)
        stats = (SolveStats * (3 * n))()
        solved = ctypes.c_int32()
        st = self._lib.tddft_polarizability_resume(self.h, n, om.ctypes.data, float(eps),
                                                   P.ctypes.data, stats, os.fsencode(path),
                                                   ctypes.byref(solved))
        if st != OK and not (st == ERR_NOT_CONVERGED and not raise_on_nonconvergence):
            self._check(st)
        return P, _stats_dict(stats, n), solved.value

    def tuning(self):
        """N-tile widths the autotuner chose for (K z, transform 1, transform 2)."""
        t = (ctypes.c_int32 * 3)()
        self._check(self._lib.tddft_tuning(self.h, t))
        return tuple(t)

    # -- timing ---------------------------------------------------------------
    def timing_enable(self, on: bool = True):
        self._check(self._lib.tddft_timing_enable(self.h, 1 if on else 0))

    def timing(self) -> dict:
        res = {}
        for i in range(self._lib.tddft_timing_count(self.h)):
            name = ctypes.c_char_p()
            n = ctypes.c_int32()
            ms = ctypes.c_double()
            fl = ctypes.c_double()
            by = ctypes.c_double()
            self._check(self._lib.tddft_timing_get(self.h, i, ctypes.byref(name), ctypes.byref(n),
                                                   ctypes.byref(ms), ctypes.byref(fl)))
            self._check(self._lib.tddft_timing_bytes(self.h, i, ctypes.byref(by)))
            res[name.value.decode()] = dict(launches=n.value, ms=ms.value, flops=fl.value,
                                            bytes=by.value)
        return res


class Batch:
    """Several molecules solved together (tddft_batch_*)."""

    def __init__(self, systems, *, restart: int = 40, max_restarts: int = 200, tol: float = 1e-6,
                 batch: int = 64, prec: str = "fp64", inner_tol: float = 1e-4,
                 stop: str = "residual", emu_slices: int = 0):
        lib = load_library()
        self._lib = lib
        marsh = [_marshal(s) for s in systems]
        arr = (_System * len(systems))(*[m[0] for m in marsh])
        o = _Options(PREC[prec], restart, max_restarts, tol, batch, None, inner_tol, 0, STOP[stop],
                     emu_slices, 0, 0, 0)
        h = ctypes.c_void_p()
        st = lib.tddft_batch_create(len(systems), arr, ctypes.byref(o), ctypes.byref(h))
        if st != OK:
            raise TddftError(st, lib.tddft_batch_last_error(None).decode())
        self.h = h
        self.n_mol = len(systems)

    def close(self):
        if getattr(self, "h", None):
            self._lib.tddft_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def polarizability(self, omega, eps, *, raise_on_nonconvergence: bool = True):
        """P [n_mol, n_omega, 3, 3] complex and stats [n_mol, n_omega, 3]."""
        om = np.ascontiguousarray(np.atleast_1d(omega), dtype=np.float64)
        n = om.size
        P = np.empty((self.n_mol, n, 3, 3), dtype=np.complex128)
        stats = (SolveStats * (3 * n * self.n_mol))()
        st = self._lib.tddft_batch_polarizability(self.h, n, om.ctypes.data, float(eps),
                                                  P.ctypes.data, stats)
        if st != OK and not (st == ERR_NOT_CONVERGED and not raise_on_nonconvergence):
            raise TddftError(st, self._lib.tddft_batch_last_error(self.h).decode())
        d = _stats_dict(stats, n * self.n_mol)
        return P, {k: v.reshape(self.n_mol, n, 3) for k, v in d.items()}


def _stats_dict(stats, n):
    return dict(
        matvecs=np.array([s.matvecs for s in stats]).reshape(n, 3),
        cycles=np.array([s.cycles for s in stats]).reshape(n, 3),
        resid=np.array([s.resid for s in stats]).reshape(n, 3),
        converged=np.array([s.converged for s in stats], dtype=bool).reshape(n, 3),
        guess_rejected=np.array([s.flags & 1 for s in stats], dtype=bool).reshape(n, 3),
        eps_p=np.array([s.eps_p for s in stats]).reshape(n, 3),
        eps_x=np.array([s.eps_x for s in stats]).reshape(n, 3))


class Mlp:
    """The guess network (tddft_mlp_*): parameters and training live on the GPU."""

    def __init__(self, n_in=10, width=256, n_out=2, max_rows=1 << 20, seed=0, stream=None):
        lib = load_library()
        self._lib = lib
        h = ctypes.c_void_p()
        st = lib.tddft_mlp_create(n_in, width, n_out, max_rows, seed,
                                  stream if stream is not None else _current_stream(),
                                  ctypes.byref(h))
        if st != OK:
            raise TddftError(st, lib.tddft_mlp_last_error(None).decode())
        self.h = h
        self.n_in, self.width, self.n_out, self.max_rows = n_in, width, n_out, max_rows
        self.n_params = lib.tddft_mlp_num_params(h)

    def close(self):
        if getattr(self, "h", None):
            self._lib.tddft_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise TddftError(st, self._lib.tddft_mlp_last_error(self.h).decode())

    def get_params(self) -> np.ndarray:
        p = np.empty(self.n_params, dtype=np.float32)
        self._check(self._lib.tddft_mlp_params(self.h, p.ctypes.data, self.n_params, 0))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self._lib.tddft_mlp_params(self.h, p.ctypes.data, self.n_params, 1))

    def save(self, path):
        """tddft_mlp_save: the parameters to a file."""
        self._check(self._lib.tddft_mlp_save(self.h, os.fsencode(path)))

    def load(self, path):
        """tddft_mlp_load: parameters of a network of this shape from a file."""
        self._check(self._lib.tddft_mlp_load(self.h, os.fsencode(path)))

    def forward(self, F, bf16: bool = False):
        import torch
        F = F.contiguous()
        Y = torch.empty((F.shape[0], self.n_out), dtype=torch.float32, device=F.device)
        self._check(self._lib.tddft_mlp_forward(self.h, F.shape[0], F.data_ptr(), Y.data_ptr(),
                                                1 if bf16 else 0))
        return Y

    def backward(self, F, dY) -> np.ndarray:
        g = np.empty(self.n_params, dtype=np.float32)
        self._check(self._lib.tddft_mlp_backward(self.h, F.shape[0], F.contiguous().data_ptr(),
                                                 dY.contiguous().data_ptr(), g.ctypes.data))
        return g

    def train_step(self, F, lin, xstar, scale, lr: float):
        import torch
        nt, n_prod = lin.shape
        loss = torch.empty(nt, dtype=torch.float64, device=lin.device)
        self._check(self._lib.tddft_mlp_train_step(
            self.h, nt, n_prod, F.contiguous().data_ptr(),
            torch.view_as_real(lin.contiguous()).data_ptr(),
            torch.view_as_real(xstar.contiguous()).data_ptr(), scale.contiguous().data_ptr(),
            loss.data_ptr(), float(lr)))
        return loss

    def combine(self, Y, lin, scale):
        import torch
        nt, n_prod = lin.shape
        x0 = torch.empty_like(lin)
        st = self._lib.tddft_guess_combine(nt, n_prod, Y.contiguous().data_ptr(),
                                           torch.view_as_real(lin.contiguous()).data_ptr(),
                                           scale.contiguous().data_ptr(),
                                           torch.view_as_real(x0).data_ptr(), _current_stream())
        if st != OK:
            raise TddftError(st, "tddft_guess_combine failed")
        return x0


def kernel_apply_centres(centres, prod_centre, z, softening: float = 1.0, diag: float = 0.05):
    """tddft_kernel_apply_centres: K z for a CUDA tensor z (n_rhs x n_prod complex)
    from the distinct product centres (n_c x 3) and each product's centre index."""
    import torch
    c = np.ascontiguousarray(centres, dtype=np.float64)
    pc = np.ascontiguousarray(prod_centre, dtype=np.int32)
    z = z.to(torch.complex128).contiguous()
    out = torch.empty_like(z)
    lib = load_library()
    st = lib.tddft_kernel_apply_centres(pc.size, c.shape[0], c.ctypes.data, pc.ctypes.data,
                                        float(softening), float(diag), z.shape[0],
                                        torch.view_as_real(z).data_ptr(),
                                        torch.view_as_real(out).data_ptr(), _current_stream())
    if st != OK:
        raise TddftError(st, "tddft_kernel_apply_centres failed")
    return out


def sweep_plan(n_omega: int):
    """tddft_sweep_plan: (pass, left, right) int arrays of an n-point sweep."""
    lib = load_library()
    out = [np.empty(n_omega, dtype=np.int32) for _ in range(3)]
    st = lib.tddft_sweep_plan(n_omega, *(a.ctypes.data for a in out))
    if st != OK:
        raise TddftError(st, "tddft_sweep_plan failed")
    return tuple(out)


def selftest_gemm(M: int, N: int, K: int, seed: int = 1, tf32: bool = False) -> float:
    """Max relative error of the split-bf16 (or TF32) tensor-core GEMM against float64."""
    lib = load_library()
    err = ctypes.c_double()
    fn = lib.tddft_selftest_gemm_tf32 if tf32 else lib.tddft_selftest_gemm
    st = fn(M, N, K, seed, ctypes.byref(err))
    if st != OK:
        raise TddftError(st, "tensor-core GEMM self-test failed")
    return err.value


def gemm_f64_emulated(A, B, slices: int = 6, out=None):
    """C = A @ B for float64 CUDA matrices (row-major, unit column stride),
    emulated on the tensor cores with `slices` integer slices per operand.
    Runs on the current torch stream."""
    import torch
    if A.dtype != torch.float64 or B.dtype != torch.float64 or not (A.is_cuda and B.is_cuda):
        raise ValueError("A and B must be float64 CUDA tensors")
    if A.dim() != 2 or B.dim() != 2 or A.shape[1] != B.shape[0]:
        raise ValueError("shapes do not match")
    if A.stride(1) != 1 or B.stride(1) != 1:
        raise ValueError("rows must be contiguous")
    M, K = A.shape
    N = B.shape[1]
    C = out if out is not None else torch.empty((M, N), dtype=torch.float64, device=A.device)
    if C.stride(1) != 1 or tuple(C.shape) != (M, N):
        raise ValueError("bad output")
    lib = load_library()
    st = lib.tddft_gemm_f64_emulated(M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                     C.data_ptr(), C.stride(0), slices, _current_stream())
    if st != OK:
        raise TddftError(st, "emulated float64 GEMM failed")
    return C


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None
