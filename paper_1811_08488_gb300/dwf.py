"""Thin ctypes binding of libdwf.so (include/dwf.h).

Only argument marshalling happens here: every step of the operator and solver
runs in the CUDA kernels of the library. Field buffers are torch tensors on
the context's device (any dtype; the native layout is described in dwf.h);
the stream is torch's current stream unless given.

The library must have been built (``python -m paper_1811_08488_gb300.build``
or ``__graft_entry__.build()``); importing this module without it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdwf.so")

DWF_FP64, DWF_FP32, DWF_FP16, DWF_BF16 = 0, 1, 2, 3
PREC = {"fp64": DWF_FP64, "fp32": DWF_FP32, "fp16": DWF_FP16, "bf16": DWF_BF16}
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "CUDA", 4: "NOT_CONVERGED",
          5: "TIMEOUT", 6: "NAN", 7: "NO_GAUGE"}
MAX_RHS = 16
MAX_EIG = 64
NOALLOC_SCRATCH_BYTES = 24 << 20

# Every symbol include/dwf.h declares.
EXPORTS = ["dwf_create", "dwf_destroy", "dwf_last_error", "dwf_solver_params_default",
           "dwf_gauge_load", "dwf_field_bytes", "dwf_field_import", "dwf_field_export",
           "dwf_dslash_eo", "dwf_m5", "dwf_m5inv", "dwf_m5inv_gemm", "dwf_mpc", "dwf_mdagm", "dwf_mdagm_noalloc",
           "dwf_block_apply",
           "dwf_block_precond", "dwf_autotune_block", "dwf_source_prep", "dwf_odd_reconstruct",
           "dwf_mpc_sym", "dwf_mdagm_sym", "dwf_source_prep_sym",
           "mspcg_solve", "dwf_profile_enable", "dwf_profile_read",
           "dwf_eig_params_default", "dwf_eig_lowmodes", "dwf_deflate", "mspcg_solve_deflated",
           "dwf_field_convert"]


class DwfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Action(C.Structure):
    _fields_ = [("dims", C.c_int * 4), ("Ls", C.c_int), ("b", C.c_double), ("c", C.c_double),
                ("M5", C.c_double), ("t_antiperiodic", C.c_int), ("recon12", C.c_int)]


class SolverParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxiter", C.c_int), ("inner_iters", C.c_int),
                ("block", C.c_int * 4), ("outer", C.c_int), ("inner", C.c_int),
                ("delta", C.c_double), ("snake", C.c_int), ("use_graph", C.c_int),
                ("io_on_host", C.c_int), ("check_every", C.c_int), ("flexible", C.c_int),
                ("schur", C.c_int), ("inner_tol", C.c_double)]


class EigParams(C.Structure):
    _fields_ = [("n_ev", C.c_int), ("degree", C.c_int), ("max_passes", C.c_int),
                ("tol", C.c_double), ("lambda_max", C.c_double), ("power_steps", C.c_int),
                ("schur", C.c_int)]


class EigInfo(C.Structure):
    _fields_ = [("passes", C.c_int), ("converged", C.c_int), ("matvecs", C.c_longlong),
                ("lambda_max", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveInfo(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("inner_iters_total", C.c_int),
                ("reliable_updates", C.c_int), ("converged", C.c_int),
                ("true_resid", C.c_double), ("seconds", C.c_double),
                ("dslash_gbs", C.c_double), ("host_syncs", C.c_int), ("device_loop", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_longlong), ("seconds", C.c_double),
                ("alg_bytes", C.c_double)]

    def as_dict(self):
        return {"name": self.name.decode(), "launches": self.launches, "seconds": self.seconds,
                "alg_bytes": self.alg_bytes}


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libdwf.so is not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    P, I, D, S = C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_size_t
    sig = {
        "dwf_create": (I, [C.POINTER(P), I, C.POINTER(Action)]),
        "dwf_destroy": (None, [P]),
        "dwf_last_error": (C.c_char_p, [P]),
        "dwf_solver_params_default": (None, [C.POINTER(SolverParams)]),
        "dwf_gauge_load": (I, [P, P, I]),
        "dwf_field_bytes": (S, [P, I, I]),
        "dwf_field_import": (I, [P, P, I, P, I, I, P]),
        "dwf_field_export": (I, [P, P, I, P, I, I, P]),
        "dwf_dslash_eo": (I, [P, P, P, I, I, I, I, D, P]),
        "dwf_m5": (I, [P, P, P, I, I, I, D, P]),
        "dwf_m5inv": (I, [P, P, P, I, I, I, D, P]),
        "dwf_m5inv_gemm": (I, [P, P, P, I, I, I, D, P]),
        "dwf_autotune_block": (I, [P, P, I, D, C.POINTER(SolverParams), I, C.POINTER(C.c_int), D, P]),
        "dwf_mpc": (I, [P, P, P, I, I, I, D, P]),
        "dwf_mdagm": (I, [P, P, P, I, I, D, P]),
        "dwf_mdagm_noalloc": (I, [P, P, P, I, I, D, P]),
        "dwf_source_prep": (I, [P, P, P, P, I, I, D, P]),
        "dwf_source_prep_sym": (I, [P, P, P, P, I, I, D, P]),
        "dwf_mpc_sym": (I, [P, P, P, I, I, I, D, P]),
        "dwf_mdagm_sym": (I, [P, P, P, I, I, D, P]),
        "dwf_odd_reconstruct": (I, [P, P, P, P, I, I, D, P]),
        "dwf_block_apply": (I, [P, P, P, C.POINTER(SolverParams), I, D, P]),
        "dwf_block_precond": (I, [P, P, P, C.POINTER(SolverParams), I, D, P]),
        "mspcg_solve": (I, [P, P, P, I, D, C.POINTER(SolverParams), C.POINTER(SolveInfo), P]),
        "dwf_profile_enable": (I, [P, I]),
        "dwf_eig_params_default": (None, [C.POINTER(EigParams)]),
        "dwf_eig_lowmodes": (I, [P, P, I, C.c_double, C.POINTER(EigParams), D, D,
                                 C.POINTER(EigInfo), P]),
        "dwf_deflate": (I, [P, P, P, P, I, D, I, I, I, I, P]),
        "mspcg_solve_deflated": (I, [P, P, P, I, D, C.POINTER(SolverParams), P, I, D, I, I,
                                     C.POINTER(SolveInfo), P]),
        "dwf_field_convert": (I, [P, P, I, P, I, I, P]),
        "dwf_profile_read": (I, [P, C.POINTER(KernelTime), I, C.POINTER(C.c_int)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def default_params(**kw) -> SolverParams:
    p = SolverParams()
    lib().dwf_solver_params_default(C.byref(p))
    for k, v in kw.items():
        if k == "block":
            for i in range(4):
                p.block[i] = int(v[i])
        elif k in ("outer", "inner") and isinstance(v, str):
            setattr(p, k, PREC[v])
        else:
            setattr(p, k, v)
    return p


def default_eig_params(**kw) -> EigParams:
    p = EigParams()
    lib().dwf_eig_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _ptr(t) -> int:
    return t.data_ptr() if hasattr(t, "data_ptr") else int(t)


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _masses(mf, nrhs=None):
    m = np.atleast_1d(np.asarray(mf, dtype=np.float64))
    if nrhs is not None and m.size == 1 and nrhs > 1:
        m = np.repeat(m, nrhs)
    return m, m.ctypes.data_as(C.POINTER(C.c_double))


class Context:
    """A DWF context: lattice, action, packed links and work buffers."""

    def __init__(self, dims, Ls, b=1.0, c=0.0, M5=1.8, t_antiperiodic=True, device=0,
                 recon12=False):
        self.dims = tuple(int(d) for d in dims)
        self.Ls = int(Ls)
        self.device = device
        a = Action()
        for i in range(4):
            a.dims[i] = self.dims[i]
        a.Ls, a.b, a.c, a.M5, a.t_antiperiodic = self.Ls, b, c, M5, int(bool(t_antiperiodic))
        a.recon12 = int(bool(recon12))
        h = C.c_void_p()
        st = lib().dwf_create(C.byref(h), device, C.byref(a))
        if st != 0:
            raise DwfError(st, lib().dwf_last_error(None).decode())
        self._h = h
        self.Vh = int(np.prod(self.dims)) // 2

    def close(self):
        if getattr(self, "_h", None):
            lib().dwf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise DwfError(st, lib().dwf_last_error(self._h).decode())
        return st

    # ------------------------------------------------------------------ fields
    def field_bytes(self, prec="fp32", nrhs=1) -> int:
        return int(lib().dwf_field_bytes(self._h, PREC.get(prec, prec), nrhs))

    def new_field(self, prec="fp32", nrhs=1, zero=True):
        import torch
        n = self.field_bytes(prec, nrhs)
        f = torch.zeros if zero else torch.empty
        return f(n, dtype=torch.uint8, device=f"cuda:{self.device}")

    def canon_shape(self, nrhs=1):
        Lx, Ly, Lz, Lt = self.dims
        return (nrhs, self.Ls, Lt, Lz, Ly, Lx // 2, 4, 3)

    def gauge_load(self, U):
        """U: complex128 [t][z][y][x][mu][3][3], numpy array or torch tensor."""
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.complex128)
            self._check(lib().dwf_gauge_load(self._h, U.ctypes.data_as(C.c_void_p), 0))
        else:
            on_dev = int(U.is_cuda)
            self._check(lib().dwf_gauge_load(self._h, C.c_void_p(U.data_ptr()), on_dev))

    def field_import(self, native, prec, canon, nrhs=1, stream=None):
        fp32 = int(str(canon.dtype).endswith("complex64"))
        self._check(lib().dwf_field_import(self._h, C.c_void_p(_ptr(native)), PREC.get(prec, prec),
                                           C.c_void_p(_ptr(canon)), fp32, nrhs, _stream(stream)))

    def field_export(self, canon, native, prec, nrhs=1, stream=None):
        fp32 = int(str(canon.dtype).endswith("complex64"))
        self._check(lib().dwf_field_export(self._h, C.c_void_p(_ptr(canon)), fp32,
                                           C.c_void_p(_ptr(native)), PREC.get(prec, prec), nrhs,
                                           _stream(stream)))

    # --------------------------------------------------------------- operators
    def dslash_eo(self, out, inp, out_parity, dagger, prec, mf, stream=None):
        m, mp = _masses(mf)
        self._check(lib().dwf_dslash_eo(self._h, C.c_void_p(_ptr(out)), C.c_void_p(_ptr(inp)),
                                        out_parity, int(dagger), PREC.get(prec, prec), m.size, mp,
                                        _stream(stream)))

    def m5(self, out, inp, dagger, prec, mf, stream=None):
        m, mp = _masses(mf)
        self._check(lib().dwf_m5(self._h, C.c_void_p(_ptr(out)), C.c_void_p(_ptr(inp)), int(dagger),
                                 PREC.get(prec, prec), m.size, mp, _stream(stream)))

    def m5inv(self, out, inp, dagger, prec, mf, stream=None):
        m, mp = _masses(mf)
        self._check(lib().dwf_m5inv(self._h, C.c_void_p(_ptr(out)), C.c_void_p(_ptr(inp)),
                                    int(dagger), PREC.get(prec, prec), m.size, mp, _stream(stream)))

    def m5inv_gemm(self, out, inp, dagger, prec, mf, stream=None):
        """dwf_m5inv_gemm: M_5^-1 (dagger: its adjoint) on the tensor cores,
        all right-hand sides of `mf` in one launch."""
        m, mp = _masses(mf)
        self._check(lib().dwf_m5inv_gemm(self._h, C.c_void_p(_ptr(out)), C.c_void_p(_ptr(inp)),
                                         int(dagger), PREC.get(prec, prec), m.size, mp,
                                         _stream(stream)))

    def mpc(self, out, inp, dagger, prec, mf, stream=None):
        m, mp = _masses(mf)
        self._check(lib().dwf_mpc(self._h, C.c_void_p(_ptr(out)), C.c_void_p(_ptr(inp)), int(dagger),
                                  PREC.get(prec, prec), m.size, mp, _stream(stream)))

    def mpc_sym(self, out, inp, dagger, prec, mf, stream=None):
        """dwf_mpc_sym: D_sym = 1 - M_5^-1 M^4_eo M_5^-1 M^4_oe (or its adjoint)."""
        m, mp = _masses(mf)
        self._check(lib().dwf_mpc_sym(self._h, C.c_void_p(_ptr(out)), C.c_void_p(_ptr(inp)),
                                      int(dagger), PREC.get(prec, prec), m.size, mp,
                                      _stream(stream)))

    def mdagm_sym(self, out, inp, prec, mf, stream=None):
        """dwf_mdagm_sym: D_sym^+ D_sym."""
        m, mp = _masses(mf)
        self._check(lib().dwf_mdagm_sym(self._h, C.c_void_p(_ptr(out)), C.c_void_p(_ptr(inp)),
                                        PREC.get(prec, prec), m.size, mp, _stream(stream)))

    def mdagm(self, out, inp, prec, mf, stream=None):
        m, mp = _masses(mf)
        self._check(lib().dwf_mdagm(self._h, C.c_void_p(_ptr(out)), C.c_void_p(_ptr(inp)),
                                    PREC.get(prec, prec), m.size, mp, _stream(stream)))

    def mdagm_noalloc(self, out, inp, prec, mf, stream=None):
        """D_PC^+ D_PC without device allocation (temporaries in the library's
        fixed scratch array of NOALLOC_SCRATCH_BYTES)."""
        m, mp = _masses(mf)
        self._check(lib().dwf_mdagm_noalloc(self._h, C.c_void_p(_ptr(out)), C.c_void_p(_ptr(inp)),
                                            PREC.get(prec, prec), m.size, mp, _stream(stream)))

    def block_apply(self, out, inp, params, mf, stream=None):
        m, mp = _masses(mf)
        self._check(lib().dwf_block_apply(self._h, C.c_void_p(_ptr(out)), C.c_void_p(_ptr(inp)),
                                          C.byref(params), m.size, mp, _stream(stream)))

    def block_precond(self, z, r, params, mf, stream=None):
        m, mp = _masses(mf)
        self._check(lib().dwf_block_precond(self._h, C.c_void_p(_ptr(z)), C.c_void_p(_ptr(r)),
                                            C.byref(params), m.size, mp, _stream(stream)))

    # ------------------------------------------------------------------- solve
    def source_prep(self, b_even, phi_even, phi_odd, prec, mf, stream=None):
        """dwf_source_prep: b = D_PC^+ (phi_e - M^4_eo M_5^-1 phi_o), native fields."""
        m, mp = _masses(mf)
        self._check(lib().dwf_source_prep(self._h, C.c_void_p(_ptr(b_even)),
                                          C.c_void_p(_ptr(phi_even)), C.c_void_p(_ptr(phi_odd)),
                                          PREC.get(prec, prec), m.size, mp, _stream(stream)))

    def source_prep_sym(self, b_even, phi_even, phi_odd, prec, mf, stream=None):
        """dwf_source_prep_sym: b = D_sym^+ M_5^-1 (phi_e - M^4_eo M_5^-1 phi_o)."""
        m, mp = _masses(mf)
        self._check(lib().dwf_source_prep_sym(self._h, C.c_void_p(_ptr(b_even)),
                                              C.c_void_p(_ptr(phi_even)),
                                              C.c_void_p(_ptr(phi_odd)), PREC.get(prec, prec),
                                              m.size, mp, _stream(stream)))

    def odd_reconstruct(self, psi_odd, psi_even, phi_odd, prec, mf, stream=None):
        """dwf_odd_reconstruct: psi_o = M_5^-1 (phi_o - M^4_oe psi_e), native fields."""
        m, mp = _masses(mf)
        self._check(lib().dwf_odd_reconstruct(self._h, C.c_void_p(_ptr(psi_odd)),
                                              C.c_void_p(_ptr(psi_even)),
                                              C.c_void_p(_ptr(phi_odd)), PREC.get(prec, prec),
                                              m.size, mp, _stream(stream)))

    def solve_full(self, phi_even, phi_odd, mf, params, stream=None):
        """Solve D psi = phi: source preparation, mspcg_solve on the normal
        equation, odd reconstruction. phi_even / phi_odd: canonical complex128
        device tensors [nrhs][...]; returns (psi_even, psi_odd, status, infos)
        in the same layout. params.schur selects the normal equation (and its
        right-hand side). Every step runs in the library's kernels."""
        import torch
        m, _ = _masses(mf)
        nrhs = m.size
        nat = {k: self.new_field("fp64", nrhs) for k in ("pe", "po", "b", "xe", "xo")}
        self.field_import(nat["pe"], "fp64", phi_even, nrhs)
        self.field_import(nat["po"], "fp64", phi_odd, nrhs)
        prep = self.source_prep_sym if params.schur else self.source_prep
        prep(nat["b"], nat["pe"], nat["po"], "fp64", list(m), stream)
        b = torch.zeros_like(phi_even)
        self.field_export(b, nat["b"], "fp64", nrhs)
        psi_e = torch.zeros_like(phi_even)
        st, info = self.solve(psi_e, b, list(m), params, stream)
        self.field_import(nat["xe"], "fp64", psi_e, nrhs)
        self.odd_reconstruct(nat["xo"], nat["xe"], nat["po"], "fp64", list(m), stream)
        psi_o = torch.zeros_like(phi_odd)
        self.field_export(psi_o, nat["xo"], "fp64", nrhs)
        return psi_e, psi_o, st, info

    def profile(self, on=True):
        """dwf_profile_enable: turn the hop-kernel timer on (resetting it) or off."""
        self._check(lib().dwf_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """dwf_profile_read: [{name, launches, seconds, alg_bytes}] per timed kernel."""
        n = C.c_int(0)
        self._check(lib().dwf_profile_read(self._h, None, 0, C.byref(n)))
        out = (KernelTime * max(1, n.value))()
        self._check(lib().dwf_profile_read(self._h, out, n.value, C.byref(n)))
        return [out[i].as_dict() for i in range(n.value)]

    def autotune_block(self, b, mf, params, trial=20, stream=None):
        """dwf_autotune_block: returns (block shape, predicted seconds)."""
        m, mp = _masses(mf)
        blk = (C.c_int * 4)()
        pred = C.c_double(0.0)
        bp = b.ctypes.data if isinstance(b, np.ndarray) else _ptr(b)
        self._check(lib().dwf_autotune_block(self._h, C.c_void_p(bp), m.size, mp, C.byref(params),
                                             int(trial), blk, C.byref(pred), _stream(stream)))
        return tuple(blk), pred.value

    def solve(self, x, b, mf, params, stream=None, raise_on_error=True):
        """mspcg_solve. x, b: canonical complex128 even fields (device tensors,
        or host numpy/pinned tensors with params.io_on_host = 1).
        Returns (status, [info dict per rhs])."""
        m, mp = _masses(mf)
        infos = (SolveInfo * m.size)()
        xp = x.ctypes.data if isinstance(x, np.ndarray) else _ptr(x)
        bp = b.ctypes.data if isinstance(b, np.ndarray) else _ptr(b)
        st = lib().mspcg_solve(self._h, C.c_void_p(xp), C.c_void_p(bp), m.size, mp,
                               C.byref(params), infos, _stream(stream))
        if st != 0 and raise_on_error and st != 4:
            raise DwfError(st, lib().dwf_last_error(self._h).decode())
        return st, [i.as_dict() for i in infos]

    # ------------------------------------------------------ low modes, deflation
    def eig_lowmodes(self, V, m, mf, params, stream=None):
        """dwf_eig_lowmodes: V holds m native FP32 fields (start vectors in,
        Ritz vectors out, ascending). Returns (theta, resid, info dict)."""
        theta = np.zeros(m)
        resid = np.zeros(m)
        info = EigInfo()
        self._check(lib().dwf_eig_lowmodes(self._h, C.c_void_p(_ptr(V)), int(m), float(mf),
                                           C.byref(params),
                                           theta.ctypes.data_as(C.POINTER(C.c_double)),
                                           resid.ctypes.data_as(C.POINTER(C.c_double)),
                                           C.byref(info), _stream(stream)))
        return theta, resid, info.as_dict()

    def field_convert(self, out, out_prec, inp, in_prec, nrhs=1, stream=None):
        """dwf_field_convert: native fields from in_prec to out_prec."""
        self._check(lib().dwf_field_convert(self._h, C.c_void_p(_ptr(out)),
                                            PREC.get(out_prec, out_prec), C.c_void_p(_ptr(inp)),
                                            PREC.get(in_prec, in_prec), int(nrhs),
                                            _stream(stream)))

    def deflate(self, z, r, V, lam, prec, nrhs=1, accumulate=False, vprec="fp32", stream=None):
        """dwf_deflate: z = (z if accumulate) + V Lambda^-1 V^+ r."""
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        self._check(lib().dwf_deflate(self._h, C.c_void_p(_ptr(z)), C.c_void_p(_ptr(r)),
                                      C.c_void_p(_ptr(V)), PREC.get(vprec, vprec),
                                      lam.ctypes.data_as(C.POINTER(C.c_double)), lam.size,
                                      PREC.get(prec, prec), int(nrhs), int(bool(accumulate)),
                                      _stream(stream)))

    def solve_deflated(self, x, b, mf, params, V, lam, coarse=True, vprec="fp32", stream=None,
                       raise_on_error=True):
        """mspcg_solve_deflated with the Ritz pairs (V, lam). Returns (status,
        [info dict per rhs])."""
        m, mp = _masses(mf)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        infos = (SolveInfo * m.size)()
        xp = x.ctypes.data if isinstance(x, np.ndarray) else _ptr(x)
        bp = b.ctypes.data if isinstance(b, np.ndarray) else _ptr(b)
        st = lib().mspcg_solve_deflated(self._h, C.c_void_p(xp), C.c_void_p(bp), m.size, mp,
                                        C.byref(params), C.c_void_p(_ptr(V)),
                                        PREC.get(vprec, vprec),
                                        lam.ctypes.data_as(C.POINTER(C.c_double)), lam.size,
                                        int(bool(coarse)), infos, _stream(stream))
        if st != 0 and raise_on_error and st != 4:
            raise DwfError(st, lib().dwf_last_error(self._h).decode())
        return st, [i.as_dict() for i in infos]
