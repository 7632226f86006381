"""Python binding of the JFNK CUDA library (argument marshalling only).

Every function here forwards to the C ABI declared in include/jfnk.h with the
same name; the numerical work runs in the library's CUDA kernels.  PyTorch
supplies device memory (the workspace and the vectors) and the stream.  The
library must have been built (`paper_1512_03662_gb300.build.build()`); there
is no CPU fallback: a missing library raises at import of the first call.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libjfnk.so")

JFNK_OK = 0
JFNK_EINVAL = -1
JFNK_ECUDA = -2
JFNK_ENOMEM = -3
JFNK_ENONFINITE = -4
JFNK_ENOCONV_GMRES = 1
JFNK_ENOCONV_NEWTON = 2

BC_PERIODIC, BC_WALL = 0, 1
ENERGY_INTERNAL, ENERGY_TOTAL = 0, 1
PRECOND_NONE, PRECOND_SOUND, PRECOND_SOUND_DIFF = 0, 1, 2
PERT_OLD, PERT_NEW = 0, 1
FP64, MIXED = 0, 1
MAX_NEWTON = 64


class jfnk_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("bc", ctypes.c_int * 3)]


class jfnk_eos(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("energy_form", ctypes.c_int)]


class jfnk_gravity(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double * 3)]


class jfnk_conductivity(ctypes.Structure):
    _fields_ = [("K0", ctypes.c_double), ("exponent", ctypes.c_double)]


class jfnk_options(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("theta", "lambda_", "alpha1", "alpha2", "eta", "newton_tol")] + \
               [(n, ctypes.c_int) for n in ("pert", "gmres_m", "gmres_max_it", "newton_min", "newton_max",
                                             "precond", "mg_cycles", "mg_nu1", "mg_nu2", "precision", "reorth",
                                             "fixed_iterations", "pc_freeze")] + \
               [("inner_tol", ctypes.c_double), ("inner_max_cycles", ctypes.c_int), ("inner_monitor", ctypes.c_int)]


class jfnk_stats(ctypes.Structure):
    _fields_ = [("newton_iterations", ctypes.c_int), ("gmres_iterations_total", ctypes.c_int),
                ("gmres_iterations", ctypes.c_int * MAX_NEWTON), ("dx_inf", ctypes.c_double * MAX_NEWTON),
                ("fhat_norm", ctypes.c_double * MAX_NEWTON), ("gmres_res", ctypes.c_double * MAX_NEWTON),
                ("gmres_converged", ctypes.c_int * MAX_NEWTON), ("converged", ctypes.c_int),
                ("jv_evaluations", ctypes.c_int), ("precond_applies", ctypes.c_int), ("jv_ms", ctypes.c_double),
                ("precond_ms", ctypes.c_double), ("ortho_ms", ctypes.c_double), ("step_ms", ctypes.c_double),
                ("jv_kernel_ms", ctypes.c_double * 5), ("kernel_launches", ctypes.c_longlong),
                ("inner_res_mean", ctypes.c_double), ("inner_res_max", ctypes.c_double),
                ("inner_cycles", ctypes.c_longlong), ("reorth_passes", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        k = self.newton_iterations
        return {"newton_iterations": k, "gmres_iterations_total": self.gmres_iterations_total,
                "gmres_iterations": list(self.gmres_iterations[:k]), "dx_inf": list(self.dx_inf[:k]),
                "fhat_norm": list(self.fhat_norm[:k]), "gmres_res": list(self.gmres_res[:k]),
                "gmres_converged": list(self.gmres_converged[:k]), "converged": bool(self.converged),
                "jv_evaluations": self.jv_evaluations, "precond_applies": self.precond_applies,
                "jv_ms": self.jv_ms, "precond_ms": self.precond_ms, "ortho_ms": self.ortho_ms,
                "step_ms": self.step_ms, "jv_kernel_ms": list(self.jv_kernel_ms),
                "kernel_launches": self.kernel_launches, "inner_res_mean": self.inner_res_mean,
                "inner_res_max": self.inner_res_max, "inner_cycles": self.inner_cycles,
                "reorth_passes": self.reorth_passes}


_lib = None


def lib():
    """The loaded libjfnk.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"JFNK CUDA library not built: {LIB_PATH} is missing "
                               "(run paper_1512_03662_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, D, I, S = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_size_t
        DP = ctypes.POINTER(ctypes.c_double)
        sig = {
            "jfnk_default_options": (None, [ctypes.POINTER(jfnk_options)]),
            "jfnk_create": (I, [ctypes.POINTER(jfnk_grid), ctypes.POINTER(jfnk_eos), ctypes.POINTER(jfnk_gravity),
                                ctypes.POINTER(jfnk_conductivity), ctypes.POINTER(jfnk_options),
                                ctypes.POINTER(P)]),
            "jfnk_workspace_bytes": (S, [P]),
            "jfnk_bind": (I, [P, P, S, P]),
            "jfnk_vector_length": (ctypes.c_longlong, [P]),
            "jfnk_set_options": (I, [P, ctypes.POINTER(jfnk_options)]),
            "jfnk_residual": (I, [P, P, P, D, P]),
            "jfnk_scaling": (I, [P, P, P, P, DP]),
            "jfnk_jv": (I, [P, P, D, P, P, DP]),
            "jfnk_precond_apply": (I, [P, P, D, P, P]),
            "jfnk_linear_solve": (I, [P, P, P, D, P, ctypes.POINTER(jfnk_stats)]),
            "jfnk_step": (I, [P, P, D, D, D, ctypes.POINTER(jfnk_stats)]),
            "jfnk_dt_from_cfl": (I, [P, P, D, DP]),
            "jfnk_set_profiling": (I, [P, I]),
            "jfnk_residual_noalloc": (I, [P, P, P, D, P]),
            "jfnk_vjp_residual": (I, [P, P, D, P, P]),
            "jfnk_si_step": (I, [P, P, D]),
            "jfnk_vjp": (I, [P, P, P, D, P, P, DP, ctypes.POINTER(jfnk_stats)]),
            "jfnk_last_error": (ctypes.c_char_p, [P]),
            "jfnk_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


EXPORTED = ["jfnk_default_options", "jfnk_create", "jfnk_workspace_bytes", "jfnk_bind", "jfnk_vector_length",
            "jfnk_set_options", "jfnk_residual", "jfnk_scaling", "jfnk_jv", "jfnk_precond_apply",
            "jfnk_linear_solve", "jfnk_step", "jfnk_dt_from_cfl", "jfnk_set_profiling", "jfnk_last_error",
            "jfnk_destroy", "jfnk_residual_noalloc", "jfnk_vjp_residual", "jfnk_vjp", "jfnk_si_step"]


class JFNKError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def default_options(**kw) -> jfnk_options:
    """jfnk_default_options with the given fields replaced (lam for lambda);
    an unknown field name raises instead of being ignored."""
    o = jfnk_options()
    lib().jfnk_default_options(ctypes.byref(o))
    names = {f[0] for f in jfnk_options._fields_}
    for k, v in kw.items():
        k = "lambda_" if k == "lam" else k
        if k not in names:
            raise TypeError(f"unknown jfnk option {k!r}")
        setattr(o, k, v)
    return o


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _resolve_device(device) -> torch.device:
    d = torch.device(device)
    if d.type == "cuda" and d.index is None:
        d = torch.device("cuda", torch.cuda.current_device())
    return d


class Solver:
    """One handle of the C library plus its torch-allocated workspace.

    The methods mirror the C entry points (jfnk_residual -> residual, ...)
    and take CUDA tensors laid out as described in include/jfnk.h."""

    def __init__(self, ndim: int, n: Sequence[int], lo: Sequence[float], hi: Sequence[float],
                 bc: Sequence[int], gamma: float, energy_form: int = 0, g: Sequence[float] = (0, 0, 0),
                 K0: float = 0.0, chi_exp: float = 3.0, options: Optional[jfnk_options] = None,
                 device: str = "cuda", stream: Optional[torch.cuda.Stream] = None):
        L = lib()
        gr = jfnk_grid(ndim, (ctypes.c_int * 3)(*n), (ctypes.c_double * 3)(*lo), (ctypes.c_double * 3)(*hi),
                       (ctypes.c_int * 3)(*bc))
        eo = jfnk_eos(gamma, energy_form)
        gv = jfnk_gravity((ctypes.c_double * 3)(*g))
        co = jfnk_conductivity(K0, chi_exp)
        self.options = options if options is not None else default_options()
        self.h = ctypes.c_void_p()
        st = L.jfnk_create(ctypes.byref(gr), ctypes.byref(eo), ctypes.byref(gv), ctypes.byref(co),
                           ctypes.byref(self.options), ctypes.byref(self.h))
        if st != JFNK_OK:
            msg = L.jfnk_last_error(self.h).decode() if self.h else "create failed"
            if self.h:
                L.jfnk_destroy(self.h)
                self.h = None
            raise JFNKError(st, msg)
        self.device = _resolve_device(device)
        self.nvec = int(L.jfnk_vector_length(self.h))
        self.vdtype = torch.float32 if self.options.precision == MIXED else torch.float64
        nbytes = int(L.jfnk_workspace_bytes(self.h))
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        off = (-base) % 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):      # the handle records the device current at jfnk_bind
            self._check(L.jfnk_bind(self.h, ctypes.c_void_p(base + off), nbytes,
                                    ctypes.c_void_p(self.stream.cuda_stream)))

    @staticmethod
    def from_workload(wl, options: Optional[jfnk_options] = None, **kw) -> "Solver":
        if options is None:
            options = default_options(theta=wl.theta, precond=wl.precond)
        return Solver(wl.ndim, wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.energy_form, wl.g, wl.K0, wl.chi_exp,
                      options, **kw)

    def _check(self, st: int, allow_positive: bool = False) -> int:
        if st < 0 or (st > 0 and not allow_positive):
            raise JFNKError(st, lib().jfnk_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            lib().jfnk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, dtype=torch.float64) -> torch.Tensor:
        return torch.empty(self.nvec, dtype=dtype, device=self.device)

    def _arg(self, t, name: str, dtype=torch.float64):
        """Device pointer of a vector argument, after checking that the C ABI
        can take it: a contiguous tensor on the handle's device with the
        expected dtype and the packed vector length.  A wrong tensor raises
        ValueError (TypeError for a non-tensor) before any library call."""
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor, not {type(t).__name__}")
        if t.device != self.device:
            raise ValueError(f"{name} is on {t.device}, the solver on {self.device}")
        if t.dtype != dtype:
            raise ValueError(f"{name} has dtype {t.dtype}, expected {dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() != self.nvec:
            raise ValueError(f"{name} has {t.numel()} elements, the packed vector has {self.nvec}")
        return ctypes.c_void_p(t.data_ptr())

    def set_options(self, options: jfnk_options):
        self._check(lib().jfnk_set_options(self.h, ctypes.byref(options)))
        self.options = options

    def set_profiling(self, on: bool):
        self._check(lib().jfnk_set_profiling(self.h, int(on)))

    def residual(self, X: torch.Tensor, Xn: torch.Tensor, dt: float, out: Optional[torch.Tensor] = None):
        px, pn = self._arg(X, "X"), self._arg(Xn, "Xn")
        F = self._vec() if out is None else out
        self._check(lib().jfnk_residual(self.h, px, pn, dt, self._arg(F, "out")))
        return F

    def residual_noalloc(self, X: torch.Tensor, Xn: torch.Tensor, dt: float, out: Optional[torch.Tensor] = None):
        """jfnk_residual_noalloc: the residual with the library's fixed scratch
        (no workspace use, nothing allocated by the call)."""
        px, pn = self._arg(X, "X"), self._arg(Xn, "Xn")
        F = self._vec() if out is None else out
        with torch.cuda.device(self.device):
            self._check(lib().jfnk_residual_noalloc(self.h, px, pn, dt, self._arg(F, "out")))
        return F

    def scaling(self, X: torch.Tensor):
        px = self._arg(X, "X")
        L, R = self._vec(), self._vec()
        xn = ctypes.c_double()
        self._check(lib().jfnk_scaling(self.h, px, _ptr(L), _ptr(R), ctypes.byref(xn)))
        return L, R, xn.value

    def jv(self, X: torch.Tensor, dt: float, v: torch.Tensor, out: Optional[torch.Tensor] = None):
        px, pv = self._arg(X, "X"), self._arg(v, "v", self.vdtype)
        Jv = self._vec(self.vdtype) if out is None else out
        d = ctypes.c_double()
        self._check(lib().jfnk_jv(self.h, px, dt, pv, self._arg(Jv, "out", self.vdtype), ctypes.byref(d)))
        return Jv, d.value

    def precond_apply(self, X: torch.Tensor, dt: float, v: torch.Tensor, out: Optional[torch.Tensor] = None):
        px, pv = self._arg(X, "X"), self._arg(v, "v", self.vdtype)
        w = self._vec(self.vdtype) if out is None else out
        self._check(lib().jfnk_precond_apply(self.h, px, dt, pv, self._arg(w, "out", self.vdtype)))
        return w

    def linear_solve(self, X: torch.Tensor, Xn: torch.Tensor, dt: float):
        px, pn = self._arg(X, "X"), self._arg(Xn, "Xn")
        dx = self._vec()
        st = jfnk_stats()
        code = self._check(lib().jfnk_linear_solve(self.h, px, pn, dt, _ptr(dx), ctypes.byref(st)),
                           allow_positive=True)
        return dx, st.as_dict(), code

    def step(self, X: torch.Tensor, dt: float, newton_tol: float = 0.0, krylov_tol: float = 0.0):
        px = self._arg(X, "X")
        st = jfnk_stats()
        code = self._check(lib().jfnk_step(self.h, px, dt, newton_tol, krylov_tol, ctypes.byref(st)),
                           allow_positive=True)
        d = st.as_dict()
        d["status"] = code
        return d

    def si_step(self, X: torch.Tensor, dt: float) -> None:
        """jfnk_si_step: one step of the semi-implicit scheme as a time
        integrator, in place in X."""
        self._check(lib().jfnk_si_step(self.h, self._arg(X, "X"), dt))

    def vjp_residual(self, X: torch.Tensor, dt: float, w: torch.Tensor) -> torch.Tensor:
        """jfnk_vjp_residual: (dG/dX)^T w at X."""
        px, pw = self._arg(X, "X"), self._arg(w, "w")
        y = self._vec()
        self._check(lib().jfnk_vjp_residual(self.h, px, dt, pw, _ptr(y)))
        return y

    def vjp(self, Xn: torch.Tensor, Xnp1: torch.Tensor, dt: float, gbar: torch.Tensor):
        """jfnk_vjp: gradients through one implicit step; returns
        (dL/dXn, dL/dK0, stats, status)."""
        pn, pn1, pg = self._arg(Xn, "Xn"), self._arg(Xnp1, "Xnp1"), self._arg(gbar, "gbar")
        gXn = self._vec()
        gK0 = ctypes.c_double()
        st = jfnk_stats()
        code = self._check(lib().jfnk_vjp(self.h, pn, pn1, dt, pg, _ptr(gXn),
                                          ctypes.byref(gK0), ctypes.byref(st)), allow_positive=True)
        return gXn, gK0.value, st.as_dict(), code

    def dt_from_cfl(self, X: torch.Tensor, cfl: float) -> float:
        px = self._arg(X, "X")
        dt = ctypes.c_double()
        self._check(lib().jfnk_dt_from_cfl(self.h, px, cfl, ctypes.byref(dt)))
        return dt.value


class JFNKStep(torch.autograd.Function):
    """One implicit step X^n -> X^{n+1} as a differentiable operation.

    forward runs jfnk_step on a copy of X^n; backward solves the transposed
    Newton system with jfnk_vjp (no unrolling of the Newton iterations) and
    returns the gradients with respect to X^n and to the conductivity
    prefactor K0 (passed as a 0-dim tensor equal to the solver's K0; the
    solver's K0 is what the step uses).  One checkpoint (X^n and X^{n+1}) is
    kept per step.  dt is held fixed."""

    @staticmethod
    def forward(ctx, Xn, K0, solver, dt, newton_tol=0.0, krylov_tol=0.0):
        X = Xn.detach().clone()
        st = solver.step(X, dt, newton_tol, krylov_tol)
        if st["status"] != JFNK_OK:
            raise JFNKError(st["status"], "implicit step did not converge")
        ctx.solver, ctx.dt = solver, dt
        ctx.save_for_backward(Xn.detach(), X)
        return X

    @staticmethod
    def backward(ctx, gbar):
        Xn, Xnp1 = ctx.saved_tensors
        gXn, gK0, st, code = ctx.solver.vjp(Xn, Xnp1, ctx.dt, gbar.contiguous().double())
        if code != JFNK_OK:
            raise JFNKError(code, "transposed solve did not converge")
        return gXn, torch.tensor(gK0, dtype=torch.float64, device=gbar.device), None, None, None, None
