"""Newton-Krylov layer (paper Sects. 4.1-4.3).  TEST INFRASTRUCTURE: see the
package docstring for who may import this.

* Scaling (Eq. jacobian_system_norm): the Newton system is solved as
  (L^-1 J R)(R^-1 dX) = -L^-1 F with diagonal
      L_rho = rho, L_e = rho e, L_u = rho_f max(|u_f|, alpha1 c_s,f),
      R_rho = rho, R_e = e,     R_u = max(|u_f|, alpha2 c_s,f),
  c_s,f and rho_f the means of the two cells beside face f.  For the total
  energy form L_E = rho eps_t, R_E = eps_t (the same rule applied to the
  energy unknown).  Wall-face slots get L = R = 1 (their entries are zero).
* Jacobian-vector product (Eqs. jacobian_free, pert_old): in scaled space
      J^ w^ = L^-1 [G(X + delta R w^) - G(X)] / delta,
      delta = lambda (lambda + ||x^||_2 / ||w^||_2),   x^ = R^-1 X,
  with G = U/dt - theta R_U (the X^n part of F cancels in the difference).
  Eq. pert_new is the alternative, with sign(0) read as +1.
* GMRES (Eq. forcing_term, Sect. 4.3 right preconditioning): start from 0,
  stop when the least-squares residual estimate is below eta ||F^||_2,
  restart length m, at most max_it iterations in total.  Classical
  Gram-Schmidt; reorth = 1 always adds a second pass, reorth = 2 adds it
  only when the first pass shrank the vector below 1/sqrt(2) of its norm
  (the selective criterion of Daniel, Gragg, Kaufman and Stewart, Math. Comp.
  30 (1976) 772-795).  Givens rotations on the Hessenberg matrix.  The preconditioned directions z_j = M^-1 v_j are kept so that the
  correction is sum_j y_j z_j; for a fixed linear M this equals the paper's
  M^-1 (V y).
* Newton (Eq. jacobian_system, nr_terminate): X^(0) = X^n, stop when
  ||R^-1 dX||_inf < eps, with at least two iterations.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import torch

from . import discretization as D

PERT_OLD = 0
PERT_NEW = 1


@dataclasses.dataclass
class Options:
    lam: float = 1e-7              # lambda of Eq. pert_old (Sect. 5.1.1 uses 1e-7)
    alpha1: float = 1e-5
    alpha2: float = 1.0
    pert: int = PERT_OLD
    gmres_m: int = 30
    gmres_max_it: int = 300
    eta: float = 1e-4
    newton_tol: float = 1e-8
    newton_min: int = 2
    newton_max: int = 20
    precond: int = 1               # 0 none, 1 sound, 2 sound + diffusion
    mg_cycles: int = 2              # V(mg_nu1, mg_nu2) cycles per preconditioner apply
    mg_nu1: int = 2
    mg_nu2: int = 2
    reorth: int = 0                # 1: always a second Gram-Schmidt pass, 2: selective (DGKS)
    fixed_iterations: bool = False # run exactly gmres_max_it / newton_max iterations
    exact_inner: bool = False      # solve the SI system with a sparse direct solver
    pc_freeze: bool = False        # SI coefficients from X^n (Sects. 3.3-3.4 write them at level n)


# ----------------------------------------------------------------------------
# scaling
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Scaling:
    L: torch.Tensor
    R: torch.Tensor
    xhat_norm: float


def scaling(P: D.Problem, X, opts: Options) -> Scaling:
    f = D.unpack(P, X)
    rho, E = f[0], f[1]
    e = D.internal_energy(P, X)
    cs = D.sound_speed(P, e)
    rp, csp = D.pad(P, rho), D.pad(P, cs)
    Ls, Rs = [rho, rho * E], [rho, E]
    for c in range(P.ndim):
        rho_f = D.crop(P, 0.5 * (D.sh(rp, c, -1) + rp))
        cs_f = D.crop(P, 0.5 * (D.sh(csp, c, -1) + csp))
        au = torch.abs(f[2 + c])
        Lu = rho_f * torch.maximum(au, opts.alpha1 * cs_f)
        Ru = torch.maximum(au, opts.alpha2 * cs_f)
        m = D.wall_slot_mask(P, c)
        Ls.append(Lu * m + (1.0 - m))
        Rs.append(Ru * m + (1.0 - m))
    L, R = D.pack(Ls), D.pack(Rs)
    xhat = D.as_tensor(X) / R
    return Scaling(L=L, R=R, xhat_norm=float(torch.linalg.vector_norm(xhat)))


def perturbation(opts: Options, sc: Scaling, X, w: torch.Tensor) -> float:
    wn = float(torch.linalg.vector_norm(w))
    if opts.pert == PERT_OLD:
        return opts.lam * (opts.lam + sc.xhat_norm / wn)
    xhat = D.as_tensor(X) / sc.R
    uv = float(torch.dot(xhat, w))
    sgn = 1.0 if uv >= 0 else -1.0
    return opts.lam * (1e-12 / opts.lam + abs(uv) / (wn * wn)) * sgn


def jv(P: D.Problem, X, G0: torch.Tensor, sc: Scaling, w: torch.Tensor, dt: float,
       opts: Options, delta: Optional[float] = None):
    """Scaled finite-difference J^ w^ (Eq. jacobian_free); returns (Jw, delta)."""
    X = D.as_tensor(X)
    if delta is None:
        delta = perturbation(opts, sc, X, w)
    Xp = X + delta * (sc.R * w)
    G1 = D.G_operator(P, Xp, dt)
    return (G1 - G0) / delta / sc.L, delta


# ----------------------------------------------------------------------------
# GMRES
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class GmresStats:
    iterations: int = 0
    restarts: int = 0
    converged: bool = False
    res_history: List[float] = dataclasses.field(default_factory=list)
    beta0: float = 0.0
    reorth_passes: int = 0


DGKS_KAPPA = 1.0 / math.sqrt(2.0)   # second pass when ||w after|| < kappa ||w before||


def gmres(apply_A: Callable[[torch.Tensor], torch.Tensor],
          apply_Minv: Callable[[torch.Tensor], torch.Tensor],
          b: torch.Tensor, eta: float, m: int, max_it: int, reorth: int = 0,
          fixed: bool = False):
    """Right-preconditioned restarted GMRES for A x = b from x = 0."""
    st = GmresStats()
    x = torch.zeros_like(b)
    beta0 = float(torch.linalg.vector_norm(b))
    st.beta0 = beta0
    if beta0 == 0.0:
        st.converged = True
        return x, st
    r = b.clone()
    total = 0
    while True:
        beta = float(torch.linalg.vector_norm(r))
        V = [r / beta]
        Z = []
        H = torch.zeros(m + 1, m, dtype=torch.float64)
        cs = torch.zeros(m, dtype=torch.float64)
        sn = torch.zeros(m, dtype=torch.float64)
        gvec = torch.zeros(m + 1, dtype=torch.float64)
        gvec[0] = beta
        k = 0
        done = False
        for j in range(m):
            if total >= max_it:
                break
            z = apply_Minv(V[j])
            Z.append(z)
            w = apply_A(z)
            wn0 = float(torch.linalg.vector_norm(w))
            h = torch.stack([torch.dot(V[i], w) for i in range(j + 1)])
            for i in range(j + 1):
                w = w - h[i] * V[i]
            hn = float(torch.linalg.vector_norm(w))
            if reorth == 1 or (reorth == 2 and hn < DGKS_KAPPA * wn0):
                h2 = torch.stack([torch.dot(V[i], w) for i in range(j + 1)])
                for i in range(j + 1):
                    w = w - h2[i] * V[i]
                h = h + h2
                hn = float(torch.linalg.vector_norm(w))
                st.reorth_passes += 1
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            # apply the previous rotations, then form the new one
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, bb = float(H[j, j]), float(H[j + 1, j])
            den = math.sqrt(a * a + bb * bb)
            c_, s_ = (1.0, 0.0) if den == 0.0 else (a / den, bb / den)
            cs[j], sn[j] = c_, s_
            H[j, j] = c_ * a + s_ * bb
            H[j + 1, j] = 0.0
            gvec[j + 1] = -s_ * gvec[j]
            gvec[j] = c_ * gvec[j]
            total += 1
            k = j + 1
            res = abs(float(gvec[j + 1]))
            st.res_history.append(res)
            if hn == 0.0:
                done = True
                break
            V.append(w / hn)
            if not fixed and res < eta * beta0:
                done = True
                break
        # least squares: upper-triangular back substitution
        y = torch.zeros(k, dtype=torch.float64)
        for i in range(k - 1, -1, -1):
            s = float(gvec[i])
            for l in range(i + 1, k):
                s -= float(H[i, l]) * float(y[l])
            y[i] = s / float(H[i, i])
        for i in range(k):
            x = x + y[i] * Z[i]
        st.iterations = total
        if done or total >= max_it:
            st.converged = (not fixed) and done or (res < eta * beta0)
            return x, st
        # restart from the true residual
        r = b - apply_A(x)
        st.restarts += 1


# ----------------------------------------------------------------------------
# Newton
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class StepStats:
    newton_iterations: int = 0
    gmres_iterations: List[int] = dataclasses.field(default_factory=list)
    converged: bool = False
    dx_inf: List[float] = dataclasses.field(default_factory=list)
    fhat_norm: List[float] = dataclasses.field(default_factory=list)
    deltas: List[float] = dataclasses.field(default_factory=list)


def newton_step(P: D.Problem, Xn, dt: float, opts: Options, on_iterate=None):
    """One implicit step: solve F_U(X) = 0 from X^(0) = X^n (Sect. 4.1)."""
    from . import precond as PC
    Xn = D.as_tensor(Xn)
    bn = D.bn_constant(P, Xn, dt)
    X = Xn.clone()
    st = StepStats()
    si = None
    for k in range(opts.newton_max):
        sc = scaling(P, X, opts)
        G0 = D.G_operator(P, X, dt)
        Fhat = (G0 - bn) / sc.L
        st.fhat_norm.append(float(torch.linalg.vector_norm(Fhat)))
        if opts.precond:
            # pc_freeze: the setup at X^(0) = X^n serves every iterate of the
            # step; the scaling sc still follows the iterate
            if si is None or not opts.pc_freeze:
                si = PC.setup(P, X, dt, opts)
            Minv = lambda v, si=si: PC.apply(si, v, sc)    # noqa: E731
        else:
            Minv = lambda v: v                             # noqa: E731

        def A(z):
            r, d = jv(P, X, G0, sc, z, dt, opts)
            st.deltas.append(d)
            return r

        dxh, gs = gmres(A, Minv, -Fhat, opts.eta, opts.gmres_m, opts.gmres_max_it,
                        opts.reorth, opts.fixed_iterations)
        st.gmres_iterations.append(gs.iterations)
        X = X + sc.R * dxh
        dinf = float(torch.max(torch.abs(dxh)))
        st.dx_inf.append(dinf)
        st.newton_iterations = k + 1
        if on_iterate is not None:
            on_iterate(k, X, dxh, gs)
        if not math.isfinite(dinf):
            break
        if not opts.fixed_iterations and k + 1 >= opts.newton_min and dinf < opts.newton_tol:
            st.converged = True
            break
    return X, st


def si_step(P: D.Problem, Xn, dt: float, opts: Options) -> torch.Tensor:
    """One step of the SI scheme used as a time integrator (Sect. 3.6):
    F_U(X^n) = -R_U(X^n); transform to the primitive residual, solve the SI
    system built at X^n, transform back and add: X^{n+1} = X^n + dX.  In the
    scaled variables of the preconditioner, dX = R M^-1(-F^) with the
    preconditioner of Sect. 4.3 (its sign convention makes M approximate
    +dF/dX).  First order in time; the paper's scheme treats the SI terms by
    backward Euler (theta = 1)."""
    from . import precond as PC
    Xn = D.as_tensor(Xn)
    sc = scaling(P, Xn, opts)
    F = D.residual(P, Xn, Xn, dt)                      # G(X^n) - b^n(X^n) = -R_U(X^n)
    si = PC.setup(P, Xn, dt, opts)
    dxh = PC.apply(si, -F / sc.L, sc)
    return Xn + sc.R * dxh
