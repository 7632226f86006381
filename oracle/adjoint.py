"""Adjoint of one implicit step (gradients through the implicit step by the
implicit-function theorem; the paper has no adjoint).  TEST INFRASTRUCTURE: see the package docstring
for who may import this.

One step defines X^{n+1}(X^n, K0) implicitly by F(X^{n+1}; X^n, K0) = 0 with
F = G(X^{n+1}) - b^n(X^n), G = U/dt - theta R_U, b^n = U(X^n)/dt +
(1-theta) R_U(X^n) (Eq. crank_nicholson).  For a loss with gradient gbar with
respect to X^{n+1}, the implicit-function theorem gives

    J^T lam = gbar,                 J = dG/dX at X^{n+1},
    dL/dX^n = (db^n/dX^n)^T lam,
    dL/dK0  = lam . (theta dR/dK0(X^{n+1}) + (1-theta) dR/dK0(X^n)).

dt is held fixed (it is not differentiated through the CFL rule).  The
transposed system is solved in the scaled form of Eq. jacobian_system_norm,
J^_T mu = R gbar with J^ = L^-1 J R and lam = L^-1 mu, by the same restarted
GMRES, right-preconditioned by the exact transpose of the physics-based
preconditioner.  Vector-Jacobian products are reverse-mode derivatives of the
oracle's residual (torch autograd), i.e. exact transposes of its Jacobian.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import torch

from . import discretization as D
from . import jfnk as J
from . import precond as PC


def vjp_G(P: D.Problem, X, dt: float, w: torch.Tensor) -> torch.Tensor:
    """(dG/dX)^T w at X."""
    X = D.as_tensor(X)
    _, f = torch.func.vjp(lambda x: D.G_operator(P, x, dt), X)
    return f(w)[0]


def vjp_bn(P: D.Problem, Xn, dt: float, w: torch.Tensor) -> torch.Tensor:
    """(db^n/dX^n)^T w."""
    Xn = D.as_tensor(Xn)
    _, f = torch.func.vjp(lambda x: D.bn_constant(P, x, dt), Xn)
    return f(w)[0]


def dR_dK0_dot(P: D.Problem, X, w: torch.Tensor) -> float:
    """w . dR_U/dK0 at X (R_U is linear in K0 through chi = K0 T^exp)."""
    K0 = torch.tensor(P.K0, dtype=torch.float64)
    def R_of(k):
        Q = dataclasses.replace(P, K0=k)
        return D.pack(D.rhs(Q, D.as_tensor(X)))
    _, f = torch.func.vjp(R_of, K0)
    return float(f(w)[0])


@dataclasses.dataclass
class AdjointResult:
    lam: torch.Tensor
    g_Xn: torch.Tensor
    g_K0: float
    gmres_iterations: int
    converged: bool


def step_adjoint(P: D.Problem, Xn, Xnp1, dt: float, gbar: torch.Tensor, opts: J.Options,
                 exact: bool = False) -> AdjointResult:
    """Gradients of a loss through one converged implicit step."""
    Xn, Xnp1 = D.as_tensor(Xn), D.as_tensor(Xnp1)
    sc = J.scaling(P, Xnp1, opts)
    masks = torch.cat([torch.ones(2 * P.ncell, dtype=torch.float64)] +
                      [D.wall_slot_mask(P, c).reshape(-1) for c in range(P.ndim)])
    gbar = gbar * masks
    if exact:
        Jm = torch.func.jacrev(lambda x: D.G_operator(P, x, dt))(Xnp1)
        keep = masks.bool()
        lam = torch.zeros_like(gbar)
        lam[keep] = torch.linalg.solve(Jm[keep][:, keep].T, gbar[keep])
        its, conv = 0, True
    else:
        def A(mu):
            return sc.R * vjp_G(P, Xnp1, dt, mu / sc.L) * masks
        if opts.precond:
            si = PC.setup(P, Xnp1, dt, opts)
            _, fT = torch.func.vjp(lambda v: PC.apply(si, v, sc), torch.zeros_like(gbar))
            Minv = lambda v: fT(v)[0] * masks            # noqa: E731  exact transpose of M^-1
        else:
            Minv = lambda v: v                           # noqa: E731
        mu, st = J.gmres(A, Minv, sc.R * gbar, opts.eta, opts.gmres_m, opts.gmres_max_it)
        lam = mu / sc.L * masks
        its, conv = st.iterations, st.converged
    g_Xn = vjp_bn(P, Xn, dt, lam) * masks
    g_K0 = 0.0
    if P.K0 != 0.0:
        g_K0 = P.theta * dR_dK0_dot(P, Xnp1, lam) + (1.0 - P.theta) * dR_dK0_dot(P, Xn, lam)
    return AdjointResult(lam=lam, g_Xn=g_Xn, g_K0=g_K0, gmres_iterations=its, converged=conv)


def kinetic_energy(P: D.Problem, X) -> torch.Tensor:
    """Loss of the adjoint problem: total kinetic energy sum_faces rho_f u_f^2/2 dV."""
    f = D.unpack(P, X)
    rp = D.pad(P, f[0])
    dV = 1.0
    for d in range(P.ndim):
        dV *= P.dx[d]
    ke = torch.zeros((), dtype=torch.float64)
    for c in range(P.ndim):
        rho_f = D.crop(P, 0.5 * (D.sh(rp, c, -1) + rp))
        u = f[2 + c] * D.wall_slot_mask(P, c)
        ke = ke + 0.5 * torch.sum(rho_f * u * u) * dV
    return ke


def kinetic_energy_grad(P: D.Problem, X) -> torch.Tensor:
    X = D.as_tensor(X).clone().requires_grad_(True)
    kinetic_energy(P, X).backward()
    return X.grad.detach()
