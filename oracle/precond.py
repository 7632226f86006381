"""Physics-based preconditioner (paper Sects. 3 and 4.3).  TEST
INFRASTRUCTURE: see the package docstring for who may import this.

M^-1 applied to a scaled Krylov vector v^ (Sect. 4.3 algorithm):
  1. v = L v^ is a residual of the conserved variables U; transform it to the
     primitive variables V = (p, e, u) with dV/dU = dV/dX . dX/dU (Sect. 3.2,
     App. B).  On the staggered grid dX/dU acts face by face for velocities:
     r_u = (r_rhou - u_f rbar_rho)/rho_f with rbar_rho the face mean.  For the
     total-energy form r_e = r_eps - <u . r_u>, with <u . a> the cell mean
     sum_d (u_d,lo a_d,lo + u_d,hi a_d,hi)/2 (the derivative of the cell
     kinetic energy).  Then r_p = dp/drho|_e r_rho + dp/de|_rho r_e.
  2. Solve the semi-implicit delta-form system J~_V dV = r_V (the paper writes
     -F~_V on the right; the sign is dropped so that M approximates J):
       sound waves (Eqs. SI3_p, SI3_e, SI3_u):
         dp/dt - th^2 dt G1 p  div(rho_f^-1 grad dp)            = r_p
         de/dt - th^2 dt (p/rho) div(rho_f^-1 grad dp)          = r_e
         du/dt + th rho_f^-1 grad dp                              = r_u
       sound waves + conduction (Eqs. SI4_p_final ... SI4_u_final) add
         -th (G3-1) div(kappa_f grad de) to the p row and
         -th rho^-1 div(kappa_f grad de) to the e row, kappa = chi / c_v.
     th is the time-scheme weight theta (the paper derives the scheme for
     backward Euler, th = 1; with theta the stiff terms of J carry theta, so
     the Laplacian carries theta^2 dt and the coupling theta).  The sound
     system is block lower triangular: dp from the Helmholtz problem, de from
     the identity th^2 dt div(..) dp = (dp/dt - r_p)/(G1 p) (the equality
     below Eq. SI3_blockstructure_V), du by back substitution.  The coupled
     system is solved jointly for (dp, de).  Coefficients come from the
     current Newton iterate.
  3. dX = dX/dV dV: drho = (dp - dp/de de)/(dp/drho), de (internal) or
     deps = de + <u . du> (total), du.  Return w^ = R^-1 dX.

Linear solver for step 2 (replaces the paper's AMG-preconditioned GMRES,
Sect. 3.4): every row pair is multiplied by B^-1, where B is the 2x2 matrix
of the coefficients in front of the two Laplacians, giving
      (1/dt) B^-1 x - [div(rho_f^-1 grad dp); div(kappa_f grad de)] = B^-1 r,
i.e. two plain variable-coefficient diffusion operators coupled only through
a cell-local 2x2 matrix (the sound-only case is the 1x1 version with
B = th^2 dt G1 p).  A fixed number of geometric multigrid V-cycles from zero
makes M^-1 a fixed linear operator:
  * levels: every direction with more than one cell is halved until all have
    one cell (grids must be powers of two); the coarsest level (one cell) is
    solved exactly;
  * coarse coefficients: the cell matrix is the mean over the children, a
    face coefficient the mean over the fine faces forming the coarse face;
    wall faces and directions with a single cell carry no flux;
  * smoother: red-black point-block Gauss-Seidel (colour = parity of i+j+k),
    nu1 sweeps red-then-black before, nu2 sweeps black-then-red after;
  * restriction: mean of the children; prolongation: cell-centred
    (bi/tri)linear interpolation, weights 3/4 and 1/4 per direction, a
    missing neighbour across a wall replaced by the parent itself.
A sparse direct solve of the unscaled system (scipy) is the exact reference,
standing for the paper's remark that eta' <= 1e-6 behaves like a direct solver.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import torch

from . import discretization as D

SOUND = 1
SOUND_DIFF = 2


# ----------------------------------------------------------------------------
# transformations (Sect. 3.2, App. B)
# ----------------------------------------------------------------------------

def _upper(P: D.Problem, q: torch.Tensor, c: int) -> torch.Tensor:
    """Value on the upper face of each cell in direction c (slot i+1; the
    upper wall face, which has no slot, is zero)."""
    up = torch.roll(q, shifts=-1, dims=D.axis(c))
    if P.bc[c] == D.BC_WALL:
        idx = [slice(None)] * 3
        idx[D.axis(c)] = -1
        up = up.clone()
        up[tuple(idx)] = 0.0
    return up


def _lower_cell(P: D.Problem, q: torch.Tensor, c: int) -> torch.Tensor:
    """Value in the cell below each slot along c (ghost-mirrored at walls)."""
    qp = D.pad(P, q)
    return D.crop(P, D.sh(qp, c, -1))


def face_mean(P: D.Problem, q: torch.Tensor, c: int) -> torch.Tensor:
    return 0.5 * (_lower_cell(P, q, c) + q)


def cell_dot(P: D.Problem, u: List[torch.Tensor], a: List[torch.Tensor]) -> torch.Tensor:
    """<u . a> = sum_d (u_d,lo a_d,lo + u_d,hi a_d,hi) / 2 at cell centres."""
    s = torch.zeros_like(u[0])
    for d in range(P.ndim):
        s = s + 0.5 * (u[d] * a[d] + _upper(P, u[d], d) * _upper(P, a[d], d))
    return s


@dataclasses.dataclass
class SIState:
    P: D.Problem
    dt: float
    kind: int
    rho: torch.Tensor
    E: torch.Tensor
    e: torch.Tensor
    u: List[torch.Tensor]
    rho_f: List[torch.Tensor]
    p: torch.Tensor
    Binv: Optional[torch.Tensor]         # (2,2,...) per cell for SOUND_DIFF
    bpp: torch.Tensor
    levels: list
    opts: object


def transform_in(si: SIState, v: torch.Tensor):
    """r_V = dV/dU v (v unscaled, packed).  Returns (r_p, r_e, [r_u_c])."""
    P = si.P
    f = D.unpack(P, v)
    r_rho, r_E = f[0], f[1]
    r_u = []
    for c in range(P.ndim):
        rb = face_mean(P, r_rho, c)
        ruc = (f[2 + c] - si.u[c] * rb) / si.rho_f[c]
        r_u.append(ruc * D.wall_slot_mask(P, c))
    r_e = (r_E - si.E * r_rho) / si.rho
    if P.energy_form == D.ENERGY_TOTAL:
        r_e = r_e - cell_dot(P, si.u, r_u)
    g1 = P.gamma - 1.0
    dpdrho = g1 * si.e
    dpde = g1 * si.rho
    r_p = dpdrho * r_rho + dpde * r_e
    return r_p, r_e, r_u


def transform_out(si: SIState, dp, de, du):
    """dX = dX/dV dV, packed."""
    P = si.P
    g1 = P.gamma - 1.0
    dpdrho = g1 * si.e
    dpde = g1 * si.rho
    drho = (dp - dpde * de) / dpdrho
    dE = de
    if P.energy_form == D.ENERGY_TOTAL:
        dE = de + cell_dot(P, si.u, du)
    return D.pack([drho, dE] + list(du))


# ----------------------------------------------------------------------------
# SI system coefficients, operators and multigrid
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Level:
    n: tuple
    h: tuple
    M: torch.Tensor            # (nf, nf, nz, ny, nx)
    K: torch.Tensor            # (nf, ndim, nz, ny, nx): coefficient on the lower face


def _level_problem(P: D.Problem, n) -> D.Problem:
    return dataclasses.replace(P, n=tuple(n))


def setup(P: D.Problem, X, dt: float, opts) -> SIState:
    """SI coefficients at the current iterate X (Sect. 3.3, 3.4)."""
    kind = opts.precond
    f = D.unpack(P, X)
    rho, E = f[0], f[1]
    u = [f[2 + c] * D.wall_slot_mask(P, c) for c in range(P.ndim)]
    e = D.internal_energy(P, X)
    p = D.pressure(P, rho, e)
    rho_f = [face_mean(P, rho, c) for c in range(P.ndim)]
    th = P.theta
    G1 = G3 = P.gamma
    bpp = th * th * dt * G1 * p
    nf = 1 if kind == SOUND else 2
    shape = P.shape
    M = torch.zeros((nf, nf) + shape, dtype=torch.float64)
    K = torch.zeros((nf, P.ndim) + shape, dtype=torch.float64)
    Binv = None
    if kind == SOUND:
        M[0, 0] = (1.0 / dt) / bpp
    else:
        bpe = th * (G3 - 1.0) * torch.ones_like(p)
        bep = th * th * dt * p / rho
        bee = th / rho
        det = bpp * bee - bpe * bep
        Binv = torch.stack([torch.stack([bee / det, -bpe / det]),
                            torch.stack([-bep / det, bpp / det])])
        M = Binv / dt
    cv = 1.0 / (P.gamma - 1.0)
    chi = D.conductivity(P, D.temperature(P, e)) if P.K0 != 0.0 else torch.zeros_like(p)
    for c in range(P.ndim):
        m = D.wall_slot_mask(P, c) if P.n[c] > 1 else torch.zeros(shape, dtype=torch.float64)
        K[0, c] = m / rho_f[c]
        if nf == 2:
            K[1, c] = m * face_mean(P, chi, c) / cv
    levels = [Level(n=tuple(P.n), h=tuple(P.dx), M=M, K=K)]
    while any(levels[-1].n[d] > 1 for d in range(P.ndim)):
        levels.append(_coarsen(P, levels[-1]))
    return SIState(P=P, dt=dt, kind=kind, rho=rho, E=E, e=e, u=u, rho_f=rho_f, p=p, Binv=Binv,
                   bpp=bpp, levels=levels, opts=opts)


def _check_pow2(n):
    for v in n:
        if v & (v - 1):
            raise ValueError("multigrid needs power-of-two grids")


def _coarsen(P: D.Problem, lv: Level) -> Level:
    _check_pow2(lv.n)
    nd = P.ndim
    cdims = [d for d in range(nd) if lv.n[d] > 1]
    nc = tuple(lv.n[d] // 2 if d in cdims else lv.n[d] for d in range(3))
    hc = tuple(lv.h[d] * 2 if d in cdims else lv.h[d] for d in range(3))

    def child_mean(q):
        # q (..., nz, ny, nx): mean over the children of each coarse cell
        for d in cdims:
            a = q.dim() - 1 - d
            sh_ = list(q.shape)
            sh_[a:a + 1] = [sh_[a] // 2, 2]
            q = q.reshape(sh_).mean(dim=a + 1)
        return q

    M = child_mean(lv.M)
    nf = lv.K.shape[0]
    K = torch.zeros((nf, nd) + (nc[2], nc[1], nc[0]), dtype=torch.float64)
    for d in range(nd):
        if nc[d] == 1:
            continue
        Kd = lv.K[:, d]
        # fine lower faces of the even children along d form the coarse face
        a = Kd.dim() - 1 - d
        idx = torch.arange(0, lv.n[d], 2)
        Kd = Kd.index_select(a, idx)
        for e in cdims:
            if e == d:
                continue
            ae = Kd.dim() - 1 - e
            sh_ = list(Kd.shape)
            sh_[ae:ae + 1] = [sh_[ae] // 2, 2]
            Kd = Kd.reshape(sh_).mean(dim=ae + 1)
        K[:, d] = Kd
    return Level(n=nc, h=hc, M=M, K=K)


def _nb(x, d, s):
    """Neighbour value along d (s = +1 upper, -1 lower), periodic index wrap;
    wall neighbours are multiplied by zero coefficients by construction."""
    return torch.roll(x, shifts=-s, dims=x.dim() - 1 - d)


def _Kup(K, d):
    return torch.roll(K, shifts=-1, dims=K.dim() - 1 - d)


def mg_apply_A(P: D.Problem, lv: Level, x: torch.Tensor) -> torch.Tensor:
    """(A x)_f = sum_g M_fg x_g - div(K_f grad x_f), x of shape (nf, nz, ny, nx)."""
    nf = x.shape[0]
    out = torch.einsum('fg...,g...->f...', lv.M, x)
    for f in range(nf):
        for d in range(P.ndim):
            if lv.n[d] == 1:
                continue
            Kl = lv.K[f, d]
            Ku = _Kup(Kl, d)
            h2 = lv.h[d] * lv.h[d]
            out[f] = out[f] - (Ku * (_nb(x[f], d, 1) - x[f]) - Kl * (x[f] - _nb(x[f], d, -1))) / h2
    return out


def _colour(n):
    k = torch.arange(n[2]).reshape(-1, 1, 1)
    j = torch.arange(n[1]).reshape(1, -1, 1)
    i = torch.arange(n[0]).reshape(1, 1, -1)
    return ((i + j + k) % 2).to(torch.bool)


def _half_sweep(P: D.Problem, lv: Level, x: torch.Tensor, rhs: torch.Tensor, colour: int):
    nf = x.shape[0]
    mask = _colour(lv.n) if colour == 1 else ~_colour(lv.n)
    diag = []
    off = []
    for f in range(nf):
        dg = torch.zeros(x.shape[1:], dtype=torch.float64)
        of = torch.zeros(x.shape[1:], dtype=torch.float64)
        for d in range(P.ndim):
            if lv.n[d] == 1:
                continue
            Kl = lv.K[f, d]
            Ku = _Kup(Kl, d)
            h2 = lv.h[d] * lv.h[d]
            dg = dg + (Kl + Ku) / h2
            of = of + (Ku * _nb(x[f], d, 1) + Kl * _nb(x[f], d, -1)) / h2
        diag.append(dg)
        off.append(of)
    if nf == 1:
        new = (rhs[0] + off[0]) / (lv.M[0, 0] + diag[0])
        x[0] = torch.where(mask, new, x[0])
    else:
        a11 = lv.M[0, 0] + diag[0]
        a12 = lv.M[0, 1]
        a21 = lv.M[1, 0]
        a22 = lv.M[1, 1] + diag[1]
        b1 = rhs[0] + off[0]
        b2 = rhs[1] + off[1]
        det = a11 * a22 - a12 * a21
        n1 = (a22 * b1 - a12 * b2) / det
        n2 = (a11 * b2 - a21 * b1) / det
        x[0] = torch.where(mask, n1, x[0])
        x[1] = torch.where(mask, n2, x[1])
    return x


def _restrict(P: D.Problem, fine: Level, coarse: Level, r: torch.Tensor) -> torch.Tensor:
    q = r
    for d in range(P.ndim):
        if fine.n[d] != coarse.n[d]:
            a = q.dim() - 1 - d
            sh_ = list(q.shape)
            sh_[a:a + 1] = [sh_[a] // 2, 2]
            q = q.reshape(sh_).mean(dim=a + 1)
    return q


def _prolong(P: D.Problem, fine: Level, coarse: Level, xc: torch.Tensor) -> torch.Tensor:
    q = xc
    for d in range(P.ndim):
        if fine.n[d] == coarse.n[d]:
            continue
        a = q.dim() - 1 - d
        ncd = coarse.n[d]
        i = torch.arange(fine.n[d])
        par = i // 2
        other = torch.where(i % 2 == 0, par - 1, par + 1)
        if P.bc[d] == D.BC_PERIODIC:
            other = other % ncd
        else:
            other = torch.where((other < 0) | (other >= ncd), par, other)
        qa = q.index_select(a, par)
        qb = q.index_select(a, other)
        q = 0.75 * qa + 0.25 * qb
    return q


def _vcycle(P: D.Problem, levels, l: int, x: torch.Tensor, rhs: torch.Tensor, nu1: int, nu2: int):
    lv = levels[l]
    if l == len(levels) - 1:
        # one cell: the Laplacians vanish, solve the local nf x nf system
        if x.shape[0] == 1:
            return rhs / lv.M[0, 0]
        a11, a12, a21, a22 = lv.M[0, 0], lv.M[0, 1], lv.M[1, 0], lv.M[1, 1]
        det = a11 * a22 - a12 * a21
        return torch.stack([(a22 * rhs[0] - a12 * rhs[1]) / det, (a11 * rhs[1] - a21 * rhs[0]) / det])
    for _ in range(nu1):
        x = _half_sweep(P, lv, x, rhs, 0)
        x = _half_sweep(P, lv, x, rhs, 1)
    r = rhs - mg_apply_A(P, lv, x)
    rc = _restrict(P, lv, levels[l + 1], r)
    xc = _vcycle(P, levels, l + 1, torch.zeros_like(rc), rc, nu1, nu2)
    x = x + _prolong(P, lv, levels[l + 1], xc)
    for _ in range(nu2):
        x = _half_sweep(P, lv, x, rhs, 1)
        x = _half_sweep(P, lv, x, rhs, 0)
    return x


def mg_solve(si: SIState, rhs: torch.Tensor, cycles: int, nu1: int = 2, nu2: int = 2) -> torch.Tensor:
    x = torch.zeros_like(rhs)
    for _ in range(cycles):
        x = _vcycle(si.P, si.levels, 0, x, rhs, nu1, nu2)
    return x


# ----------------------------------------------------------------------------
# the SI system in the paper's (unscaled) form, assembled and applied
# ----------------------------------------------------------------------------

def _laplacian(P, K, x):
    """div(K grad x) on the fine grid, K on lower faces per direction."""
    out = torch.zeros_like(x)
    for d in range(P.ndim):
        if P.n[d] == 1:
            continue
        Ku = _Kup(K[d], d)
        out = out + (Ku * (_nb(x, d, 1) - x) - K[d] * (x - _nb(x, d, -1))) / (P.dx[d] ** 2)
    return out


def paper_rows(si: SIState, dp, de):
    """Left-hand sides of the p and e rows exactly as written in the paper
    (with theta): returns (row_p, row_e)."""
    P = si.P
    th, dt = P.theta, si.dt
    G1 = G3 = P.gamma
    lvl = si.levels[0]
    Lp = _laplacian(P, [lvl.K[0, d] for d in range(P.ndim)], dp)
    row_p = dp / dt - th * th * dt * G1 * si.p * Lp
    row_e = de / dt - th * th * dt * (si.p / si.rho) * Lp
    if si.kind == SOUND_DIFF:
        Le = _laplacian(P, [lvl.K[1, d] for d in range(P.ndim)], de)
        row_p = row_p - th * (G3 - 1.0) * Le
        row_e = row_e - th / si.rho * Le
    return row_p, row_e


def assemble_paper_matrix(si: SIState):
    """Sparse matrix of the p (and e) rows, built entry by entry from the
    paper's equations (scipy CSR).  Unknown order: dp then de (cells, C order)."""
    import scipy.sparse as sp
    P = si.P
    nc = P.ncell
    nz, ny, nx = P.shape
    nf = 1 if si.kind == SOUND else 2
    th, dt = P.theta, si.dt
    G1 = G3 = P.gamma
    p = si.p.reshape(-1).numpy()
    rho = si.rho.reshape(-1).numpy()
    K0 = [si.levels[0].K[0, d].reshape(-1).numpy() for d in range(P.ndim)]
    K1 = [si.levels[0].K[1, d].reshape(-1).numpy() for d in range(P.ndim)] if nf == 2 else None
    rows, cols, vals = [], [], []

    def cid(i, j, k):
        return (k % nz) * ny * nx + (j % ny) * nx + (i % nx)

    # coefficient in front of each Laplacian in each row
    def coef(row, col, c):
        if row == 0 and col == 0:
            return th * th * dt * G1 * p[c]
        if row == 0 and col == 1:
            return th * (G3 - 1.0)
        if row == 1 and col == 0:
            return th * th * dt * p[c] / rho[c]
        return th / rho[c]

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = cid(i, j, k)
                for row in range(nf):
                    rows.append(row * nc + c)
                    cols.append(row * nc + c)
                    vals.append(1.0 / dt)
                for col in range(nf):
                    Kf = K0 if col == 0 else K1
                    for d in range(P.ndim):
                        if P.n[d] == 1:
                            continue
                        off = [0, 0, 0]
                        off[d] = 1
                        up = cid(i + off[0], j + off[1], k + off[2])
                        dn = cid(i - off[0], j - off[1], k - off[2])
                        ku, kl = Kf[d][up], Kf[d][c]
                        h2 = P.dx[d] ** 2
                        rws = range(2) if nf == 2 else range(1)
                        for row in rws:
                            if nf == 1 and row == 1:
                                continue
                            a = coef(row, col, c) / h2
                            rows += [row * nc + c] * 3
                            cols += [col * nc + up, col * nc + dn, col * nc + c]
                            vals += [-a * ku, -a * kl, a * (ku + kl)]
    n = nf * nc
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def direct_solve(si: SIState, r_p: torch.Tensor, r_e: torch.Tensor):
    import scipy.sparse.linalg as spla
    A = assemble_paper_matrix(si)
    if si.kind == SOUND:
        x = spla.spsolve(A.tocsc(), r_p.reshape(-1).numpy())
        return torch.as_tensor(x).reshape(si.P.shape), None
    b = np.concatenate([r_p.reshape(-1).numpy(), r_e.reshape(-1).numpy()])
    x = spla.spsolve(A.tocsc(), b)
    nc = si.P.ncell
    return (torch.as_tensor(x[:nc]).reshape(si.P.shape), torch.as_tensor(x[nc:]).reshape(si.P.shape))


# ----------------------------------------------------------------------------
# full preconditioner apply
# ----------------------------------------------------------------------------

def si_solve(si: SIState, r_p, r_e, r_u, exact: bool = False, cycles: Optional[int] = None):
    """Steps 2 of the algorithm: (dp, de, du) from the primitive residuals."""
    P = si.P
    opts = si.opts
    th, dt = P.theta, si.dt
    G1 = P.gamma
    if si.kind == SOUND:
        if exact:
            dp, _ = direct_solve(si, r_p, r_e)
        else:
            rhs = (r_p / si.bpp).unsqueeze(0)
            dp = mg_solve(si, rhs, opts.mg_cycles if cycles is None else cycles, opts.mg_nu1, opts.mg_nu2)[0]
        de = dt * (r_e + (dp / dt - r_p) / (G1 * si.rho))
    else:
        if exact:
            dp, de = direct_solve(si, r_p, r_e)
        else:
            B = si.Binv
            rhs = torch.stack([B[0, 0] * r_p + B[0, 1] * r_e, B[1, 0] * r_p + B[1, 1] * r_e])
            x = mg_solve(si, rhs, opts.mg_cycles if cycles is None else cycles, opts.mg_nu1, opts.mg_nu2)
            dp, de = x[0], x[1]
    du = []
    for c in range(P.ndim):
        gp = (dp - _lower_cell(P, dp, c)) / P.dx[c]
        du.append(dt * (r_u[c] - th * gp / si.rho_f[c]) * D.wall_slot_mask(P, c))
    return dp, de, du


def apply(si: SIState, vhat: torch.Tensor, sc, exact: Optional[bool] = None) -> torch.Tensor:
    """w^ = R^-1 dX/dV J~_V^-1 dV/dU L v^ (Sect. 4.3 algorithm, steps 1-3)."""
    v = sc.L * vhat
    r_p, r_e, r_u = transform_in(si, v)
    ex = si.opts.exact_inner if exact is None else exact
    dp, de, du = si_solve(si, r_p, r_e, r_u, exact=ex)
    dX = transform_out(si, dp, de, du)
    return dX / sc.R
