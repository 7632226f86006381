"""Spatial and temporal discretisation (paper Sect. 2).  TEST INFRASTRUCTURE:
see the package docstring for who may import this.

Equations (Sect. 2, Eqs. cons1-cons3 and Etot):
    d_t rho        = -div(rho u)
    d_t (rho e)    = -div(rho e u) - p div u + div(chi grad T)
    d_t (rho u)    = -div(rho u (x) u) - grad p + rho g
    d_t (rho eps_t)= -div(rho eps_t u + p u) + rho u.g + div(chi grad T)
with an ideal gas (R = 1): p = (gamma-1) rho e, T = (gamma-1) e,
chi = K0 T^chi_exp (Eq. chirad with a power-law conductivity).

The paper only names the scheme: finite volumes, velocities staggered at the
cell faces, van Leer's upwind monotonicity-preserving reconstruction, second
order and TVD (Sect. 2, "method of lines" paragraph).  The concrete reading
used here (and by the CUDA library) is:

* Reconstruction: van Leer's harmonic slope s_i = 2 a b / (a + b) if a b > 0
  else 0, with a = q_i - q_{i-1}, b = q_{i+1} - q_i.  The upwind face value is
  q_L + s_L/2 when the upwinding speed is >= 0 (ties go to the lower side),
  else q_R - s_R/2.
* Mass flux at a face: Fm = u_f rho_up.  Internal-energy flux Fm e_up plus the
  cell source -p_i (div u)_i.  Total-energy flux Fm eps_up + (p_L+p_R)/2 u_f
  and the work term sum_d g_d (Fm_d,lower + Fm_d,upper)/2.
* Momentum on face k of direction c: conserved rho_f u_f with
  rho_f = (rho_L + rho_R)/2.  Along every direction d its flux sits between
  the faces: the carrying mass flux is (Fm_d(k - 1_c) + Fm_d(k))/2, and u_c is
  reconstructed along d and upwinded by the sign of that mass flux.  Pressure
  force -(p_R - p_L)/dx_c and gravity rho_f g_c.
* Conduction: flux chi_f (T_R - T_L)/dx with chi_f = (chi_L + chi_R)/2.
* Boundaries: periodic wrap, or reflecting walls with mirror ghosts (scalars
  and tangential velocity even, normal velocity odd); wall faces carry no
  mass, momentum, energy or heat flux.
* Cell kinetic energy (total-energy form): sum_d (u_d,lower^2 + u_d,upper^2)/4.
* Time discretisation (Eq. crank_nicholson, generalised to a theta-scheme):
      F_U(X) = (U(X) - U(X^n))/dt - theta R_U(X) - (1-theta) R_U(X^n),
  theta = 1/2 is the paper's Crank-Nicolson, theta = 1 backward Euler.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import torch

GHOST = 3          # stencil radius of the momentum residual
BC_PERIODIC = 0
BC_WALL = 1
ENERGY_INTERNAL = 0
ENERGY_TOTAL = 1

_f64 = torch.float64


@dataclasses.dataclass
class Problem:
    """Grid and physics of one problem (all the residual needs)."""
    ndim: int
    n: Tuple[int, int, int]
    dx: Tuple[float, float, float]
    bc: Tuple[int, int, int]
    gamma: float
    g: Tuple[float, float, float]
    K0: float
    chi_exp: float
    energy_form: int
    theta: float

    @staticmethod
    def from_workload(wl, theta=None) -> "Problem":
        return Problem(ndim=wl.ndim, n=tuple(wl.n), dx=tuple(wl.dx), bc=tuple(wl.bc), gamma=wl.gamma,
                       g=tuple(wl.g), K0=wl.K0, chi_exp=wl.chi_exp, energy_form=wl.energy_form,
                       theta=wl.theta if theta is None else theta)

    @property
    def ncell(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def nfield(self) -> int:
        return 2 + self.ndim

    @property
    def shape(self) -> Tuple[int, int, int]:
        return (self.n[2], self.n[1], self.n[0])


# ----------------------------------------------------------------------------
# packing
# ----------------------------------------------------------------------------

def as_tensor(x) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        return x.to(_f64)
    return torch.as_tensor(x, dtype=_f64)


def unpack(P: Problem, X) -> List[torch.Tensor]:
    X = as_tensor(X)
    return [X[k * P.ncell:(k + 1) * P.ncell].reshape(P.shape) for k in range(P.nfield)]


def pack(fields: Sequence[torch.Tensor]) -> torch.Tensor:
    return torch.cat([f.reshape(-1) for f in fields])


def axis(d: int) -> int:
    """Tensor axis of direction d (x is the last, fastest axis)."""
    return 2 - d


def wall_slot_mask(P: Problem, c: int) -> torch.Tensor:
    """1 on unknown faces of direction c, 0 on the wall-face slot."""
    m = torch.ones(P.shape, dtype=_f64)
    if P.bc[c] == BC_WALL:
        idx = [slice(None)] * 3
        idx[axis(c)] = 0
        m[tuple(idx)] = 0.0
    return m


def zero_wall_slots(P: Problem, fields: List[torch.Tensor]) -> List[torch.Tensor]:
    out = list(fields[:2])
    for c in range(P.ndim):
        out.append(fields[2 + c] * wall_slot_mask(P, c))
    return out


# ----------------------------------------------------------------------------
# ghost extension and shifts
# ----------------------------------------------------------------------------

def _ghost_index(n: int, bc: int, face_normal: bool):
    """Source index and sign for padded positions k = -GHOST .. n+GHOST-1.

    Cell quantities mirror about the wall faces (k -> -k-1, k -> 2n-1-k);
    the face-normal velocity mirrors about the face positions with a sign flip
    (k -> -k, k -> 2n-k) and is zero on both wall faces (slot n is an extra
    zero appended by the caller)."""
    idx, sgn = [], []
    for k in range(-GHOST, n + GHOST):
        if bc == BC_PERIODIC:
            idx.append(k % n)
            sgn.append(1.0)
        elif not face_normal:
            if k < 0:
                idx.append(-k - 1)
            elif k >= n:
                idx.append(2 * n - 1 - k)
            else:
                idx.append(k)
            sgn.append(1.0)
        else:
            if k < 0:
                idx.append(-k)
                sgn.append(-1.0)
            elif k > n:
                idx.append(2 * n - k)
                sgn.append(-1.0)
            else:
                idx.append(k)
                sgn.append(1.0)
    top = n if face_normal else n - 1
    if any(i < 0 or i > top for i in idx):
        raise ValueError("grid too small for the stencil (need at least 4 cells per direction)")
    return torch.tensor(idx, dtype=torch.long), torch.tensor(sgn, dtype=_f64)


def pad(P: Problem, q: torch.Tensor, normal_dir: int = -1) -> torch.Tensor:
    """Extend q by GHOST ghost layers in every active direction.

    normal_dir = c marks q as the velocity normal to the faces of direction c
    (odd mirror at walls in that direction); -1 marks a cell quantity."""
    for d in range(P.ndim):
        a = axis(d)
        fn = (d == normal_dir)
        src = q
        if fn and P.bc[d] == BC_WALL:
            zshape = list(q.shape)
            zshape[a] = 1
            src = torch.cat([q, torch.zeros(zshape, dtype=_f64)], dim=a)   # upper wall face
        idx, sgn = _ghost_index(P.n[d], P.bc[d], fn and P.bc[d] == BC_WALL)
        q = src.index_select(a, idx)
        shp = [1, 1, 1]
        shp[a] = sgn.numel()
        q = q * sgn.reshape(shp)
    return q


def crop(P: Problem, q: torch.Tensor) -> torch.Tensor:
    sl = [slice(None)] * 3
    for d in range(P.ndim):
        sl[axis(d)] = slice(GHOST, GHOST + P.n[d])
    return q[tuple(sl)]


def sh(q: torch.Tensor, d: int, s: int) -> torch.Tensor:
    """sh(q, d, s)[k] = q[k + s] along direction d (wrap-around garbage only
    reaches the outer ghost layers, which are cropped)."""
    return torch.roll(q, shifts=-s, dims=axis(d))


# ----------------------------------------------------------------------------
# EOS and reconstruction
# ----------------------------------------------------------------------------

def pressure(P: Problem, rho, e):
    return (P.gamma - 1.0) * rho * e


def temperature(P: Problem, e):
    return (P.gamma - 1.0) * e


def sound_speed(P: Problem, e):
    return torch.sqrt(P.gamma * (P.gamma - 1.0) * e)


def conductivity(P: Problem, T):
    if P.chi_exp == 3.0:
        return P.K0 * (T * T * T)
    return P.K0 * T ** P.chi_exp


def vanleer_slope(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """van Leer (1974) harmonic limited slope 2ab/(a+b) if ab > 0, else 0."""
    ab = a * b
    pos = ab > 0
    den = torch.where(pos, a + b, torch.ones_like(a))
    return torch.where(pos, 2.0 * ab / den, torch.zeros_like(a))


def slope(q: torch.Tensor, d: int) -> torch.Tensor:
    return vanleer_slope(q - sh(q, d, -1), sh(q, d, 1) - q)


def upwind(q: torch.Tensor, s: torch.Tensor, speed: torch.Tensor, d: int) -> torch.Tensor:
    """Value at the lower face of each slot along d: from the lower cell
    (q + s/2 there) if speed >= 0, else from this cell (q - s/2)."""
    left = sh(q + 0.5 * s, d, -1)
    right = q - 0.5 * s
    return torch.where(speed >= 0, left, right)


# ----------------------------------------------------------------------------
# right-hand side R_U(X) and conserved variables U(X)
# ----------------------------------------------------------------------------

def _padded_state(P: Problem, X):
    f = unpack(P, X)
    rho = pad(P, f[0])
    E = pad(P, f[1])
    # the wall-face slot is read as zero whatever it holds
    u = [pad(P, f[2 + c] * wall_slot_mask(P, c), normal_dir=c) for c in range(P.ndim)]
    return rho, E, u


def cell_kinetic_energy(P: Problem, u: List[torch.Tensor]) -> torch.Tensor:
    """sum_d (u_d,lower^2 + u_d,upper^2)/4 (padded arrays in, padded out)."""
    ke = torch.zeros_like(u[0])
    for d in range(P.ndim):
        ke = ke + 0.25 * (u[d] * u[d] + sh(u[d], d, 1) * sh(u[d], d, 1))
    return ke


def rhs(P: Problem, X) -> List[torch.Tensor]:
    """R_U(X) (Eq. mol): [R_rho, R_(rho e or rho eps_t), R_(rho u_c)...],
    each of shape (nz, ny, nx); wall-face slots are zero."""
    rho, E, u = _padded_state(P, X)
    nd = P.ndim
    if P.energy_form == ENERGY_TOTAL:
        e = E - cell_kinetic_energy(P, u)
    else:
        e = E
    p = pressure(P, rho, e)
    T = temperature(P, e)
    diffusion = P.K0 != 0.0
    if diffusion:
        chi = conductivity(P, T)

    R_rho = torch.zeros_like(rho)
    R_E = torch.zeros_like(rho)
    Fm = []
    divu = torch.zeros_like(rho)
    for d in range(nd):
        h = P.dx[d]
        ud = u[d]
        rho_up = upwind(rho, slope(rho, d), ud, d)
        fm = ud * rho_up                                   # mass flux at lower faces
        Fm.append(fm)
        if P.energy_form == ENERGY_TOTAL:
            E_up = upwind(E, slope(E, d), ud, d)
            fe = fm * E_up + 0.5 * (sh(p, d, -1) + p) * ud
        else:
            e_up = upwind(e, slope(e, d), ud, d)
            fe = fm * e_up
        R_rho = R_rho - (sh(fm, d, 1) - fm) / h
        R_E = R_E - (sh(fe, d, 1) - fe) / h
        divu = divu + (sh(ud, d, 1) - ud) / h
        if diffusion:
            q = 0.5 * (sh(chi, d, -1) + chi) * (T - sh(T, d, -1)) / h    # chi grad T at lower face
            R_E = R_E + (sh(q, d, 1) - q) / h
    if P.energy_form == ENERGY_TOTAL:
        for d in range(nd):
            if P.g[d] != 0.0:
                R_E = R_E + P.g[d] * 0.5 * (Fm[d] + sh(Fm[d], d, 1))
    else:
        R_E = R_E - p * divu

    R_mom = []
    for c in range(nd):
        rho_f = 0.5 * (sh(rho, c, -1) + rho)
        Rc = -(p - sh(p, c, -1)) / P.dx[c]
        if P.g[c] != 0.0:
            Rc = Rc + rho_f * P.g[c]
        uc = u[c]
        for d in range(nd):
            m = 0.5 * (sh(Fm[d], c, -1) + Fm[d])           # carrying mass flux
            u_up = upwind(uc, slope(uc, d), m, d)
            psi = m * u_up
            Rc = Rc - (sh(psi, d, 1) - psi) / P.dx[d]
        R_mom.append(Rc)

    out = [crop(P, R_rho), crop(P, R_E)] + [crop(P, r) for r in R_mom]
    return zero_wall_slots(P, out)


def conserved(P: Problem, X) -> List[torch.Tensor]:
    """U(X) = (rho, rho e or rho eps_t, rho_f u_c) with rho_f the face mean."""
    f = unpack(P, X)
    rho = f[0]
    out = [rho, rho * f[1]]
    rp = pad(P, rho)
    for c in range(P.ndim):
        rho_f = crop(P, 0.5 * (sh(rp, c, -1) + rp))
        out.append(rho_f * f[2 + c])
    return zero_wall_slots(P, out)


def bn_constant(P: Problem, Xn, dt: float) -> torch.Tensor:
    """b^n = U(X^n)/dt + (1-theta) R_U(X^n): the part of F_U fixed by X^n."""
    U = conserved(P, Xn)
    if P.theta != 1.0:
        R = rhs(P, Xn)
        return pack([U[k] / dt + (1.0 - P.theta) * R[k] for k in range(P.nfield)])
    return pack([U[k] / dt for k in range(P.nfield)])


def G_operator(P: Problem, X, dt: float) -> torch.Tensor:
    """G(X) = U(X)/dt - theta R_U(X), so that F_U(X) = G(X) - b^n."""
    U = conserved(P, X)
    R = rhs(P, X)
    return pack([U[k] / dt - P.theta * R[k] for k in range(P.nfield)])


def residual(P: Problem, X, Xn, dt: float) -> torch.Tensor:
    """F_U(X) of Eq. crank_nicholson (theta-scheme), packed."""
    return G_operator(P, X, dt) - bn_constant(P, Xn, dt)


def residual_direct(P: Problem, X, Xn, dt: float) -> torch.Tensor:
    """The same F_U written term by term as in Eq. crank_nicholson."""
    U1, U0 = conserved(P, X), conserved(P, Xn)
    R1, R0 = rhs(P, X), rhs(P, Xn)
    return pack([(U1[k] - U0[k]) / dt - P.theta * R1[k] - (1.0 - P.theta) * R0[k]
                 for k in range(P.nfield)])


def cell_velocity_magnitude(P: Problem, X) -> torch.Tensor:
    f = unpack(P, X)
    s = torch.zeros(P.shape, dtype=_f64)
    for c in range(P.ndim):
        up = pad(P, f[2 + c], normal_dir=c)
        ubar = crop(P, 0.5 * (up + sh(up, c, 1)))
        s = s + ubar * ubar
    return torch.sqrt(s)


def internal_energy(P: Problem, X) -> torch.Tensor:
    f = unpack(P, X)
    if P.energy_form == ENERGY_TOTAL:
        _, _, u = _padded_state(P, X)
        return f[1] - crop(P, cell_kinetic_energy(P, u))
    return f[1]


def cfl_dt(P: Problem, X, cfl: float) -> float:
    """dt = CFL_hydro * min_d dx_d / max(|u_cell| + c_s)  (Sect. 1, Eq. 1),
    with u_cell the mean of the two face velocities in each direction."""
    e = internal_energy(P, X)
    speed = cell_velocity_magnitude(P, X) + sound_speed(P, e)
    hmin = min(P.dx[d] for d in range(P.ndim))
    return float(cfl * hmin / float(speed.max()))
