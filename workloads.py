"""Seeded synthetic workloads for the JFNK solver (inputs only).

This module builds initial states, grids and physical parameters for the five
test problems used by the tests and the benchmark.  It holds none of the
method's arithmetic (no residual, no Jacobian, no preconditioner): only the
analytic initial conditions, the seeded noise, and the packing of fields into
the unknown vector.  Both the CPU oracle and the CUDA path receive the same
float64 bytes produced here.

Packed unknown vector X (all problems)
--------------------------------------
Fields are stored as C-ordered arrays of shape (nz, ny, nx) (nz = 1 in 2D),
x fastest, concatenated as  [rho | e (or eps_t) | u_x | u_y | (u_z)],
each block nx*ny*nz long.  rho and e live at cell centres.  u_d lives at the
faces normal to direction d; the slot of cell i holds the velocity on the
LOWER face of cell i in direction d (position x_{i-1/2}).  In a direction with
reflecting walls the slot with index 0 is the wall face: it is present in the
vector and always zero; the upper wall face has no slot (it is zero too).
Units: gas constant R = 1, so T = p/rho and c_v = 1/(gamma-1).

Problem recipes (the paper's stellar models are not available; these analytic
problems stand in for them, following the paper's test problems of Sect. 5.1):

1. 2D Gresho-type steady vortex, 64x64 doubly periodic unit box, gamma=5/3,
   rho=1, u_max=1, background pressure p0 = 1/(gamma M^2), M = 0.01, isobaric
   density noise of relative amplitude 1e-6 (uniform in [-1,1]); backward
   Euler (theta=1), CFL_hydro = 10, 5 steps, sound-wave preconditioner.
2. 2D stratified atmosphere 256x256, gravity g=1 along -y, walls in y,
   periodic in x; polytrope of index 1.5 with density contrast 10 in discrete
   hydrostatic equilibrium; conductivity chi = K0 T^3 with K0 chosen so that
   the radiative CFL equals the hydrodynamic CFL; 8 seeded Gaussian isobaric
   temperature blobs (sigma = 0.05, relative amplitude 1e-4); Crank-Nicolson,
   CFL_hydro = 100, 10 steps, sound + diffusion preconditioner.
3. 3D vortex tube 128^3 periodic: the Gresho profile in x-y, uniform along z,
   p0 = 1/(gamma M^2) for M in {1e-2, 1e-4, 1e-6}, isobaric density noise
   1e-6; CFL_hydro = 1000, 5 steps.
4. 3D stratified box 256^3, gravity along -z, walls in z, periodic in x,y;
   polytrope of index 1.4 (superadiabatic for gamma = 5/3), density contrast
   20, discrete hydrostatic equilibrium, chi = K0 T^3 (same K0 rule); seeded
   velocity noise uniform in [-1,1]*sqrt(3)*1e-3*c_s on every unknown face
   (rms Mach 1e-3 per component); CFL_hydro = 200, 10 steps.
5. Problem 2's construction at 128^2 (and 8x8), CFL_hydro = 50, 4 steps, used
   for the adjoint.

Study workload (no noise): the advected isentropic vortex of the paper's
Sect. 3.7 on [-4, 4]^2, periodic, gamma = 7/5, beta = 0.75, u_inf = 1:
(du, dv) = beta/(2 pi) exp((1 - r^2)/2) (-y, x), dT = -(gamma-1) beta^2 /
(8 gamma pi^2) exp(1 - r^2), rho = (T_inf + dT)^(1/(gamma-1)),
e = T/(gamma-1) = rho^(gamma-1)/(gamma-1); T_inf = 1, 1e2, 1e6, 1e10 give
M_s = beta/(2 pi sqrt(gamma T_inf)) = 1e-1 ... 1e-6 (rounded).  The exact
solution at time t is the initial field shifted by u_inf t along x.

Study workload (no noise): the 3D Taylor-Green vortex of the paper's
Sect. 5.1.2 on [0, 2 pi]^3 (L = 1), 64^3 periodic, gamma = 7/5, rho_0 = 1,
u_0 = 1, u_x = sin x cos y cos z, u_y = -cos x sin y cos z, u_z = 0 sampled at
the face centres, p = p_0 + (2 + cos 2z)(cos 2x + cos 2y)/16 at the cell
centres with p_0 = 1/(gamma M_s^2); Crank-Nicolson, sound-wave
preconditioner.

Seeds: numpy.random.default_rng(problem number); the 8x8 adjoint case uses 50.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

BC_PERIODIC = 0
BC_WALL = 1

ENERGY_INTERNAL = 0
ENERGY_TOTAL = 1

PRECOND_NONE = 0
PRECOND_SOUND = 1
PRECOND_SOUND_DIFF = 2


@dataclasses.dataclass
class Workload:
    """One synthetic problem: grid, physics, initial state and run settings."""
    name: str
    ndim: int
    n: Tuple[int, int, int]            # cells along x, y, z (z = 1 in 2D)
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]
    bc: Tuple[int, int, int]           # BC_PERIODIC or BC_WALL per direction
    gamma: float
    g: Tuple[float, float, float]      # constant gravitational acceleration
    K0: float                          # chi = K0 * T**chi_exp (0 disables)
    chi_exp: float
    energy_form: int
    X0: np.ndarray                     # packed float64 state (see module doc)
    theta: float                       # 1 = backward Euler, 0.5 = Crank-Nicolson
    cfl_hydro: float
    n_steps: int
    precond: int
    seed: int

    @property
    def ncell(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def nvec(self) -> int:
        return (2 + self.ndim) * self.ncell

    @property
    def dx(self) -> Tuple[float, float, float]:
        return tuple((self.hi[d] - self.lo[d]) / self.n[d] for d in range(3))

    def fields(self, X: Optional[np.ndarray] = None) -> List[np.ndarray]:
        """Views of the packed vector as (nz, ny, nx) arrays."""
        X = self.X0 if X is None else X
        shp = (self.n[2], self.n[1], self.n[0])
        return [X[k * self.ncell:(k + 1) * self.ncell].reshape(shp) for k in range(2 + self.ndim)]


def _centres(n: int, lo: float, hi: float) -> np.ndarray:
    h = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * h


def _faces(n: int, lo: float, hi: float) -> np.ndarray:
    h = (hi - lo) / n
    return lo + np.arange(n) * h


def _pack(fields: Sequence[np.ndarray]) -> np.ndarray:
    return np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.float64).ravel() for f in fields]))


def gresho_speed(r: np.ndarray) -> np.ndarray:
    """Azimuthal speed of the Gresho-Chan vortex (u_max = 1 at r = 0.2)."""
    return np.where(r < 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))


def gresho_pressure_excess(r: np.ndarray) -> np.ndarray:
    """p - p_centre for the Gresho-Chan vortex with rho = 1 (radial balance)."""
    inner = 12.5 * r * r
    rr = np.maximum(r, 1e-300)
    mid = 12.5 * r * r - 20.0 * r + 4.0 + 4.0 * np.log(np.maximum(5.0 * rr, 1e-300))
    outer = -2.0 + 4.0 * math.log(2.0) + 0.0 * r
    return np.where(r < 0.2, inner, np.where(r < 0.4, mid, outer))


def _vortex_state(n, lo, hi, bc, ndim, gamma, mach, rng, noise_amp):
    """Gresho vortex in the x-y plane (uniform along z), centred in the box."""
    nx, ny, nz = n
    xc = 0.5 * (lo[0] + hi[0])
    yc = 0.5 * (lo[1] + hi[1])
    p0 = 1.0 / (gamma * mach * mach)
    xcell = _centres(nx, lo[0], hi[0])[None, None, :]
    ycell = _centres(ny, lo[1], hi[1])[None, :, None]
    xface = _faces(nx, lo[0], hi[0])[None, None, :]
    yface = _faces(ny, lo[1], hi[1])[None, :, None]
    shape = (nz, ny, nx)
    r_c = np.sqrt((xcell - xc) ** 2 + (ycell - yc) ** 2) + np.zeros(shape)
    p = p0 + gresho_pressure_excess(r_c)
    noise = rng.uniform(-1.0, 1.0, size=shape)
    rho = 1.0 + noise_amp * noise                       # isobaric perturbation
    e = p / ((gamma - 1.0) * rho)
    # u_x at x-faces (x_{i-1/2}, y_j), u_y at y-faces (x_i, y_{j-1/2})
    rx = np.sqrt((xface - xc) ** 2 + (ycell - yc) ** 2) + np.zeros(shape)
    ux = -gresho_speed(rx) * (ycell - yc) / np.maximum(rx, 1e-300)
    ry = np.sqrt((xcell - xc) ** 2 + (yface - yc) ** 2) + np.zeros(shape)
    uy = gresho_speed(ry) * (xcell - xc) / np.maximum(ry, 1e-300)
    fields = [rho, e, ux, uy]
    if ndim == 3:
        fields.append(np.zeros(shape))
    return fields


def _polytrope_state(n, lo, hi, bc, ndim, gamma, gdir, g, n_poly, contrast):
    """Polytropic background in discrete hydrostatic equilibrium.

    T falls linearly with height, T(h) = T_bot - g (h - lo) / (n_poly + 1), with
    T_bot / T_top = contrast**(1/n_poly) so that rho_bot / rho_top = contrast.
    The pressure obeys, cell to cell along the gravity direction,
        p_{j+1} (1 + g dh / (2 T_{j+1})) = p_j (1 - g dh / (2 T_j)),
    i.e. the face balance (p_{j+1}-p_j)/dh = -g (rho_j + rho_{j+1})/2 with
    rho = p / T; the lowest cell takes the analytic polytrope value (rho = 1
    at the bottom wall).
    """
    L = hi[gdir] - lo[gdir]
    dT = g * L / (n_poly + 1.0)
    ratio = contrast ** (1.0 / n_poly)
    T_top = dT / (ratio - 1.0)
    T_bot = T_top * ratio
    nh = n[gdir]
    h = (hi[gdir] - lo[gdir]) / nh
    hc = _centres(nh, lo[gdir], hi[gdir])
    Tc = T_bot - g * (hc - lo[gdir]) / (n_poly + 1.0)
    pc = np.empty(nh)
    pc[0] = Tc[0] * (Tc[0] / T_bot) ** n_poly
    for j in range(nh - 1):
        pc[j + 1] = pc[j] * (1.0 - g * h / (2.0 * Tc[j])) / (1.0 + g * h / (2.0 * Tc[j + 1]))
    return Tc, pc, T_bot, n_poly


def _broadcast_profile(prof, gdir, shape):
    axis = 2 - gdir
    s = [1, 1, 1]
    s[axis] = prof.size
    return prof.reshape(s) * np.ones(shape)


def _K0_rule(T, rho, gamma, dxmin):
    """K0 such that max(chi / (rho c_v)) = dx * max(c_s), with chi = K0 T^3."""
    cv = 1.0 / (gamma - 1.0)
    cs_max = float(np.max(np.sqrt(gamma * T)))
    D_per_K0 = float(np.max(T ** 3 / (rho * cv)))
    return dxmin * cs_max / D_per_K0


def make_stratified(n, ndim, seed, cfl, n_steps, n_poly, contrast, blobs, vel_noise_mach,
                    gamma=5.0 / 3.0, g=1.0, theta=0.5, precond=PRECOND_SOUND_DIFF, name="stratified"):
    nx, ny, nz = n
    gdir = ndim - 1                       # y in 2D, z in 3D
    lo = (0.0, 0.0, 0.0)
    hi = (1.0, 1.0, 1.0)
    bc = [BC_PERIODIC, BC_PERIODIC, BC_PERIODIC]
    bc[gdir] = BC_WALL
    shape = (nz, ny, nx)
    rng = np.random.default_rng(seed)
    Tc, pc, T_bot, _ = _polytrope_state(n, lo, hi, bc, ndim, gamma, gdir, g, n_poly, contrast)
    T = _broadcast_profile(Tc, gdir, shape)
    p = _broadcast_profile(pc, gdir, shape)
    if blobs > 0:
        centres = rng.uniform(0.0, 1.0, size=(blobs, ndim))
        sigma = 0.05
        pert = np.zeros(shape)
        coords = []
        for d in range(ndim):
            c = _centres(n[d], lo[d], hi[d])
            s = [1, 1, 1]
            s[2 - d] = n[d]
            coords.append(c.reshape(s))
        for b in range(blobs):
            r2 = np.zeros(shape)
            for d in range(ndim):
                dd = coords[d] - centres[b, d]
                if bc[d] == BC_PERIODIC:
                    L = hi[d] - lo[d]
                    dd = dd - L * np.round(dd / L)
                r2 = r2 + dd * dd
            pert += np.exp(-r2 / (2.0 * sigma * sigma))
        T = T * (1.0 + 1e-4 * pert)                       # isobaric: p unchanged
    rho = p / T
    e = T / (gamma - 1.0)
    dxs = [(hi[d] - lo[d]) / n[d] for d in range(ndim)]
    K0 = _K0_rule(T, rho, gamma, min(dxs))
    vel = [np.zeros(shape) for _ in range(ndim)]
    if vel_noise_mach > 0.0:
        hmin = lo[gdir]
        for d in range(ndim):
            xi = rng.uniform(-1.0, 1.0, size=shape)
            if d == gdir:
                hpos = _faces(n[gdir], lo[gdir], hi[gdir])
            else:
                hpos = _centres(n[gdir], lo[gdir], hi[gdir])
            Tf = T_bot - g * (hpos - hmin) / (n_poly + 1.0)
            cs = _broadcast_profile(np.sqrt(gamma * Tf), gdir, shape)
            u = math.sqrt(3.0) * vel_noise_mach * cs * xi
            if d == gdir:
                idx = [slice(None)] * 3
                idx[2 - gdir] = 0
                u[tuple(idx)] = 0.0                       # wall face slot
            vel[d] = u
    gv = [0.0, 0.0, 0.0]
    gv[gdir] = -g
    X0 = _pack([rho, e] + vel)
    return Workload(name=name, ndim=ndim, n=tuple(n), lo=lo, hi=hi, bc=tuple(bc), gamma=gamma,
                    g=tuple(gv), K0=K0, chi_exp=3.0, energy_form=ENERGY_INTERNAL, X0=X0,
                    theta=theta, cfl_hydro=cfl, n_steps=n_steps, precond=precond, seed=seed)


def make_vortex(n, ndim, seed, mach, cfl, n_steps, theta, gamma=5.0 / 3.0, noise_amp=1e-6,
                precond=PRECOND_SOUND, energy_form=ENERGY_INTERNAL, name="vortex"):
    lo = (0.0, 0.0, 0.0)
    hi = (1.0, 1.0, 1.0)
    bc = (BC_PERIODIC, BC_PERIODIC, BC_PERIODIC)
    rng = np.random.default_rng(seed)
    fields = _vortex_state(n, lo, hi, bc, ndim, gamma, mach, rng, noise_amp)
    if energy_form == ENERGY_TOTAL:
        # specific total energy from the analytic speed at the cell centre
        xc = _centres(n[0], lo[0], hi[0])[None, None, :] - 0.5 * (lo[0] + hi[0])
        yc = _centres(n[1], lo[1], hi[1])[None, :, None] - 0.5 * (lo[1] + hi[1])
        r = np.sqrt(xc * xc + yc * yc) + np.zeros(fields[0].shape)
        fields[1] = fields[1] + 0.5 * gresho_speed(r) ** 2
    X0 = _pack(fields)
    return Workload(name=name, ndim=ndim, n=tuple(n), lo=lo, hi=hi, bc=bc, gamma=gamma,
                    g=(0.0, 0.0, 0.0), K0=0.0, chi_exp=3.0, energy_form=energy_form, X0=X0,
                    theta=theta, cfl_hydro=cfl, n_steps=n_steps, precond=precond, seed=seed)


def make_isentropic_vortex(n: int = 64, T_inf: float = 1.0, x_shift: float = 0.0, beta: float = 0.75,
                           gamma: float = 1.4, u_inf: float = 1.0) -> Workload:
    """The advected isentropic vortex of the module docstring on an n^2 grid,
    centred at (x_shift, 0) (periodic images included), so x_shift = u_inf t
    gives the exact solution at time t."""
    lo, hi = (-4.0, -4.0, 0.0), (4.0, 4.0, 1.0)
    bc = (BC_PERIODIC, BC_PERIODIC, BC_PERIODIC)
    L = hi[0] - lo[0]

    def rel(x, y):
        # position relative to the nearest image of the centre
        dx = (x - x_shift - lo[0]) % L + lo[0]
        return dx, y

    xc, yc = _centres(n, lo[0], hi[0]), _centres(n, lo[1], hi[1])
    xf, yf = _faces(n, lo[0], hi[0]), _faces(n, lo[1], hi[1])
    Yc, Xc = np.meshgrid(yc, xc, indexing="ij")
    x, y = rel(Xc, Yc)
    dT = -(gamma - 1.0) * beta ** 2 / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - (x * x + y * y))
    T = T_inf + dT
    rho = T ** (1.0 / (gamma - 1.0))
    e = T / (gamma - 1.0)
    amp = beta / (2.0 * math.pi)
    Yx, Xx = np.meshgrid(yc, xf, indexing="ij")           # x-faces
    x, y = rel(Xx, Yx)
    u = u_inf + amp * np.exp(0.5 * (1.0 - (x * x + y * y))) * (-y)
    Yy, Xy = np.meshgrid(yf, xc, indexing="ij")           # y-faces
    x, y = rel(Xy, Yy)
    v = amp * np.exp(0.5 * (1.0 - (x * x + y * y))) * x
    X0 = _pack([a[None] for a in (rho, e, u, v)])
    return Workload(name="isentropic_vortex", ndim=2, n=(n, n, 1), lo=lo, hi=hi, bc=bc, gamma=gamma,
                    g=(0.0, 0.0, 0.0), K0=0.0, chi_exp=3.0, energy_form=ENERGY_INTERNAL, X0=X0, theta=0.5,
                    cfl_hydro=1.0, n_steps=1, precond=PRECOND_SOUND, seed=0)


def make_tgv(n: int = 64, mach: float = 1e-1, gamma: float = 1.4) -> Workload:
    """The Taylor-Green vortex of the module docstring on an n^3 grid; Mach
    number M_s = u_0 / c_s with c_s = sqrt(gamma p_0 / rho_0)."""
    lo = (0.0, 0.0, 0.0)
    hi = (2.0 * math.pi,) * 3
    bc = (BC_PERIODIC,) * 3
    xc, yc, zc = (_centres(n, lo[d], hi[d]) for d in range(3))
    xf, yf = _faces(n, lo[0], hi[0]), _faces(n, lo[1], hi[1])
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    p0 = 1.0 / (gamma * mach * mach)
    p = p0 + (2.0 + np.cos(2.0 * Z)) * (np.cos(2.0 * X) + np.cos(2.0 * Y)) / 16.0
    rho = np.ones_like(p)
    e = p / ((gamma - 1.0) * rho)
    Zx, Yx, Xx = np.meshgrid(zc, yc, xf, indexing="ij")     # x-faces
    ux = np.sin(Xx) * np.cos(Yx) * np.cos(Zx)
    Zy, Yy, Xy = np.meshgrid(zc, yf, xc, indexing="ij")     # y-faces
    uy = -np.cos(Xy) * np.sin(Yy) * np.cos(Zy)
    uz = np.zeros_like(p)
    X0 = _pack([rho, e, ux, uy, uz])
    return Workload(name="tgv3d", ndim=3, n=(n, n, n), lo=lo, hi=hi, bc=bc, gamma=gamma, g=(0.0, 0.0, 0.0),
                    K0=0.0, chi_exp=3.0, energy_form=ENERGY_INTERNAL, X0=X0, theta=0.5, cfl_hydro=1.0,
                    n_steps=100, precond=PRECOND_SOUND, seed=0)


def config(cid: int, n: Optional[Sequence[int]] = None, mach: Optional[float] = None,
           energy_form: int = ENERGY_INTERNAL) -> Workload:
    """The five problems; `n` overrides the grid (same construction), `mach`
    selects the Mach number of problem 3."""
    if cid == 1:
        nn = tuple(n) if n is not None else (64, 64)
        return make_vortex((nn[0], nn[1], 1), 2, seed=1, mach=0.01 if mach is None else mach, cfl=10.0,
                           n_steps=5, theta=1.0, energy_form=energy_form, name="gresho2d")
    if cid == 2:
        nn = tuple(n) if n is not None else (256, 256)
        return make_stratified((nn[0], nn[1], 1), 2, seed=2, cfl=100.0, n_steps=10, n_poly=1.5,
                               contrast=10.0, blobs=8, vel_noise_mach=0.0, name="strat2d")
    if cid == 3:
        nn = tuple(n) if n is not None else (128, 128, 128)
        return make_vortex(tuple(nn), 3, seed=3, mach=0.01 if mach is None else mach, cfl=1000.0,
                           n_steps=5, theta=0.5, energy_form=energy_form, name="vortextube3d")
    if cid == 4:
        nn = tuple(n) if n is not None else (256, 256, 256)
        return make_stratified(tuple(nn), 3, seed=4, cfl=200.0, n_steps=10, n_poly=1.4,
                               contrast=20.0, blobs=0, vel_noise_mach=1e-3, name="convbox3d")
    if cid == 5:
        nn = tuple(n) if n is not None else (128, 128)
        seed = 50 if tuple(nn) == (8, 8) else 5
        return make_stratified((nn[0], nn[1], 1), 2, seed=seed, cfl=50.0, n_steps=4, n_poly=1.5,
                               contrast=10.0, blobs=8, vel_noise_mach=0.0, name="adjoint2d")
    raise ValueError(f"unknown problem {cid}")


def random_state(wl: Workload, seed: int, rel: float = 0.1, vel: float = 0.3) -> np.ndarray:
    """A rough seeded state on the workload's grid (positive rho, e; random
    velocities of magnitude ~vel * c_s; wall slots zero).  Used by property
    tests that need generic, non-smooth inputs."""
    rng = np.random.default_rng(seed)
    f = [a.copy() for a in wl.fields()]
    shape = f[0].shape
    f[0] = f[0] * (1.0 + rel * rng.uniform(-1, 1, size=shape))
    f[1] = f[1] * (1.0 + rel * rng.uniform(-1, 1, size=shape))
    cs = np.sqrt(wl.gamma * (wl.gamma - 1.0) * f[1])
    for d in range(wl.ndim):
        u = vel * cs * rng.uniform(-1, 1, size=shape)
        if wl.bc[d] == BC_WALL:
            idx = [slice(None)] * 3
            idx[2 - d] = 0
            u[tuple(idx)] = 0.0
        f[2 + d] = u
    return _pack(f)


def random_vector(wl: Workload, seed: int) -> np.ndarray:
    """A seeded random vector in the packed layout with zero wall slots."""
    rng = np.random.default_rng(seed)
    shape = (wl.n[2], wl.n[1], wl.n[0])
    f = [rng.standard_normal(size=shape) for _ in range(2 + wl.ndim)]
    for d in range(wl.ndim):
        if wl.bc[d] == BC_WALL:
            idx = [slice(None)] * 3
            idx[2 - d] = 0
            f[2 + d][tuple(idx)] = 0.0
    return _pack(f)
