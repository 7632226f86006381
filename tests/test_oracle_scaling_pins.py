"""Pins of the oracle's Newton scaling (paper Sect. 4.2, Eq.
jacobian_system_norm) and of the finite-difference perturbation size (Sect.
4.3, Eqs. pert_old and pert_new) against values worked out by hand.

The states are 4x4 grids with gamma = 5/3, so c_s^2 = gamma (gamma - 1) e =
10 e / 9 and e = 0.9, 3.6, 8.1, 14.4 give c_s = 1, 2, 3, 4 exactly.  Every
expected number below was derived on paper from the equation:

    L_rho = rho,  L_e = rho e,  L_u = rho_f max(|u|, alpha1 c_s,f)
    R_rho = rho,  R_e = e,      R_u = max(|u|, alpha2 c_s,f)

with the face values rho_f, c_s,f the means of the two cells beside the face,
L = R = 1 on a wall-face slot, and in the total-energy form L_E = rho eps_t,
R_E = eps_t (c_s from e = eps_t - sum_d (u_lo^2 + u_hi^2) / 4).  A swapped
alpha1/alpha2, a cell-centred sound speed, L_E = eps_t or R_u without the
max would each change at least one of them.
"""
import math

import pytest
import torch

from oracle import discretization as D
from oracle import jfnk as J

GAMMA = 5.0 / 3.0


def _problem(bc_y, form=D.ENERGY_INTERNAL):
    return D.Problem(ndim=2, n=(4, 4, 1), dx=(0.25, 0.25, 1.0), bc=(D.BC_PERIODIC, bc_y, D.BC_PERIODIC),
                     gamma=GAMMA, g=(0.0, 0.0, 0.0), K0=0.0, chi_exp=3.0, energy_form=form, theta=0.5)


def _rows(vals):
    """A 4x4 field (x fastest) whose row j (the y index) holds vals[j]."""
    return torch.tensor([v for v in vals for _ in range(4)], dtype=torch.float64)


def _state(rho, E, ux, uy):
    return torch.cat([_rows(rho), _rows(E), _rows(ux), _rows(uy)])


def _check(sc, L, R, xhat_sq):
    assert torch.allclose(sc.L, torch.cat([_rows(v) for v in L]), rtol=1e-15, atol=0.0), (sc.L, L)
    assert torch.allclose(sc.R, torch.cat([_rows(v) for v in R]), rtol=1e-15, atol=0.0), (sc.R, R)
    assert sc.xhat_norm == pytest.approx(math.sqrt(xhat_sq), rel=1e-15)


@pytest.mark.parametrize("a1,a2", [(1e-5, 1.0), (1.0, 1.0), (1e-5, 0.5), (1.0, 0.5)])
def test_scaling_uniform_gas_at_rest_with_walls(a1, a2):
    """rho = 2, e = 0.9 (c_s = 1), u = 0, walls in y: the velocity scales are
    the floors alpha c_s; the wall-face row of u_y gets L = R = 1."""
    P = _problem(D.BC_WALL)
    X = _state([2] * 4, [0.9] * 4, [0] * 4, [0] * 4)
    sc = J.scaling(P, X, J.Options(alpha1=a1, alpha2=a2))
    L = [[2] * 4, [1.8] * 4, [2 * a1] * 4, [1, 2 * a1, 2 * a1, 2 * a1]]
    R = [[2] * 4, [0.9] * 4, [a2] * 4, [1, a2, a2, a2]]
    _check(sc, L, R, 32.0)          # rho/R_rho = e/R_e = 1 on 32 slots, u = 0


@pytest.mark.parametrize("form", [D.ENERGY_INTERNAL, D.ENERGY_TOTAL])
@pytest.mark.parametrize("a1,a2", [(1e-5, 1.0), (1.0, 0.5)])
def test_scaling_uniform_moving_gas(form, a1, a2):
    """rho = 2, e = 0.9 (c_s = 1), u_x = 0.5, u_y = -3, doubly periodic.
    Total energy: eps_t = 0.9 + (0.5^2 + 3^2) / 2 = 5.525."""
    P = _problem(D.BC_PERIODIC, form)
    E = 0.9 if form == D.ENERGY_INTERNAL else 5.525
    X = _state([2] * 4, [E] * 4, [0.5] * 4, [-3] * 4)
    sc = J.scaling(P, X, J.Options(alpha1=a1, alpha2=a2))
    if (a1, a2) == (1e-5, 1.0):
        Lux, Rux = 1.0, 1.0         # 2 max(0.5, 1e-5), max(0.5, 1)
        xhat_sq = 16 * (1 + 1 + 0.25 + 1)
    else:
        Lux, Rux = 2.0, 0.5         # 2 max(0.5, 1), max(0.5, 0.5)
        xhat_sq = 16 * (1 + 1 + 1 + 1)
    L = [[2] * 4, [2 * E] * 4, [Lux] * 4, [6] * 4]     # L_uy = 2 max(3, a1)
    R = [[2] * 4, [E] * 4, [Rux] * 4, [3] * 4]         # R_uy = max(3, a2)
    _check(sc, L, R, xhat_sq)


# Stratified 4x4, walls in y.  Rows j = 0..3 (bottom to top):
#   rho = 1, 2, 4, 8;  e = 0.9, 3.6, 8.1, 14.4  ->  c_s = 1, 2, 3, 4
#   u_x (uniform along each row) = 0, 3, -0.5, 10
#   u_y on the faces below each row = wall (0), 0.2, -4, 1
# y faces j = 1, 2, 3: rho_f = 1.5, 3, 6 and c_s,f = 1.5, 2.5, 3.5.
# x faces lie inside one row: rho_f = rho_j and c_s,f = c_s,j.
STRAT = dict(rho=[1, 2, 4, 8], e=[0.9, 3.6, 8.1, 14.4], ux=[0, 3, -0.5, 10], uy=[0, 0.2, -4, 1])
# expected velocity scales per (alpha1, alpha2): (L_ux, R_ux, L_uy, R_uy) per row
STRAT_U = {
    (1e-5, 1.0): ([1e-5, 6, 2, 80], [1, 3, 3, 10], [1, 0.3, 12, 6], [1, 1.5, 4, 3.5]),
    (1.0, 1.0): ([1, 6, 12, 80], [1, 3, 3, 10], [1, 2.25, 12, 21], [1, 1.5, 4, 3.5]),
    (1e-5, 0.5): ([1e-5, 6, 2, 80], [0.5, 3, 1.5, 10], [1, 0.3, 12, 6], [1, 0.75, 4, 1.75]),
    (1.0, 0.5): ([1, 6, 12, 80], [0.5, 3, 1.5, 10], [1, 2.25, 12, 21], [1, 0.75, 4, 1.75]),
}


def _xhat_sq(Rux, Ruy, nE):
    """||R^-1 X||^2 of the stratified state: 16 unit rho entries, nE energy
    entries (all 1) and the velocity ratios row by row."""
    s = 16.0 + nE
    for u, r in zip(STRAT["ux"], Rux):
        s += 4 * (u / r) ** 2
    for u, r in zip(STRAT["uy"], Ruy):
        s += 4 * (u / r) ** 2
    return s


@pytest.mark.parametrize("a", sorted(STRAT_U))
def test_scaling_stratified_with_walls_internal_energy(a):
    P = _problem(D.BC_WALL)
    X = _state(STRAT["rho"], STRAT["e"], STRAT["ux"], STRAT["uy"])
    sc = J.scaling(P, X, J.Options(alpha1=a[0], alpha2=a[1]))
    Lux, Rux, Luy, Ruy = STRAT_U[a]
    L = [STRAT["rho"], [0.9, 7.2, 32.4, 115.2], Lux, Luy]
    R = [STRAT["rho"], STRAT["e"], Rux, Ruy]
    _check(sc, L, R, _xhat_sq(Rux, Ruy, 16))


@pytest.mark.parametrize("a", [(1e-5, 1.0), (1.0, 0.5)])
def test_scaling_stratified_with_walls_total_energy(a):
    """Cell kinetic energies sum_d (u_lo^2 + u_hi^2)/4 per row: x gives u_x^2/2
    = 0, 4.5, 0.125, 50; y gives (0 + 0.04)/4, (0.04 + 16)/4, (16 + 1)/4,
    (1 + 0)/4 = 0.01, 4.01, 4.25, 0.25 (top and bottom faces are walls).
    eps_t = e + KE = 0.91, 12.11, 12.475, 64.65; the sound speed comes from e,
    so the velocity scales are those of the internal-energy form."""
    P = _problem(D.BC_WALL, D.ENERGY_TOTAL)
    eps = [0.91, 12.11, 12.475, 64.65]
    X = _state(STRAT["rho"], eps, STRAT["ux"], STRAT["uy"])
    sc = J.scaling(P, X, J.Options(alpha1=a[0], alpha2=a[1]))
    Lux, Rux, Luy, Ruy = STRAT_U[a]
    L = [STRAT["rho"], [0.91, 24.22, 49.9, 517.2], Lux, Luy]
    R = [STRAT["rho"], eps, Rux, Ruy]
    assert torch.allclose(sc.L, torch.cat([_rows(v) for v in L]), rtol=1e-14, atol=0.0)
    assert torch.allclose(sc.R, torch.cat([_rows(v) for v in R]), rtol=1e-14, atol=0.0)
    assert sc.xhat_norm == pytest.approx(math.sqrt(_xhat_sq(Rux, Ruy, 16)), rel=1e-14)


# ---------------------------------------------------------------------------
# perturbation size (Eqs. pert_old and pert_new)
# ---------------------------------------------------------------------------

def _moving():
    """Uniform moving gas with alpha2 = 1/2: x^ = R^-1 X is +1 on the rho,
    e and u_x slots and -1 on the u_y slots, so ||x^|| = 8."""
    P = _problem(D.BC_PERIODIC)
    X = _state([2] * 4, [0.9] * 4, [0.5] * 4, [-3] * 4)
    return P, X


def _w(**blocks):
    """A vector that is 0.5 on the named blocks (rho, e, ux, uy) and 0 elsewhere."""
    w = torch.zeros(64, dtype=torch.float64)
    for k, name in enumerate(("rho", "e", "ux", "uy")):
        if blocks.get(name):
            w[16 * k:16 * (k + 1)] = 0.5
    return w


def test_pert_old_by_hand():
    """||x^|| = 8, ||w|| = 2 (16 entries of 0.5): delta = lambda (lambda + 4)."""
    P, X = _moving()
    o = J.Options(alpha1=1.0, alpha2=0.5, lam=1e-7)
    sc = J.scaling(P, X, o)
    assert sc.xhat_norm == 8.0
    assert J.perturbation(o, sc, X, _w(rho=1)) == pytest.approx(4.0000001e-7, rel=1e-15)
    o.lam = 1e-4
    # ||w|| = 4 (64 entries of 0.5): delta = 1e-4 (1e-4 + 2)
    assert J.perturbation(o, sc, X, _w(rho=1, e=1, ux=1, uy=1)) == pytest.approx(2.0001e-4, rel=1e-15)


def test_pert_new_by_hand():
    """x^.w = +8, -8 or 0 with w.w = 4: delta = lambda (1e-12/lambda + 2)
    with the sign of x^.w, and 1e-12 when x^.w = 0 (sign(0) read as +1)."""
    P, X = _moving()
    o = J.Options(alpha1=1.0, alpha2=0.5, lam=1e-6, pert=J.PERT_NEW)
    sc = J.scaling(P, X, o)
    assert J.perturbation(o, sc, X, _w(rho=1)) == pytest.approx(2.000001e-6, rel=1e-15)
    assert J.perturbation(o, sc, X, _w(uy=1)) == pytest.approx(-2.000001e-6, rel=1e-15)
    # w.w = 8, x^.w = 8 - 8 = 0
    assert J.perturbation(o, sc, X, _w(rho=1, uy=1)) == pytest.approx(1e-12, rel=1e-15)
    # w.w = 8, x^.w = 8 + 8: lambda (1e-12/lambda + 16/8)
    assert J.perturbation(o, sc, X, _w(rho=1, ux=1)) == pytest.approx(2.000001e-6, rel=1e-15)
