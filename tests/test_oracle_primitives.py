"""Pins of the oracle's building blocks against properties the definitions
fix (van Leer's harmonic limiter, the upwind choice of Sect. 2, the ideal-gas
EOS and sound speed, the conductivity law, the CFL time step), so that a
mistake in one of them (a swapped operand, a wrong tie rule, a dropped
factor) fails here and not only through the residual's consistency pins."""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import discretization as D


def _t(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64))


def test_vanleer_slope_is_zero_at_extrema_and_sign_changes():
    a = _t([1.0, -2.0, 0.0, 3.0, 0.0, -1e-300])
    b = _t([-1.0, 3.0, 5.0, 0.0, 0.0, 1e-300])
    assert torch.all(D.vanleer_slope(a, b) == 0.0)


def test_vanleer_slope_bounds_symmetry_and_linear_exactness():
    """For ab > 0 the harmonic slope lies between min(|a|,|b|) and
    2 min(|a|,|b|) (the TVD bound), is symmetric in (a, b), odd under a sign
    flip of both, and equals a when a = b (linear data are reconstructed
    exactly)."""
    rng = np.random.default_rng(0)
    a = _t(rng.uniform(0.01, 10.0, 2000) * rng.choice([-1.0, 1.0], 2000))
    b = a.sign() * _t(rng.uniform(0.01, 10.0, 2000))
    s = D.vanleer_slope(a, b)
    m = torch.minimum(a.abs(), b.abs())
    assert torch.all(s.abs() >= m * (1 - 1e-15)) and torch.all(s.abs() <= 2 * m * (1 + 1e-15))
    assert torch.all(s.sign() == a.sign())
    assert torch.equal(s, D.vanleer_slope(b, a))
    assert torch.equal(-s, D.vanleer_slope(-a, -b))
    assert torch.allclose(D.vanleer_slope(a, a), a, rtol=1e-15, atol=0)


def test_slope_of_a_linear_profile_and_at_an_extremum():
    # along x (the last axis): q = 3 i is linear -> slope 3 away from the
    # wrap-around ends; a peak at i = 4 -> zero slope there
    q = _t(np.arange(10, dtype=np.float64) * 3.0).reshape(1, 1, 10)
    s = D.slope(q, 0)
    assert torch.allclose(s[0, 0, 1:-1], _t(np.full(8, 3.0)))
    peak = _t([0, 1, 2, 3, 5, 3, 2, 1, 0, 0]).reshape(1, 1, 10)
    assert float(D.slope(peak, 0)[0, 0, 4]) == 0.0


def test_upwind_takes_the_lower_cell_for_non_negative_speed():
    """Face i (lower face of cell i) takes q_{i-1} + s_{i-1}/2 when the speed
    is >= 0 (ties go to the lower side) and q_i - s_i/2 when it is < 0."""
    q = _t([1.0, 2.0, 4.0, 8.0]).reshape(1, 1, 4)
    s = _t([0.5, 1.0, 2.0, 4.0]).reshape(1, 1, 4)
    speed = _t([0.0, 0.0, -1.0, 2.0]).reshape(1, 1, 4)
    v = D.upwind(q, s, speed, 0)[0, 0]
    assert float(v[1]) == 1.0 + 0.25          # speed 0: lower cell 0
    assert float(v[2]) == 4.0 - 1.0           # speed < 0: this cell
    assert float(v[3]) == 4.0 + 1.0           # speed > 0: lower cell 2


def test_ideal_gas_eos_sound_speed_and_conductivity():
    wl = W.config(4, n=(8, 8, 8))
    P = D.Problem.from_workload(wl)
    rho, e = _t([1.3]), _t([2.0])
    g = P.gamma
    p = D.pressure(P, rho, e)
    assert float(p) == pytest.approx((g - 1.0) * 1.3 * 2.0, rel=1e-15)
    # c_s^2 = gamma p / rho for an ideal gas
    assert float(D.sound_speed(P, e)) ** 2 == pytest.approx(g * float(p) / 1.3, rel=1e-14)
    T = _t([0.7])
    assert float(D.conductivity(P, T)) == pytest.approx(P.K0 * 0.7 ** 3, rel=1e-15)


def test_cfl_time_step_of_a_uniform_state():
    """A uniform gas moving at velocity u in x: dt = CFL dx / (|u| + c_s)."""
    wl = W.config(1, n=(16, 16))
    P = D.Problem.from_workload(wl)
    nc = P.ncell
    X = torch.zeros(P.nfield * nc, dtype=torch.float64)
    X[:nc] = 1.0
    X[nc:2 * nc] = 3.0
    X[2 * nc:3 * nc] = 0.25
    cs = math.sqrt(P.gamma * (P.gamma - 1.0) * 3.0)
    hmin = min(P.dx[d] for d in range(P.ndim))
    assert D.cfl_dt(P, X, 10.0) == pytest.approx(10.0 * hmin / (0.25 + cs), rel=1e-14)
