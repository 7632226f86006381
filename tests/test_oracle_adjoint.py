"""Pins of the oracle's adjoint: transposed Jacobian products against finite
differences (dot-product test), the transposed GMRES solve against a dense
solve, and step gradients against central differences of full Newton steps
(8x8 stratified problem, as in the adjoint workload)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import adjoint as A
from oracle import discretization as D
from oracle import jfnk as J


def _small(seed=50):
    """8x8 version of the adjoint problem with the time step of the 128^2
    one (CFL scaled by 8/128): at CFL 50 an 8x8 grid would take a 16x longer
    step."""
    wl = W.config(5, n=(8, 8))
    P = D.Problem.from_workload(wl)
    dt = D.cfl_dt(P, wl.X0, 50.0 * 8 / 128)
    return wl, P, dt


def test_vjp_passes_the_dot_product_test_against_finite_differences():
    """w . (J v) with J v from central differences of G equals (J^T w) . v."""
    wl, P, dt = _small()
    X = torch.as_tensor(W.random_state(wl, 3, rel=0.05, vel=0.2))
    rng = np.random.default_rng(0)
    for k in range(3):
        v = torch.as_tensor(W.random_vector(wl, 10 + k)) * X.abs().clamp(min=1e-3) * 1e-3
        w = torch.as_tensor(W.random_vector(wl, 20 + k))
        h = 1e-4
        Jv = (D.G_operator(P, X + h * v, dt) - D.G_operator(P, X - h * v, dt)) / (2 * h)
        lhs = float(w @ Jv)
        rhs = float(A.vjp_G(P, X, dt, w) @ v)
        assert abs(lhs - rhs) < 1e-7 * abs(lhs), (lhs, rhs)
        Jb = (D.bn_constant(P, X + h * v, dt) - D.bn_constant(P, X - h * v, dt)) / (2 * h)
        assert abs(float(w @ Jb) - float(A.vjp_bn(P, X, dt, w) @ v)) < 1e-7 * abs(float(w @ Jb))


def test_dR_dK0_is_the_conduction_term():
    wl, P, dt = _small()
    X = torch.as_tensor(W.random_state(wl, 4, rel=0.05, vel=0.2))
    w = torch.as_tensor(W.random_vector(wl, 5))
    P0 = D.Problem.from_workload(wl)
    P0.K0 = 0.0
    cond = D.pack(D.rhs(P, X)) - D.pack(D.rhs(P0, X))          # K0 * dR/dK0
    assert A.dR_dK0_dot(P, X, w) == pytest.approx(float(w @ cond) / P.K0, rel=1e-10)


def test_transposed_gmres_matches_a_dense_solve():
    wl, P, dt = _small()
    X0 = torch.as_tensor(wl.X0)
    X1, st = J.newton_step(P, X0, dt, J.Options(precond=2, newton_tol=1e-12))
    assert st.converged
    g = torch.as_tensor(W.random_vector(wl, 7))
    o = J.Options(precond=2, eta=1e-12, reorth=1)
    r1 = A.step_adjoint(P, X0, X1, dt, g, o)
    r0 = A.step_adjoint(P, X0, X1, dt, g, o, exact=True)
    assert r1.converged
    assert float((r1.lam - r0.lam).norm() / r0.lam.norm()) < 1e-8
    assert float((r1.g_Xn - r0.g_Xn).norm() / r0.g_Xn.norm()) < 1e-8
    assert r1.g_K0 == pytest.approx(r0.g_K0, rel=1e-8)


def _run(P, X0, dt, nsteps, K0=None):
    Q = P if K0 is None else D.Problem(**{**P.__dict__, "K0": K0})
    X = X0
    traj = [X]
    for _ in range(nsteps):
        X, st = J.newton_step(Q, X, dt, J.Options(precond=2, newton_tol=1e-13, eta=1e-12, reorth=1))
        assert st.converged
        traj.append(X)
    return traj


def test_step_gradients_match_central_differences():
    """Four steps of the 8x8 stratified problem; loss = final kinetic energy;
    gradients with respect to the initial state (along a temperature-like
    direction) and to K0 agree with central differences to 1e-5."""
    wl, P, dt = _small()
    X0 = torch.as_tensor(wl.X0)
    n = 4
    traj = _run(P, X0, dt, n)
    g = A.kinetic_energy_grad(P, traj[-1])
    gK0 = 0.0
    o = J.Options(precond=2, eta=1e-12, reorth=1)
    for k in range(n, 0, -1):
        r = A.step_adjoint(P, traj[k - 1], traj[k], dt, g, o)
        gK0 += r.g_K0
        g = r.g_Xn
    # direction: isobaric temperature perturbation of the initial state
    rng = np.random.default_rng(5)
    dT = torch.as_tensor(rng.standard_normal(P.shape)).reshape(-1)
    f = D.unpack(P, X0)
    T = (P.gamma - 1) * f[1].reshape(-1)
    p = (P.gamma - 1) * f[0].reshape(-1) * f[1].reshape(-1)

    def state(eps):
        Tn = T * (1 + eps * 1e-4 * dT)
        rho = p / Tn
        e = Tn / (P.gamma - 1)
        return torch.cat([rho, e, X0[2 * P.ncell:]])

    h = 1e-3
    Lp = float(A.kinetic_energy(P, _run(P, state(h), dt, n)[-1]))
    Lm = float(A.kinetic_energy(P, _run(P, state(-h), dt, n)[-1]))
    fd = (Lp - Lm) / (2 * h)
    dX = (state(1e-6) - state(-1e-6)) / 2e-6
    ad = float(g @ dX)
    assert abs(ad - fd) < 1e-5 * abs(fd), (ad, fd)
    hk = 1e-4 * P.K0
    Lp = float(A.kinetic_energy(P, _run(P, X0, dt, n, K0=P.K0 + hk)[-1]))
    Lm = float(A.kinetic_energy(P, _run(P, X0, dt, n, K0=P.K0 - hk)[-1]))
    fdk = (Lp - Lm) / (2 * hk)
    assert abs(gK0 - fdk) < 1e-5 * abs(fdk), (gK0, fdk)
