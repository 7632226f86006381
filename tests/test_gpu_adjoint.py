"""Adjoint on the GPU against the oracle: the hand-written vector-Jacobian
product of the residual, the transposed Newton-system solve of one step,
and gradients through several steps via torch.autograd (8x8 version of the
adjoint problem, against central differences and the oracle's dense
reference gradient)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import adjoint as A
from oracle import discretization as D
from oracle import jfnk as J

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_03662_gb300 import build
    build.build()
    import paper_1512_03662_gb300 as jf
    return jf


def _dev(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.float64).cuda()


def _rel(a, b):
    a = a.detach().double().cpu()
    b = torch.as_tensor(b).double()
    return float((a - b).norm() / b.norm())


VJP_CASES = [(5, (8, 8), 0), (2, (16, 16), 0), (1, (16, 16), 1), (4, (8, 8, 8), 0), (3, (8, 8, 8), 1),
             (4, (12, 10, 6), 1)]


@pytest.mark.parametrize("cid,n,form", VJP_CASES)
def test_vjp_residual_parity(jf, cid, n, form):
    wl = W.config(cid, n=n)
    wl.energy_form = form
    P = D.Problem.from_workload(wl)
    X = torch.as_tensor(W.random_state(wl, 3, rel=0.05, vel=0.2))
    if form == D.ENERGY_TOTAL:
        X[P.ncell:2 * P.ncell] += 1.0
    dt = D.cfl_dt(P, X, 5.0)
    w = torch.as_tensor(W.random_vector(wl, 4))
    pow2 = all((v & (v - 1)) == 0 for v in wl.n[:wl.ndim])
    S = jf.Solver.from_workload(wl, jf.default_options(theta=wl.theta, precond=wl.precond if pow2 else 0))
    y = S.vjp_residual(_dev(X), dt, _dev(w))
    yo = A.vjp_G(P, X, dt, w)
    assert _rel(y, yo) < 1e-10, _rel(y, yo)


def _small(n=8):
    wl = W.config(5, n=(n, n))
    P = D.Problem.from_workload(wl)
    dt = D.cfl_dt(P, wl.X0, 50.0 * n / 128)
    return wl, P, dt


@pytest.mark.parametrize("n,m", [(8, 30), (16, 30), (16, 4)])
def test_step_adjoint_parity(jf, n, m):
    """The transposed solve (with restarts when m = 4) gives the oracle's
    gradients of one converged step (GMRES to 1e-10: measured 2e-11 to
    2e-10, asserted 1e-8)."""
    wl, P, dt = _small(n)
    o = jf.default_options(theta=wl.theta, precond=wl.precond, eta=1e-10, reorth=1, gmres_m=m, gmres_max_it=600)
    S = jf.Solver.from_workload(wl, o)
    Xn = _dev(wl.X0)
    X1 = Xn.clone()
    st = S.step(X1, dt, 1e-12, 1e-12)
    assert st["converged"]
    g = torch.as_tensor(W.random_vector(wl, 7))
    gXn, gK0, sta, code = S.vjp(Xn, X1, dt, _dev(g))
    assert code == 0, sta
    r = A.step_adjoint(P, wl.X0, X1.cpu(), dt, g, J.Options(precond=wl.precond, eta=1e-10, reorth=1),
                       exact=True)
    print("step adjoint n=%d m=%d: g_Xn %.3e g_K0 %.3e its %d" % (n, m, _rel(gXn, r.g_Xn), abs(gK0 / r.g_K0 - 1),
                                                                 sta["gmres_iterations_total"]))
    assert _rel(gXn, r.g_Xn) < 1e-8, _rel(gXn, r.g_Xn)
    assert gK0 == pytest.approx(r.g_K0, rel=1e-8)


def _kinetic_energy(P, X):
    """Loss: sum over unknown faces of rho_f u_f^2 / 2 dV (torch, any device)."""
    nc = P.ncell
    shp = P.shape
    rho = X[:nc].reshape(shp)
    dV = float(np.prod(P.dx[:P.ndim]))
    ke = X.new_zeros(())
    for c in range(P.ndim):
        ax = 2 - c
        rl = torch.roll(rho, 1, dims=ax)
        if P.bc[c] == D.BC_WALL:
            idx = [slice(None)] * 3
            idx[ax] = 0
            rl = rl.clone()
            rl[tuple(idx)] = rho[tuple(idx)]
        u = X[(2 + c) * nc:(3 + c) * nc].reshape(shp)
        if P.bc[c] == D.BC_WALL:
            m = torch.ones_like(u)
            idx = [slice(None)] * 3
            idx[ax] = 0
            m[tuple(idx)] = 0.0
            u = u * m
        ke = ke + 0.5 * torch.sum(0.5 * (rl + rho) * u * u) * dV
    return ke


def _initial_state(P, X0, dT):
    """Isobaric temperature perturbation 1e-4 dT of the initial state."""
    nc = P.ncell
    g1 = P.gamma - 1.0
    T = g1 * X0[nc:2 * nc]
    p = g1 * X0[:nc] * X0[nc:2 * nc]
    Tn = T * (1.0 + 1e-4 * dT)
    return torch.cat([p / Tn, Tn / g1, X0[2 * nc:]])


def test_autograd_gradient_through_four_steps(jf):
    """Loss = final kinetic energy after four implicit steps of the 8x8
    adjoint problem; gradients with respect to the initial temperature
    perturbation field and to K0 from JFNKStep.backward agree with central
    differences (1e-5) and with the oracle's dense reference (1e-8; measured
    about 1e-12)."""
    wl, P, dt = _small(8)
    o = jf.default_options(theta=wl.theta, precond=wl.precond, eta=1e-12, reorth=1)
    X0 = _dev(wl.X0)
    rng = np.random.default_rng(5)
    dT = _dev(rng.standard_normal(P.ncell)).requires_grad_(True)
    K0 = torch.tensor(wl.K0, dtype=torch.float64, device="cuda", requires_grad=True)
    S = jf.Solver.from_workload(wl, o)
    X = _initial_state(P, X0, dT)
    for _ in range(4):
        X = jf.JFNKStep.apply(X, K0, S, dt, 1e-13, 1e-12)
    loss = _kinetic_energy(P, X)
    loss.backward()
    g_dT = dT.grad.detach().cpu()
    g_K0 = float(K0.grad)

    def run(dTv, k0):
        wl2 = W.config(5, n=(8, 8))
        wl2.K0 = k0
        S2 = jf.Solver.from_workload(wl2, o)
        Xs = _initial_state(P, X0, dTv).detach().clone()
        for _ in range(4):
            st = S2.step(Xs, dt, 1e-13, 1e-12)
            assert st["converged"]
        return float(_kinetic_energy(P, Xs))

    # central differences along the gradient direction and for K0
    d = _dev(rng.standard_normal(P.ncell))
    h = 1e-2
    fd = (run(dT.detach() + h * d, wl.K0) - run(dT.detach() - h * d, wl.K0)) / (2 * h)
    ad = float(g_dT @ d.cpu())
    assert abs(ad - fd) < 1e-5 * abs(fd), (ad, fd)
    hk = 1e-4 * wl.K0
    fdk = (run(dT.detach(), wl.K0 + hk) - run(dT.detach(), wl.K0 - hk)) / (2 * hk)
    assert abs(g_K0 - fdk) < 1e-5 * abs(fdk), (g_K0, fdk)

    # dense reference: the oracle's exact transposed solves along the same trajectory
    Xc = _initial_state(P, X0, dT.detach()).cpu()
    traj = [Xc]
    Xs = Xc.clone()
    for _ in range(4):
        Xs, _ = J.newton_step(P, Xs, dt, J.Options(precond=wl.precond, newton_tol=1e-13, eta=1e-12, reorth=1))
        traj.append(Xs)
    g = A.kinetic_energy_grad(P, traj[-1])
    gk = 0.0
    for k in range(4, 0, -1):
        r = A.step_adjoint(P, traj[k - 1], traj[k], dt, g, J.Options(precond=wl.precond), exact=True)
        g, gk = r.g_Xn, gk + r.g_K0
    dTc = dT.detach().cpu().clone().requires_grad_(True)
    Xi = _initial_state(P, X0.cpu(), dTc)
    (Xi @ g).backward()
    print("adjoint vs dense: dT %.3e K0 %.3e; vs FD: dT %.3e K0 %.3e" % (
        _rel(g_dT, dTc.grad), abs(g_K0 / gk - 1), abs(ad / fd - 1), abs(g_K0 / fdk - 1)))
    assert _rel(g_dT, dTc.grad) < 1e-8, _rel(g_dT, dTc.grad)
    assert g_K0 == pytest.approx(gk, rel=1e-8)


def test_vjp_rejects_mixed_precision_handles(jf):
    wl, P, dt = _small(8)
    S = jf.Solver.from_workload(wl, jf.default_options(theta=wl.theta, precond=wl.precond, precision=jf.MIXED))
    X = _dev(wl.X0)
    with pytest.raises(jf.JFNKError) as e:
        S.vjp(X, X, dt, X)
    assert e.value.status == jf.JFNK_EINVAL


def test_vjp_residual_rejects_mixed_precision_handles(jf):
    """Mixed handles reserve no adjoint scratch, so the transposed product
    is refused there too."""
    wl, P, dt = _small(8)
    S = jf.Solver.from_workload(wl, jf.default_options(theta=wl.theta, precond=wl.precond, precision=jf.MIXED))
    X = _dev(wl.X0)
    with pytest.raises(jf.JFNKError) as e:
        S.vjp_residual(X, dt, X)
    assert e.value.status == jf.JFNK_EINVAL


@pytest.mark.parametrize("cid,n", [(4, (64, 64, 64)), (2, (256, 256))])
def test_vjp_residual_run_to_run_spread(jf, cid, n):
    """The reverse kernels scatter with FP64 atomic adds, whose order varies
    between runs: J^T w is reproducible to round-off, not bitwise.  Five
    calls on the same input differ from the first by a few units of
    rounding of the largest terms per entry (the spread is printed), at
    most 1e-13 normwise, and every call agrees with the oracle."""
    wl = W.config(cid, n=n)
    P = D.Problem.from_workload(wl)
    X = torch.as_tensor(W.random_state(wl, 3, rel=0.05, vel=0.2))
    dt = D.cfl_dt(P, X, 5.0)
    w = torch.as_tensor(W.random_vector(wl, 4))
    S = jf.Solver.from_workload(wl, jf.default_options(theta=wl.theta, precond=wl.precond))
    Xg, wg = _dev(X), _dev(w)
    ys = [S.vjp_residual(Xg, dt, wg).clone() for _ in range(5)]
    spread = max(float((y - ys[0]).norm() / ys[0].norm()) for y in ys[1:])
    differ = sum(int((y != ys[0]).sum()) for y in ys[1:])
    print("J^T w run-to-run, problem %d %s: normwise spread %.2e, %d of %d entries differ" % (
        cid, n, spread, differ, 4 * ys[0].numel()))
    assert spread < 1e-13, spread
    assert _rel(ys[-1], A.vjp_G(P, X, dt, w)) < 1e-10
