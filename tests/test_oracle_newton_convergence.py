"""Why Newton converges linearly on the convective box (problem 4), measured
on the oracle at 16^3 with the benchmark's time step: the finite-difference
Jacobian of Eqs. jacobian_free / pert_old is too inaccurate for the late
Newton iterations at lambda = 1e-7, not the limiter or upwind kinks.

With R_u = max(|u|, alpha2 c_s) = c_s (rms Mach 1e-3, alpha2 = 1) the
perturbation delta R w moves the face velocities by about 1e3 times more,
relative to the velocities themselves, than the scaled perturbation
suggests; the first-order truncation error of the quotient is then 1e-2 to
3e-1 of the linear residual in the directions the late Newton corrections
take.  The checks: (1) with the exact directional derivative (forward-mode
differentiation of G) each linear solve reaches the GMRES tolerance in the
true linear residual and Newton converges superlinearly; (2) with the
quotient at lambda = 1e-7 the true linear residual of the late solves stays
far above the tolerance GMRES reports, and the nonlinear residual falls by
the same factor; (3) at lambda = 1e-9 the quotient behaves like the exact
derivative; (4) no limiter or upwind branch of the face velocities flips
between X and X + delta R z at lambda <= 1e-7, so the kinks are not the
cause."""
import pytest
import torch

import workloads as W
from oracle import discretization as D
from oracle import jfnk as J
from oracle import precond as PC


def _problem4(n=16):
    wl = W.config(4, n=(n, n, n))
    wl.cfl_hydro = 200.0 * n / 256.0          # the 256^3 workload's time step
    P = D.Problem.from_workload(wl)
    X0 = torch.as_tensor(wl.X0)
    return wl, P, X0, D.cfl_dt(P, X0, wl.cfl_hydro)


def _newton(P, X0, dt, lam, exact, precond, iters=6):
    """Newton iterations of the oracle with one V(1,1) cycle per apply;
    per iteration the true relative linear residual |F^ + J^ dx| / |F^|
    (exact derivative) and the nonlinear reduction |F^(k+1)| / |F^(k)|."""
    opts = J.Options(precond=precond, lam=lam, mg_cycles=1, mg_nu1=1, mg_nu2=1)
    bn = D.bn_constant(P, X0, dt)
    X = X0.clone()
    out = []
    G = lambda x: D.G_operator(P, x, dt)                   # noqa: E731
    for _ in range(iters):
        sc = J.scaling(P, X, opts)
        G0 = G(X)
        Fhat = (G0 - bn) / sc.L
        si = PC.setup(P, X, dt, opts)
        if exact:
            A = lambda z, X=X, sc=sc: torch.func.jvp(G, (X,), (sc.R * z,))[1] / sc.L    # noqa: E731
        else:
            A = lambda z, X=X, sc=sc, G0=G0: J.jv(P, X, G0, sc, z, dt, opts)[0]          # noqa: E731
        dxh, _ = J.gmres(A, lambda v: PC.apply(si, v, sc), -Fhat, opts.eta, 30, 300)
        jt = torch.func.jvp(G, (X,), (sc.R * dxh,))[1] / sc.L
        lin = float((Fhat + jt).norm() / Fhat.norm())
        X = X + sc.R * dxh
        red = float(((G(X) - bn) / sc.L).norm() / Fhat.norm())
        out.append((lin, red, float(dxh.abs().max())))
    return out


@pytest.mark.slow
def test_late_newton_iterations_are_limited_by_the_finite_difference_jacobian():
    wl, P, X0, dt = _problem4()
    ex = _newton(P, X0, dt, 1e-7, True, wl.precond)
    fd7 = _newton(P, X0, dt, 1e-7, False, wl.precond)
    fd9 = _newton(P, X0, dt, 1e-9, False, wl.precond)
    # iterations 0-3 take the state from X^n to |dx| ~ 4e-5; from iteration 4
    # on the corrections are below 1e-6 of the scales
    for k in (4, 5):
        assert ex[k][0] < 2e-4, ex              # the linear solve meets eta = 1e-4 in truth
        assert fd9[k][0] < 2e-4, fd9
        assert fd7[k][0] > 5e-3, fd7            # the FD Jacobian leaves 1e-2 .. 3e-1
        assert fd7[k][1] > 5e-3, fd7            # and Newton reduces |F^| only that much
    # superlinear with an accurate Jacobian: iteration 4 gains four orders
    assert ex[4][1] < 1e-3 and fd9[4][1] < 1e-3, (ex[4], fd9[4])
    # the Newton stop rule |dx|_inf < 1e-8 is met at iteration 5 with the
    # accurate Jacobians, not with lambda = 1e-7
    assert ex[5][2] < 1e-8 and fd9[5][2] < 1e-8 and fd7[5][2] > 1e-8, (ex[5], fd9[5], fd7[5])


def _branch_flips(P, Xa, Xb):
    """Face velocities whose upwind sign or van Leer limiter branch (a b > 0
    along any direction) differs between states Xa and Xb."""
    fa, fb = D.unpack(P, Xa), D.unpack(P, Xb)
    up = lim = 0
    for c in range(P.ndim):
        ua, ub = fa[2 + c], fb[2 + c]
        up += int(((ua >= 0) != (ub >= 0)).sum())
        for d in range(P.ndim):
            ax = D.axis(d)
            sa = (ua - torch.roll(ua, 1, ax)) * (torch.roll(ua, -1, ax) - ua) > 0
            sb = (ub - torch.roll(ub, 1, ax)) * (torch.roll(ub, -1, ax) - ub) > 0
            lim += int((sa != sb).sum())
    return up, lim


@pytest.mark.slow
def test_finite_difference_perturbation_crosses_no_kink_at_the_working_lambda():
    """At a converged step, the perturbation of one Jacobian-free product
    along a preconditioned Krylov direction flips no upwind or limiter
    branch for lambda <= 1e-7, and the quotient's error against the exact
    derivative falls in proportion to lambda (truncation) until round-off
    takes over below lambda = 1e-8."""
    wl, P, X0, dt = _problem4()
    opts = J.Options(precond=wl.precond, mg_cycles=1, mg_nu1=1, mg_nu2=1)
    X, st = J.newton_step(P, X0, dt, opts)
    assert st.converged
    sc = J.scaling(P, X, opts)
    G0 = D.G_operator(P, X, dt)
    v = torch.as_tensor(W.random_vector(wl, 3))
    z = PC.apply(PC.setup(P, X, dt, opts), v / v.norm(), sc)
    exact = torch.func.jvp(lambda x: D.G_operator(P, x, dt), (X,), (sc.R * z,))[1] / sc.L
    err = {}
    for lam in (1e-6, 1e-7, 1e-8):
        o = J.Options(lam=lam)
        fd, delta = J.jv(P, X, G0, sc, z, dt, o)
        err[lam] = float((fd - exact).norm() / exact.norm())
        if lam <= 1e-7:
            assert _branch_flips(P, X, X + delta * sc.R * z) == (0, 0)
    assert 5.0 < err[1e-6] / err[1e-7] < 20.0, err
    assert 5.0 < err[1e-7] / err[1e-8] < 20.0, err
