"""Pins of the oracle's Newton-Krylov layer and preconditioner (paper Sects.
3.2-4.3) against exact derivatives, dense brute-force Jacobians, direct solves
and the algebra of the semi-implicit scheme."""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import discretization as D
from oracle import jfnk as J
from oracle import precond as PC


def _setup(cid, n, seed=7, rel=0.05, vel=0.2, cfl=10.0, form=0, **optkw):
    wl = W.config(cid, n=n)
    P = D.Problem.from_workload(wl)
    P.energy_form = form
    X = torch.as_tensor(W.random_state(wl, seed, rel=rel, vel=vel))
    if form == D.ENERGY_TOTAL:
        X = X.clone()
        X[P.ncell:2 * P.ncell] += 1.0                       # keep e = eps - ke positive
    dt = D.cfl_dt(P, X, cfl)
    opts = J.Options(precond=wl.precond, **optkw)
    return wl, P, X, dt, opts


# ---------------------------------------------------------------------------
# Jacobian-vector product (Eqs. jacobian_free, pert_old, pert_new)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("cid,n,form", [(1, (16, 16), 0), (2, (16, 16), 1), (4, (8, 8, 8), 0)])
def test_fd_jv_matches_exact_derivative(cid, n, form):
    """The scaled FD quotient equals L^-1 (dG/dX) R w to O(delta): the exact
    directional derivative comes from forward-mode differentiation of G."""
    wl, P, X, dt, opts = _setup(cid, n, form=form)
    sc = J.scaling(P, X, opts)
    G0 = D.G_operator(P, X, dt)
    w = torch.as_tensor(W.random_vector(wl, 3))
    Jw, delta = J.jv(P, X, G0, sc, w, dt, opts)
    _, jt = torch.func.jvp(lambda x: D.G_operator(P, x, dt), (X,), (sc.R * w,))
    exact = jt / sc.L
    assert delta == pytest.approx(opts.lam * (opts.lam + sc.xhat_norm / float(w.norm())), rel=1e-15)
    assert float((Jw - exact).norm() / exact.norm()) < 2e-5
    # a larger perturbation is proportionally less accurate (first-order FD)
    opts2 = J.Options(lam=1e-4)
    Jw2, _ = J.jv(P, X, G0, sc, w, dt, opts2)
    e1 = float((Jw - exact).norm())
    e2 = float((Jw2 - exact).norm())
    assert e2 > 30 * e1


def test_pert_new_formula():
    wl, P, X, dt, opts = _setup(1, (16, 16))
    sc = J.scaling(P, X, opts)
    w = torch.as_tensor(W.random_vector(wl, 4))
    o = J.Options(pert=J.PERT_NEW, lam=1e-6)
    d = J.perturbation(o, sc, X, w)
    xhat = X / sc.R
    uv = float(xhat @ w)
    assert d == pytest.approx(1e-6 * (1e-12 / 1e-6 + abs(uv) / float(w @ w)) * math.copysign(1, uv), rel=1e-14)


def test_dense_bruteforce_jacobian_8x8():
    """On 8x8, every column of the scaled Jacobian from central differences
    of F_U matches J^ e_j (FD Jv) and the exact derivative."""
    wl, P, X, dt, opts = _setup(5, (8, 8), cfl=5.0)
    Xn = X.clone()
    X = X + 1e-3 * torch.as_tensor(W.random_vector(wl, 9)) * X.abs()
    X = torch.as_tensor(np.where(np.asarray(D.unpack(P, X)[0].numpy()).size > 0, X.numpy(), X.numpy()))
    sc = J.scaling(P, X, opts)
    G0 = D.G_operator(P, X, dt)
    N = X.numel()
    masks = torch.cat([torch.ones(2 * P.ncell)] + [D.wall_slot_mask(P, c).reshape(-1) for c in range(P.ndim)])
    Jd = torch.zeros(N, N, dtype=torch.float64)
    h = 1e-6
    for j in range(N):
        if masks[j] == 0:
            continue
        ej = torch.zeros(N, dtype=torch.float64)
        ej[j] = 1.0
        Fp = D.residual(P, X + h * sc.R * ej, Xn, dt)
        Fm = D.residual(P, X - h * sc.R * ej, Xn, dt)
        Jd[:, j] = (Fp - Fm) / (2 * h) / sc.L
    Jex = torch.func.jacrev(lambda x: D.G_operator(P, x, dt))(X) * sc.R[None, :] / sc.L[:, None]
    Jex = Jex * masks[None, :]
    assert float((Jd - Jex).norm() / Jex.norm()) < 1e-7
    rng = np.random.default_rng(0)
    for j in rng.choice(np.nonzero(masks.numpy())[0], 12, replace=False):
        ej = torch.zeros(N, dtype=torch.float64)
        ej[j] = 1.0
        col, _ = J.jv(P, X, G0, sc, ej, dt, opts)
        assert float((col - Jd[:, j]).norm() / Jd[:, j].norm()) < 1e-5


# ---------------------------------------------------------------------------
# transformations (Sect. 3.2, App. B)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("form", [0, 1])
def test_transformations_match_the_eos_maps(form):
    """dV/dU applied to U(X+dX)-U(X) gives V(X+dX)-V(X), and dX/dV maps it
    back to dX, to second order in |dX| (V = (p, e, u))."""
    wl, P, X, dt, opts = _setup(4, (8, 8, 8), form=form, cfl=5.0)
    opts.precond = PC.SOUND
    si = PC.setup(P, X, dt, opts)
    dX0 = torch.as_tensor(W.random_vector(wl, 21)) * torch.cat(
        [X[:2 * P.ncell].abs(), torch.full((P.ndim * P.ncell,), 0.1, dtype=torch.float64)])

    def V(x):
        e = D.internal_energy(P, x)
        f = D.unpack(P, x)
        return D.pressure(P, f[0], e), e, [f[2 + c] * D.wall_slot_mask(P, c) for c in range(P.ndim)]

    errs = []
    for s in (1e-4, 5e-5):
        dX = s * dX0
        dU = D.pack(D.conserved(P, X + dX)) - D.pack(D.conserved(P, X))
        rp, re_, ru = PC.transform_in(si, dU)
        V1, V0 = V(X + dX), V(X)
        err_in = float((rp - (V1[0] - V0[0])).norm() / (V1[0] - V0[0]).norm())
        err_e = float((re_ - (V1[1] - V0[1])).norm() / (V1[1] - V0[1]).norm())
        err_u = max(float((ru[c] - (V1[2][c] - V0[2][c])).norm() / (V1[2][c] - V0[2][c]).norm())
                    for c in range(P.ndim))
        back = PC.transform_out(si, V1[0] - V0[0], V1[1] - V0[1], [V1[2][c] - V0[2][c] for c in range(P.ndim)])
        err_out = float((back - dX).norm() / dX.norm())
        errs.append((err_in, err_e, err_u, err_out))
    errs = np.array(errs)
    assert np.all(errs[0] < 1e-3), errs
    # the remainder is second order (it halves with |dX|), or zero where the
    # map is linear (p = (gamma-1) rho e is linear in U for the internal form)
    assert np.all((errs[0] < 1e-10) | (errs[0] / errs[1] > 1.8)), errs


def test_transformations_equal_the_printed_matrices():
    """For a uniform state the staggered transforms reduce to the 1D matrices
    printed in Sect. 3.2 (internal and total energy forms)."""
    gamma = 5 / 3
    rho0, e0, u0 = 1.7, 2.3, 0.4
    for form in (0, 1):
        P = D.Problem(ndim=2, n=(4, 4, 1), dx=(0.25, 0.25, 1), bc=(0, 0, 0), gamma=gamma, g=(0, 0, 0),
                      K0=0.0, chi_exp=3.0, energy_form=form, theta=1.0)
        ke = 0.5 * u0 * u0                                  # u_y = 0
        E0 = e0 + ke if form == 1 else e0
        X = torch.cat([torch.full((16,), v, dtype=torch.float64) for v in (rho0, E0, u0, 0.0)])
        si = PC.setup(P, X, 0.1, J.Options(precond=1))
        dpdrho, dpde = (gamma - 1) * e0, (gamma - 1) * rho0
        rng = np.random.default_rng(1)
        a, b, c = rng.standard_normal(3)
        v = torch.cat([torch.full((16,), v, dtype=torch.float64) for v in (a, b, c, 0.0)])
        rp, re_, ru = PC.transform_in(si, v)
        if form == 0:
            Mvu = np.array([[dpdrho - e0 / rho0 * dpde, dpde / rho0, 0.0],
                            [-e0 / rho0, 1 / rho0, 0.0],
                            [-u0 / rho0, 0.0, 1 / rho0]])
            Mxv = np.array([[1 / dpdrho, -dpde / dpdrho, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
        else:
            et = E0
            Mvu = np.array([[dpdrho - (et - u0 ** 2) / rho0 * dpde, dpde / rho0, -u0 / rho0 * dpde],
                            [-(et - u0 ** 2) / rho0, 1 / rho0, -u0 / rho0],
                            [-u0 / rho0, 0.0, 1 / rho0]])
            Mxv = np.array([[1 / dpdrho, -dpde / dpdrho, 0.0], [0.0, 1.0, u0], [0.0, 0.0, 1.0]])
        expect = Mvu @ np.array([a, b, c])
        got = np.array([float(rp[0, 0, 0]), float(re_[0, 0, 0]), float(ru[0][0, 0, 0])])
        assert np.allclose(got, expect, rtol=1e-13, atol=1e-13), (form, got, expect)
        dV = rng.standard_normal(3)
        back = PC.transform_out(si, torch.full((1, 4, 4), dV[0], dtype=torch.float64),
                                torch.full((1, 4, 4), dV[1], dtype=torch.float64),
                                [torch.full((1, 4, 4), dV[2], dtype=torch.float64),
                                 torch.zeros((1, 4, 4), dtype=torch.float64)])
        f = D.unpack(P, back)
        got = np.array([float(f[0][0, 0, 0]), float(f[1][0, 0, 0]), float(f[2][0, 0, 0])])
        assert np.allclose(got, Mxv @ dV, rtol=1e-13, atol=1e-13), (form, got, Mxv @ dV)


# ---------------------------------------------------------------------------
# semi-implicit systems and their multigrid solve (Sects. 3.3, 3.4)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nu,rate,final", [(2, 0.3, 1e-5), (1, 0.45, 1e-3)])
@pytest.mark.parametrize("cid,n", [(1, (16, 16)), (2, (16, 16)), (4, (8, 8, 8))])
def test_multigrid_converges_to_the_direct_solution(cid, n, nu, rate, final):
    """V(nu,nu) cycles against the sparse direct solve of the paper's rows:
    mean contraction per cycle measured 0.10-0.23 for V(2,2) and 0.21-0.31
    for V(1,1) (the cycle the benchmark runs)."""
    wl, P, X, dt, opts = _setup(cid, n, cfl=50.0)
    opts.mg_nu1 = opts.mg_nu2 = nu
    si = PC.setup(P, X, dt, opts)
    sc = J.scaling(P, X, opts)
    v = torch.as_tensor(W.random_vector(wl, 5))
    r_p, r_e, r_u = PC.transform_in(si, sc.L * v)
    dpx, dex, _ = PC.si_solve(si, r_p, r_e, r_u, exact=True)
    # the direct solution satisfies the paper's rows
    rp, re_ = PC.paper_rows(si, dpx, dex)
    assert float((rp - r_p).norm() / r_p.norm()) < 1e-12
    if si.kind == PC.SOUND_DIFF:
        assert float((re_ - r_e).norm() / r_e.norm()) < 1e-12
    errs = []
    for cyc in (1, 8):
        dp, de, _ = PC.si_solve(si, r_p, r_e, r_u, exact=False, cycles=cyc)
        errs.append(float((dp - dpx).norm() / dpx.norm()))
    assert errs[0] < 0.3
    assert (errs[1] / errs[0]) ** (1.0 / 7.0) < rate, errs    # mean contraction per V-cycle
    assert errs[1] < final


def test_sound_energy_row_identity():
    """With an exact dp the energy update from the identity of Sect. 3.3.4
    satisfies the paper's e row (Eq. SI3_e) exactly."""
    wl, P, X, dt, opts = _setup(1, (16, 16), cfl=30.0)
    si = PC.setup(P, X, dt, opts)
    v = torch.as_tensor(W.random_vector(wl, 6))
    r_p, r_e, r_u = PC.transform_in(si, v)
    dp, de, du = PC.si_solve(si, r_p, r_e, r_u, exact=True)
    _, re_ = PC.paper_rows(si, dp, de)
    assert float((re_ - r_e).norm() / r_e.norm()) < 1e-10
    # and du satisfies the velocity row du/dt + theta rho_f^-1 grad dp = r_u
    for c in range(P.ndim):
        gp = (dp - torch.roll(dp, 1, dims=2 - c)) / P.dx[c]
        row = du[c] / dt + P.theta * gp / si.rho_f[c]
        assert float((row - r_u[c]).norm() / r_u[c].norm()) < 1e-12


def test_pbp_is_exact_for_linear_acoustics():
    """Around a uniform state at rest the Jacobian is the linear acoustic
    operator, and the block-triangular SI preconditioner with an exact inner
    solve makes J M^-1 the identity plus a nilpotent block (Sect. 4.3):
    (J M^-1 - I)^2 = 0, so GMRES converges in 2 iterations even at
    CFL_hydro = 1000, while it stalls without preconditioning.  The exact
    derivative is used for J so that the finite-difference noise floor
    (amplified by the alpha1 = 1e-5 velocity scaling) does not blur it."""
    n = 8
    P = D.Problem(ndim=2, n=(n, n, 1), dx=(1 / n, 1 / n, 1), bc=(0, 0, 0), gamma=5 / 3, g=(0, 0, 0),
                  K0=0.0, chi_exp=3.0, energy_form=0, theta=0.5)
    N = n * n
    X = torch.cat([torch.full((N,), v, dtype=torch.float64) for v in (1.0, 1.5, 0.0, 0.0)])
    cs = math.sqrt(5 / 3 * 2 / 3 * 1.5)
    dt = 1000 * (1 / n) / cs
    opts = J.Options(precond=1, exact_inner=True)
    sc = J.scaling(P, X, opts)
    si = PC.setup(P, X, dt, opts)
    Jex = torch.func.jacrev(lambda x: D.G_operator(P, x, dt))(X) * sc.R[None, :] / sc.L[:, None]
    I4 = torch.eye(4 * N, dtype=torch.float64)
    Mi = torch.stack([PC.apply(si, I4[j], sc) for j in range(4 * N)], 1)
    E = Jex @ Mi - I4
    assert float(E.norm()) > 1e-2                           # not trivially the identity
    assert float((E @ E).norm()) < 1e-8 * float(E.norm()) ** 2 + 1e-8
    b = torch.as_tensor(np.random.default_rng(3).standard_normal(4 * N))
    _, st = J.gmres(lambda z: Jex @ z, lambda v: PC.apply(si, v, sc), b, 1e-8, 30, 30)
    assert st.converged and st.iterations <= 2, st
    _, st0 = J.gmres(lambda z: Jex @ z, lambda v: v, b, 1e-8, 30, 30)
    assert not st0.converged


# ---------------------------------------------------------------------------
# GMRES and Newton (Sect. 4.1)
# ---------------------------------------------------------------------------

def test_gmres_matches_dense_solve():
    wl, P, X, dt, opts = _setup(5, (8, 8), cfl=5.0)
    sc = J.scaling(P, X, opts)
    N = X.numel()
    Jex = torch.func.jacrev(lambda x: D.G_operator(P, x, dt))(X) * sc.R[None, :] / sc.L[:, None]
    masks = torch.cat([torch.ones(2 * P.ncell)] + [D.wall_slot_mask(P, c).reshape(-1) for c in range(P.ndim)])
    keep = masks.bool()
    A = Jex[keep][:, keep]
    b = torch.as_tensor(W.random_vector(wl, 8))
    x_direct = torch.linalg.solve(A, b[keep])
    si = PC.setup(P, X, dt, opts)
    x, st = J.gmres(lambda z: (Jex @ z) * masks, lambda v: PC.apply(si, v, sc), b, 1e-12, 30, 300)
    assert st.converged
    err = float((x[keep] - x_direct).norm() / x_direct.norm())
    cond = float(torch.linalg.cond(A))
    assert err < cond * 1e-12 * 10, (err, cond)
    # restarts: a short restart length reaches the same solution
    x2, st2 = J.gmres(lambda z: (Jex @ z) * masks, lambda v: PC.apply(si, v, sc), b, 1e-12, 5, 300)
    assert st2.restarts > 0 and float((x2[keep] - x_direct).norm() / x_direct.norm()) < cond * 1e-11


def test_newton_step_solves_the_residual_equation():
    """After a converged step F_U(X^{n+1}) is small against F_U(X^n) (Eq.
    newtimestep), and conserved totals change by dt sum F (here ~0)."""
    wl = W.config(1, n=(32, 32))
    P = D.Problem.from_workload(wl)
    X0 = torch.as_tensor(wl.X0)
    dt = D.cfl_dt(P, X0, 10.0)
    X1, st = J.newton_step(P, X0, dt, J.Options(precond=1))
    assert st.converged and 2 <= st.newton_iterations <= 6
    F0 = D.residual(P, X0, X0, dt)
    F1 = D.residual(P, X1, X0, dt)
    sc = J.scaling(P, X1, J.Options())
    assert float((F1 / sc.L).norm()) < 1e-6 * float((F0 / sc.L).norm())
    # periodic, no gravity: sum of U^{n+1} - U^n = dt sum F(X^{n+1})
    U1, U0 = D.conserved(P, X1), D.conserved(P, X0)
    Fk = D.unpack(P, F1)
    for k in (0, 2, 3):
        lhs = float((U1[k] - U0[k]).sum())
        rhs_ = dt * float(Fk[k].sum())
        assert abs(lhs - rhs_) < 1e-13 * float(U0[k].abs().sum()) + 1e-15


def test_frozen_preconditioner_reaches_the_same_step():
    """With the SI coefficients frozen at X^n (pc_freeze) the first Newton
    iteration is unchanged (X^(0) = X^n) and the step converges to the same
    X^{n+1}: the preconditioner changes the path, not the root of F_U."""
    wl = W.config(2, n=(32, 32))
    P = D.Problem.from_workload(wl)
    X0 = torch.as_tensor(wl.X0)
    dt = D.cfl_dt(P, X0, 20.0)
    first = {}

    def grab(tag):
        def f(k, X, dxh, gs):
            if k == 0:
                first[tag] = (dxh.clone(), gs.iterations)
        return f
    o = dict(precond=2, newton_tol=1e-11, eta=1e-8)
    X1, st = J.newton_step(P, X0, dt, J.Options(**o), on_iterate=grab("refresh"))
    X2, st2 = J.newton_step(P, X0, dt, J.Options(pc_freeze=True, **o), on_iterate=grab("freeze"))
    assert st.converged and st2.converged
    assert torch.equal(first["refresh"][0], first["freeze"][0])
    sc = J.scaling(P, X1, J.Options())
    assert float(((X1 - X2) / sc.R).abs().max()) < 1e-9


def test_unpreconditioned_gmres_stalls_at_large_cfl():
    """Sect. 5.1.1: without preconditioning GMRES does not converge for
    CFL_hydro >~ 10; with the sound-wave PBP it does."""
    wl = W.config(1, n=(32, 32))
    P = D.Problem.from_workload(wl)
    X0 = torch.as_tensor(wl.X0)
    dt = D.cfl_dt(P, X0, 20.0)
    o = J.Options(precond=0, gmres_max_it=60, newton_max=1, newton_min=1, alpha1=1.0)
    _, st = J.newton_step(P, X0, dt, o)
    assert st.gmres_iterations[0] == 60
    o = J.Options(precond=1, newton_max=1, newton_min=1)
    _, st = J.newton_step(P, X0, dt, o)
    assert st.gmres_iterations[0] < 30


def test_si_step_reduces_to_forward_euler():
    """As dt -> 0 the SI stepper of Sect. 3.6 becomes forward Euler in the
    unknowns: (X^{n+1} - X^n)/dt -> (dU/dX)^-1 R_U(X^n), with an error of
    order dt or smaller (the SI terms scale with dt).  Checked against a dense Jacobian
    of U(X), with the exact inner solve so that only the scheme is tested."""
    wl = W.config(1, n=(16, 16))
    P = D.Problem.from_workload(wl)
    P.theta = 1.0
    X = torch.as_tensor(W.random_state(wl, 2, rel=0.05, vel=0.2))
    JU = torch.func.jacrev(lambda x: D.pack(D.conserved(P, x)))(X)
    target = torch.linalg.solve(JU, D.pack(D.rhs(P, X)))
    errs = []
    # at M = 0.01 the acoustic SI terms make the O(dt) term large: c dt/dx = 0.016 at dt = 1e-5
    for dt in (1e-5, 1e-6):
        X1 = J.si_step(P, X, dt, J.Options(precond=1, exact_inner=True))
        errs.append(float(((X1 - X) / dt - target).norm() / target.norm()))
    assert errs[1] < 3e-3, errs
    assert errs[0] / errs[1] > 5.0, errs            # at least first order in dt


def _krylov_basis_loss(reorth, n=60, m=30):
    """Orthogonality of the GMRES basis on the diagonal operator with
    eigenvalues 2^0 ... 2^(n-1) and b = 1: max |V^T V - I| over the m basis
    vectors (with no preconditioner GMRES applies the operator to the basis
    vectors themselves, so they are captured there)."""
    d = 2.0 ** torch.arange(n, dtype=torch.float64)
    b = torch.ones(n, dtype=torch.float64)
    seen = []

    def A(v):
        seen.append(v.clone())
        return d * v
    _, st = J.gmres(A, lambda v: v, b, 1e-30, m, m, reorth=reorth, fixed=True)
    V = torch.stack(seen)
    return float((V @ V.T - torch.eye(len(seen), dtype=torch.float64)).abs().max()), st


def test_selective_reorthogonalisation_restores_an_orthogonal_basis():
    """Classical Gram-Schmidt loses orthogonality on an ill-conditioned
    Krylov sequence (30 vectors; eigenvalues spread over 2^0 ... 2^59: the
    basis drifts to 2.5e-7 from orthogonal); the selective second pass
    (Daniel, Gragg, Kaufman and Stewart 1976: re-project when the first pass
    shrank the vector below 1/sqrt(2) of its norm) keeps it at round-off,
    with fewer passes than the unconditional second pass."""
    loss0, st0 = _krylov_basis_loss(0)
    loss2, st2 = _krylov_basis_loss(2)
    loss1, st1 = _krylov_basis_loss(1)
    assert loss0 > 1e-8, loss0
    assert loss2 < 1e-14 and loss1 < 1e-14, (loss2, loss1)
    assert st0.reorth_passes == 0 and st1.reorth_passes == 30
    assert 0 < st2.reorth_passes < 30, st2.reorth_passes


def test_selective_reorthogonalisation_keeps_the_gmres_solution():
    """On a well-conditioned problem the criterion never fires and the
    solution is that of plain GMRES; with it the restarted solve of the 8x8
    Newton system still matches the dense solve."""
    d = torch.linspace(1.0, 3.0, 50, dtype=torch.float64)
    b = torch.ones(50, dtype=torch.float64)
    x0, s0 = J.gmres(lambda v: d * v, lambda v: v, b, 1e-12, 10, 100, reorth=0)
    x2, s2 = J.gmres(lambda v: d * v, lambda v: v, b, 1e-12, 10, 100, reorth=2)
    assert torch.allclose(x2, b / d, rtol=1e-10)
    assert float((x2 - x0).abs().max()) < 1e-13
