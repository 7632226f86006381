"""Parity with the oracle on grids with reflecting walls in directions the
five problems never wall (x, and all directions at once): the branch-free
neighbour offsets of the residual kernels (periodic wrap or wall mirror,
the odd mirror of the normal velocity and the zero of wall faces, chosen
per direction from the boundary type) are exercised on every direction
and in both energy forms.  Residual elementwise at 1e-9 of each field's
maximum and normwise at 1e-10; the scaling at 1e-14; the Jacobian-free
product at lambda = 1e-4 (above its finite-difference noise floor) at
1e-10; the preconditioner and the adjoint's J^T w at 1e-10; one
preconditioned implicit step with fixed iteration counts against the
oracle's own rounding sensitivity."""
import dataclasses

import numpy as np
import pytest
import torch

import workloads as W
from oracle import discretization as D
from oracle import jfnk as J

pytestmark = pytest.mark.gpu

# (problem, grid, boundary type per direction); 1 = wall
WALL_CASES = [
    (2, (16, 12, 1), (1, 1, 0)),
    (2, (12, 16, 1), (1, 0, 0)),
    (4, (12, 10, 8), (1, 1, 1)),
    (4, (8, 12, 10), (1, 0, 1)),
    (3, (10, 8, 12), (0, 1, 0)),
]


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


def _relnorm(a, b, w=None):
    a, b = a.detach().double().cpu(), torch.as_tensor(b).double()
    if w is not None:
        a, b = a / w, b / w
    return float((a - b).norm() / b.norm())


def _zero_wall_slots(wl, X):
    """Zero the normal velocity on the lower wall face of every walled
    direction (the slots the packed layout keeps for them)."""
    X = X.copy()
    shp = (wl.n[2], wl.n[1], wl.n[0])
    for d in range(wl.ndim):
        if wl.bc[d] == W.BC_WALL:
            u = X[(2 + d) * wl.ncell:(3 + d) * wl.ncell].reshape(shp)
            idx = [slice(None)] * 3
            idx[2 - d] = 0
            u[tuple(idx)] = 0.0
    return X


def _wall_case(cid, n, bc, form, seed=7, rel=0.02, vel=0.1):
    base = W.config(cid, n=n[:3] if cid in (3, 4) else n[:2])
    wl = dataclasses.replace(base, bc=bc)
    wl.energy_form = form
    P = D.Problem.from_workload(wl)
    Xn = torch.as_tensor(_zero_wall_slots(wl, wl.X0))
    if form == D.ENERGY_TOTAL:
        Xn[P.ncell:2 * P.ncell] += 0.5 * float(Xn[2 * P.ncell:].abs().max()) ** 2 + 1.0
    pert = torch.as_tensor(W.random_vector(wl, seed))
    scale = torch.cat([Xn[:2 * P.ncell].abs() * rel,
                       torch.full((P.ndim * P.ncell,), vel, dtype=torch.float64) *
                       float(torch.sqrt(wl.gamma * (wl.gamma - 1) * Xn[P.ncell:2 * P.ncell]).mean())])
    X = Xn + pert * scale
    dt = D.cfl_dt(P, Xn, wl.cfl_hydro)
    return wl, P, X, Xn, dt


def _solver(jf, wl, **kw):
    pow2 = all((v & (v - 1)) == 0 for v in wl.n[:wl.ndim])
    kw.setdefault("theta", wl.theta)
    kw.setdefault("precond", wl.precond if pow2 else 0)
    return jf.Solver.from_workload(wl, jf.default_options(**kw))


@pytest.mark.parametrize("cid,n,bc", WALL_CASES)
@pytest.mark.parametrize("form", [0, 1])
def test_residual_and_scaling_parity_with_walls(jf, cid, n, bc, form):
    wl, P, X, Xn, dt = _wall_case(cid, n, bc, form)
    assert tuple(P.bc) == bc
    S = _solver(jf, wl)
    F = S.residual(_dev(X), _dev(Xn), dt)
    Fo = D.residual(P, X, Xn, dt)
    sc = J.scaling(P, X, J.Options())
    assert _relnorm(F, Fo, sc.L) < 1e-10
    Fg = F.detach().cpu()
    for k in range(P.nfield):
        a, b = Fg[k * P.ncell:(k + 1) * P.ncell], Fo[k * P.ncell:(k + 1) * P.ncell]
        assert float((a - b).abs().max()) <= 1e-9 * float(b.abs().max()) + 1e-300, k
    L, R, xn = S.scaling(_dev(X))
    assert _relnorm(L, sc.L) < 1e-14
    assert _relnorm(R, sc.R) < 1e-14
    assert xn == pytest.approx(sc.xhat_norm, rel=1e-13)


@pytest.mark.parametrize("cid,n,bc", WALL_CASES)
@pytest.mark.parametrize("form", [0, 1])
def test_jv_parity_with_walls(jf, cid, n, bc, form):
    wl, P, X, Xn, dt = _wall_case(cid, n, bc, form)
    v = torch.as_tensor(W.random_vector(wl, 3))
    S = _solver(jf, wl, lam=1e-4)
    Jv, delta = S.jv(_dev(X), dt, _dev(v))
    oo = J.Options(lam=1e-4)
    sc = J.scaling(P, X, oo)
    Jo, do = J.jv(P, X, D.G_operator(P, X, dt), sc, v, dt, oo)
    assert delta == pytest.approx(do, rel=1e-13)
    assert _relnorm(Jv, Jo) < 1e-10, _relnorm(Jv, Jo)


# power-of-two grids (the multigrid preconditioner needs them), walled in x
# and in the direction of gravity (stratified problems 2 and 4)
PC_WALL_CASES = [
    (2, (16, 16, 1), (1, 1, 0), 2),
    (2, (16, 8, 1), (1, 1, 0), 1),
    (4, (8, 8, 8), (1, 1, 1), 2),
    (4, (8, 16, 8), (1, 0, 1), 1),
]


@pytest.mark.parametrize("cid,n,bc,pc", PC_WALL_CASES)
def test_precond_parity_with_walls(jf, cid, n, bc, pc):
    """The sound-wave (pc = 1) and sound-wave + conduction (pc = 2)
    preconditioner, two V-cycles, FP64, against the oracle's: 1e-10; the
    normal velocity stays zero on every wall face."""
    from oracle import precond as PC
    wl, P, X, Xn, dt = _wall_case(cid, n, bc, 0)
    v = torch.as_tensor(W.random_vector(wl, 5))
    S = jf.Solver.from_workload(wl, jf.default_options(theta=wl.theta, precond=pc, mg_cycles=2))
    w = S.precond_apply(_dev(X), dt, _dev(v))
    oo = J.Options(precond=pc, mg_cycles=2)
    wo = PC.apply(PC.setup(P, X, dt, oo), v, J.scaling(P, X, oo))
    assert _relnorm(w, wo) < 1e-10, _relnorm(w, wo)
    wc = w.detach().cpu()
    for c in range(P.ndim):
        if bc[c] == W.BC_WALL:
            f = wc[(2 + c) * P.ncell:(3 + c) * P.ncell].reshape(P.shape)
            idx = [slice(None)] * 3
            idx[2 - c] = 0
            assert float(f[tuple(idx)].abs().max()) == 0.0


@pytest.mark.parametrize("cid,n,bc,pc", PC_WALL_CASES)
def test_step_parity_fixed_iterations_with_walls(jf, cid, n, bc, pc):
    """Two Newton iterations of eight preconditioned GMRES iterations each
    (deterministic mode, lambda = 1e-4): the step X^{n+1} - X^n against the
    oracle's, scaled, normwise.  At these CFL numbers (100 and 200 on grids
    of 8 to 16 cells) the unconverged Krylov iterations amplify round-off:
    a 1-ulp change of X^n moves the oracle's own step by 3e-8 to 8e-4
    (measured), so the bound is a multiple of that sensitivity (and 1e-10
    where it is smaller), as in the other fixed-iteration step tests."""
    wl, P, X, Xn, dt = _wall_case(cid, n, bc, 0)
    o = jf.default_options(theta=wl.theta, precond=pc, gmres_m=8, gmres_max_it=8, newton_max=2,
                           fixed_iterations=1, lam=1e-4)
    S = jf.Solver.from_workload(wl, o)
    Xg = _dev(Xn)
    st = S.step(Xg, dt)
    assert st["newton_iterations"] == 2
    oo = J.Options(precond=pc, gmres_m=8, gmres_max_it=8, newton_max=2, fixed_iterations=True, lam=1e-4)
    Xo, _ = J.newton_step(P, Xn, dt, oo)
    sc = J.scaling(P, Xn, oo)
    err = _relnorm(Xg - _dev(Xn), Xo - Xn, sc.R)
    sens = 0.0
    for sd in (1, 2):
        rng = np.random.default_rng(sd)
        Xp = Xn * (1.0 + torch.as_tensor(rng.choice([-1.0, 1.0], Xn.numel())) * 2.0 ** -52)
        sens = max(sens, _relnorm(J.newton_step(P, Xp, dt, oo)[0] - Xp, Xo - Xn, sc.R))
    print("walled step %s: gpu-oracle %.2e, oracle 1-ulp sensitivity %.2e" % (bc, err, sens))
    assert err < max(1e-10, 4.0 * sens), (err, sens)


@pytest.mark.parametrize("cid,n,bc", WALL_CASES)
@pytest.mark.parametrize("form", [0, 1])
def test_vjp_residual_parity_with_walls(jf, cid, n, bc, form):
    """The transposed residual Jacobian product (the adjoint's J^T w, its
    wall mirrors scattered back with their signs) against the oracle's
    reverse-mode product: 1e-10."""
    from oracle import adjoint as A
    wl, P, X, Xn, dt = _wall_case(cid, n, bc, form)
    w = torch.as_tensor(W.random_vector(wl, 4))
    S = _solver(jf, wl)
    y = S.vjp_residual(_dev(X), dt, _dev(w))
    yo = A.vjp_G(P, X, dt, w)
    assert _relnorm(y, yo) < 1e-10, _relnorm(y, yo)
