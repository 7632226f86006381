"""Host logic of the C ABI that needs no GPU: handle creation and its
argument checks, the vector length and workspace plan of the five problems,
option changes after creation, and the error returned by calls made before a
workspace is bound.  No kernel is launched."""
import ctypes

import pytest

import workloads as W


@pytest.fixture(scope="module")
def jf():
    from paper_1512_03662_gb300 import build
    build.build()
    import paper_1512_03662_gb300 as jf
    return jf


def _structs(jf, ndim, n, lo, hi, bc, gamma=5.0 / 3.0, energy_form=0, g=(0.0, 0.0, 0.0), K0=0.0, chi_exp=3.0):
    gr = jf.jfnk_grid(ndim, (ctypes.c_int * 3)(*n), (ctypes.c_double * 3)(*lo), (ctypes.c_double * 3)(*hi),
                      (ctypes.c_int * 3)(*bc))
    return gr, jf.jfnk_eos(gamma, energy_form), jf.jfnk_gravity((ctypes.c_double * 3)(*g)), \
        jf.jfnk_conductivity(K0, chi_exp)


def _create(jf, structs, opt):
    L = jf.lib()
    gr, eo, gv, co = structs
    h = ctypes.c_void_p()
    st = L.jfnk_create(ctypes.byref(gr), ctypes.byref(eo), ctypes.byref(gv), ctypes.byref(co),
                       ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    msg = L.jfnk_last_error(h).decode() if h else ""
    return st, h, msg


def _wl_structs(jf, wl):
    return _structs(jf, wl.ndim, wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.energy_form, wl.g, wl.K0, wl.chi_exp)


@pytest.mark.parametrize("cid", [1, 2, 3, 4, 5])
def test_full_size_handles_plan_on_the_host(jf, cid):
    """Every problem at its full size: the packed vector has (2 + ndim) ncell
    entries, and the workspace of the mixed handle (FP32 Krylov basis and
    preconditioner) is smaller than that of the FP64 handle."""
    L = jf.lib()
    wl = W.config(cid)
    sizes = {}
    for prec in (jf.MIXED, jf.FP64):
        st, h, msg = _create(jf, _wl_structs(jf, wl),
                             jf.default_options(theta=wl.theta, precond=wl.precond, precision=prec))
        assert st == jf.JFNK_OK, msg
        assert L.jfnk_vector_length(h) == (2 + wl.ndim) * wl.ncell
        sizes[prec] = int(L.jfnk_workspace_bytes(h))
        L.jfnk_destroy(h)
    assert 0 < sizes[jf.MIXED] < sizes[jf.FP64]
    if cid == 4:
        # 256^3: about 34 GB mixed (no adjoint scratch: the adjoint runs on
        # FP64 handles only), 64 GB FP64, both far inside the 288 GB of HBM
        assert sizes[jf.MIXED] < 36e9 and sizes[jf.FP64] < 72e9


def test_workspace_grows_with_the_krylov_basis(jf):
    L = jf.lib()
    wl = W.config(2)
    b = []
    for m in (10, 30):
        st, h, msg = _create(jf, _wl_structs(jf, wl), jf.default_options(theta=wl.theta, precond=wl.precond,
                                                                          gmres_m=m))
        assert st == jf.JFNK_OK, msg
        b.append(int(L.jfnk_workspace_bytes(h)))
        L.jfnk_destroy(h)
    # 20 more basis vectors V and 20 more preconditioned directions Z, FP64
    assert b[1] - b[0] >= 40 * (2 + wl.ndim) * wl.ncell * 8


BAD_GRIDS = [
    (dict(ndim=4), "ndim"),
    (dict(n=(2, 16, 1)), "at least 4 cells"),
    (dict(bc=(0, 7, 0)), "boundary"),
    (dict(hi=(0.0, 1.0, 1.0)), "empty domain"),
    (dict(n=(16, 16, 2)), "n[2] must be 1"),
    (dict(gamma=1.0), "gamma"),
    (dict(energy_form=3), "energy form"),
    (dict(K0=-1.0), "K0"),
]


@pytest.mark.parametrize("change,words", BAD_GRIDS)
def test_create_rejects_bad_problems(jf, change, words):
    L = jf.lib()
    kw = dict(ndim=2, n=(16, 16, 1), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=(0, 1, 0))
    kw.update(change)
    st, h, msg = _create(jf, _structs(jf, **kw), jf.default_options(precond=0))
    assert st == jf.JFNK_EINVAL and words in msg, (st, msg)
    if h:
        L.jfnk_destroy(h)


BAD_OPTIONS = [
    (dict(theta=0.0), "theta"),
    (dict(gmres_m=65), "gmres_m"),
    (dict(gmres_max_it=0), "gmres_max_it"),
    (dict(newton_max=0), "newton_max"),
    (dict(precond=3), "preconditioner"),
    (dict(precision=7), "precision"),
    (dict(mg_cycles=0), "multigrid"),
    (dict(pc_freeze=2), "pc_freeze"),
    (dict(lam=0.0), "lambda"),
    (dict(pert=5), "perturbation"),
]


@pytest.mark.parametrize("change,words", BAD_OPTIONS)
def test_create_rejects_bad_options(jf, change, words):
    L = jf.lib()
    st, h, msg = _create(jf, _structs(jf, 2, (16, 16, 1), (0, 0, 0), (1, 1, 1), (0, 1, 0)),
                         jf.default_options(**change))
    assert st == jf.JFNK_EINVAL and words in msg, (st, msg)
    if h:
        L.jfnk_destroy(h)


def test_preconditioned_handles_need_power_of_two_grids(jf):
    L = jf.lib()
    structs = _structs(jf, 2, (20, 12, 1), (0, 0, 0), (1, 1, 1), (0, 1, 0))
    st, h, msg = _create(jf, structs, jf.default_options(precond=1))
    assert st == jf.JFNK_EINVAL and "power-of-two" in msg
    L.jfnk_destroy(h)
    st, h, msg = _create(jf, structs, jf.default_options(precond=0))
    assert st == jf.JFNK_OK, msg
    L.jfnk_destroy(h)


def test_options_fixed_at_creation_cannot_change(jf):
    L = jf.lib()
    st, h, msg = _create(jf, _structs(jf, 2, (16, 16, 1), (0, 0, 0), (1, 1, 1), (0, 1, 0)),
                         jf.default_options(precond=1))
    assert st == jf.JFNK_OK, msg
    ok = jf.default_options(precond=1, eta=1e-2, mg_cycles=1, mg_nu1=1, mg_nu2=1, theta=1.0)
    assert L.jfnk_set_options(h, ctypes.byref(ok)) == jf.JFNK_OK
    for change in (dict(gmres_m=10), dict(precond=2), dict(precision=jf.MIXED)):
        o = jf.default_options(**{"precond": 1, **change})
        assert L.jfnk_set_options(h, ctypes.byref(o)) == jf.JFNK_EINVAL, change
        assert "fixed at creation" in L.jfnk_last_error(h).decode()
    bad = jf.default_options(precond=1, theta=2.0)
    assert L.jfnk_set_options(h, ctypes.byref(bad)) == jf.JFNK_EINVAL
    L.jfnk_destroy(h)


def test_calls_before_binding_a_workspace_are_refused(jf):
    """Without a bound workspace every compute entry point returns
    JFNK_ENOMEM before touching the GPU; a workspace that is too small or
    misaligned is refused by jfnk_bind before it is used."""
    L = jf.lib()
    st, h, msg = _create(jf, _structs(jf, 2, (16, 16, 1), (0, 0, 0), (1, 1, 1), (0, 1, 0)),
                         jf.default_options(precond=1))
    assert st == jf.JFNK_OK, msg
    p = ctypes.c_void_p(4096)          # never dereferenced: the calls return first
    d = ctypes.c_double()
    assert L.jfnk_residual(h, p, p, ctypes.c_double(0.1), p) == jf.JFNK_ENOMEM
    assert "no workspace bound" in L.jfnk_last_error(h).decode()
    assert L.jfnk_jv(h, p, ctypes.c_double(0.1), p, p, ctypes.byref(d)) == jf.JFNK_ENOMEM
    assert L.jfnk_precond_apply(h, p, ctypes.c_double(0.1), p, p) == jf.JFNK_ENOMEM
    nbytes = int(L.jfnk_workspace_bytes(h))
    assert L.jfnk_bind(h, p, ctypes.c_size_t(nbytes - 1), None) == jf.JFNK_ENOMEM
    assert L.jfnk_bind(h, ctypes.c_void_p(4096 + 8), ctypes.c_size_t(nbytes), None) == jf.JFNK_EINVAL
    assert "256-byte aligned" in L.jfnk_last_error(h).decode()
    L.jfnk_destroy(h)


def _fake_solver(jf, nvec=64, mixed=False):
    """A Solver whose handle is never used: the argument checks of the
    binding run before any library call, so they can be tested without a
    GPU (the device is only compared, never touched)."""
    import torch
    S = object.__new__(jf.Solver)
    S.h = None
    S.device = torch.device("cuda", 0)
    S.nvec = nvec
    S.vdtype = torch.float32 if mixed else torch.float64
    return S


def test_binding_rejects_tensors_the_library_cannot_take(jf):
    """CPU tensors, a wrong dtype, a non-contiguous view or a wrong length
    raise before the pointer reaches the C ABI (a wrong tensor would make
    the kernels read or write out of bounds)."""
    import torch
    S = _fake_solver(jf)
    good_shape = torch.zeros(64, dtype=torch.float64)
    with pytest.raises(ValueError, match="is on cpu"):
        S.residual(good_shape, good_shape, 0.1)
    with pytest.raises(TypeError):
        S.step([0.0] * 64, 0.1)
    meta = dict(device="meta")
    # the checks compare metadata only, so meta tensors stand in for device tensors
    S.device = torch.device("meta")
    with pytest.raises(ValueError, match="dtype"):
        S.residual(torch.empty(64, dtype=torch.float32, **meta), torch.empty(64, dtype=torch.float64, **meta), 0.1)
    with pytest.raises(ValueError, match="contiguous"):
        S.step(torch.empty(128, dtype=torch.float64, **meta)[::2], 0.1)
    with pytest.raises(ValueError, match="elements"):
        S.dt_from_cfl(torch.empty(63, dtype=torch.float64, **meta), 1.0)
    with pytest.raises(ValueError, match="Xn"):
        S.linear_solve(torch.empty(64, dtype=torch.float64, **meta), torch.empty(65, dtype=torch.float64, **meta),
                       0.1)
    with pytest.raises(ValueError, match="gbar"):
        S.vjp(torch.empty(64, dtype=torch.float64, **meta), torch.empty(64, dtype=torch.float64, **meta), 0.1,
              torch.empty(64, dtype=torch.float32, **meta))


def test_binding_checks_krylov_vectors_against_the_handle_precision(jf):
    """Jv and preconditioner vectors are float on a mixed handle and double
    on an FP64 handle; X stays double on both."""
    import torch
    meta = dict(device="meta")
    X = torch.empty(64, dtype=torch.float64, **meta)
    for mixed, bad in ((True, torch.float64), (False, torch.float32)):
        S = _fake_solver(jf, mixed=mixed)
        S.device = torch.device("meta")
        with pytest.raises(ValueError, match="v has dtype"):
            S.jv(X, 0.1, torch.empty(64, dtype=bad, **meta))
        with pytest.raises(ValueError, match="v has dtype"):
            S.precond_apply(X, 0.1, torch.empty(64, dtype=bad, **meta))
        with pytest.raises(ValueError, match="X has dtype"):
            S.jv(X.float(), 0.1, torch.empty(64, dtype=S.vdtype, **meta))
