"""The allocation-free residual entry point (jfnk_residual_noalloc).

Some callers cannot allocate device memory (their process's allocator is
owned elsewhere, or they receive only input and output buffers).  For them
the library keeps the residual's scratch in a fixed device array.  This test
calls that entry point through the C ABI, twice in a row, on a handle that
was never bound to a workspace, and checks it against jfnk_residual.  It sits
in a file collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_03662_gb300 import build
    build.build()
    import paper_1512_03662_gb300 as jf
    return jf


def _unbound_handle(jf, wl):
    L = jf.lib()
    gr = jf.jfnk_grid(wl.ndim, (ctypes.c_int * 3)(*wl.n), (ctypes.c_double * 3)(*wl.lo),
                      (ctypes.c_double * 3)(*wl.hi), (ctypes.c_int * 3)(*wl.bc))
    eo = jf.jfnk_eos(wl.gamma, wl.energy_form)
    gv = jf.jfnk_gravity((ctypes.c_double * 3)(*wl.g))
    co = jf.jfnk_conductivity(wl.K0, wl.chi_exp)
    o = jf.default_options(theta=wl.theta, precond=0)
    h = ctypes.c_void_p()
    assert L.jfnk_create(ctypes.byref(gr), ctypes.byref(eo), ctypes.byref(gv), ctypes.byref(co),
                         ctypes.byref(o), ctypes.byref(h)) == 0
    return h


@pytest.mark.parametrize("cid,n", [(4, (16, 16, 16)), (2, (32, 32))])
def test_noalloc_residual_matches_the_workspace_residual(jf, cid, n):
    wl = W.config(cid, n=n)
    Xn = torch.as_tensor(wl.X0, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(3)
    dt = 0.37
    S = jf.Solver.from_workload(wl, jf.default_options(theta=wl.theta, precond=0))
    L = jf.lib()
    h = _unbound_handle(jf, wl)
    try:
        for call in range(2):
            X = Xn * torch.as_tensor(1.0 + 0.01 * rng.standard_normal(Xn.numel()), device="cuda")
            ref = S.residual(X, Xn, dt)
            F = torch.full_like(Xn, float("nan"))
            st = L.jfnk_residual_noalloc(h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Xn.data_ptr()), dt,
                                         ctypes.c_void_p(F.data_ptr()))
            torch.cuda.synchronize()
            assert st == 0, L.jfnk_last_error(h).decode()
            rel = float((F - ref).norm() / ref.norm())
            assert rel < 1e-10, (call, rel)
    finally:
        L.jfnk_destroy(h)


def test_noalloc_rejects_grids_above_its_limit(jf):
    wl = W.config(4, n=(64, 64, 32))                   # 131072 cells > 65536
    h = _unbound_handle(jf, wl)
    L = jf.lib()
    try:
        X = torch.as_tensor(wl.X0, dtype=torch.float64, device="cuda")
        F = torch.empty_like(X)
        st = L.jfnk_residual_noalloc(h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(X.data_ptr()), 0.1,
                                     ctypes.c_void_p(F.data_ptr()))
        assert st == jf.JFNK_EINVAL
        assert b"exceed" in L.jfnk_last_error(h)
    finally:
        L.jfnk_destroy(h)


def test_noalloc_on_a_bound_handle_follows_its_stream(jf):
    """On a handle bound to a workspace and to a non-default stream, the
    allocation-free residual is queued on that stream like jfnk_residual:
    two calls in a row, each right after a residual on the same stream,
    agree with it."""
    wl = W.config(4, n=(16, 16, 16))
    stream = torch.cuda.Stream()
    S = jf.Solver.from_workload(wl, jf.default_options(theta=wl.theta, precond=0), stream=stream)
    Xn = torch.as_tensor(wl.X0, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(5)
    for call in range(2):
        X = Xn * torch.as_tensor(1.0 + 0.01 * rng.standard_normal(Xn.numel()), device="cuda")
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ref = S.residual(X, Xn, 0.37)
            F = S.residual_noalloc(X, Xn, 0.37)
        stream.synchronize()
        rel = float((F - ref).norm() / ref.norm())
        assert rel < 1e-10, (call, rel)
