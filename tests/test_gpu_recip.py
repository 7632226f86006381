"""The reciprocal of the batched inversion in the flux kernels (recip_nr:
rcp.approx.ftz.f64 refined by two Newton-Raphson steps, Markstein 1990)
against CUDA's IEEE division 1.0 / d on the device: at most one unit in the
last place apart over the exponent range the kernels allow (|d| in
[2^-1000, 2^1000), where the inversion takes this path), mostly equal."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def probe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_03662_gb300 import build
    build.build()
    L = ctypes.CDLL(build.PROBE_LIB)
    L.fp64_recip_check.restype = ctypes.c_int
    L.fp64_recip_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p]
    return L


def _ulps(a, b):
    """Distance in units in the last place of two same-sign finite doubles."""
    ia = a.view(torch.int64)
    ib = b.view(torch.int64)
    return (ia - ib).abs()


def test_newton_raphson_reciprocal_is_within_one_ulp(probe):
    rng = np.random.default_rng(11)
    n = 1 << 22
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-999, 999, n)
    sign = rng.choice([-1.0, 1.0], n)
    d = sign * np.ldexp(mant, expo)
    # mantissa edges: powers of two, just above / below them, the largest mantissa
    edges = np.array([1.0, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0), 1.5, 1.0 + 2.0 ** -52 * 3])
    d[:len(edges)] = edges
    d[len(edges):2 * len(edges)] = -edges * 2.0 ** 999
    d[2 * len(edges):3 * len(edges)] = edges * 2.0 ** -1000
    dg = torch.as_tensor(d, device="cuda")
    r = torch.empty_like(dg)
    assert probe.fp64_recip_check(ctypes.c_void_p(dg.data_ptr()), ctypes.c_void_p(r.data_ptr()), n, None) == 0
    ref = 1.0 / dg
    torch.cuda.synchronize()
    u = _ulps(r, ref)
    assert int(u.max()) <= 1, int(u.max())
    assert bool(torch.isfinite(r).all())
    frac_exact = float((u == 0).double().mean())
    print("recip_nr: %.4f of the reciprocals equal to IEEE 1/d, the rest one ulp away" % frac_exact)
    assert frac_exact > 0.9


def test_integer_pipe_halving_equals_the_fp64_product(probe):
    """half_exact (the half mass flux of k_face_fluxes, an exponent decrement
    on the integer pipe) is bit-for-bit x * 0.5 for normal values of every
    exponent, and falls back to the product for zeros, subnormals, the
    smallest normal binade, infinities and NaN."""
    probe.fp64_half_check.restype = ctypes.c_int
    probe.fp64_half_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p]
    rng = np.random.default_rng(12)
    n = 1 << 20
    x = rng.choice([-1.0, 1.0], n) * np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-1074, 1024, n))
    tiny = np.finfo(np.float64).tiny
    special = np.array([0.0, -0.0, tiny, -tiny, 2 * tiny, np.nextafter(2 * tiny, 0), 5e-324, -5e-324,
                        np.nextafter(tiny, 0), np.inf, -np.inf, np.nan, np.finfo(np.float64).max, 1.0, -3.5])
    x[:len(special)] = special
    xg = torch.as_tensor(x, device="cuda")
    r = torch.empty_like(xg)
    assert probe.fp64_half_check(ctypes.c_void_p(xg.data_ptr()), ctypes.c_void_p(r.data_ptr()), n, None) == 0
    ref = xg * 0.5
    torch.cuda.synchronize()
    same = (r.view(torch.int64) == ref.view(torch.int64)) | (torch.isnan(r) & torch.isnan(ref))
    assert bool(same.all()), x[~same.cpu().numpy()][:8]

