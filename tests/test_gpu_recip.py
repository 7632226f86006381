"""The reciprocal of the batched inversion in the flux kernels (recip_nr:
rcp.approx.ftz.f64 refined by one third-order step of the reciprocal
iteration, Markstein 1990)
against CUDA's IEEE division 1.0 / d on the device: at most one unit in the
last place apart over the exponent range the kernels allow (|d| in
[2^-1000, 2^1000), where the inversion takes this path), mostly equal."""
import ctypes

import numpy as np
import pytest
import torch

from emu_cases import emu_operands

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



def test_integer_pipe_conversions_equal_the_conversion_instructions(probe):
    """d2f_rn (the float output of the Jacobian-free assemble) and f2d_exact
    (the float Krylov vector read by the perturbation kernel) give the bits
    of the hardware conversions for every class of input: normal values,
    half-way cases (ties to even), carries into the exponent, overflow to
    infinity, float subnormals on both sides, zeros, infinities; NaN stays
    NaN."""
    probe.fp64_conv_check.restype = ctypes.c_int
    probe.fp64_conv_check.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_longlong, ctypes.c_void_p]
    rng = np.random.default_rng(13)
    n = 1 << 21
    x = rng.choice([-1.0, 1.0], n) * np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-160, 140, n))
    # half-way doubles between two floats (ties) and their neighbours, among
    # normal floats and among float subnormals
    m = rng.integers(1 << 23, 1 << 24, 4096).astype(np.float64)
    ties = np.ldexp(m + 0.5, rng.integers(-140, 100, 4096) - 23)
    sub = np.ldexp(rng.integers(0, 1 << 23, 4096).astype(np.float64) + 0.5, -149)
    x[:4096] = ties
    x[4096:8192] = np.nextafter(ties, np.inf)
    x[8192:12288] = np.nextafter(ties, -np.inf)
    x[12288:16384] = sub
    x[16384:20480] = -np.nextafter(sub, np.inf)
    fmax = float(np.finfo(np.float32).max)
    special = np.array([0.0, -0.0, fmax, -fmax, fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -24), 2.0 ** 128,
                        2.0 ** -126, 2.0 ** -127, 2.0 ** -149, 2.0 ** -150, 3 * 2.0 ** -151, 2.0 ** -151, 1e-320,
                        np.inf, -np.inf, np.nan, np.nextafter(2.0 ** -126, 0.0), (2.0 - 2.0 ** -23) * 2.0 ** 127,
                        (2.0 - 2.0 ** -24) * 2.0 ** -127, 1e300, -1e-300])
    x[20480:20480 + len(special)] = special
    f = (rng.choice([-1.0, 1.0], n) * np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-149, 128, n))).astype(np.float32)
    f[:4096] = (rng.integers(1, 1 << 23, 4096) * np.float64(2.0 ** -149)).astype(np.float32)   # subnormals
    fspecial = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.17549435e-38, 5.877472e-39,
                         3.4028235e38], dtype=np.float32)
    f[4096:4096 + len(fspecial)] = fspecial
    xg = torch.as_tensor(x, device="cuda")
    fg = torch.as_tensor(f, device="cuda")
    xf = torch.empty(n, dtype=torch.float32, device="cuda")
    fd = torch.empty(n, dtype=torch.float64, device="cuda")
    assert probe.fp64_conv_check(ctypes.c_void_p(xg.data_ptr()), ctypes.c_void_p(fg.data_ptr()),
                                 ctypes.c_void_p(xf.data_ptr()), ctypes.c_void_p(fd.data_ptr()), n, None) == 0
    ref_f = xg.float()
    ref_d = fg.double()
    torch.cuda.synchronize()
    same_f = (xf.view(torch.int32) == ref_f.view(torch.int32)) | (torch.isnan(xf) & torch.isnan(ref_f))
    same_d = (fd.view(torch.int64) == ref_d.view(torch.int64)) | (torch.isnan(fd) & torch.isnan(ref_d))
    assert bool(same_f.all()), x[~same_f.cpu().numpy()][:8]
    assert bool(same_d.all()), f[~same_d.cpu().numpy()][:8]


def test_integer_pipe_products_and_sums_equal_dmul_dadd(probe):
    """emu::mul_rn, add_rn and sub_rn (the products and sums the flux
    kernels move off the FP64 pipe) give the bits of the DMUL / DADD
    instructions, computed by torch on the same device, for every class of
    input; NaN stays NaN."""
    probe.fp64_emu_check.restype = ctypes.c_int
    probe.fp64_emu_check.argtypes = [ctypes.c_void_p] * 5 + [ctypes.c_longlong, ctypes.c_void_p]
    n = 1 << 23
    a, b = emu_operands(n, 17)
    ag = torch.as_tensor(a, device="cuda")
    bg = torch.as_tensor(b, device="cuda")
    m = torch.empty_like(ag)
    s = torch.empty_like(ag)
    d = torch.empty_like(ag)
    assert probe.fp64_emu_check(*(ctypes.c_void_p(t.data_ptr()) for t in (ag, bg, m, s, d)), n, None) == 0
    refs = (ag * bg, ag + bg, ag - bg)
    torch.cuda.synchronize()
    for name, got, ref in zip(("mul", "add", "sub"), (m, s, d), refs):
        same = (got.view(torch.int64) == ref.view(torch.int64)) | (torch.isnan(got) & torch.isnan(ref))
        bad = (~same).nonzero().flatten()[:4].cpu().numpy()
        assert bool(same.all()), (name, a[bad], b[bad], got.cpu().numpy()[bad], ref.cpu().numpy()[bad])
