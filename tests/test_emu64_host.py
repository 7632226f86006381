"""The integer-pipe IEEE products and sums of the flux kernels (emu64.cuh),
built for the host with g++ from the same source, against the host's
binary64 arithmetic bit for bit (IEEE 754 round to nearest, ties to even):
random bit patterns, exact ties, cancellation, exponent gaps across the
alignment frame, overflow and the subnormal edge, special values.  The GPU
build is checked against the DMUL / DADD instructions in
test_gpu_recip.py."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from emu_cases import emu_operands

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1512_03662_gb300", "csrc")


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("emu") / "libemu64host.so")
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "emu64_host.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    L.emu64_host.restype = None
    L.emu64_host.argtypes = [ctypes.c_void_p] * 6 + [ctypes.c_longlong]
    return L


def _run(L, a, b):
    n = len(a)
    m, s, d = np.empty(n), np.empty(n), np.empty(n)
    fast = np.empty(n, dtype=np.uint8)
    L.emu64_host(*(x.ctypes.data for x in (a, b, m, s, d, fast)), n)
    return m, s, d, fast


def _same(x, y):
    return (x.view(np.int64) == y.view(np.int64)) | (np.isnan(x) & np.isnan(y))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_products_and_sums_are_the_ieee_results(emu, seed):
    a, b = emu_operands(1 << 20, seed)
    m, s, d, fast = _run(emu, a, b)
    with np.errstate(all="ignore"):
        refs = (a * b, a + b, a - b)
    for name, got, ref in zip(("mul", "add", "sub"), (m, s, d), refs):
        ok = _same(got, ref)
        assert ok.all(), (name, a[~ok][:4], b[~ok][:4], got[~ok][:4], ref[~ok][:4])
    # the integer path itself, not the hardware fallback, carries the
    # moderate-exponent, tie, cancellation and gap classes
    k = len(a) // 8
    assert fast[k:5 * k].mean() > 0.999


def test_signed_zeros_and_exact_cancellation(emu):
    a = np.array([0.0, -0.0, 0.0, -0.0, 1.5, -1.5, 3.0, -2.0 ** -1000])
    b = np.array([-0.0, -0.0, 0.0, 0.0, -1.5, 1.5, -0.0, 0.0])
    m, s, d, _ = _run(emu, a, b)
    assert _same(m, a * b).all() and _same(s, a + b).all() and _same(d, a - b).all()
    # x - x = +0 and -0 + -0 = -0 (round to nearest)
    assert np.signbit(s[1]) and not np.signbit(s[4]) and not np.signbit(s[0])
