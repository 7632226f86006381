"""Operand pairs shared by the host and device checks of the integer-pipe
products and sums (emu64.cuh)."""
import numpy as np


def emu_operands(n, seed):
    """Operand pairs for the integer-pipe products and sums: random bit
    patterns (every class of double), moderate exponents, short significands
    (many exact ties), nearly equal magnitudes of opposite sign (cancellation
    down to a few bits), exponent gaps around the 53 + 10 bits of the
    alignment frame, products and sums near overflow and near the subnormal
    range, and the special values."""
    rng = np.random.default_rng(seed)
    k = n // 8
    u = rng.integers(0, 2 ** 63, (2, n), dtype=np.int64).view(np.uint64) ^ \
        (rng.integers(0, 2, (2, n), dtype=np.uint64) << np.uint64(63))
    a = u[0].view(np.float64).copy()
    b = u[1].view(np.float64).copy()
    sgn = lambda m: rng.choice([-1.0, 1.0], m)
    # moderate exponents
    a[k:2 * k] = sgn(k) * np.ldexp(rng.uniform(1, 2, k), rng.integers(-100, 100, k))
    b[k:2 * k] = sgn(k) * np.ldexp(rng.uniform(1, 2, k), rng.integers(-100, 100, k))
    # short significands: exact ties of the rounding
    a[2 * k:3 * k] = sgn(k) * np.ldexp(rng.integers(1, 1 << 12, k).astype(np.float64), rng.integers(-30, 30, k))
    b[2 * k:3 * k] = sgn(k) * np.ldexp((rng.integers(1 << 40, 1 << 53, k) | 1).astype(np.float64),
                                        rng.integers(-80, 0, k))
    # cancellation: b = -(a moved by a few ulps)
    base = np.ldexp(rng.uniform(1, 2, k), rng.integers(-50, 50, k)) * sgn(k)
    steps = rng.integers(-40, 40, k)
    a[3 * k:4 * k] = base
    b[3 * k:4 * k] = -(base.view(np.int64) + steps).view(np.float64)
    # exponent gaps 40..75 (alignment and sticky bits)
    a[4 * k:5 * k] = sgn(k) * rng.uniform(1, 2, k)
    b[4 * k:5 * k] = sgn(k) * np.ldexp(rng.uniform(1, 2, k), -rng.integers(40, 76, k))
    # near overflow (products and sums) and near the subnormal range
    a[5 * k:6 * k] = sgn(k) * np.ldexp(rng.uniform(1, 2, k), rng.integers(1000, 1024, k))
    b[5 * k:6 * k] = sgn(k) * np.ldexp(rng.uniform(1, 2, k), rng.integers(-2, 24, k))
    a[6 * k:7 * k] = sgn(k) * np.ldexp(rng.uniform(1, 2, k), rng.integers(-1022, -990, k))
    b[6 * k:7 * k] = sgn(k) * np.ldexp(rng.uniform(1, 2, k), rng.integers(-40, 2, k))
    # all-ones significands (rounding carries into the exponent)
    ones = np.float64(2.0) - np.ldexp(1.0, -52)
    a[7 * k:8 * k] = sgn(k) * ones * np.ldexp(1.0, rng.integers(-20, 20, k))
    b[7 * k:8 * k] = sgn(k) * (1.0 + np.ldexp(rng.integers(0, 64, k).astype(np.float64), -52))
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.2250738585072009e-308,
                        2.2250738585072014e-308, np.finfo(np.float64).max, -np.finfo(np.float64).max, 1.0, -1.0,
                        0.5, 2.0 ** -1074 * 3, 1e-310])
    m = len(special)
    a[:m * m] = np.repeat(special, m)
    b[:m * m] = np.tile(special, m)
    return a, b
