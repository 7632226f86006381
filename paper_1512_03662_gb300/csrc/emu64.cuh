// IEEE 754 binary64 multiplication and addition, rounded to nearest with
// ties to even, computed on the integer pipes.
//
// The FP64 pipe of sm_103a issues two thread instructions per cycle per SM
// (one warp instruction every 64 cycles per scheduler), while a scheduler
// issues one warp instruction every cycle to the integer and FP32 pipes.
// The flux kernels are bound by the FP64 pipe with the other pipes almost
// idle, so part of their products and sums run here instead: each function
// returns the bits of the correctly rounded result that the DMUL / DADD
// instruction gives (IEEE 754-2008 Sect. 4.3.1, roundTiesToEven), so a
// kernel may move any of its products or sums between the two pipes
// without changing one bit of its output.
//
// Method (the textbook integer formulation of binary floating point, e.g.
// J.-M. Muller et al., Handbook of Floating-Point Arithmetic, 2nd ed., 2018,
// Sects. 7.2-7.3, and D. Goldberg, "What every computer scientist should
// know about floating-point arithmetic", ACM Comput. Surv. 23 (1991), on
// guard digits and the sticky bit):
//   product: the 53 x 53-bit significand product is formed exactly in four
//     32 x 32 -> 64-bit integer multiply-adds; its top 53 bits are the
//     significand, the next bit is the guard bit and every lower bit is
//     OR-ed into a sticky bit; round up when guard and (sticky or the
//     significand's last bit).
//   sum: the operand of smaller magnitude is aligned to the larger in a
//     64-bit frame with 10 bits below the significand; bits shifted out are
//     OR-ed into the last bit of the frame, which makes the frame value odd
//     whenever the sum is inexact, so no rounding boundary (all of them
//     multiples of 2^8 in the frame) can lie between it and the exact sum;
//     then normalisation and the same rounding rule as the product.
// Carries of the rounding step propagate into the exponent field, which
// also gives the correct infinity on overflow.
//
// The integer path handles normal and zero operands whose exact result is
// normal or zero.  mul_chk / add_chk compute without a branch and clear a
// caller's flag for everything else (subnormal operands or results,
// infinities, NaNs, overflow before rounding): the flux kernels check the
// flag once per evaluation and redo that evaluation on the FP64 pipe.
// mul_rn / add_rn, single operations, take a slow path that is the hardware
// instruction itself.  Both redo paths sit in functions that are never
// inlined, so that no FP64 instruction stands on the fast path, not even
// predicated off (a predicated-off FP64 instruction still occupies the FP64
// pipe).
//
// The functions compile for the host as well (plain C++ on the same
// integer steps), where tests check them bit for bit against the host's
// IEEE arithmetic.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define EMU_HD __host__ __device__ __forceinline__
#else
#define EMU_HD inline
#endif

namespace jfnk {
namespace emu {

EMU_HD uint32_t hi_word(double x) {
#if defined(__CUDA_ARCH__)
    return (uint32_t)__double2hiint(x);
#else
    uint64_t u;
    memcpy(&u, &x, 8);
    return (uint32_t)(u >> 32);
#endif
}

EMU_HD uint32_t lo_word(double x) {
#if defined(__CUDA_ARCH__)
    return (uint32_t)__double2loint(x);
#else
    uint64_t u;
    memcpy(&u, &x, 8);
    return (uint32_t)u;
#endif
}

EMU_HD double from_words(uint32_t hi, uint32_t lo) {
#if defined(__CUDA_ARCH__)
    return __hiloint2double((int)hi, (int)lo);
#else
    const uint64_t u = ((uint64_t)hi << 32) | lo;
    double x;
    memcpy(&x, &u, 8);
    return x;
#endif
}

EMU_HD double from_bits(uint64_t u) { return from_words((uint32_t)(u >> 32), (uint32_t)u); }

// low 32 bits of (hi:lo) >> s, 0 <= s < 32
EMU_HD uint32_t shr_pair(uint32_t lo, uint32_t hi, uint32_t s) {
#if defined(__CUDA_ARCH__)
    return __funnelshift_r(lo, hi, s);
#else
    return (uint32_t)((((uint64_t)hi << 32) | lo) >> s);
#endif
}

// number of leading zero bits of a nonzero 64-bit value
EMU_HD int clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return __builtin_clzll(x);
#endif
}

// a*b on the integer path, without a branch.  The return value is the
// correctly rounded product whenever a and b are normal or zero and the
// exact product is normal or zero; otherwise it is meaningless and ok is
// cleared (ok is never set, so a caller can check a whole sequence of
// operations once and redo it on the FP64 pipe where it failed).
EMU_HD double mul_chk(double a, double b, bool& ok) {
    const uint32_t ah = hi_word(a), al = lo_word(a), bh = hi_word(b), bl = lo_word(b);
    const uint32_t sign = (ah ^ bh) & 0x80000000u;
    // exponent fields in place (bits 20..30) and the product's before
    // normalisation; unsigned wrap-around rejects the out-of-range cases:
    // a and b normal, and the normalised exponent e0 (+1) within [1, 2046]
    const uint32_t ea = ah & 0x7ff00000u, eb = bh & 0x7ff00000u;
    const uint32_t e0 = ea + eb - 0x3ff00000u;
    const bool normal = (ea - 0x00100000u < 0x7fe00000u) & (eb - 0x00100000u < 0x7fe00000u) &
                        (e0 - 0x00100000u < 0x7fd00000u);
    // a zero times a finite number: a zero carrying the sign of the product
    const bool zero = ((((ah & 0x7fffffffu) | al) == 0u) | (((bh & 0x7fffffffu) | bl) == 0u)) &
                      (ea != 0x7ff00000u) & (eb != 0x7ff00000u);
    // significands with the hidden bit: (ma:al) and (mb:bl), 53 bits each
    const uint32_t ma = (ah & 0xfffffu) | 0x100000u, mb = (bh & 0xfffffu) | 0x100000u;
    // exact 106-bit product w3:w2:w1:w0 in four 32x32->64 multiply-adds
    const uint64_t t0 = (uint64_t)al * bl;
    const uint64_t t1 = (uint64_t)al * mb + (t0 >> 32);
    const uint64_t t2 = (uint64_t)ma * bl + (uint32_t)t1;
    const uint64_t t3 = (uint64_t)ma * mb + (t1 >> 32) + (t2 >> 32);
    const uint32_t w0 = (uint32_t)t0, w1 = (uint32_t)t2, w2 = (uint32_t)t3, w3 = (uint32_t)(t3 >> 32);
    // the product lies in [2^104, 2^106): s = 1 when bit 105 is set
    const uint32_t s = w3 >> 9;
    const uint32_t mlo = shr_pair(w1, w2, 20u + s);          // significand bits 0..31
    const uint32_t mhi = shr_pair(w2, w3, 20u + s);          // bits 32..52 (hidden bit at 20)
    // guard bit at the top of `rest`, the bits below it, w0 != 0 as bit 0;
    // round up (to nearest, ties to even) exactly when rest + 0x7fffffff +
    // the last significand bit carries out of 32 bits
    const uint32_t rest = (w1 << (12u - s)) | (uint32_t)(w0 != 0u);
    const uint32_t up = (uint32_t)(((uint64_t)rest + (0x7fffffffu + (mlo & 1u))) >> 32);
    // exponent field e0 + s: e0 + (s - 1) << 20 plus the hidden bit of mhi;
    // the rounding carry runs into the exponent (infinity on overflow)
    const uint32_t hi = sign + (e0 + (s << 20) - 0x00100000u) + mhi;
    const uint64_t bits = (((uint64_t)hi << 32) | mlo) + up;
    ok = ok & (normal | zero);
    return zero ? from_words(sign, 0u) : from_bits(bits);
}

// a+b on the integer path, without a branch; ok as for mul_chk (operands
// normal or zero, exact sum normal or zero).
EMU_HD double add_chk(double a, double b, bool& ok) {
    const uint32_t ah = hi_word(a), al = lo_word(a), bh = hi_word(b), bl = lo_word(b);
    const uint32_t am = ah & 0x7fffffffu, bm = bh & 0x7fffffffu;
    // x: the operand of larger magnitude (a on ties), y the other
    const bool swap = (bm > am) | ((bm == am) & (bl > al));
    const uint32_t xh = swap ? bh : ah, xl = swap ? bl : al;
    const uint32_t yh = swap ? ah : bh, yl = swap ? al : bl;
    const uint32_t ex = (xh >> 20) & 0x7ffu, ey = (yh >> 20) & 0x7ffu;
    const bool sub = ((ah ^ bh) & 0x80000000u) != 0u;
    // 64-bit frames: significand with hidden bit at bit 62, 10 bits below it
    const uint64_t X = ((uint64_t)((xh & 0xfffffu) | 0x100000u) << 42) | ((uint64_t)xl << 10);
    const uint64_t Y = ((uint64_t)((yh & 0xfffffu) | 0x100000u) << 42) | ((uint64_t)yl << 10);
    const uint32_t d = ex - ey < 63u ? ex - ey : 63u;          // Y >> 63 is 0: top bit at 62
    const uint64_t lost = Y & ((1ull << d) - 1ull);
    const uint64_t Ya = (Y >> d) | (uint64_t)(lost != 0ull);
    const uint64_t S0 = sub ? X - Ya : X + Ya;
    // normalise to bit 62: one place right after a carry (sticky kept),
    // left by the leading zeros after a cancellation
    const int lz = clz64(S0) - 1;                              // -1 .. 63 (63: S0 == 0)
    const uint64_t S = lz < 0 ? ((S0 >> 1) | (S0 & 1ull)) : (S0 << (uint32_t)(lz < 0 ? 0 : lz));
    const uint32_t e = ex - (uint32_t)lz;
    const uint32_t rem = (uint32_t)S & 0x3ffu;
    const uint64_t m = S >> 10;
    const uint64_t up = (uint64_t)((rem + (uint32_t)(m & 1ull)) > 0x200u);
    const uint64_t bits = ((((uint64_t)(xh & 0x80000000u)) << 32) | ((uint64_t)(e - 1u) << 52)) + m + up;
    // y == 0: the sum is x; two zeros of opposite signs give +0
    const bool yzero = ((yh & 0x7fffffffu) | yl) == 0u;
    const bool xzero = ((xh & 0x7fffffffu) | xl) == 0u;
    const bool normal = (ey != 0u) & (ex - 1u < 2046u);
    const bool exact0 = S0 == 0ull;                            // x - x: +0
    ok = ok & ((yzero & (ex != 0x7ffu)) | (normal & (exact0 | (e - 1u < 2046u))));
    const double viax = (sub & xzero) ? 0.0 : from_words(xh, xl);
    return yzero ? viax : (exact0 ? 0.0 : from_bits(bits));
}

// single operations with the range check: true and r = a*b (a+b) on the
// integer path; false (r meaningless) outside its range
EMU_HD bool mul_fast(double a, double b, double& r) {
    bool ok = true;
    r = mul_chk(a, b, ok);
    return ok;
}

EMU_HD bool add_fast(double a, double b, double& r) {
    bool ok = true;
    r = add_chk(a, b, ok);
    return ok;
}

#if defined(__CUDA_ARCH__)
__device__ __noinline__ double mul_slow(double a, double b) { return __dmul_rn(a, b); }
__device__ __noinline__ double add_slow(double a, double b) { return __dadd_rn(a, b); }
#else
inline double mul_slow(double a, double b) { return a * b; }
inline double add_slow(double a, double b) { return a + b; }
#endif

// a*b and a+b, correctly rounded, on the integer pipes
EMU_HD double mul_rn(double a, double b) {
    double r;
    if (mul_fast(a, b, r)) return r;
    return mul_slow(a, b);
}

EMU_HD double add_rn(double a, double b) {
    double r;
    if (add_fast(a, b, r)) return r;
    return add_slow(a, b);
}

// -b: the sign bit flips on the integer pipe
EMU_HD double neg(double b) { return from_words(hi_word(b) ^ 0x80000000u, lo_word(b)); }

// a - b
EMU_HD double sub_rn(double a, double b) { return add_rn(a, neg(b)); }
EMU_HD double sub_chk(double a, double b, bool& ok) { return add_chk(a, neg(b), ok); }

}  // namespace emu
}  // namespace jfnk
