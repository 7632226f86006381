// Shared device-side definitions of the JFNK library: grid descriptor,
// neighbour indexing with periodic / reflecting-wall ghosts, the van Leer
// slope, and deterministic block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "emu64.cuh"

namespace jfnk {

constexpr int kBlock = 256;          // threads per block of the pointwise kernels
constexpr int kRedBlocks = 1024;     // fixed block count of grid-stride reductions
constexpr int kMaxRedBlocks = 2048;  // cap of the occupancy-sized reduction grids

struct Grid {
    int ndim;
    int n[3];
    long long ncell;
    double dx[3], idx[3], idx2[3], tidx[3];   // tidx = 2 / dx
    double hidx[3];                           // 0.5 / dx
    int bc[3];                       // 0 periodic, 1 wall
    double gamma, gm1;
    double g[3];
    double hg[3];                    // g / 2 (the face density enters as the cell sum)
    double K0, chi_exp;
    int energy_form;                 // 0 internal e, 1 total eps_t
    double theta;
    // integer copies of the tests on the parameters above, so kernels branch
    // on them without FP64 compares: bit d of gmask = (g[d] != 0),
    // has_cond = (K0 != 0), chi3 = (chi_exp == 3)
    int gmask, has_cond, chi3;
    double igm1, igamma;             // 1/(gamma-1) = c_v and 1/gamma, formed on the host
};

inline void set_grid_flags(Grid& G) {
    G.gmask = 0;
    for (int d = 0; d < 3; ++d)
        if (G.g[d] != 0.0) G.gmask |= 1 << d;
    G.has_cond = G.K0 != 0.0;
    G.chi3 = G.chi_exp == 3.0;
    G.igm1 = 1.0 / G.gm1;
    G.igamma = 1.0 / G.gamma;
    for (int d = 0; d < 3; ++d) G.hg[d] = 0.5 * G.g[d];
}

struct Idx3 { int i[3]; };

// Launch shape of the cell kernels: x along threadIdx.x (coalesced), y and
// z from the grid, so no thread decomposes a flat index by division.
struct CellLaunch {
    dim3 grid, block;
};

inline CellLaunch cell_launch(const int n[3]) {
    int bx = 32;
    while (bx < n[0] && bx < 128) bx *= 2;
    int by = 128 / bx;
    CellLaunch L;
    L.block = dim3(bx, by, 1);
    L.grid = dim3((n[0] + bx - 1) / bx, (n[1] + by - 1) / by, n[2]);
    return L;
}

// Position of this thread in a cell_launch grid; false outside the grid.
__device__ __forceinline__ bool cell_pos(const int n[3], Idx3& P, long long& c) {
    P.i[0] = blockIdx.x * blockDim.x + threadIdx.x;
    P.i[1] = blockIdx.y * blockDim.y + threadIdx.y;
    P.i[2] = blockIdx.z;
    if (P.i[0] >= n[0] || P.i[1] >= n[1]) return false;
    c = ((long long)P.i[2] * n[1] + P.i[1]) * n[0] + P.i[0];
    return true;
}

// Position of this thread in tile `tile` of a cell_launch tiling (tiles in
// x, then y, then z order), for grid-stride kernels that visit several tiles
// per block; false outside the grid.
__device__ __forceinline__ bool cell_pos_tile(const int n[3], int tile, Idx3& P, long long& c) {
    const int gx = (n[0] + (int)blockDim.x - 1) / (int)blockDim.x;
    const int gy = (n[1] + (int)blockDim.y - 1) / (int)blockDim.y;
    const int r = tile / gx;
    P.i[0] = (tile - r * gx) * blockDim.x + threadIdx.x;
    P.i[1] = (r % gy) * blockDim.y + threadIdx.y;
    P.i[2] = r / gy;
    if (P.i[0] >= n[0] || P.i[1] >= n[1]) return false;
    c = ((long long)P.i[2] * n[1] + P.i[1]) * n[0] + P.i[0];
    return true;
}

__device__ __forceinline__ int block_linear() {
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

__device__ __forceinline__ int thread_linear() { return threadIdx.x + blockDim.x * threadIdx.y; }

__device__ __forceinline__ Idx3 decompose(const Grid& G, long long c) {
    Idx3 r;
    r.i[0] = (int)(c % G.n[0]);
    long long t = c / G.n[0];
    r.i[1] = (int)(t % G.n[1]);
    r.i[2] = (int)(t / G.n[1]);
    return r;
}

__device__ __forceinline__ long long flat(const Grid& G, int i0, int i1, int i2) {
    return ((long long)i2 * G.n[1] + i1) * G.n[0] + i0;
}

// Cell-quantity index of position k along a direction of size n: periodic
// wrap, or mirror about the wall faces (k -> -k-1, k -> 2n-1-k).  Stencil
// offsets never exceed the grid size (n >= 4, |offset| <= 3), so one
// conditional wrap replaces an integer modulo.
__device__ __forceinline__ int cell_map(int k, int n, int bc) {
    if (bc == 0) return k < 0 ? k + n : (k >= n ? k - n : k);
    if (k < 0) return -k - 1;
    if (k >= n) return 2 * n - 1 - k;
    return k;
}

// Load of a cell quantity at (pos + off) with ghost mapping in every direction.
__device__ __forceinline__ double load_cell(const Grid& G, const double* __restrict__ f, const Idx3& p,
                                            int o0, int o1, int o2) {
    int a = cell_map(p.i[0] + o0, G.n[0], G.bc[0]);
    int b = cell_map(p.i[1] + o1, G.n[1], G.bc[1]);
    int c = cell_map(p.i[2] + o2, G.n[2], G.bc[2]);
    return __ldg(f + flat(G, a, b, c));
}

// Load of the velocity normal to the faces of direction `c` at slot
// (pos + off): odd mirror about the wall faces, zero on both wall faces;
// cell mapping in the other directions.
__device__ __forceinline__ double load_normal(const Grid& G, const double* __restrict__ u, int c, const Idx3& p,
                                              int o0, int o1, int o2) {
    int k[3] = {p.i[0] + o0, p.i[1] + o1, p.i[2] + o2};
    long long flip = 0;                 // sign-bit mask of the odd mirror
    for (int d = 0; d < 3; ++d) {
        if (d == c && G.bc[d] == 1) {
            int n = G.n[d];
            int kk = k[d];
            if (kk == 0 || kk == n) return 0.0;
            if (kk < 0) { kk = -kk; flip = (long long)0x8000000000000000ULL; }
            else if (kk > n) { kk = 2 * n - kk; flip = (long long)0x8000000000000000ULL; }
            k[d] = kk;
        } else {
            k[d] = cell_map(k[d], G.n[d], G.bc[d]);
        }
    }
    double v = __ldg(u + flat(G, k[0], k[1], k[2]));
    // sign flip on the sign bit (integer pipe) instead of an FP64 multiply
    return __longlong_as_double(__double_as_longlong(v) ^ flip);
}

// ---------------------------------------------------------------------------
// Branch-free neighbour addressing of the residual kernels.  Offsets are flat
// offsets relative to the thread's own cell (pointers given at that cell):
// k * stride inside the grid; the periodic wrap or the wall mirror changes
// them only where P + k e_d leaves the grid.  The boundary type is a kernel
// parameter (uniform across the warp) and the position tests are selects,
// so no thread-dependent branch splits a warp.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int grid_stride(const Grid& G, int d) {
    return d == 0 ? 1 : (d == 1 ? G.n[0] : G.n[0] * G.n[1]);
}

// offset of the cell quantity at P + k e_d, 1 <= |k| <= 3 (k = 0: 0)
__device__ __forceinline__ int cell_off(const Grid& G, const Idx3& P, int d, int k) {
    const int i = P.i[d], n = G.n[d];
    int m = k;
    if (k < 0) {
        // i + k < 0: periodic i + k + n, wall mirror -(i + k) - 1
        const int w = G.bc[d] == 0 ? k + n : -2 * i - k - 1;
        m = i + k < 0 ? w : k;
    } else if (k > 0) {
        // i + k >= n: periodic i + k - n, wall mirror 2n - 1 - (i + k)
        const int w = G.bc[d] == 0 ? k - n : 2 * n - 1 - 2 * i - k;
        m = i + k >= n ? w : k;
    }
    return m * grid_stride(G, d);
}

// velocity normal to direction c at face slot P + k e_c (uc at the thread's
// own slot): with walls the odd mirror (sign flip on the integer pipe) and
// zero on both wall faces; periodic faces wrap like cells
__device__ __forceinline__ double normal_along(const Grid& G, const double* __restrict__ uc, const Idx3& P, int c,
                                               int k) {
    if (G.bc[c] == 0) return __ldg(uc + cell_off(G, P, c, k));
    const int i = P.i[c], n = G.n[c], kk = i + k;
    int m = k;
    bool flip = false, zero = false;
    if (k <= 0) zero = kk == 0;
    if (k >= 0) zero = zero | (kk == n);
    if (k < 0) {
        flip = kk < 0;
        m = flip ? -2 * i - k : k;                  // slot -kk
    } else if (k > 0) {
        flip = kk > n;
        m = flip ? 2 * n - 2 * i - k : k;           // slot 2n - kk
    }
    const double v = __ldg(uc + (zero ? 0 : m) * grid_stride(G, c));   // the own slot where the value is zero
    const long long f = flip ? (long long)0x8000000000000000ULL : 0ll;
    return zero ? 0.0 : __longlong_as_double(__double_as_longlong(v) ^ f);
}

// velocity normal to direction c at slot P + k e_d, d != c (tangential
// offsets map like cells); zero when the thread's own slot is a wall face
// of c
__device__ __forceinline__ double normal_across(const Grid& G, const double* __restrict__ uc, const Idx3& P, int c,
                                                int d, int k) {
    const bool wall = (G.bc[c] == 1) & (P.i[c] == 0);
    const double v = __ldg(uc + cell_off(G, P, d, k));
    return wall ? 0.0 : v;
}

// face quantity of direction d at the upper face of the cell (slot P + e_d):
// zero at an upper wall
__device__ __forceinline__ double face_up_at(const Grid& G, const double* __restrict__ f, const Idx3& P, int d) {
    const bool top = (G.bc[d] == 1) & (P.i[d] + 1 == G.n[d]);
    const double v = __ldg(f + (top ? 0 : cell_off(G, P, d, 1)));
    return top ? 0.0 : v;
}

// True when slot p is the wall face of direction c.
__device__ __forceinline__ bool is_wall_slot(const Grid& G, int c, const Idx3& p) {
    return G.bc[c] == 1 && p.i[c] == 0;
}

// van Leer (1974) harmonic slope: 2ab/(a+b) if ab > 0 else 0.
__device__ __forceinline__ double vanleer(double a, double b) {
    double ab = a * b;
    return ab > 0.0 ? (2.0 * ab) / (a + b) : 0.0;
}

// Sign tests on the bit pattern (integer pipe; the flux kernels are bound by
// the FP64 pipe).  For every non-NaN x: nonneg(x) == (x >= 0.0) (both zeros
// count), positive(x) == (x > 0.0).
// Both on the two 32-bit words: as 64-bit tests of the whole pattern the
// compiler turned nonneg into an FP64 compare (DSETP) on the FP64 pipe.
__device__ __forceinline__ bool nonneg(double x) {
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    return (hi >= 0) | ((((unsigned)hi << 1) | lo) == 0u);
}
__device__ __forceinline__ bool positive(double x) {
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    return (hi > 0) | ((hi == 0) & (lo != 0u));
}

// Upwind reconstruction without divergent branches.  With q_near the cell
// on the upwind side of the face, q_far its other neighbour and q_other the
// cell across the face, the face value is
//     q_near + s/2,   s = vanleer(q_near - q_far, q_other - q_near).
// For the right-hand (negative speed) case this is q_R - s_R/2 exactly,
// because the two differences change sign, which is exact, and s/2 =
// ab/(a+b) exactly (scaling by two commutes with rounding).  The value is
// returned split as q + num/den: num = ab and den = a + b where the limiter
// is on, num = 0 and den = 1 where it is off, so every thread divides (no
// warp split) and a thread can form all its reciprocals together.
// The arithmetic of one thread's evaluation, on the FP64 pipe (FpOps:
// plain operators, which the compiler may fuse into FMAs) or on the integer
// pipes (IntOps: emu64.cuh, the correctly rounded results of the unfused
// operations, IM for the products and IA for the sums and differences).
// The FP64 pipe of sm_103a issues one warp instruction per 64 cycles per
// scheduler, so the FP64-bound kernels move part of their arithmetic to the
// idle integer pipes.  IntOps collects one validity flag for the whole
// sequence (operands and results normal or zero) instead of branching per
// operation, so a kernel checks it once and redoes the thread's work with
// FpOps where it failed; no branch splits the integer sequence, and the
// compiler can interleave its independent chains.
struct FpOps {
    __device__ __forceinline__ double mul(double a, double b) { return a * b; }
    __device__ __forceinline__ double add(double a, double b) { return a + b; }
    __device__ __forceinline__ double sub(double a, double b) { return a - b; }
    __device__ __forceinline__ void require(bool) {}
    __device__ __forceinline__ bool valid() const { return true; }
    static constexpr bool checked = false;
};

template <bool IM, bool IA>
struct IntOps {
    bool ok = true;
    __device__ __forceinline__ double mul(double a, double b) {
        if constexpr (IM) return emu::mul_chk(a, b, ok);
        else return a * b;
    }
    __device__ __forceinline__ double add(double a, double b) {
        if constexpr (IA) return emu::add_chk(a, b, ok);
        else return a + b;
    }
    __device__ __forceinline__ double sub(double a, double b) {
        if constexpr (IA) return emu::sub_chk(a, b, ok);
        else return a - b;
    }
    __device__ __forceinline__ void require(bool c) { ok = ok & c; }
    __device__ __forceinline__ bool valid() const { return ok; }
    static constexpr bool checked = true;
};

struct Upw { double q, num, den; };
template <class O = FpOps>
__device__ __forceinline__ Upw upwind_parts(double q_near, double q_far, double q_other, O&& ops = O()) {
    const double a = ops.sub(q_near, q_far);
    const double b = ops.sub(q_other, q_near);
    const double ab = ops.mul(a, b);
    const bool on = positive(ab);
    Upw u;
    u.q = q_near;
    u.num = on ? ab : 0.0;
    u.den = on ? ops.add(a, b) : 1.0;
    return u;
}

// Float <-> double conversions on the integer pipe.  On sm_103a the
// conversion instructions run on the FP64 pipe (2 per cycle per SM), and a
// predicated-off instruction still occupies it, so these handle every
// input in integer arithmetic, with no FP64 instruction on any path, and
// give the bits of the conversion instructions (IEEE 754: the float->double
// conversion is exact, double->float rounds to nearest, ties to even; NaNs
// stay NaNs).

// (double)f
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u, mag = u & 0x7fffffffu, m = u & 0x7fffffu;
    const unsigned e = mag >> 23;
    unsigned hi, lo;
    if (e - 1u < 254u) {                              // normal: rebias by 1023 - 127 = 896
        hi = sign | ((mag >> 3) + 0x38000000u);
        lo = u << 29;
    } else if (e == 255u) {                           // infinity or NaN (quiet)
        hi = sign | 0x7ff00000u | (m >> 3) | (m ? 0x00080000u : 0u);
        lo = m << 29;
    } else if (m == 0u) {                             // zero
        hi = sign;
        lo = 0u;
    } else {                                          // subnormal float: a normal double
        const int k = 31 - __clz(m);                  // leading bit of m (value m 2^-149)
        const unsigned long long t = ((unsigned long long)m << (52 - k)) & 0xfffffffffffffULL;
        hi = sign | ((unsigned)(k + 874) << 20) | (unsigned)(t >> 32);
        lo = (unsigned)t;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// (float)x, rounded to nearest, ties to even
__device__ __forceinline__ float d2f_rn(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u, e = (hi >> 20) & 0x7ffu;
    unsigned b;
    if (e - 897u <= 1150u - 897u) {                   // normal float result: keep 23 bits, round on 29
        const unsigned m23 = ((hi & 0xfffffu) << 3) | (lo >> 29);
        const unsigned rem = lo & 0x1fffffffu;
        b = (((e - 896u) << 23) | m23) + ((rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) ? 1u : 0u);
    } else if (e == 0x7ffu) {                         // infinity or NaN (quiet)
        const bool nan = (hi & 0xfffffu) | lo;
        b = 0x7f800000u | (nan ? 0x00400000u | ((hi & 0xfffffu) << 3) | (lo >> 29) : 0u);
    } else if (e > 1150u) {                           // beyond the float range: infinity
        b = 0x7f800000u;
    } else if (e >= 873u) {                           // subnormal float (or the smallest normal)
        const unsigned long long m53 = (1ULL << 52) | ((unsigned long long)(hi & 0xfffffu) << 32) | lo;
        const unsigned s = 926u - e;                  // 30 .. 53
        const unsigned long long v = m53 >> s, r = m53 & ((1ULL << s) - 1ULL), half = 1ULL << (s - 1u);
        b = (unsigned)v + ((r > half || (r == half && (v & 1ULL))) ? 1u : 0u);
    } else {                                          // below half the smallest subnormal: zero
        b = 0u;
    }
    return __uint_as_float(sign | b);
}

// between the basis precision and double
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f2d_exact(x); }
template <typename T> __device__ __forceinline__ T from_f64(double x);
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_f64<float>(double x) { return d2f_rn(x); }

// 1/d from the hardware approximation r0 (rcp.approx.ftz.f64, MUFU pipe)
// refined by one third-order step of the reciprocal iteration: with
// e = 1 - d r0 the exact reciprocal is r0 (1 + e + e^2 + e^3 / (1 - e)), so
// r = r0 + r0 (e + e^2) leaves a relative error of about e^3 (the series
// form of Newton-Raphson refinement, P. Markstein, IBM J. Res. Dev. 34
// (1990) 111-119, taken one term further).  Three fused multiply-adds
// instead of the four of two quadratic steps; the result is within one ulp
// of the correctly rounded 1/d (the error before the last rounding is far
// below half an ulp).  Valid for normal d whose reciprocal is normal (the
// approximation flushes subnormals); callers guarantee the range.
__device__ __forceinline__ double recip_nr(double d) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    const double e = fma(-d, r, 1.0);
    return fma(fma(e, e, e), r, r);
}

// r[i] = 1/d[i], i < K, with one reciprocal: Montgomery's simultaneous
// inversion (P. L. Montgomery, Math. Comp. 48 (1987) 243-264):
// prefix products p_i = d_0 ... d_i, one reciprocal 1/p_{K-1} (recip_nr),
// then going down r_i = p_{i-1} / p_i and 1/p_{i-1} = d_i / p_i.  It costs
// 3(K-1) multiplications instead of K-1 divisions; each result carries at
// most 3K + 1 roundings instead of one.  The prefix products stay in the
// normal range when every |d_i| lies in [2^-R, 2^R), R = 1000/K (exponent
// test on the high word, integer pipe); otherwise the thread divides K
// times.
// With checked Ops (IntOps) the range test goes into its flag and there is
// no division fallback: the caller redoes the whole evaluation.
template <int K, class O = FpOps>
__device__ __forceinline__ void recip_all(const double (&d)[K], double (&r)[K], O&& ops = O()) {
    constexpr unsigned R = 1000u / K;
    bool ok = true;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const unsigned e = ((unsigned)__double2hiint(d[i]) >> 20) & 0x7ffu;
        ok = ok & (e - (1023u - R) < 2u * R);
    }
    if constexpr (std::remove_reference_t<O>::checked) ops.require(ok);
    if (std::remove_reference_t<O>::checked || ok) {
        double p[K];
        p[0] = d[0];
#pragma unroll
        for (int i = 1; i < K; ++i) p[i] = ops.mul(p[i - 1], d[i]);
        double inv = recip_nr(p[K - 1]);
#pragma unroll
        for (int i = K - 1; i > 0; --i) {
            r[i] = ops.mul(inv, p[i - 1]);
            inv = ops.mul(inv, d[i]);
        }
        r[0] = inv;
    } else {
#pragma unroll
        for (int i = 0; i < K; ++i) r[i] = 1.0 / d[i];
    }
}

// Error-free transformations (Knuth's TwoSum, FMA-based TwoProduct) used by
// the float basis and the float preconditioner output: a dot product
// accumulated as an unevaluated pair (sum, err) is as accurate as one
// accumulated in twice the working precision (Ogita, Rump & Oishi,
// "Accurate sum and dot product", 2005), without touching the FP64 pipe
// inside the loop.
struct CompF {
    float s, e;
};

// (explicitly rounded intrinsics: the compiler must not contract these into FMAs)
__device__ __forceinline__ void comp_add(CompF& a, float p) {
    float t = __fadd_rn(a.s, p);
    float bp = __fsub_rn(t, a.s);
    a.e = __fadd_rn(a.e, __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
    a.s = t;
}

__device__ __forceinline__ void comp_fma(CompF& a, float x, float y) {
    float p = __fmul_rn(x, y);
    float err = fmaf(x, y, -p);
    comp_add(a, p);
    a.e = __fadd_rn(a.e, err);
}

// Squares of float values of magnitude m stay normal floats when m lies in
// [2^-60, 2^60): a thread whose largest |x| lies outside that range redoes
// its sum of squares in double (a second loop, taken by no thread in
// practice); otherwise the compensated float sum is exact to about 2^-44 of
// the result.  The check runs once per thread, after the loop, so the loop
// itself has no FP64 instruction.
__device__ __forceinline__ bool sq_range_unsafe(float maxabs) {
    return maxabs >= 0x1p60f || (maxabs > 0.f && maxabs < 0x1p-60f);
}

template <typename T> struct Acc { typedef double type; };

// Block-wide sum of one double per thread; result valid in thread 0.
template <int BS>
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int t = threadIdx.x + blockDim.x * threadIdx.y;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = t & 31, w = t >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = (t < BS / 32) ? sh[t] : 0.0;
    if (w == 0) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

template <int BS>
__device__ __forceinline__ double block_max(double v, double* sh) {
    const int t = threadIdx.x + blockDim.x * threadIdx.y;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    int lane = t & 31, w = t >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = (t < BS / 32) ? sh[t] : 0.0;
    if (w == 0) {
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;
}

template <typename T> __device__ __forceinline__ double to_d(T v) { return (double)v; }

}  // namespace jfnk
