// GMRES kernels (paper Sect. 4.1, Eq. forcing_term; restarted GMRES of Saad &
// Schultz 1986 with classical Gram-Schmidt):
//   * multi-dot: h_i = <v_i, w> for all basis vectors in ONE pass over w,
//     accumulated in double whatever the storage type;
//   * AXPY + norm: w -= sum_i h_i s_i v_i and ||w||^2 in the same pass;
//   * lazy normalisation: v_{j+1} keeps the unnormalised w, its scale
//     s_{j+1} = 1/||w|| is applied by every reader, which saves a pass;
//   * Givens rotations and the triangular solve run on the device in one
//     thread (m <= 64), so the host only reads the residual estimate.
// Reductions are two-stage with a fixed block count and a fixed summation
// order, so results are bit-reproducible from run to run.
#include "common.cuh"
#include "kernels.h"

namespace jfnk {

// Grid of a grid-stride reduction: as many blocks as are resident on all
// SMs at once (one wave: no tail wave, every SM equally loaded), capped at
// kMaxRedBlocks.  Fixed per kernel and device, so the summation order and
// the results stay reproducible.
static int red_grid(const void* fn) {
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kBlock, 0);
    long long g = (long long)(nsm > 0 ? nsm : 1) * (occ > 0 ? occ : 1);
    return (int)(g < kMaxRedBlocks ? g : kMaxRedBlocks);
}

// one cached grid per kernel (the kernel is the template argument, so each
// instantiation has its own thread-safe static)
template <auto FN>
static int cached_grid() {
    static const int g = red_grid((const void*)FN);
    return g;
}

__global__ void k_finalize(const double* __restrict__ partials, int n, double* scal, int slot, int op) {
    __shared__ double sh[32];
    double v = (op == 2) ? 0.0 : 0.0;
    bool nan = false;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double x = partials[i];
        if (!(x == x)) nan = true;
        if (op == 2) v = fmax(v, x); else v += x;
    }
    double r = (op == 2) ? block_max<1024>(v, sh) : block_sum<1024>(v, sh);
    int anynan = __syncthreads_or(nan);
    if (threadIdx.x == 0) {
        if (anynan) r = __longlong_as_double(0x7ff8000000000000ULL);
        scal[slot] = (op == 0) ? sqrt(r) : r;
    }
}

void launch_finalize(const double* partials, int n, double* scal, int slot, int op, cudaStream_t s) {
    ++g_launch_count;
    k_finalize<<<1, 1024, 0, s>>>(partials, n, scal, slot, op);
}

__global__ void k_delta(double* scal, double lambda, int pert) {
    double zn = scal[kSlotZnorm];
    double d;
    if (pert == 0) {
        d = lambda * (lambda + scal[kSlotXhatNorm] / zn);
    } else {
        double uv = scal[kSlotTmp];
        double sgn = uv >= 0.0 ? 1.0 : -1.0;
        d = lambda * (1e-12 / lambda + fabs(uv) / (zn * zn)) * sgn;
    }
    scal[kSlotDelta] = d;
    scal[kSlotInvDelta] = 1.0 / d;
}

void launch_delta(double* scal, double lambda, int pert, cudaStream_t s) { k_delta<<<1, 1, 0, s>>>(scal, lambda, pert); }

// partial sums of x_i^2: in double for a double x; for a float x as a
// compensated float pair per thread (no FP64 instruction per element),
// converted to double once per thread, or redone in double by a thread whose
// values are too large or too small for float squares (sq_range_unsafe)
template <typename T>
__global__ void k_norm2(const T* __restrict__ x, long long n, double* __restrict__ partials) {
    __shared__ double sh[32];
    double acc = 0.0;
    CompF accf = {0.f, 0.f};
    float mx = 0.f;
    const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
    for (long long i = i0; i < n; i += st) {
        if (sizeof(T) == 8) {
            const double v = (double)x[i];
            acc += v * v;
        } else {
            const float v = (float)x[i];
            comp_fma(accf, v, v);
            mx = fmaxf(mx, fabsf(v));
        }
    }
    if (sizeof(T) != 8) {
        if (sq_range_unsafe(mx)) {
            for (long long i = i0; i < n; i += st) {
                const double v = (double)x[i];
                acc += v * v;
            }
        } else {
            acc = (double)accf.s + (double)accf.e;
        }
    }
    double s = block_sum<kBlock>(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <typename T>
void launch_norm2_partials(const T* x, long long n, double* partials, cudaStream_t s) {
    ++g_launch_count;
    k_norm2<T><<<kRedBlocks, kBlock, 0, s>>>(x, n, partials);
}
template void launch_norm2_partials<double>(const double*, long long, double*, cudaStream_t);
template void launch_norm2_partials<float>(const float*, long long, double*, cudaStream_t);

// partial sums of (a_i * ainv_i) * b_i  (used for x^ . z with x^ = X R^-1)
template <typename T>
__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ ainv, const T* __restrict__ b,
                      long long n, double* __restrict__ partials) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (a[i] * ainv[i]) * (double)b[i];
    double s = block_sum<kBlock>(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <typename T>
void launch_dot_partials(const double* a, const double* ainv, const T* b, long long n, double* partials,
                         cudaStream_t s) {
    ++g_launch_count;
    k_dot<T><<<kRedBlocks, kBlock, 0, s>>>(a, ainv, b, n, partials);
}
template void launch_dot_partials<double>(const double*, const double*, const double*, long long, double*, cudaStream_t);
template void launch_dot_partials<float>(const double*, const double*, const float*, long long, double*, cudaStream_t);

// one pass over w: partials[blk * NV + i] = sum over the block's elements of v_i * w
template <typename T, int NV>
__global__ void k_multidot(const T* __restrict__ V, long long ld, const T* __restrict__ w, long long n,
                           double* __restrict__ partials) {
    __shared__ double sh[32];
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double wk = (double)w[k];
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] += (double)V[i * ld + k] * wk;
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double s = block_sum<kBlock>(acc[i], sh);
        if (threadIdx.x == 0) partials[blockIdx.x * NV + i] = s;
    }
}

// float basis: compensated FP32 accumulation per thread, double per block
template <int NV>
__global__ void k_multidot_f32(const float* __restrict__ V, long long ld, const float* __restrict__ w, long long n,
                               double* __restrict__ partials) {
    __shared__ double sh[32];
    CompF acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = CompF{0.f, 0.f};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        float wk = w[k];
#pragma unroll
        for (int i = 0; i < NV; ++i) comp_fma(acc[i], V[i * ld + k], wk);
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double s = block_sum<kBlock>((double)acc[i].s + (double)acc[i].e, sh);
        if (threadIdx.x == 0) partials[blockIdx.x * NV + i] = s;
    }
}

// The same with 16-byte loads: each thread takes four consecutive elements
// per step, which keeps enough bytes in flight per SM to cover HBM latency
// when the basis is short (one load instruction per vector per four
// elements).  Needs ld % 4 == 0 and 16-byte aligned V and w; the n % 4 tail
// is summed element by element.
template <int NV>
__global__ void __launch_bounds__(kBlock) k_multidot_f32v(const float* __restrict__ V, long long ld,
                                                          const float* __restrict__ w, long long n,
                                                          double* __restrict__ partials) {
    __shared__ double sh[32];
    CompF acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = CompF{0.f, 0.f};
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n4 = n >> 2;
    const float4* w4 = reinterpret_cast<const float4*>(w);
    for (long long k = t0; k < n4; k += stride) {
        const float4 wk = w4[k];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const float4 v = reinterpret_cast<const float4*>(V + i * ld)[k];
            comp_fma(acc[i], v.x, wk.x);
            comp_fma(acc[i], v.y, wk.y);
            comp_fma(acc[i], v.z, wk.z);
            comp_fma(acc[i], v.w, wk.w);
        }
    }
    for (long long k = 4 * n4 + t0; k < n; k += stride) {
        const float wk = w[k];
#pragma unroll
        for (int i = 0; i < NV; ++i) comp_fma(acc[i], V[i * ld + k], wk);
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double s = block_sum<kBlock>((double)acc[i].s + (double)acc[i].e, sh);
        if (threadIdx.x == 0) partials[blockIdx.x * NV + i] = s;
    }
}

// generic fallback for any count: loops over groups of 8
template <typename T>
__global__ void k_multidot_group(const T* __restrict__ V, long long ld, int i0, int ni, int nvtot,
                                 const T* __restrict__ w, long long n, double* __restrict__ partials) {
    __shared__ double sh[32];
    double acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double wk = (double)w[k];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (i < ni) acc[i] += (double)V[(i0 + i) * ld + k] * wk;
    }
    for (int i = 0; i < ni; ++i) {
        double s = block_sum<kBlock>(acc[i], sh);
        if (threadIdx.x == 0) partials[blockIdx.x * nvtot + i0 + i] = s;
    }
}

static inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <typename T>
int launch_multidot(const T* V, long long ld, int nv, const T* w, long long n, double* partials, cudaStream_t s) {
    if (sizeof(T) == 4 && nv <= 32) {
        const float* Vf = (const float*)V;
        const float* wf = (const float*)w;
        const bool vec = ld % 4 == 0 && aligned16(V) && aligned16(w);
        int g = 0;
        ++g_launch_count;
        switch (nv) {
#define CASEF(N)                                                                                   \
    case N:                                                                                        \
        if (vec) {                                                                                 \
            g = cached_grid<k_multidot_f32v<N>>();                                                 \
            k_multidot_f32v<N><<<g, kBlock, 0, s>>>(Vf, ld, wf, n, partials);                       \
        } else {                                                                                   \
            g = cached_grid<k_multidot_f32<N>>();                                                  \
            k_multidot_f32<N><<<g, kBlock, 0, s>>>(Vf, ld, wf, n, partials);                        \
        }                                                                                          \
        return g;
            CASEF(1) CASEF(2) CASEF(3) CASEF(4) CASEF(5) CASEF(6) CASEF(7) CASEF(8)
            CASEF(9) CASEF(10) CASEF(11) CASEF(12) CASEF(13) CASEF(14) CASEF(15) CASEF(16)
            CASEF(17) CASEF(18) CASEF(19) CASEF(20) CASEF(21) CASEF(22) CASEF(23) CASEF(24)
            CASEF(25) CASEF(26) CASEF(27) CASEF(28) CASEF(29) CASEF(30) CASEF(31) CASEF(32)
#undef CASEF
        }
    }
    int g = 0;
    switch (nv) {
#define CASE(N)                                                                                    \
    case N:                                                                                        \
        ++g_launch_count;                                                                          \
        g = cached_grid<k_multidot<T, N>>();                                                       \
        k_multidot<T, N><<<g, kBlock, 0, s>>>(V, ld, w, n, partials);                               \
        return g;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
        CASE(9) CASE(10) CASE(11) CASE(12) CASE(13) CASE(14) CASE(15) CASE(16)
#undef CASE
        default:
            g = cached_grid<k_multidot_group<T>>();
            for (int i0 = 0; i0 < nv; i0 += 8) {
                int ni = nv - i0 < 8 ? nv - i0 : 8;
                ++g_launch_count;
                k_multidot_group<T><<<g, kBlock, 0, s>>>(V, ld, i0, ni, nv, w, n, partials);
            }
            return g;
    }
}
template int launch_multidot<double>(const double*, long long, int, const double*, long long, double*, cudaStream_t);
template int launch_multidot<float>(const float*, long long, int, const float*, long long, double*, cudaStream_t);

// hcol[i] (+)= vscale[i] * sum_b partials[b * nv + i]; one block per i
__global__ void k_multidot_finalize(const double* __restrict__ partials, int nblocks, int nv,
                                    const double* __restrict__ vscale, double* hcol, int accumulate) {
    __shared__ double sh[32];
    int i = blockIdx.x;
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[b * nv + i];
    double r = block_sum<kBlock>(v, sh);
    if (threadIdx.x == 0) {
        double h = r * vscale[i];
        hcol[i] = accumulate ? hcol[i] + h : h;
    }
}

void launch_multidot_finalize(const double* partials, int nblocks, int nv, const double* vscale, double* hcol,
                              int accumulate, cudaStream_t s) {
    ++g_launch_count;
    k_multidot_finalize<<<nv, kBlock, 0, s>>>(partials, nblocks, nv, vscale, hcol, accumulate);
}

// w -= sum_i (h_i s_i) v_i ; partial ||w||^2
template <typename T, int NV>
__global__ void k_axpy_norm(T* __restrict__ w, const T* __restrict__ V, long long ld, const double* __restrict__ hcol,
                            const double* __restrict__ vscale, long long n, double* __restrict__ partials) {
    __shared__ double sh[32];
    __shared__ double coef[64];
    if (threadIdx.x < NV) coef[threadIdx.x] = hcol[threadIdx.x] * vscale[threadIdx.x];
    __syncthreads();
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double x = (double)w[k];
#pragma unroll
        for (int i = 0; i < NV; ++i) x -= coef[i] * (double)V[i * ld + k];
        T xs = (T)x;
        w[k] = xs;
        double xd = (double)xs;
        acc += xd * xd;
    }
    double s = block_sum<kBlock>(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <typename T>
__global__ void k_axpy_norm_dyn(T* __restrict__ w, const T* __restrict__ V, long long ld, int nv,
                                const double* __restrict__ hcol, const double* __restrict__ vscale, long long n,
                                double* __restrict__ partials) {
    __shared__ double sh[32];
    __shared__ double coef[64];
    if (threadIdx.x < nv) coef[threadIdx.x] = hcol[threadIdx.x] * vscale[threadIdx.x];
    __syncthreads();
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double x = (double)w[k];
        for (int i = 0; i < nv; ++i) x -= coef[i] * (double)V[i * ld + k];
        T xs = (T)x;
        w[k] = xs;
        double xd = (double)xs;
        acc += xd * xd;
    }
    double s = block_sum<kBlock>(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// float basis: w -= sum_i c_i v_i with c_i split into float hi + lo parts and
// the sum kept as a compensated pair; ||w||^2 of the rounded result, compensated.
template <int NV>
__global__ void k_axpy_norm_f32(float* __restrict__ w, const float* __restrict__ V, long long ld,
                                const double* __restrict__ hcol, const double* __restrict__ vscale, long long n,
                                double* __restrict__ partials) {
    __shared__ double sh[32];
    __shared__ float chi[32], clo[32];
    if (threadIdx.x < NV) {
        double c = -(hcol[threadIdx.x] * vscale[threadIdx.x]);
        float h = (float)c;
        chi[threadIdx.x] = h;
        clo[threadIdx.x] = (float)(c - (double)h);
    }
    __syncthreads();
    CompF nrm{0.f, 0.f};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        CompF x{w[k], 0.f};
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float v = V[i * ld + k];
            comp_fma(x, chi[i], v);
            x.e = fmaf(clo[i], v, x.e);
        }
        float xs = x.s + x.e;
        w[k] = xs;
        comp_fma(nrm, xs, xs);
    }
    double s = block_sum<kBlock>((double)nrm.s + (double)nrm.e, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// The same with 16-byte loads and stores (four consecutive elements per
// thread and step); needs ld % 4 == 0 and 16-byte aligned w and V.
template <int NV>
__global__ void __launch_bounds__(kBlock) k_axpy_norm_f32v(float* __restrict__ w, const float* __restrict__ V,
                                                           long long ld, const double* __restrict__ hcol,
                                                           const double* __restrict__ vscale, long long n,
                                                           double* __restrict__ partials) {
    __shared__ double sh[32];
    __shared__ float chi[32], clo[32];
    if (threadIdx.x < NV) {
        double c = -(hcol[threadIdx.x] * vscale[threadIdx.x]);
        float h = (float)c;
        chi[threadIdx.x] = h;
        clo[threadIdx.x] = (float)(c - (double)h);
    }
    __syncthreads();
    CompF nrm{0.f, 0.f};
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n4 = n >> 2;
    float4* w4 = reinterpret_cast<float4*>(w);
    for (long long k = t0; k < n4; k += stride) {
        const float4 wk = w4[k];
        CompF x0{wk.x, 0.f}, x1{wk.y, 0.f}, x2{wk.z, 0.f}, x3{wk.w, 0.f};
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const float4 v = reinterpret_cast<const float4*>(V + i * ld)[k];
            const float ch = chi[i], cl = clo[i];
            comp_fma(x0, ch, v.x);
            x0.e = fmaf(cl, v.x, x0.e);
            comp_fma(x1, ch, v.y);
            x1.e = fmaf(cl, v.y, x1.e);
            comp_fma(x2, ch, v.z);
            x2.e = fmaf(cl, v.z, x2.e);
            comp_fma(x3, ch, v.w);
            x3.e = fmaf(cl, v.w, x3.e);
        }
        float4 o;
        o.x = x0.s + x0.e;
        o.y = x1.s + x1.e;
        o.z = x2.s + x2.e;
        o.w = x3.s + x3.e;
        w4[k] = o;
        comp_fma(nrm, o.x, o.x);
        comp_fma(nrm, o.y, o.y);
        comp_fma(nrm, o.z, o.z);
        comp_fma(nrm, o.w, o.w);
    }
    for (long long k = 4 * n4 + t0; k < n; k += stride) {
        CompF x{w[k], 0.f};
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float v = V[i * ld + k];
            comp_fma(x, chi[i], v);
            x.e = fmaf(clo[i], v, x.e);
        }
        float xs = x.s + x.e;
        w[k] = xs;
        comp_fma(nrm, xs, xs);
    }
    double sum = block_sum<kBlock>((double)nrm.s + (double)nrm.e, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = sum;
}

template <typename T>
int launch_axpy_norm(T* w, const T* V, long long ld, int nv, const double* hcol, const double* vscale, long long n,
                     double* partials, cudaStream_t s) {
    if (sizeof(T) == 4 && nv <= 32) {
        float* wf = (float*)w;
        const float* Vf = (const float*)V;
        const bool vec = ld % 4 == 0 && aligned16(V) && aligned16(w);
        int g = 0;
        ++g_launch_count;
        switch (nv) {
#define CASEF(N)                                                                                   \
    case N:                                                                                        \
        if (vec) {                                                                                 \
            g = cached_grid<k_axpy_norm_f32v<N>>();                                                \
            k_axpy_norm_f32v<N><<<g, kBlock, 0, s>>>(wf, Vf, ld, hcol, vscale, n, partials);        \
        } else {                                                                                   \
            g = cached_grid<k_axpy_norm_f32<N>>();                                                 \
            k_axpy_norm_f32<N><<<g, kBlock, 0, s>>>(wf, Vf, ld, hcol, vscale, n, partials);         \
        }                                                                                          \
        return g;
            CASEF(1) CASEF(2) CASEF(3) CASEF(4) CASEF(5) CASEF(6) CASEF(7) CASEF(8)
            CASEF(9) CASEF(10) CASEF(11) CASEF(12) CASEF(13) CASEF(14) CASEF(15) CASEF(16)
            CASEF(17) CASEF(18) CASEF(19) CASEF(20) CASEF(21) CASEF(22) CASEF(23) CASEF(24)
            CASEF(25) CASEF(26) CASEF(27) CASEF(28) CASEF(29) CASEF(30) CASEF(31) CASEF(32)
#undef CASEF
        }
    }
    int g = 0;
    switch (nv) {
#define CASE(N)                                                                                    \
    case N:                                                                                        \
        ++g_launch_count;                                                                          \
        g = cached_grid<k_axpy_norm<T, N>>();                                                      \
        k_axpy_norm<T, N><<<g, kBlock, 0, s>>>(w, V, ld, hcol, vscale, n, partials);                \
        return g;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
        CASE(9) CASE(10) CASE(11) CASE(12) CASE(13) CASE(14) CASE(15) CASE(16)
#undef CASE
        default:
            ++g_launch_count;
            g = cached_grid<k_axpy_norm_dyn<T>>();
            k_axpy_norm_dyn<T><<<g, kBlock, 0, s>>>(w, V, ld, nv, hcol, vscale, n, partials);
            return g;
    }
}
template int launch_axpy_norm<double>(double*, const double*, long long, int, const double*, const double*, long long,
                                      double*, cudaStream_t);
template int launch_axpy_norm<float>(float*, const float*, long long, int, const double*, const double*, long long,
                                     double*, cudaStream_t);

// With w = delta J^ z (kModeJvD) the Gram-Schmidt pass ran on delta times the
// true vector: every coefficient and the norm carry the factor delta, and the
// normalised v_{j+1} is the same, so only the Hessenberg column is rescaled.
__global__ void k_set_subdiag(double* scal, double* hcol, int j, double* vscale, int col_scale_slot) {
    double nrm = scal[kSlotTmp];
    hcol[j + 1] = nrm;
    vscale[j + 1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    if (col_scale_slot >= 0) {
        const double f = scal[col_scale_slot];
        for (int i = 0; i <= j + 1; ++i) hcol[i] *= f;
    }
}

void launch_set_subdiag(double* scal, double* hcol, int j, double* vscale, cudaStream_t s, int col_scale_slot) {
    ++g_launch_count;
    k_set_subdiag<<<1, 1, 0, s>>>(scal, hcol, j, vscale, col_scale_slot);
}

// Column j of the Hessenberg matrix H (column-major, leading dim ldh): apply
// the previous rotations, form rotation j, update g; scal[kSlotRes] = |g_{j+1}|.
__global__ void k_givens(double* H, int ldh, int j, double* cs, double* sn, double* g, double* scal) {
    double* h = H + (long long)j * ldh;
    for (int i = 0; i < j; ++i) {
        double t = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
    }
    double a = h[j], b = h[j + 1];
    double den = sqrt(a * a + b * b);
    double c = 1.0, s = 0.0;
    if (den != 0.0) { c = a / den; s = b / den; }
    cs[j] = c;
    sn[j] = s;
    h[j] = c * a + s * b;
    h[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    scal[kSlotRes] = fabs(g[j + 1]);
}

void launch_givens(double* H, int ldh, int j, double* cs, double* sn, double* g, double* scal, cudaStream_t s) {
    ++g_launch_count;
    k_givens<<<1, 1, 0, s>>>(H, ldh, j, cs, sn, g, scal);
}

__global__ void k_backsolve(const double* H, int ldh, int k, const double* g, double* y) {
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < k; ++l) s -= H[(long long)l * ldh + i] * y[l];
        y[i] = s / H[(long long)i * ldh + i];
    }
}

void launch_backsolve(const double* H, int ldh, int k, const double* g, double* y, cudaStream_t s) {
    ++g_launch_count;
    k_backsolve<<<1, 1, 0, s>>>(H, ldh, k, g, y);
}

// x += sum_{i<k} y_i Z_i
template <typename T>
__global__ void k_update(double* __restrict__ x, const T* __restrict__ Z, long long ld, int k,
                         const double* __restrict__ y, long long n) {
    __shared__ double ys[64];
    if (threadIdx.x < k) ys[threadIdx.x] = y[threadIdx.x];
    __syncthreads();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double v = x[e];
        for (int i = 0; i < k; ++i) v = v + ys[i] * (double)Z[i * ld + e];
        x[e] = v;
    }
}

// The same for a float basis: the products and their sum run on the FP32
// pipe as an unevaluated pair (TwoProduct, TwoSum; each y_i split into two
// floats), four elements per thread with 16-byte loads.  In double, the k
// FMAs per element bound this pass by the FP64 pipe (k up to 30 at 84
// million unknowns).  Columns of Z start on 16-byte boundaries (ld is a
// multiple of 64) and x is 256-byte aligned; the last n mod 4 elements take
// the scalar loop.
__global__ void __launch_bounds__(kBlock) k_update_f32v(double* __restrict__ x, const float* __restrict__ Z,
                                                        long long ld, int k, const double* __restrict__ y,
                                                        long long n) {
    __shared__ float yh[64], yl[64];
    if (threadIdx.x < k) {
        const double c = y[threadIdx.x];
        const float h = (float)c;
        yh[threadIdx.x] = h;
        yl[threadIdx.x] = (float)(c - (double)h);
    }
    __syncthreads();
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n4 = n >> 2;
    for (long long q = t0; q < n4; q += stride) {
        CompF a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f}, a3{0.f, 0.f};
#pragma unroll 4
        for (int i = 0; i < k; ++i) {
            const float4 v = reinterpret_cast<const float4*>(Z + i * ld)[q];
            const float h = yh[i], l = yl[i];
            comp_fma(a0, h, v.x);
            a0.e = fmaf(l, v.x, a0.e);
            comp_fma(a1, h, v.y);
            a1.e = fmaf(l, v.y, a1.e);
            comp_fma(a2, h, v.z);
            a2.e = fmaf(l, v.z, a2.e);
            comp_fma(a3, h, v.w);
            a3.e = fmaf(l, v.w, a3.e);
        }
        double2* xp = reinterpret_cast<double2*>(x) + 2 * q;
        double2 lo = xp[0], hi = xp[1];
        lo.x += (double)a0.s + (double)a0.e;
        lo.y += (double)a1.s + (double)a1.e;
        hi.x += (double)a2.s + (double)a2.e;
        hi.y += (double)a3.s + (double)a3.e;
        xp[0] = lo;
        xp[1] = hi;
    }
    for (long long e = 4 * n4 + t0; e < n; e += stride) {
        CompF a{0.f, 0.f};
        for (int i = 0; i < k; ++i) {
            const float z = Z[i * ld + e];
            comp_fma(a, yh[i], z);
            a.e = fmaf(yl[i], z, a.e);
        }
        x[e] += (double)a.s + (double)a.e;
    }
}

template <typename T>
void launch_update(double* x, const T* Z, long long ld, int k, const double* y, long long n, cudaStream_t s) {
    ++g_launch_count;
    if (sizeof(T) == 4 && ld % 4 == 0) {
        const int g = cached_grid<k_update_f32v>();
        k_update_f32v<<<g, kBlock, 0, s>>>(x, (const float*)Z, ld, k, y, n);
    } else {
        k_update<T><<<kRedBlocks, kBlock, 0, s>>>(x, Z, ld, k, y, n);
    }
}
template void launch_update<double>(double*, const double*, long long, int, const double*, long long, cudaStream_t);
template void launch_update<float>(double*, const float*, long long, int, const double*, long long, cudaStream_t);

// dst = src * (alpha, or scal[slot], or 1/scal[slot])
template <typename TS, typename TD>
__global__ void k_scale_copy(const TS* __restrict__ src, double alpha, const double* scal, int slot, int invert,
                             TD* __restrict__ dst, long long n) {
    double a = alpha;
    if (slot >= 0) a = invert ? 1.0 / scal[slot] : scal[slot];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dst[e] = (TD)((double)src[e] * a);
}

template <typename TS, typename TD>
void launch_scale_copy(const TS* src, double alpha, const double* scal, int slot, int invert, TD* dst, long long n,
                       cudaStream_t s) {
    ++g_launch_count;
    k_scale_copy<TS, TD><<<kRedBlocks, kBlock, 0, s>>>(src, alpha, scal, slot, invert, dst, n);
}
template void launch_scale_copy<double, double>(const double*, double, const double*, int, int, double*, long long, cudaStream_t);
template void launch_scale_copy<double, float>(const double*, double, const double*, int, int, float*, long long, cudaStream_t);
template void launch_scale_copy<float, float>(const float*, double, const double*, int, int, float*, long long, cudaStream_t);
template void launch_scale_copy<float, double>(const float*, double, const double*, int, int, double*, long long, cudaStream_t);

// X += R dxh ; partial max |dxh| (NaN propagates)
__global__ void k_newton_update(double* __restrict__ X, const double* __restrict__ R, const double* __restrict__ dxh,
                                long long n, double* __restrict__ partials) {
    __shared__ double sh[32];
    double m = 0.0;
    bool nan = false;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double d = dxh[e];
        X[e] = X[e] + R[e] * d;
        double a = fabs(d);
        if (!(a == a)) nan = true;
        m = fmax(m, a);
    }
    double r = block_max<kBlock>(m, sh);
    int anynan = __syncthreads_or(nan);
    if (threadIdx.x == 0) partials[blockIdx.x] = anynan ? __longlong_as_double(0x7ff8000000000000ULL) : r;
}

void launch_newton_update(double* X, const double* R, const double* dxh, long long n, double* partials,
                          cudaStream_t s) {
    ++g_launch_count;
    k_newton_update<<<kRedBlocks, kBlock, 0, s>>>(X, R, dxh, n, partials);
}

template <typename T>
__global__ void k_zero(T* x, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        x[e] = (T)0;
}

template <typename T>
void launch_zero(T* x, long long n, cudaStream_t s) { k_zero<T><<<kRedBlocks, kBlock, 0, s>>>(x, n); }
template void launch_zero<double>(double*, long long, cudaStream_t);
template void launch_zero<float>(float*, long long, cudaStream_t);

// r = b - r with b = -(G0 - b^n) L^-1 (the Newton right-hand side, rebuilt in
// double for a GMRES restart); r holds J^ x on entry
template <typename T>
__global__ void k_restart_residual(T* r, const double* __restrict__ G0, const double* __restrict__ bn,
                                   const double* __restrict__ Linv, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double b = -((G0[e] - bn[e]) * Linv[e]);
        r[e] = (T)(b - (double)r[e]);
    }
}

template <typename T>
void launch_restart_residual(T* r, const double* G0, const double* bn, const double* Linv, long long n,
                             cudaStream_t s) {
    ++g_launch_count;
    k_restart_residual<T><<<kRedBlocks, kBlock, 0, s>>>(r, G0, bn, Linv, n);
}
template void launch_restart_residual<double>(double*, const double*, const double*, const double*, long long,
                                              cudaStream_t);
template void launch_restart_residual<float>(float*, const double*, const double*, const double*, long long,
                                             cudaStream_t);

// start of a GMRES cycle: g = (beta, 0, ...), vscale[0] = 1/beta
__global__ void k_init_cycle(double* scal, double* g, double* vscale, int m) {
    double beta = scal[kSlotBeta];
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    vscale[0] = beta > 0.0 ? 1.0 / beta : 0.0;
}

void launch_init_cycle(double* scal, double* g, double* vscale, int m, cudaStream_t s) {
    ++g_launch_count;
    k_init_cycle<<<1, 1, 0, s>>>(scal, g, vscale, m);
}

// column += other (second Gram-Schmidt pass)
__global__ void k_add_col(double* col, const double* other, int n) {
    int i = threadIdx.x;
    if (i < n) col[i] += other[i];
}

// P = L^-1/dt, Q = theta L^-1, C = L^-1 G(X) of the Jacobian-free assemble;
// entries from u_begin on (the momentum rows, whose conserved value the
// assemble forms as 2 rho_f u) take P = L^-1/(2 dt)
__global__ void k_jv_coeffs(const double* __restrict__ Linv, const double* __restrict__ G0, double idt, double idt_h,
                            double theta, double* __restrict__ P, double* __restrict__ Q, double* __restrict__ C,
                            long long n, long long u_begin) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const double li = Linv[e];
        P[e] = (e < u_begin ? idt : idt_h) * li;
        Q[e] = theta * li;
        C[e] = G0[e] * li;
    }
}

void launch_jv_coeffs(const double* Linv, const double* G0, double dt, double theta, double* P, double* Q, double* C,
                      long long n, long long u_begin, cudaStream_t s) {
    ++g_launch_count;
    k_jv_coeffs<<<kRedBlocks, kBlock, 0, s>>>(Linv, G0, 1.0 / dt, 0.5 / dt, theta, P, Q, C, n, u_begin);
}

void launch_add_col(double* col, const double* other, int n, cudaStream_t s) {
    ++g_launch_count;
    k_add_col<<<1, 64, 0, s>>>(col, other, n);
}

}  // namespace jfnk
