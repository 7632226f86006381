// FP64 throughput probe: the measured peak that the FP64-bound stencil
// kernels are compared against; and checks, run by the tests, of device
// functions of the solver's kernels: the Newton-Raphson reciprocal
// (recip_nr) against IEEE division, and the integer-pipe float/double
// conversions (f2d_exact, d2f_rn) against the conversion instructions,
// and the integer-pipe products and sums (emu::mul_rn, emu::add_rn,
// emu::sub_rn) against the DMUL / DADD instructions.
//
// Every thread runs eight independent chains of fused multiply-adds
// x <- x * a + b (one DFMA instruction, two flops each), so the FP64 pipe
// always has independent work to issue and the measured rate is its issue
// limit.  With 0 < a < 1 and b = 1 - a every chain converges to 1.0 and
// stays a normal number.  Each thread writes the sum of its chains so that
// no chain is dead code.  This is not part of the solver library: bench.py
// loads it on its own to time the probe with CUDA events.
#include <cuda_runtime.h>

#include "common.cuh"
#include "emu64.cuh"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_dfma_probe(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_recip_check(const double* __restrict__ d, double* __restrict__ r, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) r[i] = jfnk::recip_nr(d[i]);
}

__global__ void k_conv_check(const double* __restrict__ x, const float* __restrict__ f, float* __restrict__ xf,
                             double* __restrict__ fd, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) {
        xf[i] = jfnk::d2f_rn(x[i]);
        fd[i] = jfnk::f2d_exact(f[i]);
    }
}

__global__ void k_emu_check(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ m,
                            double* __restrict__ s, double* __restrict__ d, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) {
        m[i] = jfnk::emu::mul_rn(a[i], b[i]);
        s[i] = jfnk::emu::add_rn(a[i], b[i]);
        d[i] = jfnk::emu::sub_rn(a[i], b[i]);
    }
}

}  // namespace

extern "C" {

// xf[i] = d2f_rn(x[i]) and fd[i] = f2d_exact(f[i]) for i < n (device arrays),
// queued on `stream`.
int fp64_conv_check(const double* x, const float* f, float* xf, double* fd, long long n, void* stream) {
    if (!x || !f || !xf || !fd || n <= 0) return (int)cudaErrorInvalidValue;
    const long long blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
    k_conv_check<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(x, f, xf, fd, n);
    return (int)cudaGetLastError();
}

// r[i] = recip_nr(d[i]) (the reciprocal of the batched inversion in the
// residual kernels) for i < n, queued on `stream`; d and r are device
// arrays of n doubles.
int fp64_recip_check(const double* d, double* r, long long n, void* stream) {
    if (!d || !r || n <= 0) return (int)cudaErrorInvalidValue;
    const long long blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
    k_recip_check<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d, r, n);
    return (int)cudaGetLastError();
}

// m[i] = a[i] * b[i], s[i] = a[i] + b[i], d[i] = a[i] - b[i] on the integer
// pipes (emu64.cuh) for i < n, queued on `stream`; all device arrays of n
// doubles.
int fp64_emu_check(const double* a, const double* b, double* m, double* s, double* d, long long n, void* stream) {
    if (!a || !b || !m || !s || !d || n <= 0) return (int)cudaErrorInvalidValue;
    const long long blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
    k_emu_check<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(a, b, m, s, d, n);
    return (int)cudaGetLastError();
}

// DFMA instructions one launch executes per thread.
long long fp64_probe_fma_per_thread(int iters) { return (long long)iters * kChains; }

// Queue one probe launch of `blocks` x 256 threads on `stream`; out holds
// blocks * 256 doubles.  Returns the cudaError_t of the launch.
int fp64_probe_launch(double* out, int blocks, int iters, double a, void* stream) {
    if (!out || blocks <= 0 || iters <= 0 || !(a > 0.0 && a < 1.0)) return (int)cudaErrorInvalidValue;
    k_dfma_probe<<<blocks, 256, 0, (cudaStream_t)stream>>>(out, iters, a, 1.0 - a);
    return (int)cudaGetLastError();
}

}  // extern "C"
