// jfnk_residual_noalloc: the residual entry point for callers that cannot
// allocate device memory.
//
// jfnk_residual needs scratch (the X^n part b^n, p and T per cell, and the
// face and momentum fluxes) that normally lives in the workspace the caller
// allocates and binds.  Some callers cannot make that allocation: code that
// runs where the process's device allocator belongs to another framework or
// is locked down, plugins handed only the input and output buffers, or code
// that must not trigger an allocation at that point of its run.  This entry
// point keeps its scratch in a fixed array in the library's own device
// memory instead, so it needs only the caller's input and output buffers and
// a created handle (no jfnk_bind).
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (JFNK_NOALLOC_MAX_CELLS * 23 doubles, 12.1 MB) until the
// process exits.  Host code reaches it only through the address returned by
// cudaGetSymbolAddress, fetched once per device on the first call made with
// that device current and kept in an atomic per-device slot (concurrent
// first calls from several host threads store the same address).  A handle
// bound with jfnk_bind must be called with its own device current.  Every
// call shares the one array, so calls that overlap on the GPU (different
// streams, or different host threads) race; callers must serialise them.  No
// scratch needs clearing: each call writes every scratch value before
// reading it.
#include <atomic>
#include <cstdio>
#include <string>

#include "../../include/jfnk.h"
#include "common.cuh"
#include "kernels.h"

using namespace jfnk;

namespace {

constexpr long long kNoallocFields = 23;   // 5 b^n + p + T + chi + 3 Fm + 3 FE + 9 Psi (3D; 2D uses 15)
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kNoallocFields * JFNK_NOALLOC_MAX_CELLS];

std::atomic<void*> g_scratch_ptr[kMaxDevices];

// Device address of the scratch array on device dev, which must be current
// (fetched once per device; a race between first calls stores one address).
cudaError_t scratch_for_device(int dev, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    void* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev].store(p, std::memory_order_release);
    }
    *out = (double*)p;
    return cudaSuccess;
}

}  // namespace

// Grid and stream of a handle (defined with the handle in engine.cu).
const jfnk::Grid* jfnk_handle_grid(const jfnk_handle* h);
cudaStream_t jfnk_handle_stream(const jfnk_handle* h);
int jfnk_handle_device(const jfnk_handle* h);
void jfnk_handle_set_error(jfnk_handle* h, const char* msg);

extern "C" jfnk_status jfnk_residual_noalloc(jfnk_handle* h, const double* X, const double* Xn, double dt,
                                             double* F) {
    if (!h) return JFNK_EINVAL;
    if (!X || !Xn || !F || !(dt > 0.0)) {
        jfnk_handle_set_error(h, "bad arguments to jfnk_residual_noalloc");
        return JFNK_EINVAL;
    }
    const Grid& G = *jfnk_handle_grid(h);
    if (G.ncell > JFNK_NOALLOC_MAX_CELLS) {
        char buf[160];
        snprintf(buf, sizeof buf, "jfnk_residual_noalloc: %lld cells exceed the fixed scratch limit of %d cells",
                 G.ncell, JFNK_NOALLOC_MAX_CELLS);
        jfnk_handle_set_error(h, buf);
        return JFNK_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && jfnk_handle_device(h) >= 0 && jfnk_handle_device(h) != dev) {
        char buf[160];
        snprintf(buf, sizeof buf, "jfnk_residual_noalloc: handle bound on device %d but device %d is current",
                 jfnk_handle_device(h), dev);
        jfnk_handle_set_error(h, buf);
        return JFNK_EINVAL;
    }
    double* base = nullptr;
    if (e == cudaSuccess) e = scratch_for_device(dev, &base);
    if (e != cudaSuccess) {
        std::string m = std::string("jfnk_residual_noalloc: device address lookup failed: ") + cudaGetErrorString(e);
        jfnk_handle_set_error(h, m.c_str());
        return JFNK_ECUDA;
    }
    const long long nc = G.ncell, nd = G.ndim;
    double* bn = base;
    double* p = bn + (2 + nd) * nc;
    double* T = p + nc;
    double* chi = T + nc;
    double* Fm = chi + nc;
    double* FE = Fm + nd * nc;
    double* Psi = FE + nd * nc;
    cudaStream_t s = jfnk_handle_stream(h);
    launch_eos(G, Xn, p, T, chi, s);
    launch_fluxes(G, Xn, p, T, chi, Fm, FE, Psi, s);
    launch_assemble<kModeBn, double>(G, Xn, p, Fm, FE, Psi, nullptr, nullptr, nullptr, nullptr, 0, dt, bn,
                                     (double*)nullptr, s);
    launch_eos(G, X, p, T, chi, s);
    launch_fluxes(G, X, p, T, chi, Fm, FE, Psi, s);
    launch_assemble<kModeRes, double>(G, X, p, Fm, FE, Psi, bn, nullptr, nullptr, nullptr, 0, dt, F,
                                      (double*)nullptr, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        std::string m = std::string("jfnk_residual_noalloc: ") + cudaGetErrorString(e);
        jfnk_handle_set_error(h, m.c_str());
        return JFNK_ECUDA;
    }
    return JFNK_OK;
}
