// Host build of the integer-pipe products and sums of the flux kernels
// (paper_1512_03662_gb300/csrc/emu64.cuh compiles for the host on the same
// integer steps), loaded by tests/test_emu64_host.py through ctypes and
// compared there bit for bit with the host's IEEE arithmetic.
#include "emu64.cuh"

extern "C" {

// m = a*b, s = a+b, d = a-b elementwise; fast[i] = 1 where both the product
// and the sum took the integer path (not the hardware fallback)
void emu64_host(const double* a, const double* b, double* m, double* s, double* d, unsigned char* fast, long long n) {
    for (long long i = 0; i < n; ++i) {
        m[i] = jfnk::emu::mul_rn(a[i], b[i]);
        s[i] = jfnk::emu::add_rn(a[i], b[i]);
        d[i] = jfnk::emu::sub_rn(a[i], b[i]);
        double t;
        fast[i] = (unsigned char)(jfnk::emu::mul_fast(a[i], b[i], t) && jfnk::emu::add_fast(a[i], b[i], t));
    }
}
}
