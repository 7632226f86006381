// Physics-based preconditioner (paper Sects. 3.2-3.4 and 4.3).
//
//   w = R^-1 dX/dV J~_V^-1 dV/dU L v
//
// k_precond_in   v -> r_V = dV/dU L v, factored as dV/dX dX/dU (App. B); the
//                velocity rows act face by face, r_u = (r_rhou - u rbar_rho)/rho_f;
//                the multigrid right-hand side is B^-1 (r_p, r_e), B the 2x2
//                matrix of the Laplacian coefficients of the p and e rows
//                (1x1, B = theta^2 dt Gamma1 p, for the sound-only scheme).
// k_si_setup     cell matrix M = B^-1/dt and face coefficients K_p = 1/rho_f,
//                K_e = chi_f/c_v of the equivalent system
//                    M x - [div(K_p grad dp); div(K_e grad de)] = B^-1 r,
//                from the current Newton iterate.
// multigrid      fixed V-cycles: red-black (point-block) Gauss-Seidel,
//                mean restriction, cell-centred linear prolongation, exact
//                one-cell coarsest level; coarse coefficients by averaging.
// k_precond_out  de from the identity of Sect. 3.3.4 (sound scheme) or from
//                the coupled solve; du_f = dt (r_u - theta rho_f^-1 grad dp);
//                dX = dX/dV dV; z = R^-1 dX and partial sums of |z|^2.
// The multigrid runs in the basis precision T (float in mixed mode); the
// pointwise transforms compute in double and store T.
#include "common.cuh"
#include "kernels.h"

namespace jfnk {

static inline unsigned nb(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

struct LvlDev {
    int n[3];
    long long nc;
    double ih2[3];
    float ih2f[3];   // the same in float, so FP32 kernels convert nothing
};

static inline LvlDev lvl(const MGLevel& L) {
    LvlDev d;
    for (int i = 0; i < 3; ++i) { d.n[i] = L.n[i]; d.ih2[i] = L.ih2[i]; d.ih2f[i] = (float)L.ih2[i]; }
    d.nc = L.ncell;
    return d;
}

template <typename T> __device__ __forceinline__ T ih2_of(const LvlDev& L, int d);
template <> __device__ __forceinline__ double ih2_of<double>(const LvlDev& L, int d) { return L.ih2[d]; }
template <> __device__ __forceinline__ float ih2_of<float>(const LvlDev& L, int d) { return L.ih2f[d]; }

// Storage index of cell (a,b,c) in a multigrid array.  With an even x extent
// the arrays are colour-split: all cells with i+j+k even first, then the odd
// ones, each in x-fastest order (the two cells of an x pair share flat/2), so
// a red-black half sweep reads and writes contiguous memory.  Levels with an
// odd x extent (a single cell along x) keep the natural order.
__device__ __forceinline__ long long rb_index(int n0, int n1, long long nc, int a, int b, int c) {
    long long f = ((long long)c * n1 + b) * n0 + a;
    if (n0 & 1) return f;
    return (long long)((a + b + c) & 1) * (nc >> 1) + (f >> 1);
}

__device__ __forceinline__ long long lflat(const LvlDev& L, int a, int b, int c) {
    return rb_index(L.n[0], L.n[1], L.nc, a, b, c);
}

// index of fine-level cell P in the level-0 multigrid arrays
__device__ __forceinline__ long long mg0(const Grid& G, const Idx3& P) {
    return rb_index(G.n[0], G.n[1], G.ncell, P.i[0], P.i[1], P.i[2]);
}

__device__ __forceinline__ int wrapi(int k, int n) { return k < 0 ? k + n : (k >= n ? k - n : k); }

__device__ __forceinline__ double conductivity_si(const Grid& G, double T) {
    return G.chi3 ? G.K0 * (T * T * T) : G.K0 * pow(T, G.chi_exp);
}

// ---------------------------------------------------------------------------
// coefficients at the current iterate (once per Newton iteration)
// ---------------------------------------------------------------------------

__device__ __forceinline__ double e_internal_at(const Grid& G, const double* X, const Idx3& P, int o0, int o1, int o2) {
    const long long nc = G.ncell;
    double E = load_cell(G, X + nc, P, o0, o1, o2);
    if (G.energy_form == 0) return E;
    Idx3 Q;
    Q.i[0] = cell_map(P.i[0] + o0, G.n[0], G.bc[0]);
    Q.i[1] = cell_map(P.i[1] + o1, G.n[1], G.bc[1]);
    Q.i[2] = cell_map(P.i[2] + o2, G.n[2], G.bc[2]);
    double ke = 0.0;
    for (int d = 0; d < G.ndim; ++d) {
        const double* u = X + (2 + d) * nc;
        int o[3] = {0, 0, 0};
        o[d] = 1;
        double ul = load_normal(G, u, d, Q, 0, 0, 0);
        double uu = load_normal(G, u, d, Q, o[0], o[1], o[2]);
        ke = ke + 0.25 * (ul * ul + uu * uu);
    }
    return E - ke;
}

// Per-cell coefficient fields of the transforms, in the basis precision T.
// Field order (index * ncell): see PcField.  All divisions of the
// preconditioner happen here, once per Newton iteration, and they reduce to
// reciprocals of rho, e, b_pp and the face densities (one batched
// inversion) and of det B: every other quotient is a product with those.
// B is the 2x2 matrix of Laplacian coefficients of the p and e rows (sound
// scheme: b_pp alone), B^-1 its inverse.
template <int ND, typename T>
__global__ void k_pc_setup(Grid G, const double* __restrict__ X, const double* __restrict__ L,
                           const double* __restrict__ Rinv, double dt, double idt, int nf, T* __restrict__ C,
                           T* __restrict__ M, T* __restrict__ K) {
    Idx3 P;
    long long cc;
    if (!cell_pos(G.n, P, cc)) return;
    const long long nc = G.ncell;
    const double rho = X[cc];
    const double E = X[nc + cc];
    const double e = e_internal_at(G, X, P, 0, 0, 0);
    const double p = G.gm1 * rho * e;
    const double th = G.theta;
    const double bpp = th * th * dt * G.gamma * p;
    double rl[ND], den[3 + ND], inv[3 + ND];
    den[0] = rho;
    den[1] = e;
    den[2] = bpp;
#pragma unroll
    for (int c = 0; c < ND; ++c) {
        int o[3] = {0, 0, 0};
        o[c] = -1;
        rl[c] = load_cell(G, X, P, o[0], o[1], o[2]);
        den[3 + c] = 0.5 * (rl[c] + rho);           // rho_f on the lower face
    }
    recip_all<3 + ND>(den, inv);
    const double irho = inv[0], ie = inv[1], ibpp = inv[2];
    double b00, b01, b10, b11;
    if (nf == 2) {
        const double bpe = th * G.gm1;
        const double bep = th * th * dt * p * irho;
        const double bee = th * irho;
        const double idet = 1.0 / (bpp * bee - bpe * bep);
        b00 = bee * idet;
        b01 = -bpe * idet;
        b10 = -bep * idet;
        b11 = bpp * idet;
    } else {
        b00 = ibpp;
        b01 = b10 = b11 = 0.0;
    }
    const long long mi = mg0(G, P);
    if (nf == 1) {
        M[mi] = from_f64<T>(idt * ibpp);
    } else {
        M[0 * nc + mi] = from_f64<T>(b00 * idt);
        M[1 * nc + mi] = from_f64<T>(b01 * idt);
        M[2 * nc + mi] = from_f64<T>(b10 * idt);
        M[3 * nc + mi] = from_f64<T>(b11 * idt);
    }
    const double chi0 = (G.has_cond) ? conductivity_si(G, G.gm1 * e) : 0.0;
    const double dpdrho = G.gm1 * e, dpde = G.gm1 * rho;
    C[PcLr * nc + cc] = from_f64<T>(L[cc]);
    C[PcLE * nc + cc] = from_f64<T>(L[nc + cc]);
    C[PcInvRho * nc + cc] = from_f64<T>(irho);
    C[PcE * nc + cc] = from_f64<T>(E);
    C[PcDpdrho * nc + cc] = from_f64<T>(dpdrho);
    C[PcDpde * nc + cc] = from_f64<T>(dpde);
    C[PcInvDpdrho * nc + cc] = from_f64<T>(G.igm1 * ie);
    C[PcCde * nc + cc] = from_f64<T>(G.igamma * irho);
    // r_p = Pr r_rho + PE r_E - dpde <u.r_u>: first row of dV/dU in the
    // product form printed in Sect. 3.2 (no cancellation between terms)
    const double Eir = E * irho;
    const double Pr = dpdrho - dpde * Eir, PE = dpde * irho;
    C[PcPr * nc + cc] = from_f64<T>(Pr);
    C[PcPE * nc + cc] = from_f64<T>(PE);
    if (sizeof(T) == 8) {
        C[PcQ0 * nc + cc] = from_f64<T>(b00);
        if (nf == 2) {
            C[PcQ1 * nc + cc] = from_f64<T>(b01);
            C[PcQ2 * nc + cc] = from_f64<T>(b10);
            C[PcQ3 * nc + cc] = from_f64<T>(b11);
        }
    } else {
        // rhs = B^-1 (r_p, r_e) with r_e = (r_E - E r_rho)/rho - <u.r_u>,
        // folded in double (no cancellation in FP32)
        C[PcQ0 * nc + cc] = from_f64<T>(b00 * Pr - b01 * Eir);
        C[PcQ1 * nc + cc] = from_f64<T>(b00 * PE + b01 * irho);
        C[PcQ2 * nc + cc] = from_f64<T>(b00 * dpde + b01);
        C[PcQ3 * nc + cc] = from_f64<T>(b10 * Pr - b11 * Eir);
        C[PcQ4 * nc + cc] = from_f64<T>(b10 * PE + b11 * irho);
        C[PcQ5 * nc + cc] = from_f64<T>(b10 * dpde + b11);
    }
    C[PcRinvR * nc + cc] = from_f64<T>(Rinv[cc]);
    C[PcRinvE * nc + cc] = from_f64<T>(Rinv[nc + cc]);
#pragma unroll
    for (int c = 0; c < ND; ++c) {
        const bool wall = is_wall_slot(G, c, P);
        int o[3] = {0, 0, 0};
        o[c] = -1;
        const double irhof = inv[3 + c];
        const double m = (wall || G.n[c] == 1) ? 0.0 : 1.0;
        K[(0 * ND + c) * nc + mi] = from_f64<T>(m * irhof);
        if (nf == 2) {
            double chil = 0.0;
            if (G.has_cond) chil = conductivity_si(G, G.gm1 * e_internal_at(G, X, P, o[0], o[1], o[2]));
            K[(1 * ND + c) * nc + mi] = from_f64<T>(m * (0.5 * (chil + chi0)) * G.gm1);
        }
        const double u = wall ? 0.0 : X[(2 + c) * nc + cc];
        C[(PcLu + c) * nc + cc] = from_f64<T>(L[(2 + c) * nc + cc]);
        C[(PcU + c) * nc + cc] = from_f64<T>(u);
        C[(PcInvRhof + c) * nc + cc] = from_f64<T>(wall ? 0.0 : irhof);
        C[(PcThf + c) * nc + cc] = from_f64<T>(wall ? 0.0 : G.theta * G.idx[c] * irhof);
        C[(PcRinvU + c) * nc + cc] = from_f64<T>(Rinv[(2 + c) * nc + cc]);
    }
}

#define CELL_LAUNCH_T(KERNEL, T, ...)                                                     \
    do {                                                                                  \
        CellLaunch cl_ = cell_launch(G.n);                                                \
        ++g_launch_count;                                                                 \
        if (G.ndim == 3) KERNEL<3, T><<<cl_.grid, cl_.block, 0, s>>>(__VA_ARGS__);        \
        else KERNEL<2, T><<<cl_.grid, cl_.block, 0, s>>>(__VA_ARGS__);                    \
    } while (0)

template <typename T>
void launch_pc_setup(const Grid& G, const double* X, const double* L, const double* Rinv, double dt, int nf, T* C,
                     MGLevel& L0, cudaStream_t s) {
    CELL_LAUNCH_T(k_pc_setup, T, G, X, L, Rinv, dt, 1.0 / dt, nf, C, (T*)L0.M, (T*)L0.K);
}
template void launch_pc_setup<double>(const Grid&, const double*, const double*, const double*, double, int, double*,
                                      MGLevel&, cudaStream_t);
template void launch_pc_setup<float>(const Grid&, const double*, const double*, const double*, double, int, float*,
                                     MGLevel&, cudaStream_t);

// The scaling fields of C alone, as k_pc_setup writes them (the frozen-
// coefficient option renews only these at later Newton iterates).
template <int ND, typename T>
__global__ void k_pc_rescale(Grid G, const double* __restrict__ L, const double* __restrict__ Rinv,
                             T* __restrict__ C) {
    Idx3 P;
    long long cc;
    if (!cell_pos(G.n, P, cc)) return;
    const long long nc = G.ncell;
    C[PcLr * nc + cc] = from_f64<T>(L[cc]);
    C[PcLE * nc + cc] = from_f64<T>(L[nc + cc]);
    C[PcRinvR * nc + cc] = from_f64<T>(Rinv[cc]);
    C[PcRinvE * nc + cc] = from_f64<T>(Rinv[nc + cc]);
#pragma unroll
    for (int c = 0; c < ND; ++c) {
        C[(PcLu + c) * nc + cc] = from_f64<T>(L[(2 + c) * nc + cc]);
        C[(PcRinvU + c) * nc + cc] = from_f64<T>(Rinv[(2 + c) * nc + cc]);
    }
}

template <typename T>
void launch_pc_rescale(const Grid& G, const double* L, const double* Rinv, T* C, cudaStream_t s) {
    CELL_LAUNCH_T(k_pc_rescale, T, G, L, Rinv, C);
}
template void launch_pc_rescale<double>(const Grid&, const double*, const double*, double*, cudaStream_t);
template void launch_pc_rescale<float>(const Grid&, const double*, const double*, float*, cudaStream_t);

// ---------------------------------------------------------------------------
// coarse coefficients
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool lvl_pos(const LvlDev& L, int i[3], long long& c) {
    i[0] = blockIdx.x * blockDim.x + threadIdx.x;
    i[1] = blockIdx.y * blockDim.y + threadIdx.y;
    i[2] = blockIdx.z;
    if (i[0] >= L.n[0] || i[1] >= L.n[1]) return false;
    c = lflat(L, i[0], i[1], i[2]);
    return true;
}

// mean over the children of coarse cell (a,b,c), pairs along x, then y, then z
template <typename T>
__device__ __forceinline__ double child_mean(const T* f, const LvlDev& F, const int cd[3], int a, int b, int c) {
    int nx = cd[0] ? 2 : 1, ny = cd[1] ? 2 : 1, nz = cd[2] ? 2 : 1;
    int x0 = cd[0] ? 2 * a : a, y0 = cd[1] ? 2 * b : b, z0 = cd[2] ? 2 * c : c;
    double zs[2];
    for (int kz = 0; kz < nz; ++kz) {
        double ys[2];
        for (int ky = 0; ky < ny; ++ky) {
            double v0 = (double)f[lflat(F, x0, y0 + ky, z0 + kz)];
            ys[ky] = (nx == 2) ? (v0 + (double)f[lflat(F, x0 + 1, y0 + ky, z0 + kz)]) / 2.0 : v0;
        }
        zs[kz] = (ny == 2) ? (ys[0] + ys[1]) / 2.0 : ys[0];
    }
    return (nz == 2) ? (zs[0] + zs[1]) / 2.0 : zs[0];
}

template <typename T>
__global__ void k_coarsen(int nf, int ndim, LvlDev F, LvlDev C, const T* __restrict__ Mf, const T* __restrict__ Kf,
                          T* __restrict__ Mc, T* __restrict__ Kc) {
    int ic[3];
    long long cc;
    if (!lvl_pos(C, ic, cc)) return;
    const int a = ic[0], b = ic[1], c = ic[2];
    int cd[3] = {F.n[0] != C.n[0], F.n[1] != C.n[1], F.n[2] != C.n[2]};
    for (int q = 0; q < nf * nf; ++q) Mc[q * C.nc + cc] = (T)child_mean(Mf + q * F.nc, F, cd, a, b, c);
    for (int f = 0; f < nf; ++f) {
        for (int d = 0; d < ndim; ++d) {
            const T* k = Kf + (f * ndim + d) * F.nc;
            double v = 0.0;
            if (C.n[d] > 1) {
                // fine lower faces of the even children along d, mean over the other coarsened dims
                int cd2[3] = {cd[0], cd[1], cd[2]};
                cd2[d] = 0;
                int fx = cd[0] ? 2 * a : a, fy = cd[1] ? 2 * b : b, fz = cd[2] ? 2 * c : c;
                int nx = cd2[0] ? 2 : 1, ny = cd2[1] ? 2 : 1, nz = cd2[2] ? 2 : 1;
                double zs[2];
                for (int kz = 0; kz < nz; ++kz) {
                    double ys[2];
                    for (int ky = 0; ky < ny; ++ky) {
                        double v0 = (double)k[lflat(F, fx, fy + ky, fz + kz)];
                        ys[ky] = (nx == 2) ? (v0 + (double)k[lflat(F, fx + 1, fy + ky, fz + kz)]) / 2.0 : v0;
                    }
                    zs[kz] = (ny == 2) ? (ys[0] + ys[1]) / 2.0 : ys[0];
                }
                v = (nz == 2) ? (zs[0] + zs[1]) / 2.0 : zs[0];
            }
            Kc[(f * ndim + d) * C.nc + cc] = (T)v;
        }
    }
}

template <typename T>
void launch_coarsen(const Grid& G, int nf, const MGLevel& F, MGLevel& C, cudaStream_t s) {
    CellLaunch cl = cell_launch(C.n);
    ++g_launch_count;
    k_coarsen<T><<<cl.grid, cl.block, 0, s>>>(nf, G.ndim, lvl(F), lvl(C), (const T*)F.M, (const T*)F.K, (T*)C.M,
                                              (T*)C.K);
}
template void launch_coarsen<double>(const Grid&, int, const MGLevel&, MGLevel&, cudaStream_t);
template void launch_coarsen<float>(const Grid&, int, const MGLevel&, MGLevel&, cudaStream_t);

// ---------------------------------------------------------------------------
// transform in: r_V and the multigrid right-hand side
// ---------------------------------------------------------------------------

// r_rho at the cell (pos + off) with ghost mapping
template <typename T, typename TV>
__device__ __forceinline__ T rrho_at(const Grid& G, const T* C, const TV* v, T s, const Idx3& P, int o0, int o1,
                                     int o2) {
    int a = cell_map(P.i[0] + o0, G.n[0], G.bc[0]);
    int b = cell_map(P.i[1] + o1, G.n[1], G.bc[1]);
    int c = cell_map(P.i[2] + o2, G.n[2], G.bc[2]);
    long long j = flat(G, a, b, c);
    return C[PcLr * G.ncell + j] * (s * (T)v[j]);
}

// r_u on the lower face of cell Q in direction c (zero at a wall slot)
template <typename T, typename TV>
__device__ __forceinline__ T ru_at(const Grid& G, const T* C, const TV* v, T s, int c, const Idx3& Q) {
    const long long nc = G.ncell;
    const long long j = flat(G, Q.i[0], Q.i[1], Q.i[2]);
    int o[3] = {0, 0, 0};
    o[c] = -1;
    T rl = rrho_at<T, TV>(G, C, v, s, Q, o[0], o[1], o[2]);
    T r0 = C[PcLr * nc + j] * (s * (T)v[j]);
    T rb = (T)0.5 * (rl + r0);
    T ruv = C[(PcLu + c) * nc + j] * (s * (T)v[(2 + c) * nc + j]);
    return (ruv - C[(PcU + c) * nc + j] * rb) * C[(PcInvRhof + c) * nc + j];
}

template <int ND, typename T>
__global__ void k_precond_in(Grid G, const T* __restrict__ C, const T* __restrict__ v,
                             const double* __restrict__ vscale, int vslot, int nf, T* __restrict__ rp,
                             T* __restrict__ re, T* __restrict__ ru, T* __restrict__ rhs, T* __restrict__ x0,
                             int zero_x) {
    Idx3 P;
    long long cc;
    if (!cell_pos(G.n, P, cc)) return;
    const long long nc = G.ncell;
    const T s = vslot >= 0 ? (T)vscale[vslot] : (T)1;
    T r_rho = C[PcLr * nc + cc] * (s * v[cc]);
    T r_E = C[PcLE * nc + cc] * (s * v[nc + cc]);
    T r_e = (r_E - C[PcE * nc + cc] * r_rho) * C[PcInvRho * nc + cc];
    T ruv[ND];
    T dot_ur = (T)0;
#pragma unroll
    for (int c = 0; c < ND; ++c) ruv[c] = ru_at<T, T>(G, C, v, s, c, P);
    if (G.energy_form == 1) {
        T dot = (T)0;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            Idx3 Q = P;
            T uu = (T)0, au = (T)0;
            if (!(G.bc[d] == 1 && P.i[d] + 1 == G.n[d])) {
                Q.i[d] = (P.i[d] + 1 == G.n[d]) ? 0 : P.i[d] + 1;
                uu = C[(PcU + d) * nc + flat(G, Q.i[0], Q.i[1], Q.i[2])];
                au = ru_at<T, T>(G, C, v, s, d, Q);
            }
            dot = dot + (T)0.5 * (C[(PcU + d) * nc + cc] * ruv[d] + uu * au);
        }
        r_e = r_e - dot;
        dot_ur = dot;
    }
#pragma unroll
    for (int c = 0; c < ND; ++c) ru[c * nc + cc] = ruv[c];
    // r_p and r_e are kept for the back substitution of the sound-only scheme
    if (nf == 1) re[cc] = r_e;
    const long long mi = mg0(G, P);
    if (sizeof(T) == 8) {
        // double: the oracle's order, r_p = dp/drho r_rho + dp/de r_e, rhs = B^-1 (r_p, r_e)
        T r_p = C[PcDpdrho * nc + cc] * r_rho + C[PcDpde * nc + cc] * r_e;
        if (nf == 1) {
            rp[cc] = r_p;
            rhs[mi] = r_p * C[PcQ0 * nc + cc];
        } else {
            rhs[mi] = C[PcQ0 * nc + cc] * r_p + C[PcQ1 * nc + cc] * r_e;
            rhs[nc + mi] = C[PcQ2 * nc + cc] * r_p + C[PcQ3 * nc + cc] * r_e;
        }
    } else {
        // float: folded coefficients (see PcQ*), free of cancellation
        if (nf == 1) rp[cc] = C[PcPr * nc + cc] * r_rho + C[PcPE * nc + cc] * r_E - C[PcDpde * nc + cc] * dot_ur;
        rhs[mi] = C[PcQ0 * nc + cc] * r_rho + C[PcQ1 * nc + cc] * r_E - C[PcQ2 * nc + cc] * dot_ur;
        if (nf == 2)
            rhs[nc + mi] = C[PcQ3 * nc + cc] * r_rho + C[PcQ4 * nc + cc] * r_E - C[PcQ5 * nc + cc] * dot_ur;
    }
    // the first half sweep can take a zero start without reading x
    if (zero_x) {
        x0[mi] = (T)0;
        if (nf == 2) x0[nc + mi] = (T)0;
    }
}

template <typename T>
void launch_precond_in(const Grid& G, const T* C, const T* v, const double* vscale, int vslot, int nf, T* rp, T* re,
                       T* ru, MGLevel& L0, cudaStream_t s, int zero_x) {
    CELL_LAUNCH_T(k_precond_in, T, G, C, v, vscale, vslot, nf, rp, re, ru, (T*)L0.rhs, (T*)L0.x, zero_x);
}
template void launch_precond_in<double>(const Grid&, const double*, const double*, const double*, int, int, double*,
                                        double*, double*, MGLevel&, cudaStream_t, int);
template void launch_precond_in<float>(const Grid&, const float*, const float*, const double*, int, int, float*,
                                       float*, float*, MGLevel&, cudaStream_t, int);

// ---------------------------------------------------------------------------
// multigrid
// ---------------------------------------------------------------------------

__device__ __forceinline__ int wrap_up(int i, int n) { return i + 1 == n ? 0 : i + 1; }
__device__ __forceinline__ int wrap_dn(int i, int n) { return i == 0 ? n - 1 : i - 1; }

// Storage indices of the upper and lower neighbours of (a,b,c) along d
// (periodic wrap; wall neighbours carry zero face coefficients).
__device__ __forceinline__ void nb_index(const LvlDev& L, int d, int a, int b, int c, long long& ju, long long& jd) {
    if (d == 0) {
        ju = lflat(L, wrap_up(a, L.n[0]), b, c);
        jd = lflat(L, wrap_dn(a, L.n[0]), b, c);
    } else if (d == 1) {
        ju = lflat(L, a, wrap_up(b, L.n[1]), c);
        jd = lflat(L, a, wrap_dn(b, L.n[1]), c);
    } else {
        ju = lflat(L, a, b, wrap_up(c, L.n[2]));
        jd = lflat(L, a, b, wrap_dn(c, L.n[2]));
    }
}

// Red-black Gauss-Seidel half sweep over the cells of one colour (parity of
// i+j+k).  With an even x extent each thread takes one cell of the colour
// (compact mapping); otherwise threads of the other colour return.  Loops
// over directions and fields are unrolled at compile time (ND, NF) so all
// per-thread arrays stay in registers.  ZS: x is zero on entry, so the
// neighbour values are not read (first half sweep of a level that starts
// from zero; the cells of the other colour are overwritten before they are
// read).  A run-time flag in its place cost the kernel 12 registers and a
// quarter of its occupancy.
template <typename T, int NF, int ND, bool ZS>
__device__ __forceinline__ void smooth_cell(const LvlDev& Lv, const T* M, const T* K, T* x, const T* rhs, int a,
                                            int b, int c, int tr) {
    const long long cc = lflat(Lv, a, b, c);
    T dg[NF], of[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) { dg[f] = (T)0; of[f] = (T)0; }
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        if (Lv.n[d] == 1) continue;
        long long ju, jd;
        nb_index(Lv, d, a, b, c, ju, jd);
        const T ih2 = ih2_of<T>(Lv, d);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const T* Kd = K + (long long)(f * ND + d) * Lv.nc;
            T Kl = Kd[cc], Ku = Kd[ju];
            dg[f] = dg[f] + (Kl + Ku) * ih2;
            if (!ZS) {
                const T* xf = x + (long long)f * Lv.nc;
                of[f] = of[f] + (Ku * xf[ju] + Kl * xf[jd]) * ih2;
            }
        }
    }
    if (NF == 1) {
        x[cc] = (rhs[cc] + of[0]) / (M[cc] + dg[0]);
    } else {
        // tr: the transposed system (off-diagonal entries of the cell matrix swapped)
        T m01 = M[Lv.nc + cc], m10 = M[2 * Lv.nc + cc];
        T a11 = M[cc] + dg[0], a12 = tr ? m10 : m01, a21 = tr ? m01 : m10, a22 = M[3 * Lv.nc + cc] + dg[NF - 1];
        T b1 = rhs[cc] + of[0], b2 = rhs[Lv.nc + cc] + of[NF - 1];
        T det = a11 * a22 - a12 * a21;
        x[cc] = (a22 * b1 - a12 * b2) / det;
        x[Lv.nc + cc] = (a11 * b2 - a21 * b1) / det;
    }
}

template <typename T, int NF, int ND, bool ZS>
__global__ void k_smooth(LvlDev Lv, const T* __restrict__ M, const T* __restrict__ K, T* x,
                         const T* __restrict__ rhs, int colour, int compact, int tr) {
    const int b = blockIdx.y * blockDim.y + threadIdx.y;
    const int c = blockIdx.z;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = compact ? 2 * t + ((b + c + colour) & 1) : t;
    if (a >= Lv.n[0] || b >= Lv.n[1]) return;
    if (((a + b + c) & 1) != colour) return;
    smooth_cell<T, NF, ND, ZS>(Lv, M, K, x, rhs, a, b, c, tr);
}

#define MG_DISPATCH(KERNEL, GRID, BLOCK, ...)                                                 \
    do {                                                                                      \
        ++g_launch_count;                                                                     \
        if (nf == 1 && G.ndim == 3) KERNEL<T, 1, 3><<<GRID, BLOCK, 0, s>>>(__VA_ARGS__);      \
        else if (nf == 1) KERNEL<T, 1, 2><<<GRID, BLOCK, 0, s>>>(__VA_ARGS__);                \
        else if (G.ndim == 3) KERNEL<T, 2, 3><<<GRID, BLOCK, 0, s>>>(__VA_ARGS__);            \
        else KERNEL<T, 2, 2><<<GRID, BLOCK, 0, s>>>(__VA_ARGS__);                             \
    } while (0)

template <typename T, bool ZS>
static void smooth_launch(const Grid& G, int nf, MGLevel& Lv, int colour, cudaStream_t s, int tr) {
    int compact = (Lv.n[0] % 2 == 0) ? 1 : 0;
    int nx[3] = {compact ? Lv.n[0] / 2 : Lv.n[0], Lv.n[1], Lv.n[2]};
    CellLaunch cl = cell_launch(nx);
    ++g_launch_count;
    const LvlDev L = lvl(Lv);
    const T *M = (const T*)Lv.M, *K = (const T*)Lv.K, *rhs = (const T*)Lv.rhs;
    T* x = (T*)Lv.x;
    if (nf == 1 && G.ndim == 3) k_smooth<T, 1, 3, ZS><<<cl.grid, cl.block, 0, s>>>(L, M, K, x, rhs, colour, compact, tr);
    else if (nf == 1) k_smooth<T, 1, 2, ZS><<<cl.grid, cl.block, 0, s>>>(L, M, K, x, rhs, colour, compact, tr);
    else if (G.ndim == 3) k_smooth<T, 2, 3, ZS><<<cl.grid, cl.block, 0, s>>>(L, M, K, x, rhs, colour, compact, tr);
    else k_smooth<T, 2, 2, ZS><<<cl.grid, cl.block, 0, s>>>(L, M, K, x, rhs, colour, compact, tr);
}

template <typename T>
void launch_smooth(const Grid& G, int nf, MGLevel& Lv, int colour, cudaStream_t s, int tr, int zero_start) {
    if (zero_start) smooth_launch<T, true>(G, nf, Lv, colour, s, tr);
    else smooth_launch<T, false>(G, nf, Lv, colour, s, tr);
}
template void launch_smooth<double>(const Grid&, int, MGLevel&, int, cudaStream_t, int, int);
template void launch_smooth<float>(const Grid&, int, MGLevel&, int, cudaStream_t, int, int);

// residual rhs - A x at fine cell (a,b,c), field f
template <typename T, int NF, int ND>
__device__ __forceinline__ T fine_residual(const LvlDev& F, const T* M, const T* K, const T* x, const T* rhs, int f,
                                           int a, int b, int c, int tr) {
    const long long cc = lflat(F, a, b, c);
    T out;
    if (NF == 1) out = M[cc] * x[cc];
    else if (!tr) out = M[(f * 2 + 0) * F.nc + cc] * x[cc] + M[(f * 2 + 1) * F.nc + cc] * x[F.nc + cc];
    else out = M[(0 * 2 + f) * F.nc + cc] * x[cc] + M[(1 * 2 + f) * F.nc + cc] * x[F.nc + cc];
    const T* xf = x + (long long)f * F.nc;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        if (F.n[d] == 1) continue;
        long long ju, jd;
        nb_index(F, d, a, b, c, ju, jd);
        const T* Kd = K + (long long)(f * ND + d) * F.nc;
        T Kl = Kd[cc], Ku = Kd[ju];
        out = out - (Ku * (xf[ju] - xf[cc]) - Kl * (xf[cc] - xf[jd])) * ih2_of<T>(F, d);
    }
    return rhs[(long long)f * F.nc + cc] - out;
}

template <typename T, int NF, int ND>
__device__ __forceinline__ void residual_cell(const LvlDev& F, const T* M, const T* K, const T* x, const T* rhs,
                                              T* r, int a, int b, int c, int tr) {
    const long long cc = lflat(F, a, b, c);
#pragma unroll
    for (int f = 0; f < NF; ++f)
        r[(long long)f * F.nc + cc] = fine_residual<T, NF, ND>(F, M, K, x, rhs, f, a, b, c, tr);
}

// fine residual r = rhs - A x: one thread per fine cell, or (red_only) per
// colour-0 cell with the compact mapping of the smoother
template <typename T, int NF, int ND>
__global__ void k_residual_mg(LvlDev F, const T* __restrict__ M, const T* __restrict__ K, const T* __restrict__ x,
                             const T* __restrict__ rhs, T* __restrict__ r, int tr, int red_only, int compact) {
    const int b = blockIdx.y * blockDim.y + threadIdx.y;
    const int c = blockIdx.z;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = compact ? 2 * t + ((b + c) & 1) : t;
    if (a >= F.n[0] || b >= F.n[1]) return;
    if (red_only && ((a + b + c) & 1)) return;
    residual_cell<T, NF, ND>(F, M, K, x, rhs, r, a, b, c, tr);
}

// coarse right-hand side = mean of the children's residuals (pairs along x,
// then y, then z; colour-1 children count as zero when red_only); the coarse
// correction starts from zero
template <typename T, int NF, int ND>
__device__ __forceinline__ void restrict_cell(const LvlDev& F, const LvlDev& C, const T* r, T* rhsc, T* xc,
                                              const int ic[3], long long cc, int red_only, int zero_xc) {
    const bool cx = F.n[0] != C.n[0], cy = F.n[1] != C.n[1], cz = F.n[2] != C.n[2];
    const int x0 = cx ? 2 * ic[0] : ic[0], y0 = cy ? 2 * ic[1] : ic[1], z0 = cz ? 2 * ic[2] : ic[2];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const T* q = r + (long long)f * F.nc;
        auto child = [&](int xx, int yy, int zz) -> T {
            return (red_only && ((xx + yy + zz) & 1)) ? (T)0 : q[lflat(F, xx, yy, zz)];
        };
        auto xm = [&](int yy, int zz) -> T {
            T a = child(x0, yy, zz);
            return cx ? (a + child(x0 + 1, yy, zz)) / (T)2 : a;
        };
        auto ym = [&](int zz) -> T {
            T a = xm(y0, zz);
            return cy ? (a + xm(y0 + 1, zz)) / (T)2 : a;
        };
        T a = ym(z0);
        rhsc[(long long)f * C.nc + cc] = cz ? (a + ym(z0 + 1)) / (T)2 : a;
        if (zero_xc) xc[(long long)f * C.nc + cc] = (T)0;
    }
}

template <typename T, int NF, int ND>
__global__ void k_restrict(LvlDev F, LvlDev C, const T* __restrict__ r, T* __restrict__ rhsc, T* __restrict__ xc,
                           int red_only, int zero_xc) {
    int ic[3];
    long long cc;
    if (!lvl_pos(C, ic, cc)) return;
    restrict_cell<T, NF, ND>(F, C, r, rhsc, xc, ic, cc, red_only, zero_xc);
}

// Residual and restriction in one pass, after a pre-smoothing sweep (the
// colour-1 residual is zero): one thread per coarse cell evaluates the
// residuals of its colour-0 children where the restriction needs them, in
// the same pair order as restrict_cell, so the coarse right-hand side is
// bitwise that of the two-kernel path, without writing and re-reading the
// fine residual.
template <typename T, int NF, int ND>
__global__ void k_residual_restrict(LvlDev F, LvlDev C, const T* __restrict__ M, const T* __restrict__ K,
                                    const T* __restrict__ x, const T* __restrict__ rhs, T* __restrict__ rhsc,
                                    int tr) {
    // one thread per coarse cell and field: blockIdx.z runs over the coarse
    // z index of field 0, then of field 1
    int ic[3];
    ic[0] = blockIdx.x * blockDim.x + threadIdx.x;
    ic[1] = blockIdx.y * blockDim.y + threadIdx.y;
    const int f = blockIdx.z / C.n[2];
    ic[2] = blockIdx.z - f * C.n[2];
    if (ic[0] >= C.n[0] || ic[1] >= C.n[1]) return;
    const long long cc = lflat(C, ic[0], ic[1], ic[2]);
    const bool cx = F.n[0] != C.n[0], cy = F.n[1] != C.n[1], cz = F.n[2] != C.n[2];
    const int x0 = cx ? 2 * ic[0] : ic[0], y0 = cy ? 2 * ic[1] : ic[1], z0 = cz ? 2 * ic[2] : ic[2];
    {
        auto child = [&](int xx, int yy, int zz) -> T {
            return ((xx + yy + zz) & 1) ? (T)0 : fine_residual<T, NF, ND>(F, M, K, x, rhs, f, xx, yy, zz, tr);
        };
        auto xm = [&](int yy, int zz) -> T {
            T a = child(x0, yy, zz);
            return cx ? (a + child(x0 + 1, yy, zz)) / (T)2 : a;
        };
        auto ym = [&](int zz) -> T {
            T a = xm(y0, zz);
            return cy ? (a + xm(y0 + 1, zz)) / (T)2 : a;
        };
        T a = ym(z0);
        rhsc[(long long)f * C.nc + cc] = cz ? (a + ym(z0 + 1)) / (T)2 : a;
    }
}

template <typename T>
void launch_restrict(const Grid& G, int nf, MGLevel& F, MGLevel& C, cudaStream_t s, int tr, int red_only) {
    CellLaunch cl = cell_launch(C.n);
    if (red_only) {
        // after a pre-smoothing sweep the coarse level starts with a
        // zero-start half sweep, so its x needs no zeroing
        dim3 grid = cl.grid;
        grid.z *= nf;
        MG_DISPATCH(k_residual_restrict, grid, cl.block, lvl(F), lvl(C), (const T*)F.M, (const T*)F.K,
                    (const T*)F.x, (const T*)F.rhs, (T*)C.rhs, tr);
        return;
    }
    CellLaunch fl = cell_launch(F.n);
    MG_DISPATCH(k_residual_mg, fl.grid, fl.block, lvl(F), (const T*)F.M, (const T*)F.K, (const T*)F.x,
                (const T*)F.rhs, (T*)F.r, tr, 0, 0);
    MG_DISPATCH(k_restrict, cl.grid, cl.block, lvl(F), lvl(C), (const T*)F.r, (T*)C.rhs, (T*)C.x, 0, 1);
}
template void launch_restrict<double>(const Grid&, int, MGLevel&, MGLevel&, cudaStream_t, int, int);
template void launch_restrict<float>(const Grid&, int, MGLevel&, MGLevel&, cudaStream_t, int, int);

// r = rhs - A x on every cell of level F (the inner-solve residual that the
// preconditioner's accuracy monitor and its tolerance-driven cycling read)
template <typename T>
void launch_mg_residual(const Grid& G, int nf, MGLevel& F, cudaStream_t s) {
    CellLaunch fl = cell_launch(F.n);
    MG_DISPATCH(k_residual_mg, fl.grid, fl.block, lvl(F), (const T*)F.M, (const T*)F.K, (const T*)F.x,
                (const T*)F.rhs, (T*)F.r, 0, 0, 0);
}
template void launch_mg_residual<double>(const Grid&, int, MGLevel&, cudaStream_t);
template void launch_mg_residual<float>(const Grid&, int, MGLevel&, cudaStream_t);

// Cell-centred linear prolongation x_f += P x_c for one coarse cell: load
// the coarse neighbourhood once (3 values along each coarsened direction)
// and update the cell's 2^k children.  A child at offset
// delta along a coarsened direction interpolates 3/4 of its parent and 1/4
// of the parent's neighbour on its side (periodic wrap; at a wall the parent
// itself), along x, then y, then z.
template <typename T, int NF, int ND>
__device__ __forceinline__ void prolong_cell(int bc0, int bc1, int bc2, const LvlDev& F, const LvlDev& C,
                                             const T* xc, T* xf, const int ic[3]) {
    const bool cd[3] = {F.n[0] != C.n[0], F.n[1] != C.n[1], F.n[2] != C.n[2]};
    const int bc[3] = {bc0, bc1, bc2};
    // coarse indices at offsets -1, 0, +1 along each direction
    int nb[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int i = ic[d], n = C.n[d];
        nb[d][1] = i;
        if (!cd[d]) {
            nb[d][0] = nb[d][2] = i;
        } else if (bc[d] == 0) {
            nb[d][0] = wrapi(i - 1, n);
            nb[d][2] = wrapi(i + 1, n);
        } else {
            nb[d][0] = i - 1 < 0 ? i : i - 1;
            nb[d][2] = i + 1 >= n ? i : i + 1;
        }
    }
    const T w0 = (T)0.75, w1 = (T)0.25;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const T* q = xc + (long long)f * C.nc;
        T* out = xf + (long long)f * F.nc;
        T v[3][3][3];       // v[z][y][x], offsets -1..+1 (only 0 along a direction not coarsened)
#pragma unroll
        for (int kz = 0; kz < 3; ++kz)
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int kx = 0; kx < 3; ++kx)
                    v[kz][ky][kx] = q[lflat(C, nb[0][kx], nb[1][ky], nb[2][kz])];
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
            if (dz && !cd[2]) continue;
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                if (dy && !cd[1]) continue;
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    if (dx && !cd[0]) continue;
                    // the other parent lies at offset -1 for child 0 and +1 for child 1
                    auto along_x = [&](int yy, int zz) -> T {
                        const T a = v[zz][yy][1], o = dx ? v[zz][yy][2] : v[zz][yy][0];
                        return cd[0] ? w0 * a + w1 * o : a;
                    };
                    auto along_y = [&](int zz) -> T {
                        const T a = along_x(1, zz), o = dy ? along_x(2, zz) : along_x(0, zz);
                        return cd[1] ? w0 * a + w1 * o : a;
                    };
                    const T a = along_y(1), o = dz ? along_y(2) : along_y(0);
                    const T val = cd[2] ? w0 * a + w1 * o : a;
                    const int fx = cd[0] ? 2 * ic[0] + dx : ic[0];
                    const int fy = cd[1] ? 2 * ic[1] + dy : ic[1];
                    const int fz = cd[2] ? 2 * ic[2] + dz : ic[2];
                    const long long j = lflat(F, fx, fy, fz);
                    out[j] = out[j] + val;
                }
            }
        }
    }
}

// one thread per coarse cell and field (blockIdx.z runs over field, then
// coarse z): one field's 27 coarse values live at a time, which halves the
// registers of the two-field case (128 -> 64) and doubles its occupancy
template <typename T, int ND>
__global__ void k_prolong(int bc0, int bc1, int bc2, LvlDev F, LvlDev C, const T* __restrict__ xc,
                          T* __restrict__ xf) {
    const int f = blockIdx.z / C.n[2];
    int ic[3];
    ic[0] = blockIdx.x * blockDim.x + threadIdx.x;
    ic[1] = blockIdx.y * blockDim.y + threadIdx.y;
    ic[2] = blockIdx.z - f * C.n[2];
    if (ic[0] >= C.n[0] || ic[1] >= C.n[1]) return;
    prolong_cell<T, 1, ND>(bc0, bc1, bc2, F, C, xc + (long long)f * C.nc, xf + (long long)f * F.nc, ic);
}

template <typename T>
void launch_prolong(const Grid& G, int nf, MGLevel& F, MGLevel& C, cudaStream_t s) {
    CellLaunch cl = cell_launch(C.n);
    cl.grid.z = (unsigned)(C.n[2] * nf);
    ++g_launch_count;
    if (G.ndim == 3)
        k_prolong<T, 3><<<cl.grid, cl.block, 0, s>>>(G.bc[0], G.bc[1], G.bc[2], lvl(F), lvl(C), (const T*)C.x, (T*)F.x);
    else
        k_prolong<T, 2><<<cl.grid, cl.block, 0, s>>>(G.bc[0], G.bc[1], G.bc[2], lvl(F), lvl(C), (const T*)C.x, (T*)F.x);
}
template void launch_prolong<double>(const Grid&, int, MGLevel&, MGLevel&, cudaStream_t);
template void launch_prolong<float>(const Grid&, int, MGLevel&, MGLevel&, cudaStream_t);

template <typename T>
__device__ __forceinline__ void coarsest_cell(int nf, const T* M, const T* rhs, T* x, int tr) {
    if (nf == 1) {
        x[0] = rhs[0] / M[0];
    } else {
        T a11 = M[0], a12 = tr ? M[2] : M[1], a21 = tr ? M[1] : M[2], a22 = M[3];
        T det = a11 * a22 - a12 * a21;
        x[0] = (a22 * rhs[0] - a12 * rhs[1]) / det;
        x[1] = (a11 * rhs[1] - a21 * rhs[0]) / det;
    }
}

template <typename T>
__global__ void k_coarsest(int nf, const T* __restrict__ M, const T* __restrict__ rhs, T* __restrict__ x, int tr) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    coarsest_cell<T>(nf, M, rhs, x, tr);
}

template <typename T>
void launch_coarsest(int nf, MGLevel& C, cudaStream_t s, int tr) {
    ++g_launch_count;
    k_coarsest<T><<<1, 32, 0, s>>>(nf, (const T*)C.M, (const T*)C.rhs, (T*)C.x, tr);
}
template void launch_coarsest<double>(int, MGLevel&, cudaStream_t, int);
template void launch_coarsest<float>(int, MGLevel&, cudaStream_t, int);

// The coarse end of a V-cycle in one block.  Below a few thousand cells a
// level's kernels last 4-8 us each whatever their size (launch and
// dependency latency, about 11 launches per level), so the levels from the
// first one at or below kTailCells down to the single-cell level run as
// phases of one kernel separated by block barriers: the same per-cell
// functions in the same order of phases as the separate launches (results
// agree to rounding: the compiler may contract multiply-adds differently in
// the two contexts).  Every phase visits its cells with a block-stride loop;
// x, rhs and r are written and read within the kernel, so they are read
// through plain (coherent) loads.
struct TailLevel {
    LvlDev L;
    const void* M;
    const void* K;
    void* x;
    void* rhs;
    void* r;
};
struct TailArgs {
    TailLevel lv[kTailMaxLevels];
    int nlev;
    int bc[3];
    int nu1, nu2, tr;
};

template <typename T, int NF, int ND, bool ZS>
__device__ __forceinline__ void tail_smooth(const TailLevel& V, int colour, int tr) {
    const LvlDev& L = V.L;
    const int compact = (L.n[0] % 2 == 0) ? 1 : 0;
    const int nx = compact ? L.n[0] / 2 : L.n[0];
    const int total = nx * L.n[1] * L.n[2];
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int t = i % nx, rem = i / nx, b = rem % L.n[1], c = rem / L.n[1];
        const int a = compact ? 2 * t + ((b + c + colour) & 1) : t;
        if (((a + b + c) & 1) != colour) continue;
        smooth_cell<T, NF, ND, ZS>(L, (const T*)V.M, (const T*)V.K, (T*)V.x, (const T*)V.rhs, a, b, c, tr);
    }
}

template <typename T, int NF, int ND>
__global__ void __launch_bounds__(kTailThreads) k_vcycle_tail(TailArgs A) {
    const int red_only = A.nu1 > 0 ? 1 : 0;
    // descent: pre-smoothing (the first half sweep of every coarse level
    // starts from zero), residual on colour 0 and restriction
    for (int l = 0; l + 1 < A.nlev; ++l) {
        const TailLevel& V = A.lv[l];
        const TailLevel& W = A.lv[l + 1];
        for (int k = 0; k < A.nu1; ++k) {
            if (k == 0) tail_smooth<T, NF, ND, true>(V, 0, A.tr);
            else tail_smooth<T, NF, ND, false>(V, 0, A.tr);
            __syncthreads();
            tail_smooth<T, NF, ND, false>(V, 1, A.tr);
            __syncthreads();
        }
        {
            const LvlDev& F = V.L;
            const int compact = (red_only && F.n[0] % 2 == 0) ? 1 : 0;
            const int nx = compact ? F.n[0] / 2 : F.n[0];
            const int total = nx * F.n[1] * F.n[2];
            for (int i = threadIdx.x; i < total; i += blockDim.x) {
                const int t = i % nx, rem = i / nx, b = rem % F.n[1], c = rem / F.n[1];
                const int a = compact ? 2 * t + ((b + c) & 1) : t;
                if (red_only && ((a + b + c) & 1)) continue;
                residual_cell<T, NF, ND>(F, (const T*)V.M, (const T*)V.K, (const T*)V.x, (const T*)V.rhs, (T*)V.r, a,
                                         b, c, A.tr);
            }
        }
        __syncthreads();
        {
            const LvlDev& C = W.L;
            const int total = C.n[0] * C.n[1] * C.n[2];
            for (int i = threadIdx.x; i < total; i += blockDim.x) {
                int ic[3];
                ic[0] = i % C.n[0];
                ic[1] = (i / C.n[0]) % C.n[1];
                ic[2] = i / (C.n[0] * C.n[1]);
                restrict_cell<T, NF, ND>(V.L, C, (const T*)V.r, (T*)W.rhs, (T*)W.x, ic, lflat(C, ic[0], ic[1], ic[2]),
                                         red_only, red_only ? 0 : 1);
            }
        }
        __syncthreads();
    }
    const TailLevel& Z = A.lv[A.nlev - 1];
    if (threadIdx.x == 0) coarsest_cell<T>(NF, (const T*)Z.M, (const T*)Z.rhs, (T*)Z.x, A.tr);
    __syncthreads();
    // ascent: prolongation and post-smoothing
    for (int l = A.nlev - 2; l >= 0; --l) {
        const TailLevel& V = A.lv[l];
        const TailLevel& W = A.lv[l + 1];
        const LvlDev& C = W.L;
        const int total = C.n[0] * C.n[1] * C.n[2];
        for (int i = threadIdx.x; i < total; i += blockDim.x) {
            int ic[3];
            ic[0] = i % C.n[0];
            ic[1] = (i / C.n[0]) % C.n[1];
            ic[2] = i / (C.n[0] * C.n[1]);
            prolong_cell<T, NF, ND>(A.bc[0], A.bc[1], A.bc[2], V.L, C, (const T*)W.x, (T*)V.x, ic);
        }
        __syncthreads();
        for (int k = 0; k < A.nu2; ++k) {
            tail_smooth<T, NF, ND, false>(V, 1, A.tr);
            __syncthreads();
            tail_smooth<T, NF, ND, false>(V, 0, A.tr);
            __syncthreads();
        }
    }
}

template <typename T>
void launch_vcycle_tail(const Grid& G, int nf, const MGLevel* levels, int nlev, int nu1, int nu2, cudaStream_t s,
                        int tr) {
    TailArgs A;
    A.nlev = nlev;
    for (int d = 0; d < 3; ++d) A.bc[d] = G.bc[d];
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.tr = tr;
    for (int l = 0; l < nlev; ++l) {
        A.lv[l].L = lvl(levels[l]);
        A.lv[l].M = levels[l].M;
        A.lv[l].K = levels[l].K;
        A.lv[l].x = levels[l].x;
        A.lv[l].rhs = levels[l].rhs;
        A.lv[l].r = levels[l].r;
    }
    ++g_launch_count;
    if (nf == 1 && G.ndim == 3) k_vcycle_tail<T, 1, 3><<<1, kTailThreads, 0, s>>>(A);
    else if (nf == 1) k_vcycle_tail<T, 1, 2><<<1, kTailThreads, 0, s>>>(A);
    else if (G.ndim == 3) k_vcycle_tail<T, 2, 3><<<1, kTailThreads, 0, s>>>(A);
    else k_vcycle_tail<T, 2, 2><<<1, kTailThreads, 0, s>>>(A);
}
template void launch_vcycle_tail<double>(const Grid&, int, const MGLevel*, int, int, int, cudaStream_t, int);
template void launch_vcycle_tail<float>(const Grid&, int, const MGLevel*, int, int, int, cudaStream_t, int);

// ---------------------------------------------------------------------------
// back substitution and transform out
// ---------------------------------------------------------------------------

// du on the lower face of cell Q in direction c
template <typename T>
__device__ __forceinline__ T du_at(const Grid& G, const T* C, T dt, const T* ru, const T* dp, int c, const Idx3& Q) {
    const long long nc = G.ncell;
    const long long j = flat(G, Q.i[0], Q.i[1], Q.i[2]);
    int o[3] = {0, 0, 0};
    o[c] = -1;
    int a = cell_map(Q.i[0] + o[0], G.n[0], G.bc[0]);
    int b = cell_map(Q.i[1] + o[1], G.n[1], G.bc[1]);
    int cz = cell_map(Q.i[2] + o[2], G.n[2], G.bc[2]);
    Idx3 L;
    L.i[0] = a; L.i[1] = b; L.i[2] = cz;
    // dp lives in the (colour-split) multigrid array of level 0
    return dt * (ru[c * nc + j] - C[(PcThf + c) * nc + j] * (dp[mg0(G, Q)] - dp[mg0(G, L)]));
}

// One wave of blocks, each visiting cell tiles with a grid stride and
// reducing its partial |z|^2 once: with one tile per block the block-wide
// reduction (two barriers per 128 cells) cost a quarter of the kernel.
template <int ND, typename T>
__global__ void k_precond_out(Grid G, const T* __restrict__ C, double dt_d, double idt_d, int nf,
                              const T* __restrict__ rp,
                              const T* __restrict__ re, const T* __restrict__ ru, const T* __restrict__ x,
                              T* __restrict__ z, double* __restrict__ partials, int ntiles) {
    __shared__ double sh[32];
    // |z|^2: in double for a double z; for a float z as a compensated float
    // pair (no FP64 instruction per element), converted once per thread, or
    // redone in double from the stored z by a thread whose values are too
    // large or too small for float squares (sq_range_unsafe)
    double acc = 0.0;
    CompF accf = {0.f, 0.f};
    float mx = 0.f;
    const long long nc = G.ncell;
    const T dt = (T)dt_d, idt = (T)idt_d;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        Idx3 P;
        long long cc;
        if (!cell_pos_tile(G.n, tile, P, cc)) continue;
        const long long mi = mg0(G, P);
        const T dp = x[mi];
        T de;
        if (nf == 1) de = dt * (re[cc] + (dp * idt - rp[cc]) * C[PcCde * nc + cc]);
        else de = x[nc + mi];
        T du[ND];
#pragma unroll
        for (int c = 0; c < ND; ++c) du[c] = du_at<T>(G, C, dt, ru, x, c, P);
        T dE = de;
        if (G.energy_form == 1) {
            T dot = (T)0;
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                T uu = (T)0, au = (T)0;
                if (!(G.bc[d] == 1 && P.i[d] + 1 == G.n[d])) {
                    Idx3 Q = P;
                    Q.i[d] = (P.i[d] + 1 == G.n[d]) ? 0 : P.i[d] + 1;
                    uu = C[(PcU + d) * nc + flat(G, Q.i[0], Q.i[1], Q.i[2])];
                    au = du_at<T>(G, C, dt, ru, x, d, Q);
                }
                dot = dot + (T)0.5 * (C[(PcU + d) * nc + cc] * du[d] + uu * au);
            }
            dE = de + dot;
        }
        T drho = (dp - C[PcDpde * nc + cc] * de) * C[PcInvDpdrho * nc + cc];
        T out[2 + ND];
        out[0] = drho * C[PcRinvR * nc + cc];
        out[1] = dE * C[PcRinvE * nc + cc];
#pragma unroll
        for (int c = 0; c < ND; ++c) out[2 + c] = du[c] * C[(PcRinvU + c) * nc + cc];
#pragma unroll
        for (int k = 0; k < 2 + ND; ++k) {
            z[k * nc + cc] = out[k];
            if (sizeof(T) == 8) {
                const double zd = (double)out[k];
                acc += zd * zd;
            } else {
                const float zf = (float)out[k];
                comp_fma(accf, zf, zf);
                mx = fmaxf(mx, fabsf(zf));
            }
        }
    }
    if (sizeof(T) != 8) {
        if (sq_range_unsafe(mx)) {
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
                Idx3 P;
                long long cc;
                if (!cell_pos_tile(G.n, tile, P, cc)) continue;
#pragma unroll
                for (int k = 0; k < 2 + ND; ++k) {
                    const double zd = (double)z[k * nc + cc];
                    acc += zd * zd;
                }
            }
        } else {
            acc = (double)accf.s + (double)accf.e;
        }
    }
    double s = block_sum<128>(acc, sh);
    if (thread_linear() == 0) partials[blockIdx.x] = s;
}

// blocks of one wave of k_precond_out (occupancy query, once per kernel)
template <auto FN>
static int one_wave(int threads) {
    static const int g = [threads] {
        int dev = 0, nsm = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, FN, threads, 0);
        long long w = (long long)(nsm > 0 ? nsm : 1) * (occ > 0 ? occ : 1);
        return (int)(w < kMaxRedBlocks ? w : kMaxRedBlocks);
    }();
    return g;
}

template <typename T>
int launch_precond_out(const Grid& G, const T* C, double dt, int nf, const T* rp, const T* re, const T* ru,
                       const MGLevel& L0, T* z, double* partials, cudaStream_t s) {
    CellLaunch cl = cell_launch(G.n);
    const long long nt = (long long)cl.grid.x * cl.grid.y * cl.grid.z;
    const int ntiles = (int)nt;
    int g = G.ndim == 3 ? one_wave<k_precond_out<3, T>>(cl.block.x * cl.block.y)
                        : one_wave<k_precond_out<2, T>>(cl.block.x * cl.block.y);
    if (g > ntiles) g = ntiles;
    ++g_launch_count;
    if (G.ndim == 3)
        k_precond_out<3, T><<<g, cl.block, 0, s>>>(G, C, dt, 1.0 / dt, nf, rp, re, ru, (const T*)L0.x, z, partials,
                                                   ntiles);
    else
        k_precond_out<2, T><<<g, cl.block, 0, s>>>(G, C, dt, 1.0 / dt, nf, rp, re, ru, (const T*)L0.x, z, partials,
                                                   ntiles);
    return g;
}
template int launch_precond_out<double>(const Grid&, const double*, double, int, const double*, const double*,
                                        const double*, const MGLevel&, double*, double*, cudaStream_t);
template int launch_precond_out<float>(const Grid&, const float*, double, int, const float*, const float*,
                                       const float*, const MGLevel&, float*, double*, cudaStream_t);

}  // namespace jfnk
