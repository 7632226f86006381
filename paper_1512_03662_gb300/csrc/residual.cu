// Finite-volume right-hand side R_U(X) of the paper's Sect. 2 on the
// staggered grid, and the residual-type operators built from it:
//   G(X)  = U(X)/dt - theta R_U(X)                 (Jv, Newton set-up)
//   b^n   = U(X^n)/dt + (1-theta) R_U(X^n)          (Eq. crank_nicholson)
//   F_U   = G(X) - b^n
//   Jv    = L^-1 [G(X + delta R v) - G(X)] / delta   (Eqs. jacobian_free, pert_old)
//
// The evaluation is split so that every van Leer slope and every flux is
// computed once per slot (the FP64 rate of sm_103a, about 0.6 TFMA/s, binds
// these kernels, not HBM).  The flux kernels form their products on the
// integer pipes (emu64.cuh: the same correctly rounded bits, checked once per
// evaluation, redone on the FP64 pipe where an operand left the normal
// range) and address neighbours with branch-free offsets (common.cuh), so
// the FP64 pipe keeps the sums and the fused multiply-adds only:
//   k_eos          p, T per cell (perturbed state written first by k_perturb)
//   k_face_fluxes  mass flux Fm_d and energy flux FE_d (advective part minus
//                  conduction) on the lower face of every cell, per direction
//   k_mom_fluxes   momentum fluxes Psi_cd: for c == d at cell centres, for
//                  c != d on the edges between faces; stored doubled (carried
//                  by the sum of two mass fluxes, not their mean: exact, and
//                  the assemble takes the 1/2 into 1/(2 dx))
//   k_assemble     divergences, sources, U(X) and the requested combination
//
// Reconstruction (van Leer 1974): slope 2ab/(a+b) if ab > 0 else 0; the
// upwind face value is q_L + s_L/2 when the upwinding speed is >= 0, else
// q_R - s_R/2.  Only the slope on the upwind side is evaluated.
#include "common.cuh"
#include "kernels.h"

namespace jfnk {

long long g_launch_count = 0;

template <typename TZ>
__global__ void k_perturb(Grid G, const double* __restrict__ X, const TZ* __restrict__ z,
                          const double* __restrict__ R, const double* __restrict__ scal, int delta_slot,
                          double* __restrict__ Xp, long long nvec) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= nvec) return;
    const double delta = scal[delta_slot];
    // R_rho = rho and R_e = e (Eq. jacobian_system_norm; k_scaling stores
    // them as copies of X): the density and energy rows take R from X
    // instead of reading it again
    const double x = X[k];
    const double r = k < 2 * G.ncell ? x : R[k];
    Xp[k] = x + delta * (r * to_f64(z[k]));
}

__device__ __forceinline__ double conductivity(const Grid& G, double T) {
    return G.chi3 ? G.K0 * (T * T * T) : G.K0 * pow(T, G.chi_exp);
}

// p, T and (with conduction) chi = K0 T^exp per cell, each formed once for
// all the faces that use it.  This kernel stays on the FP64 pipe: it is
// bound by memory latency, and its six products on the integer pipes made
// it slower (0.20 -> 0.23 ms at 256^3, the ALU pipe 74 % busy).
template <int ND>
__global__ void k_eos(Grid G, const double* __restrict__ X, double* __restrict__ p, double* __restrict__ T,
                      double* __restrict__ chi) {
    Idx3 P;
    long long c;
    if (!cell_pos(G.n, P, c)) return;
    const long long nc = G.ncell;
    double rho = X[c];
    double e = X[nc + c];
    if (G.energy_form == 1) {
        double ke = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const double* u = X + (2 + d) * nc + c;
            const double ul = normal_along(G, u, P, d, 0);
            const double uu = normal_along(G, u, P, d, 1);
            ke = ke + 0.25 * (ul * ul + uu * uu);
        }
        e = e - ke;
    }
    p[c] = G.gm1 * rho * e;
    const double Tc = G.gm1 * e;
    T[c] = Tc;
    if (G.has_cond) chi[c] = conductivity(G, Tc);
}

// Mass and energy flux of the lower face of direction d of one cell (its
// own reciprocal batch of two); with checked Ops nothing is written unless
// every operation was in range.
template <int ND, int EF, class O>
__device__ __forceinline__ bool face_flux_dir(O ops, const Grid& G, const double* __restrict__ X,
                                              const double* __restrict__ p, const double* __restrict__ T,
                                              const double* __restrict__ chi, double* __restrict__ Fm,
                                              double* __restrict__ FE, int d, const Idx3& P, long long c) {
    const long long nc = G.ncell;
    const double* rho = X + c;
    const double* E = X + nc + c;
    const double u = normal_along(G, X + (2 + d) * nc + c, P, d, 0);
    const int om2 = cell_off(G, P, d, -2), om1 = cell_off(G, P, d, -1), op1 = cell_off(G, P, d, 1);
    const double r0 = __ldg(rho), e0 = __ldg(E);
    const double r2 = __ldg(rho + om2), e2 = __ldg(E + om2);
    const double r1 = __ldg(rho + om1), e1 = __ldg(E + om1);
    const double r3 = __ldg(rho + op1), e3 = __ldg(E + op1);
    // upwind side: cell i-1 for u >= 0 (ties to the lower side), else cell i
    const bool left = nonneg(u);
    const Upw ur = upwind_parts(left ? r1 : r0, left ? r2 : r3, left ? r0 : r1, ops);
    const Upw ue = upwind_parts(left ? e1 : e0, left ? e2 : e3, left ? e0 : e1, ops);
    // one reciprocal for the two limited slopes
    double den[2] = {ur.den, ue.den}, inv[2];
    recip_all<2>(den, inv, ops);
    const double fm = ops.mul(u, fma(ur.num, inv[0], ur.q));
    double fe = ops.mul(fm, fma(ue.num, inv[1], ue.q));
    if constexpr (EF == 1) {
        const double pl = __ldg(p + c + om1);
        fe = fe + 0.5 * (pl + __ldg(p + c)) * u;
    }
    if (G.has_cond) {
        // q = chi_f (T_c - T_l) / dx with chi_f the mean of the two cells
        const double Tl = __ldg(T + c + om1);
        const double chil = __ldg(chi + c + om1);
        const double sq = ops.mul(chil + __ldg(chi + c), G.hidx[d]);
        fe = fma(-sq, __ldg(T + c) - Tl, fe);
    }
    if (!ops.valid()) return false;
    Fm[d * nc + c] = fm;                  // mass flux (every consumer takes half the sum of two)
    FE[d * nc + c] = fe;
    return true;
}

// products of the face fluxes on the integer pipes, sums on the FP64 pipe
using FaceOps = IntOps<true, false>;

// the FP64-pipe redo of one direction, out of line: inlined, the compiler
// predicates part of it into the fast path, where its FP64 instructions
// still occupy the FP64 pipe with every lane switched off
template <int ND, int EF>
__device__ __noinline__ void face_flux_dir_fp64(const Grid G, const double* __restrict__ X,
                                                const double* __restrict__ p, const double* __restrict__ T,
                                                const double* __restrict__ chi, double* __restrict__ Fm,
                                                double* __restrict__ FE, int d, const Idx3 P, long long c) {
    face_flux_dir<ND, EF>(FpOps(), G, X, p, T, chi, Fm, FE, d, P, c);
}

// one direction at a time (a reciprocal batch of two instead of 2 ND keeps
// the live state small); at least 6 blocks of 128 threads per SM: 80
// registers.  The energy form EF (0: internal, 1: total) is a template
// parameter: as a runtime test its pressure-work term was predicated, and
// its FP64 instructions occupied the FP64 pipe with every lane off.
template <int ND, int EF>
__global__ void __launch_bounds__(128, 6) k_face_fluxes(Grid G, const double* __restrict__ X, const double* __restrict__ p,
                              const double* __restrict__ T, const double* __restrict__ chi, double* __restrict__ Fm,
                              double* __restrict__ FE) {
    Idx3 P;
    long long c;
    if (!cell_pos(G.n, P, c)) return;
#pragma unroll
    for (int d = 0; d < ND; ++d)
        if (!face_flux_dir<ND, EF>(FaceOps(), G, X, p, T, chi, Fm, FE, d, P, c))
            face_flux_dir_fp64<ND, EF>(G, X, p, T, chi, Fm, FE, d, P, c);
}

// Momentum fluxes Psi_cd (d = 0..ND-1) of component c at one cell; with
// checked Ops nothing is written unless every operation was in range.
template <int ND, class O>
__device__ __forceinline__ bool mom_fluxes_component(O ops, const Grid& G, const double* __restrict__ X,
                                                     const double* __restrict__ Fm, double* __restrict__ Psi,
                                                     int c, const Idx3& P, long long cc) {
    const long long nc = G.ncell;
    constexpr int nd = ND;
    const double* uc = X + (2 + c) * nc + cc;         // pointers at the thread's own slot
    // pass 1: loads, carrying mass flux and split upwind value
    double mf[nd];
    Upw up[nd];
#pragma unroll
    for (int d = 0; d < nd; ++d) {
        double m, q_near, q_far, q_other;
        const double* fmd = Fm + d * nc + cc;
        if (c == d) {
            // flux at the cell centre between faces i and i+1 along c, carried
            // by the mean of the two mass fluxes (here their sum: Psi doubled)
            m = __ldg(fmd) + face_up_at(G, fmd, P, c);
            const double um = normal_along(G, uc, P, c, -1);
            const double u0 = normal_along(G, uc, P, c, 0);
            const double u1 = normal_along(G, uc, P, c, 1);
            const double u2 = normal_along(G, uc, P, c, 2);
            const bool left = nonneg(m);
            q_near = left ? u0 : u1;
            q_far = left ? um : u2;
            q_other = left ? u1 : u0;
        } else {
            // flux on the edge between c-face i_c and d-face i_d
            m = __ldg(fmd + cell_off(G, P, c, -1)) + __ldg(fmd);
            const double u2 = normal_across(G, uc, P, c, d, -2);
            const double u1 = normal_across(G, uc, P, c, d, -1);
            const double u0 = normal_across(G, uc, P, c, d, 0);
            const double u3 = normal_across(G, uc, P, c, d, 1);
            const bool left = nonneg(m);
            q_near = left ? u1 : u0;
            q_far = left ? u2 : u3;
            q_other = left ? u0 : u1;
        }
        mf[d] = m;
        up[d] = upwind_parts(q_near, q_far, q_other, ops);
    }
    // pass 2: one division for the nd limited slopes of component c (a
    // batch of nd keeps the kernel near 56 registers; one batch of nd^2
    // needed 102 and ran 20 % slower at the lower occupancy)
    double den[nd], inv[nd], psi[nd];
#pragma unroll
    for (int d = 0; d < nd; ++d) den[d] = up[d].den;
    recip_all<nd>(den, inv, ops);
#pragma unroll
    for (int d = 0; d < nd; ++d) psi[d] = ops.mul(mf[d], fma(up[d].num, inv[d], up[d].q));
    if (!ops.valid()) return false;
#pragma unroll
    for (int d = 0; d < nd; ++d) Psi[(c * nd + d) * nc + cc] = psi[d];
    return true;
}

// products of the momentum fluxes on the integer pipes, sums on the FP64 pipe
using MomOps = IntOps<true, false>;

// the FP64-pipe redo of one component, out of line (see face_flux_dir_fp64)
template <int ND>
__device__ __noinline__ void mom_fluxes_component_fp64(const Grid G, const double* __restrict__ X,
                                                       const double* __restrict__ Fm, double* __restrict__ Psi,
                                                       int c, const Idx3 P, long long cc) {
    mom_fluxes_component<ND>(FpOps(), G, X, Fm, Psi, c, P, cc);
}

// 128-thread blocks, at least 10 resident per SM (48 registers); the
// components run as a loop (not unrolled), which keeps the straight-line
// code, and the instruction-cache misses of its warps, three times smaller
template <int ND>
__global__ void __launch_bounds__(128, 10) k_mom_fluxes(Grid G, const double* __restrict__ X,
                                                        const double* __restrict__ Fm, double* __restrict__ Psi) {
    Idx3 P;
    long long cc;
    if (!cell_pos(G.n, P, cc)) return;
#pragma unroll 1
    for (int c = 0; c < ND; ++c)
        if (!mom_fluxes_component<ND>(MomOps(), G, X, Fm, Psi, c, P, cc))
            mom_fluxes_component_fp64<ND>(G, X, Fm, Psi, c, P, cc);
}

// Divergences and sources Rv and conserved variables Uv of one cell, the
// products on the integer pipes with checked Ops (false, nothing valid,
// where one was out of range)
template <int ND, class O>
__device__ __forceinline__ bool assemble_terms(O ops, const Grid& G, const double* __restrict__ X,
                                               const double* __restrict__ p, const double* __restrict__ Fm,
                                               const double* __restrict__ FE, const double* __restrict__ Psi,
                                               const Idx3& P, long long cc, double (&Uv)[2 + ND],
                                               double (&Rv)[2 + ND]) {
    const long long nc = G.ncell;
    constexpr int nd = ND;
    double Rr = 0.0, RE = 0.0, divu = 0.0;
#pragma unroll
    for (int d = 0; d < nd; ++d) {
        const double* fmd = Fm + d * nc + cc;              // pointers at the thread's own cell
        const double* fed = FE + d * nc + cc;
        const double fm0 = __ldg(fmd), fm1 = face_up_at(G, fmd, P, d);
        const double fe0 = __ldg(fed), fe1 = face_up_at(G, fed, P, d);
        Rr = Rr - (fm1 - fm0) * G.idx[d];
        RE = RE - (fe1 - fe0) * G.idx[d];
        if (G.energy_form == 0) {
            const double* ud = X + (2 + d) * nc + cc;
            const double u0 = normal_along(G, ud, P, d, 0);
            const double u1 = normal_along(G, ud, P, d, 1);
            divu = divu + (u1 - u0) * G.idx[d];
        } else if ((G.gmask >> d) & 1) {
            RE = RE + G.hg[d] * (fm0 + fm1);
        }
    }
    const double pc = __ldg(p + cc);
    if (G.energy_form == 0) RE = RE - pc * divu;

    const double rho = __ldg(X + cc);
    Uv[0] = rho;            Rv[0] = Rr;
    Uv[1] = ops.mul(rho, __ldg(X + nc + cc)); Rv[1] = RE;
#pragma unroll
    for (int c = 0; c < nd; ++c) {
        // every thread evaluates (wall slots read mirrored, in-range cells)
        // and wall slots select zero, so no branch splits the warp
        const int om1 = cell_off(G, P, c, -1);
        const double pl = __ldg(p + cc + om1);
        const double rl = __ldg(X + cc + om1);
        // rs = rl + rho = 2 rho_f: the 1/2 of the face mean is carried by
        // g/2 here and by the halved 1/dt factors of the momentum rows below
        // (exact powers of two: the results are those of rho_f itself)
        const double rs = rl + rho;
        double Rc = ops.mul(pl - pc, G.idx[c]);
        if ((G.gmask >> c) & 1) Rc = fma(rs, G.hg[c], Rc);
#pragma unroll
        for (int d = 0; d < nd; ++d) {
            const double* ps = Psi + (c * nd + d) * nc + cc;
            double a, b;
            if (c == d) {
                b = __ldg(ps);
                a = __ldg(ps + om1);                          // centre i-1 along c
                Rc = Rc - (b - a) * G.hidx[c];         // Psi stored doubled
            } else {
                a = __ldg(ps);
                b = face_up_at(G, ps, P, d);
                Rc = Rc - (b - a) * G.hidx[d];
            }
        }
        const bool wall = is_wall_slot(G, c, P);
        Uv[2 + c] = wall ? 0.0 : ops.mul(rs, __ldg(X + (2 + c) * nc + cc));        // 2 rho_f u
        Rv[2 + c] = wall ? 0.0 : Rc;
    }
    return ops.valid();
}

template <int ND> struct AsmTerms { double U[2 + ND], R[2 + ND]; };

// the FP64-pipe redo, out of line (see face_flux_dir_fp64); the terms come
// back by value so that the caller's arrays stay in registers
template <int ND>
__device__ __noinline__ AsmTerms<ND> assemble_terms_fp64(const Grid G, const double* __restrict__ X,
                                                         const double* __restrict__ p, const double* __restrict__ Fm,
                                                         const double* __restrict__ FE,
                                                         const double* __restrict__ Psi, const Idx3 P, long long cc) {
    AsmTerms<ND> t;
    assemble_terms<ND>(FpOps(), G, X, p, Fm, FE, Psi, P, cc, t.U, t.R);
    return t;
}

template <int ND, int MODE, typename TO>
__global__ void k_assemble(Grid G, const double* __restrict__ X, const double* __restrict__ p,
                           const double* __restrict__ Fm, const double* __restrict__ FE,
                           const double* __restrict__ Psi, const double* __restrict__ bn,
                           const double* __restrict__ G0, const double* __restrict__ Linv,
                           const double* __restrict__ scal, int delta_slot, double dt_inv, double dt_inv_h,
                           double* __restrict__ outd, TO* __restrict__ outb) {
    Idx3 P;
    long long cc;
    if (!cell_pos(G.n, P, cc)) return;
    const long long nc = G.ncell;
    constexpr int nd = ND;
    const double th = G.theta;
    double inv_delta = 0.0;
    if (MODE == kModeJv) inv_delta = scal[kSlotInvDelta];

    double Uv[2 + ND], Rv[2 + ND];
    if (!assemble_terms<ND>(IntOps<true, false>(), G, X, p, Fm, FE, Psi, P, cc, Uv, Rv)) {
        const AsmTerms<ND> t = assemble_terms_fp64<ND>(G, X, p, Fm, FE, Psi, P, cc);
#pragma unroll
        for (int k = 0; k < 2 + ND; ++k) {
            Uv[k] = t.U[k];
            Rv[k] = t.R[k];
        }
    }
#pragma unroll
    for (int k = 0; k < 2 + nd; ++k) {
        const long long j = k * nc + cc;
        const bool wall = (k >= 2) && is_wall_slot(G, k - 2, P);
        const double di = k >= 2 ? dt_inv_h : dt_inv;      // momentum rows hold 2 rho_f u
        if (MODE == kModeG) {
            outd[j] = Uv[k] * di - th * Rv[k];
        } else if (MODE == kModeBn) {
            outd[j] = Uv[k] * di + (1.0 - th) * Rv[k];
        } else if (MODE == kModeRes) {
            outd[j] = Uv[k] * di - th * Rv[k] - bn[j];
        } else if (MODE == kModeNewton) {
            double g = Uv[k] * di - th * Rv[k];
            outd[j] = g;
            outb[j] = wall ? (TO)0 : from_f64<TO>(-((g - bn[j]) * Linv[j]));
        } else {
            // kModeJv: L^-1 (G(X+dw) - G(X)) / delta with bn, G0, Linv holding
            // Q = theta L^-1, C = L^-1 G(X) and P = L^-1/dt, halved on the
            // momentum rows (launch_jv_coeffs):
            // (U P - R Q - C) / delta, two FMAs and a product per unknown;
            // kModeJvD leaves out the 1/delta (GMRES applies it to its
            // Hessenberg column): two FMAs per unknown
            const double q = fma(Rv[k], bn[j], G0[j]);
            const double d = fma(Uv[k], Linv[j], -q);
            outb[j] = wall ? (TO)0 : from_f64<TO>(MODE == kModeJv ? d * inv_delta : d);
        }
    }
}

// --------------------------------------------------------------------------
// scaling L, R (Eq. jacobian_system_norm) and ||R^-1 X||^2 partial sums
// --------------------------------------------------------------------------

__device__ __forceinline__ double internal_e(const Grid& G, const double* X, const Idx3& P, int o0, int o1, int o2) {
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

// L, R, their inverses and the squares of x_hat = R^-1 X of one cell; the
// products of the batched inversion on the integer pipes with checked Ops
// (nothing written, false, where one was out of range)
template <int ND, class O>
__device__ __forceinline__ bool scaling_cell(O ops, const Grid& G, const double* __restrict__ X, double alpha1,
                                             double alpha2, double* __restrict__ L, double* __restrict__ R,
                                             double* __restrict__ Linv, double* __restrict__ Rinv, const Idx3& P,
                                             long long cc, double& acc) {
    const long long nc = G.ncell;
    double rho = X[cc], E = X[nc + cc];
    double Lv[2 + ND], Rv[2 + ND];
    Lv[0] = rho; Rv[0] = rho;
    Lv[1] = rho * E; Rv[1] = E;
    double e0 = internal_e(G, X, P, 0, 0, 0);
    double cs0 = sqrt(G.gamma * G.gm1 * e0);
#pragma unroll
    for (int c = 0; c < ND; ++c) {
        if (is_wall_slot(G, c, P)) { Lv[2 + c] = 1.0; Rv[2 + c] = 1.0; continue; }
        int o[3] = {0, 0, 0};
        o[c] = -1;
        double rl = load_cell(G, X, P, o[0], o[1], o[2]);
        double el = internal_e(G, X, P, o[0], o[1], o[2]);
        double csl = sqrt(G.gamma * G.gm1 * el);
        double rho_f = 0.5 * (rl + rho);
        double cs_f = 0.5 * (csl + cs0);
        double au = fabs(X[(2 + c) * nc + cc]);
        Lv[2 + c] = rho_f * fmax(au, alpha1 * cs_f);
        Rv[2 + c] = fmax(au, alpha2 * cs_f);
    }
    // all 2(2+ND) reciprocals with one division
    double den[2 * (2 + ND)], inv[2 * (2 + ND)];
#pragma unroll
    for (int k = 0; k < 2 + ND; ++k) {
        den[k] = Lv[k];
        den[2 + ND + k] = Rv[k];
    }
    recip_all<2 * (2 + ND)>(den, inv, ops);
    if (!ops.valid()) return false;
    double a = 0.0;
#pragma unroll
    for (int k = 0; k < 2 + ND; ++k) {
        long long j = k * nc + cc;
        L[j] = Lv[k];
        R[j] = Rv[k];
        Linv[j] = inv[k];
        Rinv[j] = inv[2 + ND + k];
        double xh = X[j] * inv[2 + ND + k];
        if (k >= 2 && is_wall_slot(G, k - 2, P)) xh = 0.0;
        a += xh * xh;
    }
    acc = a;
    return true;
}

template <int ND>
__device__ __noinline__ double scaling_cell_fp64(const Grid G, const double* __restrict__ X, double alpha1,
                                                 double alpha2, double* __restrict__ L, double* __restrict__ R,
                                                 double* __restrict__ Linv, double* __restrict__ Rinv, const Idx3 P,
                                                 long long cc) {
    double acc = 0.0;
    scaling_cell<ND>(FpOps(), G, X, alpha1, alpha2, L, R, Linv, Rinv, P, cc, acc);
    return acc;
}

// at least 6 blocks of 128 threads per SM (80 registers; 126 without the
// bound ran slower)
template <int ND>
__global__ void __launch_bounds__(128, 6) k_scaling(Grid G, const double* __restrict__ X, double alpha1, double alpha2,
                          double* __restrict__ L, double* __restrict__ R, double* __restrict__ Linv,
                          double* __restrict__ Rinv, double* __restrict__ partials) {
    __shared__ double sh[32];
    Idx3 P;
    long long cc;
    double acc = 0.0;
    if (cell_pos(G.n, P, cc)) {
        if (!scaling_cell<ND>(IntOps<true, false>(), G, X, alpha1, alpha2, L, R, Linv, Rinv, P, cc, acc))
            acc = scaling_cell_fp64<ND>(G, X, alpha1, alpha2, L, R, Linv, Rinv, P, cc);
    }
    double s = block_sum<128>(acc, sh);
    if (thread_linear() == 0) partials[block_linear()] = s;
}

// max over cells of |u_cell| + c_s (Sect. 1, CFL_hydro)
template <int ND>
__global__ void k_signal_speed(Grid G, const double* __restrict__ X, double* __restrict__ partials) {
    __shared__ double sh[32];
    Idx3 P;
    long long cc;
    double v = 0.0;
    if (cell_pos(G.n, P, cc)) {
        const long long nc = G.ncell;
        double s = 0.0;
        for (int c = 0; c < ND; ++c) {
            int o[3] = {0, 0, 0};
            o[c] = 1;
            double u0 = load_normal(G, X + (2 + c) * nc, c, P, 0, 0, 0);
            double u1 = load_normal(G, X + (2 + c) * nc, c, P, o[0], o[1], o[2]);
            double ub = 0.5 * (u0 + u1);
            s = s + ub * ub;
        }
        double e = internal_e(G, X, P, 0, 0, 0);
        v = sqrt(s) + sqrt(G.gamma * G.gm1 * e);
        if (!(v == v)) v = __longlong_as_double(0x7ff8000000000000ULL);
    }
    double m = block_max<128>(v, sh);
    if (thread_linear() == 0) partials[block_linear()] = m;
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------

static inline unsigned nblk(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

#define CELL_LAUNCH(KERNEL, ...)                                                          \
    do {                                                                                  \
        CellLaunch cl_ = cell_launch(G.n);                                                \
        ++g_launch_count;                                                                 \
        if (G.ndim == 3) KERNEL<3><<<cl_.grid, cl_.block, 0, s>>>(__VA_ARGS__);           \
        else KERNEL<2><<<cl_.grid, cl_.block, 0, s>>>(__VA_ARGS__);                       \
    } while (0)

void launch_eos(const Grid& G, const double* X, double* p, double* T, double* chi, cudaStream_t s) {
    CELL_LAUNCH(k_eos, G, X, p, T, chi);
}

template <typename TZ>
void launch_perturb(const Grid& G, const double* X, const TZ* z, const double* R, const double* scal, int slot,
                    double* Xp, cudaStream_t s) {
    long long nvec = (2 + G.ndim) * G.ncell;
    ++g_launch_count;
    k_perturb<TZ><<<nblk(nvec), kBlock, 0, s>>>(G, X, z, R, scal, slot, Xp, nvec);
}
template void launch_perturb<double>(const Grid&, const double*, const double*, const double*, const double*, int,
                                     double*, cudaStream_t);
template void launch_perturb<float>(const Grid&, const double*, const float*, const double*, const double*, int,
                                    double*, cudaStream_t);

void launch_face_fluxes(const Grid& G, const double* X, const double* p, const double* T, const double* chi,
                        double* Fm, double* FE, cudaStream_t s) {
    const CellLaunch cl = cell_launch(G.n);
    ++g_launch_count;
    if (G.ndim == 3) {
        if (G.energy_form == 1) k_face_fluxes<3, 1><<<cl.grid, cl.block, 0, s>>>(G, X, p, T, chi, Fm, FE);
        else k_face_fluxes<3, 0><<<cl.grid, cl.block, 0, s>>>(G, X, p, T, chi, Fm, FE);
    } else {
        if (G.energy_form == 1) k_face_fluxes<2, 1><<<cl.grid, cl.block, 0, s>>>(G, X, p, T, chi, Fm, FE);
        else k_face_fluxes<2, 0><<<cl.grid, cl.block, 0, s>>>(G, X, p, T, chi, Fm, FE);
    }
}

void launch_mom_fluxes(const Grid& G, const double* X, const double* Fm, double* Psi, cudaStream_t s) {
    CELL_LAUNCH(k_mom_fluxes, G, X, Fm, Psi);
}

void launch_fluxes(const Grid& G, const double* X, const double* p, const double* T, const double* chi, double* Fm,
                   double* FE, double* Psi, cudaStream_t s) {
    launch_face_fluxes(G, X, p, T, chi, Fm, FE, s);
    launch_mom_fluxes(G, X, Fm, Psi, s);
}

template <int MODE, typename TO>
void launch_assemble(const Grid& G, const double* X, const double* p, const double* Fm, const double* FE,
                     const double* Psi, const double* bn, const double* G0, const double* Linv, const double* scal,
                     int slot, double dt, double* outd, TO* outb, cudaStream_t s) {
    CellLaunch cl = cell_launch(G.n);
    ++g_launch_count;
    if (G.ndim == 3)
        k_assemble<3, MODE, TO><<<cl.grid, cl.block, 0, s>>>(G, X, p, Fm, FE, Psi, bn, G0, Linv, scal, slot, 1.0 / dt,
                                                           0.5 / dt, outd, outb);
    else
        k_assemble<2, MODE, TO><<<cl.grid, cl.block, 0, s>>>(G, X, p, Fm, FE, Psi, bn, G0, Linv, scal, slot, 1.0 / dt,
                                                           0.5 / dt, outd, outb);
}
#define INST(M, T)                                                                                             \
    template void launch_assemble<M, T>(const Grid&, const double*, const double*, const double*, const double*, \
                                        const double*, const double*, const double*, const double*,           \
                                        const double*, int, double, double*, T*, cudaStream_t);
INST(kModeG, double)
INST(kModeBn, double)
INST(kModeRes, double)
INST(kModeNewton, double)
INST(kModeNewton, float)
INST(kModeJv, double)
INST(kModeJv, float)
INST(kModeJvD, double)
INST(kModeJvD, float)
#undef INST

void launch_scaling(const Grid& G, const double* X, double a1, double a2, double* L, double* R, double* Linv,
                    double* Rinv, double* partials, cudaStream_t s) {
    CELL_LAUNCH(k_scaling, G, X, a1, a2, L, R, Linv, Rinv, partials);
}

void launch_signal_speed(const Grid& G, const double* X, double* partials, cudaStream_t s) {
    CELL_LAUNCH(k_signal_speed, G, X, partials);
}

unsigned cell_blocks(const Grid& G) {
    CellLaunch cl = cell_launch(G.n);
    return cl.grid.x * cl.grid.y * cl.grid.z;
}

}  // namespace jfnk
