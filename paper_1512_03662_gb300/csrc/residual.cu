// Finite-volume right-hand side R_U(X) of the paper's Sect. 2 on the
// staggered grid, and the residual-type operators built from it:
//   G(X)  = U(X)/dt - theta R_U(X)                 (Jv, Newton set-up)
//   b^n   = U(X^n)/dt + (1-theta) R_U(X^n)          (Eq. crank_nicholson)
//   F_U   = G(X) - b^n
//   Jv    = L^-1 [G(X + delta R v) - G(X)] / delta   (Eqs. jacobian_free, pert_old)
//
// The evaluation is split so that every van Leer slope and every flux is
// computed once per slot (the FP64 rate of sm_103a, about 0.6 TFMA/s, binds
// these kernels, not HBM):
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
// all the faces that use it
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
            const double* u = X + (2 + d) * nc;
            int o[3] = {0, 0, 0};
            o[d] = 1;
            double ul = load_normal(G, u, d, P, 0, 0, 0);
            double uu = load_normal(G, u, d, P, o[0], o[1], o[2]);
            ke = ke + 0.25 * (ul * ul + uu * uu);
        }
        e = e - ke;
    }
    p[c] = G.gm1 * rho * e;
    const double Tc = G.gm1 * e;
    T[c] = Tc;
    if (G.has_cond) chi[c] = conductivity(G, Tc);
}

template <int ND>
__global__ void k_face_fluxes(Grid G, const double* __restrict__ X, const double* __restrict__ p,
                              const double* __restrict__ T, const double* __restrict__ chi, double* __restrict__ Fm,
                              double* __restrict__ FE) {
    Idx3 P;
    long long c;
    if (!cell_pos(G.n, P, c)) return;
    const long long nc = G.ncell;
    const double* rho = X;
    const double* E = X + nc;
    const double r0 = __ldg(rho + c), e0 = __ldg(E + c);
    // pass 1: loads and the split upwind values of rho and E on every face
    double u[ND];
    Upw up[2 * ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        int o[3] = {0, 0, 0};
        u[d] = load_normal(G, X + (2 + d) * nc, d, P, 0, 0, 0);
        o[d] = -2; const double r2 = load_cell(G, rho, P, o[0], o[1], o[2]), e2 = load_cell(G, E, P, o[0], o[1], o[2]);
        o[d] = -1; const double r1 = load_cell(G, rho, P, o[0], o[1], o[2]), e1 = load_cell(G, E, P, o[0], o[1], o[2]);
        o[d] = 1;  const double r3 = load_cell(G, rho, P, o[0], o[1], o[2]), e3 = load_cell(G, E, P, o[0], o[1], o[2]);
        // upwind side: cell i-1 for u >= 0 (ties to the lower side), else cell i
        const bool left = nonneg(u[d]);
        up[2 * d] = upwind_parts(left ? r1 : r0, left ? r2 : r3, left ? r0 : r1);
        up[2 * d + 1] = upwind_parts(left ? e1 : e0, left ? e2 : e3, left ? e0 : e1);
    }
    // pass 2: one division for all limited slopes of the cell
    double den[2 * ND], inv[2 * ND];
#pragma unroll
    for (int k = 0; k < 2 * ND; ++k) den[k] = up[k].den;
    recip_all<2 * ND>(den, inv);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        int o[3] = {0, 0, 0};
        const double rho_up = up[2 * d].q + up[2 * d].num * inv[2 * d];
        const double E_up = up[2 * d + 1].q + up[2 * d + 1].num * inv[2 * d + 1];
        double fm = u[d] * rho_up;
        double fe = fm * E_up;
        o[d] = -1;
        if (G.energy_form == 1) {
            double pl = load_cell(G, p, P, o[0], o[1], o[2]);
            fe = fe + 0.5 * (pl + __ldg(p + c)) * u[d];
        }
        if (G.has_cond) {
            // q = chi_f (T_c - T_l) / dx with chi_f the mean of the two cells
            const double Tl = load_cell(G, T, P, o[0], o[1], o[2]);
            const double chil = load_cell(G, chi, P, o[0], o[1], o[2]);
            const double sq = (chil + __ldg(chi + c)) * G.hidx[d];
            fe = fma(-sq, __ldg(T + c) - Tl, fe);
        }
        Fm[d * nc + c] = fm;                  // mass flux (every consumer takes half the sum of two)
        FE[d * nc + c] = fe;
    }
}

// Fm_d at slot (pos + off) where the offset is along a direction in which Fm_d
// behaves as a cell quantity (any direction other than d).
__device__ __forceinline__ double load_Fm_cell(const Grid& G, const double* Fm_d, const Idx3& P, int o0, int o1, int o2) {
    return load_cell(G, Fm_d, P, o0, o1, o2);
}

// Fm_d at the upper face (slot + 1 along d): zero at an upper wall.
__device__ __forceinline__ double load_face_up(const Grid& G, const double* f, int d, const Idx3& P) {
    if (G.bc[d] == 1 && P.i[d] + 1 == G.n[d]) return 0.0;
    int o[3] = {0, 0, 0};
    o[d] = 1;
    return load_cell(G, f, P, o[0], o[1], o[2]);
}

// 128-thread blocks, at least 10 resident per SM: 48 registers (no spills)
// instead of 54, 40 warps per SM instead of 36
template <int ND>
__global__ void __launch_bounds__(128, 10) k_mom_fluxes(Grid G, const double* __restrict__ X,
                                                        const double* __restrict__ Fm, double* __restrict__ Psi) {
    Idx3 P;
    long long cc;
    if (!cell_pos(G.n, P, cc)) return;
    const long long nc = G.ncell;
    constexpr int nd = ND;
    // pass 1 per component c: loads, carrying mass flux and split upwind value
    double mf[nd * nd];
    Upw up[nd * nd];
#pragma unroll
    for (int c = 0; c < nd; ++c) {
        const double* uc = X + (2 + c) * nc;
#pragma unroll
        for (int d = 0; d < nd; ++d) {
            double m, q_near, q_far, q_other;
            int o[3] = {0, 0, 0};
            if (c == d) {
                // flux at the cell centre between faces i and i+1 along c, carried
                // by the mean of the two mass fluxes (here their sum: Psi doubled)
                m = __ldg(Fm + c * nc + cc) + load_face_up(G, Fm + c * nc, c, P);
                o[c] = -1; const double um = load_normal(G, uc, c, P, o[0], o[1], o[2]);
                const double u0 = load_normal(G, uc, c, P, 0, 0, 0);
                o[c] = 1;  const double u1 = load_normal(G, uc, c, P, o[0], o[1], o[2]);
                o[c] = 2;  const double u2 = load_normal(G, uc, c, P, o[0], o[1], o[2]);
                const bool left = nonneg(m);
                q_near = left ? u0 : u1;
                q_far = left ? um : u2;
                q_other = left ? u1 : u0;
            } else {
                // flux on the edge between c-face i_c and d-face i_d
                o[c] = -1;
                m = load_Fm_cell(G, Fm + d * nc, P, o[0], o[1], o[2]) + __ldg(Fm + d * nc + cc);
                o[c] = 0;
                o[d] = -2; const double u2 = load_normal(G, uc, c, P, o[0], o[1], o[2]);
                o[d] = -1; const double u1 = load_normal(G, uc, c, P, o[0], o[1], o[2]);
                const double u0 = load_normal(G, uc, c, P, 0, 0, 0);
                o[d] = 1;  const double u3 = load_normal(G, uc, c, P, o[0], o[1], o[2]);
                const bool left = nonneg(m);
                q_near = left ? u1 : u0;
                q_far = left ? u2 : u3;
                q_other = left ? u0 : u1;
            }
            mf[c * nd + d] = m;
            up[c * nd + d] = upwind_parts(q_near, q_far, q_other);
        }
        // pass 2: one division for the nd limited slopes of component c (a
        // batch of nd keeps the kernel near 56 registers; one batch of nd^2
        // needed 102 and ran 20 % slower at the lower occupancy)
        double den[nd], inv[nd];
#pragma unroll
        for (int d = 0; d < nd; ++d) den[d] = up[c * nd + d].den;
        recip_all<nd>(den, inv);
#pragma unroll
        for (int d = 0; d < nd; ++d)
            Psi[(c * nd + d) * nc + cc] = mf[c * nd + d] * (up[c * nd + d].q + up[c * nd + d].num * inv[d]);
    }
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

    double Rr = 0.0, RE = 0.0, divu = 0.0;
#pragma unroll
    for (int d = 0; d < nd; ++d) {
        const double* fmd = Fm + d * nc;
        const double* fed = FE + d * nc;
        double fm0 = __ldg(fmd + cc), fm1 = load_face_up(G, fmd, d, P);
        double fe0 = __ldg(fed + cc), fe1 = load_face_up(G, fed, d, P);
        Rr = Rr - (fm1 - fm0) * G.idx[d];
        RE = RE - (fe1 - fe0) * G.idx[d];
        if (G.energy_form == 0) {
            const double* ud = X + (2 + d) * nc;
            double u0 = load_normal(G, ud, d, P, 0, 0, 0);
            int o[3] = {0, 0, 0};
            o[d] = 1;
            double u1 = load_normal(G, ud, d, P, o[0], o[1], o[2]);
            divu = divu + (u1 - u0) * G.idx[d];
        } else if ((G.gmask >> d) & 1) {
            RE = RE + G.hg[d] * (fm0 + fm1);
        }
    }
    const double pc = __ldg(p + cc);
    if (G.energy_form == 0) RE = RE - pc * divu;

    const double rho = __ldg(X + cc);
    double Uv[2 + ND], Rv[2 + ND];
    Uv[0] = rho;            Rv[0] = Rr;
    Uv[1] = rho * __ldg(X + nc + cc); Rv[1] = RE;
#pragma unroll
    for (int c = 0; c < nd; ++c) {
        if (is_wall_slot(G, c, P)) { Uv[2 + c] = 0.0; Rv[2 + c] = 0.0; continue; }
        int o[3] = {0, 0, 0};
        o[c] = -1;
        double pl = load_cell(G, p, P, o[0], o[1], o[2]);
        double rl = load_cell(G, X, P, o[0], o[1], o[2]);
        // rs = rl + rho = 2 rho_f: the 1/2 of the face mean is carried by
        // g/2 here and by the halved 1/dt factors of the momentum rows below
        // (exact powers of two: the results are those of rho_f itself)
        const double rs = rl + rho;
        double Rc = -(pc - pl) * G.idx[c];
        if ((G.gmask >> c) & 1) Rc = fma(rs, G.hg[c], Rc);
#pragma unroll
        for (int d = 0; d < nd; ++d) {
            const double* ps = Psi + (c * nd + d) * nc;
            double a, b;
            if (c == d) {
                b = __ldg(ps + cc);
                a = load_cell(G, ps, P, o[0], o[1], o[2]);      // centre i-1 along c
                Rc = Rc - (b - a) * G.hidx[c];              // Psi stored doubled
            } else {
                a = __ldg(ps + cc);
                b = load_face_up(G, ps, d, P);
                Rc = Rc - (b - a) * G.hidx[d];
            }
        }
        Uv[2 + c] = rs * __ldg(X + (2 + c) * nc + cc);        // 2 rho_f u
        Rv[2 + c] = Rc;
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

template <int ND>
__global__ void k_scaling(Grid G, const double* __restrict__ X, double alpha1, double alpha2,
                          double* __restrict__ L, double* __restrict__ R, double* __restrict__ Linv,
                          double* __restrict__ Rinv, double* __restrict__ partials) {
    __shared__ double sh[32];
    Idx3 P;
    long long cc;
    double acc = 0.0;
    if (cell_pos(G.n, P, cc)) {
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
        recip_all<2 * (2 + ND)>(den, inv);
#pragma unroll
        for (int k = 0; k < 2 + ND; ++k) {
            long long j = k * nc + cc;
            L[j] = Lv[k];
            R[j] = Rv[k];
            Linv[j] = inv[k];
            Rinv[j] = inv[2 + ND + k];
            double xh = X[j] * inv[2 + ND + k];
            if (k >= 2 && is_wall_slot(G, k - 2, P)) xh = 0.0;
            acc += xh * xh;
        }
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
    CELL_LAUNCH(k_face_fluxes, G, X, p, T, chi, Fm, FE);
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
