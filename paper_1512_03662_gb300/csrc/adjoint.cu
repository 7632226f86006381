// Adjoint kernels: vector-Jacobian products of the residual and the transpose
// of the physics-based preconditioner.
//
// y = (a dU/dX + b dR_U/dX)^T w at a state X, with (a, b) = (1/dt, -theta)
// for G = U/dt - theta R_U and (1/dt, 1 - theta) for b^n.  Each forward
// kernel of residual.cu has a reverse kernel here that recomputes its local
// forward values and scatters the adjoints of its inputs with atomic adds, in
// the reverse order of the forward pass:
//   k_vjp_assemble   adjoints of the half mass fluxes, energy fluxes,
//                    momentum fluxes and p, plus the direct terms (U, gravity,
//                    p div u)
//   k_vjp_mom        momentum fluxes -> velocities and half mass fluxes
//   k_vjp_face       face fluxes -> rho, e or eps_t, velocities, T, chi (and p)
//   k_vjp_eos        p, T, chi -> rho, e (and the kinetic energy for eps_t)
// The derivative of the van Leer face value q_near + ab/(a+b) is
// d/dq_near = 1 + h_a - h_b, d/dq_far = -h_a, d/dq_other = h_b with
// h_a = b^2/(a+b)^2, h_b = a^2/(a+b)^2 where ab > 0 (zero otherwise); the
// upwind switch contributes nothing (piecewise derivative).  Atomic
// accumulation makes the sums order-dependent at round-off level.
//
// The transposed preconditioner applies the transposes of the pointwise
// transforms and back substitutions exactly, and solves the transposed
// multigrid system with the same V-cycle on the transposed cell matrices.
#include "common.cuh"
#include "kernels.h"

namespace jfnk {


// storage slot and sign of the velocity normal to direction c at position
// (pos + off); false for a wall face (a constant zero, no adjoint).
__device__ __forceinline__ bool normal_slot(const Grid& G, int c, const Idx3& P, int o0, int o1, int o2,
                                            long long& j, double& sgn) {
    int k[3] = {P.i[0] + o0, P.i[1] + o1, P.i[2] + o2};
    sgn = 1.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d == c && G.bc[d] == 1) {
            int n = G.n[d];
            int kk = k[d];
            if (kk == 0 || kk == n) return false;
            if (kk < 0) { kk = -kk; sgn = -sgn; }
            else if (kk > n) { kk = 2 * n - kk; sgn = -sgn; }
            k[d] = kk;
        } else {
            k[d] = cell_map(k[d], G.n[d], G.bc[d]);
        }
    }
    j = flat(G, k[0], k[1], k[2]);
    return true;
}

__device__ __forceinline__ long long cell_slot(const Grid& G, const Idx3& P, int o0, int o1, int o2) {
    return flat(G, cell_map(P.i[0] + o0, G.n[0], G.bc[0]), cell_map(P.i[1] + o1, G.n[1], G.bc[1]),
                cell_map(P.i[2] + o2, G.n[2], G.bc[2]));
}

// slot of the face above cell P along d (false at an upper wall)
__device__ __forceinline__ bool up_slot(const Grid& G, int d, const Idx3& P, long long& j) {
    if (G.bc[d] == 1 && P.i[d] + 1 == G.n[d]) return false;
    int o[3] = {0, 0, 0};
    o[d] = 1;
    j = cell_slot(G, P, o[0], o[1], o[2]);
    return true;
}

// van Leer face value and its partial derivatives
struct UpwindD {
    double v, dn, df, dot;
};

// value and derivatives from the differences and inv = 1/(a+b) (any value
// where the limiter is off): with s = a + b, h_a = (b/s)^2, h_b = (a/s)^2
__device__ __forceinline__ UpwindD upwind_d_finish(double q_near, double a, double b, bool on, double inv) {
    const double ai = a * inv, bi = b * inv;
    const double ha = on ? bi * bi : 0.0, hb = on ? ai * ai : 0.0;
    UpwindD r;
    r.v = q_near + (on ? (a * b) * inv : 0.0);
    r.dn = 1.0 + ha - hb;
    r.df = -ha;
    r.dot = hb;
    return r;
}

// branch-free, one reciprocal
__device__ __forceinline__ UpwindD upwind_d(double q_near, double q_far, double q_other) {
    const double a = q_near - q_far;
    const double b = q_other - q_near;
    const bool on = positive(a * b);
    return upwind_d_finish(q_near, a, b, on, 1.0 / (on ? a + b : 1.0));
}

// two face values with one division (batched inversion)
__device__ __forceinline__ void upwind_d2(double qn1, double qf1, double qo1, double qn2, double qf2, double qo2,
                                          UpwindD& r1, UpwindD& r2) {
    const double a1 = qn1 - qf1, b1 = qo1 - qn1, a2 = qn2 - qf2, b2 = qo2 - qn2;
    const bool on1 = positive(a1 * b1), on2 = positive(a2 * b2);
    const double den[2] = {on1 ? a1 + b1 : 1.0, on2 ? a2 + b2 : 1.0};
    double inv[2];
    recip_all<2>(den, inv);
    r1 = upwind_d_finish(qn1, a1, b1, on1, inv[0]);
    r2 = upwind_d_finish(qn2, a2, b2, on2, inv[1]);
}

__device__ __forceinline__ double cond_dchi(const Grid& G, double T) {
    return G.chi3 ? 3.0 * G.K0 * (T * T) : G.K0 * G.chi_exp * pow(T, G.chi_exp - 1.0);
}

struct AdjBufs {
    double* Fmhb;   // nd fields
    double* FEb;    // nd fields
    double* Psib;   // nd*nd fields
    double* pb;
    double* Tb;
    double* chib;
    double* Xb;     // packed
};

// --------------------------------------------------------------------------
// reverse of k_assemble
// --------------------------------------------------------------------------
template <int ND>
__global__ void k_vjp_assemble(Grid G, const double* __restrict__ X, const double* __restrict__ p,
                               const double* __restrict__ w, double a_u, double b_r, AdjBufs A) {
    Idx3 P;
    long long cc;
    if (!cell_pos(G.n, P, cc)) return;
    const long long nc = G.ncell;
    const double Rr = b_r * w[cc], RE = b_r * w[nc + cc];
    const double Ur = a_u * w[cc], UE = a_u * w[nc + cc];
    const double rho = X[cc], E = X[nc + cc];
    double rhob = Ur + UE * E;
    atomicAdd(A.Xb + nc + cc, UE * rho);
    double divu = 0.0;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        long long ju;
        const bool hasup = up_slot(G, d, P, ju);
        atomicAdd(A.Fmhb + d * nc + cc, Rr * G.tidx[d]);
        atomicAdd(A.FEb + d * nc + cc, RE * G.idx[d]);
        if (hasup) {
            atomicAdd(A.Fmhb + d * nc + ju, -Rr * G.tidx[d]);
            atomicAdd(A.FEb + d * nc + ju, -RE * G.idx[d]);
        }
        if (G.energy_form == 0) {
            const double* ud = X + (2 + d) * nc;
            int o[3] = {0, 0, 0};
            o[d] = 1;
            double u0 = load_normal(G, ud, d, P, 0, 0, 0);
            double u1 = load_normal(G, ud, d, P, o[0], o[1], o[2]);
            divu = divu + (u1 - u0) * G.idx[d];
            const double pc = p[cc];
            if (!is_wall_slot(G, d, P)) atomicAdd(A.Xb + (2 + d) * nc + cc, RE * pc * G.idx[d]);
            long long js;
            double sg;
            if (normal_slot(G, d, P, o[0], o[1], o[2], js, sg)) atomicAdd(A.Xb + (2 + d) * nc + js, -sg * RE * pc * G.idx[d]);
        } else if (((G.gmask >> d) & 1)) {
            atomicAdd(A.Fmhb + d * nc + cc, RE * G.g[d]);
            if (hasup) atomicAdd(A.Fmhb + d * nc + ju, RE * G.g[d]);
        }
    }
    if (G.energy_form == 0) atomicAdd(A.pb + cc, -RE * divu);
#pragma unroll
    for (int c = 0; c < ND; ++c) {
        if (is_wall_slot(G, c, P)) continue;
        const double Ru = b_r * w[(2 + c) * nc + cc];
        const double Uu = a_u * w[(2 + c) * nc + cc];
        int o[3] = {0, 0, 0};
        o[c] = -1;
        const long long jl = cell_slot(G, P, o[0], o[1], o[2]);
        atomicAdd(A.pb + cc, -Ru * G.idx[c]);
        atomicAdd(A.pb + jl, Ru * G.idx[c]);
        const double uc = X[(2 + c) * nc + cc];
        const double rho_f = 0.5 * (X[jl] + rho);
        double rfb = Uu * uc;                              // adjoint of rho_f
        if (((G.gmask >> c) & 1)) rfb += Ru * G.g[c];
        rhob += 0.5 * rfb;
        atomicAdd(A.Xb + jl, 0.5 * rfb);
        atomicAdd(A.Xb + (2 + c) * nc + cc, Uu * rho_f);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            double* ps = A.Psib + (c * ND + d) * nc;
            if (c == d) {
                atomicAdd(ps + cc, -Ru * G.idx[c]);
                atomicAdd(ps + jl, Ru * G.idx[c]);
            } else {
                atomicAdd(ps + cc, Ru * G.idx[d]);
                long long ju;
                if (up_slot(G, d, P, ju)) atomicAdd(ps + ju, -Ru * G.idx[d]);
            }
        }
    }
    atomicAdd(A.Xb + cc, rhob);
}

// --------------------------------------------------------------------------
// reverse of k_mom_fluxes (Fm: the forward mass fluxes; m is the carrying
// mean of two of them, which the adjoint buffers below differentiate as the
// sum of two half fluxes)
// --------------------------------------------------------------------------
template <int ND>
__global__ void k_vjp_mom(Grid G, const double* __restrict__ X, const double* __restrict__ Fm, AdjBufs A) {
    Idx3 P;
    long long cc;
    if (!cell_pos(G.n, P, cc)) return;
    const long long nc = G.ncell;
#pragma unroll
    for (int c = 0; c < ND; ++c) {
        const double* uc = X + (2 + c) * nc;
        double* ub = A.Xb + (2 + c) * nc;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const double psib = A.Psib[(c * ND + d) * nc + cc];
            if (psib == 0.0) continue;
            int on[3] = {0, 0, 0}, of[3] = {0, 0, 0}, oo[3] = {0, 0, 0};
            double m;
            long long jm1 = -1, jm2 = -1;
            if (c == d) {
                long long ju;
                const bool hasup = up_slot(G, c, P, ju);
                m = 0.5 * (Fm[c * nc + cc] + (hasup ? Fm[c * nc + ju] : 0.0));
                jm1 = c * nc + cc;
                jm2 = hasup ? c * nc + ju : -1;
                const bool left = nonneg(m);
                on[c] = left ? 0 : 1;
                of[c] = left ? -1 : 2;
                oo[c] = left ? 1 : 0;
            } else {
                int o[3] = {0, 0, 0};
                o[c] = -1;
                const long long jl = cell_slot(G, P, o[0], o[1], o[2]);
                m = 0.5 * (Fm[d * nc + jl] + Fm[d * nc + cc]);
                jm1 = d * nc + jl;
                jm2 = d * nc + cc;
                const bool left = nonneg(m);
                on[d] = left ? -1 : 0;
                of[d] = left ? -2 : 1;
                oo[d] = left ? 0 : -1;
            }
            const double qn = load_normal(G, uc, c, P, on[0], on[1], on[2]);
            const double qf = load_normal(G, uc, c, P, of[0], of[1], of[2]);
            const double qo = load_normal(G, uc, c, P, oo[0], oo[1], oo[2]);
            const UpwindD U = upwind_d(qn, qf, qo);
            const double mb = psib * U.v;
            atomicAdd(A.Fmhb + jm1, mb);
            if (jm2 >= 0) atomicAdd(A.Fmhb + jm2, mb);
            const double upb = psib * m;
            long long j;
            double sg;
            if (normal_slot(G, c, P, on[0], on[1], on[2], j, sg)) atomicAdd(ub + j, sg * upb * U.dn);
            if (U.df != 0.0 && normal_slot(G, c, P, of[0], of[1], of[2], j, sg)) atomicAdd(ub + j, sg * upb * U.df);
            if (U.dot != 0.0 && normal_slot(G, c, P, oo[0], oo[1], oo[2], j, sg)) atomicAdd(ub + j, sg * upb * U.dot);
        }
    }
}

// --------------------------------------------------------------------------
// reverse of k_face_fluxes
// --------------------------------------------------------------------------
template <int ND>
__global__ void k_vjp_face(Grid G, const double* __restrict__ X, const double* __restrict__ p,
                           const double* __restrict__ T, const double* __restrict__ chi, AdjBufs A) {
    Idx3 P;
    long long c;
    if (!cell_pos(G.n, P, c)) return;
    const long long nc = G.ncell;
    const double* rho = X;
    const double* E = X + nc;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const double fmhb = A.Fmhb[d * nc + c];
        const double feb = A.FEb[d * nc + c];
        if (fmhb == 0.0 && feb == 0.0) continue;
        const bool wall = is_wall_slot(G, d, P);
        const double u = load_normal(G, X + (2 + d) * nc, d, P, 0, 0, 0);
        const bool left = nonneg(u);
        int on[3] = {0, 0, 0}, of[3] = {0, 0, 0}, oo[3] = {0, 0, 0};
        on[d] = left ? -1 : 0;
        of[d] = left ? -2 : 1;
        oo[d] = left ? 0 : -1;
        const long long jn = cell_slot(G, P, on[0], on[1], on[2]);
        const long long jf = cell_slot(G, P, of[0], of[1], of[2]);
        const long long jo = cell_slot(G, P, oo[0], oo[1], oo[2]);
        UpwindD Ur, Ue;
        upwind_d2(rho[jn], rho[jf], rho[jo], E[jn], E[jf], E[jo], Ur, Ue);
        const double fm = u * Ur.v;
        const double fmb = 0.5 * fmhb + feb * Ue.v;
        const double Eupb = feb * fm;
        int ol[3] = {0, 0, 0};
        ol[d] = -1;
        const long long jl = cell_slot(G, P, ol[0], ol[1], ol[2]);
        if (!wall) {
            double ubar = fmb * Ur.v;
            if (G.energy_form == 1) ubar += feb * 0.5 * (p[jl] + p[c]);
            atomicAdd(A.Xb + (2 + d) * nc + c, ubar);
            const double rupb = fmb * u;
            atomicAdd(A.Xb + jn, rupb * Ur.dn);
            if (Ur.df != 0.0) atomicAdd(A.Xb + jf, rupb * Ur.df);
            if (Ur.dot != 0.0) atomicAdd(A.Xb + jo, rupb * Ur.dot);
            atomicAdd(A.Xb + nc + jn, Eupb * Ue.dn);
            if (Ue.df != 0.0) atomicAdd(A.Xb + nc + jf, Eupb * Ue.df);
            if (Ue.dot != 0.0) atomicAdd(A.Xb + nc + jo, Eupb * Ue.dot);
            if (G.energy_form == 1) {
                atomicAdd(A.pb + jl, 0.5 * feb * u);
                atomicAdd(A.pb + c, 0.5 * feb * u);
            }
        }
        if (G.has_cond) {
            // FE contains -q, q = (chi_L + chi_R)/2 (T_R - T_L) / dx
            const double qb = -feb;
            const double Tl = T[jl], Tc = T[c];
            const double chif = 0.5 * (chi[jl] + chi[c]);      // chi of the forward k_eos
            const double dT = (Tc - Tl) * G.idx[d];
            atomicAdd(A.chib + jl, 0.5 * qb * dT);
            atomicAdd(A.chib + c, 0.5 * qb * dT);
            atomicAdd(A.Tb + c, qb * chif * G.idx[d]);
            atomicAdd(A.Tb + jl, -qb * chif * G.idx[d]);
        }
    }
}

// --------------------------------------------------------------------------
// reverse of k_eos; finishes Xb (wall slots cleared)
// --------------------------------------------------------------------------
template <int ND>
__global__ void k_vjp_eos(Grid G, const double* __restrict__ X, const double* __restrict__ T, AdjBufs A) {
    Idx3 P;
    long long cc;
    if (!cell_pos(G.n, P, cc)) return;
    const long long nc = G.ncell;
    const double rho = X[cc];
    const double Tc = T[cc];
    const double e = Tc / G.gm1;
    double Tbt = A.Tb[cc];
    if (G.has_cond) Tbt += A.chib[cc] * cond_dchi(G, Tc);
    const double pbv = A.pb[cc];
    const double eb = pbv * G.gm1 * rho + Tbt * G.gm1;
    atomicAdd(A.Xb + cc, pbv * G.gm1 * e);
    atomicAdd(A.Xb + nc + cc, eb);
    if (G.energy_form == 1) {
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const double* ud = X + (2 + d) * nc;
            long long j;
            double sg;
            if (!is_wall_slot(G, d, P)) atomicAdd(A.Xb + (2 + d) * nc + cc, -eb * 0.5 * ud[cc]);
            int o[3] = {0, 0, 0};
            o[d] = 1;
            if (normal_slot(G, d, P, o[0], o[1], o[2], j, sg))
                atomicAdd(A.Xb + (2 + d) * nc + j, -eb * 0.5 * ud[j]);
        }
    }
}

// w . dR_U/dK0: the conduction divergence without K0, dotted with w_E
template <int ND>
__global__ void k_dRdK0_dot(Grid G, const double* __restrict__ T, const double* __restrict__ w,
                            double* __restrict__ partials) {
    __shared__ double sh[32];
    Idx3 P;
    long long cc;
    double acc = 0.0;
    if (cell_pos(G.n, P, cc)) {
        const long long nc = G.ncell;
        double div = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            int o[3] = {0, 0, 0};
            o[d] = -1;
            const long long jl = cell_slot(G, P, o[0], o[1], o[2]);
            const double Tl = T[jl], Tc = T[cc];
            const double kl = G.chi3 ? Tl * Tl * Tl : pow(Tl, G.chi_exp);
            const double kc = G.chi3 ? Tc * Tc * Tc : pow(Tc, G.chi_exp);
            const double q0 = 0.5 * (kl + kc) * (Tc - Tl) * G.idx[d];
            double q1 = 0.0;
            long long ju;
            if (up_slot(G, d, P, ju)) {
                const double Tu = T[ju];
                const double ku = G.chi3 ? Tu * Tu * Tu : pow(Tu, G.chi_exp);
                q1 = 0.5 * (kc + ku) * (Tu - Tc) * G.idx[d];
            }
            div = div + (q1 - q0) * G.idx[d];
        }
        acc = w[nc + cc] * div;
    }
    double s = block_sum<128>(acc, sh);
    if (thread_linear() == 0) partials[block_linear()] = s;
}

#define CELL_LAUNCH_A(KERNEL, ...)                                                        \
    do {                                                                                  \
        CellLaunch cl_ = cell_launch(G.n);                                                \
        ++g_launch_count;                                                                 \
        if (G.ndim == 3) KERNEL<3><<<cl_.grid, cl_.block, 0, s>>>(__VA_ARGS__);           \
        else KERNEL<2><<<cl_.grid, cl_.block, 0, s>>>(__VA_ARGS__);                       \
    } while (0)

void launch_vjp(const Grid& G, const double* X, const double* p, const double* T, const double* chi, const double* Fm,
                const double* w, double a_u, double b_r, double* adj, double* Xb, cudaStream_t s) {
    const long long nc = G.ncell, nd = G.ndim;
    AdjBufs A;
    A.Fmhb = adj;
    A.FEb = A.Fmhb + nd * nc;
    A.Psib = A.FEb + nd * nc;
    A.pb = A.Psib + nd * nd * nc;
    A.Tb = A.pb + nc;
    A.chib = A.Tb + nc;
    A.Xb = Xb;
    const long long nadj = (2 * nd + nd * nd + 3) * nc;
    launch_zero<double>(adj, nadj, s);
    launch_zero<double>(Xb, (2 + nd) * nc, s);
    CELL_LAUNCH_A(k_vjp_assemble, G, X, p, w, a_u, b_r, A);
    CELL_LAUNCH_A(k_vjp_mom, G, X, Fm, A);
    CELL_LAUNCH_A(k_vjp_face, G, X, p, T, chi, A);
    CELL_LAUNCH_A(k_vjp_eos, G, X, T, A);
}

long long vjp_scratch_doubles(const Grid& G) {
    const long long nc = G.ncell, nd = G.ndim;
    return (2 * nd + nd * nd + 3) * nc;
}

void launch_dRdK0_dot(const Grid& G, const double* T, const double* w, double* partials, cudaStream_t s) {
    CELL_LAUNCH_A(k_dRdK0_dot, G, T, w, partials);
}

// --------------------------------------------------------------------------
// transposed preconditioner (FP64)
// --------------------------------------------------------------------------

__device__ __forceinline__ long long mg0_index(const Grid& G, const Idx3& P) {
    long long f = ((long long)P.i[2] * G.n[1] + P.i[1]) * G.n[0] + P.i[0];
    if (G.n[0] & 1) return f;
    return (long long)((P.i[0] + P.i[1] + P.i[2]) & 1) * (G.ncell >> 1) + (f >> 1);
}

// Stage 1: y -> adjoints of (dp, de, du) through R^-1, dX/dV and the back
// substitution; writes the multigrid right-hand side (transposed system),
// the adjoints of r_u and r_e, and the direct part of the adjoint of r_p.
template <int ND>
__global__ void k_precondT_out(Grid G, const double* __restrict__ C, double dt, int nf, const double* __restrict__ y,
                               double* __restrict__ rub, double* __restrict__ reb, double* __restrict__ rpb,
                               double* __restrict__ rhs, double* __restrict__ x0) {
    Idx3 P;
    long long cc;
    if (!cell_pos(G.n, P, cc)) return;
    const long long nc = G.ncell;
    // adjoint of dX = R^-1 y (diagonal), then of dX/dV
    const double drhob = y[cc] * C[PcRinvR * nc + cc];
    const double dEb = y[nc + cc] * C[PcRinvE * nc + cc];
    double dpb = drhob * C[PcInvDpdrho * nc + cc];
    double deb = dEb - C[PcDpde * nc + cc] * C[PcInvDpdrho * nc + cc] * drhob;
    // du adjoint at the faces of this cell (own slot), including the
    // eps_t = e + <u.du> term for the total energy form
    double dub[ND];
#pragma unroll
    for (int c = 0; c < ND; ++c) {
        dub[c] = y[(2 + c) * nc + cc] * C[(PcRinvU + c) * nc + cc];
        if (G.energy_form == 1 && !is_wall_slot(G, c, P)) {
            int o[3] = {0, 0, 0};
            o[c] = -1;
            const long long jl = cell_slot(G, P, o[0], o[1], o[2]);
            const double dEbl = y[nc + jl] * C[PcRinvE * nc + jl];
            dub[c] += 0.5 * C[(PcU + c) * nc + cc] * (dEb + dEbl);
        }
    }
    // back substitution: du_c(k) = dt (r_u - thf (dp(k) - dp(k-1)))
#pragma unroll
    for (int c = 0; c < ND; ++c) {
        rub[c * nc + cc] = dt * dub[c];
        dpb -= dt * C[(PcThf + c) * nc + cc] * dub[c];
        long long ju;
        if (up_slot(G, c, P, ju)) {
            double yu = y[(2 + c) * nc + ju] * C[(PcRinvU + c) * nc + ju];
            if (G.energy_form == 1) {
                const double dEbu = y[nc + ju] * C[PcRinvE * nc + ju];
                yu += 0.5 * C[(PcU + c) * nc + ju] * (dEbu + dEb);
            }
            dpb += dt * C[(PcThf + c) * nc + ju] * yu;
        }
    }
    const long long mi = mg0_index(G, P);
    if (nf == 1) {
        // de = dt (r_e + (dp/dt - r_p) cde)
        reb[cc] = dt * deb;
        rpb[cc] = -dt * C[PcCde * nc + cc] * deb;
        rhs[mi] = dpb + deb * C[PcCde * nc + cc];
        x0[mi] = 0.0;
    } else {
        reb[cc] = 0.0;
        rpb[cc] = 0.0;
        rhs[mi] = dpb;
        rhs[nc + mi] = deb;
        x0[mi] = 0.0;
        x0[nc + mi] = 0.0;
    }
}

// Adjoints of r_p and r_e at a cell (slot j, multigrid index mi): the direct
// parts from stage 1 plus B^-T applied to the transposed multigrid solution.
struct RpRe {
    double rp, re;
};

__device__ __forceinline__ RpRe rp_re_bar(const double* C, long long nc, int nf, const double* xmg,
                                          const double* reb, const double* rpb, long long j, long long mi) {
    RpRe r;
    r.rp = rpb[j];
    r.re = reb[j];
    if (nf == 1) {
        r.rp += C[PcQ0 * nc + j] * xmg[mi];
    } else {
        const double y0 = xmg[mi], y1 = xmg[nc + mi];
        r.rp += C[PcQ0 * nc + j] * y0 + C[PcQ2 * nc + j] * y1;
        r.re += C[PcQ1 * nc + j] * y0 + C[PcQ3 * nc + j] * y1;
    }
    return r;
}

// total adjoint of r_e at cell Q (r_p = dpdrho r_rho + dpde r_e also uses r_e)
__device__ __forceinline__ double reb_total(const Grid& G, const double* C, int nf, const double* xmg,
                                            const double* reb, const double* rpb, const Idx3& Q) {
    const long long nc = G.ncell;
    const long long j = flat(G, Q.i[0], Q.i[1], Q.i[2]);
    RpRe r = rp_re_bar(C, nc, nf, xmg, reb, rpb, j, mg0_index(G, Q));
    return r.re + C[PcDpde * nc + j] * r.rp;
}

// total adjoint of r_u_c on the lower face of cell Q (adds, for the total
// energy form, the -<u.r_u> term of r_e of the two cells beside the face)
__device__ __forceinline__ double rub_total(const Grid& G, const double* C, int nf, const double* xmg,
                                            const double* reb, const double* rpb, const double* rub, int c,
                                            const Idx3& Q) {
    const long long nc = G.ncell;
    const long long j = flat(G, Q.i[0], Q.i[1], Q.i[2]);
    double v = rub[c * nc + j];
    if (G.energy_form == 1 && !is_wall_slot(G, c, Q)) {
        Idx3 L = Q;
        L.i[c] = cell_map(Q.i[c] - 1, G.n[c], G.bc[c]);
        v -= 0.5 * C[(PcU + c) * nc + j] *
             (reb_total(G, C, nf, xmg, reb, rpb, Q) + reb_total(G, C, nf, xmg, reb, rpb, L));
    }
    return v;
}

// Stage 2: adjoints of (r_p, r_e, r_u) -> z = L (dV/dU)^T (...), through B^-T.
template <int ND>
__global__ void k_precondT_in(Grid G, const double* __restrict__ C, int nf, const double* __restrict__ xmg,
                              const double* __restrict__ rub, const double* __restrict__ reb,
                              const double* __restrict__ rpb, double* __restrict__ z) {
    Idx3 P;
    long long cc;
    if (!cell_pos(G.n, P, cc)) return;
    const long long nc = G.ncell;
    const RpRe r = rp_re_bar(C, nc, nf, xmg, reb, rpb, cc, mg0_index(G, P));
    // r_p = dpdrho r_rho + dpde r_e ; r_e = (r_E - E r_rho) invrho [- <u.r_u>]
    const double reb_t = r.re + C[PcDpde * nc + cc] * r.rp;
    double rrho_b = C[PcDpdrho * nc + cc] * r.rp - C[PcE * nc + cc] * C[PcInvRho * nc + cc] * reb_t;
    const double rE_b = C[PcInvRho * nc + cc] * reb_t;
    // r_u_c(k) = (L_u v_u - u_c rbar_rho) invrhof, rbar_rho the face mean of r_rho
#pragma unroll
    for (int c = 0; c < ND; ++c) {
        const double own = rub_total(G, C, nf, xmg, reb, rpb, rub, c, P);
        rrho_b -= 0.5 * C[(PcU + c) * nc + cc] * C[(PcInvRhof + c) * nc + cc] * own;
        long long ju;
        if (up_slot(G, c, P, ju)) {
            Idx3 U = P;
            U.i[c] = (P.i[c] + 1 == G.n[c]) ? 0 : P.i[c] + 1;
            const double up = rub_total(G, C, nf, xmg, reb, rpb, rub, c, U);
            rrho_b -= 0.5 * C[(PcU + c) * nc + ju] * C[(PcInvRhof + c) * nc + ju] * up;
        }
        z[(2 + c) * nc + cc] = C[(PcLu + c) * nc + cc] * C[(PcInvRhof + c) * nc + cc] * own;
    }
    z[cc] = C[PcLr * nc + cc] * rrho_b;
    z[nc + cc] = C[PcLE * nc + cc] * rE_b;
}

void launch_precondT_out(const Grid& G, const double* C, double dt, int nf, const double* y, double* rub, double* reb,
                         double* rpb, MGLevel& L0, cudaStream_t s) {
    CELL_LAUNCH_A(k_precondT_out, G, C, dt, nf, y, rub, reb, rpb, (double*)L0.rhs, (double*)L0.x);
}

void launch_precondT_in(const Grid& G, const double* C, int nf, const MGLevel& L0, const double* rub,
                        const double* reb, const double* rpb, double* z, cudaStream_t s) {
    CELL_LAUNCH_A(k_precondT_in, G, C, nf, (const double*)L0.x, rub, reb, rpb, z);
}

// out = x * y elementwise
__global__ void k_mul(const double* __restrict__ x, const double* __restrict__ y, double* __restrict__ out,
                      long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        out[e] = x[e] * y[e];
}

void launch_mul(const double* x, const double* y, double* out, long long n, cudaStream_t s) {
    ++g_launch_count;
    k_mul<<<kRedBlocks, kBlock, 0, s>>>(x, y, out, n);
}

// out = a - b elementwise
__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                      long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        out[e] = a[e] - b[e];
}

void launch_sub(const double* a, const double* b, double* out, long long n, cudaStream_t s) {
    ++g_launch_count;
    k_sub<<<kRedBlocks, kBlock, 0, s>>>(a, b, out, n);
}

// zero the wall-face slots of a packed vector
template <int ND>
__global__ void k_mask_walls(Grid G, double* __restrict__ v) {
    Idx3 P;
    long long cc;
    if (!cell_pos(G.n, P, cc)) return;
#pragma unroll
    for (int c = 0; c < ND; ++c)
        if (is_wall_slot(G, c, P)) v[(2 + c) * G.ncell + cc] = 0.0;
}

void launch_mask_walls(const Grid& G, double* v, cudaStream_t s) { CELL_LAUNCH_A(k_mask_walls, G, v); }

}  // namespace jfnk
