// Host-side launch interface between the solver engine and the kernels.
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace jfnk {

// number of kernels launched through the launchers below (profiling aid)
extern long long g_launch_count;

// kModeJvD: the Jacobian-free product times delta, L^-1 (G(X + delta R w) - G(X));
// GMRES takes the 1/delta into its Hessenberg column instead
enum { kModeG = 0, kModeBn = 1, kModeRes = 2, kModeNewton = 3, kModeJv = 4, kModeJvD = 5 };

// device scalar slots (double array `scal` in the workspace)
enum {
    kSlotXhatNorm = 0,   // ||R^-1 X||_2
    kSlotDelta = 1,      // perturbation delta of the current Jv
    kSlotBeta = 2,       // ||b||_2 of the current GMRES cycle
    kSlotRes = 3,        // GMRES residual estimate |g_{j+1}|
    kSlotDxInf = 4,      // ||dxhat||_inf
    kSlotZnorm = 5,      // ||z||_2 of the last preconditioned vector
    kSlotMaxSpeed = 6,   // max |u| + c_s
    kSlotTmp = 7,
    kSlotBeta0 = 8,
    kSlotInvDelta = 9,   // 1/delta of the current Jv (one division, not one per thread)
    kSlotInnerB = 10,    // ||b||_2 of the finest-level SI system of the current preconditioner apply
    kSlotInnerR = 11,    // ||b - A x||_2 after its V-cycles
    kSlotWnorm0 = 12,    // ||w||_2 of the new Arnoldi vector before Gram-Schmidt (selective second pass)
    kNumSlots = 16
};

// residual.cu
// p, T and, when the grid has conduction, chi = K0 T^exp per cell
void launch_eos(const Grid& G, const double* X, double* p, double* T, double* chi, cudaStream_t s);
template <typename TZ>
void launch_perturb(const Grid& G, const double* X, const TZ* z, const double* R, const double* scal, int slot,
                    double* Xp, cudaStream_t s);
void launch_face_fluxes(const Grid& G, const double* X, const double* p, const double* T, const double* chi,
                        double* Fm, double* FE, cudaStream_t s);
void launch_mom_fluxes(const Grid& G, const double* X, const double* Fm, double* Psi, cudaStream_t s);
void launch_fluxes(const Grid& G, const double* X, const double* p, const double* T, const double* chi, double* Fm,
                   double* FE, double* Psi, cudaStream_t s);
template <int MODE, typename TO>
void launch_assemble(const Grid& G, const double* X, const double* p, const double* Fm, const double* FE,
                     const double* Psi, const double* bn, const double* G0, const double* Linv, const double* scal,
                     int slot, double dt, double* outd, TO* outb, cudaStream_t s);
void launch_scaling(const Grid& G, const double* X, double a1, double a2, double* L, double* R, double* Linv,
                    double* Rinv, double* partials, cudaStream_t s);
void launch_signal_speed(const Grid& G, const double* X, double* partials, cudaStream_t s);
unsigned cell_blocks(const Grid& G);

// krylov.cu
// finalize: scal[slot] = op(partials[0..n)) with op 0 = sqrt(sum), 1 = sum, 2 = max
void launch_finalize(const double* partials, int n, double* scal, int slot, int op, cudaStream_t s);
// delta = lambda (lambda + xhat / ||z||) (pert 0) or the pert_new rule (pert 1,
// uses scal[kSlotTmp] = xhat . z and scal[kSlotZnorm])
void launch_delta(double* scal, double lambda, int pert, cudaStream_t s);
template <typename T>
void launch_norm2_partials(const T* x, long long n, double* partials, cudaStream_t s);
template <typename T>
void launch_dot_partials(const double* a, const double* ainv_scale, const T* b, long long n, double* partials,
                         cudaStream_t s);
// multi-dot and AXPY + norm return the number of blocks (partial sums per
// vector) of their occupancy-sized grid, at most kMaxRedBlocks
template <typename T>
int launch_multidot(const T* V, long long ld, int nv, const T* w, long long n, double* partials, cudaStream_t s);
void launch_multidot_finalize(const double* partials, int nblocks, int nv, const double* vscale, double* hcol,
                              int accumulate, cudaStream_t s);
template <typename T>
int launch_axpy_norm(T* w, const T* V, long long ld, int nv, const double* hcol, const double* vscale, long long n,
                     double* partials, cudaStream_t s);
// hcol[j+1] = norm, vscale[j+1] = 1/norm
// h_{j+1,j} = ||w|| (scal[kSlotTmp]) and the lazy scale 1/||w|| of v_{j+1};
// with col_scale_slot >= 0 the whole column 0..j+1 is then multiplied by
// scal[col_scale_slot] (w was formed as delta J^ z)
void launch_set_subdiag(double* scal, double* hcol, int j, double* vscale, cudaStream_t s, int col_scale_slot = -1);
void launch_givens(double* H, int ldh, int j, double* cs, double* sn, double* g, double* scal, cudaStream_t s);
void launch_backsolve(const double* H, int ldh, int k, const double* g, double* y, cudaStream_t s);
template <typename T>
void launch_update(double* x, const T* Z, long long ld, int k, const double* y, long long n, cudaStream_t s);
template <typename TS, typename TD>
void launch_scale_copy(const TS* src, double alpha, const double* scal, int slot, int invert, TD* dst, long long n,
                       cudaStream_t s);
void launch_newton_update(double* X, const double* R, const double* dxh, long long n, double* partials,
                          cudaStream_t s);
template <typename T>
void launch_zero(T* x, long long n, cudaStream_t s);
template <typename T>
void launch_restart_residual(T* r, const double* G0, const double* bn, const double* Linv, long long n,
                             cudaStream_t s);
void launch_init_cycle(double* scal, double* g, double* vscale, int m, cudaStream_t s);
void launch_add_col(double* col, const double* other, int n, cudaStream_t s);
// coefficients of the Jacobian-free product for one linearisation:
// P = L^-1 / dt, Q = theta L^-1, C = L^-1 G(X)
void launch_jv_coeffs(const double* Linv, const double* G0, double dt, double theta, double* P, double* Q, double* C,
                      long long n, long long u_begin, cudaStream_t s);

// precond.cu
struct MGLevel {
    int n[3];
    long long ncell;
    double h[3], ih2[3];
    void* M;     // nf*nf fields
    void* K;     // nf*ndim fields (coefficient on the lower face)
    void* x;     // nf fields
    void* rhs;   // nf fields
    void* r;     // nf fields: residual scratch for the restriction
};

// per-cell coefficient fields of the preconditioner transforms
// PcQ0..PcQ5: FP64 mode: B^-1 entries (b00, b01, b10, b11) applied to
// (r_p, r_e) as the oracle does; FP32 mode: the same map folded with the
// transform, rhs_p = Q0 r_rho + Q1 r_E - Q2 <u.r_u>, rhs_e = Q3 r_rho + Q4 r_E
// - Q5 <u.r_u>, coefficients formed in double so no FP32 cancellation occurs.
enum {
    PcLr = 0, PcLE, PcInvRho, PcE, PcDpdrho, PcDpde, PcInvDpdrho, PcCde,
    PcQ0, PcQ1, PcQ2, PcQ3, PcQ4, PcQ5, PcPr, PcPE, PcRinvR, PcRinvE,
    PcLu, PcU = PcLu + 3, PcInvRhof = PcU + 3, PcThf = PcInvRhof + 3, PcRinvU = PcThf + 3,
    PcNumFields = PcRinvU + 3
};

template <typename T>
void launch_pc_setup(const Grid& G, const double* X, const double* L, const double* Rinv, double dt, int nf, T* C,
                     MGLevel& L0, cudaStream_t s);
template <typename T>
void launch_coarsen(const Grid& G, int nf, const MGLevel& F, MGLevel& C, cudaStream_t s);
// renew only the scaling fields (L and R^-1) of the coefficient array C
template <typename T>
void launch_pc_rescale(const Grid& G, const double* L, const double* Rinv, T* C, cudaStream_t s);
// zero_x = 1: also zero the level-0 multigrid unknowns (needed when the
// V-cycle does not start with a zero-start half sweep)
template <typename T>
void launch_precond_in(const Grid& G, const T* C, const T* v, const double* vscale, int vslot, int nf, T* rp, T* re,
                       T* ru, MGLevel& L0, cudaStream_t s, int zero_x);
// tr = 1: the transposed multigrid system (cell matrices transposed);
// zero_start = 1: x is zero on entry (no neighbour loads)
template <typename T>
void launch_smooth(const Grid& G, int nf, MGLevel& Lv, int colour, cudaStream_t s, int tr = 0, int zero_start = 0);
// red_only = 1 after at least one pre-smoothing sweep (the last half sweep
// leaves a zero residual on colour-1 cells): residual and restriction read
// colour-0 cells only
template <typename T>
void launch_restrict(const Grid& G, int nf, MGLevel& F, MGLevel& C, cudaStream_t s, int tr = 0, int red_only = 0);
template <typename T>
void launch_mg_residual(const Grid& G, int nf, MGLevel& F, cudaStream_t s);
template <typename T>
void launch_prolong(const Grid& G, int nf, MGLevel& F, MGLevel& C, cudaStream_t s);
template <typename T>
void launch_coarsest(int nf, MGLevel& C, cudaStream_t s, int tr = 0);
// the levels levels[0 .. nlev-1] (the last one the single-cell level) of a
// V-cycle in one single-block kernel; levels[0] starts from zero
constexpr long long kTailCells = 4096;
constexpr int kTailMaxLevels = 16;
constexpr int kTailThreads = 512;
template <typename T>
void launch_vcycle_tail(const Grid& G, int nf, const MGLevel* levels, int nlev, int nu1, int nu2, cudaStream_t s,
                        int tr);
template <typename T>
int launch_precond_out(const Grid& G, const T* C, double dt, int nf, const T* rp, const T* re, const T* ru,
                       const MGLevel& L0, T* z, double* partials, cudaStream_t s);

// adjoint.cu
// y = (a dU/dX + b dR/dX)^T w at X (p, T, chi and mass fluxes of X precomputed);
// adj: vjp_scratch_doubles(G) doubles of scratch
void launch_vjp(const Grid& G, const double* X, const double* p, const double* T, const double* chi, const double* Fmh,
                const double* w, double a_u, double b_r, double* adj, double* Xb, cudaStream_t s);
long long vjp_scratch_doubles(const Grid& G);
// partial sums of w_E . (conduction divergence / K0) (T of the state given)
void launch_dRdK0_dot(const Grid& G, const double* T, const double* w, double* partials, cudaStream_t s);
void launch_precondT_out(const Grid& G, const double* C, double dt, int nf, const double* y, double* rub, double* reb,
                         double* rpb, MGLevel& L0, cudaStream_t s);
void launch_precondT_in(const Grid& G, const double* C, int nf, const MGLevel& L0, const double* rub,
                        const double* reb, const double* rpb, double* z, cudaStream_t s);
void launch_mul(const double* x, const double* y, double* out, long long n, cudaStream_t s);
void launch_sub(const double* a, const double* b, double* out, long long n, cudaStream_t s);
void launch_mask_walls(const Grid& G, double* v, cudaStream_t s);

}  // namespace jfnk
