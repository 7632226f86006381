// C ABI of the JFNK library and the host-side solver engine.
//
// The engine drives the device kernels on the caller's stream: Newton
// iterations (Sect. 4.1), restarted right-preconditioned GMRES (Sects. 4.1,
// 4.3) with the Jacobian-free product (Sect. 4.2) and the physics-based
// preconditioner (Sects. 3, 4.3).  All vectors live in the caller-provided
// workspace; the host only reads convergence scalars (a few doubles per
// GMRES iteration) through a pinned buffer.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/jfnk.h"
#include "common.cuh"
#include "kernels.h"

using namespace jfnk;

struct jfnk_handle {
    Grid G;
    jfnk_options opt;
    int nf;            // fields of the SI system: 1 sound, 2 sound + conduction, 0 none
    int mixed;
    long long nc, nvec;
    size_t ws_bytes;
    char* ws;
    cudaStream_t stream;
    int device;        // device current at jfnk_bind (-1: never bound)
    long long inner_cycles;   // V-cycles run by preconditioner applies (host count)
    double* hpin;      // pinned host scalars
    std::string err;
    int profiling;
    cudaEvent_t ev[16];
    // workspace carve-up
    double *bn, *G0, *L, *R, *Linv, *Rinv, *Xp, *dxh, *p, *T, *chi, *Fm, *FE, *Psi, *partials, *scal;
    double *H, *cs, *sn, *g, *y, *vscale, *hc2;
    void *V, *Z, *rp, *re, *ru, *C;
    // adjoint (FP64): VJP scratch, its output, transposed-preconditioner
    // temporaries, right-hand side, multiplier and a scaled input vector
    double *adj, *Xb, *rub, *reb, *rpb, *b64, *lam, *w64;
    // coefficients of the Jacobian-free product of the current linearisation:
    // jvP = L^-1/dt, jvQ = theta L^-1, jvC = L^-1 G(X)
    double *jvP, *jvQ, *jvC;
    long long npartials;
    long long ldv;     // column stride of V and Z: nvec rounded up to 64 (16-byte aligned columns)
    std::vector<MGLevel> levels;
    size_t tail_level; // first level of the single-block V-cycle tail (levels.size(): none)
    size_t elt;        // bytes per basis element
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

jfnk_status fail(jfnk_handle* h, jfnk_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    return st;
}

#define CUDA_TRY(h, call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return fail(h, JFNK_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define CUDA_CHECK_VOID(call) (void)(call)

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Carve the workspace (or, with base == nullptr, only measure it).
size_t plan(jfnk_handle* h, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        void* p = base ? (void*)(base + off) : nullptr;
        off += align256(bytes);
        return p;
    };
    const long long nc = h->nc, nv = h->nvec;
    const int nd = h->G.ndim, m = h->opt.gmres_m;
    h->bn = (double*)take(nv * 8);
    h->G0 = (double*)take(nv * 8);
    h->L = (double*)take(nv * 8);
    h->R = (double*)take(nv * 8);
    h->Linv = (double*)take(nv * 8);
    h->Rinv = (double*)take(nv * 8);
    h->Xp = (double*)take(nv * 8);
    h->dxh = (double*)take(nv * 8);
    h->p = (double*)take(nc * 8);
    h->T = (double*)take(nc * 8);
    h->chi = (double*)take(nc * 8);
    h->Fm = (double*)take(nd * nc * 8);
    h->FE = (double*)take(nd * nc * 8);
    h->Psi = (double*)take((long long)nd * nd * nc * 8);
    long long cb = cell_blocks(h->G);
    h->npartials = std::max<long long>(cb, (long long)std::max(kRedBlocks, kMaxRedBlocks) * (m + 1));
    h->partials = (double*)take(h->npartials * 8);
    h->scal = (double*)take(kNumSlots * 8);
    h->H = (double*)take((size_t)(m + 1) * m * 8);
    h->cs = (double*)take(m * 8);
    h->sn = (double*)take(m * 8);
    h->g = (double*)take((m + 1) * 8);
    h->y = (double*)take(m * 8);
    h->vscale = (double*)take((m + 1) * 8);
    h->hc2 = (double*)take((m + 1) * 8);
    // the adjoint (jfnk_vjp, jfnk_vjp_residual) runs on FP64 handles only:
    // mixed handles reserve none of its scratch
    h->adj = h->Xb = h->rub = h->reb = h->rpb = h->b64 = h->lam = h->w64 = nullptr;
    if (!h->mixed) {
        h->adj = (double*)take(vjp_scratch_doubles(h->G) * 8);
        h->Xb = (double*)take(nv * 8);
        h->rub = (double*)take(nd * nc * 8);
        h->reb = (double*)take(nc * 8);
        h->rpb = (double*)take(nc * 8);
        h->b64 = (double*)take(nv * 8);
        h->lam = (double*)take(nv * 8);
        h->w64 = (double*)take(nv * 8);
    }
    h->jvP = (double*)take(nv * 8);
    h->jvQ = (double*)take(nv * 8);
    h->jvC = (double*)take(nv * 8);
    const size_t e = h->elt;
    h->V = take((size_t)(m + 1) * h->ldv * e);
    h->Z = take((size_t)m * h->ldv * e);
    if (h->nf > 0) {
        h->rp = take(nc * e);
        h->re = take(nc * e);
        h->ru = take(nd * nc * e);
        h->C = take((size_t)PcNumFields * nc * e);
        for (auto& L : h->levels) {
            L.M = take((size_t)h->nf * h->nf * L.ncell * e);
            L.K = take((size_t)h->nf * nd * L.ncell * e);
            L.x = take((size_t)h->nf * L.ncell * e);
            L.rhs = take((size_t)h->nf * L.ncell * e);
            L.r = take((size_t)h->nf * L.ncell * e);
        }
    }
    return off;
}

void build_levels(jfnk_handle* h) {
    h->levels.clear();
    h->tail_level = (size_t)-1;
    if (h->nf == 0) return;
    MGLevel L;
    for (int d = 0; d < 3; ++d) {
        L.n[d] = h->G.n[d];
        L.h[d] = h->G.dx[d];
        L.ih2[d] = 1.0 / (L.h[d] * L.h[d]);
    }
    L.ncell = h->nc;
    h->levels.push_back(L);
    for (;;) {
        MGLevel C = h->levels.back();
        bool any = false;
        for (int d = 0; d < h->G.ndim; ++d)
            if (C.n[d] > 1) {
                C.n[d] /= 2;
                C.h[d] *= 2;
                C.ih2[d] = 1.0 / (C.h[d] * C.h[d]);
                any = true;
            }
        if (!any) break;
        C.ncell = (long long)C.n[0] * C.n[1] * C.n[2];
        h->levels.push_back(C);
    }
    // the coarse levels (which start from zero) at or below kTailCells run
    // as one single-block kernel when that covers at least two levels
    const size_t nl = h->levels.size();
    h->tail_level = nl;
    for (size_t l = 1; l + 1 < nl; ++l)
        if (h->levels[l].ncell <= kTailCells && nl - l <= (size_t)kTailMaxLevels) {
            h->tail_level = l;
            break;
        }
}

jfnk_status check_bound(jfnk_handle* h) {
    if (!h) return JFNK_EINVAL;
    if (!h->ws) return fail(h, JFNK_ENOMEM, "no workspace bound (call jfnk_bind)");
    return JFNK_OK;
}

jfnk_status sync_read(jfnk_handle* h) {
    CUDA_TRY(h, cudaMemcpyAsync(h->hpin, h->scal, kNumSlots * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    CUDA_TRY(h, cudaGetLastError());
    return JFNK_OK;
}

unsigned cblocks(jfnk_handle* h) { return cell_blocks(h->G); }

// G-type evaluation of state Xs into the assemble mode
template <int MODE, typename TO>
void eval(jfnk_handle* h, const double* Xs, double dt, double* outd, TO* outb) {
    cudaStream_t s = h->stream;
    launch_eos(h->G, Xs, h->p, h->T, h->chi, s);
    launch_fluxes(h->G, Xs, h->p, h->T, h->chi, h->Fm, h->FE, h->Psi, s);
    launch_assemble<MODE, TO>(h->G, Xs, h->p, h->Fm, h->FE, h->Psi, h->bn, h->G0, h->Linv, h->scal, kSlotDelta, dt,
                              outd, outb, s);
}

void scaling(jfnk_handle* h, const double* X) {
    launch_scaling(h->G, X, h->opt.alpha1, h->opt.alpha2, h->L, h->R, h->Linv, h->Rinv, h->partials, h->stream);
    launch_finalize(h->partials, (int)cblocks(h), h->scal, kSlotXhatNorm, 0, h->stream);
}

template <typename T>
T* Vcol(jfnk_handle* h, int j) { return (T*)h->V + (long long)j * h->ldv; }
template <typename T>
T* Zcol(jfnk_handle* h, int j) { return (T*)h->Z + (long long)j * h->ldv; }

// coefficients of the preconditioner at X (needs the scaling of X)
void si_setup(jfnk_handle* h, const double* X, double dt) {
    if (h->nf == 0) return;
    if (h->mixed) launch_pc_setup<float>(h->G, X, h->L, h->Rinv, dt, h->nf, (float*)h->C, h->levels[0], h->stream);
    else launch_pc_setup<double>(h->G, X, h->L, h->Rinv, dt, h->nf, (double*)h->C, h->levels[0], h->stream);
    for (size_t l = 0; l + 1 < h->levels.size(); ++l) {
        if (h->mixed) launch_coarsen<float>(h->G, h->nf, h->levels[l], h->levels[l + 1], h->stream);
        else launch_coarsen<double>(h->G, h->nf, h->levels[l], h->levels[l + 1], h->stream);
    }
}

// one V-cycle from level l; tr = 1 solves the transposed system
template <typename T>
// x_l starts at zero on coarse levels and, in the first cycle, on level 0
// (zero_start: the first half sweep reads no neighbours; the other colour is
// overwritten before it is read)
void vcycle(jfnk_handle* h, size_t l, int tr = 0, bool first = false) {
    cudaStream_t s = h->stream;
    auto& Lv = h->levels;
    if (l + 1 == Lv.size()) {
        launch_coarsest<T>(h->nf, Lv[l], s, tr);
        return;
    }
    if (l == h->tail_level) {
        launch_vcycle_tail<T>(h->G, h->nf, &Lv[l], (int)(Lv.size() - l), h->opt.mg_nu1, h->opt.mg_nu2, s, tr);
        return;
    }
    for (int k = 0; k < h->opt.mg_nu1; ++k) {
        launch_smooth<T>(h->G, h->nf, Lv[l], 0, s, tr, (k == 0 && (l > 0 || first)) ? 1 : 0);
        launch_smooth<T>(h->G, h->nf, Lv[l], 1, s, tr);
    }
    launch_restrict<T>(h->G, h->nf, Lv[l], Lv[l + 1], s, tr, h->opt.mg_nu1 > 0 ? 1 : 0);
    vcycle<T>(h, l + 1, tr);
    launch_prolong<T>(h->G, h->nf, Lv[l], Lv[l + 1], s);
    for (int k = 0; k < h->opt.mg_nu2; ++k) {
        launch_smooth<T>(h->G, h->nf, Lv[l], 1, s, tr);
        launch_smooth<T>(h->G, h->nf, Lv[l], 0, s, tr);
    }
}

// z = M^-1 (scale * v); partial |z|^2 -> scal[kSlotZnorm]
template <typename T>
void precond(jfnk_handle* h, const double* X, double dt, const T* v, int vslot, T* z) {
    cudaStream_t s = h->stream;
    if (h->nf == 0) {
        if (vslot >= 0) launch_scale_copy<T, T>(v, 1.0, h->vscale, vslot, 0, z, h->nvec, s);
        else launch_scale_copy<T, T>(v, 1.0, nullptr, -1, 0, z, h->nvec, s);
        launch_norm2_partials<T>(z, h->nvec, h->partials, s);
        launch_finalize(h->partials, kRedBlocks, h->scal, kSlotZnorm, 0, s);
        return;
    }
    (void)X;
    launch_precond_in<T>(h->G, (const T*)h->C, v, h->vscale, vslot, h->nf, (T*)h->rp, (T*)h->re, (T*)h->ru,
                         h->levels[0], s, h->opt.mg_nu1 > 0 ? 0 : 1);
    MGLevel& L0 = h->levels[0];
    const long long n0 = (long long)h->nf * L0.ncell;
    const bool adaptive = h->opt.inner_tol > 0.0;
    if (adaptive || h->opt.inner_monitor) {
        launch_norm2_partials<T>((const T*)L0.rhs, n0, h->partials, s);
        launch_finalize(h->partials, kRedBlocks, h->scal, kSlotInnerB, 0, s);
    }
    auto inner_residual = [&]() {
        launch_mg_residual<T>(h->G, h->nf, L0, s);
        launch_norm2_partials<T>((const T*)L0.r, n0, h->partials, s);
        launch_finalize(h->partials, kRedBlocks, h->scal, kSlotInnerR, 0, s);
    };
    if (adaptive) {
        // cycle until ||b - A x|| <= inner_tol ||b|| (a sync per cycle)
        for (int c = 0; c < h->opt.inner_max_cycles; ++c) {
            vcycle<T>(h, 0, 0, c == 0);
            ++h->inner_cycles;
            inner_residual();
            if (sync_read(h) != JFNK_OK) break;       // the error resurfaces at the caller's next sync
            if (!(h->hpin[kSlotInnerR] > h->opt.inner_tol * h->hpin[kSlotInnerB])) break;
        }
    } else {
        for (int c = 0; c < h->opt.mg_cycles; ++c) vcycle<T>(h, 0, 0, c == 0);
        h->inner_cycles += h->opt.mg_cycles;
        if (h->opt.inner_monitor) inner_residual();
    }
    const int np = launch_precond_out<T>(h->G, (const T*)h->C, dt, h->nf, (const T*)h->rp, (const T*)h->re,
                                         (const T*)h->ru, h->levels[0], z, h->partials, s);
    launch_finalize(h->partials, np, h->scal, kSlotZnorm, 0, s);
}

// out = J^ z (basis precision), requires scaling, G0 of X; delta_scaled:
// out = delta J^ z (the Arnoldi vectors of GMRES, which takes the 1/delta
// into its Hessenberg column)
template <typename TZ, typename T>
void jv(jfnk_handle* h, const double* X, double dt, const TZ* z, int znorm_ready, T* out, bool delta_scaled = false) {
    cudaStream_t s = h->stream;
    if (!znorm_ready) {
        launch_norm2_partials<TZ>(z, h->nvec, h->partials, s);
        launch_finalize(h->partials, kRedBlocks, h->scal, kSlotZnorm, 0, s);
    }
    if (h->opt.pert == JFNK_PERT_NEW) {
        launch_dot_partials<TZ>(X, h->Rinv, z, h->nvec, h->partials, s);
        launch_finalize(h->partials, kRedBlocks, h->scal, kSlotTmp, 1, s);
    }
    launch_delta(h->scal, h->opt.lambda, h->opt.pert, s);
    const bool prof = h->profiling != 0;
    if (prof) cudaEventRecord(h->ev[0], s);
    launch_perturb<TZ>(h->G, X, z, h->R, h->scal, kSlotDelta, h->Xp, s);
    if (prof) cudaEventRecord(h->ev[1], s);
    launch_eos(h->G, h->Xp, h->p, h->T, h->chi, s);
    if (prof) cudaEventRecord(h->ev[2], s);
    launch_face_fluxes(h->G, h->Xp, h->p, h->T, h->chi, h->Fm, h->FE, s);
    if (prof) cudaEventRecord(h->ev[3], s);
    launch_mom_fluxes(h->G, h->Xp, h->Fm, h->Psi, s);
    if (prof) cudaEventRecord(h->ev[4], s);
    if (delta_scaled)
        launch_assemble<kModeJvD, T>(h->G, h->Xp, h->p, h->Fm, h->FE, h->Psi, h->jvQ, h->jvC, h->jvP, h->scal,
                                     kSlotDelta, dt, nullptr, out, s);
    else
        launch_assemble<kModeJv, T>(h->G, h->Xp, h->p, h->Fm, h->FE, h->Psi, h->jvQ, h->jvC, h->jvP, h->scal,
                                    kSlotDelta, dt, nullptr, out, s);
    if (prof) cudaEventRecord(h->ev[5], s);
}

double ev_ms(jfnk_handle* h, int a, int b) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, h->ev[a], h->ev[b]) != cudaSuccess) return 0.0;
    return t;
}

struct Timer {
    jfnk_handle* h;
    int a, b;
    bool on;
    Timer(jfnk_handle* hh, int ia) : h(hh), a(ia), b(ia + 1), on(hh->profiling != 0) {
        if (on) cudaEventRecord(h->ev[a], h->stream);
    }
    void stop() {
        if (on) cudaEventRecord(h->ev[b], h->stream);
    }
    static double ms(jfnk_handle* h, int a) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, h->ev[a], h->ev[a + 1]) != cudaSuccess) return 0.0;
        return t;
    }
};

struct SolveOut {
    int iterations = 0;
    int converged = 0;
    double res = 0.0;
    double beta0 = 0.0;
    int jv = 0, pc = 0;
    double jv_ms = 0, pc_ms = 0, or_ms = 0;
    double kms[5] = {0, 0, 0, 0, 0};
    double inner_sum = 0, inner_max = 0;
    int inner_n = 0;
    int reorth = 0;      // second Gram-Schmidt passes
};

// Classical Gram-Schmidt of the new Arnoldi vector Vn = V[j+1] against
// V[0..j]: coefficients into hcol, partial sums of |Vn|^2 after the
// projection left in h->partials (the count is returned in nb).  reorth = 1
// adds a second pass always; reorth = 2 adds it only when the first pass
// shrank the vector below kDgksKappa of its norm (the selective criterion of
// Daniel, Gragg, Kaufman and Stewart, Math. Comp. 30 (1976) 772-795), which
// the host decides from two norms read back; `passes` counts second passes.
constexpr double kDgksKappa = 0.70710678118654752440;   // 1/sqrt(2)

template <typename T>
jfnk_status gram_schmidt(jfnk_handle* h, const T* V, T* Vn, int j, double* hcol, int& nb, int& passes) {
    cudaStream_t s = h->stream;
    const long long n = h->nvec, ld = h->ldv;
    if (h->opt.reorth == 2) {
        launch_norm2_partials<T>(Vn, n, h->partials, s);
        launch_finalize(h->partials, kRedBlocks, h->scal, kSlotWnorm0, 0, s);
    }
    nb = launch_multidot<T>(V, ld, j + 1, Vn, n, h->partials, s);
    launch_multidot_finalize(h->partials, nb, j + 1, h->vscale, hcol, 0, s);
    nb = launch_axpy_norm<T>(Vn, V, ld, j + 1, hcol, h->vscale, n, h->partials, s);
    bool second = h->opt.reorth == 1;
    if (h->opt.reorth == 2) {
        launch_finalize(h->partials, nb, h->scal, kSlotTmp, 0, s);
        jfnk_status st = sync_read(h);
        if (st != JFNK_OK) return st;
        second = h->hpin[kSlotTmp] < kDgksKappa * h->hpin[kSlotWnorm0];
    }
    if (second) {
        nb = launch_multidot<T>(V, ld, j + 1, Vn, n, h->partials, s);
        launch_multidot_finalize(h->partials, nb, j + 1, h->vscale, h->hc2, 0, s);
        nb = launch_axpy_norm<T>(Vn, V, ld, j + 1, h->hc2, h->vscale, n, h->partials, s);
        launch_add_col(hcol, h->hc2, j + 1, s);
        ++passes;
    }
    return JFNK_OK;
}

// GMRES on J^ M^-1, RHS in V[0] (unnormalised), solution accumulated in dxh.
template <typename T>
jfnk_status gmres(jfnk_handle* h, const double* X, double dt, double eta, SolveOut& so) {
    cudaStream_t s = h->stream;
    const int m = h->opt.gmres_m;
    const int ldh = m + 1;
    const long long n = h->nvec;
    jfnk_status st;
    launch_zero<double>(h->dxh, n, s);
    launch_norm2_partials<T>(Vcol<T>(h, 0), n, h->partials, s);
    launch_finalize(h->partials, kRedBlocks, h->scal, kSlotBeta, 0, s);
    if ((st = sync_read(h)) != JFNK_OK) return st;
    const double beta0 = h->hpin[kSlotBeta];
    so.beta0 = beta0;
    if (!std::isfinite(beta0)) return fail(h, JFNK_ENONFINITE, "non-finite residual norm");
    if (beta0 == 0.0) {
        so.converged = 1;
        return JFNK_OK;
    }
    int total = 0;
    double res = beta0;
    for (;;) {
        launch_init_cycle(h->scal, h->g, h->vscale, m, s);
        int k = 0;
        bool done = false;
        for (int j = 0; j < m; ++j) {
            if (total >= h->opt.gmres_max_it) break;
            {
                Timer t(h, 6);
                precond<T>(h, X, dt, Vcol<T>(h, j), j, Zcol<T>(h, j));
                t.stop();
            }
            jv<T, T>(h, X, dt, Zcol<T>(h, j), 1, Vcol<T>(h, j + 1), true);
            {
                Timer t(h, 8);
                double* hcol = h->H + (long long)j * ldh;
                int nb = 0;
                if ((st = gram_schmidt<T>(h, Vcol<T>(h, 0), Vcol<T>(h, j + 1), j, hcol, nb, so.reorth)) != JFNK_OK)
                    return st;
                launch_finalize(h->partials, nb, h->scal, kSlotTmp, 0, s);
                launch_set_subdiag(h->scal, hcol, j, h->vscale, s, kSlotInvDelta);
                launch_givens(h->H, ldh, j, h->cs, h->sn, h->g, h->scal, s);
                t.stop();
            }
            if ((st = sync_read(h)) != JFNK_OK) return st;
            if (h->profiling) {
                so.pc_ms += Timer::ms(h, 6);
                so.or_ms += Timer::ms(h, 8);
                for (int q = 0; q < 5; ++q) so.kms[q] += ev_ms(h, q, q + 1);
                so.jv_ms += ev_ms(h, 0, 5);
            }
            if ((h->opt.inner_monitor || h->opt.inner_tol > 0.0) && h->nf > 0) {
                const double b = h->hpin[kSlotInnerB];
                const double ratio = b > 0.0 ? h->hpin[kSlotInnerR] / b : 0.0;
                so.inner_sum += ratio;
                so.inner_max = std::max(so.inner_max, ratio);
                so.inner_n++;
            }
            so.jv++;
            so.pc++;
            total++;
            k = j + 1;
            res = h->hpin[kSlotRes];
            const double hn = h->hpin[kSlotTmp];
            if (!std::isfinite(res) || !std::isfinite(hn))
                return fail(h, JFNK_ENONFINITE, "non-finite value in GMRES iteration %d", total);
            if (hn == 0.0) { done = true; break; }
            if (!h->opt.fixed_iterations && res < eta * beta0) { done = true; break; }
        }
        if (k > 0) {
            launch_backsolve(h->H, ldh, k, h->g, h->y, s);
            launch_update<T>(h->dxh, (const T*)h->Z, h->ldv, k, h->y, n, s);
        }
        so.iterations = total;
        so.res = res / beta0;
        if (done || total >= h->opt.gmres_max_it || k == 0) {
            so.converged = res < eta * beta0 ? 1 : 0;
            return JFNK_OK;
        }
        // restart from the true residual r = b - J^ dxh
        jv<double, T>(h, X, dt, h->dxh, 0, Vcol<T>(h, 0));
        so.jv++;
        launch_restart_residual<T>(Vcol<T>(h, 0), h->G0, h->bn, h->Linv, n, s);
        launch_norm2_partials<T>(Vcol<T>(h, 0), n, h->partials, s);
        launch_finalize(h->partials, kRedBlocks, h->scal, kSlotBeta, 0, s);
    }
}

// scaling, G0, RHS in V[0] and the preconditioner at iterate X (b^n must be
// set); full_setup = false keeps the SI coefficients of the previous setup
// and renews only the scaling fields
template <typename T>
void linearize(jfnk_handle* h, const double* X, double dt, bool full_setup) {
    scaling(h, X);
    eval<kModeNewton, T>(h, X, dt, h->G0, Vcol<T>(h, 0));
    launch_jv_coeffs(h->Linv, h->G0, dt, h->opt.theta, h->jvP, h->jvQ, h->jvC, h->nvec, 2 * h->nc, h->stream);
    if (full_setup) {
        si_setup(h, X, dt);
    } else if (h->nf > 0) {
        if (h->mixed) launch_pc_rescale<float>(h->G, h->L, h->Rinv, (float*)h->C, h->stream);
        else launch_pc_rescale<double>(h->G, h->L, h->Rinv, (double*)h->C, h->stream);
    }
}

template <typename T>
jfnk_status newton_solve(jfnk_handle* h, const double* X, double dt, double eta, SolveOut& so, bool full_setup) {
    linearize<T>(h, X, dt, full_setup);
    return gmres<T>(h, X, dt, eta, so);
}

// one step of the SI scheme as a time integrator (Sect. 3.6), in place in X
template <typename T>
void si_step(jfnk_handle* h, double* X, double dt) {
    cudaStream_t s = h->stream;
    eval<kModeBn, double>(h, X, dt, h->bn, (double*)nullptr);     // b^n at X^n
    linearize<T>(h, X, dt, true);          // scaling, V[0] = -F^ = L^-1 R_U(X^n), SI setup at X^n
    precond<T>(h, X, dt, Vcol<T>(h, 0), -1, Zcol<T>(h, 0));
    launch_scale_copy<T, double>(Zcol<T>(h, 0), 1.0, nullptr, -1, 0, h->dxh, h->nvec, s);
    launch_newton_update(X, h->R, h->dxh, h->nvec, h->partials, s);
}

// ---------------------------------------------------------------------------
// adjoint (FP64 handles)
// ---------------------------------------------------------------------------

// out = (a dU/dX + b dR/dX)^T w at Xs
void vjp_apply(jfnk_handle* h, const double* Xs, const double* w, double a, double b, double* out) {
    cudaStream_t s = h->stream;
    launch_eos(h->G, Xs, h->p, h->T, h->chi, s);
    launch_face_fluxes(h->G, Xs, h->p, h->T, h->chi, h->Fm, h->FE, s);
    launch_vjp(h->G, Xs, h->p, h->T, h->chi, h->Fm, w, a, b, h->adj, out, s);
}

// z = M^-T y (transpose of the scaled physics-based preconditioner)
void precond_T(jfnk_handle* h, double dt, const double* y, double* z) {
    cudaStream_t s = h->stream;
    if (h->nf == 0) {
        CUDA_CHECK_VOID(cudaMemcpyAsync(z, y, h->nvec * 8, cudaMemcpyDeviceToDevice, s));
        return;
    }
    launch_precondT_out(h->G, (const double*)h->C, dt, h->nf, y, h->rub, h->reb, h->rpb, h->levels[0], s);
    for (int c = 0; c < h->opt.mg_cycles; ++c) vcycle<double>(h, 0, 1, c == 0);
    launch_precondT_in(h->G, (const double*)h->C, h->nf, h->levels[0], h->rub, h->reb, h->rpb, z, s);
}

// out = J^T z in scaled form: R (dG/dX)^T (L^-1 z) at Xs
void jT_apply(jfnk_handle* h, const double* Xs, double dt, const double* z, double* out) {
    cudaStream_t s = h->stream;
    launch_mul(h->Linv, z, h->w64, h->nvec, s);
    vjp_apply(h, Xs, h->w64, 1.0 / dt, -h->opt.theta, h->Xb);
    launch_mul(h->R, h->Xb, out, h->nvec, s);
}

// Restarted GMRES on J^T M^-T (right preconditioned), RHS in V[0] and b64.
jfnk_status gmres_adj(jfnk_handle* h, const double* X, double dt, double eta, SolveOut& so) {
    cudaStream_t s = h->stream;
    const int m = h->opt.gmres_m;
    const int ldh = m + 1;
    const long long n = h->nvec;
    jfnk_status st;
    double* V = (double*)h->V;
    double* Z = (double*)h->Z;
    launch_zero<double>(h->dxh, n, s);
    launch_norm2_partials<double>(V, n, h->partials, s);
    launch_finalize(h->partials, kRedBlocks, h->scal, kSlotBeta, 0, s);
    if ((st = sync_read(h)) != JFNK_OK) return st;
    const double beta0 = h->hpin[kSlotBeta];
    so.beta0 = beta0;
    if (!std::isfinite(beta0)) return fail(h, JFNK_ENONFINITE, "non-finite adjoint right-hand side");
    if (beta0 == 0.0) {
        so.converged = 1;
        return JFNK_OK;
    }
    int total = 0;
    double res = beta0;
    for (;;) {
        launch_init_cycle(h->scal, h->g, h->vscale, m, s);
        int k = 0;
        bool done = false;
        for (int j = 0; j < m; ++j) {
            if (total >= h->opt.gmres_max_it) break;
            const long long ld = h->ldv;
            double* Vj = V + (long long)j * ld;
            double* Zj = Z + (long long)j * ld;
            double* Vn = V + (long long)(j + 1) * ld;
            launch_scale_copy<double, double>(Vj, 1.0, h->vscale, j, 0, h->w64, n, s);
            precond_T(h, dt, h->w64, Zj);
            jT_apply(h, X, dt, Zj, Vn);
            double* hcol = h->H + (long long)j * ldh;
            int nb = 0;
            if ((st = gram_schmidt<double>(h, V, Vn, j, hcol, nb, so.reorth)) != JFNK_OK) return st;
            launch_finalize(h->partials, nb, h->scal, kSlotTmp, 0, s);
            launch_set_subdiag(h->scal, hcol, j, h->vscale, s);
            launch_givens(h->H, ldh, j, h->cs, h->sn, h->g, h->scal, s);
            if ((st = sync_read(h)) != JFNK_OK) return st;
            so.jv++;
            so.pc++;
            total++;
            k = j + 1;
            res = h->hpin[kSlotRes];
            const double hn = h->hpin[kSlotTmp];
            if (!std::isfinite(res) || !std::isfinite(hn))
                return fail(h, JFNK_ENONFINITE, "non-finite value in adjoint GMRES iteration %d", total);
            if (hn == 0.0) { done = true; break; }
            if (res < eta * beta0) { done = true; break; }
        }
        if (k > 0) {
            launch_backsolve(h->H, ldh, k, h->g, h->y, s);
            launch_update<double>(h->dxh, Z, h->ldv, k, h->y, n, s);
        }
        so.iterations = total;
        so.res = res / beta0;
        if (done || total >= h->opt.gmres_max_it || k == 0) {
            so.converged = res < eta * beta0 ? 1 : 0;
            return JFNK_OK;
        }
        jT_apply(h, X, dt, h->dxh, V);                 // restart from b - A x
        launch_sub(h->b64, V, V, n, s);
        launch_norm2_partials<double>(V, n, h->partials, s);
        launch_finalize(h->partials, kRedBlocks, h->scal, kSlotBeta, 0, s);
    }
}

jfnk_status validate_options(jfnk_handle* h, const jfnk_options* o) {
    if (!(o->theta > 0.0 && o->theta <= 1.0)) return fail(h, JFNK_EINVAL, "theta must be in (0, 1]");
    if (o->gmres_m < 1 || o->gmres_m > 64) return fail(h, JFNK_EINVAL, "gmres_m must be in [1, 64]");
    if (o->gmres_max_it < 1) return fail(h, JFNK_EINVAL, "gmres_max_it must be >= 1");
    if (o->newton_max < 1 || o->newton_max > JFNK_MAX_NEWTON) return fail(h, JFNK_EINVAL, "newton_max out of range");
    if (o->precond < 0 || o->precond > 2) return fail(h, JFNK_EINVAL, "unknown preconditioner");
    if (o->precision != JFNK_FP64 && o->precision != JFNK_MIXED) return fail(h, JFNK_EINVAL, "unknown precision");
    if (o->mg_cycles < 1 || o->mg_nu1 < 0 || o->mg_nu2 < 0) return fail(h, JFNK_EINVAL, "bad multigrid cycle counts");
    if (o->pc_freeze != 0 && o->pc_freeze != 1) return fail(h, JFNK_EINVAL, "pc_freeze must be 0 or 1");
    if (o->reorth < 0 || o->reorth > 2) return fail(h, JFNK_EINVAL, "reorth must be 0, 1 or 2");
    if (!(o->lambda > 0.0)) return fail(h, JFNK_EINVAL, "lambda must be positive");
    if (!(o->inner_tol >= 0.0) || o->inner_max_cycles < 1 || (o->inner_monitor != 0 && o->inner_monitor != 1))
        return fail(h, JFNK_EINVAL, "bad inner tolerance options");
    if (o->pert != JFNK_PERT_OLD && o->pert != JFNK_PERT_NEW) return fail(h, JFNK_EINVAL, "unknown perturbation rule");
    return JFNK_OK;
}

}  // namespace

// accessors for the allocation-free entry point (noalloc.cu)
const jfnk::Grid* jfnk_handle_grid(const jfnk_handle* h) { return &h->G; }
cudaStream_t jfnk_handle_stream(const jfnk_handle* h) { return h->stream; }
int jfnk_handle_device(const jfnk_handle* h) { return h->device; }
void jfnk_handle_set_error(jfnk_handle* h, const char* msg) { h->err = msg; }

extern "C" {

void jfnk_default_options(jfnk_options* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->theta = 0.5;
    o->lambda = 1e-7;
    o->alpha1 = 1e-5;
    o->alpha2 = 1.0;
    o->eta = 1e-4;
    o->newton_tol = 1e-8;
    o->pert = JFNK_PERT_OLD;
    o->gmres_m = 30;
    o->gmres_max_it = 300;
    o->newton_min = 2;
    o->newton_max = 20;
    o->precond = JFNK_PRECOND_SOUND;
    o->mg_cycles = 2;
    o->mg_nu1 = 2;
    o->mg_nu2 = 2;
    o->precision = JFNK_FP64;
    o->reorth = 0;
    o->fixed_iterations = 0;
    o->pc_freeze = 0;
    o->inner_tol = 0.0;
    o->inner_max_cycles = 50;
    o->inner_monitor = 0;
}

jfnk_status jfnk_create(const jfnk_grid* grid, const jfnk_eos* eos, const jfnk_gravity* gravity,
                        const jfnk_conductivity* cond, const jfnk_options* opt, jfnk_handle** out) {
    if (!out || !grid || !eos) return JFNK_EINVAL;
    *out = nullptr;
    jfnk_handle* h = new jfnk_handle();
    h->ws = nullptr;
    h->hpin = nullptr;
    h->stream = 0;
    h->device = -1;
    h->inner_cycles = 0;
    h->profiling = 0;
    for (auto& e : h->ev) e = nullptr;
    if (opt) h->opt = *opt;
    else jfnk_default_options(&h->opt);
    jfnk_status st = validate_options(h, &h->opt);
    if (st != JFNK_OK) { *out = h; return st; }
    Grid& G = h->G;
    G.ndim = grid->ndim;
    if (G.ndim != 2 && G.ndim != 3) { *out = h; return fail(h, JFNK_EINVAL, "ndim must be 2 or 3"); }
    for (int d = 0; d < 3; ++d) {
        G.n[d] = grid->n[d];
        G.bc[d] = grid->bc[d];
        if (d < G.ndim) {
            if (G.n[d] < 4) { *out = h; return fail(h, JFNK_EINVAL, "need at least 4 cells per direction"); }
            if (G.bc[d] != 0 && G.bc[d] != 1) { *out = h; return fail(h, JFNK_EINVAL, "unknown boundary type"); }
            if (!(grid->hi[d] > grid->lo[d])) { *out = h; return fail(h, JFNK_EINVAL, "empty domain"); }
            G.dx[d] = (grid->hi[d] - grid->lo[d]) / G.n[d];
        } else {
            if (G.n[d] != 1) { *out = h; return fail(h, JFNK_EINVAL, "n[2] must be 1 in 2D"); }
            G.dx[d] = 1.0;
            G.bc[d] = 0;
        }
        G.idx[d] = 1.0 / G.dx[d];
        G.idx2[d] = G.idx[d] * G.idx[d];
        G.tidx[d] = 2.0 * G.idx[d];
        G.hidx[d] = 0.5 * G.idx[d];
    }
    G.ncell = (long long)G.n[0] * G.n[1] * G.n[2];
    if (!(eos->gamma > 1.0)) { *out = h; return fail(h, JFNK_EINVAL, "gamma must exceed 1"); }
    if (eos->energy_form != 0 && eos->energy_form != 1) { *out = h; return fail(h, JFNK_EINVAL, "unknown energy form"); }
    G.gamma = eos->gamma;
    G.gm1 = eos->gamma - 1.0;
    G.energy_form = eos->energy_form;
    for (int d = 0; d < 3; ++d) G.g[d] = (gravity && d < G.ndim) ? gravity->g[d] : 0.0;
    G.K0 = cond ? cond->K0 : 0.0;
    G.chi_exp = cond ? cond->exponent : 3.0;
    if (G.K0 < 0.0) { *out = h; return fail(h, JFNK_EINVAL, "K0 must be >= 0"); }
    G.theta = h->opt.theta;
    set_grid_flags(G);
    h->nc = G.ncell;
    h->nvec = (2 + G.ndim) * G.ncell;
    h->ldv = (h->nvec + 63) / 64 * 64;
    h->nf = h->opt.precond == JFNK_PRECOND_SOUND ? 1 : (h->opt.precond == JFNK_PRECOND_SOUND_DIFF ? 2 : 0);
    h->mixed = h->opt.precision == JFNK_MIXED;
    h->elt = h->mixed ? sizeof(float) : sizeof(double);
    if (h->nf > 0)
        for (int d = 0; d < G.ndim; ++d)
            if (!pow2(G.n[d])) { *out = h; return fail(h, JFNK_EINVAL, "preconditioned solves need power-of-two grids"); }
    build_levels(h);
    h->ws_bytes = plan(h, nullptr);
    *out = h;
    return JFNK_OK;
}

size_t jfnk_workspace_bytes(const jfnk_handle* h) { return h ? h->ws_bytes : 0; }

long long jfnk_vector_length(const jfnk_handle* h) { return h ? h->nvec : 0; }

jfnk_status jfnk_bind(jfnk_handle* h, void* ws, size_t bytes, void* stream) {
    if (!h) return JFNK_EINVAL;
    if (!ws || bytes < h->ws_bytes) return fail(h, JFNK_ENOMEM, "workspace of %zu bytes, need %zu", bytes, h->ws_bytes);
    if (((uintptr_t)ws) & 255) return fail(h, JFNK_EINVAL, "workspace must be 256-byte aligned");
    int dev = 0;
    CUDA_TRY(h, cudaGetDevice(&dev));
    h->ws = (char*)ws;
    h->stream = (cudaStream_t)stream;
    h->device = dev;
    plan(h, h->ws);
    if (!h->hpin) CUDA_TRY(h, cudaMallocHost((void**)&h->hpin, kNumSlots * sizeof(double)));
    return JFNK_OK;
}

jfnk_status jfnk_set_options(jfnk_handle* h, const jfnk_options* o) {
    if (!h || !o) return JFNK_EINVAL;
    jfnk_status st = validate_options(h, o);
    if (st != JFNK_OK) return st;
    if (o->precision != h->opt.precision || o->gmres_m != h->opt.gmres_m || o->precond != h->opt.precond)
        return fail(h, JFNK_EINVAL, "precision, gmres_m and precond are fixed at creation");
    h->opt = *o;
    h->G.theta = o->theta;
    return JFNK_OK;
}

jfnk_status jfnk_set_profiling(jfnk_handle* h, int on) {
    if (!h) return JFNK_EINVAL;
    if (on && !h->ev[0])
        for (auto& e : h->ev) CUDA_TRY(h, cudaEventCreate(&e));
    h->profiling = on;
    return JFNK_OK;
}

jfnk_status jfnk_residual(jfnk_handle* h, const double* X, const double* Xn, double dt, double* F) {
    jfnk_status st = check_bound(h);
    if (st) return st;
    if (!X || !Xn || !F || !(dt > 0.0)) return fail(h, JFNK_EINVAL, "bad arguments to jfnk_residual");
    eval<kModeBn, double>(h, Xn, dt, h->bn, (double*)nullptr);
    eval<kModeRes, double>(h, X, dt, F, (double*)nullptr);
    CUDA_TRY(h, cudaGetLastError());
    return JFNK_OK;
}

jfnk_status jfnk_scaling(jfnk_handle* h, const double* X, double* L, double* R, double* xhat_norm) {
    jfnk_status st = check_bound(h);
    if (st) return st;
    if (!X) return fail(h, JFNK_EINVAL, "bad arguments to jfnk_scaling");
    scaling(h, X);
    if (L) CUDA_TRY(h, cudaMemcpyAsync(L, h->L, h->nvec * 8, cudaMemcpyDeviceToDevice, h->stream));
    if (R) CUDA_TRY(h, cudaMemcpyAsync(R, h->R, h->nvec * 8, cudaMemcpyDeviceToDevice, h->stream));
    if (xhat_norm) {
        if ((st = sync_read(h)) != JFNK_OK) return st;
        *xhat_norm = h->hpin[kSlotXhatNorm];
    }
    CUDA_TRY(h, cudaGetLastError());
    return JFNK_OK;
}

jfnk_status jfnk_jv(jfnk_handle* h, const double* X, double dt, const void* v, void* Jv, double* delta_used) {
    jfnk_status st = check_bound(h);
    if (st) return st;
    if (!X || !v || !Jv || !(dt > 0.0)) return fail(h, JFNK_EINVAL, "bad arguments to jfnk_jv");
    scaling(h, X);
    eval<kModeG, double>(h, X, dt, h->G0, (double*)nullptr);
    launch_jv_coeffs(h->Linv, h->G0, dt, h->opt.theta, h->jvP, h->jvQ, h->jvC, h->nvec, 2 * h->nc, h->stream);
    if (h->mixed) jv<float, float>(h, X, dt, (const float*)v, 0, (float*)Jv);
    else jv<double, double>(h, X, dt, (const double*)v, 0, (double*)Jv);
    if (delta_used) {
        if ((st = sync_read(h)) != JFNK_OK) return st;
        *delta_used = h->hpin[kSlotDelta];
    }
    CUDA_TRY(h, cudaGetLastError());
    return JFNK_OK;
}

jfnk_status jfnk_precond_apply(jfnk_handle* h, const double* X, double dt, const void* v, void* w) {
    jfnk_status st = check_bound(h);
    if (st) return st;
    if (!X || !v || !w || !(dt > 0.0)) return fail(h, JFNK_EINVAL, "bad arguments to jfnk_precond_apply");
    scaling(h, X);
    si_setup(h, X, dt);
    if (h->mixed) precond<float>(h, X, dt, (const float*)v, -1, (float*)w);
    else precond<double>(h, X, dt, (const double*)v, -1, (double*)w);
    CUDA_TRY(h, cudaGetLastError());
    return JFNK_OK;
}

jfnk_status jfnk_linear_solve(jfnk_handle* h, const double* X, const double* Xn, double dt, double* dxhat,
                              jfnk_stats* stats) {
    jfnk_status st = check_bound(h);
    if (st) return st;
    if (!X || !Xn || !dxhat || !(dt > 0.0)) return fail(h, JFNK_EINVAL, "bad arguments to jfnk_linear_solve");
    eval<kModeBn, double>(h, Xn, dt, h->bn, (double*)nullptr);
    SolveOut so;
    h->inner_cycles = 0;
    st = h->mixed ? newton_solve<float>(h, X, dt, h->opt.eta, so, true)
                  : newton_solve<double>(h, X, dt, h->opt.eta, so, true);
    if (st < 0) return st;
    CUDA_TRY(h, cudaMemcpyAsync(dxhat, h->dxh, h->nvec * 8, cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->newton_iterations = 1;
        stats->gmres_iterations[0] = so.iterations;
        stats->gmres_iterations_total = so.iterations;
        stats->gmres_res[0] = so.res;
        stats->gmres_converged[0] = so.converged;
        stats->fhat_norm[0] = so.beta0;
        stats->jv_evaluations = so.jv;
        stats->precond_applies = so.pc;
        stats->inner_res_mean = so.inner_n > 0 ? so.inner_sum / so.inner_n : 0.0;
        stats->inner_res_max = so.inner_max;
        stats->inner_cycles = h->inner_cycles;
        stats->reorth_passes = so.reorth;
    }
    return so.converged ? JFNK_OK : JFNK_ENOCONV_GMRES;
}

jfnk_status jfnk_step(jfnk_handle* h, double* X, double dt, double newton_tol, double krylov_tol,
                      jfnk_stats* stats) {
    jfnk_status st = check_bound(h);
    if (st) return st;
    if (!X || !(dt > 0.0)) return fail(h, JFNK_EINVAL, "bad arguments to jfnk_step");
    const double ntol = newton_tol > 0.0 ? newton_tol : h->opt.newton_tol;
    const double eta = krylov_tol > 0.0 ? krylov_tol : h->opt.eta;
    jfnk_stats local;
    jfnk_stats* S = stats ? stats : &local;
    memset(S, 0, sizeof *S);
    if (h->profiling) cudaEventRecord(h->ev[10], h->stream);
    const long long launches0 = g_launch_count;
    h->inner_cycles = 0;
    double inner_sum = 0.0;
    int inner_n = 0;
    eval<kModeBn, double>(h, X, dt, h->bn, (double*)nullptr);      // X holds X^n here
    bool gmres_fail = false;
    for (int k = 0; k < h->opt.newton_max; ++k) {
        SolveOut so;
        // X^(0) = X^n: with pc_freeze the first setup is the one at X^n
        const bool full = k == 0 || !h->opt.pc_freeze;
        st = h->mixed ? newton_solve<float>(h, X, dt, eta, so, full) : newton_solve<double>(h, X, dt, eta, so, full);
        if (st < 0) return st;
        launch_newton_update(X, h->R, h->dxh, h->nvec, h->partials, h->stream);
        launch_finalize(h->partials, kRedBlocks, h->scal, kSlotDxInf, 2, h->stream);
        if ((st = sync_read(h)) != JFNK_OK) return st;
        const double dinf = h->hpin[kSlotDxInf];
        S->newton_iterations = k + 1;
        S->gmres_iterations[k] = so.iterations;
        S->gmres_iterations_total += so.iterations;
        S->gmres_res[k] = so.res;
        S->gmres_converged[k] = so.converged;
        S->fhat_norm[k] = so.beta0;
        S->dx_inf[k] = dinf;
        S->jv_evaluations += so.jv;
        S->precond_applies += so.pc;
        S->jv_ms += so.jv_ms;
        S->precond_ms += so.pc_ms;
        S->ortho_ms += so.or_ms;
        for (int q = 0; q < 5; ++q) S->jv_kernel_ms[q] += so.kms[q];
        inner_sum += so.inner_sum;
        inner_n += so.inner_n;
        S->reorth_passes += so.reorth;
        S->inner_res_max = std::max(S->inner_res_max, so.inner_max);
        if (!so.converged) gmres_fail = true;
        if (!std::isfinite(dinf)) return fail(h, JFNK_ENONFINITE, "non-finite Newton correction");
        if (!h->opt.fixed_iterations && k + 1 >= h->opt.newton_min && dinf < ntol) {
            S->converged = 1;
            break;
        }
    }
    if (h->profiling) {
        cudaEventRecord(h->ev[11], h->stream);
        cudaEventSynchronize(h->ev[11]);
        S->step_ms = Timer::ms(h, 10);
    }
    S->kernel_launches = g_launch_count - launches0;
    S->inner_res_mean = inner_n > 0 ? inner_sum / inner_n : 0.0;
    S->inner_cycles = h->inner_cycles;
    if (!S->converged && !h->opt.fixed_iterations) return JFNK_ENOCONV_NEWTON;
    (void)gmres_fail;
    return JFNK_OK;
}

jfnk_status jfnk_si_step(jfnk_handle* h, double* X, double dt) {
    jfnk_status st = check_bound(h);
    if (st) return st;
    if (!X || !(dt > 0.0)) return fail(h, JFNK_EINVAL, "bad arguments to jfnk_si_step");
    if (h->nf == 0) return fail(h, JFNK_EINVAL, "jfnk_si_step needs the SI preconditioner (precond 1 or 2)");
    if (h->mixed) si_step<float>(h, X, dt);
    else si_step<double>(h, X, dt);
    CUDA_TRY(h, cudaGetLastError());
    return JFNK_OK;
}

jfnk_status jfnk_vjp(jfnk_handle* h, const double* Xn, const double* Xnp1, double dt, const double* gbar, double* gXn,
                     double* gK0, jfnk_stats* stats) {
    jfnk_status st = check_bound(h);
    if (st) return st;
    if (!Xn || !Xnp1 || !gbar || !gXn || !(dt > 0.0)) return fail(h, JFNK_EINVAL, "bad arguments to jfnk_vjp");
    if (h->mixed) return fail(h, JFNK_EINVAL, "jfnk_vjp needs an FP64 handle");
    cudaStream_t s = h->stream;
    const long long n = h->nvec;
    scaling(h, Xnp1);
    si_setup(h, Xnp1, dt);
    double* V0 = (double*)h->V;
    launch_mul(h->R, gbar, V0, n, s);
    launch_mask_walls(h->G, V0, s);
    CUDA_TRY(h, cudaMemcpyAsync(h->b64, V0, n * 8, cudaMemcpyDeviceToDevice, s));
    SolveOut so;
    st = gmres_adj(h, Xnp1, dt, h->opt.eta, so);
    if (st < 0) return st;
    launch_mul(h->Linv, h->dxh, h->lam, n, s);
    vjp_apply(h, Xn, h->lam, 1.0 / dt, 1.0 - h->opt.theta, gXn);
    double gk = 0.0;
    if (h->G.K0 != 0.0) {
        const double wts[2] = {h->opt.theta, 1.0 - h->opt.theta};
        const double* states[2] = {Xnp1, Xn};
        for (int q = 0; q < 2; ++q) {
            launch_eos(h->G, states[q], h->p, h->T, h->chi, s);
            launch_dRdK0_dot(h->G, h->T, h->lam, h->partials, s);
            launch_finalize(h->partials, (int)cblocks(h), h->scal, kSlotTmp, 1, s);
            if ((st = sync_read(h)) != JFNK_OK) return st;
            gk += wts[q] * h->hpin[kSlotTmp];
        }
    } else {
        CUDA_TRY(h, cudaStreamSynchronize(s));
    }
    CUDA_TRY(h, cudaGetLastError());
    if (gK0) *gK0 = gk;
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->newton_iterations = 1;
        stats->gmres_iterations[0] = so.iterations;
        stats->gmres_iterations_total = so.iterations;
        stats->gmres_res[0] = so.res;
        stats->gmres_converged[0] = so.converged;
        stats->fhat_norm[0] = so.beta0;
    }
    return so.converged ? JFNK_OK : JFNK_ENOCONV_GMRES;
}

jfnk_status jfnk_vjp_residual(jfnk_handle* h, const double* X, double dt, const double* w, double* y) {
    jfnk_status st = check_bound(h);
    if (st) return st;
    if (!X || !w || !y || !(dt > 0.0)) return fail(h, JFNK_EINVAL, "bad arguments to jfnk_vjp_residual");
    if (h->mixed) return fail(h, JFNK_EINVAL, "jfnk_vjp_residual needs an FP64 handle");
    vjp_apply(h, X, w, 1.0 / dt, -h->opt.theta, y);
    CUDA_TRY(h, cudaGetLastError());
    return JFNK_OK;
}

jfnk_status jfnk_dt_from_cfl(jfnk_handle* h, const double* X, double cfl, double* dt) {
    jfnk_status st = check_bound(h);
    if (st) return st;
    if (!X || !dt || !(cfl > 0.0)) return fail(h, JFNK_EINVAL, "bad arguments to jfnk_dt_from_cfl");
    launch_signal_speed(h->G, X, h->partials, h->stream);
    launch_finalize(h->partials, (int)cblocks(h), h->scal, kSlotMaxSpeed, 2, h->stream);
    if ((st = sync_read(h)) != JFNK_OK) return st;
    double vmax = h->hpin[kSlotMaxSpeed];
    if (!std::isfinite(vmax) || !(vmax > 0.0)) return fail(h, JFNK_ENONFINITE, "non-finite or zero signal speed");
    double hmin = h->G.dx[0];
    for (int d = 1; d < h->G.ndim; ++d) hmin = std::min(hmin, h->G.dx[d]);
    *dt = cfl * hmin / vmax;
    return JFNK_OK;
}

const char* jfnk_last_error(const jfnk_handle* h) { return h ? h->err.c_str() : "null handle"; }

void jfnk_destroy(jfnk_handle* h) {
    if (!h) return;
    if (h->hpin) cudaFreeHost(h->hpin);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    delete h;
}

}  // extern "C"
