// Internal state of the GMG-PCG solver (not part of the ABI): its levels,
// the solver handle and the functions that the setup, the solve and the
// lockstep translation units share.
#pragma once

#include <atomic>
#include <vector>

#include "pa_internal.h"

namespace pa {


constexpr int kRedThreads = 256;
// Reductions: up to 8 CTAs of 256 threads per SM, enough loads in flight to
// stream HBM; the persistent coarse CG keeps to 2 CTAs per SM (its grid
// barriers cost more with more CTAs).
constexpr int kRedBlocks = 8 * 152;
constexpr int kCoopBlocks = 2 * 152;

// device scalar slots
enum Slot {
    S_RZ = 0, S_PQ, S_ALPHA, S_BETA, S_RR, S_BB, S_ZQ, S_ZR,
    C_RZ = 16, C_PQ, C_ALPHA, C_BETA, C_RR, C_BB, C_TOL2,
    P_NUM = 24, P_DEN,
    NSLOT = 32
};
enum FlagSlot { F_BREAK = 0, F_CDONE = 1, F_CIT = 2, F_CTIMEOUT = 3, NFLAG = 4 };

struct Dev {
    double *scal;       // [NSLOT]
    int *flag;          // [NFLAG]
    double *partial;    // [3][kRedBlocks]
    unsigned *counter;  // [1]
};

// Coarse basis of one axis at the fine nodes (transfers between p-levels):
// L[a*(pf+1) + j] = coarse basis a at fine node j (1D).
struct XferTab {
    double L[kMaxD * kMaxD];
};

// Coefficients of the cheb_order smoothing steps of a level: step k sets
// d = cd[k] d + cr[k] Dinv (r - A e), then e += d (cd[0] = 0).
constexpr int kMaxCheb = 8;
struct ChebCoef {
    double cd[kMaxCheb] = {}, cr[kMaxCheb] = {};
};

// ---------------------------------------------------------------- levels --
struct Level {
    int p = 0;
    pa_op *op = nullptr;    // FP64 operator (level 0: the caller's)
    pa_op *op32 = nullptr;  // FP32 operator (mixed mode, smoothed levels)
    bool own_op = false;
    int64_t n = 0;
    double *dinv = nullptr;
    float *dinv32 = nullptr;
    // work vectors (FP64 and FP32 copies for mixed mode)
    double *r = nullptr, *e = nullptr, *t = nullptr, *d = nullptr;
    float *r32 = nullptr, *e32 = nullptr, *t32 = nullptr, *d32 = nullptr;
    double *xa = nullptr, *xb = nullptr;  // transfer temporaries (fine size of this level)
    float *xa32 = nullptr, *xb32 = nullptr;
    XferTab xt{};  // coarse (next level) basis at this level's nodes
    bool hdown = false;  // the next level is this mesh coarsened once (p = 1 both), not a lower degree
    double lmax = 0.0;
    double theta = 0.0, delta = 0.0;
    ChebCoef cheb{};  // smoothing-step coefficients
    // coarse CG vectors
    double *cx = nullptr, *cr = nullptr, *cp = nullptr, *cq = nullptr;
    double *stencil = nullptr;  // assembled p = 1 coarse matrix (81 planes of n), or null
};

// One level of the h-hierarchy below the p = 1 level (assembled stencils).
struct HLevel {
    Grid g{};                   // grid of this level (nodes Mx x My x Mz)
    int64_t n = 0;              // 3 Nn
    double *vals = nullptr;     // stencil (81 planes of n); level 0 borrows the p = 1 stencil
    uint8_t *ess = nullptr;     // essential mask (level 0 borrows the operator's)
    double *dinv = nullptr;     // 1 / diag
    double *r = nullptr, *e = nullptr, *t = nullptr, *d = nullptr;  // level 0: r is the coarse CG residual
    double *e2 = nullptr;       // second iterate buffer of the fused smoothing steps
    double *xa = nullptr, *xb = nullptr;  // transfer temporaries (size of this level)
    double theta = 0.0, delta = 0.0, lmax = 0.0;
    ChebCoef cheb{};            // smoothing-step coefficients
    double *Ainv = nullptr;     // dense inverse on the coarsest level
};

}  // namespace pa

namespace pa {
struct StepGraphs {
    cudaGraphExec_t init = nullptr, iter = nullptr;
};
}  // namespace pa

struct pa_solver {
    std::vector<pa::Level> lv;
    bool use_graphs = true;
    cudaStream_t stream = nullptr;  // the solver's own stream (capture needs a non-legacy stream)
    pa::StepGraphs g64, g32, gmx;
    unsigned *bar = nullptr;      // grid barrier state of the persistent coarse CG
    double *coop_part = nullptr;  // its per-CTA partial sums [3][3][kRedBlocks]
    int coop_blocks = 0;          // co-resident CTAs (0: no cooperative launch)
    bool allow_coop = true;
    std::vector<pa::HLevel> hl;   // h-multigrid under the p = 1 level (empty: Jacobi-CG coarse)
    bool use_hmg = true;
    double *xin = nullptr, *bin = nullptr;  // FP64 solve operates on these copies
    int mode = PA_SOLVE_FP64;
    int cheb_order = 2;
    // Chebyshev target interval [cheb_lo, cheb_hi] * lambda_max(D^-1 A) and
    // the power iterations that estimate lambda_max
    double cheb_lo = 0.05, cheb_hi = 1.2;
    int cheb_kind = 1;  // 1: first-kind Chebyshev on the interval, 4: fourth kind on [0, cheb_hi]
    int power_its = 10;
    // bound of the persistent coarse kernel's grid-barrier waits, in SM
    // clock cycles (2 s at the device's clock by default)
    long long wait_cycles = 4000000000LL;
    int clock_khz = 2000000;  // SM clock of the device (its attribute, read at creation)
    // test hook: the inner solve with this index (1-based) of the next
    // iterative-refinement solve reports a breakdown (0: none)
    int inject_inner_failure = 0;
    // set by the owner (the server) to end the solve between CG steps
    const std::atomic<int> *cancel = nullptr;
    double coarse_rtol = 1e-2;
    int coarse_maxit = 50;
    pa::Dev dev{};
    double *h_scal = nullptr;  // pinned mirror of a few scalars
    int *h_flag = nullptr;
    // outer vectors (FP64)
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *t = nullptr;
    // inner (mixed) vectors
    float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *x32 = nullptr, *b32 = nullptr;
    std::vector<void *> allocs;
    // Phase filter of lockstep capture (several solvers stepped together):
    // the step functions run with only the kernels of phase ph_target
    // emitted; phases are separated by the operator applies, and the apply
    // that ends phase ph_target is recorded (ph_op, ph_x, ph_y) instead of
    // launched.  Off: every kernel and apply is launched as usual.
    int64_t coarse_its = 0;  // coarse iterations of the current solve (graph mode)
    bool ph_on = false;
    int ph_target = 0, ph_counter = 0;
    pa_op *ph_op = nullptr;
    const void *ph_x = nullptr;
    void *ph_y = nullptr;
};

namespace pa {

// setup (pa_solver_setup.cu)
double read_scalar(pa_solver *s, int slot, cudaStream_t st);

// flexible CG, V-cycle and coarse solves (pa_solver.cu)
// vectors of one flexible CG (x_zero: x starts at 0)
template <typename T>
struct FcgVecs {
    T *x, *b, *r, *z, *p, *q;
    bool x_zero;
};
FcgVecs<double> outer_vecs(pa_solver *s);
template <typename T, typename TP> int fcg_init_a(pa_solver *s, const FcgVecs<T> &v, cudaStream_t st);
template <typename T, typename TP> int fcg_init_b(pa_solver *s, const FcgVecs<T> &v, cudaStream_t st);
template <typename T, typename TP> int fcg_iter_a(pa_solver *s, const FcgVecs<T> &v, cudaStream_t st);
template <typename T, typename TP> int fcg_iter_b(pa_solver *s, const FcgVecs<T> &v, cudaStream_t st);
int build_coarse_graph(pa_solver *s, cudaStream_t st, cudaGraphExec_t *out);
int solve_begin(pa_solver *s, const double *b, double *x, double *bb_out, pa_solve_info *inf, bool *trivial);
int solve_finish(pa_solver *s, double *x, int rc_loop, bool converged, double bb, double tol2, pa_solve_info *inf);

}  // namespace pa
