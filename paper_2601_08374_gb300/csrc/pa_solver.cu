// GMG-preconditioned CG solver (Sec. 3): p-levels on the fine mesh, then
// optional h-levels at p = 1 on uniformly coarsened meshes; V(1,1) cycle
// with Chebyshev-Jacobi smoothing on every level but the coarsest (Sec. 3.1),
// interpolation prolongation and its exact transpose as restriction (GLL
// spaces between p-levels, natural injection between h-levels, Sec. 3); on
// the coarsest level an assembled 27-point stencil solved inexactly by FP64
// CG preconditioned by a geometric multigrid of Galerkin stencils (Sec. 3.2,
// in place of AMG; Jacobi-CG selectable); an outer flexible CG.
//
// All vectors and scalars stay on the device.  Dot products are
// deterministic two-level reductions (fixed block partition, last block sums
// the partials in order), and the coefficients alpha/beta are formed on the
// device, so an iteration enqueues without host round trips; the host reads
// one residual norm per outer iteration to test convergence.  Each CG step
// is captured once into a CUDA graph whose coarse CG is a conditional WHILE
// node driven by a device-side stop flag, so a step is one graph launch and
// the coarse solve runs only the iterations it needs (an eager path with a
// fixed-length coarse loop of early-returning kernels remains as fallback).
//
// Mixed modes: PA_SOLVE_MIXED is iterative refinement in FP64 (residual
// b - A x with the FP64 operator, FP64 norms) around an inner flexible CG in
// FP32 storage with FP64 dot products, preconditioned by an FP32 V-cycle;
// PA_SOLVE_MIXED_FCG is the FP64 flexible CG preconditioned by the FP32
// V-cycle.  The coarse-level solve is FP64 in every mode.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "pa_internal.h"

namespace pa {
namespace {

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
enum FlagSlot { F_BREAK = 0, F_CDONE = 1, F_CIT = 2, NFLAG = 4 };  // slot 3: coarse barrier timeout

struct Dev {
    double *scal;       // [NSLOT]
    int *flag;          // [NFLAG]
    double *partial;    // [3][kRedBlocks]
    unsigned *counter;  // [1]
};

template <typename T>
__device__ inline double dd(T v) { return (double)v; }

// Block-level sum of up to 3 values; result valid in thread 0.
template <int K>
__device__ inline void block_sum(double (&v)[K])
{
    __shared__ double sh[K][kRedThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double x = (lane < (int)(blockDim.x >> 5)) ? sh[k][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            v[k] = x;
        }
    }
}

// Publishes the block partials; returns true in thread 0 of the last block,
// with tot[] holding the grid sums.  The last block adds the partials with
// all its threads in a fixed assignment and a fixed tree, so the result is
// deterministic for a given grid size.
template <int K>
__device__ inline bool grid_sum(Dev d, double (&v)[K], double (&tot)[K])
{
    block_sum<K>(v);
    __shared__ bool last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) d.partial[k * kRedBlocks + blockIdx.x] = v[k];
        __threadfence();
        unsigned prev = atomicAdd(d.counter, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double acc = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            acc += ((volatile double *)d.partial)[k * kRedBlocks + b];
        w[k] = acc;
    }
    block_sum<K>(w);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) tot[k] = w[k];
        *d.counter = 0u;
        return true;
    }
    return false;
}

#define GRID_STRIDE(i, n) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------- outer / inner FCG
// pq = (p, q); alpha = rz / pq (breakdown flag if pq <= 0 or not finite)
template <typename T>
__global__ void k_fcg_pq(Dev d, const T *p, const T *q, int64_t n, int slot_base)
{
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(i, n) v[0] += dd(p[i] * q[i]);
    if (grid_sum<1>(d, v, tot)) {
        double pq = tot[0];
        d.scal[slot_base + S_PQ] = pq;
        if (!(pq > 0.0) || !isfinite(pq)) {
            d.flag[F_BREAK] = 1;
            d.scal[slot_base + S_ALPHA] = 0.0;
        } else {
            d.scal[slot_base + S_ALPHA] = d.scal[slot_base + S_RZ] / pq;
        }
    }
}

// x += alpha p ; r -= alpha q ; rr = (r, r)
template <typename T, typename TX>
__global__ void k_fcg_update(Dev d, TX *x, T *r, const T *p, const T *q, int64_t n, int slot_base)
{
    const T alpha = (T)d.scal[slot_base + S_ALPHA];
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(i, n)
    {
        x[i] = (TX)(x[i] + (TX)(alpha * p[i]));
        const T ri = r[i] - alpha * q[i];
        r[i] = ri;
        v[0] += dd(ri * ri);
    }
    if (grid_sum<1>(d, v, tot)) {
        d.scal[slot_base + S_RR] = tot[0];
        if (!isfinite(tot[0])) d.flag[F_BREAK] = 1;
    }
}

// zr = (z, r), zq = (z, q); flexible (Polak-Ribiere) beta = -alpha zq / rz;
// rz <- zr.  With q = A p and r_new = r_old - alpha q this is
// (z, r_new - r_old) / rz_old.
template <typename T>
__global__ void k_fcg_beta(Dev d, const T *z, const T *r, const T *q, int64_t n, int slot_base)
{
    double v[2] = {0.0, 0.0}, tot[2];
    GRID_STRIDE(i, n)
    {
        const T zi = z[i];
        v[0] += dd(zi * r[i]);
        v[1] += dd(zi * q[i]);
    }
    if (grid_sum<2>(d, v, tot)) {
        double rz_old = d.scal[slot_base + S_RZ];
        double beta = -d.scal[slot_base + S_ALPHA] * tot[1] / rz_old;
        if (!isfinite(beta)) {
            d.flag[F_BREAK] = 1;
            beta = 0.0;
        }
        d.scal[slot_base + S_BETA] = beta;
        d.scal[slot_base + S_RZ] = tot[0];
        d.scal[slot_base + S_ZR] = tot[0];
        d.scal[slot_base + S_ZQ] = tot[1];
    }
}

// p = z + beta p
template <typename T>
__global__ void k_fcg_p(Dev d, T *p, const T *z, int64_t n, int slot_base)
{
    const T beta = (T)d.scal[slot_base + S_BETA];
    GRID_STRIDE(i, n) p[i] = z[i] + beta * p[i];
}

// rz = (r, z), rr = (r, r), p = z   (FCG start)
template <typename T>
__global__ void k_fcg_start(Dev d, T *p, const T *z, const T *r, int64_t n, int slot_base)
{
    double v[2] = {0.0, 0.0}, tot[2];
    GRID_STRIDE(i, n)
    {
        const T zi = z[i], ri = r[i];
        p[i] = zi;
        v[0] += dd(ri * zi);
        v[1] += dd(ri * ri);
    }
    if (grid_sum<2>(d, v, tot)) {
        d.scal[slot_base + S_RZ] = tot[0];
        d.scal[slot_base + S_RR] = tot[1];
        if (!isfinite(tot[0]) || !isfinite(tot[1])) d.flag[F_BREAK] = 1;
    }
}

// out[slot] = (a, a)
template <typename T>
__global__ void k_norm2(Dev d, const T *a, int64_t n, int slot)
{
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(i, n) v[0] += dd(a[i] * a[i]);
    if (grid_sum<1>(d, v, tot)) d.scal[slot] = tot[0];
}

// r = b - t
template <typename TB, typename TT, typename TR>
__global__ void k_sub(TR *r, const TB *b, const TT *t, int64_t n)
{
    GRID_STRIDE(i, n) r[i] = (TR)(dd(b[i]) - dd(t[i]));
}

// y = (TY) (s * x)
template <typename TX, typename TY>
__global__ void k_scale_copy(TY *y, const TX *x, double s, int64_t n)
{
    if (s == 1.0) {
        GRID_STRIDE(i, n) y[i] = (TY)x[i];
    } else {
        GRID_STRIDE(i, n) y[i] = (TY)(s * dd(x[i]));
    }
}

// x += s * d
template <typename TX, typename TD>
__global__ void k_axpy(TX *x, const TD *dv, double s, int64_t n)
{
    GRID_STRIDE(i, n) x[i] = (TX)(dd(x[i]) + s * dd(dv[i]));
}

// ------------------------------------------------------------- coarse CG
// start: x = 0, r = b, p = Dinv r, rz = (r, Dinv r), bb = (b, b), done = bb == 0
__global__ void k_cg_start(Dev d, double *x, double *r, double *p, const double *b, const double *dinv, int64_t n,
                           double tol2)
{
    double v[2] = {0.0, 0.0}, tot[2];
    GRID_STRIDE(i, n)
    {
        double bi = b[i], zi = dinv[i] * bi;
        x[i] = 0.0;
        r[i] = bi;
        p[i] = zi;
        v[0] += bi * zi;
        v[1] += bi * bi;
    }
    if (grid_sum<2>(d, v, tot)) {
        d.scal[C_RZ] = tot[0];
        d.scal[C_BB] = tot[1];
        d.scal[C_RR] = tot[1];
        d.scal[C_TOL2] = tol2;
        d.flag[F_CDONE] = (tot[1] == 0.0 || !isfinite(tot[1])) ? 1 : 0;
        d.flag[F_CIT] = 0;
    }
}

__global__ void k_cg_pq(Dev d, const double *p, const double *q, int64_t n)
{
    if (d.flag[F_CDONE]) return;
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(i, n) v[0] += p[i] * q[i];
    if (grid_sum<1>(d, v, tot)) {
        double pq = tot[0];
        if (!(pq > 0.0) || !isfinite(pq)) {
            d.flag[F_CDONE] = 1;  // stop on breakdown; x keeps the last iterate
            d.scal[C_ALPHA] = 0.0;
        } else {
            d.scal[C_ALPHA] = d.scal[C_RZ] / pq;
        }
    }
}

// x += alpha p; r -= alpha q; rr = (r, r); rzn = (r, Dinv r); beta = rzn / rz
__global__ void k_cg_update(Dev d, double *x, double *r, const double *p, const double *q, const double *dinv,
                            int64_t n)
{
    if (d.flag[F_CDONE]) return;
    const double alpha = d.scal[C_ALPHA];
    double v[2] = {0.0, 0.0}, tot[2];
    GRID_STRIDE(i, n)
    {
        x[i] += alpha * p[i];
        double ri = r[i] - alpha * q[i];
        r[i] = ri;
        v[0] += ri * ri;
        v[1] += ri * dinv[i] * ri;
    }
    if (grid_sum<2>(d, v, tot)) {
        d.scal[C_RR] = tot[0];
        d.scal[C_BETA] = tot[1] / d.scal[C_RZ];
        d.scal[C_RZ] = tot[1];
        if (tot[0] <= d.scal[C_TOL2] * d.scal[C_BB] || !isfinite(tot[0])) d.flag[F_CDONE] = 1;
    }
}

__global__ void k_cg_p(Dev d, double *p, const double *r, const double *dinv, int64_t n)
{
    if (d.flag[F_CDONE]) return;
    const double beta = d.scal[C_BETA];
    GRID_STRIDE(i, n) p[i] = dinv[i] * r[i] + beta * p[i];
}

// ------------------------------------------------ assembled coarse matrix
// The coarsest level (p = 1) is assembled once, as the coarse level of the
// paper's hierarchy is (Sec. 3.2), into a 27-point nodal stencil: row (c, i),
// column (d, i + offset) with offset in {-1,0,1}^3.  Values are stored as 81
// planes of N (plane s*3 + d, s the stencil index) so that consecutive rows
// read consecutive addresses.  Each entry sums the element-matrix entries of
// the (at most 8) elements holding both nodes, in increasing element order.
struct P1Tables {
    double M[2][2], C[2][2], K[2][2];  // sum_q w B_i B_j, w G_i B_j, w G_i G_j
};

__global__ void k_assemble_p1(const double *__restrict__ geo, double *__restrict__ vals, P1Tables t, Grid g)
{
    const int64_t Nn = g.Nn, nrow = 3 * Nn;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < nrow;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(row / Nn);
        const int64_t i = row - c * Nn;
        const int ix = (int)(i % g.Mx), iy = (int)((i / g.Mx) % g.My), iz = (int)(i / ((int64_t)g.Mx * g.My));
        double acc[81];
        for (int k = 0; k < 81; ++k) acc[k] = 0.0;
        for (int ez = iz - 1; ez <= iz; ++ez)
            for (int ey = iy - 1; ey <= iy; ++ey)
                for (int ex = ix - 1; ex <= ix; ++ex) {
                    if (ex < 0 || ey < 0 || ez < 0 || ex >= g.nx || ey >= g.ny || ez >= g.nz) continue;
                    const int64_t e = ex + (int64_t)g.nx * (ey + (int64_t)g.ny * ez);
                    const double *gp = geo + e * kGeoStride;
                    const double cl = gp[9], cm = gp[10];
                    double Ji[9];
                    for (int k = 0; k < 9; ++k) Ji[k] = gp[k];
                    // C[m][n][d] = lambda detJ Ji[m][c] Ji[n][d] + mu detJ Ji[m][d] Ji[n][c]
                    //              + mu detJ delta_cd (Ji Ji^T)[m][n]
                    double Cmn[3][3][3];
                    for (int m = 0; m < 3; ++m)
                        for (int n = 0; n < 3; ++n) {
                            double jj = Ji[m * 3] * Ji[n * 3] + Ji[m * 3 + 1] * Ji[n * 3 + 1] + Ji[m * 3 + 2] * Ji[n * 3 + 2];
                            for (int d = 0; d < 3; ++d)
                                Cmn[m][n][d] = cl * Ji[m * 3 + c] * Ji[n * 3 + d] + cm * Ji[m * 3 + d] * Ji[n * 3 + c] +
                                               (c == d ? cm * jj : 0.0);
                        }
                    const int a[3] = {ix - ex, iy - ey, iz - ez};
                    for (int bz = 0; bz < 2; ++bz)
                        for (int by = 0; by < 2; ++by)
                            for (int bx = 0; bx < 2; ++bx) {
                                const int b[3] = {bx, by, bz};
                                double S[3][3];
                                for (int m = 0; m < 3; ++m)
                                    for (int n = 0; n < 3; ++n) {
                                        double v = 1.0;
                                        for (int k = 0; k < 3; ++k) {
                                            const int ak = a[k], bk = b[k];
                                            v *= (k == m && k == n) ? t.K[ak][bk]
                                                 : (k == m)         ? t.C[ak][bk]
                                                 : (k == n)         ? t.C[bk][ak]
                                                                    : t.M[ak][bk];
                                        }
                                        S[m][n] = v;
                                    }
                                const int sidx = (ex + bx - ix + 1) + 3 * (ey + by - iy + 1) + 9 * (ez + bz - iz + 1);
                                for (int d = 0; d < 3; ++d) {
                                    double v = 0.0;
                                    for (int m = 0; m < 3; ++m)
                                        for (int n = 0; n < 3; ++n) v += S[m][n] * Cmn[m][n][d];
                                    acc[sidx * 3 + d] += v;
                                }
                            }
                }
        for (int k = 0; k < 81; ++k) vals[(int64_t)k * nrow + row] = acc[k];
    }
}

// Row of y = A p on an assembled stencil level whose planes are masked
// (k_mask_stencil): essential rows are identity rows, couplings to essential
// dofs and to neighbours outside the grid are zero.  The row is then a
// branch-free sum of 81 terms; a neighbour outside the grid is read at the
// row's own node (its coefficient is 0), so all loads are independent and in
// flight together.  One partial sum per column component.
__device__ inline double stencil_row(const double *__restrict__ vals, const double *__restrict__ p, const Grid &g,
                                     int64_t row)
{
    const int Nn = (int)g.Nn, Mx = g.Mx, My = g.My, Mz = g.Mz;
    const int64_t nrow = 3 * (int64_t)Nn;
    const int c = (int)(row / Nn);
    const int i = (int)(row - (int64_t)c * Nn);
    const int ix = i % Mx, t = i / Mx, iy = t % My, iz = t / My;
    const int ox[3] = {ix > 0 ? -1 : 0, 0, ix < Mx - 1 ? 1 : 0};
    const int oy[3] = {iy > 0 ? -Mx : 0, 0, iy < My - 1 ? Mx : 0};
    const int oz[3] = {iz > 0 ? -Mx * My : 0, 0, iz < Mz - 1 ? Mx * My : 0};
    double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int sz = 0; sz < 3; ++sz)
#pragma unroll
        for (int sy = 0; sy < 3; ++sy)
#pragma unroll
            for (int sx = 0; sx < 3; ++sx) {
                const int sidx = sx + 3 * sy + 9 * sz;
                const int j = i + ox[sx] + oy[sy] + oz[sz];
#pragma unroll
                for (int d2 = 0; d2 < 3; ++d2)
                    acc[d2] = fma(vals[(int64_t)(sidx * 3 + d2) * nrow + row], p[(int64_t)d2 * Nn + j], acc[d2]);
            }
    return (acc[0] + acc[1]) + acc[2];
}

// Three lanes per stencil row: lanes 3r, 3r + 1, 3r + 2 of a warp take row
// base + r (r = 0..9; lanes 30, 31 idle), lane d2 summing the 27 products
// with the neighbours' component d2 in stencil_row's order, and the row's
// first lane adding the three sums as stencil_row does (same bits).  On a
// small level one thread per row leaves most SMs idle while each active SM
// works through 81 FP64 products per thread; three lanes spread them over
// three times the SMs.
__device__ inline double stencil_part(const double *__restrict__ vals, const double *__restrict__ p, const Grid &g,
                                      int64_t row, int d2)
{
    const int Nn = (int)g.Nn, Mx = g.Mx, My = g.My, Mz = g.Mz;
    const int64_t nrow = 3 * (int64_t)Nn;
    const int c = (int)(row / Nn);
    const int i = (int)(row - (int64_t)c * Nn);
    const int ix = i % Mx, t = i / Mx, iy = t % My, iz = t / My;
    const int ox[3] = {ix > 0 ? -1 : 0, 0, ix < Mx - 1 ? 1 : 0};
    const int oy[3] = {iy > 0 ? -Mx : 0, 0, iy < My - 1 ? Mx : 0};
    const int oz[3] = {iz > 0 ? -Mx * My : 0, 0, iz < Mz - 1 ? Mx * My : 0};
    const double *pd = p + (int64_t)d2 * Nn;
    double acc = 0.0;
#pragma unroll
    for (int sz = 0; sz < 3; ++sz)
#pragma unroll
        for (int sy = 0; sy < 3; ++sy)
#pragma unroll
            for (int sx = 0; sx < 3; ++sx) {
                const int sidx = sx + 3 * sy + 9 * sz;
                acc = fma(vals[(int64_t)(sidx * 3 + d2) * nrow + row], pd[i + ox[sx] + oy[sy] + oz[sz]], acc);
            }
    return acc;
}

// The row sum on the row's first lane (all 32 lanes must call it together).
__device__ inline double stencil_row3(const double *__restrict__ vals, const double *__restrict__ p, const Grid &g,
                                      int64_t row, int d2, bool valid)
{
    const double part = valid ? stencil_part(vals, p, g, row, d2) : 0.0;
    const double p1 = __shfl_down_sync(0xffffffffu, part, 1);
    const double p2 = __shfl_down_sync(0xffffffffu, part, 2);
    return (part + p1) + p2;
}

// Warp-strided loop over groups of ten rows: row, d2 and valid (the lane
// has a row and the row exists) for each lane; the loop bounds are uniform
// over the warp, so the shuffles see every lane.
#define ROW3_LOOP(nrow_expr, BODY)                                                                       \
    {                                                                                                    \
        const int64_t nrow_ = (nrow_expr);                                                               \
        const int lane_ = threadIdx.x & 31, r_ = lane_ / 3, d2 = lane_ - 3 * r_;                        \
        const int64_t w0_ = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;                     \
        const int64_t nw_ = ((int64_t)gridDim.x * blockDim.x) >> 5;                                      \
        for (int64_t base_ = w0_ * 10; base_ < nrow_; base_ += nw_ * 10) {                               \
            const int64_t row = base_ + r_;                                                              \
            const bool valid = lane_ < 30 && row < nrow_;                                                \
            BODY                                                                                         \
        }                                                                                                \
    }

// CTAs of 128 threads (4 warps, 40 rows) for a three-lanes-per-row kernel
unsigned row3_blocks(int64_t nrow, int64_t cap = 152 * 16)
{
    int64_t b = ((nrow + 9) / 10 + 3) / 4;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// Masks an assembled stencil level in place for stencil_row: zero
// coefficients towards neighbours outside the grid and towards essential
// dofs, identity rows on essential dofs.  The Galerkin products and the dense
// coarsest matrix leave essential rows and columns out, so they read the
// same values from masked planes.
__global__ void k_mask_stencil(double *__restrict__ vals, const uint8_t *__restrict__ ess, Grid g)
{
    const int64_t Nn = g.Nn, nrow = 3 * Nn;
    GRID_STRIDE(row, nrow)
    {
        const int c = (int)(row / Nn);
        const int64_t i = row - c * Nn;
        const int ix = (int)(i % g.Mx), iy = (int)((i / g.Mx) % g.My), iz = (int)(i / ((int64_t)g.Mx * g.My));
        const bool erow = ess && ess[row];
        for (int sidx = 0; sidx < 27; ++sidx) {
            const int dx = sidx % 3 - 1, dy = (sidx / 3) % 3 - 1, dz = sidx / 9 - 1;
            const bool inside = ix + dx >= 0 && ix + dx < g.Mx && iy + dy >= 0 && iy + dy < g.My && iz + dz >= 0 &&
                                iz + dz < g.Mz;
            const int64_t j = i + dx + (int64_t)g.Mx * (dy + (int64_t)g.My * dz);
            for (int d2 = 0; d2 < 3; ++d2) {
                double &v = vals[(int64_t)(sidx * 3 + d2) * nrow + row];
                if (!inside) v = 0.0;
                else if (erow) v = (sidx == 13 && d2 == c) ? 1.0 : 0.0;
                else if (ess && ess[d2 * Nn + j]) v = 0.0;
            }
        }
    }
}

// q = A p with the assembled stencil (constrained rows/columns as the
// operator: essential columns read as 0, essential rows return p), fused with
// pq = (p, q) and alpha = rz / pq.
__global__ void k_cg_spmv_pq(Dev d, const double *__restrict__ vals, const double *__restrict__ p,
                             double *__restrict__ q, Grid g)
{
    if (d.flag[F_CDONE]) return;
    double v[1] = {0.0}, tot[1];
    ROW3_LOOP(3 * g.Nn, {
        const double y = stencil_row3(vals, p, g, row, d2, valid);
        if (valid && d2 == 0) {
            q[row] = y;
            v[0] += p[row] * y;
        }
    })
    if (grid_sum<1>(d, v, tot)) {
        double pq = tot[0];
        if (!(pq > 0.0) || !isfinite(pq)) {
            d.flag[F_CDONE] = 1;
            d.scal[C_ALPHA] = 0.0;
        } else {
            d.scal[C_ALPHA] = d.scal[C_RZ] / pq;
        }
    }
}

// ------------------------------------------------- persistent coarse CG
// The whole Jacobi-CG of the assembled coarse level in one cooperative
// launch (all CTAs co-resident): three grid barriers per iteration replace
// four kernel launches.  Every CTA adds the per-CTA partial sums itself in
// the same fixed order, so all CTAs take the same decisions and the result
// is deterministic.  The barrier's spin is bounded by time; on expiry the
// kernel raises F_CTIMEOUT and returns.  The bound is the solver's wait
// budget (PA_SOLVER_OPT_WAIT_LIMIT, 2 s by default) in SM clock cycles.
enum { F_CTIMEOUT = 3 };

__device__ inline bool grid_barrier(unsigned *bar, int *timeout_flag, long long limit_cycles)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (clock64() - t0 > limit_cycles || *(volatile int *)timeout_flag) {
                    atomicExch(timeout_flag, 1);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Sum over CTAs of K per-CTA partials (same order in every CTA); all threads
// receive the totals.
template <int K>
__device__ inline void all_sum(const double *part, double (&tot)[K])
{
    __shared__ double res[K];
    double w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double acc = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) acc += ((volatile const double *)part)[k * kRedBlocks + b];
        w[k] = acc;
    }
    block_sum<K>(w);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) res[k] = w[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) tot[k] = res[k];
    __syncthreads();
}

template <int K>
__device__ inline void publish(double *part, double (&v)[K])
{
    block_sum<K>(v);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) part[k * kRedBlocks + blockIdx.x] = v[k];
}

__global__ void __launch_bounds__(256) k_cg_coop(Dev d, const double *__restrict__ vals, double *__restrict__ x,
                                                 double *__restrict__ r, double *__restrict__ p, double *__restrict__ q,
                                                 const double *__restrict__ dinv, const double *__restrict__ b,
                                                 const uint8_t *__restrict__ ess, Grid g, double tol2, int maxit,
                                                 unsigned *bar, double *part, long long wait_cycles)
{
    const int64_t n = 3 * g.Nn;
    double *pA = part, *pB = part + 3 * kRedBlocks, *pC = part + 6 * kRedBlocks;
    int *tflag = d.flag + F_CTIMEOUT;
    // start: x = 0, r = b, p = Dinv b
    double v2[2] = {0.0, 0.0}, t2[2];
    GRID_STRIDE(i, n)
    {
        const double bi = b[i], zi = dinv[i] * bi;
        x[i] = 0.0;
        r[i] = bi;
        p[i] = zi;
        v2[0] += bi * zi;
        v2[1] += bi * bi;
    }
    publish<2>(pC, v2);
    if (!grid_barrier(bar, tflag, wait_cycles)) return;
    all_sum<2>(pC, t2);
    double rz = t2[0];
    const double bb = t2[1];
    double rr = bb;
    int it = 0;
    bool stop = !(bb > 0.0) || !isfinite(bb);
    while (!stop && it < maxit) {
        double v1[1] = {0.0}, t1[1];
        GRID_STRIDE(row, n)
        {
            const double y = stencil_row(vals, p, g, row);
            q[row] = y;
            v1[0] += p[row] * y;
        }
        publish<1>(pA, v1);
        if (!grid_barrier(bar, tflag, wait_cycles)) return;
        all_sum<1>(pA, t1);
        const double pq = t1[0];
        if (!(pq > 0.0) || !isfinite(pq)) break;
        const double alpha = rz / pq;
        v2[0] = v2[1] = 0.0;
        GRID_STRIDE(i, n)
        {
            x[i] += alpha * p[i];
            const double ri = r[i] - alpha * q[i];
            r[i] = ri;
            v2[0] += ri * ri;
            v2[1] += ri * dinv[i] * ri;
        }
        publish<2>(pB, v2);
        if (!grid_barrier(bar, tflag, wait_cycles)) return;
        all_sum<2>(pB, t2);
        rr = t2[0];
        const double beta = t2[1] / rz;
        rz = t2[1];
        ++it;
        if (rr <= tol2 * bb || !isfinite(rr)) break;
        GRID_STRIDE(i, n) p[i] = dinv[i] * r[i] + beta * p[i];
        if (!grid_barrier(bar, tflag, wait_cycles)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d.scal[C_RR] = rr;
        d.scal[C_BB] = bb;
        d.flag[F_CIT] = it;
    }
}


// ------------------------------------------------------ h-multigrid (p = 1)
// Geometric coarsening of the assembled p = 1 level below the p-hierarchy
// (the paper's hierarchy has h-levels at p = 1 under its p-levels, Sec. 3).
// Along an axis with M fine nodes the coarse nodes sit at the even fine
// indices and at the last node: Mc = (M + 1) / 2 for odd M, M / 2 + 1 for
// even M.  Prolongation is linear interpolation between coarse nodes (per
// component); restriction is its exact transpose; coarse operators are the
// Galerkin products P^T A P in the same 27-point stencil form.
__host__ __device__ inline int h_coarse_size(int M) { return (M & 1) ? (M + 1) / 2 : M / 2 + 1; }

__host__ __device__ inline int h_pos(int J, int Mf, int Mc) { return (J == Mc - 1) ? Mf - 1 : 2 * J; }

// coarse parents of fine index i along one axis: 1 or 2 (index, weight)
__host__ __device__ inline int h_parents(int i, int Mf, int Mc, int *J, double *w)
{
    if (i == Mf - 1) {
        J[0] = Mc - 1;
        w[0] = 1.0;
        return 1;
    }
    if ((i & 1) == 0) {
        J[0] = i / 2;
        w[0] = 1.0;
        return 1;
    }
    J[0] = (i - 1) / 2;
    w[0] = 0.5;
    J[1] = (i + 1) / 2;
    w[1] = 0.5;
    return 2;
}

// weight of coarse index J in the interpolation of fine index i (0 if none)
__host__ __device__ inline double h_weight(int i, int J, int Mf, int Mc)
{
    int Jp[2];
    double w[2];
    const int n = h_parents(i, Mf, Mc, Jp, w);
    for (int k = 0; k < n; ++k)
        if (Jp[k] == J) return w[k];
    return 0.0;
}

// y = A x on an assembled stencil level (constrained like the operator)
__global__ void k_stencil_apply(const double *__restrict__ vals, const double *__restrict__ x, double *__restrict__ y,
                                Grid g)
{
    ROW3_LOOP(3 * g.Nn, {
        const double v = stencil_row3(vals, x, g, row, d2, valid);
        if (valid && d2 == 0) y[row] = v;
    })
}

// One Chebyshev step on a stencil level fused with its operator apply:
// d = cd d + cr Dinv (r - A e_in); e_out = e_in + d (e_in and e_out distinct)
__global__ void k_stencil_cheb(const double *__restrict__ vals, const double *__restrict__ ein,
                               double *__restrict__ eout, double *__restrict__ dv, const double *__restrict__ r,
                               const double *__restrict__ dinv, double cd, double cr, Grid g)
{
    ROW3_LOOP(3 * g.Nn, {
        const double ae = stencil_row3(vals, ein, g, row, d2, valid);
        if (valid && d2 == 0) {
            const double rk = r[row] - ae;
            const double di = (cd != 0.0 ? cd * dv[row] : 0.0) + cr * dinv[row] * rk;
            dv[row] = di;
            eout[row] = ein[row] + di;
        }
    })
}

// h-prolongation (natural injection of the trilinear space, Sec. 3) in one
// pass: ef += P ec, each fine dof gathering its (at most 8) coarse parents,
// summed x inside y inside z.
template <typename T>
__device__ inline T hprolong_val(const T *__restrict__ ec, const Grid &gf, const Grid &gc, int64_t o)
{
    const int64_t Nnf = gf.Nn, Nnc = gc.Nn;
    {
        const int c = (int)(o / Nnf);
        const int64_t i = o - c * Nnf;
        const int fx = (int)(i % gf.Mx), fy = (int)((i / gf.Mx) % gf.My), fz = (int)(i / ((int64_t)gf.Mx * gf.My));
        int Jx[2], Jy[2], Jz[2];
        double wx[2], wy[2], wz[2];
        const int nx = h_parents(fx, gf.Mx, gc.Mx, Jx, wx), ny = h_parents(fy, gf.My, gc.My, Jy, wy),
                  nz = h_parents(fz, gf.Mz, gc.Mz, Jz, wz);
        T sz = 0;
        for (int kz = 0; kz < nz; ++kz) {
            T sy = 0;
            for (int ky = 0; ky < ny; ++ky) {
                const T *row = ec + c * Nnc + (int64_t)gc.Mx * (Jy[ky] + (int64_t)gc.My * Jz[kz]);
                T sx = 0;
                for (int kx = 0; kx < nx; ++kx) sx += (T)wx[kx] * row[Jx[kx]];
                sy += (T)wy[ky] * sx;
            }
            sz += (T)wz[kz] * sy;
        }
        return sz;
    }
}

template <typename T>
__global__ void k_hprolong_add(T *__restrict__ ef, const T *__restrict__ ec, Grid gf, Grid gc)
{
    GRID_STRIDE(o, 3 * gf.Nn) ef[o] = ef[o] + hprolong_val(ec, gf, gc, o);
}

// h-restriction out = R (in - in2) (in2 may be null): each coarse dof
// gathers its fine children (at most 3 per axis) with the transposed
// weights, summed x inside y inside z.  One z-plane (iz = pz - 1 + k): the
// plane's weight (0 when the plane is outside the grid or has no weight)
// and its y/x sum.
template <typename T>
__device__ inline T hrestrict_plane(const T *__restrict__ in, const T *__restrict__ in2, const Grid &gf,
                                    const Grid &gc, int64_t o, int k, T &wz)
{
    const int64_t Nnf = gf.Nn, Nnc = gc.Nn;
    const int c = (int)(o / Nnc);
    const int64_t I = o - c * Nnc;
    const int Jx = (int)(I % gc.Mx), Jy = (int)((I / gc.Mx) % gc.My), Jz = (int)(I / ((int64_t)gc.Mx * gc.My));
    const int px = h_pos(Jx, gf.Mx, gc.Mx), py = h_pos(Jy, gf.My, gc.My), iz = h_pos(Jz, gf.Mz, gc.Mz) - 1 + k;
    wz = (iz < 0 || iz >= gf.Mz) ? (T)0 : (T)h_weight(iz, Jz, gf.Mz, gc.Mz);
    T sy = 0;
    if (wz == (T)0) return sy;
    for (int iy = py - 1; iy <= py + 1; ++iy) {
        if (iy < 0 || iy >= gf.My) continue;
        const T wy = (T)h_weight(iy, Jy, gf.My, gc.My);
        if (wy == (T)0) continue;
        const int64_t base = c * Nnf + (int64_t)gf.Mx * (iy + (int64_t)gf.My * iz);
        T sx = 0;
        for (int ix = px - 1; ix <= px + 1; ++ix) {
            if (ix < 0 || ix >= gf.Mx) continue;
            const T wx = (T)h_weight(ix, Jx, gf.Mx, gc.Mx);
            if (wx == (T)0) continue;
            sx += wx * (in2 ? in[base + ix] - in2[base + ix] : in[base + ix]);
        }
        sy += wy * sx;
    }
    return sy;
}

// The three z-planes on three lanes (ROW3_LOOP's lane layout); the row's
// first lane adds them in plane order.  All 32 lanes must call it together.
template <typename T>
__device__ inline T hrestrict_val3(const T *__restrict__ in, const T *__restrict__ in2, const Grid &gf, const Grid &gc,
                                   int64_t o, int k, bool valid)
{
    T wz = 0;
    const T sy = valid ? hrestrict_plane(in, in2, gf, gc, o, k, wz) : (T)0;
    const T w1 = __shfl_down_sync(0xffffffffu, wz, 1), s1 = __shfl_down_sync(0xffffffffu, sy, 1);
    const T w2 = __shfl_down_sync(0xffffffffu, wz, 2), s2 = __shfl_down_sync(0xffffffffu, sy, 2);
    T sz = 0;
    if (wz != (T)0) sz += wz * sy;
    if (w1 != (T)0) sz += w1 * s1;
    if (w2 != (T)0) sz += w2 * s2;
    return sz;
}

// First Chebyshev step from a zero iterate of an h-level, taken by the
// kernel that produces the level's right-hand side: e = d = cr Dinv r
// (the step needs no operator apply, so it costs no dependent stage).
struct FirstStep {
    double *e = nullptr, *d = nullptr;  // null: no fused step
    const double *dinv = nullptr;
    double cr = 0.0;
};

__device__ inline void first_step(const FirstStep &f, int64_t i, double r)
{
    if (f.e) {
        const double di = 0.0 + f.cr * f.dinv[i] * r;
        f.d[i] = di;
        f.e[i] = di;
    }
}

// (three lanes per coarse dof, row3_blocks CTAs of 128 threads)
template <typename T>
__global__ void k_hrestrict(T *__restrict__ out, const T *__restrict__ in, const T *__restrict__ in2, Grid gf, Grid gc,
                            const uint8_t *__restrict__ ess)
{
    ROW3_LOOP(3 * gc.Nn, {
        const T v = hrestrict_val3(in, in2, gf, gc, row, d2, valid);
        if (valid && d2 == 0) out[row] = (ess && ess[row]) ? (T)0 : v;
    })
}

// The same restriction followed by the coarse level's first Chebyshev step
// from a zero iterate (e = d = cr Dinv r), which needs no operator apply.
__global__ void k_hrestrict_first(double *__restrict__ out, const double *__restrict__ in,
                                  const double *__restrict__ in2, Grid gf, Grid gc, const uint8_t *__restrict__ ess,
                                  FirstStep f)
{
    ROW3_LOOP(3 * gc.Nn, {
        const double r3 = hrestrict_val3(in, in2, gf, gc, row, d2, valid);
        if (valid && d2 == 0) {
            const double v = (ess && ess[row]) ? 0.0 : r3;
            out[row] = v;
            first_step(f, row, v);
        }
    })
}

// Galerkin coarse stencil: one thread per coarse row (c, I); essential fine
// rows and columns are left out of the product (the constrained operator).
__global__ void k_rap_stencil(const double *__restrict__ fv, const uint8_t *__restrict__ fess, Grid gf,
                              double *__restrict__ cv, Grid gc)
{
    const int64_t nrow_c = 3 * gc.Nn, nrow_f = 3 * gf.Nn;
    GRID_STRIDE(row, nrow_c)
    {
        const int c = (int)(row / gc.Nn);
        const int64_t I = row - c * gc.Nn;
        const int Ic[3] = {(int)(I % gc.Mx), (int)((I / gc.Mx) % gc.My), (int)(I / ((int64_t)gc.Mx * gc.My))};
        const int Mf[3] = {gf.Mx, gf.My, gf.Mz}, Mc[3] = {gc.Mx, gc.My, gc.Mz};
        double acc[81];
        for (int k = 0; k < 81; ++k) acc[k] = 0.0;
        int pos[3];
        for (int a = 0; a < 3; ++a) pos[a] = h_pos(Ic[a], Mf[a], Mc[a]);
        for (int iz = pos[2] - 1; iz <= pos[2] + 1; ++iz) {
            if (iz < 0 || iz >= Mf[2]) continue;
            const double wz = h_weight(iz, Ic[2], Mf[2], Mc[2]);
            if (wz == 0.0) continue;
            for (int iy = pos[1] - 1; iy <= pos[1] + 1; ++iy) {
                if (iy < 0 || iy >= Mf[1]) continue;
                const double wy = h_weight(iy, Ic[1], Mf[1], Mc[1]);
                if (wy == 0.0) continue;
                for (int ix = pos[0] - 1; ix <= pos[0] + 1; ++ix) {
                    if (ix < 0 || ix >= Mf[0]) continue;
                    const double wx = h_weight(ix, Ic[0], Mf[0], Mc[0]);
                    if (wx == 0.0) continue;
                    const double wi = wx * wy * wz;
                    const int64_t i = ix + (int64_t)gf.Mx * (iy + (int64_t)gf.My * iz);
                    const int64_t frow = c * gf.Nn + i;
                    if (fess && fess[frow]) continue;
                    for (int dz = -1; dz <= 1; ++dz) {
                        const int jz = iz + dz;
                        if (jz < 0 || jz >= Mf[2]) continue;
                        int Jz[2];
                        double wjz[2];
                        const int nz2 = h_parents(jz, Mf[2], Mc[2], Jz, wjz);
                        for (int dy = -1; dy <= 1; ++dy) {
                            const int jy = iy + dy;
                            if (jy < 0 || jy >= Mf[1]) continue;
                            int Jy[2];
                            double wjy[2];
                            const int ny2 = h_parents(jy, Mf[1], Mc[1], Jy, wjy);
                            for (int dx = -1; dx <= 1; ++dx) {
                                const int jx = ix + dx;
                                if (jx < 0 || jx >= Mf[0]) continue;
                                int Jx[2];
                                double wjx[2];
                                const int nx2 = h_parents(jx, Mf[0], Mc[0], Jx, wjx);
                                const int fs = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                                const int64_t j = jx + (int64_t)gf.Mx * (jy + (int64_t)gf.My * jz);
                                for (int d = 0; d < 3; ++d) {
                                    if (fess && fess[d * gf.Nn + j]) continue;
                                    const double a = wi * fv[(int64_t)(fs * 3 + d) * nrow_f + frow];
                                    if (a == 0.0) continue;
                                    for (int kz = 0; kz < nz2; ++kz)
                                        for (int ky = 0; ky < ny2; ++ky)
                                            for (int kx = 0; kx < nx2; ++kx) {
                                                const int cs = (Jx[kx] - Ic[0] + 1) + 3 * (Jy[ky] - Ic[1] + 1) +
                                                               9 * (Jz[kz] - Ic[2] + 1);
                                                acc[cs * 3 + d] += a * wjx[kx] * wjy[ky] * wjz[kz];
                                            }
                                }
                            }
                        }
                    }
                }
            }
        }
        for (int k = 0; k < 81; ++k) cv[(int64_t)k * nrow_c + row] = acc[k];
    }
}

// y = Ainv x with a dense (coarsest-level) inverse, one thread per row
// y = Ainv x (dense, n <= 1280): one warp per row, lane-strided partial
// sums combined by a fixed butterfly.
__global__ void k_dense_matvec(const double *__restrict__ Ainv, const double *__restrict__ x, double *__restrict__ y,
                               int64_t n)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarp) {
        const double *row = Ainv + i * n;
        double s2 = 0.0;
        for (int64_t j = lane; j < n; j += 32) s2 = fma(row[j], x[j], s2);
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) y[i] = s2;
    }
}

// preconditioned coarse CG (z = M r from the h-cycle)
// start 1: x = 0, r = b, bb = (b, b), done = bb == 0
__global__ void k_pcg_start1(Dev d, double *x, double *r, const double *b, int64_t n, double tol2, FirstStep f)
{
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(i, n)
    {
        const double bi = b[i];
        x[i] = 0.0;
        r[i] = bi;
        v[0] += bi * bi;
        first_step(f, i, bi);
    }
    if (grid_sum<1>(d, v, tot)) {
        d.scal[C_BB] = tot[0];
        d.scal[C_RR] = tot[0];
        d.scal[C_TOL2] = tol2;
        d.scal[C_RZ] = 0.0;  // no previous direction: the first one is z
        d.flag[F_CDONE] = (tot[0] == 0.0 || !isfinite(tot[0])) ? 1 : 0;
        d.flag[F_CIT] = 0;
    }
}

// x += alpha p; r -= alpha q; rr = (r, r); done when rr <= tol2 bb
__global__ void k_pcg_update(Dev d, double *x, double *r, const double *p, const double *q, int64_t n, FirstStep f)
{
    if (d.flag[F_CDONE]) return;
    const double alpha = d.scal[C_ALPHA];
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(i, n)
    {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        v[0] += ri * ri;
        first_step(f, i, ri);
    }
    if (grid_sum<1>(d, v, tot)) {
        d.scal[C_RR] = tot[0];
        if (tot[0] <= d.scal[C_TOL2] * d.scal[C_BB] || !isfinite(tot[0])) d.flag[F_CDONE] = 1;
    }
}

// rz_new = (r, z); beta = rz_new / rz (0 when there is no previous
// direction, rz = 0); rz = rz_new
__global__ void k_pcg_beta(Dev d, const double *r, const double *z, int64_t n)
{
    if (d.flag[F_CDONE]) return;
    double v[1] = {0.0}, tot[1];
    GRID_STRIDE(i, n) v[0] += r[i] * z[i];
    if (grid_sum<1>(d, v, tot)) {
        const double rz = d.scal[C_RZ];
        d.scal[C_BETA] = rz != 0.0 ? tot[0] / rz : 0.0;
        d.scal[C_RZ] = tot[0];
    }
}

// p = z + beta p (p = z when beta = 0: the old p is not read)
__global__ void k_pcg_p(Dev d, double *p, const double *z, int64_t n)
{
    if (d.flag[F_CDONE]) return;
    const double beta = d.scal[C_BETA];
    GRID_STRIDE(i, n) p[i] = beta != 0.0 ? z[i] + beta * p[i] : z[i];
}

// Loop condition of the graph's coarse WHILE node: continue while the coarse
// CG has not stopped and the iteration cap is not reached.
__global__ void k_cg_cond(Dev d, int maxit, cudaGraphConditionalHandle h)
{
    if (threadIdx.x == 0) {
        int it = ++d.flag[F_CIT];
        cudaGraphSetConditional(h, (!d.flag[F_CDONE] && it < maxit) ? 1u : 0u);
    }
}

// ------------------------------------------------------------ smoothing
// Chebyshev step: rk = r - t (t may be null: rk = r);
// d = cd d + cr Dinv rk; e = d (first step from a zero guess) or e += d.
template <typename T>
__global__ void k_cheb(T *e, T *dv, const T *r, const T *t, const T *dinv, double cd, double cr, int first_zero,
                       int64_t n)
{
    const T cdt = (T)cd, crt = (T)cr;
    GRID_STRIDE(i, n)
    {
        const T rk = t ? r[i] - t[i] : r[i];
        const T di = (cd != 0.0 ? cdt * dv[i] : T(0)) + crt * dinv[i] * rk;
        dv[i] = di;
        e[i] = first_zero ? di : e[i] + di;
    }
}

template <typename T>
__global__ void k_recip(T *dinv, const T *dg, int64_t n)
{
    GRID_STRIDE(i, n) dinv[i] = (T)(1.0 / dd(dg[i]));
}

// deterministic pseudo-random start vector (splitmix64 of the index), zero on
// essential dofs
__global__ void k_random(double *v, const uint8_t *ess, int64_t n, uint64_t seed)
{
    GRID_STRIDE(i, n)
    {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        double u = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        v[i] = (ess && ess[i]) ? 0.0 : u;
    }
}

// ------------------------------------------------------------- transfers
// One axis of the global tensor-product interpolation between the degree-pc
// and degree-pf GLL spaces on the same n-element axis.  Arrays are
// [3][Nz][Ny][Nx]; `ax` is the axis being changed (0 = x, 1 = y, 2 = z).
// L[a*(pf+1) + j] = coarse basis a at fine node j (1D).
struct XferTab {
    double L[kMaxD * kMaxD];
};

template <typename T>
__global__ void k_prolong_axis(T *out, const T *in, int ax, int Nx, int Ny, int Nz, int n, int pc, int pf,
                               XferTab tab, int accumulate)
{
    // out dims: axis `ax` fine (n pf + 1), others as given (already in their final size)
    const int Mf = n * pf + 1, Mc = n * pc + 1;
    int dims[3] = {Nx, Ny, Nz};
    dims[ax] = Mf;
    int64_t total = 3LL * dims[0] * dims[1] * dims[2];
    GRID_STRIDE(o, total)
    {
        int64_t t = o;
        int i0 = (int)(t % dims[0]); t /= dims[0];
        int i1 = (int)(t % dims[1]); t /= dims[1];
        int i2 = (int)(t % dims[2]);
        int c = (int)(t / dims[2]);
        int idx[3] = {i0, i1, i2};
        int i = idx[ax];
        int k = i / pf;
        if (k > n - 1) k = n - 1;
        int jl = i - k * pf;
        int cdims[3] = {dims[0], dims[1], dims[2]};
        cdims[ax] = Mc;
        T s = T(0);
        for (int a = 0; a <= pc; ++a) {
            const double w = tab.L[a * (pf + 1) + jl];
            if (w == 0.0) continue;
            idx[ax] = k * pc + a;
            int64_t ci = (((int64_t)c * cdims[2] + idx[2]) * cdims[1] + idx[1]) * cdims[0] + idx[0];
            s += (T)w * in[ci];
        }
        out[o] = accumulate ? out[o] + s : s;
    }
}

// Exact transpose of k_prolong_axis along one axis.  in2 (optional) is
// subtracted from in on the fly; ess (optional, on the output L-vector) zeroes
// essential entries.
template <typename T>
__global__ void k_restrict_axis(T *out, const T *in, const T *in2, int ax, int Nx, int Ny, int Nz, int n, int pc,
                                int pf, XferTab tab, const uint8_t *ess)
{
    const int Mf = n * pf + 1, Mc = n * pc + 1;
    int dims[3] = {Nx, Ny, Nz};  // input dims (axis `ax` fine)
    int odims[3] = {Nx, Ny, Nz};
    dims[ax] = Mf;
    odims[ax] = Mc;
    int64_t total = 3LL * odims[0] * odims[1] * odims[2];
    GRID_STRIDE(o, total)
    {
        int64_t t = o;
        int i0 = (int)(t % odims[0]); t /= odims[0];
        int i1 = (int)(t % odims[1]); t /= odims[1];
        int i2 = (int)(t % odims[2]);
        int c = (int)(t / odims[2]);
        int idx[3] = {i0, i1, i2};
        int jc = idx[ax];
        T s = T(0);
        int kk = jc / pc;
        for (int k = kk - 1; k <= kk; ++k) {
            if (k < 0 || k > n - 1) continue;
            int a = jc - k * pc;
            if (a < 0 || a > pc) continue;
            for (int jl = 0; jl <= pf; ++jl) {
                int i = k * pf + jl;
                int owner = i / pf;
                if (owner > n - 1) owner = n - 1;
                if (owner != k) continue;
                const double w = tab.L[a * (pf + 1) + jl];
                if (w == 0.0) continue;
                idx[ax] = i;
                int64_t fi = (((int64_t)c * dims[2] + idx[2]) * dims[1] + idx[1]) * dims[0] + idx[0];
                T v = in[fi];
                if (in2) v -= in2[fi];
                s += (T)w * v;
            }
        }
        if (ess && ess[o]) s = T(0);
        out[o] = s;
    }
}

// Grid of a reduction kernel: about 4 elements per thread, at most kRedBlocks.
// one element per thread up to the cap: small vectors (coarse levels) spread
// over many SMs instead of waiting on a few
unsigned red_blocks(int64_t n)
{
    int64_t b = (n + kRedThreads - 1) / kRedThreads;
    if (b > kRedBlocks) b = kRedBlocks;
    if (b < 1) b = 1;
    return (unsigned)b;
}

unsigned blocks_for(int64_t n, int th = 256)
{
    int64_t b = (n + th - 1) / th;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

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
namespace {

template <typename T>
int dalloc(pa_solver *s, T **ptr, int64_t n)
{
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(T) * (size_t)(n > 0 ? n : 1));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? set_error(PA_ENOMEM, "solver: device allocation")
                                                                 : cuda_error(e, "solver: cudaMalloc");
    s->allocs.push_back(p);
    *ptr = static_cast<T *>(p);
    return PA_OK;
}

// coarse essential mask: coarse dof j is essential when the coarse basis
// function j is non-zero at some essential fine dof (exact for essential sets
// made of whole element faces).
std::vector<uint8_t> coarse_mask(const std::vector<uint8_t> &fine, const Grid &gf, int pc, const Basis1D &bc,
                                 const Basis1D &bf)
{
    const int pf = gf.p;
    std::vector<double> val((size_t)(pc + 1) * (pf + 1)), der(val.size());
    lagrange_product(pc + 1, bc.nodes.data(), pf + 1, bf.nodes.data(), val.data(), der.data());
    const int Mxc = gf.nx * pc + 1, Myc = gf.ny * pc + 1, Mzc = gf.nz * pc + 1;
    const int64_t Nnc = (int64_t)Mxc * Myc * Mzc;
    std::vector<uint8_t> out((size_t)3 * Nnc, 0);
    auto owners = [&](int i, int n, int *cj) {
        int k = std::min(i / pf, n - 1), jl = i - k * pf, cnt = 0;
        for (int a = 0; a <= pc; ++a)
            if (std::fabs(val[a * (pf + 1) + jl]) > 1e-14) cj[cnt++] = k * pc + a;
        return cnt;
    };
    int cx[kMaxD + 1], cy[kMaxD + 1], cz[kMaxD + 1];
    for (int c = 0; c < 3; ++c)
        for (int64_t gn = 0; gn < gf.Nn; ++gn) {
            if (!fine[(size_t)c * gf.Nn + gn]) continue;
            int gx = (int)(gn % gf.Mx), gy = (int)((gn / gf.Mx) % gf.My), gz = (int)(gn / ((int64_t)gf.Mx * gf.My));
            int nxa = owners(gx, gf.nx, cx), nya = owners(gy, gf.ny, cy), nza = owners(gz, gf.nz, cz);
            for (int k = 0; k < nza; ++k)
                for (int j = 0; j < nya; ++j)
                    for (int i = 0; i < nxa; ++i)
                        out[(size_t)c * Nnc + cx[i] + (int64_t)Mxc * (cy[j] + (int64_t)Myc * cz[k])] = 1;
        }
    return out;
}

// Element data of one level's mesh: the fine operator's, or the mesh whose
// uniform refinement is the level above (Sec. 3: the h-levels of the
// hierarchy come from r uniform refinements of a coarse mesh).
struct LevelMesh {
    int nx = 0, ny = 0, nz = 0;
    std::vector<double> affine;  // [ne][12]: J row-major, x0
    std::vector<double> mat;     // [ne][2] (lambda_e, mu_e), or empty
    std::vector<double> cv;      // [ne][36] Voigt matrices, or empty
    double lambda = 0.0, mu = 0.0;
};

LevelMesh mesh_of(const pa_op *op)
{
    LevelMesh m;
    m.nx = op->g.nx;
    m.ny = op->g.ny;
    m.nz = op->g.nz;
    m.affine = op->h_affine;
    m.mat = op->h_mat;
    m.cv = op->h_cv;
    m.lambda = op->lambda;
    m.mu = op->mu;
    return m;
}

// Undo one uniform refinement: coarse element (I, J, K) is the union of the
// fine elements (2I + a, 2J + b, 2K + c), a, b, c in {0, 1}.  Its map is
// x0 = x0 of child (0,0,0), J = 2 J of that child.  Fails unless every
// dimension is even, every child's map is the matching eighth of that map
// (to rounding) and the children share one material.
int coarsen_mesh(const LevelMesh &f, LevelMesh &c)
{
    if ((f.nx & 1) || (f.ny & 1) || (f.nz & 1))
        return set_error(PA_EINVAL, "solver: h-coarsening needs even element counts in x, y and z");
    c = LevelMesh();
    c.nx = f.nx / 2;
    c.ny = f.ny / 2;
    c.nz = f.nz / 2;
    c.lambda = f.lambda;
    c.mu = f.mu;
    const int64_t nec = (int64_t)c.nx * c.ny * c.nz;
    c.affine.assign((size_t)nec * 12, 0.0);
    if (!f.mat.empty()) c.mat.assign((size_t)nec * 2, 0.0);
    if (!f.cv.empty()) c.cv.assign((size_t)nec * 36, 0.0);
    auto fe = [&](int ix, int iy, int iz) { return (int64_t)ix + (int64_t)f.nx * (iy + (int64_t)f.ny * iz); };
    for (int K = 0; K < c.nz; ++K)
        for (int J = 0; J < c.ny; ++J)
            for (int I = 0; I < c.nx; ++I) {
                const int64_t E = (int64_t)I + (int64_t)c.nx * (J + (int64_t)c.ny * K);
                const double *a0 = f.affine.data() + 12 * fe(2 * I, 2 * J, 2 * K);
                double *A = c.affine.data() + 12 * E;
                double scale = 0.0;
                for (int k = 0; k < 9; ++k) {
                    A[k] = 2.0 * a0[k];
                    scale = std::max(scale, std::fabs(A[k]));
                }
                for (int k = 0; k < 3; ++k) A[9 + k] = a0[9 + k];
                const double tol = 1e-12 * scale;
                for (int cc = 0; cc < 2; ++cc)
                    for (int bb = 0; bb < 2; ++bb)
                        for (int aa = 0; aa < 2; ++aa) {
                            const int64_t e = fe(2 * I + aa, 2 * J + bb, 2 * K + cc);
                            const double *ae = f.affine.data() + 12 * e;
                            const double off[3] = {0.5 * aa, 0.5 * bb, 0.5 * cc};
                            bool ok = true;
                            for (int k = 0; k < 9; ++k) ok = ok && std::fabs(ae[k] - 0.5 * A[k]) <= tol;
                            for (int i = 0; i < 3; ++i) {
                                const double x0 = A[9 + i] + A[3 * i] * off[0] + A[3 * i + 1] * off[1] + A[3 * i + 2] * off[2];
                                ok = ok && std::fabs(ae[9 + i] - x0) <= tol + 1e-12 * std::fabs(x0);
                            }
                            if (!ok) return set_error(PA_EINVAL, "solver: mesh is not a uniform refinement (h-coarsening)");
                            if (!f.mat.empty()) {
                                if (f.mat[2 * e] != f.mat[2 * fe(2 * I, 2 * J, 2 * K)] ||
                                    f.mat[2 * e + 1] != f.mat[2 * fe(2 * I, 2 * J, 2 * K) + 1])
                                    return set_error(PA_EINVAL, "solver: material varies inside a coarse element");
                            }
                            if (!f.cv.empty()) {
                                for (int k = 0; k < 36; ++k)
                                    if (f.cv[36 * e + k] != f.cv[36 * fe(2 * I, 2 * J, 2 * K) + k])
                                        return set_error(PA_EINVAL, "solver: material varies inside a coarse element");
                            }
                        }
                if (!f.mat.empty()) {
                    c.mat[2 * E] = f.mat[2 * fe(2 * I, 2 * J, 2 * K)];
                    c.mat[2 * E + 1] = f.mat[2 * fe(2 * I, 2 * J, 2 * K) + 1];
                }
                if (!f.cv.empty())
                    std::copy(f.cv.begin() + 36 * fe(2 * I, 2 * J, 2 * K), f.cv.begin() + 36 * fe(2 * I, 2 * J, 2 * K) + 36,
                              c.cv.begin() + 36 * E);
            }
    return PA_OK;
}

int make_level_op(const LevelMesh &lm, int p, int precision, const std::vector<uint8_t> &mask, pa_op **out)
{
    pa_mesh m;
    m.nx = lm.nx;
    m.ny = lm.ny;
    m.nz = lm.nz;
    m.affine = lm.affine;
    int rc = pa_op_setup(&m, p, 0, lm.lambda, lm.mu, precision, mask.empty() ? nullptr : mask.data(), out);
    if (rc == PA_OK && !lm.mat.empty()) rc = pa_op_set_material(*out, lm.mat.data());
    if (rc == PA_OK && !lm.cv.empty()) rc = pa_op_set_anisotropic(*out, lm.cv.data());
    if (rc && *out) {
        pa_op_destroy(*out);
        *out = nullptr;
    }
    return rc;
}

// blocking read of one device scalar
double read_scalar(pa_solver *s, int slot, cudaStream_t st)
{
    cudaMemcpyAsync(s->h_scal + slot, s->dev.scal + slot, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return s->h_scal[slot];
}

// Chebyshev centre and half-width of the interval [cheb_lo, cheb_hi] * lam
void cheb_interval(const pa_solver *s, double lam, double *theta, double *delta)
{
    const double a = s->cheb_lo * lam, b = s->cheb_hi * lam;
    *theta = 0.5 * (a + b);
    *delta = 0.5 * (b - a);
}

// power iteration for lambda_max(D^-1 A) of level l (FP64), power_its (10 by
// default, Sec. 3.1) steps from a fixed pseudo-random start
int estimate_lmax(pa_solver *s, Level &L, cudaStream_t st)
{
    const int64_t n = L.n;
    k_random<<<blocks_for(n), 256, 0, st>>>(L.e, L.op->d_ess, n, 0x1234567ull + (uint64_t)L.p);
    double lam = 0.0;
    for (int it = 0; it < s->power_its; ++it) {
        k_norm2<double><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, L.e, n, P_DEN);
        int rc = op_apply_async(L.op, L.e, L.t, false, st, nullptr);
        if (rc) return rc;
        // d = Dinv (A e)   (k_cheb with a zero guess, cd = 0, cr = 1)
        k_cheb<double><<<blocks_for(n), 256, 0, st>>>(L.d, L.r, L.t, nullptr, L.dinv, 0.0, 1.0, 1, n);
        k_norm2<double><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, L.d, n, P_NUM);
        PA_CUDA_TRY(cudaMemcpyAsync(s->h_scal + P_NUM, s->dev.scal + P_NUM, 2 * sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
        PA_CUDA_TRY(cudaStreamSynchronize(st));
        const double num = s->h_scal[P_NUM], den = s->h_scal[P_DEN];
        if (!(den > 0.0) || !(num > 0.0) || !std::isfinite(num))
            return set_error(PA_EBREAKDOWN, "solver: power iteration broke down");
        lam = std::sqrt(num / den);
        k_scale_copy<double, double><<<blocks_for(n), 256, 0, st>>>(L.e, L.d, 1.0 / std::sqrt(num), n);
    }
    PA_CUDA_TRY(cudaGetLastError());
    L.lmax = lam;
    cheb_interval(s, lam, &L.theta, &L.delta);
    return PA_OK;
}


// ------------------------------------------------------- h-hierarchy setup
int h_power_lmax(pa_solver *s, HLevel &H, cudaStream_t st)
{
    const int64_t n = H.n;
    k_random<<<blocks_for(n), 256, 0, st>>>(H.e, H.ess, n, 0x5151ull + (uint64_t)n);
    double lam = 0.0;
    for (int it = 0; it < s->power_its; ++it) {
        k_norm2<double><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, H.e, n, P_DEN);
        k_stencil_apply<<<row3_blocks(n), 128, 0, st>>>(H.vals, H.e, H.t, H.g);
        k_cheb<double><<<blocks_for(n), 256, 0, st>>>(H.d, H.r, H.t, nullptr, H.dinv, 0.0, 1.0, 1, n);
        k_norm2<double><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, H.d, n, P_NUM);
        PA_CUDA_TRY(cudaMemcpyAsync(s->h_scal + P_NUM, s->dev.scal + P_NUM, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        PA_CUDA_TRY(cudaStreamSynchronize(st));
        const double num = s->h_scal[P_NUM], den = s->h_scal[P_DEN];
        if (!(den > 0.0) || !(num > 0.0) || !std::isfinite(num)) return set_error(PA_EBREAKDOWN, "solver: h-level power iteration");
        lam = std::sqrt(num / den);
        k_scale_copy<double, double><<<blocks_for(n), 256, 0, st>>>(H.e, H.d, 1.0 / std::sqrt(num), n);
    }
    H.lmax = lam;
    cheb_interval(s, lam, &H.theta, &H.delta);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

// Cholesky inverse of a small SPD matrix (host, in place on a copy).
bool spd_inverse(std::vector<double> &A, int n)
{
    std::vector<double> L((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(d > 0.0)) return false;
        const double ljj = std::sqrt(d);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double v = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = v / ljj;
        }
    }
    // inverse columns by forward/back substitution
    std::vector<double> col(n);
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= L[(size_t)i * n + k] * col[k];
            col[i] = v / L[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double v = col[i];
            for (int k = i + 1; k < n; ++k) v -= L[(size_t)k * n + i] * col[k];
            col[i] = v / L[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i) A[(size_t)i * n + c] = col[i];
    }
    return true;
}

// h-coarse essential mask: coarse dof j is essential when its interpolation
// reaches an essential fine dof (the 0/1 fine mask restricted); exact for
// essential sets made of whole faces.
std::vector<uint8_t> h_coarse_mask(const std::vector<uint8_t> &fm, const Grid &gf, const Grid &gc)
{
    std::vector<uint8_t> cm((size_t)3 * gc.Nn, 0);
    const int Mf[3] = {gf.Mx, gf.My, gf.Mz}, Mc[3] = {gc.Mx, gc.My, gc.Mz};
    for (int comp = 0; comp < 3; ++comp)
        for (int64_t i = 0; i < gf.Nn; ++i) {
            if (!fm[(size_t)(comp * gf.Nn + i)]) continue;
            const int f[3] = {(int)(i % gf.Mx), (int)((i / gf.Mx) % gf.My), (int)(i / ((int64_t)gf.Mx * gf.My))};
            int J[3][2], nJ[3];
            double w[3][2];
            for (int a = 0; a < 3; ++a) nJ[a] = h_parents(f[a], Mf[a], Mc[a], J[a], w[a]);
            for (int kz = 0; kz < nJ[2]; ++kz)
                for (int ky = 0; ky < nJ[1]; ++ky)
                    for (int kx = 0; kx < nJ[0]; ++kx)
                        cm[(size_t)(comp * gc.Nn + J[0][kx] + (int64_t)gc.Mx * (J[1][ky] + (int64_t)gc.My * J[2][kz]))] = 1;
        }
    return cm;
}

// Builds the h-hierarchy under the p = 1 level: Galerkin stencils, masks,
// diagonals, Chebyshev intervals, and a dense inverse on the coarsest level.
int build_h_levels(pa_solver *s, cudaStream_t st)
{
    Level &L = s->lv.back();
    if (!L.stencil) return PA_OK;
    const int64_t kMaxDense = 320;
    HLevel H0;
    H0.g = L.op->g;
    H0.n = L.n;
    H0.vals = L.stencil;
    H0.ess = L.op->d_ess;
    H0.dinv = L.dinv;
    s->hl.push_back(H0);
    while (true) {
        HLevel &F = s->hl.back();
        if (F.n <= kMaxDense) break;
        Grid c = F.g;
        c.Mx = h_coarse_size(F.g.Mx);
        c.My = h_coarse_size(F.g.My);
        c.Mz = h_coarse_size(F.g.Mz);
        if (c.Mx == F.g.Mx && c.My == F.g.My && c.Mz == F.g.Mz) break;
        c.nx = c.Mx - 1;
        c.ny = c.My - 1;
        c.nz = c.Mz - 1;
        c.p = 1;
        c.ne = (int64_t)c.nx * c.ny * c.nz;
        c.Nn = (int64_t)c.Mx * c.My * c.Mz;
        HLevel C;
        C.g = c;
        C.n = 3 * c.Nn;
        int rc;
        if ((rc = dalloc(s, &C.vals, 81 * C.n))) return rc;
        k_rap_stencil<<<blocks_for(C.n, 64), 64, 0, st>>>(F.vals, F.ess, F.g, C.vals, c);
        PA_CUDA_TRY(cudaGetLastError());
        if (F.ess) {
            // coarse essential dofs: those whose interpolation reaches an
            // essential fine dof (restrict the fine mask as a 0/1 field)
            std::vector<uint8_t> fm((size_t)F.n);
            PA_CUDA_TRY(cudaMemcpyAsync(fm.data(), F.ess, F.n, cudaMemcpyDeviceToHost, st));
            PA_CUDA_TRY(cudaStreamSynchronize(st));
            std::vector<uint8_t> cm = h_coarse_mask(fm, F.g, c);
            if ((rc = dalloc(s, &C.ess, C.n))) return rc;
            PA_CUDA_TRY(cudaMemcpyAsync(C.ess, cm.data(), C.n, cudaMemcpyHostToDevice, st));
            PA_CUDA_TRY(cudaStreamSynchronize(st));
        }
        if ((rc = dalloc(s, &C.dinv, C.n))) return rc;
        k_mask_stencil<<<blocks_for(C.n, 128), 128, 0, st>>>(C.vals, C.ess, c);
        PA_CUDA_TRY(cudaGetLastError());
        s->hl.push_back(C);
    }
    // work vectors, diagonals, Chebyshev intervals, coarsest inverse
    for (size_t k = 0; k < s->hl.size(); ++k) {
        HLevel &H = s->hl[k];
        int rc;
        // level 0 reads its right-hand side from the coarse CG residual in place
        if (k == 0) H.r = L.cr;
        else if ((rc = dalloc(s, &H.r, H.n))) return rc;
        if ((rc = dalloc(s, &H.e, H.n)) || (rc = dalloc(s, &H.e2, H.n)) || (rc = dalloc(s, &H.t, H.n)) ||
            (rc = dalloc(s, &H.d, H.n)) || (rc = dalloc(s, &H.xa, H.n)) || (rc = dalloc(s, &H.xb, H.n)))
            return rc;
        if (k > 0) {
            // diagonal = stencil centre entry (s = 13) of the own component; 1 on essential rows
            std::vector<double> cen((size_t)H.n);
            std::vector<uint8_t> em;
            for (int comp = 0; comp < 3; ++comp)
                PA_CUDA_TRY(cudaMemcpyAsync(cen.data() + comp * H.g.Nn, H.vals + (int64_t)(13 * 3 + comp) * H.n + comp * H.g.Nn,
                                            sizeof(double) * H.g.Nn, cudaMemcpyDeviceToHost, st));
            if (H.ess) {
                em.resize((size_t)H.n);
                PA_CUDA_TRY(cudaMemcpyAsync(em.data(), H.ess, H.n, cudaMemcpyDeviceToHost, st));
            }
            PA_CUDA_TRY(cudaStreamSynchronize(st));
            for (int64_t i = 0; i < H.n; ++i) cen[(size_t)i] = (H.ess && em[(size_t)i]) ? 1.0 : 1.0 / cen[(size_t)i];
            PA_CUDA_TRY(cudaMemcpyAsync(H.dinv, cen.data(), sizeof(double) * H.n, cudaMemcpyHostToDevice, st));
            PA_CUDA_TRY(cudaStreamSynchronize(st));
        }
        if (k + 1 < s->hl.size()) {
            if ((rc = h_power_lmax(s, H, st))) return rc;
        }
    }
    // dense inverse of the coarsest level (constrained: identity on essential dofs)
    HLevel &Hc = s->hl.back();
    if (Hc.n > 4 * kMaxDense) return set_error(PA_EINVAL, "solver: h-hierarchy coarsest level too large for a dense solve");
    const int n = (int)Hc.n;
    std::vector<double> V((size_t)81 * n);
    std::vector<uint8_t> em((size_t)n, 0);
    PA_CUDA_TRY(cudaMemcpyAsync(V.data(), Hc.vals, sizeof(double) * V.size(), cudaMemcpyDeviceToHost, st));
    if (Hc.ess) PA_CUDA_TRY(cudaMemcpyAsync(em.data(), Hc.ess, n, cudaMemcpyDeviceToHost, st));
    PA_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> A((size_t)n * n, 0.0);
    const Grid &g = Hc.g;
    for (int row = 0; row < n; ++row) {
        if (em[row]) {
            A[(size_t)row * n + row] = 1.0;
            continue;
        }
        const int c = (int)(row / g.Nn);
        const int64_t i = row - c * g.Nn;
        const int ix = (int)(i % g.Mx), iy = (int)((i / g.Mx) % g.My), iz = (int)(i / ((int64_t)g.Mx * g.My));
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (ix + dx < 0 || ix + dx >= g.Mx || iy + dy < 0 || iy + dy >= g.My || iz + dz < 0 || iz + dz >= g.Mz)
                        continue;
                    const int sidx = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                    const int64_t j = i + dx + (int64_t)g.Mx * (dy + (int64_t)g.My * dz);
                    for (int d = 0; d < 3; ++d) {
                        const int64_t col = d * g.Nn + j;
                        if (em[col]) continue;
                        A[(size_t)row * n + col] += V[(size_t)(sidx * 3 + d) * n + row];
                    }
                }
    }
    // symmetrise the rounding, then invert
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const double m = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
            A[(size_t)i * n + j] = A[(size_t)j * n + i] = m;
        }
    if (!spd_inverse(A, n)) return set_error(PA_EBREAKDOWN, "solver: coarsest h-level matrix is not SPD");
    int rc = dalloc(s, &Hc.Ainv, (int64_t)n * n);
    if (rc) return rc;
    PA_CUDA_TRY(cudaMemcpyAsync(Hc.Ainv, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice, st));
    PA_CUDA_TRY(cudaStreamSynchronize(st));
    return PA_OK;
}

// The first-step arguments of h-level H (cr of the first Chebyshev step)
FirstStep h_first_step(const HLevel &H)
{
    FirstStep f;
    f.e = H.e;
    f.d = H.d;
    f.dinv = H.dinv;
    f.cr = 1.0 / H.theta;
    return f;
}

// ... of the first h-level, which the coarse CG's start and update kernels
// take (none when the first level is the dense bottom)
FirstStep coarse_first_step(pa_solver *s) { return s->hl.size() > 1 ? h_first_step(s->hl[0]) : FirstStep{}; }

// Chebyshev smoothing on an h-level (stencil operator) of the iterate in
// buffer e.  The step from a zero iterate needs no operator apply: the
// kernel that produced the level's right-hand side has already taken it
// into H.e and H.d (first_step), so pre-smoothing starts at the second
// step.  Every other step is one fused kernel (stencil apply and update)
// from one iterate buffer into the other (H.e / H.e2).  Returns the buffer
// with the result.
double *h_smooth(pa_solver *s, HLevel &H, double *e, bool from_zero, cudaStream_t st)
{
    const int64_t n = H.n;
    const double sigma = H.theta / H.delta;
    double rho_prev = 1.0 / sigma;
    double *cur = e;
    for (int k = 0; k < s->cheb_order; ++k) {
        double cd, cr;
        if (k == 0) {
            cd = 0.0;
            cr = 1.0 / H.theta;
        } else {
            const double rho = 1.0 / (2.0 * sigma - rho_prev);
            cd = rho * rho_prev;
            cr = 2.0 * rho / H.delta;
            rho_prev = rho;
        }
        if (k == 0 && from_zero) {
            continue;  // taken by the producer of H.r
        } else {
            double *nxt = cur == H.e ? H.e2 : H.e;
            k_stencil_cheb<<<row3_blocks(n), 128, 0, st>>>(H.vals, cur, nxt, H.d, H.r, H.dinv, cd, cr, H.g);
            cur = nxt;
        }
    }
    return cur;
}

// h-V(1,1) cycle from h-level k: e_k ~ A_k^-1 r_k; returns the buffer of
// level k holding e_k.  Launch errors are left for the caller's check.
double *h_vcycle(pa_solver *s, size_t k, cudaStream_t st)
{
    HLevel &F = s->hl[k];
    if (k + 1 == s->hl.size()) {
        k_dense_matvec<<<(unsigned)((F.n * 32 + 255) / 256), 256, 0, st>>>(F.Ainv, F.r, F.e, F.n);
        return F.e;
    }
    HLevel &C = s->hl[k + 1];
    double *e = h_smooth(s, F, F.e, true, st);
    k_stencil_apply<<<row3_blocks(F.n), 128, 0, st>>>(F.vals, e, F.t, F.g);
    // restrict r - t (with the coarse level's first smoothing step unless it
    // is the dense bottom), then the coarse correction prolonged and added
    if (k + 2 < s->hl.size())
        k_hrestrict_first<<<row3_blocks(C.n), 128, 0, st>>>(C.r, F.r, F.t, F.g, C.g, C.ess, h_first_step(C));
    else
        k_hrestrict<double><<<row3_blocks(C.n), 128, 0, st>>>(C.r, F.r, F.t, F.g, C.g, C.ess);
    const double *ec = h_vcycle(s, k + 1, st);
    k_hprolong_add<double><<<blocks_for(F.n, 64), 64, 0, st>>>(e, ec, F.g, C.g);
    return h_smooth(s, F, e, false, st);
}

// h-multigrid preconditioned coarse CG: on a ladder of h-levels, or (a
// coarse level small enough for it) on the dense inverse alone
bool use_hmg(pa_solver *s) { return s->use_hmg && !s->hl.empty() && s->hl.back().Ainv != nullptr; }

// h-multigrid preconditioned coarse CG, with the loop rotated so that each
// iteration applies the preconditioner once and the last one applies none
// after convergence:
//   start:     x = 0, r = b, rz = 0 (the first direction is z itself)
//   iteration: z = M r; beta = (r, z) / rz (0 at first); p = z + beta p;
//              q = A p, alpha = rz / (p, q); x += alpha p; r -= alpha q;
//              stop when (r, r) <= tol^2 (b, b)
int coarse_start_hmg(pa_solver *s, Level &L, cudaStream_t st)
{
    k_pcg_start1<<<red_blocks(L.n), kRedThreads, 0, st>>>(s->dev, L.cx, L.cr, L.r, L.n, s->coarse_rtol * s->coarse_rtol,
                                                          coarse_first_step(s));
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

int coarse_iter_hmg(pa_solver *s, Level &L, cudaStream_t st)
{
    const int64_t n = L.n;
    const double *z = h_vcycle(s, 0, st);  // reads L.cr in place
    k_pcg_beta<<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, L.cr, z, n);
    k_pcg_p<<<blocks_for(n), 256, 0, st>>>(s->dev, L.cp, z, n);
    k_cg_spmv_pq<<<row3_blocks(n, kRedBlocks), 128, 0, st>>>(s->dev, L.stencil, L.cp, L.cq, L.op->g);
    k_pcg_update<<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, L.cx, L.cr, L.cp, L.cq, n, coarse_first_step(s));
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

// ------------------------------------------------------------ V-cycle (T)
template <typename T>
struct LV {
    static T *r(Level &L);
    static T *e(Level &L);
    static T *t(Level &L);
    static T *d(Level &L);
    static T *dinv(Level &L);
    static T *xa(Level &L);
    static T *xb(Level &L);
    static pa_op *op(Level &L);
};
template <> double *LV<double>::r(Level &L) { return L.r; }
template <> double *LV<double>::e(Level &L) { return L.e; }
template <> double *LV<double>::t(Level &L) { return L.t; }
template <> double *LV<double>::d(Level &L) { return L.d; }
template <> double *LV<double>::dinv(Level &L) { return L.dinv; }
template <> double *LV<double>::xa(Level &L) { return L.xa; }
template <> double *LV<double>::xb(Level &L) { return L.xb; }
template <> pa_op *LV<double>::op(Level &L) { return L.op; }
template <> float *LV<float>::r(Level &L) { return L.r32; }
template <> float *LV<float>::e(Level &L) { return L.e32; }
template <> float *LV<float>::t(Level &L) { return L.t32; }
template <> float *LV<float>::d(Level &L) { return L.d32; }
template <> float *LV<float>::dinv(Level &L) { return L.dinv32; }
template <> float *LV<float>::xa(Level &L) { return L.xa32; }
template <> float *LV<float>::xb(Level &L) { return L.xb32; }
template <> pa_op *LV<float>::op(Level &L) { return L.op32; }

// True when the kernels of the code being run are to be launched (always,
// unless a lockstep capture filters one phase).
inline bool emit(const pa_solver *s) { return !s->ph_on || s->ph_counter == s->ph_target; }

// An operator apply of a step function: launched, or under the phase filter
// recorded when it ends the filtered phase; either way the next phase starts.
int step_apply(pa_solver *s, pa_op *op, const void *x, void *y, cudaStream_t st)
{
    if (!s->ph_on) return op_apply_async(op, x, y, false, st, nullptr);
    if (s->ph_counter == s->ph_target) {
        s->ph_op = op;
        s->ph_x = x;
        s->ph_y = y;
    }
    ++s->ph_counter;
    return PA_OK;
}

// A phase boundary without an apply (keeps the phases of solvers whose step
// skips an apply aligned with the others').
void step_gap(pa_solver *s)
{
    if (s->ph_on) ++s->ph_counter;
}

// Chebyshev smoothing of A e = r on level L (cheb_order steps); from a zero
// guess the first step needs no operator apply.
template <typename T>
int smooth(pa_solver *s, Level &L, bool from_zero, cudaStream_t st)
{
    const int64_t n = L.n;
    T *e = LV<T>::e(L), *dv = LV<T>::d(L), *r = LV<T>::r(L), *t = LV<T>::t(L), *dinv = LV<T>::dinv(L);
    pa_op *op = LV<T>::op(L);
    const double sigma = L.theta / L.delta;
    double rho_prev = 1.0 / sigma;
    for (int k = 0; k < s->cheb_order; ++k) {
        const T *tt = nullptr;
        if (!(k == 0 && from_zero)) {
            int rc = step_apply(s, op, e, t, st);
            if (rc) return rc;
            tt = t;
        }
        double cd, cr;
        if (k == 0) {
            cd = 0.0;
            cr = 1.0 / L.theta;
        } else {
            double rho = 1.0 / (2.0 * sigma - rho_prev);
            cd = rho * rho_prev;
            cr = 2.0 * rho / L.delta;
            rho_prev = rho;
        }
        if (emit(s))
            k_cheb<T><<<blocks_for(n), 256, 0, st>>>(e, dv, r, tt, dinv, cd, cr, (k == 0 && from_zero) ? 1 : 0, n);
    }
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

// rc = R (r - t) of level l into level l+1 (T storage)
template <typename T>
void restrict_to(Level &F, Level &C, const T *r, const T *t, T *out, cudaStream_t st)
{
    if (F.hdown) {
        k_hrestrict<T><<<row3_blocks(3 * C.op->g.Nn), 128, 0, st>>>(out, r, t, F.op->g, C.op->g, C.op->d_ess);
        return;
    }
    const Grid &g = F.op->g;
    const int n_[3] = {g.nx, g.ny, g.nz};
    const int pf = F.p, pc = C.p;
    const int Mf[3] = {g.Mx, g.My, g.Mz};
    const int Mc[3] = {n_[0] * pc + 1, n_[1] * pc + 1, n_[2] * pc + 1};
    T *xa = LV<T>::xa(F), *xb = LV<T>::xb(F);
    // x axis: [3][Mzf][Myf][Mxf] -> [3][Mzf][Myf][Mxc]
    int64_t n1 = 3LL * Mf[2] * Mf[1] * Mc[0];
    k_restrict_axis<T><<<blocks_for(n1), 256, 0, st>>>(xa, r, t, 0, Mf[0], Mf[1], Mf[2], n_[0], pc, pf, F.xt, nullptr);
    int64_t n2 = 3LL * Mf[2] * Mc[1] * Mc[0];
    k_restrict_axis<T><<<blocks_for(n2), 256, 0, st>>>(xb, xa, nullptr, 1, Mc[0], Mf[1], Mf[2], n_[1], pc, pf, F.xt,
                                                       nullptr);
    int64_t n3 = 3LL * Mc[2] * Mc[1] * Mc[0];
    k_restrict_axis<T><<<blocks_for(n3), 256, 0, st>>>(out, xb, nullptr, 2, Mc[0], Mc[1], Mf[2], n_[2], pc, pf, F.xt,
                                                       C.op->d_ess);
}

// e_f += P e_c
template <typename T>
void prolong_add(Level &F, Level &C, const T *ec, T *ef, cudaStream_t st)
{
    if (F.hdown) {
        k_hprolong_add<T><<<blocks_for(3 * F.op->g.Nn), 256, 0, st>>>(ef, ec, F.op->g, C.op->g);
        return;
    }
    const Grid &g = F.op->g;
    const int n_[3] = {g.nx, g.ny, g.nz};
    const int pf = F.p, pc = C.p;
    const int Mf[3] = {g.Mx, g.My, g.Mz};
    const int Mc[3] = {n_[0] * pc + 1, n_[1] * pc + 1, n_[2] * pc + 1};
    T *xa = LV<T>::xa(F), *xb = LV<T>::xb(F);
    int64_t n1 = 3LL * Mc[2] * Mc[1] * Mf[0];
    k_prolong_axis<T><<<blocks_for(n1), 256, 0, st>>>(xa, ec, 0, Mc[0], Mc[1], Mc[2], n_[0], pc, pf, F.xt, 0);
    int64_t n2 = 3LL * Mc[2] * Mf[1] * Mf[0];
    k_prolong_axis<T><<<blocks_for(n2), 256, 0, st>>>(xb, xa, 1, Mf[0], Mc[1], Mc[2], n_[1], pc, pf, F.xt, 0);
    int64_t n3 = 3LL * Mf[2] * Mf[1] * Mf[0];
    k_prolong_axis<T><<<blocks_for(n3), 256, 0, st>>>(ef, xb, 2, Mf[0], Mf[1], Mc[2], n_[2], pc, pf, F.xt, 1);
}

// ---------------------------------------------------------- coarse solve
// FP64 Jacobi-CG on the coarsest level: L.cx ~ A^-1 L.r.  The start kernel
// resets the device stop flag and iteration counter; every iteration's
// kernels return at once after the flag is set.
int coarse_start(pa_solver *s, Level &L, cudaStream_t st)
{
    if (use_hmg(s)) return coarse_start_hmg(s, L, st);
    k_cg_start<<<red_blocks(L.n), kRedThreads, 0, st>>>(s->dev, L.cx, L.cr, L.cp, L.r, L.dinv, L.n,
                                                   s->coarse_rtol * s->coarse_rtol);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

int coarse_iter(pa_solver *s, Level &L, cudaStream_t st)
{
    if (use_hmg(s)) return coarse_iter_hmg(s, L, st);
    const int64_t n = L.n;
    if (L.stencil) {
        // FP64 work per row: three lanes per row spread it over the SMs
        k_cg_spmv_pq<<<row3_blocks(n, kRedBlocks), 128, 0, st>>>(s->dev, L.stencil, L.cp, L.cq, L.op->g);
    } else {
        int rc = op_apply_async(L.op, L.cp, L.cq, false, st, s->dev.flag + F_CDONE);
        if (rc) return rc;
        k_cg_pq<<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, L.cp, L.cq, n);
    }
    k_cg_update<<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, L.cx, L.cr, L.cp, L.cq, L.dinv, n);
    k_cg_p<<<blocks_for(n), 256, 0, st>>>(s->dev, L.cp, L.cr, L.dinv, n);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

// The persistent cooperative coarse CG applies when the coarse level is
// assembled, Jacobi-preconditioned (h-multigrid off) and co-resident CTAs
// are available.  (The h-multigrid PCG as one cooperative launch, with a
// grid barrier between its ~26 dependent stages per iteration, measured
// slower than the launched kernels in the step graph at every CTA count.)
bool use_coop(pa_solver *s)
{
    return !use_hmg(s) && s->allow_coop && s->coop_blocks > 0 && s->lv.back().stencil != nullptr;
}

int coarse_coop(pa_solver *s, cudaStream_t st)
{
    Level &L = s->lv.back();
    PA_CUDA_TRY(cudaMemsetAsync(s->bar, 0, 2 * sizeof(unsigned), st));
    Dev dv = s->dev;
    const double *vals = L.stencil, *dinv = L.dinv, *b = L.r;
    double *x = L.cx, *r = L.cr, *p = L.cp, *q = L.cq;
    const uint8_t *ess = L.op->d_ess;
    Grid g = L.op->g;
    double tol2 = s->coarse_rtol * s->coarse_rtol;
    int maxit = s->coarse_maxit;
    unsigned *bar = s->bar;
    double *part = s->coop_part;
    long long wait_cycles = s->wait_cycles;
    void *args[] = {&dv, &vals, &x, &r, &p, &q, &dinv, &b, &ess, &g, &tol2, &maxit, &bar, &part, &wait_cycles};
    PA_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_cg_coop, dim3(s->coop_blocks), dim3(256), args, 0, st));
    return PA_OK;
}

// Eager coarse solve: the persistent kernel, or a fixed number of launches
// of the iteration kernels (which return at once after convergence).
int coarse_eager(pa_solver *s, cudaStream_t st)
{
    if (use_coop(s)) return coarse_coop(s, st);
    Level &L = s->lv.back();
    for (int it = 0; it < s->coarse_maxit; ++it) {
        int rc = coarse_iter(s, L, st);
        if (rc) return rc;
    }
    return PA_OK;
}

// ------------------------------------------------------------- V(1,1) cycle
// Down half: pre-smoothing, residual and restriction from level 0 to the
// coarsest level, whose FP64 right-hand side ends in L.r; then the coarse
// CG start.  Input: LV<T>::r(level 0).
template <typename T>
int vcycle_down(pa_solver *s, cudaStream_t st)
{
    const int nl = (int)s->lv.size();
    for (int l = 0; l < nl - 1; ++l) {
        Level &L = s->lv[l], &C = s->lv[l + 1];
        int rc = smooth<T>(s, L, true, st);
        if (rc) return rc;
        rc = step_apply(s, LV<T>::op(L), LV<T>::e(L), LV<T>::t(L), st);
        if (rc) return rc;
        if (emit(s)) restrict_to<T>(L, C, LV<T>::r(L), LV<T>::t(L), LV<T>::r(C), st);
    }
    if (!emit(s)) return PA_OK;
    Level &Lc = s->lv.back();
    if constexpr (sizeof(T) == 4) k_scale_copy<float, double><<<blocks_for(Lc.n), 256, 0, st>>>(Lc.r, Lc.r32, 1.0, Lc.n);
    if (!use_coop(s)) {
        int rc = coarse_start(s, Lc, st);
        if (rc) return rc;
    }
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

// Up half: coarse correction into LV<T>::e(coarsest), then prolongation and
// post-smoothing back to level 0.  Output: LV<T>::e(level 0).
template <typename T>
int vcycle_up(pa_solver *s, cudaStream_t st)
{
    const int nl = (int)s->lv.size();
    Level &Lc = s->lv.back();
    if (emit(s)) k_scale_copy<double, T><<<blocks_for(Lc.n), 256, 0, st>>>(LV<T>::e(Lc), Lc.cx, 1.0, Lc.n);
    for (int l = nl - 2; l >= 0; --l) {
        Level &L = s->lv[l], &C = s->lv[l + 1];
        if (emit(s)) prolong_add<T>(L, C, LV<T>::e(C), LV<T>::e(L), st);
        int rc = smooth<T>(s, L, false, st);
        if (rc) return rc;
    }
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

// ------------------------------------------------------------ flexible CG
// One FCG step is two segments around the coarse solve of its V-cycle:
//   init  A: r = b - A x (or x = 0, r = b), V-cycle down
//   init  B: V-cycle up, z = M r, p = z, rz = (r, z), rr = (r, r)
//   iter  A: q = A p, alpha, x += alpha p, r -= alpha q, V-cycle down
//   iter  B: V-cycle up, z = M r, beta, p = z + beta p
// Both B segments end with an asynchronous copy of rr and the flags to
// pinned host memory.
template <typename T>
struct FcgVecs {
    T *x, *b, *r, *z, *p, *q;
    bool x_zero;
};

template <typename T, typename TP>
int fcg_init_a(pa_solver *s, const FcgVecs<T> &v, cudaStream_t st)
{
    Level &L0 = s->lv[0];
    const int64_t n = L0.n;
    if (v.x_zero) {
        if (emit(s)) {
            PA_CUDA_TRY(cudaMemsetAsync(v.x, 0, sizeof(T) * n, st));
            k_scale_copy<T, T><<<blocks_for(n), 256, 0, st>>>(v.r, v.b, 1.0, n);
        }
        step_gap(s);  // in the place of the apply below
    } else {
        int rc = step_apply(s, LV<T>::op(L0), v.x, v.q, st);
        if (rc) return rc;
        if (emit(s)) k_sub<T, T, T><<<blocks_for(n), 256, 0, st>>>(v.r, v.b, v.q, n);
    }
    if (emit(s)) k_scale_copy<T, TP><<<blocks_for(n), 256, 0, st>>>(LV<TP>::r(L0), v.r, 1.0, n);
    return vcycle_down<TP>(s, st);
}

template <typename T>
int publish_scalars(pa_solver *s, cudaStream_t st)
{
    PA_CUDA_TRY(cudaMemcpyAsync(s->h_scal + S_RR, s->dev.scal + S_RR, sizeof(double), cudaMemcpyDeviceToHost, st));
    PA_CUDA_TRY(cudaMemcpyAsync(s->h_flag, s->dev.flag, sizeof(int) * NFLAG, cudaMemcpyDeviceToHost, st));
    return PA_OK;
}

template <typename T, typename TP>
int fcg_init_b(pa_solver *s, const FcgVecs<T> &v, cudaStream_t st)
{
    Level &L0 = s->lv[0];
    const int64_t n = L0.n;
    int rc = vcycle_up<TP>(s, st);
    if (rc) return rc;
    if (!emit(s)) return PA_OK;
    k_scale_copy<TP, T><<<blocks_for(n), 256, 0, st>>>(v.z, LV<TP>::e(L0), 1.0, n);
    k_fcg_start<T><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, v.p, v.z, v.r, n, 0);
    PA_CUDA_TRY(cudaGetLastError());
    return publish_scalars<T>(s, st);
}

template <typename T, typename TP>
int fcg_iter_a(pa_solver *s, const FcgVecs<T> &v, cudaStream_t st)
{
    Level &L0 = s->lv[0];
    const int64_t n = L0.n;
    int rc = step_apply(s, LV<T>::op(L0), v.p, v.q, st);
    if (rc) return rc;
    if (emit(s)) {
        k_fcg_pq<T><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, v.p, v.q, n, 0);
        k_fcg_update<T, T><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, v.x, v.r, v.p, v.q, n, 0);
        k_scale_copy<T, TP><<<blocks_for(n), 256, 0, st>>>(LV<TP>::r(L0), v.r, 1.0, n);
    }
    return vcycle_down<TP>(s, st);
}

template <typename T, typename TP>
int fcg_iter_b(pa_solver *s, const FcgVecs<T> &v, cudaStream_t st)
{
    Level &L0 = s->lv[0];
    const int64_t n = L0.n;
    int rc = vcycle_up<TP>(s, st);
    if (rc) return rc;
    if (!emit(s)) return PA_OK;
    k_scale_copy<TP, T><<<blocks_for(n), 256, 0, st>>>(v.z, LV<TP>::e(L0), 1.0, n);
    k_fcg_beta<T><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, v.z, v.r, v.q, n, 0);
    k_fcg_p<T><<<blocks_for(n), 256, 0, st>>>(s->dev, v.p, v.z, n, 0);
    PA_CUDA_TRY(cudaGetLastError());
    return publish_scalars<T>(s, st);
}

// Captures [segment A] -> WHILE(coarse CG iteration) -> [segment B] into an
// executable graph; the loop's condition is set on the device after every
// coarse iteration (stop flag or iteration cap), so only the iterations the
// coarse solve needs are executed.
template <typename FA, typename FB>
int build_step_graph(pa_solver *s, cudaStream_t st, FA seg_a, FB seg_b, cudaGraphExec_t *out)
{
    if (use_coop(s)) {
        // one capture: segment A, the persistent coarse CG, segment B
        cudaGraph_t g = nullptr;
        PA_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
        int r = seg_a();
        if (!r) r = coarse_coop(s, st);
        if (!r) r = seg_b();
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (r) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e != cudaSuccess) return cuda_error(e, "solver graph: cudaStreamEndCapture");
        e = cudaGraphInstantiate(out, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
        return PA_OK;
    }
    cudaGraph_t G = nullptr, gA = nullptr, gB = nullptr, gBody = nullptr;
    int rc = PA_OK;
    auto capture = [&](cudaGraph_t *g, auto &&fn) -> int {
        PA_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
        int r = fn();
        cudaGraph_t tmp = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &tmp);
        if (r) {
            if (tmp) cudaGraphDestroy(tmp);
            return r;
        }
        if (e != cudaSuccess) return cuda_error(e, "solver graph: cudaStreamEndCapture");
        *g = tmp;
        return PA_OK;
    };
    do {
        if (cudaGraphCreate(&G, 0) != cudaSuccess) { rc = cuda_error(cudaGetLastError(), "cudaGraphCreate"); break; }
        if ((rc = capture(&gA, seg_a))) break;
        cudaGraphNode_t nA, nC, nB, nBody;
        cudaError_t e = cudaGraphAddChildGraphNode(&nA, G, nullptr, 0, gA);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaGraphAddChildGraphNode"); break; }
        cudaGraphConditionalHandle h;
        e = cudaGraphConditionalHandleCreate(&h, G, 1, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaGraphConditionalHandleCreate"); break; }
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&nC, G, &nA, nullptr, 1, &cp);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaGraphAddNode(conditional)"); break; }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        Level &Lc = s->lv.back();
        const int maxit = s->coarse_maxit;
        if ((rc = capture(&gBody, [&]() -> int {
                 int r = coarse_iter(s, Lc, st);
                 if (r) return r;
                 k_cg_cond<<<1, 32, 0, st>>>(s->dev, maxit, h);
                 PA_CUDA_TRY(cudaGetLastError());
                 return PA_OK;
             })))
            break;
        e = cudaGraphAddChildGraphNode(&nBody, body, nullptr, 0, gBody);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaGraphAddChildGraphNode(body)"); break; }
        if ((rc = capture(&gB, seg_b))) break;
        e = cudaGraphAddChildGraphNode(&nB, G, &nC, 1, gB);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaGraphAddChildGraphNode"); break; }
        e = cudaGraphInstantiate(out, G, 0);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaGraphInstantiate"); break; }
    } while (false);
    if (gA) cudaGraphDestroy(gA);
    if (gB) cudaGraphDestroy(gB);
    if (gBody) cudaGraphDestroy(gBody);
    if (G) cudaGraphDestroy(G);
    return rc;
}

// Flexible CG on level 0 in storage T (FP64 outer solve, or the FP32 inner
// solve of the mixed mode).  Stops when (r, r) <= tol2 * bb or after maxit
// iterations.  With graphs, each step is one graph launch; otherwise the
// same segments run eagerly with the fixed-length coarse loop.
template <typename T, typename TP = T>
int fcg(pa_solver *s, const FcgVecs<T> &v, StepGraphs &sg, double tol2, double bb, int maxit, int *iters,
        cudaStream_t st)
{
    int rc;
    if (s->use_graphs && !sg.init) {
        rc = build_step_graph(
            s, st, [&]() { return fcg_init_a<T, TP>(s, v, st); }, [&]() { return fcg_init_b<T, TP>(s, v, st); }, &sg.init);
        if (!rc)
            rc = build_step_graph(
                s, st, [&]() { return fcg_iter_a<T, TP>(s, v, st); }, [&]() { return fcg_iter_b<T, TP>(s, v, st); }, &sg.iter);
        if (rc) {
            // fall back to eager execution for this solver
            if (sg.init) cudaGraphExecDestroy(sg.init);
            if (sg.iter) cudaGraphExecDestroy(sg.iter);
            sg.init = sg.iter = nullptr;
            s->use_graphs = false;
            cudaGetLastError();
        }
    }
    auto step = [&](bool init) -> int {
        if (s->use_graphs) {
            PA_CUDA_TRY(cudaGraphLaunch(init ? sg.init : sg.iter, st));
        } else {
            int r = init ? fcg_init_a<T, TP>(s, v, st) : fcg_iter_a<T, TP>(s, v, st);
            if (r) return r;
            r = coarse_eager(s, st);
            if (r) return r;
            r = init ? fcg_init_b<T, TP>(s, v, st) : fcg_iter_b<T, TP>(s, v, st);
            if (r) return r;
        }
        PA_CUDA_TRY(cudaStreamSynchronize(st));
        if (s->use_graphs) s->coarse_its += s->h_flag[F_CIT];
        return PA_OK;
    };
    rc = step(true);
    if (rc) return rc;
    double rr = s->h_scal[S_RR];
    int it = 0;
    if (s->h_flag[F_CTIMEOUT]) return set_error(PA_ETIMEOUT, "solver: coarse-solve grid barrier timed out");
    if (s->h_flag[F_BREAK]) {
        *iters = 0;
        return set_error(PA_EBREAKDOWN, "solver: non-finite value in the first preconditioned residual");
    }
    while (rr > tol2 * bb && it < maxit) {
        if (s->cancel && s->cancel->load(std::memory_order_relaxed)) {
            *iters = it;
            return set_error(PA_ECANCELED, "solver: solve canceled");
        }
        rc = step(false);
        if (rc) return rc;
        rr = s->h_scal[S_RR];
        ++it;
        if (s->h_flag[F_CTIMEOUT]) {
            *iters = it;
            return set_error(PA_ETIMEOUT, "solver: coarse-solve grid barrier timed out");
        }
        if (s->h_flag[F_BREAK]) {
            *iters = it;
            return set_error(PA_EBREAKDOWN, "solver: CG breakdown (p^T A p <= 0 or non-finite value)");
        }
    }
    *iters = it;
    return PA_OK;
}

// Start of a solve: flags cleared, (b, b) computed; b = 0 gives x = 0 at
// once (*trivial), non-finite b is rejected; b and x copied into the
// solver's own vectors.  Blocks until (b, b) is on the host.
int solve_begin(pa_solver *s, const double *b, double *x, double *bb_out, pa_solve_info *inf, bool *trivial)
{
    cudaStream_t st = s->stream;
    const int64_t n = s->lv[0].n;
    *inf = pa_solve_info{};
    *trivial = false;
    s->coarse_its = 0;
    for (size_t l = 0; l < s->lv.size() && l < 8; ++l) inf->lambda_max[l] = s->lv[l].lmax;
    PA_CUDA_TRY(cudaMemsetAsync(s->dev.flag, 0, sizeof(int) * NFLAG, st));
    k_norm2<double><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, b, n, S_BB);
    const double bb = read_scalar(s, S_BB, st);
    inf->b_norm = std::sqrt(bb);
    *bb_out = bb;
    if (bb == 0.0) {
        PA_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
        PA_CUDA_TRY(cudaStreamSynchronize(st));
        inf->rel_residual = 0.0;
        inf->tolerance_met = 1;
        *trivial = true;
        return PA_OK;
    }
    if (!std::isfinite(bb)) return set_error(PA_EINVAL, "pa_gmg_pcg_solve: b has non-finite entries");
    PA_CUDA_TRY(cudaMemcpyAsync(s->xin, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    PA_CUDA_TRY(cudaMemcpyAsync(s->bin, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    return PA_OK;
}

// End of a solve: the true FP64 residual of the solver's iterate, which is
// copied to x.  rc_loop is the iteration loop's return code (breakdown is
// reported as a status with the residual; other errors are returned as is).
int solve_finish(pa_solver *s, double *x, int rc_loop, bool converged, double bb, double tol2, pa_solve_info *inf)
{
    cudaStream_t st = s->stream;
    Level &L0 = s->lv[0];
    const int64_t n = L0.n;
    int status = PA_OK;
    if (rc_loop == PA_EBREAKDOWN) status = PA_EBREAKDOWN;
    else if (rc_loop) return rc_loop;
    int rc = op_apply_async(L0.op, s->xin, s->t, false, st, nullptr);
    if (rc) return rc;
    k_sub<double, double, double><<<blocks_for(n), 256, 0, st>>>(s->r, s->bin, s->t, n);
    k_norm2<double><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, s->r, n, S_RR);
    PA_CUDA_TRY(cudaMemcpyAsync(x, s->xin, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    const double rr = read_scalar(s, S_RR, st);
    PA_CUDA_TRY(cudaGetLastError());
    inf->rel_residual = std::sqrt(rr / bb);
    inf->tolerance_met = rr <= tol2 * bb ? 1 : 0;
    inf->coarse_iterations = (int)std::min<int64_t>(s->coarse_its, 0x7fffffff);
    if (status == PA_OK && !converged) status = PA_ENOTCONV;
    inf->status = status;
    if (status == PA_ENOTCONV) set_error(PA_ENOTCONV, "pa_gmg_pcg_solve: iteration cap reached");
    return status;
}

FcgVecs<double> outer_vecs(pa_solver *s) { return FcgVecs<double>{s->xin, s->bin, s->r, s->z, s->p, s->q, false}; }

// Executable graph of the coarse solve alone: a WHILE node whose body is one
// coarse iteration; the condition is set on the device after every
// iteration (stop flag or iteration cap).
int build_coarse_graph(pa_solver *s, cudaStream_t st, cudaGraphExec_t *out)
{
    cudaGraph_t G = nullptr, gBody = nullptr;
    int rc = PA_OK;
    do {
        cudaError_t e = cudaGraphCreate(&G, 0);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaGraphCreate"); break; }
        cudaGraphConditionalHandle h;
        e = cudaGraphConditionalHandleCreate(&h, G, 1, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaGraphConditionalHandleCreate"); break; }
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t nC, nBody;
        e = cudaGraphAddNode(&nC, G, nullptr, nullptr, 0, &cp);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaGraphAddNode(conditional)"); break; }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        Level &Lc = s->lv.back();
        const int maxit = s->coarse_maxit;
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaStreamBeginCapture"); break; }
        int r = coarse_iter(s, Lc, st);
        if (!r) k_cg_cond<<<1, 32, 0, st>>>(s->dev, maxit, h);
        e = cudaStreamEndCapture(st, &gBody);
        if (r) { rc = r; break; }
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaStreamEndCapture"); break; }
        e = cudaGraphAddChildGraphNode(&nBody, body, nullptr, 0, gBody);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaGraphAddChildGraphNode(body)"); break; }
        e = cudaGraphInstantiate(out, G, 0);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaGraphInstantiate"); break; }
    } while (false);
    if (gBody) cudaGraphDestroy(gBody);
    if (G) cudaGraphDestroy(G);
    return rc;
}

// ------------------------------------------------------------ lockstep
// Several solvers advanced together, one flexible-CG step per tick.  Each
// solver's step is captured once per phase (the kernels between two
// operator applies) into small executable graphs on its own stream; a tick
// runs phase j of every member, then the applies that end phase j -- one per
// member, all on the same level -- as one batched launch per (precision,
// degree) on the lockstep's stream, then phase j + 1.  The coarse solve of
// each member is its own device-controlled loop between the two halves of
// the step.  Members join and leave between ticks.  The kernels, their
// order per member and the applies' arithmetic are those of the solver's
// own step, so a member's iterates are bitwise those of its solo solve.
struct ApplyRec {
    pa_op *op = nullptr;
    const void *x = nullptr;
    void *y = nullptr;
};

struct Segment {
    std::vector<cudaGraphExec_t> g;  // per phase (null: nothing to launch)
    std::vector<ApplyRec> ap;        // apply ending each phase but the last (op null: none)
};

struct LockMember {
    pa_solver *s = nullptr;
    double *x_out = nullptr;
    void *tag = nullptr;
    double bb = 0.0, tol2 = 0.0;
    int maxit = 0, it = 0;
    bool started = false;
    cudaEvent_t ev = nullptr;
    Segment a[2], b[2];  // [0] first step, [1] iteration step
    cudaGraphExec_t coarse = nullptr;
    pa_solve_info info{};
};

void free_segment(Segment &sg)
{
    for (cudaGraphExec_t g : sg.g)
        if (g) cudaGraphExecDestroy(g);
    sg.g.clear();
    sg.ap.clear();
}

void free_member(LockMember &m)
{
    for (int k = 0; k < 2; ++k) {
        free_segment(m.a[k]);
        free_segment(m.b[k]);
    }
    if (m.coarse) cudaGraphExecDestroy(m.coarse);
    if (m.ev) cudaEventDestroy(m.ev);
    m.coarse = nullptr;
    m.ev = nullptr;
}

// Captures every phase of a step segment of solver s into sg.
template <typename F>
int capture_segment(pa_solver *s, F fn, Segment &sg)
{
    cudaStream_t st = s->stream;
    s->ph_on = true;
    s->ph_target = -1;  // count the phases: nothing is emitted
    s->ph_counter = 0;
    int rc = fn();
    const int napply = s->ph_counter;
    for (int j = 0; !rc && j <= napply; ++j) {
        s->ph_target = j;
        s->ph_counter = 0;
        s->ph_op = nullptr;
        s->ph_x = nullptr;
        s->ph_y = nullptr;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            rc = cuda_error(e, "lockstep: cudaStreamBeginCapture");
            break;
        }
        int r = fn();
        e = cudaStreamEndCapture(st, &g);
        if (!r && e != cudaSuccess) r = cuda_error(e, "lockstep: cudaStreamEndCapture");
        if (!r && s->ph_counter != napply) r = set_error(PA_EINVAL, "lockstep: step phases differ between captures");
        cudaGraphExec_t ex = nullptr;
        if (!r) {
            size_t nn = 0;
            e = cudaGraphGetNodes(g, nullptr, &nn);
            if (e != cudaSuccess) r = cuda_error(e, "lockstep: cudaGraphGetNodes");
            else if (nn > 0 && (e = cudaGraphInstantiate(&ex, g, 0)) != cudaSuccess)
                r = cuda_error(e, "lockstep: cudaGraphInstantiate");
        }
        if (g) cudaGraphDestroy(g);
        if (r) {
            rc = r;
            break;
        }
        sg.g.push_back(ex);
        if (j < napply) sg.ap.push_back(ApplyRec{s->ph_op, s->ph_x, s->ph_y});
    }
    s->ph_on = false;
    return rc;
}

template <typename TP>
int capture_member(LockMember &m)
{
    pa_solver *s = m.s;
    FcgVecs<double> v = outer_vecs(s);
    const cudaStream_t st = s->stream;
    int rc = capture_segment(s, [&]() { return fcg_init_a<double, TP>(s, v, st); }, m.a[0]);
    if (!rc) rc = capture_segment(s, [&]() { return fcg_iter_a<double, TP>(s, v, st); }, m.a[1]);
    if (!rc) rc = capture_segment(s, [&]() { return fcg_init_b<double, TP>(s, v, st); }, m.b[0]);
    if (!rc) rc = capture_segment(s, [&]() { return fcg_iter_b<double, TP>(s, v, st); }, m.b[1]);
    if (!rc && (m.a[0].g.size() != m.a[1].g.size() || m.b[0].g.size() != m.b[1].g.size()))
        rc = set_error(PA_EINVAL, "lockstep: first and later steps have different phases");
    if (!rc) rc = build_coarse_graph(s, st, &m.coarse);
    return rc;
}

}  // namespace

struct Lockstep {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<LockMember> m;
    std::vector<LockstepDone> done;
};

namespace {

// Finishes member m (true residual, solution copy) into L.done.
void retire(Lockstep &L, LockMember &m, int rc_loop, bool converged)
{
    LockstepDone d;
    d.tag = m.tag;
    m.info.iterations = m.it;
    int st = solve_finish(m.s, m.x_out, rc_loop, converged, m.bb, m.tol2, &m.info);
    d.status = st;
    if (st != PA_OK) d.error = pa_last_error();
    d.info = m.info;
    L.done.push_back(d);
    free_member(m);
}

// Runs phases 0 .. n-1 of one segment kind for all members, batching the
// applies between phases; the last phase is launched but not joined.
int run_segment(Lockstep &L, bool second_half)
{
    // members may have different hierarchies, so different numbers of
    // phases: phase round j runs phase j of every member that has one, then
    // the applies that end those phases as one batched launch
    auto seg = [&](LockMember &m) -> Segment & {
        return second_half ? m.b[m.started ? 1 : 0] : m.a[m.started ? 1 : 0];
    };
    size_t nph = 0;
    for (LockMember &m : L.m) nph = std::max(nph, seg(m).g.size());
    std::vector<pa_op *> ops;
    std::vector<const void *> xs;
    std::vector<void *> ys;
    for (size_t j = 0; j < nph; ++j) {
        for (LockMember &m : L.m) {
            Segment &sg = seg(m);
            if (j < sg.g.size() && sg.g[j]) PA_CUDA_TRY(cudaGraphLaunch(sg.g[j], m.s->stream));
        }
        ops.clear();
        xs.clear();
        ys.clear();
        for (LockMember &m : L.m) {
            Segment &sg = seg(m);
            if (j + 1 >= sg.g.size()) continue;  // its last phase (or none): no apply follows
            const ApplyRec &ap = sg.ap[j];
            if (!ap.op) continue;
            PA_CUDA_TRY(cudaEventRecord(m.ev, m.s->stream));
            PA_CUDA_TRY(cudaStreamWaitEvent(L.st, m.ev, 0));
            ops.push_back(ap.op);
            xs.push_back(ap.x);
            ys.push_back(ap.y);
        }
        if (ops.empty()) continue;
        int rc = apply_batch_async(ops.data(), xs.data(), ys.data(), (int)ops.size(), L.st);
        if (rc) return rc;
        PA_CUDA_TRY(cudaEventRecord(L.ev, L.st));
        for (LockMember &m : L.m) {
            Segment &sg = seg(m);
            if (j + 1 < sg.g.size() && sg.ap[j].op) PA_CUDA_TRY(cudaStreamWaitEvent(m.s->stream, L.ev, 0));
        }
    }
    return PA_OK;
}

}  // namespace

int lockstep_create(Lockstep **out)
{
    *out = nullptr;
    Lockstep *L = new (std::nothrow) Lockstep;
    if (!L) return set_error(PA_ENOMEM, "lockstep: host allocation");
    cudaError_t e = cudaStreamCreateWithFlags(&L->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        lockstep_destroy(L);
        return cuda_error(e, "lockstep: stream or event creation");
    }
    *out = L;
    return PA_OK;
}

void lockstep_destroy(Lockstep *L)
{
    if (!L) return;
    for (LockMember &m : L->m) free_member(m);
    if (L->ev) cudaEventDestroy(L->ev);
    if (L->st) cudaStreamDestroy(L->st);
    delete L;
}

int lockstep_active(const Lockstep *L) { return (int)L->m.size(); }

void lockstep_take_done(Lockstep *L, std::vector<LockstepDone> &out)
{
    for (LockstepDone &d : L->done) out.push_back(d);
    L->done.clear();
}

int lockstep_add(Lockstep *L, pa_solver *s, const double *b, double *x, double rtol, int maxit, void *tag)
{
    if (s->mode != PA_SOLVE_FP64 && s->mode != PA_SOLVE_MIXED_FCG)
        return set_error(PA_EINVAL, "lockstep: only the flexible-CG modes (FP64, MIXED_FCG) step in lockstep");
    // a grid-wide persistent coarse kernel must not run beside other members
    s->allow_coop = false;
    LockMember m;
    m.s = s;
    m.x_out = x;
    m.tag = tag;
    m.maxit = maxit;
    m.tol2 = rtol * rtol;
    bool trivial = false;
    int rc = solve_begin(s, b, x, &m.bb, &m.info, &trivial);
    if (rc || trivial) {
        LockstepDone d;
        d.tag = tag;
        d.status = rc;
        if (rc) d.error = pa_last_error();
        d.info = m.info;
        d.info.status = rc;
        L->done.push_back(d);
        return PA_OK;
    }
    rc = s->mode == PA_SOLVE_FP64 ? capture_member<double>(m) : capture_member<float>(m);
    if (!rc && cudaEventCreateWithFlags(&m.ev, cudaEventDisableTiming) != cudaSuccess)
        rc = cuda_error(cudaGetLastError(), "lockstep: cudaEventCreate");
    if (rc) {
        free_member(m);
        return rc;
    }
    L->m.push_back(m);
    return PA_OK;
}

void solver_set_cancel(pa_solver *s, const std::atomic<int> *flag) { s->cancel = flag; }

int lockstep_cancel(Lockstep *L, void *tag)
{
    for (size_t i = 0; i < L->m.size(); ++i) {
        if (L->m[i].tag != tag) continue;
        LockMember m = L->m[i];
        L->m.erase(L->m.begin() + (std::ptrdiff_t)i);
        retire(*L, m, set_error(PA_ECANCELED, "solver: solve canceled"), false);
        return PA_OK;
    }
    return set_error(PA_EINVAL, "lockstep: no member with this tag");
}

// Members of any hierarchy step together; one lockstep per solve mode keeps
// each lane's members of one precision mix.
int lockstep_key(const pa_solver *s) { return s->mode; }

int lockstep_tick(Lockstep *L)
{
    if (L->m.empty()) return PA_OK;
    int rc = run_segment(*L, false);
    if (rc) return rc;
    for (LockMember &m : L->m) PA_CUDA_TRY(cudaGraphLaunch(m.coarse, m.s->stream));
    rc = run_segment(*L, true);
    if (rc) return rc;
    for (LockMember &m : L->m) PA_CUDA_TRY(cudaStreamSynchronize(m.s->stream));
    // convergence test of every member, as in the solo loop
    std::vector<LockMember> keep;
    for (LockMember &m : L->m) {
        pa_solver *s = m.s;
        const double rr = s->h_scal[S_RR];
        s->coarse_its += s->h_flag[F_CIT];
        if (m.started) ++m.it;
        m.started = true;
        if (s->h_flag[F_CTIMEOUT]) {
            retire(*L, m, set_error(PA_ETIMEOUT, "solver: coarse-solve grid barrier timed out"), false);
            continue;
        }
        if (s->h_flag[F_BREAK]) {
            retire(*L, m,
                   set_error(PA_EBREAKDOWN, m.it == 0 ? "solver: non-finite value in the first preconditioned residual"
                                                      : "solver: CG breakdown (p^T A p <= 0 or non-finite value)"),
                   false);
            continue;
        }
        if (rr <= m.tol2 * m.bb || m.it >= m.maxit) {
            retire(*L, m, PA_OK, rr <= m.tol2 * m.bb);
            continue;
        }
        keep.push_back(m);
    }
    L->m.swap(keep);
    return PA_OK;
}

namespace {
}  // namespace
}  // namespace pa

using namespace pa;

extern "C" {

int pa_op_assemble_p1(const pa_op *op, double *vals, void *stream)
{
    if (!op || !vals) return set_error(PA_EINVAL, "pa_op_assemble_p1: null argument");
    if (op->p != 1 || op->precision != PA_FP64) return set_error(PA_EINVAL, "pa_op_assemble_p1: needs an FP64 p = 1 operator");
    const Basis1D &bb = op->basis;
    P1Tables t{};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            for (int q = 0; q < bb.Q; ++q) {
                const double w = bb.qwts[q];
                t.M[i][j] += w * bb.B[i * bb.Q + q] * bb.B[j * bb.Q + q];
                t.C[i][j] += w * bb.G[i * bb.Q + q] * bb.B[j * bb.Q + q];
                t.K[i][j] += w * bb.G[i * bb.Q + q] * bb.G[j * bb.Q + q];
            }
    const int64_t n = op->ndofs();
    k_assemble_p1<<<blocks_for(n, 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const double *>(op->d_geo), vals, t, op->g);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

// p = 1 on both sides and the fine mesh twice as fine in every direction:
// the h-transfer (natural injection of the trilinear space)
static bool h_pair(const pa_op *c, const pa_op *f)
{
    return c->p == 1 && f->p == 1 && f->g.nx == 2 * c->g.nx && f->g.ny == 2 * c->g.ny && f->g.nz == 2 * c->g.nz;
}

static int transfer_check(const pa_op *c, const pa_op *f)
{
    if (!c || !f) return set_error(PA_EINVAL, "transfer: null operator");
    if (c->precision != PA_FP64 || f->precision != PA_FP64) return set_error(PA_EINVAL, "transfer: FP64 operators only");
    if (h_pair(c, f)) return PA_OK;
    if (c->g.nx != f->g.nx || c->g.ny != f->g.ny || c->g.nz != f->g.nz)
        return set_error(PA_EINVAL, "transfer: operators live on different meshes");
    if (!(c->p < f->p)) return set_error(PA_EINVAL, "transfer: coarse degree must be below fine degree");
    return PA_OK;
}

static XferTab transfer_table(const pa_op *c, const pa_op *f)
{
    XferTab t{};
    std::vector<double> val((size_t)(c->p + 1) * (f->p + 1)), der(val.size());
    lagrange_product(c->p + 1, c->basis.nodes.data(), f->p + 1, f->basis.nodes.data(), val.data(), der.data());
    for (size_t i = 0; i < val.size(); ++i) t.L[i] = std::fabs(val[i]) < 1e-15 ? 0.0 : val[i];
    return t;
}

int pa_op_prolong(const pa_op *coarse, const pa_op *fine, const double *xc, double *xf, void *stream)
{
    int rc = transfer_check(coarse, fine);
    if (rc) return rc;
    if (!xc || !xf) return set_error(PA_EINVAL, "pa_op_prolong: null vector");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (h_pair(coarse, fine)) {
        PA_CUDA_TRY(cudaMemsetAsync(xf, 0, sizeof(double) * (size_t)fine->ndofs(), st));
        k_hprolong_add<double><<<blocks_for(fine->ndofs()), 256, 0, st>>>(xf, xc, fine->g, coarse->g);
        PA_CUDA_TRY(cudaGetLastError());
        return PA_OK;
    }
    Level F, C;
    F.op = const_cast<pa_op *>(fine);
    F.p = fine->p;
    C.op = const_cast<pa_op *>(coarse);
    C.p = coarse->p;
    F.xt = transfer_table(coarse, fine);
    // the fine operator's staging vectors serve as sweep temporaries
    F.xa = static_cast<double *>(fine->d_xh);
    F.xb = static_cast<double *>(fine->d_yh);
    PA_CUDA_TRY(cudaMemsetAsync(xf, 0, sizeof(double) * (size_t)fine->ndofs(), st));
    prolong_add<double>(F, C, xc, xf, st);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

int pa_op_restrict(const pa_op *coarse, const pa_op *fine, const double *rf, double *rc_out, void *stream)
{
    int rc = transfer_check(coarse, fine);
    if (rc) return rc;
    if (!rf || !rc_out) return set_error(PA_EINVAL, "pa_op_restrict: null vector");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (h_pair(coarse, fine)) {
        k_hrestrict<double><<<row3_blocks(coarse->ndofs()), 128, 0, st>>>(rc_out, rf, nullptr, fine->g, coarse->g, nullptr);
        PA_CUDA_TRY(cudaGetLastError());
        return PA_OK;
    }
    Level F, C;
    F.op = const_cast<pa_op *>(fine);
    F.p = fine->p;
    pa_op cmask_free = pa_op();  // restriction without essential masking
    cmask_free.d_ess = nullptr;
    C.op = &cmask_free;
    C.p = coarse->p;
    F.xt = transfer_table(coarse, fine);
    F.xa = static_cast<double *>(fine->d_xh);
    F.xb = static_cast<double *>(fine->d_yh);
    restrict_to<double>(F, C, rf, nullptr, rc_out, st);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

int pa_solver_destroy(pa_solver *s)
{
    if (!s) return PA_OK;
    for (auto &L : s->lv) {
        if (L.own_op) pa_op_destroy(L.op);
        pa_op_destroy(L.op32);
    }
    for (StepGraphs *g : {&s->g64, &s->g32, &s->gmx}) {
        if (g->init) cudaGraphExecDestroy(g->init);
        if (g->iter) cudaGraphExecDestroy(g->iter);
    }
    if (s->stream) cudaStreamDestroy(s->stream);
    for (void *p : s->allocs) cudaFree(p);
    cudaFree(s->dev.scal);
    cudaFree(s->dev.flag);
    cudaFree(s->dev.partial);
    cudaFree(s->dev.counter);
    cudaFreeHost(s->h_scal);
    cudaFreeHost(s->h_flag);
    delete s;
    return PA_OK;
}

int pa_solver_create(pa_op *fine, int nlev, const int *p_levels, int cheb_order, double coarse_rtol, int coarse_maxit,
                     int mode, pa_solver **out)
{
    return pa_solver_create_hp(fine, nlev, p_levels, 0, cheb_order, coarse_rtol, coarse_maxit, mode, out);
}

int pa_solver_create_hp(pa_op *fine, int nlev, const int *p_levels, int h_levels, int cheb_order, double coarse_rtol,
                        int coarse_maxit, int mode, pa_solver **out)
{
    if (!out) return set_error(PA_EINVAL, "pa_solver_create: null output");
    *out = nullptr;
    if (!fine || !p_levels || nlev < 1 || nlev > 8) return set_error(PA_EINVAL, "pa_solver_create: bad levels");
    if (h_levels < 0 || nlev + h_levels > 8) return set_error(PA_EINVAL, "pa_solver_create: at most 8 levels in all");
    if (h_levels > 0 && p_levels[nlev - 1] != 1)
        return set_error(PA_EINVAL, "pa_solver_create: h-levels need the last degree to be 1");
    if (fine->precision != PA_FP64) return set_error(PA_EINVAL, "pa_solver_create: fine operator must be FP64");
    if (p_levels[0] != fine->p) return set_error(PA_EINVAL, "pa_solver_create: p_levels[0] must be the fine degree");
    for (int l = 1; l < nlev; ++l)
        if (p_levels[l] >= p_levels[l - 1] || p_levels[l] < 1)
            return set_error(PA_EINVAL, "pa_solver_create: degrees must decrease");
    if (cheb_order < 1 || cheb_order > 8) return set_error(PA_EINVAL, "pa_solver_create: cheb_order in 1..8");
    if (coarse_maxit < 1 || !(coarse_rtol >= 0.0)) return set_error(PA_EINVAL, "pa_solver_create: bad coarse parameters");
    if (mode != PA_SOLVE_FP64 && mode != PA_SOLVE_MIXED && mode != PA_SOLVE_MIXED_FCG)
        return set_error(PA_EINVAL, "pa_solver_create: bad mode");
    const bool fp32_levels = mode != PA_SOLVE_FP64;

    pa_solver *s = new (std::nothrow) pa_solver;
    if (!s) return set_error(PA_ENOMEM, "pa_solver_create: host allocation");
    s->mode = mode;
    s->cheb_order = cheb_order;
    s->coarse_rtol = coarse_rtol;
    s->coarse_maxit = coarse_maxit;
    int rc = PA_OK;
#define TRY(x)                        \
    do {                              \
        rc = (x);                     \
        if (rc) {                     \
            pa_solver_destroy(s);     \
            return rc;                \
        }                             \
    } while (0)
#define TRYC(x) TRY(((x) == cudaSuccess) ? PA_OK : cuda_error(cudaGetLastError(), #x))
    TRYC(cudaMalloc((void **)&s->dev.scal, sizeof(double) * NSLOT));
    TRYC(cudaMalloc((void **)&s->dev.flag, sizeof(int) * NFLAG));
    TRYC(cudaMalloc((void **)&s->dev.partial, sizeof(double) * 3 * kRedBlocks));
    TRYC(cudaMalloc((void **)&s->dev.counter, sizeof(unsigned)));
    TRYC(cudaMemset(s->dev.counter, 0, sizeof(unsigned)));
    TRYC(cudaMemset(s->dev.flag, 0, sizeof(int) * NFLAG));
    TRYC(cudaMemset(s->dev.scal, 0, sizeof(double) * NSLOT));
    TRYC(cudaMallocHost((void **)&s->h_scal, sizeof(double) * NSLOT));
    TRYC(cudaMallocHost((void **)&s->h_flag, sizeof(int) * NFLAG));
    TRYC(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    TRY(dalloc(s, &s->bar, 2));
    TRY(dalloc(s, &s->coop_part, 9 * (int64_t)kRedBlocks));
    {
        int dev = 0, coop = 0, nsm = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_coop, 256, 0) == cudaSuccess)
            s->coop_blocks = std::min(kCoopBlocks, per_sm * nsm);
        int khz = 0;
        if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) == cudaSuccess && khz > 0) s->clock_khz = khz;
        s->wait_cycles = (long long)(2.0 * s->clock_khz * 1e3);
        cudaGetLastError();
    }

    const int ntot = nlev + h_levels;
    s->lv.resize(ntot);
    std::vector<uint8_t> mask = fine->h_ess;
    LevelMesh cur = mesh_of(fine);  // mesh of the level being built
    for (int l = 0; l < ntot; ++l) {
        Level &L = s->lv[l];
        L.p = l < nlev ? p_levels[l] : 1;
        if (l == 0) {
            L.op = fine;
        } else if (l < nlev) {
            // p-coarsening: same mesh, lower degree
            const pa_op *F = s->lv[l - 1].op;
            if (!mask.empty()) {
                Basis1D bc;
                bc.build(L.p, L.p + 2);
                mask = coarse_mask(mask, F->g, L.p, bc, F->basis);
            }
            TRY(make_level_op(cur, L.p, PA_FP64, mask, &L.op));
            L.own_op = true;
        } else {
            // h-coarsening: p = 1 on the mesh whose uniform refinement is the level above
            const pa_op *F = s->lv[l - 1].op;
            LevelMesh c;
            TRY(coarsen_mesh(cur, c));
            if (!mask.empty()) {
                Grid gc{};
                gc.nx = c.nx;
                gc.ny = c.ny;
                gc.nz = c.nz;
                gc.p = 1;
                gc.Mx = c.nx + 1;
                gc.My = c.ny + 1;
                gc.Mz = c.nz + 1;
                gc.ne = (int64_t)c.nx * c.ny * c.nz;
                gc.Nn = (int64_t)gc.Mx * gc.My * gc.Mz;
                mask = h_coarse_mask(mask, F->g, gc);
            }
            cur = std::move(c);
            TRY(make_level_op(cur, 1, PA_FP64, mask, &L.op));
            L.own_op = true;
            s->lv[l - 1].hdown = true;
        }
        L.n = L.op->ndofs();
        if (fp32_levels) TRY(make_level_op(cur, L.p, PA_FP32, L.op->h_ess, &L.op32));
    }
    const int nlev_all = ntot;
    cudaStream_t st = s->stream;
    for (int l = 0; l < nlev_all; ++l) {
        Level &L = s->lv[l];
        const int64_t n = L.n;
        TRY(dalloc(s, &L.dinv, n));
        TRY(dalloc(s, &L.r, n));
        TRY(dalloc(s, &L.e, n));
        TRY(dalloc(s, &L.t, n));
        TRY(dalloc(s, &L.d, n));
        TRY(pa_op_diag(L.op, L.t, st));
        k_recip<double><<<blocks_for(n), 256, 0, st>>>(L.dinv, L.t, n);
        if (l < nlev_all - 1) {
            TRY(dalloc(s, &L.xa, n));
            TRY(dalloc(s, &L.xb, n));
            if (!L.hdown) {
                const int pc = p_levels[l + 1];
                Basis1D bc;
                bc.build(pc, pc + 2);
                std::vector<double> val((size_t)(pc + 1) * (L.p + 1)), der(val.size());
                lagrange_product(pc + 1, bc.nodes.data(), L.p + 1, L.op->basis.nodes.data(), val.data(), der.data());
                for (size_t i = 0; i < val.size(); ++i) L.xt.L[i] = std::fabs(val[i]) < 1e-15 ? 0.0 : val[i];
            }
            TRY(estimate_lmax(s, L, st));
        } else {
            TRY(dalloc(s, &L.cx, n));
            TRY(dalloc(s, &L.cr, n));
            TRY(dalloc(s, &L.cp, n));
            TRY(dalloc(s, &L.cq, n));
            if (L.p == 1 && L.op->g.Nn < (1LL << 30) && L.op->h_cv.empty()) {
                // assemble the coarse matrix (same quadrature as the operator);
                // its kernels index nodes in 32 bits
                TRY(dalloc(s, &L.stencil, 81 * n));
                TRY(pa_op_assemble_p1(L.op, L.stencil, st));
                k_mask_stencil<<<blocks_for(n, 128), 128, 0, st>>>(L.stencil, L.op->d_ess, L.op->g);
            }
        }
        if (fp32_levels) {
            TRY(dalloc(s, &L.r32, n));
            TRY(dalloc(s, &L.e32, n));
            TRY(dalloc(s, &L.dinv32, n));
            TRY(dalloc(s, &L.t32, n));
            TRY(dalloc(s, &L.d32, n));
            TRY(dalloc(s, &L.xa32, n));
            TRY(dalloc(s, &L.xb32, n));
            k_scale_copy<double, float><<<blocks_for(n), 256, 0, st>>>(L.dinv32, L.dinv, 1.0, n);
            // one eager apply per FP32 operator before any graph capture
            TRY(op_apply_async(L.op32, L.dinv32, L.t32, false, st, nullptr));
        }
    }
    if (s->lv.back().stencil) TRY(build_h_levels(s, st));
    const int64_t n0 = s->lv[0].n;
    TRY(dalloc(s, &s->xin, n0));
    TRY(dalloc(s, &s->bin, n0));
    TRY(dalloc(s, &s->r, n0));
    TRY(dalloc(s, &s->z, n0));
    TRY(dalloc(s, &s->p, n0));
    TRY(dalloc(s, &s->q, n0));
    TRY(dalloc(s, &s->t, n0));
    if (mode == PA_SOLVE_MIXED) {
        TRY(dalloc(s, &s->r32, n0));
        TRY(dalloc(s, &s->z32, n0));
        TRY(dalloc(s, &s->p32, n0));
        TRY(dalloc(s, &s->q32, n0));
        TRY(dalloc(s, &s->x32, n0));
        TRY(dalloc(s, &s->b32, n0));
    }
    TRYC(cudaStreamSynchronize(st));
    TRYC(cudaGetLastError());
#undef TRY
#undef TRYC
    *out = s;
    clear_error();
    return PA_OK;
}

int pa_solver_set_option(pa_solver *s, int option, double value)
{
    if (!s) return set_error(PA_EINVAL, "pa_solver_set_option: null solver");
    switch (option) {
    case PA_SOLVER_OPT_GRAPHS:
    case PA_SOLVER_OPT_PERSISTENT_COARSE:
    case PA_SOLVER_OPT_COARSE_HMG: {
        // both change what the step graphs contain: drop any built graphs
        for (StepGraphs *g : {&s->g64, &s->g32, &s->gmx}) {
            if (g->init) cudaGraphExecDestroy(g->init);
            if (g->iter) cudaGraphExecDestroy(g->iter);
            g->init = g->iter = nullptr;
        }
        if (option == PA_SOLVER_OPT_GRAPHS) s->use_graphs = value != 0.0;
        else if (option == PA_SOLVER_OPT_PERSISTENT_COARSE) s->allow_coop = value != 0.0;
        else s->use_hmg = value != 0.0;
        return PA_OK;
    }
    case PA_SOLVER_OPT_CHEB_LOWER:
    case PA_SOLVER_OPT_CHEB_UPPER:
    case PA_SOLVER_OPT_POWER_ITERS: {
        if (option == PA_SOLVER_OPT_POWER_ITERS) {
            if (!(value >= 1.0 && value <= 1000.0)) return set_error(PA_EINVAL, "pa_solver_set_option: power iterations in 1..1000");
        } else {
            const double lo = option == PA_SOLVER_OPT_CHEB_LOWER ? value : s->cheb_lo;
            const double hi = option == PA_SOLVER_OPT_CHEB_UPPER ? value : s->cheb_hi;
            if (!(lo > 0.0) || !(hi > lo) || !(hi < 100.0))
                return set_error(PA_EINVAL, "pa_solver_set_option: need 0 < lower < upper < 100 (fractions of lambda_max)");
        }
        // the step graphs hold the Chebyshev coefficients as kernel arguments
        for (StepGraphs *g : {&s->g64, &s->g32, &s->gmx}) {
            if (g->init) cudaGraphExecDestroy(g->init);
            if (g->iter) cudaGraphExecDestroy(g->iter);
            g->init = g->iter = nullptr;
        }
        if (option == PA_SOLVER_OPT_CHEB_LOWER) s->cheb_lo = value;
        else if (option == PA_SOLVER_OPT_CHEB_UPPER) s->cheb_hi = value;
        else s->power_its = (int)value;
        cudaStream_t st = s->stream;
        // smoothed levels are the ones with an estimate (the assembled p = 1
        // level is solved, not smoothed; the last h-level is a dense solve)
        for (Level &L : s->lv) {
            if (!(L.lmax > 0.0)) continue;
            if (option == PA_SOLVER_OPT_POWER_ITERS) {
                if (int rc = estimate_lmax(s, L, st)) return rc;
            } else {
                cheb_interval(s, L.lmax, &L.theta, &L.delta);
            }
        }
        for (HLevel &H : s->hl) {
            if (!(H.lmax > 0.0)) continue;
            if (option == PA_SOLVER_OPT_POWER_ITERS) {
                if (int rc = h_power_lmax(s, H, st)) return rc;
            } else {
                cheb_interval(s, H.lmax, &H.theta, &H.delta);
            }
        }
        PA_CUDA_TRY(cudaStreamSynchronize(st));
        return PA_OK;
    }
    case PA_SOLVER_OPT_WAIT_LIMIT: {
        if (!(value > 0.0 && value <= 60.0)) return set_error(PA_EINVAL, "pa_solver_set_option: wait limit in (0, 60] s");
        // the limit is a kernel argument of the captured step graphs
        for (StepGraphs *g : {&s->g64, &s->g32, &s->gmx}) {
            if (g->init) cudaGraphExecDestroy(g->init);
            if (g->iter) cudaGraphExecDestroy(g->iter);
            g->init = g->iter = nullptr;
        }
        s->wait_cycles = std::max(1LL, (long long)(value * s->clock_khz * 1e3));
        return PA_OK;
    }
    case PA_SOLVER_OPT_INJECT_INNER_FAILURE:
        if (!(value >= 0.0 && value <= 1e6)) return set_error(PA_EINVAL, "pa_solver_set_option: inner-failure index >= 0");
        s->inject_inner_failure = (int)value;
        return PA_OK;
    default: return set_error(PA_EINVAL, "pa_solver_set_option: unknown option");
    }
}

int pa_gmg_pcg_solve(pa_solver *s, const double *b, double *x, double rtol, int maxit, pa_solve_info *info,
                     void *stream)
{
    if (!s || !b || !x) return set_error(PA_EINVAL, "pa_gmg_pcg_solve: null argument");
    if (!(rtol > 0.0) || maxit < 0) return set_error(PA_EINVAL, "pa_gmg_pcg_solve: bad tolerance or cap");
    // the caller's stream first finishes producing b and x; the solve runs on
    // the solver's own stream
    PA_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    cudaStream_t st = s->stream;
    Level &L0 = s->lv[0];
    const int64_t n = L0.n;
    pa_solve_info inf{};
    double bb = 0.0;
    bool trivial = false;
    int rc = solve_begin(s, b, x, &bb, &inf, &trivial);
    if (rc || trivial) {
        if (info) *info = inf;
        return rc;
    }
    double *xs = s->xin, *bs = s->bin;
    const double tol2 = rtol * rtol;
    bool converged = false;
    if (s->mode == PA_SOLVE_FP64 || s->mode == PA_SOLVE_MIXED_FCG) {
        int it = 0;
        FcgVecs<double> v = outer_vecs(s);
        if (s->mode == PA_SOLVE_FP64) rc = fcg<double>(s, v, s->g64, tol2, bb, maxit, &it, st);
        else rc = fcg<double, float>(s, v, s->gmx, tol2, bb, maxit, &it, st);
        inf.iterations = it;
        converged = (rc == PA_OK) && s->h_scal[S_RR] <= tol2 * bb;
    } else {
        // iterative refinement: r = b - A x (FP64), inner FCG in FP32 on A d = r.
        // Stops at the tolerance, or when a refinement step no longer halves
        // the FP64 residual (its rounding floor).
        int total_inner = 0, refine = 0;
        double rr_prev = -1.0;
        bool inner_truncated = false;  // the last inner solve was cut short by maxit
        FcgVecs<float> v{s->x32, s->b32, s->r32, s->z32, s->p32, s->q32, true};
        while (true) {
            rc = op_apply_async(L0.op, xs, s->t, false, st, nullptr);
            if (rc) break;
            k_sub<double, double, double><<<blocks_for(n), 256, 0, st>>>(s->r, bs, s->t, n);
            k_norm2<double><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, s->r, n, S_RR);
            double rr = read_scalar(s, S_RR, st);
            if (!std::isfinite(rr)) {
                rc = set_error(PA_EBREAKDOWN, "solver: non-finite residual");
                break;
            }
            if (rr <= tol2 * bb) {
                converged = true;
                break;
            }
            if (rr_prev >= 0.0 && rr > 0.25 * rr_prev && !inner_truncated && rr <= 1e6 * tol2 * bb) {
                // stagnation within 1e3 of the tolerance: the FP64 residual
                // floor.  Farther away, a refinement step that gained less
                // than 2x (the FP32 inner residual drifted from the true one)
                // is followed by another until the iteration cap.
                converged = true;
                break;
            }
            if (total_inner >= maxit) break;
            rr_prev = rr;
            // the residual scaled to unit norm is the FP32 right-hand side
            const double sc = 1.0 / std::sqrt(rr);
            k_scale_copy<double, float><<<blocks_for(n), 256, 0, st>>>(s->b32, s->r, sc, n);
            int it = 0;
            // inner solve: relative reduction 1e-4 or at most 50 iterations
            const int inner_cap = std::min(50, maxit - total_inner);
            if (s->inject_inner_failure == refine + 1) {
                // host-side fault injection (test hook, one shot): this inner
                // solve reports a breakdown without running
                s->inject_inner_failure = 0;
                rc = set_error(PA_EBREAKDOWN, "solver: inner solve failure injected (PA_SOLVER_OPT_INJECT_INNER_FAILURE)");
                break;
            }
            rc = fcg<float>(s, v, s->g32, 1e-8, 1.0, inner_cap, &it, st);
            if (rc) break;
            inner_truncated = inner_cap < 50 && it == inner_cap;
            total_inner += it;
            ++refine;
            k_axpy<double, float><<<blocks_for(n), 256, 0, st>>>(xs, s->x32, 1.0 / sc, n);
            if (it == 0) break;
        }
        inf.iterations = total_inner;
        inf.inner_iterations = total_inner;
        inf.refinements = refine;
    }
    const int status = solve_finish(s, x, rc, converged, bb, tol2, &inf);
    if (info) *info = inf;
    return status;
}

int pa_gmg_pcg_solve_batch(pa_solver *const *solvers, const double *const *b, double *const *x, int count,
                           double rtol, int maxit, pa_solve_info *infos, void *stream)
{
    if (count < 0 || (count > 0 && (!solvers || !b || !x)))
        return set_error(PA_EINVAL, "pa_gmg_pcg_solve_batch: bad arguments");
    if (!(rtol > 0.0) || maxit < 0) return set_error(PA_EINVAL, "pa_gmg_pcg_solve_batch: bad tolerance or cap");
    for (int k = 0; k < count; ++k) {
        if (!solvers[k] || !b[k] || !x[k]) return set_error(PA_EINVAL, "pa_gmg_pcg_solve_batch: null entry");
        for (int j = 0; j < k; ++j)
            if (solvers[j] == solvers[k]) return set_error(PA_EINVAL, "pa_gmg_pcg_solve_batch: a solver appears twice");
    }
    PA_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    Lockstep *L = nullptr;
    int rc = lockstep_create(&L);
    if (rc) return rc;
    std::vector<int> status(count, PA_OK);
    std::vector<std::string> errors(count);
    for (int k = 0; k < count && !rc; ++k) rc = lockstep_add(L, solvers[k], b[k], x[k], rtol, maxit, (void *)(intptr_t)k);
    while (!rc && lockstep_active(L) > 0) rc = lockstep_tick(L);
    std::vector<LockstepDone> done;
    lockstep_take_done(L, done);
    lockstep_destroy(L);
    if (rc) return rc;
    int first = PA_OK;
    std::string first_err;
    for (const LockstepDone &d : done) {
        const int k = (int)(intptr_t)d.tag;
        if (infos) infos[k] = d.info;
        status[k] = d.status;
        errors[k] = d.error;
    }
    for (int k = 0; k < count; ++k)
        if (status[k] != PA_OK && first == PA_OK) {
            first = status[k];
            first_err = errors[k];
        }
    if (first != PA_OK) set_error(first, first_err);
    return first;
}

}  // extern "C"
