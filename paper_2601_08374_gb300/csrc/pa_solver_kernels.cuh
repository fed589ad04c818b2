// Device kernels and launch helpers of the GMG-PCG solver (internal; each
// translation unit of the solver that launches them includes this header,
// and the kernels it does not use are not instantiated or are dropped).
#pragma once
// a unit need not use every helper defined here
#pragma nv_diag_suppress 177

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "pa_internal.h"

#include "pa_solver_state.h"

namespace pa {
namespace {


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
}  // namespace pa
