// Register-tiled variant of the fused element kernel (same dataflow as
// pa_apply.cuh, Sec. 4.2-4.5).
//
// Every 1D sweep is done by one thread per 1D line: the thread loads the
// line's inputs once into registers and produces all outputs of the line
// with fully unrolled loops, so the 1D tables B, G, Bw, Gw are compile-time
// indexed kernel parameters (constant-bank operands of the FMAs) and each
// shared-memory word read feeds Q (or D) FMAs.  The Z sweep, the pointwise
// stress and the transposed Z sweep are fused per (qx, qy) column: the
// column's 9 x D inputs and 9 x D accumulators live in registers and the
// transposed result overwrites the column in place.
//
// Shared-memory layouts are chosen so that, in both the producing and the
// consuming sweep, the index that varies across the lanes of a warp has an
// odd word stride (no bank conflicts):
//   S0  x_e / y_e staging   [c][iz][iy][ix]      (ix padded to DP, odd)
//   S1  X-sweep out         [c][iz][ch][qx][iy]  (iy padded to DP)
//   S2  Y-sweep out / Z^T   [qy][qx][c][k][iz]   (column stride CS, odd)
//   S3  Y^T-sweep out       [c][iz][iy][k*Q+qx]  (row stride BS = 2Q+1)
// Buffer A holds S0 then S2 then the output staging; buffer B holds S1
// then S3.  The E-vector leaves through a coalesced copy of the staging.
//
// FP32 runs on paired FMA instructions (__ffma2_rn: two fmaf in one
// instruction, the same FMA work in half the issue slots) wherever two sums
// share an operand and their other operands load as pairs: the forward X
// and Y sweeps two quadrature outputs at a time (even Q), the transposed
// sweeps and the Z^T sweep two node outputs at a time, with the weights from
// the transposed tables BwT, GwT.  Each sum keeps its terms and their order,
// so the results are bitwise those of the scalar form.  Measured against the
// scalar form: p = 6 0.0608 -> 0.0540 ms, p = 8 0.0715 -> 0.0658 ms per
// launch on the ~3M-dof sweep meshes.
#pragma once

#include <cstdint>
#include <type_traits>

#include "pa_internal.h"

namespace pa {

// TWO: the fused Z stage runs in two passes (z_columns_2pass) whose
// quadrature values [col][qz][9] (column stride QS, odd) share buffer B.
template <typename T, int D, int Q, bool TWO = false>
struct LineLayout {
    static constexpr int DP = D | 1;                      // odd pitch for ix / iy
    static constexpr int CS = (9 * D) | 1;                // odd column stride of S2
    static constexpr int BS = 2 * Q + 1;                  // odd row stride of S3
    static constexpr int QS = (9 * Q) | 1;                // odd column stride of the quadrature values
    static constexpr int S0 = 3 * D * D * DP;
    static constexpr int S1 = 3 * D * 2 * Q * DP;
    static constexpr int S2 = Q * Q * CS;
    static constexpr int S3 = 3 * D * D * BS;
    static constexpr int SQ = TWO ? Q * Q * QS : 0;
    static constexpr int A = S0 > S2 ? S0 : S2;
    static constexpr int B13 = S1 > S3 ? S1 : S3;
    static constexpr int B = B13 > SQ ? B13 : SQ;
    static constexpr int per_elem = A + B;
    // bytes of the per-CTA element table (global base node of each element),
    // placed after the value buffers
    __host__ __device__ static size_t table_offset(int epb) { return (((size_t)epb * per_elem * sizeof(T)) + 15) & ~(size_t)15; }
};

__device__ __forceinline__ int sel3(int k, int x0, int x1, int x2) { return k == 0 ? x0 : (k == 1 ? x1 : x2); }
template <typename T>
__device__ __forceinline__ T sel3v(int k, T x0, T x1, T x2) { return k == 0 ? x0 : (k == 1 ? x1 : x2); }

// The fused Z stage (Z sweep, pointwise stress of Eq. 7, Q reconstruction,
// Z^T sweep) with one column (el, qx, qy) per three lanes: lane 10 c + k of
// a warp holds the three channels of displacement component c of column
// slot k (3 D inputs and 3 D accumulators instead of 9 D each), lanes 30
// and 31 idle.  At each quadrature point the lanes of a column exchange by
// shuffles the gradient entries the symmetric stress needs: du[c'][c] of
// the other two components and their diagonal entries; lane c = 0 adds the
// divergence in component order and broadcasts it.  Each lane keeps J^-1
// with its columns rotated to the order c, c + 1, c + 2 (mod 3).
template <typename T, int D, int Q, bool ROLLED = false>
__device__ __forceinline__ void z_columns_split(const T *geo0, const Tables<T> &tab, T *bufA, int astride, int ne_blk,
                                                int tid, int nt)
{
    using L = LineLayout<T, D, Q>;
    constexpr int CS = L::CS;
    constexpr int kUnrollQz = ROLLED ? 1 : Q;  // as in z_columns
    // FP32: Z^T on node pairs from the transposed tables, as in z_columns
    constexpr bool PT = sizeof(T) == 4;
    constexpr int NA = PT ? (D + 1) / 2 : D;
    using AccT = std::conditional_t<PT, float2, T>;
    constexpr unsigned kMask = 0x3fffffffu;  // lanes 0..29
    const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
    const int c = lane / 10, slot = lane - 10 * c;
    if (c >= 3) return;
    const int cn = c == 2 ? 0 : c + 1, cp = c == 0 ? 2 : c - 1;
    const int ln = slot + 10 * cn, lp = slot + 10 * cp;
    const int total = ne_blk * Q * Q;
    for (int base = warp * 10; base < total; base += nwarp * 10) {
        const int o = base + slot;
        const bool act = o < total;
        const int oo = act ? o : base;  // a lane past the end works on a valid column and writes nothing
        const int el = oo / (Q * Q), col = oo - el * (Q * Q);
        T *cpt = bufA + (size_t)el * astride + col * CS + c * 3 * D;
        T in[3][D];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int i = 0; i < D; ++i) in[k][i] = cpt[k * D + i];
        const T *geo = geo0 + (size_t)el * kGeoStride;
        T R[3][3];  // R[n][r] = Ji[n][(c + r) mod 3]
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            const T j0 = geo[n * 3 + 0], j1 = geo[n * 3 + 1], j2 = geo[n * 3 + 2];
            R[n][0] = sel3v(c, j0, j1, j2);
            R[n][1] = sel3v(cn, j0, j1, j2);
            R[n][2] = sel3v(cp, j0, j1, j2);
        }
        const T cl = geo[9], cm = geo[10], m2 = cm + cm;
        AccT acc[3][NA];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                if constexpr (PT) acc[k][i] = make_float2(0.f, 0.f);
                else acc[k][i] = T(0);
            }
#pragma unroll(kUnrollQz)
        for (int qz = 0; qz < Q; ++qz) {
            T bq[D], gq[D], bwq[D], gwq[D];
            if constexpr (ROLLED)
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    bq[i] = tab.B[i * Q + qz];
                    gq[i] = tab.G[i * Q + qz];
                    bwq[i] = tab.Bw[i * Q + qz];
                    gwq[i] = tab.Gw[i * Q + qz];
                }
            // unrolled, the tables stay constant-bank operands of the FMAs
            auto tB = [&](int i) { if constexpr (ROLLED) return bq[i]; else return tab.B[i * Q + qz]; };
            auto tG = [&](int i) { if constexpr (ROLLED) return gq[i]; else return tab.G[i * Q + qz]; };
            auto tBw = [&](int i) { if constexpr (ROLLED) return bwq[i]; else return tab.Bw[i * Q + qz]; };
            auto tGw = [&](int i) { if constexpr (ROLLED) return gwq[i]; else return tab.Gw[i * Q + qz]; };
            T g0 = T(0), g1 = T(0), g2 = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                g0 = fma(in[0][i], tB(i), g0);
                g1 = fma(in[1][i], tB(i), g1);
                g2 = fma(in[2][i], tG(i), g2);
            }
            // du[c][(c + r) mod 3]
            const T u0 = fma(R[0][0], g0, fma(R[1][0], g1, R[2][0] * g2));
            const T u1 = fma(R[0][1], g0, fma(R[1][1], g1, R[2][1] * g2));
            const T u2 = fma(R[0][2], g0, fma(R[1][2], g1, R[2][2] * g2));
            const T from_n = __shfl_sync(kMask, u2, ln);  // du[cn][c]
            const T from_p = __shfl_sync(kMask, u1, lp);  // du[cp][c]
            const T dn = __shfl_sync(kMask, u0, ln), dp = __shfl_sync(kMask, u0, lp);
            const T div = __shfl_sync(kMask, (u0 + dn) + dp, slot);  // (du00 + du11) + du22 from lane c = 0
            const T ld = cl * div;
            const T s0 = fma(m2, u0, ld);      // sigma[c][c]
            const T s1 = cm * (u1 + from_n);   // sigma[c][cn]
            const T s2 = cm * (u2 + from_p);   // sigma[c][cp]
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const T qv = fma(s0, R[m][0], fma(s1, R[m][1], s2 * R[m][2]));
                if constexpr (PT) {
                    const float2 qd = make_float2(qv, qv);
                    const float *wt = (m == 2 ? tab.GwT : tab.BwT) + qz * kTStride;
#pragma unroll
                    for (int j = 0; j < NA; ++j)
                        acc[m][j] = __ffma2_rn(qd, make_float2(wt[2 * j], wt[2 * j + 1]), acc[m][j]);
                } else {
#pragma unroll
                    for (int i = 0; i < D; ++i)
                        acc[m][i] = fma(qv, (m == 2 ? tGw(i) : tBw(i)), acc[m][i]);
                }
            }
        }
        if (act)
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int j = 0; j < NA; ++j) {
                    if constexpr (PT) {
                        cpt[k * D + 2 * j] = acc[k][j].x;
                        if (2 * j + 1 < D) cpt[k * D + 2 * j + 1] = acc[k][j].y;
                    } else {
                        cpt[k * D + j] = acc[k][j];
                    }
                }
    }
}

// The fused Z stage with one thread per column (el, qx, qy): the column's
// 9 x D inputs (channels [c][k], k = d/dxi, d/deta, interpolated) and 9 x D
// accumulators in registers; Z sweep, pointwise stress of Eq. 7, Q
// reconstruction and Z^T sweep, the result written back in place.  Columns
// of element el start at bufA + el * astride, column col at col * CS; its
// geometry record at geo0 + el * kGeoStride.
template <typename T, int D, int Q, bool ROLLED = false>
__device__ __forceinline__ void z_columns(const T *geo0, const Tables<T> &tab, T *bufA, int astride, int ne_blk,
                                          int tid, int nt)
{
    constexpr int CS = LineLayout<T, D, Q>::CS;
    // ROLLED: the qz loop is not unrolled (smaller code; the table columns of
    // each qz are loaded once per iteration); same arithmetic either way
    constexpr int kUnrollQz = ROLLED ? 1 : Q;
    // FP32: the Z^T sweep accumulates nodes i, i + 1 of a channel on one
    // paired FMA (__ffma2_rn, two fmaf per instruction) with the weight pair
    // from the transposed tables; for an odd D the last pair's second lane
    // runs on a zero weight and is not stored.  Same terms, same order.
    constexpr bool PT = sizeof(T) == 4;
    constexpr int NA = PT ? (D + 1) / 2 : D;
    using AccT = std::conditional_t<PT, float2, T>;
    for (int o = tid; o < ne_blk * Q * Q; o += nt) {
        int el = o / (Q * Q), col = o - el * Q * Q;  // col = qy*Q + qx
        T *cp = bufA + (size_t)el * astride + col * CS;
        T in[9][D];
#pragma unroll
        for (int ch = 0; ch < 9; ++ch)
#pragma unroll
            for (int i = 0; i < D; ++i) in[ch][i] = cp[ch * D + i];
        const T *geo = geo0 + (size_t)el * kGeoStride;
        T Ji[9], cj[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) Ji[i] = geo[i];
        const T cl = geo[9], cm = geo[10], m2 = cm + cm;
        // mu detJ J^-1: each shear stress is one 6-term dot with it
#pragma unroll
        for (int i = 0; i < 9; ++i) cj[i] = cm * Ji[i];
        AccT acc[9][NA];
#pragma unroll
        for (int ch = 0; ch < 9; ++ch)
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                if constexpr (PT) acc[ch][i] = make_float2(0.f, 0.f);
                else acc[ch][i] = T(0);
            }
#pragma unroll(kUnrollQz)
        for (int qz = 0; qz < Q; ++qz) {
            T bq[D], gq[D], bwq[D], gwq[D];
            if constexpr (ROLLED)
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    bq[i] = tab.B[i * Q + qz];
                    gq[i] = tab.G[i * Q + qz];
                    bwq[i] = tab.Bw[i * Q + qz];
                    gwq[i] = tab.Gw[i * Q + qz];
                }
            // unrolled, the tables stay constant-bank operands of the FMAs
            auto tB = [&](int i) { if constexpr (ROLLED) return bq[i]; else return tab.B[i * Q + qz]; };
            auto tG = [&](int i) { if constexpr (ROLLED) return gq[i]; else return tab.G[i * Q + qz]; };
            auto tBw = [&](int i) { if constexpr (ROLLED) return bwq[i]; else return tab.Bw[i * Q + qz]; };
            auto tGw = [&](int i) { if constexpr (ROLLED) return gwq[i]; else return tab.Gw[i * Q + qz]; };
            T gr[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T g0 = T(0), g1 = T(0), g2 = T(0);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    g0 = fma(in[c * 3 + 0][i], tB(i), g0);
                    g1 = fma(in[c * 3 + 1][i], tB(i), g1);
                    g2 = fma(in[c * 3 + 2][i], tG(i), g2);
                }
                gr[c][0] = g0;
                gr[c][1] = g1;
                gr[c][2] = g2;
            }
            // Voigt stress (Eq. 7): the diagonal of grad u, then each shear
            // stress mu detJ (du_ab + du_ba) as one 6-term dot
            T dg[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) dg[c] = fma(Ji[c], gr[c][0], fma(Ji[3 + c], gr[c][1], Ji[6 + c] * gr[c][2]));
            const T ld = cl * (dg[0] + dg[1] + dg[2]);
            T s[3][3];
            s[0][0] = fma(m2, dg[0], ld);
            s[1][1] = fma(m2, dg[1], ld);
            s[2][2] = fma(m2, dg[2], ld);
            auto shear = [&](int ia, int ib) {
                return fma(cj[ib], gr[ia][0], fma(cj[3 + ib], gr[ia][1], fma(cj[6 + ib], gr[ia][2],
                       fma(cj[ia], gr[ib][0], fma(cj[3 + ia], gr[ib][1], cj[6 + ia] * gr[ib][2])))));
            };
            s[0][1] = s[1][0] = shear(0, 1);
            s[0][2] = s[2][0] = shear(0, 2);
            s[1][2] = s[2][1] = shear(1, 2);
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    T qv = fma(s[c][0], Ji[m * 3 + 0], fma(s[c][1], Ji[m * 3 + 1], s[c][2] * Ji[m * 3 + 2]));
                    if constexpr (PT) {
                        const float2 qd = make_float2(qv, qv);
                        const float *wt = (m == 2 ? tab.GwT : tab.BwT) + qz * kTStride;
#pragma unroll
                        for (int j = 0; j < NA; ++j)
                            acc[c * 3 + m][j] = __ffma2_rn(qd, make_float2(wt[2 * j], wt[2 * j + 1]), acc[c * 3 + m][j]);
                    } else {
#pragma unroll
                        for (int i = 0; i < D; ++i)
                            acc[c * 3 + m][i] = fma(qv, (m == 2 ? tGw(i) : tBw(i)), acc[c * 3 + m][i]);
                    }
                }
        }
#pragma unroll
        for (int ch = 0; ch < 9; ++ch)
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                if constexpr (PT) {
                    cp[ch * D + 2 * j] = acc[ch][j].x;
                    if (2 * j + 1 < D) cp[ch * D + 2 * j + 1] = acc[ch][j].y;
                } else {
                    cp[ch * D + j] = acc[ch][j];
                }
            }
    }
}

// FP32 form of z_columns on paired FMAs (__ffma2_rn: two independent FP32
// FMAs in one instruction, each rounded as one fmaf).  The channels d/dxi
// and d/deta of a component share their Z-sweep weight, and the Q
// reconstructions m = 0, 1 of a component share their Z^T weight, so those
// accumulators advance two at a time; the third channels of components 0
// and 1 pair up the same way, that of component 2 stays scalar.  Every
// accumulator receives the same terms in the same order as in z_columns, so
// the results are bitwise z_columns'.  The paired FMA runs at the scalar
// FMA's rate (measured: 80.4 against 78.6 TFLOP/s over the whole GPU); it
// saves issue slots, not pipe cycles.  The plane kernel (p <= 4) uses this
// form (measured 5-7 % faster); the line kernels keep z_columns, where the
// paired registers cost occupancy (p = 6: 164 -> 182 registers, 16 %
// slower).
template <int D, int Q, bool ROLLED = false>
__device__ __forceinline__ void z_columns_f2(const float *geo0, const Tables<float> &tab, float *bufA, int astride,
                                             int ne_blk, int tid, int nt)
{
    constexpr int CS = LineLayout<float, D, Q>::CS;
    constexpr int kUnrollQz = ROLLED ? 1 : Q;
    for (int o = tid; o < ne_blk * Q * Q; o += nt) {
        int el = o / (Q * Q), col = o - el * Q * Q;  // col = qy*Q + qx
        float *cp = bufA + (size_t)el * astride + col * CS;
        // channel pairs: (c, 0) with (c, 1) for each c; (0, 2) with (1, 2);
        // (2, 2) alone
        float2 in01[3][D], in2p[D];
        float in22[D];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < D; ++i) in01[c][i] = make_float2(cp[(3 * c) * D + i], cp[(3 * c + 1) * D + i]);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            in2p[i] = make_float2(cp[2 * D + i], cp[5 * D + i]);
            in22[i] = cp[8 * D + i];
        }
        const float *geo = geo0 + (size_t)el * kGeoStride;
        float Ji[9], cj[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) Ji[i] = geo[i];
        const float cl = geo[9], cm = geo[10], m2 = cm + cm;
#pragma unroll
        for (int i = 0; i < 9; ++i) cj[i] = cm * Ji[i];
        float2 acc01[3][D], acc2p[D];
        float acc22[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
#pragma unroll
            for (int c = 0; c < 3; ++c) acc01[c][i] = make_float2(0.f, 0.f);
            acc2p[i] = make_float2(0.f, 0.f);
            acc22[i] = 0.f;
        }
#pragma unroll(kUnrollQz)
        for (int qz = 0; qz < Q; ++qz) {
            float bq[D], gq[D], bwq[D], gwq[D];
            if constexpr (ROLLED)
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    bq[i] = tab.B[i * Q + qz];
                    gq[i] = tab.G[i * Q + qz];
                    bwq[i] = tab.Bw[i * Q + qz];
                    gwq[i] = tab.Gw[i * Q + qz];
                }
            auto tB = [&](int i) { if constexpr (ROLLED) return bq[i]; else return tab.B[i * Q + qz]; };
            auto tG = [&](int i) { if constexpr (ROLLED) return gq[i]; else return tab.G[i * Q + qz]; };
            auto tBw = [&](int i) { if constexpr (ROLLED) return bwq[i]; else return tab.Bw[i * Q + qz]; };
            auto tGw = [&](int i) { if constexpr (ROLLED) return gwq[i]; else return tab.Gw[i * Q + qz]; };
            float2 g01[3], g2p = make_float2(0.f, 0.f);
            float g22 = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) g01[c] = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const float b = tB(i), g = tG(i);
#pragma unroll
                for (int c = 0; c < 3; ++c) g01[c] = __ffma2_rn(in01[c][i], make_float2(b, b), g01[c]);
                g2p = __ffma2_rn(in2p[i], make_float2(g, g), g2p);
                g22 = fmaf(in22[i], g, g22);
            }
            float gr[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                gr[c][0] = g01[c].x;
                gr[c][1] = g01[c].y;
            }
            gr[0][2] = g2p.x;
            gr[1][2] = g2p.y;
            gr[2][2] = g22;
            // Voigt stress (Eq. 7), as in z_columns
            float dg[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                dg[c] = fmaf(Ji[c], gr[c][0], fmaf(Ji[3 + c], gr[c][1], Ji[6 + c] * gr[c][2]));
            const float ld = cl * (dg[0] + dg[1] + dg[2]);
            float s[3][3];
            s[0][0] = fmaf(m2, dg[0], ld);
            s[1][1] = fmaf(m2, dg[1], ld);
            s[2][2] = fmaf(m2, dg[2], ld);
            auto shear = [&](int ia, int ib) {
                return fmaf(cj[ib], gr[ia][0], fmaf(cj[3 + ib], gr[ia][1], fmaf(cj[6 + ib], gr[ia][2],
                       fmaf(cj[ia], gr[ib][0], fmaf(cj[3 + ia], gr[ib][1], cj[6 + ia] * gr[ib][2])))));
            };
            s[0][1] = s[1][0] = shear(0, 1);
            s[0][2] = s[2][0] = shear(0, 2);
            s[1][2] = s[2][1] = shear(1, 2);
            float qv[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int m = 0; m < 3; ++m)
                    qv[c][m] = fmaf(s[c][0], Ji[m * 3 + 0], fmaf(s[c][1], Ji[m * 3 + 1], s[c][2] * Ji[m * 3 + 2]));
            const float2 q2 = make_float2(qv[0][2], qv[1][2]);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const float bw = tBw(i), gw = tGw(i);
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    acc01[c][i] = __ffma2_rn(make_float2(qv[c][0], qv[c][1]), make_float2(bw, bw), acc01[c][i]);
                acc2p[i] = __ffma2_rn(q2, make_float2(gw, gw), acc2p[i]);
                acc22[i] = fmaf(qv[2][2], gw, acc22[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cp[(3 * c) * D + i] = acc01[c][i].x;
                cp[(3 * c + 1) * D + i] = acc01[c][i].y;
            }
            cp[2 * D + i] = acc2p[i].x;
            cp[5 * D + i] = acc2p[i].y;
            cp[8 * D + i] = acc22[i];
        }
    }
}

// The fused Z stage in two passes per column, to halve the registers a
// thread holds (9 D inputs, then 9 D accumulators, instead of both): pass 1
// runs the Z sweep, the pointwise stress of Eq. 7 and the Q reconstruction
// and stores the column's 9 quadrature values per point to qbuf; pass 2
// runs the Z^T sweep from them.  Every accumulator receives the same terms
// in the same order as in z_columns, so the results are bitwise the same.
template <typename T, int D, int Q>
__device__ __forceinline__ void z_columns_2pass(const T *geo0, const Tables<T> &tab, T *bufA, int astride, T *qbuf,
                                                int qstride, int ne_blk, int tid, int nt)
{
    constexpr int CS = LineLayout<T, D, Q>::CS;
    constexpr int QS = LineLayout<T, D, Q, true>::QS;
    for (int o = tid; o < ne_blk * Q * Q; o += nt) {
        const int el = o / (Q * Q), col = o - el * Q * Q;  // col = qy*Q + qx
        T *cp = bufA + (size_t)el * astride + col * CS;
        T *qp = qbuf + (size_t)el * qstride + col * QS;
        {
            T in[9][D];
#pragma unroll
            for (int ch = 0; ch < 9; ++ch)
#pragma unroll
                for (int i = 0; i < D; ++i) in[ch][i] = cp[ch * D + i];
            const T *geo = geo0 + (size_t)el * kGeoStride;
            T Ji[9], cj[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) Ji[i] = geo[i];
            const T cl = geo[9], cm = geo[10], m2 = cm + cm;
#pragma unroll
            for (int i = 0; i < 9; ++i) cj[i] = cm * Ji[i];
            // both qz loops stay rolled, with the table columns of one qz
            // loaded per iteration: unrolled, the compiler hoists every
            // point's loads and the register saving is lost
#pragma unroll 1
            for (int qz = 0; qz < Q; ++qz) {
                T bq[D], gq[D];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    bq[i] = tab.B[i * Q + qz];
                    gq[i] = tab.G[i * Q + qz];
                }
                T gr[3][3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    T g0 = T(0), g1 = T(0), g2 = T(0);
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        g0 = fma(in[c * 3 + 0][i], bq[i], g0);
                        g1 = fma(in[c * 3 + 1][i], bq[i], g1);
                        g2 = fma(in[c * 3 + 2][i], gq[i], g2);
                    }
                    gr[c][0] = g0;
                    gr[c][1] = g1;
                    gr[c][2] = g2;
                }
                T dg[3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    dg[c] = fma(Ji[c], gr[c][0], fma(Ji[3 + c], gr[c][1], Ji[6 + c] * gr[c][2]));
                const T ld = cl * (dg[0] + dg[1] + dg[2]);
                T sg[3][3];
                sg[0][0] = fma(m2, dg[0], ld);
                sg[1][1] = fma(m2, dg[1], ld);
                sg[2][2] = fma(m2, dg[2], ld);
                auto shear = [&](int ia, int ib) {
                    return fma(cj[ib], gr[ia][0], fma(cj[3 + ib], gr[ia][1], fma(cj[6 + ib], gr[ia][2],
                           fma(cj[ia], gr[ib][0], fma(cj[3 + ia], gr[ib][1], cj[6 + ia] * gr[ib][2])))));
                };
                sg[0][1] = sg[1][0] = shear(0, 1);
                sg[0][2] = sg[2][0] = shear(0, 2);
                sg[1][2] = sg[2][1] = shear(1, 2);
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int m = 0; m < 3; ++m)
                        qp[qz * 9 + c * 3 + m] =
                            fma(sg[c][0], Ji[m * 3 + 0], fma(sg[c][1], Ji[m * 3 + 1], sg[c][2] * Ji[m * 3 + 2]));
            }
        }
        T acc[9][D];
#pragma unroll
        for (int ch = 0; ch < 9; ++ch)
#pragma unroll
            for (int i = 0; i < D; ++i) acc[ch][i] = T(0);
#pragma unroll 1
        for (int qz = 0; qz < Q; ++qz) {
            T bwq[D], gwq[D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                bwq[i] = tab.Bw[i * Q + qz];
                gwq[i] = tab.Gw[i * Q + qz];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const T qv = qp[qz * 9 + c * 3 + m];
#pragma unroll
                    for (int i = 0; i < D; ++i)
                        acc[c * 3 + m][i] = fma(qv, (m == 2 ? gwq[i] : bwq[i]), acc[c * 3 + m][i]);
                }
        }
#pragma unroll
        for (int ch = 0; ch < 9; ++ch)
#pragma unroll
            for (int i = 0; i < D; ++i) cp[ch * D + i] = acc[ch][i];
    }
}

// FUSE: the gather is done by the X-sweep threads (one contiguous line of D
// values each) and the X^T-sweep threads write their line of the E-vector
// directly, instead of separate gather / store phases through shared memory.
// SPLIT: the fused Z stage runs three lanes per column (z_columns_split).
template <typename T, int D, int Q, bool FUSE, bool SPLIT = false, bool TWO = false>
__device__ __forceinline__ void line_body(const ApplyArgs<T> &a, const Tables<T> &tab, int epb, int64_t blk)
{
    using L = LineLayout<T, D, Q, TWO>;
    constexpr int D3 = D * D * D, DP = L::DP, CS = L::CS, BS = L::BS;
    // FP32, even Q: the forward X and Y sweeps produce two quadrature
    // outputs per paired FMA (__ffma2_rn, two fmaf per instruction)
    constexpr bool kPairQ = sizeof(T) == 4 && Q % 2 == 0;
    // FP32: the transposed Y and X sweeps produce two node outputs per paired
    // FMA, with weight pairs from the transposed tables
    constexpr bool kPairT = sizeof(T) == 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *bufA = reinterpret_cast<T *>(smem_raw);
    T *bufB = bufA + (size_t)epb * L::A;

    if (a.skip && *a.skip) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t e0 = blk * epb;
    const int ne_blk = (int)((a.g.ne - e0) < epb ? (a.g.ne - e0) : epb);
    if (ne_blk <= 0) return;
    const int p = D - 1;
    const int64_t Nn = a.g.Nn;
    const int64_t Mx = a.g.Mx, MxMy = (int64_t)a.g.Mx * a.g.My;
    int64_t *gbase = reinterpret_cast<int64_t *>(smem_raw + L::table_offset(epb));
    for (int el = tid; el < ne_blk; el += nt) {
        // global node of the element's local node (0,0,0): one runtime
        // division per element instead of one per gathered value
        const int64_t e = e0 + el;
        const int64_t t = e / a.g.nx;
        const int ex = (int)(e - t * a.g.nx), ey = (int)(t % a.g.ny), ez = (int)(t / a.g.ny);
        gbase[el] = (int64_t)ex * p + Mx * ((int64_t)ey * p) + MxMy * ((int64_t)ez * p);
    }
    __syncthreads();

    // ---- gather x_e into S0 [c][iz][iy][ix]
    if (!FUSE)
    for (int o = tid; o < ne_blk * 3 * D3; o += nt) {
        int el = o / (3 * D3), r = o - el * 3 * D3;
        int ix = r % D, iy = (r / D) % D, iz = (r / (D * D)) % D, c = r / D3;
        int64_t k = c * Nn + gbase[el] + ix + Mx * iy + MxMy * iz;
        const bool in = PA_INB(a.g, k, 3 * Nn);
        T v = in ? a.x[k] : T(0);
        if (in && a.ess && a.ess[k]) v = T(0);
        bufA[(size_t)el * L::A + ((c * D + iz) * D + iy) * DP + ix] = v;
    }
    if (!FUSE) __syncthreads();

    // ---- X sweep: line (el, c, iz, iy) -> S1 [c][iz][ch][qx][iy]
    for (int o = tid; o < ne_blk * 3 * D * D; o += nt) {
        int el = o / (3 * D * D), r = o - el * 3 * D * D;
        int iy = r % D, iz = (r / D) % D, c = r / (D * D);
        T xv[D];
        if (FUSE) {
            const int64_t k0 = c * Nn + gbase[el] + Mx * iy + MxMy * iz;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const bool in = PA_INB(a.g, k0 + i, 3 * Nn);
                T v = in ? a.x[k0 + i] : T(0);
                if (in && a.ess && a.ess[k0 + i]) v = T(0);
                xv[i] = v;
            }
        } else {
            const T *in = bufA + (size_t)el * L::A + ((c * D + iz) * D + iy) * DP;
#pragma unroll
            for (int i = 0; i < D; ++i) xv[i] = in[i];
        }
        T *out = bufB + (size_t)el * L::B + (c * D + iz) * 2 * Q * DP + iy;
        if constexpr (kPairQ) {
            // outputs q, q + 1 on paired FMAs (table pairs adjacent and
            // 8-byte aligned for an even Q); same sums, same order
            float2 xd[D];
#pragma unroll
            for (int i = 0; i < D; ++i) xd[i] = make_float2(xv[i], xv[i]);
#pragma unroll
            for (int q = 0; q < Q; q += 2) {
                float2 u = make_float2(0.f, 0.f), v = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    u = __ffma2_rn(xd[i], make_float2(tab.B[i * Q + q], tab.B[i * Q + q + 1]), u);
                    v = __ffma2_rn(xd[i], make_float2(tab.G[i * Q + q], tab.G[i * Q + q + 1]), v);
                }
                out[(0 * Q + q) * DP] = u.x;
                out[(0 * Q + q + 1) * DP] = u.y;
                out[(1 * Q + q) * DP] = v.x;
                out[(1 * Q + q + 1) * DP] = v.y;
            }
        } else {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                T u = T(0), v = T(0);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    u = fma(xv[i], tab.B[i * Q + q], u);
                    v = fma(xv[i], tab.G[i * Q + q], v);
                }
                out[(0 * Q + q) * DP] = u;
                out[(1 * Q + q) * DP] = v;
            }
        }
    }
    __syncthreads();

    // ---- Y sweep: line (el, c, iz, qx) -> S2 [qy][qx][c][k][iz]
    for (int o = tid; o < ne_blk * 3 * D * Q; o += nt) {
        int el = o / (3 * D * Q), r = o - el * 3 * D * Q;
        int qx = r % Q, iz = (r / Q) % D, c = r / (Q * D);
        const T *in = bufB + (size_t)el * L::B + (c * D + iz) * 2 * Q * DP + qx * DP;
        T uv[D], vv[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            uv[i] = in[i];
            vv[i] = in[Q * DP + i];
        }
        T *out = bufA + (size_t)el * L::A + qx * CS + (c * 3) * D + iz;
        if constexpr (kPairQ) {
            float2 ud[D], vd[D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                ud[i] = make_float2(uv[i], uv[i]);
                vd[i] = make_float2(vv[i], vv[i]);
            }
#pragma unroll
            for (int q = 0; q < Q; q += 2) {
                float2 d0 = make_float2(0.f, 0.f), d1 = make_float2(0.f, 0.f), d2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    const float2 b2 = make_float2(tab.B[i * Q + q], tab.B[i * Q + q + 1]);
                    d0 = __ffma2_rn(vd[i], b2, d0);                                                  // d/dxi
                    d1 = __ffma2_rn(ud[i], make_float2(tab.G[i * Q + q], tab.G[i * Q + q + 1]), d1);  // d/deta
                    d2 = __ffma2_rn(ud[i], b2, d2);                                                  // interpolated
                }
                T *o2 = out + q * Q * CS;
                o2[0 * D] = d0.x;
                o2[1 * D] = d1.x;
                o2[2 * D] = d2.x;
                o2 += Q * CS;
                o2[0 * D] = d0.y;
                o2[1 * D] = d1.y;
                o2[2 * D] = d2.y;
            }
        } else {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                T d0 = T(0), d1 = T(0), d2 = T(0);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    d0 = fma(vv[i], tab.B[i * Q + q], d0);  // d/dxi
                    d1 = fma(uv[i], tab.G[i * Q + q], d1);  // d/deta
                    d2 = fma(uv[i], tab.B[i * Q + q], d2);  // interpolated, G follows along z
                }
                T *o2 = out + q * Q * CS;
                o2[0 * D] = d0;
                o2[1 * D] = d1;
                o2[2 * D] = d2;
            }
        }
    }
    __syncthreads();

    // ---- Z sweep + pointwise + Z^T sweep: column (el, qx, qy), in place
    const T *geo0 = a.geo + e0 * kGeoStride;  // the tile's geometry records
    if constexpr (SPLIT) z_columns_split<T, D, Q>(geo0, tab, bufA, L::A, ne_blk, tid, nt);
    else if constexpr (TWO) z_columns_2pass<T, D, Q>(geo0, tab, bufA, L::A, bufB, L::B, ne_blk, tid, nt);
    else z_columns<T, D, Q>(geo0, tab, bufA, L::A, ne_blk, tid, nt);
    __syncthreads();

    // ---- Y^T sweep: line (el, c, iz, qx) -> S3 [c][iz][iy][k*Q + qx]
    for (int o = tid; o < ne_blk * 3 * D * Q; o += nt) {
        int el = o / (3 * D * Q), r = o - el * 3 * D * Q;
        int qx = r % Q, iz = (r / Q) % D, c = r / (Q * D);
        const T *in = bufA + (size_t)el * L::A + qx * CS + (c * 3) * D + iz;
        T t0[Q], t1[Q], t2[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const T *col = in + q * Q * CS;
            t0[q] = col[0 * D];
            t1[q] = col[1 * D];
            t2[q] = col[2 * D];
        }
        T *out = bufB + (size_t)el * L::B + ((c * D + iz) * D) * BS + qx;
        if constexpr (kPairT) {
            // outputs iy, iy + 1 on paired FMAs, weight pairs from the
            // transposed tables (an odd D's last second lane unused)
            float2 t0d[Q], t1d[Q], t2d[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                t0d[q] = make_float2(t0[q], t0[q]);
                t1d[q] = make_float2(t1[q], t1[q]);
                t2d[q] = make_float2(t2[q], t2[q]);
            }
#pragma unroll
            for (int iy = 0; iy < D; iy += 2) {
                float2 u0 = make_float2(0.f, 0.f), u12 = make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const float2 bw = make_float2(tab.BwT[q * kTStride + iy], tab.BwT[q * kTStride + iy + 1]);
                    u0 = __ffma2_rn(t0d[q], bw, u0);
                    u12 = __ffma2_rn(t1d[q], make_float2(tab.GwT[q * kTStride + iy], tab.GwT[q * kTStride + iy + 1]), u12);
                    u12 = __ffma2_rn(t2d[q], bw, u12);
                }
                out[iy * BS] = u0.x;
                out[iy * BS + Q] = u12.x;
                if (iy + 1 < D) {
                    out[(iy + 1) * BS] = u0.y;
                    out[(iy + 1) * BS + Q] = u12.y;
                }
            }
        } else {
#pragma unroll
            for (int iy = 0; iy < D; ++iy) {
                T u0 = T(0), u12 = T(0);
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    u0 = fma(t0[q], tab.Bw[iy * Q + q], u0);
                    u12 = fma(t1[q], tab.Gw[iy * Q + q], u12);
                    u12 = fma(t2[q], tab.Bw[iy * Q + q], u12);
                }
                out[iy * BS] = u0;
                out[iy * BS + Q] = u12;
            }
        }
    }
    __syncthreads();

    // ---- X^T sweep: line (el, c, iz, iy) -> staging [c][iz][iy][ix] in A
    for (int o = tid; o < ne_blk * 3 * D * D; o += nt) {
        int el = o / (3 * D * D), r = o - el * 3 * D * D;
        int iy = r % D, iz = (r / D) % D, c = r / (D * D);
        const T *in = bufB + (size_t)el * L::B + ((c * D + iz) * D + iy) * BS;
        T u0[Q], u12[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            u0[q] = in[q];
            u12[q] = in[Q + q];
        }
        T *out = FUSE ? a.ye + (e0 + el) * 3 * D3 + ((c * D + iz) * D + iy) * D
                      : bufA + (size_t)el * L::A + ((c * D + iz) * D + iy) * DP;
        // (a line of D entries: its first and last index checked)
        if (FUSE && !(PA_INB(a.g, (e0 + el) * 3 * D3 + ((c * D + iz) * D + iy) * D, a.g.ne * 3 * D3) &&
                      PA_INB(a.g, (e0 + el) * 3 * D3 + ((c * D + iz) * D + iy) * D + D - 1, a.g.ne * 3 * D3)))
            continue;
        if constexpr (kPairT) {
            float2 u0d[Q], u12d[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                u0d[q] = make_float2(u0[q], u0[q]);
                u12d[q] = make_float2(u12[q], u12[q]);
            }
#pragma unroll
            for (int ix = 0; ix < D; ix += 2) {
                float2 y = make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    y = __ffma2_rn(u0d[q], make_float2(tab.GwT[q * kTStride + ix], tab.GwT[q * kTStride + ix + 1]), y);
                    y = __ffma2_rn(u12d[q], make_float2(tab.BwT[q * kTStride + ix], tab.BwT[q * kTStride + ix + 1]), y);
                }
                out[ix] = y.x;
                if (ix + 1 < D) out[ix + 1] = y.y;
            }
        } else {
#pragma unroll
            for (int ix = 0; ix < D; ++ix) {
                T y = T(0);
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    y = fma(u0[q], tab.Gw[ix * Q + q], y);
                    y = fma(u12[q], tab.Bw[ix * Q + q], y);
                }
                out[ix] = y;
            }
        }
    }
    if (FUSE) return;
    __syncthreads();

    // ---- coalesced store of the CTA's contiguous E-vector block
    T *ye = a.ye + e0 * 3 * D3;
    for (int o = tid; o < ne_blk * 3 * D3; o += nt) {
        int el = o / (3 * D3), r = o - el * 3 * D3;
        int ix = r % D, rest = r / D;  // rest = (c*D + iz)*D + iy
        if (PA_INB(a.g, e0 * 3 * D3 + o, a.g.ne * 3 * D3)) ye[o] = bufA[(size_t)el * L::A + rest * DP + ix];
    }
}

template <typename T, int D, int Q, bool FUSE, bool SPLIT = false, bool TWO = false>
__global__ void __launch_bounds__(256) pa_apply_line_kernel(ApplyArgs<T> a, Tables<T> tab, int epb)
{
    line_body<T, D, Q, FUSE, SPLIT, TWO>(a, tab, epb, blockIdx.x);
}

// Several operators of the same degree and precision in one launch: CTA b
// belongs to the operator k with cta_start[k] <= b < cta_start[k + 1].
template <typename T, int D, int Q, bool FUSE, bool SPLIT = false, bool TWO = false>
__global__ void __launch_bounds__(256) pa_apply_line_batch_kernel(BatchArgs<T> bt, Tables<T> tab, int epb)
{
    int k = 0;
    while (k + 1 < bt.count && (int64_t)blockIdx.x >= bt.cta_start[k + 1]) ++k;
    line_body<T, D, Q, FUSE, SPLIT, TWO>(bt.args[k], tab, epb, (int64_t)blockIdx.x - bt.cta_start[k]);
}

template <typename T, int D, int Q, bool TWO = false>
size_t line_smem_bytes(int epb)
{
    return LineLayout<T, D, Q, TWO>::table_offset(epb) + sizeof(int64_t) * (size_t)epb;
}

template <typename T, int D, int Q, bool FUSE, bool SPLIT = false, bool TWO = false>
int launch_line(const ApplyArgs<T> &a, const Tables<T> &tab, const ApplyLaunch &cfg, cudaStream_t s)
{
    if (cfg.threads > 256) return set_error(PA_EINVAL, "line kernel: at most 256 threads per CTA");
    size_t smem = line_smem_bytes<T, D, Q, TWO>(cfg.epb);
    auto kern = pa_apply_line_kernel<T, D, Q, FUSE, SPLIT, TWO>;
    static bool smem_set[kMaxAttrDevices] = {};
    if (int rc = max_smem_once(kern, smem_set)) return rc;
    int64_t nblk = (a.g.ne + cfg.epb - 1) / cfg.epb;
    if (nblk <= 0) return PA_OK;
    kern<<<(unsigned)nblk, cfg.threads, smem, s>>>(a, tab, cfg.epb);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

template <typename T, int D, int Q, bool FUSE, bool SPLIT = false, bool TWO = false>
int launch_line_batch(const BatchArgs<T> &b, const Tables<T> &tab, const ApplyLaunch &cfg, cudaStream_t s)
{
    if (cfg.threads > 256) return set_error(PA_EINVAL, "line kernel: at most 256 threads per CTA");
    const size_t smem = line_smem_bytes<T, D, Q, TWO>(cfg.epb);
    auto kern = pa_apply_line_batch_kernel<T, D, Q, FUSE, SPLIT, TWO>;
    static bool smem_set[kMaxAttrDevices] = {};
    if (int rc = max_smem_once(kern, smem_set)) return rc;
    const int64_t nblk = b.cta_start[b.count];
    if (nblk <= 0) return PA_OK;
    kern<<<(unsigned)nblk, cfg.threads, smem, s>>>(b, tab, cfg.epb);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

}  // namespace pa

