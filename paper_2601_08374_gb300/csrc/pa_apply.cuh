// Fused element kernel of the PA elasticity apply (Sec. 4.2-4.5).
//
// One CTA owns EPB consecutive elements.  Every stage of the element-local
// dataflow runs inside the CTA with shared-memory hand-off between the 1D
// sweeps; nothing but the input L-vector, the 12-value geometry record and
// the output E-vector touches global memory:
//   P0  gather      x_e(ix,iy,iz,c)       <- x_L (essential dofs read as 0)
//   P1  X sweep     u = sum_ix x B, v = sum_ix x G                  (Sec. 4.4)
//   P2  Y sweep     d_xi = sum_iy v B, d_eta = sum u G, u_xy = sum u B
//   P3  Z sweep     reference gradient at (qx,qy,qz), then
//       pointwise   grad u = J^-T grad_ref u, Voigt stress with
//                   lambda detJ, mu detJ (Sec. 4.5, Eq. 7), and
//                   Q_{c,m} = sum_i sigma_{c,i} (J^-1)_{m,i}         (Sec. 4.5)
//   P4  Z^T sweep   T_m = sum_qz Q_{c,m} (G if m = 2 else B) w
//   P5  Y^T sweep   U0 = sum_qy T_0 B w,  U12 = sum_qy (T_1 G + T_2 B) w
//   P6  X^T sweep   y_e = sum_qx (U0 G + U12 B) w                    -> E-vector
// The quadrature weight w_q of each direction is folded into the transposed
// tables (Bw, Gw), so the pointwise stage works with unweighted stress.
// Summing the m = 1 and m = 2 channels before the X^T sweep (both end with
// B along x) mirrors the two-channel X sweep of the forward pass.
//
// Each sweep is a flattened loop over all outputs of the CTA's elements, one
// dot product per output, two independent outputs per thread per step.
#pragma once

#include <cstdint>

#include "pa_internal.h"

namespace pa {

template <typename T, int D, int Q>
struct FlatLayout {
    static constexpr int D3 = D * D * D;
    static constexpr int Q3 = Q * Q * Q;
    static constexpr int nX = 3 * D3;           // gathered input
    static constexpr int n1 = 6 * D * D * Q;    // X sweep out  [c][2][iz][iy][qx]
    static constexpr int n2 = 9 * D * Q * Q;    // Y sweep out  [c][3][iz][qy][qx]
    static constexpr int n3 = 9 * Q3;           // Q values     [c][3][qz][qy][qx]
    static constexpr int n4 = 9 * D * Q * Q;    // Z^T out      [c][3][iz][qy][qx]
    static constexpr int n5 = 6 * D * D * Q;    // Y^T out      [c][2][iz][iy][qx]
    static constexpr int bufA = (nX > n2 ? (nX > n4 ? nX : n4) : (n2 > n4 ? n2 : n4));
    static constexpr int bufB = (n1 > n3 ? (n1 > n5 ? n1 : n5) : (n3 > n5 ? n3 : n5));
    static constexpr int tab = 4 * D * Q;
    static constexpr int per_elem = bufA + bufB;
    // byte offset of the per-CTA element table (global base node per element)
    __host__ __device__ static size_t table_offset(int epb) { return (((size_t)tab + (size_t)epb * per_elem) * sizeof(T) + 15) & ~(size_t)15; }
    // byte offset of the per-CTA coefficient table (10 values per element)
    __host__ __device__ static size_t coef_offset(int epb) { return (table_offset(epb) + sizeof(int64_t) * (size_t)epb + 15) & ~(size_t)15; }
};

// PART 0: the whole fused dataflow.  PART 1 / 2 (ablation of Table 8 only):
// the forward half up to the Q values, written to a.qvec, and the transposed
// half from a.qvec -- the two-kernel form with the quadrature values making
// a round trip through HBM.  FULLC (ablation only): the stress from the full
// 81-term contraction sigma_ij = sum_kl C_ijkl du_kl with the element's
// tensor read from a.ctensor, in place of the Voigt arithmetic of Eq. 7.
// ANISO: anisotropic material (Eq. 2): the Voigt stress sigma_V = C_V eps_V
// with the element's symmetric 6x6 matrix (times detJ) from a.cvoigt,
// eps_V = [du00, du11, du22, du01 + du10, du02 + du20, du12 + du21].
template <typename T, int D, int Q, int PART = 0, bool FULLC = false, bool ANISO = false>
__device__ __forceinline__ void flat_body(const ApplyArgs<T> &a, const Tables<T> &tab, int epb, int64_t blk)
{
    using L = FlatLayout<T, D, Q>;
    constexpr int D3 = L::D3, Q3 = L::Q3, DQ = D * Q;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sB = reinterpret_cast<T *>(smem_raw);  // tables
    T *sG = sB + DQ;
    T *sBw = sG + DQ;
    T *sGw = sBw + DQ;
    T *bufA = sB + L::tab;
    T *bufB = bufA + (size_t)epb * L::bufA;

    if (a.skip && *a.skip) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t e0 = blk * epb;
    const int ne_blk = (int)((a.g.ne - e0) < epb ? (a.g.ne - e0) : epb);
    if (ne_blk <= 0) return;

    for (int i = tid; i < DQ; i += nt) {
        sB[i] = tab.B[i];
        sG[i] = tab.G[i];
        sBw[i] = tab.Bw[i];
        sGw[i] = tab.Gw[i];
    }

    const int p = D - 1;
    const int64_t Nn = a.g.Nn;
    const int64_t Mx = a.g.Mx, MxMy = (int64_t)a.g.Mx * a.g.My;
    int64_t *gbase = reinterpret_cast<int64_t *>(smem_raw + L::table_offset(epb));
    // isotropic pointwise stage: per element mu detJ J^-1 (9) and 2 mu detJ
    constexpr bool kIso = !ANISO && !FULLC;
    T *coef = reinterpret_cast<T *>(smem_raw + L::coef_offset(epb));
    for (int el = tid; el < ne_blk; el += nt) {
        const int64_t e = e0 + el;
        const int64_t t = e / a.g.nx;
        const int ex = (int)(e - t * a.g.nx), ey = (int)(t % a.g.ny), ez = (int)(t / a.g.ny);
        gbase[el] = (int64_t)ex * p + Mx * ((int64_t)ey * p) + MxMy * ((int64_t)ez * p);
        if (kIso && PART != 2) {
            const T *geo = a.geo + e * kGeoStride;
            const T cm = geo[10];
#pragma unroll
            for (int k = 0; k < 9; ++k) coef[el * 10 + k] = cm * geo[k];
            coef[el * 10 + 9] = cm + cm;
        }
    }
    __syncthreads();
    if (PART != 2) {
    // ---- P0: gather x_e[el][c][iz][iy][ix] into bufA
    {
        const int total = ne_blk * L::nX;
        for (int o = tid; o < total; o += nt) {
            int el = o / L::nX, r = o - el * L::nX;
            int c = r / D3, a3 = r - c * D3;
            int iz = a3 / (D * D), iy = (a3 / D) % D, ix = a3 % D;
            int64_t k = c * Nn + gbase[el] + ix + Mx * iy + MxMy * iz;
            const bool in = PA_INB(a.g, k, 3 * Nn);
            T v = in ? a.x[k] : T(0);
            if (in && a.ess && a.ess[k]) v = T(0);
            bufA[(size_t)el * L::bufA + r] = v;
        }
    }
    __syncthreads();

    // ---- P1: X sweep.  out [el][c][ch][iz][iy][qx] in bufB
    {
        const int total = ne_blk * L::n1;
        for (int o = tid; o < total; o += 2 * nt) {
            int oo[2] = {o, o + nt};
            T acc[2] = {T(0), T(0)};
            const T *in[2];
            const T *tb[2];
            for (int u = 0; u < 2; ++u) {
                int q = oo[u] < total ? oo[u] : o;
                int el = q / L::n1, r = q - el * L::n1;
                int qx = r % Q, line = r / Q;  // line = ((c*2+ch)*D+iz)*D+iy
                int iy = line % D, iz = (line / D) % D, ch = (line / (D * D)) % 2, c = line / (2 * D * D);
                in[u] = bufA + (size_t)el * L::bufA + c * D3 + (iz * D + iy) * D;
                tb[u] = (ch == 0 ? sB : sG) + qx;
            }
#pragma unroll
            for (int ix = 0; ix < D; ++ix) {
                acc[0] = fma(in[0][ix], tb[0][ix * Q], acc[0]);
                acc[1] = fma(in[1][ix], tb[1][ix * Q], acc[1]);
            }
            for (int u = 0; u < 2; ++u)
                if (oo[u] < total) {
                    int el = oo[u] / L::n1;
                    bufB[(size_t)el * L::bufB + (oo[u] - el * L::n1)] = acc[u];
                }
        }
    }
    __syncthreads();

    // ---- P2: Y sweep.  out [el][c][k][iz][qy][qx] in bufA
    {
        const int total = ne_blk * L::n2;
        for (int o = tid; o < total; o += 2 * nt) {
            int oo[2] = {o, o + nt};
            T acc[2] = {T(0), T(0)};
            const T *in[2];
            const T *tb[2];
            for (int u = 0; u < 2; ++u) {
                int q = oo[u] < total ? oo[u] : o;
                int el = q / L::n2, r = q - el * L::n2;
                int qx = r % Q, qy = (r / Q) % Q, iz = (r / (Q * Q)) % D, ck = r / (Q * Q * D);
                int k = ck % 3, c = ck / 3;
                // k = 0: sum v B ; k = 1: sum u G ; k = 2: sum u B
                int ch = (k == 0) ? 1 : 0;
                in[u] = bufB + (size_t)el * L::bufB + (((c * 2 + ch) * D + iz) * D) * Q + qx;
                tb[u] = (k == 1 ? sG : sB) + qy;
            }
#pragma unroll
            for (int iy = 0; iy < D; ++iy) {
                acc[0] = fma(in[0][iy * Q], tb[0][iy * Q], acc[0]);
                acc[1] = fma(in[1][iy * Q], tb[1][iy * Q], acc[1]);
            }
            for (int u = 0; u < 2; ++u)
                if (oo[u] < total) {
                    int el = oo[u] / L::n2;
                    bufA[(size_t)el * L::bufA + (oo[u] - el * L::n2)] = acc[u];
                }
        }
    }
    __syncthreads();

    // ---- P3: Z sweep + pointwise.  out Q values [el][c][m][qz][qy][qx] in bufB
    {
        const int total = ne_blk * Q3;
        for (int o = tid; o < total; o += nt) {
            int el = o / Q3, r = o - el * Q3;
            int qx = r % Q, qy = (r / Q) % Q, qz = r / (Q * Q);
            const T *s2 = bufA + (size_t)el * L::bufA + qy * Q + qx;
            T gr[3][3];  // gr[c][n] = d u_c / d xi_n
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T g0 = T(0), g1 = T(0), g2 = T(0);
#pragma unroll
                for (int iz = 0; iz < D; ++iz) {
                    T bz = sB[iz * Q + qz], gz = sG[iz * Q + qz];
                    g0 = fma(s2[((c * 3 + 0) * D + iz) * Q * Q], bz, g0);
                    g1 = fma(s2[((c * 3 + 1) * D + iz) * Q * Q], bz, g1);
                    g2 = fma(s2[((c * 3 + 2) * D + iz) * Q * Q], gz, g2);
                }
                gr[c][0] = g0;
                gr[c][1] = g1;
                gr[c][2] = g2;
            }
            const T *geo = a.geo + (e0 + el) * kGeoStride;
            T Ji[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) Ji[i] = geo[i];
            const T cl = geo[9];
            // physical gradient du[c][j] = sum_n Ji[n][j] gr[c][n]
            T du[3][3];
            if constexpr (!kIso) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        du[c][j] = fma(Ji[0 * 3 + j], gr[c][0], fma(Ji[1 * 3 + j], gr[c][1], Ji[2 * 3 + j] * gr[c][2]));
            }
            T s[3][3];
            if constexpr (ANISO) {
                const T *cv = a.cvoigt + (e0 + el) * 21;
                const T ev[6] = {du[0][0], du[1][1], du[2][2], du[0][1] + du[1][0], du[0][2] + du[2][0],
                                 du[1][2] + du[2][1]};
                T sv[6];
#pragma unroll
                for (int I = 0; I < 6; ++I) {
                    T acc = T(0);
#pragma unroll
                    for (int J = 0; J < 6; ++J) {
                        const int r = I < J ? I : J, c2 = I < J ? J : I;
                        acc = fma(cv[r * 6 - r * (r - 1) / 2 + (c2 - r)], ev[J], acc);
                    }
                    sv[I] = acc;
                }
                s[0][0] = sv[0];
                s[1][1] = sv[1];
                s[2][2] = sv[2];
                s[0][1] = s[1][0] = sv[3];
                s[0][2] = s[2][0] = sv[4];
                s[1][2] = s[2][1] = sv[5];
            } else if constexpr (FULLC) {
                const T *C = a.ctensor + (e0 + el) * 81;
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        T acc = T(0);
#pragma unroll
                        for (int k = 0; k < 3; ++k)
#pragma unroll
                            for (int l = 0; l < 3; ++l) acc = fma(C[((i * 3 + j) * 3 + k) * 3 + l], du[k][l], acc);
                        s[i][j] = acc;
                    }
            } else {
                // Voigt stress (Eq. 7), order [00, 11, 22, 01, 02, 12]: only
                // the diagonal of grad u is formed; each shear stress
                // mu detJ (du_ab + du_ba) is one 6-term dot of the reference
                // gradient with the element's mu detJ J^-1 (two FP64
                // instructions fewer per pair than forming du_ab and du_ba)
                const T *cj = coef + el * 10;
                T dg[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) dg[c] = fma(Ji[c], gr[c][0], fma(Ji[3 + c], gr[c][1], Ji[6 + c] * gr[c][2]));
                const T ld = cl * (dg[0] + dg[1] + dg[2]), m2 = cj[9];
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
            }
            T *s3 = bufB + (size_t)el * L::bufB + r;
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int m = 0; m < 3; ++m)
                    s3[(c * 3 + m) * Q3] = fma(s[c][0], Ji[m * 3 + 0], fma(s[c][1], Ji[m * 3 + 1], s[c][2] * Ji[m * 3 + 2]));
        }
    }
    __syncthreads();
    }  // PART != 2
    if (PART == 1) {
        // the Q values of the CTA's elements to HBM (contiguous block)
        T *qv = a.qvec + e0 * L::n3;
        for (int o = tid; o < ne_blk * L::n3; o += nt) {
            const int el = o / L::n3;
            qv[o] = bufB[(size_t)el * L::bufB + (o - el * L::n3)];
        }
        return;
    }
    if (PART == 2) {
        const T *qv = a.qvec + e0 * L::n3;
        for (int o = tid; o < ne_blk * L::n3; o += nt) {
            const int el = o / L::n3;
            bufB[(size_t)el * L::bufB + (o - el * L::n3)] = qv[o];
        }
        __syncthreads();
    }

    // ---- P4: Z^T sweep.  out [el][c][m][iz][qy][qx] in bufA
    {
        const int total = ne_blk * L::n4;
        for (int o = tid; o < total; o += 2 * nt) {
            int oo[2] = {o, o + nt};
            T acc[2] = {T(0), T(0)};
            const T *in[2];
            const T *tb[2];
            for (int u = 0; u < 2; ++u) {
                int q = oo[u] < total ? oo[u] : o;
                int el = q / L::n4, r = q - el * L::n4;
                int qxy = r % (Q * Q), iz = (r / (Q * Q)) % D, cm = r / (Q * Q * D);
                int m = cm % 3;
                in[u] = bufB + (size_t)el * L::bufB + cm * Q3 + qxy;
                tb[u] = (m == 2 ? sGw : sBw) + iz * Q;
            }
#pragma unroll
            for (int qz = 0; qz < Q; ++qz) {
                acc[0] = fma(in[0][qz * Q * Q], tb[0][qz], acc[0]);
                acc[1] = fma(in[1][qz * Q * Q], tb[1][qz], acc[1]);
            }
            for (int u = 0; u < 2; ++u)
                if (oo[u] < total) {
                    int el = oo[u] / L::n4;
                    bufA[(size_t)el * L::bufA + (oo[u] - el * L::n4)] = acc[u];
                }
        }
    }
    __syncthreads();

    // ---- P5: Y^T sweep.  out [el][c][k][iz][iy][qx] in bufB
    //      k = 0: U0 = sum_qy T0 Bw ; k = 1: U12 = sum_qy T1 Gw + T2 Bw
    {
        const int total = ne_blk * L::n5;
        for (int o = tid; o < total; o += 2 * nt) {
            int oo[2] = {o, o + nt};
            T acc[2] = {T(0), T(0)};
            const T *in0[2];
            const T *in1[2];
            const T *t0[2];
            const T *t1[2];
            for (int u = 0; u < 2; ++u) {
                int q = oo[u] < total ? oo[u] : o;
                int el = q / L::n5, r = q - el * L::n5;
                int qx = r % Q, iy = (r / Q) % D, iz = (r / (Q * D)) % D, ck = r / (Q * D * D);
                int k = ck % 2, c = ck / 2;
                const T *base = bufA + (size_t)el * L::bufA + qx;
                if (k == 0) {
                    in0[u] = base + ((c * 3 + 0) * D + iz) * Q * Q;
                    t0[u] = sBw + iy * Q;
                    in1[u] = in0[u];
                    t1[u] = nullptr;
                } else {
                    in0[u] = base + ((c * 3 + 1) * D + iz) * Q * Q;
                    t0[u] = sGw + iy * Q;
                    in1[u] = base + ((c * 3 + 2) * D + iz) * Q * Q;
                    t1[u] = sBw + iy * Q;
                }
            }
#pragma unroll
            for (int qy = 0; qy < Q; ++qy) {
                acc[0] = fma(in0[0][qy * Q], t0[0][qy], acc[0]);
                acc[1] = fma(in0[1][qy * Q], t0[1][qy], acc[1]);
            }
            for (int u = 0; u < 2; ++u)
                if (t1[u]) {
                    T s = acc[u];
#pragma unroll
                    for (int qy = 0; qy < Q; ++qy) s = fma(in1[u][qy * Q], t1[u][qy], s);
                    acc[u] = s;
                }
            for (int u = 0; u < 2; ++u)
                if (oo[u] < total) {
                    int el = oo[u] / L::n5;
                    bufB[(size_t)el * L::bufB + (oo[u] - el * L::n5)] = acc[u];
                }
        }
    }
    __syncthreads();

    // ---- P6: X^T sweep.  out E-vector ye[e][c][iz][iy][ix]
    {
        const int total = ne_blk * 3 * D3;
        for (int o = tid; o < total; o += 2 * nt) {
            int oo[2] = {o, o + nt};
            T acc[2] = {T(0), T(0)};
            const T *in[2];
            int ixs[2];
            for (int u = 0; u < 2; ++u) {
                int q = oo[u] < total ? oo[u] : o;
                int el = q / (3 * D3), r = q - el * (3 * D3);
                int ix = r % D, iy = (r / D) % D, iz = (r / (D * D)) % D, c = r / D3;
                in[u] = bufB + (size_t)el * L::bufB + (((c * 2) * D + iz) * D + iy) * Q;
                ixs[u] = ix;
            }
            const int off1 = D * D * Q;  // channel 1 (U12)
#pragma unroll
            for (int qx = 0; qx < Q; ++qx) {
                acc[0] = fma(in[0][qx], sGw[ixs[0] * Q + qx], acc[0]);
                acc[1] = fma(in[1][qx], sGw[ixs[1] * Q + qx], acc[1]);
                acc[0] = fma(in[0][off1 + qx], sBw[ixs[0] * Q + qx], acc[0]);
                acc[1] = fma(in[1][off1 + qx], sBw[ixs[1] * Q + qx], acc[1]);
            }
            for (int u = 0; u < 2; ++u)
                if (oo[u] < total && PA_INB(a.g, e0 * 3 * D3 + oo[u], a.g.ne * 3 * D3)) a.ye[e0 * 3 * D3 + oo[u]] = acc[u];
        }
    }
}

template <typename T, int D, int Q>
__global__ void __launch_bounds__(512) pa_apply_flat_kernel(ApplyArgs<T> a, Tables<T> tab, int epb)
{
    flat_body<T, D, Q>(a, tab, epb, blockIdx.x);
}

// Several operators of the same degree and precision in one launch: CTA b
// belongs to the operator k with cta_start[k] <= b < cta_start[k + 1].
template <typename T, int D, int Q>
__global__ void __launch_bounds__(512) pa_apply_flat_batch_kernel(BatchArgs<T> bt, Tables<T> tab, int epb)
{
    int k = 0;
    while (k + 1 < bt.count && (int64_t)blockIdx.x >= bt.cta_start[k + 1]) ++k;
    flat_body<T, D, Q>(bt.args[k], tab, epb, (int64_t)blockIdx.x - bt.cta_start[k]);
}

// The fused kernel with an anisotropic material.
template <typename T, int D, int Q>
__global__ void __launch_bounds__(512) pa_apply_flat_aniso_kernel(ApplyArgs<T> a, Tables<T> tab, int epb)
{
    flat_body<T, D, Q, 0, false, true>(a, tab, epb, blockIdx.x);
}

// The two halves of the fused kernel as separate launches (ablation).
template <typename T, int D, int Q, int PART, bool FULLC>
__global__ void __launch_bounds__(512) pa_apply_flat_part_kernel(ApplyArgs<T> a, Tables<T> tab, int epb)
{
    flat_body<T, D, Q, PART, FULLC>(a, tab, epb, blockIdx.x);
}

template <typename T, int D, int Q>
size_t flat_smem_bytes(int epb)
{
    return FlatLayout<T, D, Q>::coef_offset(epb) + sizeof(T) * 10 * (size_t)epb;
}

template <typename T, int D, int Q>
int launch_flat(const ApplyArgs<T> &a, const Tables<T> &tab, const ApplyLaunch &cfg, cudaStream_t s)
{
    size_t smem = flat_smem_bytes<T, D, Q>(cfg.epb);
    auto kern = a.cvoigt ? pa_apply_flat_aniso_kernel<T, D, Q> : pa_apply_flat_kernel<T, D, Q>;
    static bool smem_set[2][kMaxAttrDevices] = {};
    if (int rc = max_smem_once(kern, smem_set[a.cvoigt ? 1 : 0])) return rc;
    int64_t nblk = (a.g.ne + cfg.epb - 1) / cfg.epb;
    if (nblk <= 0) return PA_OK;
    kern<<<(unsigned)nblk, cfg.threads, smem, s>>>(a, tab, cfg.epb);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

template <typename T, int D, int Q>
int launch_flat_batch(const BatchArgs<T> &b, const Tables<T> &tab, const ApplyLaunch &cfg, cudaStream_t s)
{
    const size_t smem = flat_smem_bytes<T, D, Q>(cfg.epb);
    auto kern = pa_apply_flat_batch_kernel<T, D, Q>;
    static bool smem_set[kMaxAttrDevices] = {};
    if (int rc = max_smem_once(kern, smem_set)) return rc;
    const int64_t nblk = b.cta_start[b.count];
    if (nblk <= 0) return PA_OK;
    kern<<<(unsigned)nblk, cfg.threads, smem, s>>>(b, tab, cfg.epb);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

}  // namespace pa

