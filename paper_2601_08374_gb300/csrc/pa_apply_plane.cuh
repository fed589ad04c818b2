// Plane-fused variant of the element kernel (variant 5; same dataflow as
// pa_apply.cuh, Sec. 4.2-4.5), written for a part whose FP32 apply is bound
// by instruction issue: it keeps the shared-memory round trips and the
// barriers per element to the minimum the three contraction directions
// allow.
//
//   stage A  one thread per plane (el, c, iz): gathers the D x D plane of
//            displacement component c at z-node iz into registers, then the
//            X sweep and the Y sweep (Sec. 4.4) in registers, one qx at a
//            time; writes the three Y-sweep channels of every (qx, qy)
//            column to shared memory.
//   stage B  one thread (or three lanes) per column (el, qx, qy): Z sweep,
//            Voigt stress of Eq. 7, Q reconstruction, Z^T sweep, in place
//            (the column code of the register-tiled line variant).
//   stage C  one thread per plane (el, c, iz): the Y^T and X^T sweeps
//            (Sec. 4.5) in registers, one qx at a time, accumulating the
//            plane's D x D outputs, which it writes to the E-vector.
//
// Two barriers per CTA pass instead of six; each shared word written feeds
// D or Q FMAs of the next stage.  In FP32, stages A and B run on paired FMAs
// (__ffma2_rn: two fmaf per instruction, half the issue slots for the same
// FMA work).  The sums run in the same order as in the line variants, so
// the results are bitwise theirs.
#pragma once

#include <cstdint>

#include "pa_apply_line.cuh"
#include "pa_internal.h"

namespace pa {

template <typename T, int D, int Q>
struct PlaneLayout {
    static constexpr int CS = LineLayout<T, D, Q>::CS;  // odd column stride
    // per-element stride: the Q^2 columns plus a pad chosen (by counting the
    // banks the stage-A stores, stage-C loads and column loads of a warp
    // touch) so that no access pattern is worse than 2-way
    static constexpr int PAD = D == 2 ? 7 : D == 3 ? 13 : D == 4 ? 7 : D == 8 ? 15 : 0;
    static constexpr int A = Q * Q * CS + PAD;
    // from p = 4 on, the per-qx loops of the plane stages and the qz loop of
    // the column stage stay rolled: unrolled, each stage is tens of KB of
    // code and instruction-cache misses stall the warps (measured: rolled is
    // faster from p = 4, unrolled below)
    static constexpr bool ROLL = D >= 5;
    static constexpr int kUnroll = ROLL ? 1 : Q;
    __host__ __device__ static size_t table_offset(int epb) { return (((size_t)epb * A * sizeof(T)) + 15) & ~(size_t)15; }
};

// Shared memory of a CTA: the column buffers, the elements' base nodes and
// (geometry recomputed in the kernel) the tile's geometry records.
template <typename T, int D, int Q>
size_t plane_smem_bytes(int epb)
{
    return PlaneLayout<T, D, Q>::table_offset(epb) + (sizeof(int64_t) + kGeoStride * sizeof(T)) * (size_t)epb;
}

// The geometry record of an element (J^-1 row-major, lambda detJ, mu detJ,
// detJ; the PA data of Sec. 4.4 for an affine element) from the 9 entries
// of its map's J, recomputed in the element kernel: the unassembled (UA)
// evaluation of the data D that the paper contrasts with PA (Sec. 2).
template <typename T>
__device__ __forceinline__ void ua_record(const T *__restrict__ J, T lambda, T mu, T *rec)
{
    const T c0 = J[4] * J[8] - J[5] * J[7], c1 = J[5] * J[6] - J[3] * J[8], c2 = J[3] * J[7] - J[4] * J[6];
    const T det = J[0] * c0 + J[1] * c1 + J[2] * c2;
    const T id = T(1) / det;
    rec[0] = c0 * id;
    rec[1] = (J[2] * J[7] - J[1] * J[8]) * id;
    rec[2] = (J[1] * J[5] - J[2] * J[4]) * id;
    rec[3] = c1 * id;
    rec[4] = (J[0] * J[8] - J[2] * J[6]) * id;
    rec[5] = (J[2] * J[3] - J[0] * J[5]) * id;
    rec[6] = c2 * id;
    rec[7] = (J[1] * J[6] - J[0] * J[7]) * id;
    rec[8] = (J[0] * J[4] - J[1] * J[3]) * id;
    rec[9] = lambda * det;
    rec[10] = mu * det;
    rec[11] = det;
}

// Stage A for plane (el, c, iz): x-plane [iy][ix] in registers, then per qx
// the X-sweep values u[iy] = sum_ix x B, v[iy] = sum_ix x G and from them the
// Y-sweep channels d/dxi = sum_iy v B, d/deta = sum_iy u G, interpolated =
// sum_iy u B of every column (qx, qy).
template <typename T, int D, int Q>
__device__ __forceinline__ void plane_forward(const ApplyArgs<T> &a, const Tables<T> &tab, T *colbase, int64_t k0,
                                              int64_t Mx)
{
    constexpr int CS = PlaneLayout<T, D, Q>::CS;
    T xv[D][D];
#pragma unroll
    for (int iy = 0; iy < D; ++iy)
#pragma unroll
        for (int ix = 0; ix < D; ++ix) {
            const int64_t k = k0 + Mx * iy + ix;
            const bool in = PA_INB(a.g, k, 3 * a.g.Nn);
            T v = in ? a.x[k] : T(0);
            if (in && a.ess && a.ess[k]) v = T(0);
            xv[iy][ix] = v;
        }
    // the table columns of one qx are loaded once per iteration (the loop
    // is rolled from p = 4 on, see PlaneLayout::ROLL)
#pragma unroll(PlaneLayout<T, D, Q>::kUnroll)
    for (int qx = 0; qx < Q; ++qx) {
        T bq[D], gq[D];
#pragma unroll
        for (int ix = 0; ix < D; ++ix) {
            bq[ix] = tab.B[ix * Q + qx];
            gq[ix] = tab.G[ix * Q + qx];
        }
        T u[D], v[D];
#pragma unroll
        for (int iy = 0; iy < D; ++iy) {
            T su = T(0), sv = T(0);
#pragma unroll
            for (int ix = 0; ix < D; ++ix) {
                su = fma(xv[iy][ix], bq[ix], su);
                sv = fma(xv[iy][ix], gq[ix], sv);
            }
            u[iy] = su;
            v[iy] = sv;
        }
#pragma unroll
        for (int qy = 0; qy < Q; ++qy) {
            T d0 = T(0), d1 = T(0), d2 = T(0);
#pragma unroll
            for (int iy = 0; iy < D; ++iy) {
                d0 = fma(v[iy], tab.B[iy * Q + qy], d0);  // d/dxi
                d1 = fma(u[iy], tab.G[iy * Q + qy], d1);  // d/deta
                d2 = fma(u[iy], tab.B[iy * Q + qy], d2);  // interpolated, G follows along z
            }
            T *o = colbase + (qy * Q + qx) * CS;
            o[0 * D] = d0;
            o[1 * D] = d1;
            o[2 * D] = d2;
        }
    }
}

// Stage C for plane (el, c, iz): per qx the Y^T sweep of the column channels
// (u0[iy] = sum_qy t0 Bw, u12[iy] = sum_qy t1 Gw + t2 Bw), accumulated into
// the plane's outputs by the X^T sweep y[iy][ix] += u0 Gw + u12 Bw.
template <typename T, int D, int Q>
__device__ __forceinline__ void plane_backward(const Tables<T> &tab, const T *colbase, T *out)
{
    constexpr int CS = PlaneLayout<T, D, Q>::CS;
    T acc[D][D];
#pragma unroll
    for (int iy = 0; iy < D; ++iy)
#pragma unroll
        for (int ix = 0; ix < D; ++ix) acc[iy][ix] = T(0);
#pragma unroll(PlaneLayout<T, D, Q>::kUnroll)
    for (int qx = 0; qx < Q; ++qx) {
        T gwq[D], bwq[D];
#pragma unroll
        for (int ix = 0; ix < D; ++ix) {
            gwq[ix] = tab.Gw[ix * Q + qx];
            bwq[ix] = tab.Bw[ix * Q + qx];
        }
        T t0[Q], t1[Q], t2[Q];
#pragma unroll
        for (int qy = 0; qy < Q; ++qy) {
            const T *col = colbase + (qy * Q + qx) * CS;
            t0[qy] = col[0 * D];
            t1[qy] = col[1 * D];
            t2[qy] = col[2 * D];
        }
#pragma unroll
        for (int iy = 0; iy < D; ++iy) {
            T u0 = T(0), u12 = T(0);
#pragma unroll
            for (int qy = 0; qy < Q; ++qy) {
                u0 = fma(t0[qy], tab.Bw[iy * Q + qy], u0);
                u12 = fma(t1[qy], tab.Gw[iy * Q + qy], u12);
                u12 = fma(t2[qy], tab.Bw[iy * Q + qy], u12);
            }
#pragma unroll
            for (int ix = 0; ix < D; ++ix) {
                acc[iy][ix] = fma(u0, gwq[ix], acc[iy][ix]);
                acc[iy][ix] = fma(u12, bwq[ix], acc[iy][ix]);
            }
        }
    }
#pragma unroll
    for (int iy = 0; iy < D; ++iy)
#pragma unroll
        for (int ix = 0; ix < D; ++ix) out[iy * D + ix] = acc[iy][ix];
}

// FP32 stage A on paired FMAs (__ffma2_rn, two fmaf in one instruction):
// the X sweep runs two rows iy of the plane at a time (the last row of an
// odd D alone), the Y sweep two quadrature rows qy at a time (the last of
// an odd Q alone).  Same terms in the same order per sum as plane_forward:
// bitwise its results (measured 2-3 % faster at p = 2, 4; paired forms of
// stage C, over outputs ix or over rows iy with the transposed tables,
// measured within 1 % of the scalar stage and are not used).
template <int D, int Q>
__device__ __forceinline__ void plane_forward_f2(const ApplyArgs<float> &a, const Tables<float> &tab,
                                                 float *colbase, int64_t k0, int64_t Mx)
{
    constexpr int CS = PlaneLayout<float, D, Q>::CS;
    constexpr int H = D / 2, HQ = Q / 2;
    float2 xp[H][D];  // rows 2h and 2h + 1
    float xl[D];      // row D - 1 of an odd D
#pragma unroll
    for (int iy = 0; iy < D; ++iy)
#pragma unroll
        for (int ix = 0; ix < D; ++ix) {
            const int64_t k = k0 + Mx * iy + ix;
            const bool in = PA_INB(a.g, k, 3 * a.g.Nn);
            float v = in ? a.x[k] : 0.f;
            if (in && a.ess && a.ess[k]) v = 0.f;
            if (iy < 2 * H) {
                if (iy & 1) xp[iy >> 1][ix].y = v;
                else xp[iy >> 1][ix].x = v;
            } else {
                xl[ix] = v;
            }
        }
#pragma unroll(PlaneLayout<float, D, Q>::kUnroll)
    for (int qx = 0; qx < Q; ++qx) {
        float bq[D], gq[D];
#pragma unroll
        for (int ix = 0; ix < D; ++ix) {
            bq[ix] = tab.B[ix * Q + qx];
            gq[ix] = tab.G[ix * Q + qx];
        }
        float u[D], v[D];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            float2 su = make_float2(0.f, 0.f), sv = make_float2(0.f, 0.f);
#pragma unroll
            for (int ix = 0; ix < D; ++ix) {
                su = __ffma2_rn(xp[h][ix], make_float2(bq[ix], bq[ix]), su);
                sv = __ffma2_rn(xp[h][ix], make_float2(gq[ix], gq[ix]), sv);
            }
            u[2 * h] = su.x;
            u[2 * h + 1] = su.y;
            v[2 * h] = sv.x;
            v[2 * h + 1] = sv.y;
        }
        if constexpr (D & 1) {
            float su = 0.f, sv = 0.f;
#pragma unroll
            for (int ix = 0; ix < D; ++ix) {
                su = fmaf(xl[ix], bq[ix], su);
                sv = fmaf(xl[ix], gq[ix], sv);
            }
            u[D - 1] = su;
            v[D - 1] = sv;
        }
#pragma unroll
        for (int j = 0; j < HQ; ++j) {
            const int qy = 2 * j;
            float2 d0 = make_float2(0.f, 0.f), d1 = make_float2(0.f, 0.f), d2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int iy = 0; iy < D; ++iy) {
                const float2 b2 = make_float2(tab.B[iy * Q + qy], tab.B[iy * Q + qy + 1]);
                const float2 g2 = make_float2(tab.G[iy * Q + qy], tab.G[iy * Q + qy + 1]);
                d0 = __ffma2_rn(make_float2(v[iy], v[iy]), b2, d0);  // d/dxi
                d1 = __ffma2_rn(make_float2(u[iy], u[iy]), g2, d1);  // d/deta
                d2 = __ffma2_rn(make_float2(u[iy], u[iy]), b2, d2);  // interpolated
            }
            float *o = colbase + (qy * Q + qx) * CS;
            o[0 * D] = d0.x;
            o[1 * D] = d1.x;
            o[2 * D] = d2.x;
            o += Q * CS;
            o[0 * D] = d0.y;
            o[1 * D] = d1.y;
            o[2 * D] = d2.y;
        }
        if constexpr (Q & 1) {
            constexpr int qy = Q - 1;
            float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
            for (int iy = 0; iy < D; ++iy) {
                d0 = fmaf(v[iy], tab.B[iy * Q + qy], d0);
                d1 = fmaf(u[iy], tab.G[iy * Q + qy], d1);
                d2 = fmaf(u[iy], tab.B[iy * Q + qy], d2);
            }
            float *o = colbase + (qy * Q + qx) * CS;
            o[0 * D] = d0;
            o[1 * D] = d1;
            o[2 * D] = d2;
        }
    }
}

template <typename T, int D, int Q, bool SPLIT>
__device__ __forceinline__ void plane_body(const ApplyArgs<T> &a, const Tables<T> &tab, int epb, int64_t blk)
{
    using L = PlaneLayout<T, D, Q>;
    constexpr int D3 = D * D * D;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);

    if (a.skip && *a.skip) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t e0 = blk * epb;
    const int ne_blk = (int)((a.g.ne - e0) < epb ? (a.g.ne - e0) : epb);
    if (ne_blk <= 0) return;
    const int p = D - 1;
    const int64_t Nn = a.g.Nn;
    const int64_t Mx = a.g.Mx, MxMy = (int64_t)a.g.Mx * a.g.My;
    int64_t *gbase = reinterpret_cast<int64_t *>(smem_raw + L::table_offset(epb));
    T *geo_s = reinterpret_cast<T *>(gbase + epb);  // the tile's geometry records
    for (int el = tid; el < ne_blk; el += nt) {
        const int64_t e = e0 + el;
        const int64_t t = e / a.g.nx;
        const int ex = (int)(e - t * a.g.nx), ey = (int)(t % a.g.ny), ez = (int)(t / a.g.ny);
        gbase[el] = (int64_t)ex * p + Mx * ((int64_t)ey * p) + MxMy * ((int64_t)ez * p);
        if (a.ua) ua_record(a.geo + e * kUaStride, a.ua_lambda, a.ua_mu, geo_s + (size_t)el * kGeoStride);
    }
    // stored records: one coalesced copy of the tile's records to shared
    // memory, which the column threads read (measured at p = 1: 5.5 % less
    // element time than each column thread loading its element's record)
    if (!a.ua)
        for (int k = tid; k < ne_blk * kGeoStride; k += nt) geo_s[k] = a.geo[e0 * kGeoStride + k];
    __syncthreads();
    const T *geo0 = geo_s;  // the tile's geometry records

    // stage A: plane (el, c, iz) -> columns [qy][qx][c][k][iz]
    // from p = 2 on the element index varies fastest across the threads, so
    // that neighbouring lanes gather neighbouring nodes of x (measured: p = 3
    // 3-5 %, p = 2, 4 1-2 % faster than the plane index fastest); at p = 1
    // with 32 elements per CTA that order puts two lanes on one shared-memory
    // bank in the column stores, and the plane index stays fastest
    for (int o = tid; o < ne_blk * 3 * D; o += nt) {
        int el, r;
        if constexpr (D >= 3) {
            r = o / ne_blk;
            el = o - r * ne_blk;
        } else {
            el = o / (3 * D);
            r = o - el * 3 * D;
        }
        const int c = r / D, iz = r - c * D;
        T *cb = buf + (size_t)el * L::A + c * 3 * D + iz;
        if constexpr (sizeof(T) == 4) plane_forward_f2<D, Q>(a, tab, cb, c * Nn + gbase[el] + MxMy * iz, Mx);
        else plane_forward<T, D, Q>(a, tab, cb, c * Nn + gbase[el] + MxMy * iz, Mx);
    }
    __syncthreads();

    // stage B: Z sweep, pointwise stress, Z^T sweep per column, in place
    if constexpr (SPLIT) z_columns_split<T, D, Q, L::ROLL>(geo0, tab, buf, L::A, ne_blk, tid, nt);
    else if constexpr (sizeof(T) == 4) z_columns_f2<D, Q, L::ROLL>(geo0, tab, buf, L::A, ne_blk, tid, nt);
    else z_columns<T, D, Q, L::ROLL>(geo0, tab, buf, L::A, ne_blk, tid, nt);
    __syncthreads();

    // stage C: plane (el, c, iz) -> E-vector [e][c][iz][iy][ix]
    for (int o = tid; o < ne_blk * 3 * D; o += nt) {
        const int el = o / (3 * D), r = o - el * 3 * D;
        const int c = r / D, iz = r - c * D;
        const int64_t ob = (e0 + el) * 3 * D3 + (c * D + iz) * D * D;  // a plane of D^2 entries
        if (!(PA_INB(a.g, ob, a.g.ne * 3 * D3) && PA_INB(a.g, ob + D * D - 1, a.g.ne * 3 * D3))) continue;
        plane_backward<T, D, Q>(tab, buf + (size_t)el * L::A + c * 3 * D + iz, a.ye + ob);
    }
}

template <typename T, int D, int Q, bool SPLIT>
__global__ void __launch_bounds__(256) pa_apply_plane_kernel(ApplyArgs<T> a, Tables<T> tab, int epb)
{
    plane_body<T, D, Q, SPLIT>(a, tab, epb, blockIdx.x);
}

// Several operators of the same degree and precision in one launch: CTA b
// belongs to the operator k with cta_start[k] <= b < cta_start[k + 1].
template <typename T, int D, int Q, bool SPLIT>
__global__ void __launch_bounds__(256) pa_apply_plane_batch_kernel(BatchArgs<T> bt, Tables<T> tab, int epb)
{
    int k = 0;
    while (k + 1 < bt.count && (int64_t)blockIdx.x >= bt.cta_start[k + 1]) ++k;
    plane_body<T, D, Q, SPLIT>(bt.args[k], tab, epb, (int64_t)blockIdx.x - bt.cta_start[k]);
}

template <typename T, int D, int Q, bool SPLIT>
int launch_plane(const ApplyArgs<T> &a, const Tables<T> &tab, const ApplyLaunch &cfg, cudaStream_t s)
{
    if (cfg.threads > 256) return set_error(PA_EINVAL, "plane kernel: at most 256 threads per CTA");
    const size_t smem = plane_smem_bytes<T, D, Q>(cfg.epb);
    auto kern = pa_apply_plane_kernel<T, D, Q, SPLIT>;
    static bool smem_set[kMaxAttrDevices] = {};
    if (int rc = max_smem_once(kern, smem_set)) return rc;
    const int64_t nblk = (a.g.ne + cfg.epb - 1) / cfg.epb;
    if (nblk <= 0) return PA_OK;
    kern<<<(unsigned)nblk, cfg.threads, smem, s>>>(a, tab, cfg.epb);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

template <typename T, int D, int Q, bool SPLIT>
int launch_plane_batch(const BatchArgs<T> &b, const Tables<T> &tab, const ApplyLaunch &cfg, cudaStream_t s)
{
    if (cfg.threads > 256) return set_error(PA_EINVAL, "plane kernel: at most 256 threads per CTA");
    const size_t smem = plane_smem_bytes<T, D, Q>(cfg.epb);
    auto kern = pa_apply_plane_batch_kernel<T, D, Q, SPLIT>;
    static bool smem_set[kMaxAttrDevices] = {};
    if (int rc = max_smem_once(kern, smem_set)) return rc;
    const int64_t nblk = b.cta_start[b.count];
    if (nblk <= 0) return PA_OK;
    kern<<<(unsigned)nblk, cfg.threads, smem, s>>>(b, tab, cfg.epb);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

}  // namespace pa
