// The optimisation stack of the paper measured stage by stage on the GPU
// (Table 8: baseline, + sum factorisation, + Voigt notation, + fusion), for
// measurement and parity only; the production apply is the fused kernel.
//
//   stage 0  baseline: two kernels with the quadrature values (Q values,
//            the paper's QVec) making a round trip through HBM; the
//            gradients at the quadrature points and the transposed
//            contraction as dense products with the full 3D basis-gradient
//            tables (O(p^6) per element, the tables streamed from L2/HBM);
//            the stress from the full 81-term contraction with C_ijkl.
//   stage 1  + sum factorisation: the same two kernels with the 1D sweeps.
//   stage 2  + Voigt notation: the structured stress of Eq. 7.
//   stage 3  + fusion: the production kernel (pa_op_apply), Q values on chip.
// Every stage computes the same operator (FP64 only).
#include <cmath>
#include <vector>

#include "pa_apply.cuh"

namespace pa {
namespace {

constexpr int kDenseThreads = 256;

// C_ijkl = lambda detJ delta_ij delta_kl + mu detJ (delta_ik delta_jl +
// delta_il delta_jk) of every element, from its geometry record.
__global__ void ctensor_kernel(const double *__restrict__ geo, double *__restrict__ C, int64_t ne)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        const double cl = geo[e * kGeoStride + 9], cm = geo[e * kGeoStride + 10];
        for (int t = 0; t < 81; ++t) {
            const int i = t / 27, j = (t / 9) % 3, k = (t / 3) % 3, l = t % 3;
            C[e * 81 + t] = (i == j && k == l ? cl : 0.0) + (i == k && j == l ? cm : 0.0) + (i == l && j == k ? cm : 0.0);
        }
    }
}

// Stage 0, first kernel: one CTA per element, one thread per quadrature
// point: the reference gradient as dense sums over the element's D^3 nodes
// with dphi[m][a][alpha] (coalesced over alpha), J^-T, the full-tensor
// stress, Q_{c,m} = sum_i sigma_{c,i} Ji[m][i], to qvec[e][c][m][alpha].
template <int D, int Q>
__global__ void __launch_bounds__(kDenseThreads) dense_fwd_kernel(ApplyArgs<double> a, const double *__restrict__ dphi)
{
    constexpr int D3 = D * D * D, Q3 = Q * Q * Q;
    __shared__ double xe[3 * D3];
    const int64_t e = blockIdx.x;
    const int tid = threadIdx.x;
    const Grid &g = a.g;
    const int p = D - 1;
    const int64_t ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / ((int64_t)g.nx * g.ny);
    for (int o = tid; o < 3 * D3; o += blockDim.x) {
        const int c = o / D3, r = o - c * D3, ix = r % D, iy = (r / D) % D, iz = r / (D * D);
        const int64_t k = c * g.Nn + (ex * p + ix) + (int64_t)g.Mx * ((ey * p + iy) + (int64_t)g.My * (ez * p + iz));
        xe[o] = (a.ess && a.ess[k]) ? 0.0 : a.x[k];
    }
    __syncthreads();
    const double *geo = a.geo + e * kGeoStride;
    const double *C = a.ctensor + e * 81;
    for (int al = tid; al < Q3; al += blockDim.x) {
        double gr[3][3] = {};  // gr[c][m] = d u_c / d xi_m
        for (int m = 0; m < 3; ++m)
            for (int ai = 0; ai < D3; ++ai) {
                const double t = dphi[((int64_t)m * D3 + ai) * Q3 + al];
                for (int c = 0; c < 3; ++c) gr[c][m] = fma(xe[c * D3 + ai], t, gr[c][m]);
            }
        double du[3][3];
        for (int c = 0; c < 3; ++c)
            for (int j = 0; j < 3; ++j)
                du[c][j] = fma(geo[0 * 3 + j], gr[c][0], fma(geo[1 * 3 + j], gr[c][1], geo[2 * 3 + j] * gr[c][2]));
        double s[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc = fma(C[((i * 3 + j) * 3 + k) * 3 + l], du[k][l], acc);
                s[i][j] = acc;
            }
        double *qv = a.qvec + e * 9 * Q3;
        for (int c = 0; c < 3; ++c)
            for (int m = 0; m < 3; ++m)
                qv[(c * 3 + m) * Q3 + al] = fma(s[c][0], geo[m * 3 + 0], fma(s[c][1], geo[m * 3 + 1], s[c][2] * geo[m * 3 + 2]));
    }
}

// Stage 0, second kernel: one CTA per element, one thread per node: the
// transposed contraction as a dense sum over the Q^3 quadrature points
// with dphiw[m][alpha][a] (weights folded, coalesced over a), into the
// E-vector.
template <int D, int Q>
__global__ void __launch_bounds__(kDenseThreads) dense_bwd_kernel(ApplyArgs<double> a, const double *__restrict__ dphiw)
{
    constexpr int D3 = D * D * D, Q3 = Q * Q * Q;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *qs = reinterpret_cast<double *>(smem_raw);  // [9][Q3]
    const int64_t e = blockIdx.x;
    const double *qv = a.qvec + e * 9 * Q3;
    for (int o = threadIdx.x; o < 9 * Q3; o += blockDim.x) qs[o] = qv[o];
    __syncthreads();
    for (int ai = threadIdx.x; ai < D3; ai += blockDim.x) {
        double y[3] = {0.0, 0.0, 0.0};
        for (int m = 0; m < 3; ++m)
            for (int al = 0; al < Q3; ++al) {
                const double t = dphiw[((int64_t)m * Q3 + al) * D3 + ai];
                for (int c = 0; c < 3; ++c) y[c] = fma(qs[(c * 3 + m) * Q3 + al], t, y[c]);
            }
        for (int c = 0; c < 3; ++c) a.ye[(e * 3 + c) * D3 + ai] = y[c];
    }
}

template <int D, int Q>
int stage_elements(pa_op *op, int stage, const ApplyArgs<double> &a, cudaStream_t s)
{
    const Tables<double> &tab = op->tab64;
    const int64_t ne = op->g.ne;
    if (stage == 0) {
        constexpr int D3 = D * D * D, Q3 = Q * Q * Q;
        const double *dphi = static_cast<const double *>(op->d_abl[2]);
        const double *dphiw = static_cast<const double *>(op->d_abl[3]);
        dense_fwd_kernel<D, Q><<<(unsigned)ne, kDenseThreads, 0, s>>>(a, dphi);
        PA_CUDA_TRY(cudaGetLastError());
        const size_t smem = sizeof(double) * 9 * Q3;
        static bool smem_set[kMaxAttrDevices] = {};
        if (int rc = max_smem_once(dense_bwd_kernel<D, Q>, smem_set)) return rc;
        (void)D3;
        dense_bwd_kernel<D, Q><<<(unsigned)ne, kDenseThreads, smem, s>>>(a, dphiw);
        PA_CUDA_TRY(cudaGetLastError());
        return PA_OK;
    }
    // stages 1, 2: the fused kernel's halves with the production launch shape
    ApplyLaunch cfg = op->launch.variant == 0 ? op->launch : default_apply_launch(op->p, PA_FP64);
    if (cfg.variant != 0) cfg = ApplyLaunch{0, 1, 256};
    const size_t smem = flat_smem_bytes<double, D, Q>(cfg.epb);
    const int64_t nblk = (ne + cfg.epb - 1) / cfg.epb;
    auto k1 = stage == 1 ? pa_apply_flat_part_kernel<double, D, Q, 1, true> : pa_apply_flat_part_kernel<double, D, Q, 1, false>;
    auto k2 = pa_apply_flat_part_kernel<double, D, Q, 2, false>;
    PA_CUDA_TRY(cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    PA_CUDA_TRY(cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    k1<<<(unsigned)nblk, cfg.threads, smem, s>>>(a, tab, cfg.epb);
    PA_CUDA_TRY(cudaGetLastError());
    k2<<<(unsigned)nblk, cfg.threads, smem, s>>>(a, tab, cfg.epb);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

// Lazily allocated buffers of the ablation stages.
int stage_buffers(pa_op *op, int stage, cudaStream_t s)
{
    const Grid &g = op->g;
    const int D = op->p + 1, Q = op->q;
    const int64_t D3 = (int64_t)D * D * D, Q3 = (int64_t)Q * Q * Q;
    if (!op->d_abl[0]) PA_CUDA_TRY(cudaMalloc(&op->d_abl[0], sizeof(double) * (size_t)(g.ne * 9 * Q3)));
    if (!op->d_abl[1]) {
        PA_CUDA_TRY(cudaMalloc(&op->d_abl[1], sizeof(double) * (size_t)(g.ne * 81)));
        ctensor_kernel<<<(unsigned)std::min<int64_t>((g.ne + 255) / 256, 152 * 8), 256, 0, s>>>(
            static_cast<const double *>(op->d_geo), static_cast<double *>(op->d_abl[1]), g.ne);
        PA_CUDA_TRY(cudaGetLastError());
    }
    if (stage == 0 && !op->d_abl[2]) {
        // dense tables from the 1D tables: dphi[m][a][alpha] = d Phi_a / d xi_m
        const Basis1D &b = op->basis;
        std::vector<double> t1((size_t)(3 * D3 * Q3)), t2((size_t)(3 * D3 * Q3));
        for (int64_t ai = 0; ai < D3; ++ai) {
            const int ix = (int)(ai % D), iy = (int)((ai / D) % D), iz = (int)(ai / (D * D));
            for (int64_t al = 0; al < Q3; ++al) {
                const int qx = (int)(al % Q), qy = (int)((al / Q) % Q), qz = (int)(al / (Q * Q));
                const double bx = b.B[ix * Q + qx], by = b.B[iy * Q + qy], bz = b.B[iz * Q + qz];
                const double gx = b.G[ix * Q + qx], gy = b.G[iy * Q + qy], gz = b.G[iz * Q + qz];
                const double w = b.qwts[qx] * b.qwts[qy] * b.qwts[qz];
                const double d[3] = {gx * by * bz, bx * gy * bz, bx * by * gz};
                for (int m = 0; m < 3; ++m) {
                    t1[(size_t)((m * D3 + ai) * Q3 + al)] = d[m];
                    t2[(size_t)((m * Q3 + al) * D3 + ai)] = w * d[m];
                }
            }
        }
        PA_CUDA_TRY(cudaMalloc(&op->d_abl[2], sizeof(double) * t1.size()));
        PA_CUDA_TRY(cudaMalloc(&op->d_abl[3], sizeof(double) * t2.size()));
        PA_CUDA_TRY(cudaMemcpy(op->d_abl[2], t1.data(), sizeof(double) * t1.size(), cudaMemcpyHostToDevice));
        PA_CUDA_TRY(cudaMemcpy(op->d_abl[3], t2.data(), sizeof(double) * t2.size(), cudaMemcpyHostToDevice));
    }
    return PA_OK;
}

}  // namespace
}  // namespace pa

using namespace pa;

extern "C" int pa_op_apply_stage(pa_op *op, int stage, const void *x, void *y, void *stream)
{
    if (!op || !x || !y) return set_error(PA_EINVAL, "pa_op_apply_stage: null argument");
    if (x == y) return set_error(PA_EINVAL, "pa_op_apply_stage: x and y must not alias");
    if (stage < 0 || stage > 3) return set_error(PA_EINVAL, "pa_op_apply_stage: stage must be in 0..3");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (stage == 3) return op_apply_async(op, x, y, false, s, nullptr);
    if (op->precision != PA_FP64) return set_error(PA_EINVAL, "pa_op_apply_stage: stages 0-2 are FP64 only");
    if (op->d_cv) return set_error(PA_EINVAL, "pa_op_apply_stage: stages 0-2 take the isotropic material only");
    int rc = stage_buffers(op, stage, s);
    if (rc) return rc;
    ApplyArgs<double> a;
    a.x = static_cast<const double *>(x);
    a.ye = static_cast<double *>(op->d_ye);
    a.geo = static_cast<const double *>(op->d_geo);
    a.ess = op->d_ess;
    a.skip = nullptr;
    a.g = op->g;
    a.qvec = static_cast<double *>(op->d_abl[0]);
    a.ctensor = static_cast<const double *>(op->d_abl[1]);
    switch (op->p) {
    case 1: rc = stage_elements<2, 3>(op, stage, a, s); break;
    case 2: rc = stage_elements<3, 4>(op, stage, a, s); break;
    case 3: rc = stage_elements<4, 5>(op, stage, a, s); break;
    case 4: rc = stage_elements<5, 6>(op, stage, a, s); break;
    case 5: rc = stage_elements<6, 7>(op, stage, a, s); break;
    case 6: rc = stage_elements<7, 8>(op, stage, a, s); break;
    case 7: rc = stage_elements<8, 9>(op, stage, a, s); break;
    case 8: rc = stage_elements<9, 10>(op, stage, a, s); break;
    default: return set_error(PA_EINVAL, "pa_op_apply_stage: p must be in 1..8");
    }
    if (rc) return rc;
    return launch_assemble<double>(a.ye, static_cast<double *>(y), a.x, op->d_ess, 0.0, false, op->g, s);
}
