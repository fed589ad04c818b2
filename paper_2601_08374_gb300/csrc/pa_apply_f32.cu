// Instantiations of the fused element kernels for float, p = 1..8 (q = p + 2):
// variant 0 = flattened shared-memory sweeps, variant 1 = register-tiled lines,
// variant 2 = register-tiled lines with the gather and store fused into the X sweeps,
// variant 3 = variant 2 with the fused Z stage split over three lanes per column,
// variant 4 = the contractions on the tensor cores (tcgen05, three-pass TF32; p <= 6),
// variant 5 = plane-fused sweeps (X+Y and Y^T+X^T per plane in registers, p <= 6),
// variant 6 = variant 5 with the fused Z stage split over three lanes per column,
// variant 7 = variant 2 with the fused Z stage in two passes (half the registers).
#include <cstring>

#include "pa_apply.cuh"
#include "pa_apply_line.cuh"
#include "pa_apply_plane.cuh"
#include "pa_apply_tc.cuh"

namespace pa {
namespace {

// Variants 1 and 2 keep 18 D values per thread in the fused Z stage; in FP64
// that fits the register file only up to D = 5 (variant 3 keeps 6 D).
template <int D>
constexpr bool line_ok = sizeof(float) == 4 || D <= 5;

template <int D, int Q>
size_t smem_for(const ApplyLaunch &c)
{
    if (c.variant == 0) return flat_smem_bytes<float, D, Q>(c.epb);
    if (c.variant == 4) {
        // one shape: 384 threads, floor(128 / Q^2) elements per CTA
        if (tc_elems(D, Q) == 0 || c.threads != kTcThreads || c.epb != tc_elems(D, Q)) return 0;
        return tc_smem_bytes();
    }
    if (c.threads > 256) return 0;
    // variant 5 keeps 18 D column values per thread: up to D = 7
    if (c.variant == 5) return D <= 7 ? plane_smem_bytes<float, D, Q>(c.epb) : 0;
    if (c.variant == 6) return plane_smem_bytes<float, D, Q>(c.epb);
    if (c.variant == 7) return line_smem_bytes<float, D, Q, true>(c.epb);
    if (c.variant == 3 || line_ok<D>) return line_smem_bytes<float, D, Q>(c.epb);
    return 0;
}

template <int D, int Q>
int launch_for(const ApplyArgs<float> &a, const Tables<float> &tab, const ApplyLaunch &c, cudaStream_t s)
{
    if (c.variant == 0) return launch_flat<float, D, Q>(a, tab, c, s);
    if (c.variant == 3) return launch_line<float, D, Q, true, true>(a, tab, c, s);
    if (c.variant == 6) return launch_plane<float, D, Q, true>(a, tab, c, s);
    if (c.variant == 7) return launch_line<float, D, Q, true, false, true>(a, tab, c, s);
    if (c.variant == 5) {
        if constexpr (D <= 7) return launch_plane<float, D, Q, false>(a, tab, c, s);
        return set_error(PA_EINVAL, "apply variant 5 is instantiated for p <= 6 only");
    }
    if (c.variant == 4) {
        if constexpr (D <= 8 && Q <= 8) return launch_tc<D, Q>(a, tc_tables(tab, D, Q), s);
        return set_error(PA_EINVAL, "apply variant 4 is instantiated for p <= 6 only");
    }
    if constexpr (line_ok<D>) return c.variant == 1 ? launch_line<float, D, Q, false>(a, tab, c, s)
                                                    : launch_line<float, D, Q, true>(a, tab, c, s);
    return set_error(PA_EINVAL, "apply variants 1 and 2 are not instantiated for this degree and precision");
}

template <int D, int Q>
int launch_batch_for(const BatchArgs<float> &b, const Tables<float> &tab, const ApplyLaunch &c, cudaStream_t s)
{
    if (c.variant == 0) return launch_flat_batch<float, D, Q>(b, tab, c, s);
    if (c.variant == 3) return launch_line_batch<float, D, Q, true, true>(b, tab, c, s);
    if (c.variant == 6) return launch_plane_batch<float, D, Q, true>(b, tab, c, s);
    if (c.variant == 7) return launch_line_batch<float, D, Q, true, false, true>(b, tab, c, s);
    if (c.variant == 5) {
        if constexpr (D <= 7) return launch_plane_batch<float, D, Q, false>(b, tab, c, s);
        return set_error(PA_EINVAL, "apply variant 5 is instantiated for p <= 6 only");
    }
    if (c.variant == 4) {
        // batches of operators run the fused line variant
        ApplyLaunch l2;
        l2.variant = 2;
        l2.epb = 2;
        l2.threads = 128;
        return launch_line_batch<float, D, Q, true>(b, tab, l2, s);
    }
    if constexpr (line_ok<D>) return c.variant == 1 ? launch_line_batch<float, D, Q, false>(b, tab, c, s)
                                                    : launch_line_batch<float, D, Q, true>(b, tab, c, s);
    return set_error(PA_EINVAL, "apply variants 1 and 2 are not instantiated for this degree and precision");
}

}  // namespace

// TF32 hi / lo parts of the five tables of variant 4 (hi = the operand
// rounded to TF32, lo = the exact FP32 remainder).
TcTables tc_tables(const Tables<float> &tab, int D, int Q)
{
    TcTables t;
    std::memset(&t, 0, sizeof(t));
    auto split = [&](int k, int n, int r, float v) {
        uint32_t u;
        std::memcpy(&u, &v, 4);
        u = (u + 0x1000u) & 0xFFFFE000u;  // nearest TF32 (ties away from zero)
        float h;
        std::memcpy(&h, &u, 4);
        t.hi[k][n][r] = h;
        t.lo[k][n][r] = v - h;
    };
    for (int i = 0; i < D; ++i)
        for (int q = 0; q < Q; ++q) {
            split(0, q, i, tab.B[i * Q + q]);       // [B | G]: N = q, K = i
            split(0, Q + q, i, tab.G[i * Q + q]);
            split(1, q, i, tab.B[i * Q + q]);       // [B]
            split(2, q, i, tab.G[i * Q + q]);       // [G]
            split(3, i, q, tab.Bw[i * Q + q]);      // [Bw]: N = i, K = q
            split(4, i, q, tab.Gw[i * Q + q]);      // [Gw]
        }
    return t;
}

template <>
size_t apply_smem_bytes<float>(int p, const ApplyLaunch &cfg)
{
    switch (p) {
    case 1: return smem_for<2, 3>(cfg);
    case 2: return smem_for<3, 4>(cfg);
    case 3: return smem_for<4, 5>(cfg);
    case 4: return smem_for<5, 6>(cfg);
    case 5: return smem_for<6, 7>(cfg);
    case 6: return smem_for<7, 8>(cfg);
    case 7: return smem_for<8, 9>(cfg);
    case 8: return smem_for<9, 10>(cfg);
    default: return 0;
    }
}

template <>
int launch_apply_elements<float>(const ApplyArgs<float> &a, const Tables<float> &tab, const ApplyLaunch &cfg,
                               cudaStream_t s)
{
    if (cfg.threads < 32 || cfg.threads > 512 || cfg.epb < 1) return set_error(PA_EINVAL, "bad apply launch config");
    const size_t smem = apply_smem_bytes<float>(a.g.p, cfg);
    if (smem == 0 || smem > 227 * 1024) return set_error(PA_EINVAL, "apply launch config not admissible");
    switch (a.g.p) {
    case 1: return launch_for<2, 3>(a, tab, cfg, s);
    case 2: return launch_for<3, 4>(a, tab, cfg, s);
    case 3: return launch_for<4, 5>(a, tab, cfg, s);
    case 4: return launch_for<5, 6>(a, tab, cfg, s);
    case 5: return launch_for<6, 7>(a, tab, cfg, s);
    case 6: return launch_for<7, 8>(a, tab, cfg, s);
    case 7: return launch_for<8, 9>(a, tab, cfg, s);
    case 8: return launch_for<9, 10>(a, tab, cfg, s);
    default: return set_error(PA_EINVAL, "p must be in 1..8");
    }
}

template <>
int launch_apply_batch<float>(const BatchArgs<float> &b, int p, const Tables<float> &tab, const ApplyLaunch &cfg,
                              cudaStream_t s)
{
    const size_t smem = apply_smem_bytes<float>(p, cfg);
    if (smem == 0 || smem > 227 * 1024) return set_error(PA_EINVAL, "apply launch config not admissible");
    switch (p) {
    case 1: return launch_batch_for<2, 3>(b, tab, cfg, s);
    case 2: return launch_batch_for<3, 4>(b, tab, cfg, s);
    case 3: return launch_batch_for<4, 5>(b, tab, cfg, s);
    case 4: return launch_batch_for<5, 6>(b, tab, cfg, s);
    case 5: return launch_batch_for<6, 7>(b, tab, cfg, s);
    case 6: return launch_batch_for<7, 8>(b, tab, cfg, s);
    case 7: return launch_batch_for<8, 9>(b, tab, cfg, s);
    case 8: return launch_batch_for<9, 10>(b, tab, cfg, s);
    default: return set_error(PA_EINVAL, "p must be in 1..8");
    }
}

}  // namespace pa
