// Instantiations of the fused element kernels for double, p = 1..8 (q = p + 2):
// variant 0 = flattened shared-memory sweeps, variant 1 = register-tiled lines,
// variant 2 = register-tiled lines with the gather and store fused into the X sweeps,
// variant 3 = variant 2 with the fused Z stage split over three lanes per column.
#include "pa_apply.cuh"
#include "pa_apply_line.cuh"

namespace pa {
namespace {

// Variants 1 and 2 keep 18 D values per thread in the fused Z stage; in FP64
// that fits the register file only up to D = 5 (variant 3 keeps 6 D).
template <int D>
constexpr bool line_ok = sizeof(double) == 4 || D <= 5;

template <int D, int Q>
size_t smem_for(const ApplyLaunch &c)
{
    if (c.variant == 0) return flat_smem_bytes<double, D, Q>(c.epb);
    if (c.variant >= 4) return 0;  // FP32 only
    if (c.threads > 256) return 0;
    if (c.variant == 3 || line_ok<D>) return line_smem_bytes<double, D, Q>(c.epb);
    return 0;
}

template <int D, int Q>
int launch_for(const ApplyArgs<double> &a, const Tables<double> &tab, const ApplyLaunch &c, cudaStream_t s)
{
    if (c.variant == 0) return launch_flat<double, D, Q>(a, tab, c, s);
    if (c.variant == 3) return launch_line<double, D, Q, true, true>(a, tab, c, s);
    if constexpr (line_ok<D>) return c.variant == 1 ? launch_line<double, D, Q, false>(a, tab, c, s)
                                                    : launch_line<double, D, Q, true>(a, tab, c, s);
    return set_error(PA_EINVAL, "apply variants 1 and 2 are not instantiated for this degree and precision");
}

template <int D, int Q>
int launch_batch_for(const BatchArgs<double> &b, const Tables<double> &tab, const ApplyLaunch &c, cudaStream_t s)
{
    if (c.variant == 0) return launch_flat_batch<double, D, Q>(b, tab, c, s);
    if (c.variant == 3) return launch_line_batch<double, D, Q, true, true>(b, tab, c, s);
    if constexpr (line_ok<D>) return c.variant == 1 ? launch_line_batch<double, D, Q, false>(b, tab, c, s)
                                                    : launch_line_batch<double, D, Q, true>(b, tab, c, s);
    return set_error(PA_EINVAL, "apply variants 1 and 2 are not instantiated for this degree and precision");
}

}  // namespace

template <>
size_t apply_smem_bytes<double>(int p, const ApplyLaunch &cfg)
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
int launch_apply_elements<double>(const ApplyArgs<double> &a, const Tables<double> &tab, const ApplyLaunch &cfg,
                               cudaStream_t s)
{
    if (cfg.threads < 32 || cfg.threads > 512 || cfg.epb < 1) return set_error(PA_EINVAL, "bad apply launch config");
    const size_t smem = apply_smem_bytes<double>(a.g.p, cfg);
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
int launch_apply_batch<double>(const BatchArgs<double> &b, int p, const Tables<double> &tab, const ApplyLaunch &cfg,
                              cudaStream_t s)
{
    const size_t smem = apply_smem_bytes<double>(p, cfg);
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
