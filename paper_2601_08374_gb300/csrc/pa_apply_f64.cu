// Instantiations of the fused element kernel for double, p = 1..8 (q = p + 2).
#include "pa_apply.cuh"

namespace pa {

template <>
size_t apply_smem_bytes<double>(int p, const ApplyLaunch &cfg)
{
    switch (p) {
    case 1: return flat_smem_bytes<double, 2, 3>(cfg.epb);
    case 2: return flat_smem_bytes<double, 3, 4>(cfg.epb);
    case 3: return flat_smem_bytes<double, 4, 5>(cfg.epb);
    case 4: return flat_smem_bytes<double, 5, 6>(cfg.epb);
    case 5: return flat_smem_bytes<double, 6, 7>(cfg.epb);
    case 6: return flat_smem_bytes<double, 7, 8>(cfg.epb);
    case 7: return flat_smem_bytes<double, 8, 9>(cfg.epb);
    case 8: return flat_smem_bytes<double, 9, 10>(cfg.epb);
    default: return 0;
    }
}

template <>
int launch_apply_elements<double>(const ApplyArgs<double> &a, const Tables<double> &tab, const ApplyLaunch &cfg,
                               cudaStream_t s)
{
    if (cfg.threads < 32 || cfg.threads > 512 || cfg.epb < 1) return set_error(PA_EINVAL, "bad apply launch config");
    if (apply_smem_bytes<double>(a.g.p, cfg) > 227 * 1024) return set_error(PA_EINVAL, "apply launch config exceeds shared memory");
    switch (a.g.p) {
    case 1: return launch_flat<double, 2, 3>(a, tab, cfg, s);
    case 2: return launch_flat<double, 3, 4>(a, tab, cfg, s);
    case 3: return launch_flat<double, 4, 5>(a, tab, cfg, s);
    case 4: return launch_flat<double, 5, 6>(a, tab, cfg, s);
    case 5: return launch_flat<double, 6, 7>(a, tab, cfg, s);
    case 6: return launch_flat<double, 7, 8>(a, tab, cfg, s);
    case 7: return launch_flat<double, 8, 9>(a, tab, cfg, s);
    case 8: return launch_flat<double, 9, 10>(a, tab, cfg, s);
    default: return set_error(PA_EINVAL, "p must be in 1..8");
    }
}

}  // namespace pa
