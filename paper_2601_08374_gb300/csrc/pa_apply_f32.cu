// Instantiations of the fused element kernel for float, p = 1..8 (q = p + 2).
#include "pa_apply.cuh"

namespace pa {

template <>
size_t apply_smem_bytes<float>(int p, const ApplyLaunch &cfg)
{
    switch (p) {
    case 1: return flat_smem_bytes<float, 2, 3>(cfg.epb);
    case 2: return flat_smem_bytes<float, 3, 4>(cfg.epb);
    case 3: return flat_smem_bytes<float, 4, 5>(cfg.epb);
    case 4: return flat_smem_bytes<float, 5, 6>(cfg.epb);
    case 5: return flat_smem_bytes<float, 6, 7>(cfg.epb);
    case 6: return flat_smem_bytes<float, 7, 8>(cfg.epb);
    case 7: return flat_smem_bytes<float, 8, 9>(cfg.epb);
    case 8: return flat_smem_bytes<float, 9, 10>(cfg.epb);
    default: return 0;
    }
}

template <>
int launch_apply_elements<float>(const ApplyArgs<float> &a, const Tables<float> &tab, const ApplyLaunch &cfg,
                               cudaStream_t s)
{
    if (cfg.threads < 32 || cfg.threads > 512 || cfg.epb < 1) return set_error(PA_EINVAL, "bad apply launch config");
    if (apply_smem_bytes<float>(a.g.p, cfg) > 227 * 1024) return set_error(PA_EINVAL, "apply launch config exceeds shared memory");
    switch (a.g.p) {
    case 1: return launch_flat<float, 2, 3>(a, tab, cfg, s);
    case 2: return launch_flat<float, 3, 4>(a, tab, cfg, s);
    case 3: return launch_flat<float, 4, 5>(a, tab, cfg, s);
    case 4: return launch_flat<float, 5, 6>(a, tab, cfg, s);
    case 5: return launch_flat<float, 6, 7>(a, tab, cfg, s);
    case 6: return launch_flat<float, 7, 8>(a, tab, cfg, s);
    case 7: return launch_flat<float, 8, 9>(a, tab, cfg, s);
    case 8: return launch_flat<float, 9, 10>(a, tab, cfg, s);
    default: return set_error(PA_EINVAL, "p must be in 1..8");
    }
}

}  // namespace pa
