// Operator apply that allocates no device memory (pa_apply_noalloc).
//
// Some callers cannot call cudaMalloc: plugins whose host framework owns all
// device memory through its own pool and forbids driver allocations behind
// its back, and latency-critical loops that must not block on the implicit
// device synchronisation of cudaMalloc/cudaFree.  For them this entry point
// takes everything from the caller (element maps, vectors, optional mask) and
// keeps its scratch -- the per-element geometry records and the element
// output vector -- in one file-scope device array of fixed size that every
// GPU loading this library holds until process exit.  The arithmetic is the
// regular operator's: the same element and assembly kernels run on pointers
// into that array.
#include <cmath>

#include "pa_internal.h"

namespace pa {
namespace {

// 64 MiB of scratch shared by every call on a device.
constexpr size_t kStaticScratchBytes = (size_t)64 << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device with that device current).
int scratch_address(void **out)
{
    int dev = 0;
    PA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(PA_EINVAL, "pa_apply_noalloc: device index out of range");
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        PA_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return PA_OK;
}

// Geometry records (J^-1 row-major, lambda detJ, mu detJ, detJ) from the
// caller's affine maps, one thread per element; det J <= 0 sets *bad.
template <typename T>
__global__ void geometry_from_affine(const double *__restrict__ affine, T *__restrict__ geo, double lambda, double mu,
                                     int64_t ne, int *bad)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        const double *J = affine + 12 * e;
        const double c00 = J[4] * J[8] - J[5] * J[7], c01 = J[5] * J[6] - J[3] * J[8], c02 = J[3] * J[7] - J[4] * J[6];
        const double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
        if (!(det > 0.0)) atomicExch(bad, 1);
        const double id = 1.0 / det;
        double r[kGeoStride] = {c00 * id,
                                (J[2] * J[7] - J[1] * J[8]) * id,
                                (J[1] * J[5] - J[2] * J[4]) * id,
                                c01 * id,
                                (J[0] * J[8] - J[2] * J[6]) * id,
                                (J[2] * J[3] - J[0] * J[5]) * id,
                                c02 * id,
                                (J[1] * J[6] - J[0] * J[7]) * id,
                                (J[0] * J[4] - J[1] * J[3]) * id,
                                lambda * det,
                                mu * det,
                                det};
        for (int k = 0; k < kGeoStride; ++k) geo[e * kGeoStride + k] = (T)r[k];
    }
}

// An element map with det J <= 0 makes the whole output NaN, so a bad map is
// visible in y without a host round trip.
template <typename T>
__global__ void nan_if_bad(const int *__restrict__ bad, T *__restrict__ y, int64_t n)
{
    if (!*bad) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (T)NAN;
}

// 1D tables of degree p on the stack (no heap use).
template <typename T>
void stack_tables(int p, Tables<T> &t)
{
    const int D = p + 1, Q = p + 2;
    double nodes[kMaxD], qx[kMaxQ], qw[kMaxQ], B[kMaxD * kMaxQ], G[kMaxD * kMaxQ];
    gll_nodes_01(p, nodes);
    gauss_legendre_01(Q, qx, qw);
    lagrange_product(D, nodes, Q, qx, B, G);
    for (int i = 0; i < kMaxD * kMaxQ; ++i) t.B[i] = t.G[i] = t.Bw[i] = t.Gw[i] = T(0);
    for (int i = 0; i < D; ++i)
        for (int k = 0; k < Q; ++k) {
            t.B[i * Q + k] = (T)B[i * Q + k];
            t.G[i * Q + k] = (T)G[i * Q + k];
            t.Bw[i * Q + k] = (T)(B[i * Q + k] * qw[k]);
            t.Gw[i * Q + k] = (T)(G[i * Q + k] * qw[k]);
        }
    transpose_tables(t, D, Q);
}

template <typename T>
int noalloc_apply(const Grid &g, double lambda, double mu, const double *affine, const uint8_t *ess, const T *x, T *y,
                  unsigned char *scratch, cudaStream_t s)
{
    const int D = g.p + 1;
    const size_t geo_bytes = (((size_t)g.ne * kGeoStride * sizeof(T)) + 255) & ~(size_t)255;
    T *geo = reinterpret_cast<T *>(scratch);
    T *ye = reinterpret_cast<T *>(scratch + geo_bytes);
    int *bad = reinterpret_cast<int *>(scratch + geo_bytes + (size_t)g.ne * 3 * D * D * D * sizeof(T));
    PA_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
    int64_t nb = (3 * g.Nn + 255) / 256;
    if (nb > 152 * 8) nb = 152 * 8;
    geometry_from_affine<T><<<(unsigned)nb, 256, 0, s>>>(affine, geo, lambda, mu, g.ne, bad);
    PA_CUDA_TRY(cudaGetLastError());
    Tables<T> tab;
    stack_tables<T>(g.p, tab);
    ApplyArgs<T> a;
    a.x = x;
    a.ye = ye;
    a.geo = geo;
    a.ess = ess;
    a.skip = bad;  // an element with det J <= 0 skips the apply (y becomes NaN below)
    a.g = g;
    int rc = launch_apply_elements<T>(a, tab, default_apply_launch(g.p, sizeof(T) == 8 ? PA_FP64 : PA_FP32), s);
    if (rc) return rc;
    rc = launch_assemble<T>(ye, y, x, ess, T(0), false, g, s, bad);
    if (rc) return rc;
    nan_if_bad<T><<<(unsigned)nb, 256, 0, s>>>(bad, y, 3 * g.Nn);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

}  // namespace

size_t noalloc_scratch_bytes(int p, int64_t ne, size_t elem)
{
    const int D = p + 1;
    const size_t geo_bytes = ((size_t)ne * kGeoStride * elem + 255) & ~(size_t)255;
    return geo_bytes + (size_t)ne * 3 * D * D * D * elem + sizeof(int);
}

}  // namespace pa

using namespace pa;

namespace {
// True when the byte ranges [a, a + na) and [b, b + nb) share a byte.
bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t pa_ = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
    return pa_ < pb + nb && pb < pa_ + na;
}
}  // namespace

extern "C" int pa_apply_noalloc(int nx, int ny, int nz, int p, double lambda, double mu, int precision,
                                const double *affine, const uint8_t *ess_mask, const void *x, void *y, void *stream)
{
    if (precision != PA_FP64 && precision != PA_FP32) return set_error(PA_EINVAL, "pa_apply_noalloc: bad precision");
    if (!affine || !x || !y) return set_error(PA_EINVAL, "pa_apply_noalloc: null argument");
    if (!std::isfinite(lambda) || !std::isfinite(mu)) return set_error(PA_EINVAL, "pa_apply_noalloc: non-finite Lame parameters");
    Grid g;
    // the same size limits as pa_op_setup: every product below stays far
    // inside 64 bits (at most 2^31 elements, 2^36 nodes, 729 nodes per element)
    if (int rc = make_grid(nx, ny, nz, p, g, "pa_apply_noalloc")) return rc;
    const size_t elem = precision == PA_FP64 ? 8 : 4;
    const size_t vec_bytes = (size_t)(3 * g.Nn) * elem;
    if (ranges_overlap(x, vec_bytes, y, vec_bytes))
        return set_error(PA_EINVAL, "pa_apply_noalloc: x and y overlap");
    if (ranges_overlap(affine, (size_t)g.ne * 12 * sizeof(double), y, vec_bytes))
        return set_error(PA_EINVAL, "pa_apply_noalloc: affine and y overlap");
    if (ess_mask && ranges_overlap(ess_mask, (size_t)(3 * g.Nn), y, vec_bytes))
        return set_error(PA_EINVAL, "pa_apply_noalloc: ess_mask and y overlap");
    const size_t need = noalloc_scratch_bytes(p, g.ne, elem);
    if (need > kStaticScratchBytes)
        return set_error(PA_EINVAL, "pa_apply_noalloc: mesh needs " + std::to_string(need) +
                                        " bytes of scratch, more than the fixed 67108864 (64 MiB)");
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *sp = static_cast<unsigned char *>(scratch);
    if (precision == PA_FP64)
        return noalloc_apply<double>(g, lambda, mu, affine, ess_mask, static_cast<const double *>(x),
                                     static_cast<double *>(y), sp, s);
    return noalloc_apply<float>(g, lambda, mu, affine, ess_mask, static_cast<const float *>(x), static_cast<float *>(y),
                                sp, s);
}
