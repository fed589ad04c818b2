// C ABI of the PA elasticity operator: errors, mesh, operator setup/apply,
// diagonal and load vector (declarations and contracts in pa_elasticity.h).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <climits>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "pa_internal.h"

namespace pa {

static thread_local std::string g_last_error;

int set_error(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_error(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return PA_ECUDA;
}

void clear_error() { g_last_error.clear(); }

static double det3(const double *J)
{
    return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
           J[2] * (J[3] * J[7] - J[4] * J[6]);
}

// Inverse by the adjugate.
static void inverse3(const double *J, double det, double *Ji)
{
    double id = 1.0 / det;
    Ji[0] = (J[4] * J[8] - J[5] * J[7]) * id;
    Ji[1] = (J[2] * J[7] - J[1] * J[8]) * id;
    Ji[2] = (J[1] * J[5] - J[2] * J[4]) * id;
    Ji[3] = (J[5] * J[6] - J[3] * J[8]) * id;
    Ji[4] = (J[0] * J[8] - J[2] * J[6]) * id;
    Ji[5] = (J[2] * J[3] - J[0] * J[5]) * id;
    Ji[6] = (J[3] * J[7] - J[4] * J[6]) * id;
    Ji[7] = (J[1] * J[6] - J[0] * J[7]) * id;
    Ji[8] = (J[0] * J[4] - J[1] * J[3]) * id;
}

// Geometry records of every element from the host copies of the maps and
// of the material: J^-1 (row-major), lambda_e detJ, mu_e detJ, detJ
// (constant per affine element, Sec. 4.4; material constant per element,
// the PA data D of Sec. 4.5), uploaded in the operator's precision.
int upload_geometry(pa_op *op)
{
    const Grid &g = op->g;
    const size_t geo_bytes = (size_t)g.ne * kGeoStride * op->elem;
    std::vector<unsigned char> geo;
    try {
        geo.resize(geo_bytes);
    } catch (...) {
        return set_error(PA_ENOMEM, "geometry records: host allocation");
    }
    for (int64_t e = 0; e < g.ne; ++e) {
        const double *J = op->h_affine.data() + 12 * e;
        double det = det3(J), Ji[9];
        inverse3(J, det, Ji);
        const double lam = op->h_mat.empty() ? op->lambda : op->h_mat[2 * e];
        const double mu = op->h_mat.empty() ? op->mu : op->h_mat[2 * e + 1];
        double rec[kGeoStride] = {Ji[0], Ji[1], Ji[2], Ji[3], Ji[4], Ji[5], Ji[6], Ji[7], Ji[8],
                                  lam * det, mu * det, det};
        for (int k = 0; k < kGeoStride; ++k) {
            if (op->precision == PA_FP64) reinterpret_cast<double *>(geo.data())[e * kGeoStride + k] = rec[k];
            else reinterpret_cast<float *>(geo.data())[e * kGeoStride + k] = (float)rec[k];
        }
    }
    PA_CUDA_TRY(cudaMemcpy(op->d_geo, geo.data(), geo_bytes, cudaMemcpyHostToDevice));
    return PA_OK;
}

// Launch table per degree and precision: the shapes the autotuner picks for
// the ~3M-dof operator sweep on GB300 (variant, elements per CTA, threads).
ApplyLaunch default_apply_launch(int p, int precision)
{
    static const int v64[kMaxP + 1] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    static const int epb64[kMaxP + 1] = {0, 32, 12, 6, 4, 2, 1, 1, 1};
    static const int thr64[kMaxP + 1] = {0, 384, 256, 256, 256, 256, 256, 256, 512};
    static const int v32[kMaxP + 1] = {0, 5, 5, 5, 5, 2, 2, 2, 3};
    static const int epb32[kMaxP + 1] = {0, 32, 16, 8, 8, 2, 2, 1, 1};
    static const int thr32[kMaxP + 1] = {0, 96, 96, 96, 96, 128, 128, 96, 96};
    ApplyLaunch c;
    if (precision == PA_FP64) {
        c.variant = v64[p];
        c.epb = epb64[p];
        c.threads = thr64[p];
    } else {
        c.variant = v32[p];
        c.epb = epb32[p];
        c.threads = thr32[p];
    }
    return c;
}

template <typename T>
static int apply_impl(pa_op *op, const T *x, T *y, bool accumulate, cudaStream_t s, const int *skip)
{
    ApplyArgs<T> a;
    a.x = x;
    a.ye = static_cast<T *>(op->d_ye);
    a.geo = static_cast<const T *>(op->d_geo);
    a.ess = op->d_ess;
    a.skip = skip;
    a.g = op->g;
    a.cvoigt = static_cast<const T *>(op->d_cv);
    a.err = op->d_err;
    a.wait_cycles = op->wait_cycles;
    if (op->geometry_mode == PA_GEOMETRY_UA) {
        a.geo = static_cast<const T *>(op->d_ua);
        a.ua = 1;
        a.ua_lambda = (T)op->lambda;
        a.ua_mu = (T)op->mu;
    }
    const Tables<T> *tab;
    if constexpr (sizeof(T) == 8) tab = &op->tab64;
    else tab = &op->tab32;
    // an anisotropic material runs in the flattened variant
    const ApplyLaunch launch = (op->d_cv && op->launch.variant != 0) ? default_apply_launch(op->p, PA_FP64)
                                                                      : op->launch;
    cudaEvent_t *ev = nullptr;
    if (op->prof_on && op->prof_count * 3 + 3 <= (int)op->prof_ev.size()) {
        ev = &op->prof_ev[op->prof_count * 3];
        ++op->prof_count;
        PA_CUDA_TRY(cudaEventRecord(ev[0], s));
    }
    int rc = launch_apply_elements<T>(a, *tab, launch, s);
    if (rc) return rc;
    if (ev) PA_CUDA_TRY(cudaEventRecord(ev[1], s));
    rc = launch_assemble<T>(a.ye, y, x, op->d_ess, T(0), accumulate, op->g, s, skip);
    if (rc) return rc;
    if (ev) PA_CUDA_TRY(cudaEventRecord(ev[2], s));
    return PA_OK;
}

int op_apply_async(pa_op *op, const void *x, void *y, bool accumulate, cudaStream_t s, const int *skip)
{
    if (op->precision == PA_FP64)
        return apply_impl<double>(op, static_cast<const double *>(x), static_cast<double *>(y), accumulate, s, skip);
    return apply_impl<float>(op, static_cast<const float *>(x), static_cast<float *>(y), accumulate, s, skip);
}

template <typename T>
int apply_batch_group(pa_op *const *ops, const void *const *xs, void *const *ys, const std::vector<int> &idx,
                      cudaStream_t s)
{
    for (size_t c0 = 0; c0 < idx.size(); c0 += kMaxBatch) {
        const size_t m = std::min(idx.size() - c0, (size_t)kMaxBatch);
        pa_op *first = ops[idx[c0]];
        ApplyLaunch cfg = first->launch;
        // a shape fitted to one small mesh (fewer elements per CTA than the
        // default) is undone: the batch as a whole has the elements to fill
        // the SMs
        const ApplyLaunch dflt = default_apply_launch(first->p, first->precision);
        if (cfg.variant == dflt.variant && cfg.threads == dflt.threads && cfg.epb < dflt.epb) cfg = dflt;
        BatchArgs<T> b{};
        AssembleBatch<T> ab{};
        b.count = ab.count = (int)m;
        b.cta_start[0] = ab.node_start[0] = 0;
        for (size_t j = 0; j < m; ++j) {
            pa_op *op = ops[idx[c0 + j]];
            ApplyArgs<T> &a = b.args[j];
            a.x = static_cast<const T *>(xs[idx[c0 + j]]);
            a.ye = static_cast<T *>(op->d_ye);
            a.geo = static_cast<const T *>(op->d_geo);
            a.ess = op->d_ess;
            a.skip = nullptr;
            a.g = op->g;
            b.cta_start[j + 1] = b.cta_start[j] + (op->g.ne + cfg.epb - 1) / cfg.epb;
            ab.node_start[j + 1] = ab.node_start[j] + op->g.Nn;
            ab.ye[j] = a.ye;
            ab.y[j] = static_cast<T *>(ys[idx[c0 + j]]);
            ab.x[j] = a.x;
            ab.ess[j] = op->d_ess;
            ab.g[j] = op->g;
        }
        const Tables<T> *tab;
        if constexpr (sizeof(T) == 8) tab = &first->tab64;
        else tab = &first->tab32;
        int rc = launch_apply_batch<T>(b, first->p, *tab, cfg, s);
        if (rc) return rc;
        rc = launch_assemble_batch<T>(ab, s);
        if (rc) return rc;
    }
    return PA_OK;
}

int make_grid(int nx, int ny, int nz, int p, Grid &g, const char *who)
{
    const std::string w(who);
    if (nx < 1 || ny < 1 || nz < 1) return set_error(PA_EINVAL, w + ": dimensions must be >= 1");
    if (p < 1 || p > kMaxP) return set_error(PA_EINVAL, w + ": p must be in 1..8");
    // every factor is below 2^31, so each product below is formed only when
    // it cannot leave int64
    const int64_t kMaxElems = (int64_t)1 << 31, kMaxNodes = (int64_t)1 << 36;
    const int64_t nxy = (int64_t)nx * ny;
    if (nxy > kMaxElems || nz > kMaxElems / nxy) return set_error(PA_EINVAL, w + ": too many elements (more than 2^31)");
    const int64_t ne = nxy * nz;
    const int64_t mx = (int64_t)nx * p + 1, my = (int64_t)ny * p + 1, mz = (int64_t)nz * p + 1;
    if (mx > INT32_MAX || my > INT32_MAX || mz > INT32_MAX)
        return set_error(PA_EINVAL, w + ": nodes per direction (n p + 1) exceed 2^31 - 1");
    const int64_t mxy = mx * my;
    if (mxy > kMaxNodes || mz > kMaxNodes / mxy) return set_error(PA_EINVAL, w + ": too many nodes (more than 2^36)");
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.p = p;
    g.Mx = (int)mx;
    g.My = (int)my;
    g.Mz = (int)mz;
    g.ne = ne;
    g.Nn = mx * my * mz;
    return PA_OK;
}
}  // namespace pa

using namespace pa;

extern "C" {

const char *pa_last_error(void) { return g_last_error.c_str(); }

int pa_version(void) { return 100; }

int pa_lame(double E, double nu, double *lambda, double *mu)
{
    if (!lambda || !mu) return set_error(PA_EINVAL, "pa_lame: null output");
    if (!(E > 0) || !(nu > -1.0) || !(nu < 0.5)) return set_error(PA_EINVAL, "pa_lame: need E > 0, -1 < nu < 1/2");
    *lambda = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    *mu = E / (2.0 * (1.0 + nu));
    return PA_OK;
}


int pa_mesh_create(int nx, int ny, int nz, const double *box, const double *affine, pa_mesh **out)
{
    if (!out) return set_error(PA_EINVAL, "pa_mesh_create: null output");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return set_error(PA_EINVAL, "pa_mesh_create: dimensions must be >= 1");
    int64_t ne = (int64_t)nx * ny * nz;
    if (ne > (int64_t)1 << 31) return set_error(PA_EINVAL, "pa_mesh_create: too many elements");
    pa_mesh *m = new (std::nothrow) pa_mesh;
    if (!m) return set_error(PA_ENOMEM, "pa_mesh_create: host allocation");
    m->nx = nx;
    m->ny = ny;
    m->nz = nz;
    try {
        m->affine.assign((size_t)ne * 12, 0.0);
    } catch (...) {
        delete m;
        return set_error(PA_ENOMEM, "pa_mesh_create: host allocation");
    }
    if (affine) {
        std::memcpy(m->affine.data(), affine, sizeof(double) * 12 * (size_t)ne);
    } else {
        double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
        if (box)
            for (int i = 0; i < 3; ++i) {
                lo[i] = box[i];
                hi[i] = box[3 + i];
            }
        double h[3] = {(hi[0] - lo[0]) / nx, (hi[1] - lo[1]) / ny, (hi[2] - lo[2]) / nz};
        for (int ez = 0; ez < nz; ++ez)
            for (int ey = 0; ey < ny; ++ey)
                for (int ex = 0; ex < nx; ++ex) {
                    double *A = m->affine.data() + 12 * ((size_t)ex + (size_t)nx * (ey + (size_t)ny * ez));
                    A[0] = h[0];
                    A[4] = h[1];
                    A[8] = h[2];
                    A[9] = lo[0] + ex * h[0];
                    A[10] = lo[1] + ey * h[1];
                    A[11] = lo[2] + ez * h[2];
                }
    }
    for (int64_t e = 0; e < ne; ++e) {
        double d = det3(m->affine.data() + 12 * e);
        if (!(d > 0.0) || !std::isfinite(d)) {
            delete m;
            return set_error(PA_EINVAL, "pa_mesh_create: element " + std::to_string(e) + " has det J <= 0");
        }
    }
    *out = m;
    clear_error();
    return PA_OK;
}

int pa_mesh_destroy(pa_mesh *mesh)
{
    delete mesh;
    return PA_OK;
}

int pa_op_destroy(pa_op *op)
{
    if (!op) return PA_OK;
    for (cudaEvent_t e : op->prof_ev) cudaEventDestroy(e);
    cudaFree(op->d_geo);
    cudaFree(op->d_affine);
    cudaFree(op->d_ess);
    cudaFree(op->d_ye);
    cudaFree(op->d_xh);
    cudaFree(op->d_yh);
    for (void *q : op->d_abl) cudaFree(q);
    cudaFree(op->d_cv);
    cudaFree(op->d_ua);
    cudaFree(op->d_err);
    delete op;
    return PA_OK;
}

int pa_op_setup(const pa_mesh *mesh, int p, int q, double lambda, double mu, int precision,
                const uint8_t *ess_mask, pa_op **out)
{
    if (!out) return set_error(PA_EINVAL, "pa_op_setup: null output");
    *out = nullptr;
    if (!mesh) return set_error(PA_EINVAL, "pa_op_setup: null mesh");
    if (p < 1 || p > kMaxP) return set_error(PA_EINVAL, "pa_op_setup: p must be in 1..8");
    if (q == 0) q = p + 2;
    if (q != p + 2) return set_error(PA_EINVAL, "pa_op_setup: only q = p + 2 is instantiated");
    if (precision != PA_FP64 && precision != PA_FP32) return set_error(PA_EINVAL, "pa_op_setup: bad precision");
    if (!std::isfinite(lambda) || !std::isfinite(mu)) return set_error(PA_EINVAL, "pa_op_setup: non-finite Lame parameters");

    pa_op *op = new (std::nothrow) pa_op;
    if (!op) return set_error(PA_ENOMEM, "pa_op_setup: host allocation");
    op->p = p;
    op->q = q;
    op->precision = precision;
    op->lambda = lambda;
    op->mu = mu;
    op->elem = precision == PA_FP64 ? 8 : 4;
    Grid &g = op->g;
    if (int rc = make_grid(mesh->nx, mesh->ny, mesh->nz, p, g, "pa_op_setup")) {
        delete op;
        return rc;
    }
    op->basis.build(p, q);
    fill_tables(op->basis, op->tab64);
    fill_tables(op->basis, op->tab32);
    op->launch = default_apply_launch(p, precision);
    {
        // a mesh too small to give every SM two CTAs of the default shape
        // gets fewer elements per CTA (the default shapes come from meshes
        // of ~3M dofs; a solver's coarse p-levels and small requests are
        // far smaller)
        const int64_t two_per_sm = 2 * 152;
        if (g.ne < two_per_sm * op->launch.epb)
            op->launch.epb = (int)std::max<int64_t>(1, g.ne / two_per_sm);
    }

    const int D = p + 1;
    const size_t D3 = (size_t)D * D * D;
    const size_t geo_bytes = (size_t)g.ne * kGeoStride * op->elem;
    cudaError_t err;
    const size_t N = (size_t)3 * g.Nn;
    if ((err = cudaMalloc(&op->d_geo, geo_bytes)) != cudaSuccess ||
        (err = cudaMalloc((void **)&op->d_affine, sizeof(double) * 12 * (size_t)g.ne)) != cudaSuccess ||
        (err = cudaMalloc(&op->d_ye, (size_t)g.ne * 3 * D3 * op->elem)) != cudaSuccess ||
        (err = cudaMalloc(&op->d_xh, N * op->elem)) != cudaSuccess ||
        (err = cudaMalloc(&op->d_yh, N * op->elem)) != cudaSuccess ||
        (err = cudaMalloc((void **)&op->d_err, sizeof(int))) != cudaSuccess ||
        (err = cudaMemset(op->d_err, 0, sizeof(int))) != cudaSuccess) {
        int rc = err == cudaErrorMemoryAllocation ? set_error(PA_ENOMEM, "pa_op_setup: device allocation failed")
                                                  : cuda_error(err, "pa_op_setup: cudaMalloc");
        pa_op_destroy(op);
        return rc;
    }
    g.flags = op->d_err;  // status flags the kernels may set (bounds build)
    if ((err = cudaMemcpy(op->d_affine, mesh->affine.data(), sizeof(double) * 12 * (size_t)g.ne,
                          cudaMemcpyHostToDevice)) != cudaSuccess) {
        pa_op_destroy(op);
        return cuda_error(err, "pa_op_setup: cudaMemcpy");
    }
    try {
        op->h_affine = mesh->affine;
        if (ess_mask) op->h_ess.assign(ess_mask, ess_mask + N);
    } catch (...) {
        pa_op_destroy(op);
        return set_error(PA_ENOMEM, "pa_op_setup: host allocation");
    }
    if (int rc = upload_geometry(op)) {
        pa_op_destroy(op);
        return rc;
    }
    if (ess_mask) {
        if ((err = cudaMalloc((void **)&op->d_ess, N)) != cudaSuccess ||
            (err = cudaMemcpy(op->d_ess, ess_mask, N, cudaMemcpyHostToDevice)) != cudaSuccess) {
            pa_op_destroy(op);
            return cuda_error(err, "pa_op_setup: essential mask");
        }
    }
    *out = op;
    clear_error();
    return PA_OK;
}

int pa_op_info(const pa_op *op, int64_t *ndofs, int64_t *nelem, int *p, int *precision)
{
    if (!op) return set_error(PA_EINVAL, "pa_op_info: null op");
    if (ndofs) *ndofs = op->ndofs();
    if (nelem) *nelem = op->g.ne;
    if (p) *p = op->p;
    if (precision) *precision = op->precision;
    return PA_OK;
}

int pa_op_apply(pa_op *op, const void *x, void *y, void *stream)
{
    if (!op || !x || !y) return set_error(PA_EINVAL, "pa_op_apply: null argument");
    if (x == y) return set_error(PA_EINVAL, "pa_op_apply: x and y must not alias");
    return op_apply_async(op, x, y, false, static_cast<cudaStream_t>(stream), nullptr);
}

int pa_op_apply_add(pa_op *op, const void *x, void *y, void *stream)
{
    if (!op || !x || !y) return set_error(PA_EINVAL, "pa_op_apply_add: null argument");
    if (x == y) return set_error(PA_EINVAL, "pa_op_apply_add: x and y must not alias");
    return op_apply_async(op, x, y, true, static_cast<cudaStream_t>(stream), nullptr);
}

int pa_op_apply_batch(pa_op *const *ops, const void *const *xs, void *const *ys, int count, void *stream)
{
    if (count < 0 || (count > 0 && (!ops || !xs || !ys))) return set_error(PA_EINVAL, "pa_op_apply_batch: bad arguments");
    for (int k = 0; k < count; ++k) {
        if (!ops[k] || !xs[k] || !ys[k]) return set_error(PA_EINVAL, "pa_op_apply_batch: null entry");
        if (xs[k] == ys[k]) return set_error(PA_EINVAL, "pa_op_apply_batch: x and y must not alias");
        for (int j = 0; j < k; ++j)
            if (ops[j] == ops[k]) return set_error(PA_EINVAL, "pa_op_apply_batch: an operator appears twice");
    }
    return apply_batch_async(ops, xs, ys, count, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace pa {

int apply_batch_async(pa_op *const *ops, const void *const *xs, void *const *ys, int count, cudaStream_t s)
{
    // anisotropic operators and operators with UA geometry are applied one
    // by one (the batched kernels take the isotropic material and the stored
    // geometry records)
    auto single = [](const pa_op *op) { return op->d_cv != nullptr || op->geometry_mode == PA_GEOMETRY_UA; };
    bool any_single = false;
    for (int k = 0; k < count; ++k) any_single = any_single || single(ops[k]);
    if (any_single) {
        std::vector<pa_op *> o2;
        std::vector<const void *> x2;
        std::vector<void *> y2;
        for (int k = 0; k < count; ++k) {
            if (single(ops[k])) {
                int rc = op_apply_async(ops[k], xs[k], ys[k], false, s, nullptr);
                if (rc) return rc;
            } else {
                o2.push_back(ops[k]);
                x2.push_back(xs[k]);
                y2.push_back(ys[k]);
            }
        }
        if (o2.empty()) return PA_OK;
        return apply_batch_async(o2.data(), x2.data(), y2.data(), (int)o2.size(), s);
    }
    // operators the persistent multi launch reproduces bitwise: one launch
    // pair per precision for any mix of degrees
    std::vector<int> multi[2], rest;
    for (int k = 0; k < count; ++k) {
        if (multi_eligible(ops[k])) multi[ops[k]->precision == PA_FP64 ? 0 : 1].push_back(k);
        else rest.push_back(k);
    }
    if (!multi[0].empty())
        if (int rc = apply_multi_group<double>(ops, xs, ys, multi[0], s)) return rc;
    if (!multi[1].empty())
        if (int rc = apply_multi_group<float>(ops, xs, ys, multi[1], s)) return rc;
    // the others: groups of equal (precision, degree), in first-appearance order
    std::vector<std::vector<int>> groups;
    std::vector<std::pair<int, int>> keys;
    for (int k : rest) {
        std::pair<int, int> key{ops[k]->precision, ops[k]->p};
        size_t g = 0;
        while (g < keys.size() && keys[g] != key) ++g;
        if (g == keys.size()) {
            keys.push_back(key);
            groups.emplace_back();
        }
        groups[g].push_back(k);
    }
    for (size_t g = 0; g < groups.size(); ++g) {
        int rc = keys[g].first == PA_FP64 ? apply_batch_group<double>(ops, xs, ys, groups[g], s)
                                          : apply_batch_group<float>(ops, xs, ys, groups[g], s);
        if (rc) return rc;
    }
    return PA_OK;
}

}  // namespace pa

extern "C" {

int pa_op_apply_host(pa_op *op, const void *x_host, void *y_host, void *stream)
{
    if (!op || !x_host || !y_host) return set_error(PA_EINVAL, "pa_op_apply_host: null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t bytes = (size_t)op->ndofs() * op->elem;
    PA_CUDA_TRY(cudaMemcpyAsync(op->d_xh, x_host, bytes, cudaMemcpyHostToDevice, s));
    int rc = pa_op_apply(op, op->d_xh, op->d_yh, stream);
    if (rc) return rc;
    PA_CUDA_TRY(cudaMemcpyAsync(y_host, op->d_yh, bytes, cudaMemcpyDeviceToHost, s));
    PA_CUDA_TRY(cudaStreamSynchronize(s));
    return PA_OK;
}

int pa_op_apply_host_batch(pa_op *const *ops, const void *const *x_host, void *const *y_host, int count, void *stream)
{
    if (count < 0 || (count > 0 && (!ops || !x_host || !y_host)))
        return set_error(PA_EINVAL, "pa_op_apply_host_batch: bad arguments");
    for (int k = 0; k < count; ++k) {
        if (!ops[k] || !x_host[k] || !y_host[k]) return set_error(PA_EINVAL, "pa_op_apply_host_batch: null entry");
        for (int j = 0; j < k; ++j)
            if (ops[j] == ops[k]) return set_error(PA_EINVAL, "pa_op_apply_host_batch: an operator appears twice");
    }
    if (count == 0) return PA_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStream_t up = nullptr, down = nullptr;
    std::vector<cudaEvent_t> ev((size_t)2 * count + 1, nullptr);
    int rc = PA_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking);
    for (size_t i = 0; e == cudaSuccess && i < ev.size(); ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) rc = cuda_error(e, "pa_op_apply_host_batch: stream or event creation");
    // the copies start after the caller's earlier work on `stream`
    if (!rc && (e = cudaEventRecord(ev[2 * count], s)) == cudaSuccess) e = cudaStreamWaitEvent(up, ev[2 * count], 0);
    if (!rc && e != cudaSuccess) rc = cuda_error(e, "pa_op_apply_host_batch: ordering");
    // every input goes up back to back on one stream ...
    for (int k = 0; !rc && k < count; ++k) {
        const size_t bytes = (size_t)ops[k]->ndofs() * ops[k]->elem;
        e = cudaMemcpyAsync(ops[k]->d_xh, x_host[k], bytes, cudaMemcpyHostToDevice, up);
        if (e == cudaSuccess) e = cudaEventRecord(ev[k], up);
        if (e != cudaSuccess) rc = cuda_error(e, "pa_op_apply_host_batch: host-to-device copy");
    }
    // ... each apply starts when its input has landed, and its result goes
    // down on a third stream while the next operators compute
    for (int k = 0; !rc && k < count; ++k) {
        if ((e = cudaStreamWaitEvent(s, ev[k], 0)) != cudaSuccess) {
            rc = cuda_error(e, "pa_op_apply_host_batch: ordering");
            break;
        }
        rc = pa_op_apply(ops[k], ops[k]->d_xh, ops[k]->d_yh, stream);
        if (rc) break;
        const size_t bytes = (size_t)ops[k]->ndofs() * ops[k]->elem;
        e = cudaEventRecord(ev[count + k], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(down, ev[count + k], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(y_host[k], ops[k]->d_yh, bytes, cudaMemcpyDeviceToHost, down);
        if (e != cudaSuccess) rc = cuda_error(e, "pa_op_apply_host_batch: device-to-host copy");
    }
    // all three streams drained before the resources go
    if (up) cudaStreamSynchronize(up);
    if (down && (e = cudaStreamSynchronize(down)) != cudaSuccess && !rc) rc = cuda_error(e, "pa_op_apply_host_batch: sync");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess && !rc) rc = cuda_error(e, "pa_op_apply_host_batch: sync");
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (up) cudaStreamDestroy(up);
    if (down) cudaStreamDestroy(down);
    return rc;
}

int pa_op_diag(pa_op *op, void *d, void *stream)
{
    if (!op || !d) return set_error(PA_EINVAL, "pa_op_diag: null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    if (op->precision == PA_FP64) {
        rc = launch_diag_elements<double>(static_cast<const double *>(op->d_geo), static_cast<double *>(op->d_ye),
                                          op->basis, op->g, s, static_cast<const double *>(op->d_cv));
        if (!rc)
            rc = launch_assemble<double>(static_cast<const double *>(op->d_ye), static_cast<double *>(d), nullptr,
                                         op->d_ess, 1.0, false, op->g, s);
    } else {
        rc = launch_diag_elements<float>(static_cast<const float *>(op->d_geo), static_cast<float *>(op->d_ye),
                                         op->basis, op->g, s, static_cast<const float *>(op->d_cv));
        if (!rc)
            rc = launch_assemble<float>(static_cast<const float *>(op->d_ye), static_cast<float *>(d), nullptr,
                                        op->d_ess, 1.0f, false, op->g, s);
    }
    return rc;
}

int pa_op_rhs(pa_op *op, const double *f0, int nmodes, const double *modes, void *F, void *stream)
{
    if (!op || !F) return set_error(PA_EINVAL, "pa_op_rhs: null argument");
    if (nmodes > 0 && !modes) return set_error(PA_EINVAL, "pa_op_rhs: modes is null");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    if (op->precision == PA_FP64) {
        rc = launch_rhs_elements<double>(op->d_affine, static_cast<double *>(op->d_ye), op->basis, op->g, f0, nmodes,
                                         modes, s);
        if (!rc)
            rc = launch_assemble<double>(static_cast<const double *>(op->d_ye), static_cast<double *>(F), nullptr,
                                         op->d_ess, 0.0, false, op->g, s);
    } else {
        rc = launch_rhs_elements<float>(op->d_affine, static_cast<float *>(op->d_ye), op->basis, op->g, f0, nmodes,
                                        modes, s);
        if (!rc)
            rc = launch_assemble<float>(static_cast<const float *>(op->d_ye), static_cast<float *>(F), nullptr,
                                        op->d_ess, 0.0f, false, op->g, s);
    }
    return rc;
}

int pa_op_set_material(pa_op *op, const double *lambda_mu)
{
    if (!op) return set_error(PA_EINVAL, "pa_op_set_material: null op");
    const int64_t ne = op->g.ne;
    if (!lambda_mu) {
        op->h_mat.clear();
        return upload_geometry(op);
    }
    if (op->geometry_mode == PA_GEOMETRY_UA)
        return set_error(PA_EINVAL, "pa_op_set_material: UA geometry takes the operator's constant material");
    for (int64_t k = 0; k < 2 * ne; ++k)
        if (!std::isfinite(lambda_mu[k])) return set_error(PA_EINVAL, "pa_op_set_material: non-finite material");
    try {
        op->h_mat.assign(lambda_mu, lambda_mu + 2 * ne);
    } catch (...) {
        return set_error(PA_ENOMEM, "pa_op_set_material: host allocation");
    }
    return upload_geometry(op);
}

int pa_op_check(pa_op *op)
{
    if (!op) return set_error(PA_EINVAL, "pa_op_check: null op");
    int flag = 0;
    PA_CUDA_TRY(cudaMemcpy(&flag, op->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!flag) return PA_OK;
    PA_CUDA_TRY(cudaMemset(op->d_err, 0, sizeof(int)));
    if (flag & 1)
        return set_error(PA_ETIMEOUT, "pa_op_check: a tensor-core wait of an apply timed out (its result is not valid)");
    return set_error(PA_EINVAL, "pa_op_check: an index outside its array was met (bounds-checking build)");
}

int pa_op_set_anisotropic(pa_op *op, const double *cvoigt)
{
    if (!op) return set_error(PA_EINVAL, "pa_op_set_anisotropic: null op");
    const int64_t ne = op->g.ne;
    if (!cvoigt) {
        op->h_cv.clear();
        cudaFree(op->d_cv);
        op->d_cv = nullptr;
        return PA_OK;
    }
    if (op->geometry_mode == PA_GEOMETRY_UA)
        return set_error(PA_EINVAL, "pa_op_set_anisotropic: UA geometry takes the isotropic material");
    for (int64_t e = 0; e < ne; ++e)
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                const double v = cvoigt[e * 36 + i * 6 + j];
                if (!std::isfinite(v)) return set_error(PA_EINVAL, "pa_op_set_anisotropic: non-finite entry");
                if (v != cvoigt[e * 36 + j * 6 + i]) return set_error(PA_EINVAL, "pa_op_set_anisotropic: matrix not symmetric");
            }
    std::vector<unsigned char> up;
    try {
        op->h_cv.assign(cvoigt, cvoigt + 36 * ne);
        up.resize((size_t)ne * 21 * op->elem);
    } catch (...) {
        return set_error(PA_ENOMEM, "pa_op_set_anisotropic: host allocation");
    }
    for (int64_t e = 0; e < ne; ++e) {
        const double det = det3(op->h_affine.data() + 12 * e);
        int k = 0;
        for (int i = 0; i < 6; ++i)
            for (int j = i; j < 6; ++j, ++k) {
                const double v = det * cvoigt[e * 36 + i * 6 + j];
                if (op->precision == PA_FP64) reinterpret_cast<double *>(up.data())[e * 21 + k] = v;
                else reinterpret_cast<float *>(up.data())[e * 21 + k] = (float)v;
            }
    }
    if (!op->d_cv) PA_CUDA_TRY(cudaMalloc(&op->d_cv, up.size()));
    PA_CUDA_TRY(cudaMemcpy(op->d_cv, up.data(), up.size(), cudaMemcpyHostToDevice));
    return PA_OK;
}

int pa_op_traction(pa_op *op, int face, const double *t, void *F, void *stream)
{
    if (!op || !t || !F) return set_error(PA_EINVAL, "pa_op_traction: null argument");
    if (face < 0 || face > 5) return set_error(PA_EINVAL, "pa_op_traction: face must be in 0..5");
    // integrals of the 1D basis functions over [0,1] with the operator's rule
    double m1[kMaxD] = {};
    const Basis1D &b = op->basis;
    for (int i = 0; i < b.D; ++i)
        for (int q = 0; q < b.Q; ++q) m1[i] += b.qwts[q] * b.B[i * b.Q + q];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (op->precision == PA_FP64)
        return launch_traction<double>(op->d_affine, static_cast<double *>(F), op->d_ess, m1, face, t, op->g, s);
    return launch_traction<float>(op->d_affine, static_cast<float *>(F), op->d_ess, m1, face, t, op->g, s);
}

int pa_op_set_launch(pa_op *op, int variant, int elems_per_block, int threads)
{
    if (!op) return set_error(PA_EINVAL, "pa_op_set_launch: null op");
    if (variant < 0 || variant > kMaxVariant || elems_per_block < 1 || threads < 32 || threads > 512 || threads % 32)
        return set_error(PA_EINVAL, "pa_op_set_launch: bad shape");
    if (op->geometry_mode == PA_GEOMETRY_UA && variant != 5)
        return set_error(PA_EINVAL, "pa_op_set_launch: UA geometry runs in the plane kernel (variant 5)");
    ApplyLaunch c;
    c.variant = variant;
    c.epb = elems_per_block;
    c.threads = threads;
    size_t smem = op->precision == PA_FP64 ? apply_smem_bytes<double>(op->p, c) : apply_smem_bytes<float>(op->p, c);
    if (smem == 0 || smem > 227 * 1024) return set_error(PA_EINVAL, "pa_op_set_launch: shared memory too large");
    op->launch = c;
    return PA_OK;
}

int pa_op_set_geometry_mode(pa_op *op, int mode)
{
    if (!op) return set_error(PA_EINVAL, "pa_op_set_geometry_mode: null op");
    if (mode == PA_GEOMETRY_STORED) {
        cudaFree(op->d_ua);
        op->d_ua = nullptr;
        op->geometry_mode = PA_GEOMETRY_STORED;
        return PA_OK;
    }
    if (mode != PA_GEOMETRY_UA) return set_error(PA_EINVAL, "pa_op_set_geometry_mode: unknown mode");
    if (op->precision != PA_FP32 || op->p > 6)
        return set_error(PA_EINVAL, "pa_op_set_geometry_mode: UA geometry runs in the FP32 plane kernel (p <= 6)");
    if (!op->h_mat.empty() || op->d_cv)
        return set_error(PA_EINVAL, "pa_op_set_geometry_mode: UA geometry takes the constant isotropic material");
    if (op->geometry_mode == PA_GEOMETRY_UA) return PA_OK;
    const int64_t ne = op->g.ne;
    std::vector<float> J;
    try {
        J.resize((size_t)ne * kUaStride);
    } catch (...) {
        return set_error(PA_ENOMEM, "pa_op_set_geometry_mode: host allocation");
    }
    for (int64_t e = 0; e < ne; ++e)
        for (int k = 0; k < kUaStride; ++k) J[(size_t)e * kUaStride + k] = (float)op->h_affine[12 * e + k];
    void *d = nullptr;
    if (cudaMalloc(&d, J.size() * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(PA_ENOMEM, "pa_op_set_geometry_mode: device allocation");
    }
    const cudaError_t e = cudaMemcpy(d, J.data(), J.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_error(e, "pa_op_set_geometry_mode: upload");
    }
    op->d_ua = d;
    op->geometry_mode = PA_GEOMETRY_UA;
    if (op->launch.variant != 5) {
        // the plane kernel's shape: the default for p <= 4, one element per CTA above
        ApplyLaunch c = default_apply_launch(op->p, PA_FP32);
        if (c.variant != 5) {
            c.variant = 5;
            c.epb = 1;
            c.threads = 128;
        }
        op->launch = c;
    }
    return PA_OK;
}

int pa_op_get_launch(const pa_op *op, int *variant, int *elems_per_block, int *threads)
{
    if (!op) return set_error(PA_EINVAL, "pa_op_get_launch: null op");
    if (variant) *variant = op->launch.variant;
    if (elems_per_block) *elems_per_block = op->launch.epb;
    if (threads) *threads = op->launch.threads;
    return PA_OK;
}

int pa_op_set_wait_limit(pa_op *op, double seconds)
{
    if (!op) return set_error(PA_EINVAL, "pa_op_set_wait_limit: null op");
    if (!(seconds > 0.0 && seconds <= 60.0)) return set_error(PA_EINVAL, "pa_op_set_wait_limit: seconds in (0, 60]");
    int dev = 0, khz = 0;
    PA_CUDA_TRY(cudaGetDevice(&dev));
    PA_CUDA_TRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    op->wait_cycles = std::max(1LL, (long long)(seconds * (double)khz * 1e3));
    return PA_OK;
}

int pa_op_autotune(pa_op *op, void *stream)
{
    NvtxRange nvtx("pa_op_autotune");
    if (!op) return set_error(PA_EINVAL, "pa_op_autotune: null op");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)op->ndofs() * op->elem;
    PA_CUDA_TRY(cudaMemsetAsync(op->d_xh, 0x3f, bytes, s));  // finite, non-zero pattern
    cudaEvent_t e0, e1;
    PA_CUDA_TRY(cudaEventCreate(&e0));
    PA_CUDA_TRY(cudaEventCreate(&e1));
    const ApplyLaunch keep = op->launch;
    ApplyLaunch best = keep;
    float best_ms = 1e30f;
    static const int epbs[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64};
    static const int thrs[] = {64, 96, 128, 160, 192, 256, 384, 512};
    int rc = PA_OK;
    for (int v = 0; v <= kMaxVariant && rc == PA_OK; ++v)
        for (int ep : epbs)
            for (int th : thrs) {
                if (v == 4) {
                    // the tensor-core variant has one shape: floor(128 / Q^2) elements, 384 threads
                    if (ep != epbs[0] || th != thrs[0]) continue;
                    ep = 128 / (op->q * op->q);
                    th = 384;
                }
                if (pa_op_set_launch(op, v, ep, th) != PA_OK) continue;
                if ((int64_t)ep > op->g.ne) continue;
                float best_here = 1e30f;
                for (int rep = 0; rep < 4 && rc == PA_OK; ++rep) {
                    cudaEventRecord(e0, s);
                    rc = pa_op_apply(op, op->d_xh, op->d_yh, stream);
                    cudaEventRecord(e1, s);
                    if (rc == PA_OK && cudaEventSynchronize(e1) == cudaSuccess) {
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if (rep > 0 && ms < best_here) best_here = ms;
                    }
                }
                if (rc != PA_OK) break;
                if (best_here < best_ms) {
                    best_ms = best_here;
                    best = op->launch;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    op->launch = (rc == PA_OK) ? best : keep;
    clear_error();
    return rc;
}

int pa_op_profile(pa_op *op, int enable)
{
    if (!op) return set_error(PA_EINVAL, "pa_op_profile: null op");
    if (enable && op->prof_ev.empty()) {
        const int n = 3 * 4096;
        op->prof_ev.resize(n);
        for (int i = 0; i < n; ++i) {
            cudaError_t e = cudaEventCreate(&op->prof_ev[i]);
            if (e != cudaSuccess) {
                for (int j = 0; j < i; ++j) cudaEventDestroy(op->prof_ev[j]);
                op->prof_ev.clear();
                return cuda_error(e, "pa_op_profile: cudaEventCreate");
            }
        }
    }
    if (enable) op->prof_count = 0;
    op->prof_on = enable != 0;
    return PA_OK;
}

int pa_op_profile_read(pa_op *op, double *element_ms, double *assemble_ms, int64_t *applies)
{
    if (!op) return set_error(PA_EINVAL, "pa_op_profile_read: null op");
    double te = 0.0, ta = 0.0;
    if (op->prof_count > 0) {
        PA_CUDA_TRY(cudaEventSynchronize(op->prof_ev[op->prof_count * 3 - 1]));
        for (int i = 0; i < op->prof_count; ++i) {
            float a = 0.f, b = 0.f;
            PA_CUDA_TRY(cudaEventElapsedTime(&a, op->prof_ev[3 * i], op->prof_ev[3 * i + 1]));
            PA_CUDA_TRY(cudaEventElapsedTime(&b, op->prof_ev[3 * i + 1], op->prof_ev[3 * i + 2]));
            te += a;
            ta += b;
        }
    }
    if (element_ms) *element_ms = te;
    if (assemble_ms) *assemble_ms = ta;
    if (applies) *applies = op->prof_count;
    return PA_OK;
}

}  // extern "C"
