// Element-to-node assembly, the closed-form PA diagonal and the load vector.
#include <cstdint>

#include <algorithm>

#include "pa_internal.h"

namespace pa {

namespace {

__host__ __device__ inline void node_coords(int64_t gn, const Grid &g, int &gx, int &gy, int &gz)
{
    gx = (int)(gn % g.Mx);
    int64_t t = gn / g.Mx;
    gy = (int)(t % g.My);
    gz = (int)(t / g.My);
}

// Elements along one axis that hold global index gi: up to two (lower first).
__device__ inline int axis_owners(int gi, int n, int p, int *e, int *i)
{
    int k = gi / p, r = gi - k * p, cnt = 0;
    if (r == 0) {
        if (k - 1 >= 0) { e[cnt] = k - 1; i[cnt] = p; ++cnt; }
        if (k < n) { e[cnt] = k; i[cnt] = 0; ++cnt; }
    } else {
        e[cnt] = k; i[cnt] = r; ++cnt;
    }
    return cnt;
}

unsigned grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > (int64_t)152 * 64) b = (int64_t)152 * 64;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

// ------------------------------------------------------------- assembly --
// Owner-computes Gather-transpose (G^T of the operator chain, Sec. 2.2):
// every global node sums the E-vector entries of the (at most 8) elements
// that hold it, in increasing element order, so the result is
// deterministic.  Essential rows take xin (constrained operator) or
// ess_value.
template <typename T>
__device__ __forceinline__ void assemble_node(const T *__restrict__ ye, T *__restrict__ y, const T *__restrict__ xin,
                                              const uint8_t *__restrict__ ess, T ess_value, int accumulate,
                                              const Grid &g, int64_t gn)
{
    const int p = g.p, D = p + 1, D3 = D * D * D;
    int gx, gy, gz;
    node_coords(gn, g, gx, gy, gz);
    int ex[2], ix[2], ey[2], iy[2], ez[2], iz[2];
    int nx_ = axis_owners(gx, g.nx, p, ex, ix);
    int ny_ = axis_owners(gy, g.ny, p, ey, iy);
    int nz_ = axis_owners(gz, g.nz, p, ez, iz);
    T acc0 = T(0), acc1 = T(0), acc2 = T(0);
    for (int c = 0; c < nz_; ++c)
        for (int b = 0; b < ny_; ++b)
            for (int a = 0; a < nx_; ++a) {
                int64_t e = ex[a] + (int64_t)g.nx * (ey[b] + (int64_t)g.ny * ez[c]);
                int loc = ix[a] + D * (iy[b] + D * iz[c]);
                const T *base = ye + e * 3 * D3 + loc;
                acc0 += base[0];
                acc1 += base[D3];
                acc2 += base[2 * D3];
            }
    T acc[3] = {acc0, acc1, acc2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        int64_t k = c * g.Nn + gn;
        T v = acc[c];
        if (ess && ess[k]) v = xin ? xin[k] : ess_value;
        y[k] = accumulate ? y[k] + v : v;
    }
}

// The same node sum specialised on the degree, with 32-bit node arithmetic
// (grids of fewer than 2^31 nodes): the divisions by p and by the grid
// extents are the costly part of a node's work.  Same additions in the same
// order as assemble_node.
// Elements of one axis that hold grid coordinate gi (degree P, ne elements
// along the axis), with the node's local index in each: one owner inside an
// element, two on an element boundary (the lower element first).  Both
// entries are written at fixed indices, so the arrays stay in registers.
template <int P>
__device__ __forceinline__ int axis_owners_p(int gi, int ne, int e[2], int li[2])
{
    const int k = gi / P, r = gi - k * P;
    if (r == 0) {
        const bool lo = k >= 1, hi = k < ne;
        e[0] = lo ? k - 1 : k;
        li[0] = lo ? P : 0;
        e[1] = k;
        li[1] = 0;
        return (int)lo + (int)hi;
    }
    e[0] = e[1] = k;
    li[0] = li[1] = r;
    return 1;
}

// Sum of the (at most 8) E-vector entries of global node (gx, gy, gz) given
// its owners along each axis: z owners outermost, then y, then x, each in
// increasing element order.  Fixed-length loops guarded by the counts.
template <typename T, int P>
__device__ __forceinline__ void node_sum_p(const T *__restrict__ ye, const Grid &g, const int ex[2], const int ix[2],
                                           int cx, const int ey[2], const int iy[2], int cy, const int ez[2],
                                           const int iz[2], int cz, T acc[3])
{
    constexpr int D = P + 1, D3 = D * D * D;
    T acc0 = T(0), acc1 = T(0), acc2 = T(0);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                if (c >= cz || b >= cy || a >= cx) continue;
                const int el = ex[a] + g.nx * (ey[b] + g.ny * ez[c]);
                const int loc = ix[a] + D * (iy[b] + D * iz[c]);
                if (!(PA_INB(g, (int64_t)el * (3 * D3) + loc, g.ne * 3 * D3) &&
                      PA_INB(g, (int64_t)el * (3 * D3) + loc + 2 * D3, g.ne * 3 * D3)))
                    continue;
                const T *base = ye + (int64_t)el * (3 * D3) + loc;
                acc0 += base[0];
                acc1 += base[D3];
                acc2 += base[2 * D3];
            }
    acc[0] = acc0;
    acc[1] = acc1;
    acc[2] = acc2;
}

template <typename T, int P>
__device__ __forceinline__ void assemble_node_p(const T *__restrict__ ye, T *__restrict__ y, const T *__restrict__ xin,
                                                const uint8_t *__restrict__ ess, T ess_value, int accumulate,
                                                const Grid &g, int gn)
{
    const int t = gn / g.Mx;
    int ex[2], ix[2], ey[2], iy[2], ez[2], iz[2];
    const int cx = axis_owners_p<P>(gn - t * g.Mx, g.nx, ex, ix);
    const int cy = axis_owners_p<P>(t % g.My, g.ny, ey, iy);
    const int cz = axis_owners_p<P>(t / g.My, g.nz, ez, iz);
    T acc[3];
    node_sum_p<T, P>(ye, g, ex, ix, cx, ey, iy, cy, ez, iz, cz, acc);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int64_t k = c * g.Nn + gn;
        T v = acc[c];
        if (ess && ess[k]) v = xin ? xin[k] : ess_value;
        y[k] = accumulate ? y[k] + v : v;
    }
}

// The node sum organised by node rows: a CTA takes whole rows (gy, gz) of
// the grid, so the y and z owners are the same for all its threads and only
// every P-th node along x (an element boundary) has a second owner; no
// division by a grid extent per node.  Same additions in the same order as
// assemble_node_p.
template <typename T, int P>
__global__ void __launch_bounds__(256) assemble_rows_kernel(const T *__restrict__ ye, T *__restrict__ y,
                                                            const T *__restrict__ xin, const uint8_t *__restrict__ ess,
                                                            T ess_value, int accumulate, Grid g,
                                                            const int *__restrict__ skip)
{
    // R rows per pass (rows row0 + r * gridDim.x): their loads are issued
    // before any of their stores, so a thread keeps R node sums in flight.
    // Measured against one row per pass: p = 2, 4 5 % faster with two rows
    // (FP64 and FP32), p = 6, 8 within +-4 % and four rows slower everywhere
    constexpr int R = P <= 4 ? 2 : 1;
    if (skip && *skip) return;
    const int64_t rows = (int64_t)g.My * g.Mz;
    for (int64_t row0 = blockIdx.x; row0 < rows; row0 += (int64_t)R * gridDim.x) {
        for (int gx = threadIdx.x; gx < g.Mx; gx += blockDim.x) {
            int ex[2], ix[2];
            const int cx = axis_owners_p<P>(gx, g.nx, ex, ix);
            T acc[R][3];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int64_t row = row0 + (int64_t)r * gridDim.x;
                if (row >= rows) break;
                int ey[2], iy[2], ez[2], iz[2];
                const int cy = axis_owners_p<P>((int)(row % g.My), g.ny, ey, iy);
                const int cz = axis_owners_p<P>((int)(row / g.My), g.nz, ez, iz);
                node_sum_p<T, P>(ye, g, ex, ix, cx, ey, iy, cy, ez, iz, cz, acc[r]);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int64_t row = row0 + (int64_t)r * gridDim.x;
                if (row >= rows) break;
                const int64_t gn = gx + (int64_t)g.Mx * row;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int64_t k = c * g.Nn + gn;
                    T v = acc[r][c];
                    if (ess && ess[k]) v = xin ? xin[k] : ess_value;
                    y[k] = accumulate ? y[k] + v : v;
                }
            }
        }
    }
}

template <typename T, int P>
__global__ void assemble_kernel_p(const T *__restrict__ ye, T *__restrict__ y, const T *__restrict__ xin,
                                  const uint8_t *__restrict__ ess, T ess_value, int accumulate, Grid g,
                                  const int *__restrict__ skip)
{
    if (skip && *skip) return;
    // the loop counter is 64-bit: near 2^31 nodes a 32-bit counter plus the
    // grid stride would overflow; the node arithmetic inside stays 32-bit
    for (int64_t gn = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gn < g.Nn; gn += (int64_t)gridDim.x * blockDim.x)
        assemble_node_p<T, P>(ye, y, xin, ess, ess_value, accumulate, g, (int)gn);
}

template <typename T, int P>
__global__ void assemble_batch_kernel_p(AssembleBatch<T> b)
{
    const int64_t total = b.node_start[b.count];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < b.count && t >= b.node_start[k + 1]) ++k;
        assemble_node_p<T, P>(b.ye[k], b.y[k], b.x[k], b.ess[k], T(0), 0, b.g[k], (int)(t - b.node_start[k]));
    }
}

template <typename T>
__global__ void assemble_kernel(const T *__restrict__ ye, T *__restrict__ y, const T *__restrict__ xin,
                                const uint8_t *__restrict__ ess, T ess_value, int accumulate, Grid g,
                                const int *__restrict__ skip)
{
    if (skip && *skip) return;
    for (int64_t gn = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gn < g.Nn;
         gn += (int64_t)gridDim.x * blockDim.x)
        assemble_node<T>(ye, y, xin, ess, ess_value, accumulate, g, gn);
}

// The node sums of several operators in one launch (constrained rows take x).
template <typename T>
__global__ void assemble_batch_kernel(AssembleBatch<T> b)
{
    const int64_t total = b.node_start[b.count];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < b.count && t >= b.node_start[k + 1]) ++k;
        assemble_node<T>(b.ye[k], b.y[k], b.x[k], b.ess[k], T(0), 0, b.g[k], t - b.node_start[k]);
    }
}

// Node sums of operators of any degree (AssembleMulti): every node finds
// its operator by bisection over the prefix sums and runs the node sum of
// that operator's degree.
template <typename T>
__global__ void __launch_bounds__(256) assemble_multi_kernel(AssembleMulti<T> m)
{
    const int64_t total = m.node_start[m.count];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = m.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (m.node_start[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const int k = lo;
        const int gn = (int)(t - m.node_start[k]);
        switch (m.g[k].p) {
#define PA_ASM_MULTI(P) \
    case P: assemble_node_p<T, P>(m.ye[k], m.y[k], m.x[k], m.ess[k], T(0), 0, m.g[k], gn); break;
            PA_ASM_MULTI(1) PA_ASM_MULTI(2) PA_ASM_MULTI(3) PA_ASM_MULTI(4)
            PA_ASM_MULTI(5) PA_ASM_MULTI(6) PA_ASM_MULTI(7) PA_ASM_MULTI(8)
#undef PA_ASM_MULTI
        default: break;
        }
    }
}

template <typename T>
int launch_assemble_multi(const AssembleMulti<T> &b, cudaStream_t s)
{
    const int64_t nodes = b.node_start[b.count];
    if (nodes <= 0) return PA_OK;
    assemble_multi_kernel<T><<<grid_for(nodes, 256), 256, 0, s>>>(b);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}
template int launch_assemble_multi<double>(const AssembleMulti<double> &, cudaStream_t);
template int launch_assemble_multi<float>(const AssembleMulti<float> &, cudaStream_t);

constexpr int64_t kNode32 = (int64_t)1 << 31;

template <typename T>
int launch_assemble_batch(const AssembleBatch<T> &b, cudaStream_t s)
{
    const int th = 256;
    const unsigned nb = grid_for(b.node_start[b.count], th);
    bool same_p = true, small = true;
    for (int k = 0; k < b.count; ++k) {
        same_p = same_p && b.g[k].p == b.g[0].p;
        small = small && b.g[k].Nn < kNode32;
    }
    if (b.count > 0 && same_p && small) {
        switch (b.g[0].p) {
#define PA_ASM_BATCH(P) \
    case P: assemble_batch_kernel_p<T, P><<<nb, th, 0, s>>>(b); break;
            PA_ASM_BATCH(1) PA_ASM_BATCH(2) PA_ASM_BATCH(3) PA_ASM_BATCH(4)
            PA_ASM_BATCH(5) PA_ASM_BATCH(6) PA_ASM_BATCH(7) PA_ASM_BATCH(8)
#undef PA_ASM_BATCH
        default: assemble_batch_kernel<T><<<nb, th, 0, s>>>(b);
        }
    } else {
        assemble_batch_kernel<T><<<nb, th, 0, s>>>(b);
    }
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}
template int launch_assemble_batch<double>(const AssembleBatch<double> &, cudaStream_t);
template int launch_assemble_batch<float>(const AssembleBatch<float> &, cudaStream_t);

template <typename T>
int launch_assemble(const T *ye, T *y, const T *xin, const uint8_t *ess, T ess_value, bool accumulate,
                    const Grid &g, cudaStream_t s, const int *skip)
{
    const int th = 256;
    const unsigned nb = grid_for(g.Nn, th);
    const int acc = accumulate ? 1 : 0;
    if (g.Nn < kNode32) {
        // rows of Mx nodes: one CTA per row at a time, its width Mx rounded up to a warp
        const int64_t rows = (int64_t)g.My * g.Mz;
        const int rth = (int)std::min<int64_t>(256, ((int64_t)g.Mx + 31) / 32 * 32);
        const unsigned rb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(rows, (int64_t)152 * 16));
        // p = 1: every node is an element boundary along x and the rows
        // gain nothing (measured 46 vs 43 us at 100^3 nodes); the per-node
        // form stays there
        switch (g.p) {
        case 1: assemble_kernel_p<T, 1><<<nb, th, 0, s>>>(ye, y, xin, ess, ess_value, acc, g, skip); break;
#define PA_ASM(P) \
    case P: assemble_rows_kernel<T, P><<<rb, rth, 0, s>>>(ye, y, xin, ess, ess_value, acc, g, skip); break;
            PA_ASM(2) PA_ASM(3) PA_ASM(4) PA_ASM(5) PA_ASM(6) PA_ASM(7) PA_ASM(8)
#undef PA_ASM
        default: assemble_kernel<T><<<nb, th, 0, s>>>(ye, y, xin, ess, ess_value, acc, g, skip);
        }
    } else {
        assemble_kernel<T><<<nb, th, 0, s>>>(ye, y, xin, ess, ess_value, acc, g, skip);
    }
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}
template int launch_assemble<double>(const double *, double *, const double *, const uint8_t *, double, bool,
                                     const Grid &, cudaStream_t, const int *);
template int launch_assemble<float>(const float *, float *, const float *, const uint8_t *, float, bool,
                                    const Grid &, cudaStream_t, const int *);

// -------------------------------------------------------------- traction --
// Neumann load of a constant traction t on one face of the box (the boundary
// term of the weak form, Eq. 1), added to F node by node.  On an element's
// face the basis is the product of the two tangential 1D bases (the nodal
// basis along the normal is 1 at the face node and 0 elsewhere), so the
// face integral of a node's basis function is dS_e m1[ib] m1[ic], with m1
// the integrals of the 1D basis functions and dS_e = |dx/du x dx/dv| of the
// element's affine map; a node sums the (at most 4) faces that hold it in
// increasing element order.  Essential entries are set to 0.
struct TractionArgs {
    double m1[kMaxD];
    double t[3];
    int face;
};

template <typename T>
__global__ void traction_kernel(const double *__restrict__ affine, T *__restrict__ F, const uint8_t *__restrict__ ess,
                                TractionArgs ta, Grid g)
{
    const int ax = ta.face / 2, side = ta.face % 2;
    const int bx = ax == 0 ? 1 : 0, cx = ax == 2 ? 1 : 2;
    const int M[3] = {g.Mx, g.My, g.Mz}, ne[3] = {g.nx, g.ny, g.nz};
    const int64_t nface = (int64_t)M[bx] * M[cx];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nface; k += (int64_t)gridDim.x * blockDim.x) {
        int gi[3];
        gi[ax] = side ? M[ax] - 1 : 0;
        gi[bx] = (int)(k % M[bx]);
        gi[cx] = (int)(k / M[bx]);
        int eb[2], ib[2], ec[2], ic[2];
        const int nb = axis_owners(gi[bx], ne[bx], g.p, eb, ib);
        const int nc = axis_owners(gi[cx], ne[cx], g.p, ec, ic);
        int ei[3];
        ei[ax] = side ? ne[ax] - 1 : 0;
        double acc = 0.0;
        for (int kc = 0; kc < nc; ++kc)
            for (int kb = 0; kb < nb; ++kb) {
                ei[bx] = eb[kb];
                ei[cx] = ec[kc];
                const int64_t e = ei[0] + (int64_t)g.nx * (ei[1] + (int64_t)g.ny * ei[2]);
                const double *J = affine + 12 * e;
                const double u0 = J[0 * 3 + bx], u1 = J[1 * 3 + bx], u2 = J[2 * 3 + bx];
                const double v0 = J[0 * 3 + cx], v1 = J[1 * 3 + cx], v2 = J[2 * 3 + cx];
                const double c0 = u1 * v2 - u2 * v1, c1 = u2 * v0 - u0 * v2, c2 = u0 * v1 - u1 * v0;
                acc += sqrt(c0 * c0 + c1 * c1 + c2 * c2) * ta.m1[ib[kb]] * ta.m1[ic[kc]];
            }
        const int64_t gn = gi[0] + (int64_t)g.Mx * (gi[1] + (int64_t)g.My * gi[2]);
        for (int c = 0; c < 3; ++c) {
            const int64_t kk = c * g.Nn + gn;
            F[kk] = (ess && ess[kk]) ? T(0) : (T)((double)F[kk] + ta.t[c] * acc);
        }
    }
}

template <typename T>
int launch_traction(const double *affine, T *F, const uint8_t *ess, const double *m1, int face, const double *t,
                    const Grid &g, cudaStream_t s)
{
    TractionArgs ta{};
    for (int i = 0; i <= g.p; ++i) ta.m1[i] = m1[i];
    for (int c = 0; c < 3; ++c) ta.t[c] = t[c];
    ta.face = face;
    const int ax = face / 2;
    const int64_t M[3] = {g.Mx, g.My, g.Mz};
    const int64_t nface = M[ax == 0 ? 1 : 0] * M[ax == 2 ? 1 : 2];
    traction_kernel<T><<<grid_for(nface, 256), 256, 0, s>>>(affine, F, ess, ta, g);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}
template int launch_traction<double>(const double *, double *, const uint8_t *, const double *, int, const double *,
                                     const Grid &, cudaStream_t);
template int launch_traction<float>(const double *, float *, const uint8_t *, const double *, int, const double *,
                                    const Grid &, cudaStream_t);

// -------------------------------------------------------------- diagonal --
struct DiagTables {
    double M[kMaxD], C[kMaxD], K[kMaxD];  // sum_q w B^2, w B G, w G^2
};

// Element part of diag(A) in closed form: for dof (a, c) of element e,
//   sum_mn [ (lambda+mu) detJ Ji[m][c] Ji[n][c] + mu detJ (Ji Ji^T)[m][n] ] S^a_mn
// where S^a_mn = sum_alpha w d_m Phi_a d_n Phi_a factorises into products of
// the 1D sums M, C, K (tensor-product basis, Eq. 6).
template <typename T>
__global__ void diag_elements_kernel(const T *__restrict__ geo, T *__restrict__ ye, DiagTables t, Grid g,
                                     const T *__restrict__ cv)
{
    const int D = g.p + 1, D3 = D * D * D;
    const int64_t total = g.ne * D3;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = o / D3;
        int a = (int)(o - e * D3);
        int i3[3] = {a % D, (a / D) % D, a / (D * D)};
        double S[3][3];
        for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n) {
                double v = 1.0;
                for (int k = 0; k < 3; ++k) {
                    int i = i3[k];
                    v *= (k == m && k == n) ? t.K[i] : ((k == m || k == n) ? t.C[i] : t.M[i]);
                }
                S[m][n] = v;
            }
        const T *gp = geo + e * kGeoStride;
        double Ji[9];
        for (int k = 0; k < 9; ++k) Ji[k] = (double)gp[k];
        double cl = (double)gp[9], cm = (double)gp[10];
        double JJ[3][3];
        for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n)
                JJ[m][n] = Ji[m * 3 + 0] * Ji[n * 3 + 0] + Ji[m * 3 + 1] * Ji[n * 3 + 1] + Ji[m * 3 + 2] * Ji[n * 3 + 2];
        if (cv) {
            // anisotropic: sum_mn S_mn sum_jl Ji[m][j] C_cjcl Ji[n][l], C_cjcl the
            // Voigt entry (v(c,j), v(c,l)) of the element's matrix (times detJ)
            const int vi[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
            const T *ce = cv + e * 21;
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int m = 0; m < 3; ++m)
                    for (int n = 0; n < 3; ++n) {
                        double k2 = 0.0;
                        for (int j = 0; j < 3; ++j)
                            for (int l = 0; l < 3; ++l) {
                                int r = vi[c][j], q = vi[c][l];
                                if (r > q) { const int tmp = r; r = q; q = tmp; }
                                k2 += Ji[m * 3 + j] * (double)ce[r * 6 - r * (r - 1) / 2 + (q - r)] * Ji[n * 3 + l];
                            }
                        s += k2 * S[m][n];
                    }
                ye[(e * 3 + c) * D3 + a] = (T)s;
            }
            continue;
        }
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int m = 0; m < 3; ++m)
                for (int n = 0; n < 3; ++n)
                    s += ((cl + cm) * Ji[m * 3 + c] * Ji[n * 3 + c] + cm * JJ[m][n]) * S[m][n];
            ye[(e * 3 + c) * D3 + a] = (T)s;
        }
    }
}

template <typename T>
int launch_diag_elements(const T *geo, T *ye, const Basis1D &b, const Grid &g, cudaStream_t s, const T *cv)
{
    DiagTables t{};
    for (int i = 0; i < b.D; ++i) {
        t.M[i] = b.Md[i];
        t.C[i] = b.Cd[i];
        t.K[i] = b.Kd[i];
    }
    const int th = 256;
    int64_t total = g.ne * b.D * b.D * b.D;
    diag_elements_kernel<T><<<grid_for(total, th), th, 0, s>>>(geo, ye, t, g, cv);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}
template int launch_diag_elements<double>(const double *, double *, const Basis1D &, const Grid &, cudaStream_t,
                                          const double *);
template int launch_diag_elements<float>(const float *, float *, const Basis1D &, const Grid &, cudaStream_t,
                                         const float *);

// ----------------------------------------------------------- load vector --
constexpr int kMaxModes = 16;
struct RhsParams {
    double B[kMaxD * kMaxQ];
    double qx[kMaxQ], qw[kMaxQ];
    double f0[3];
    double modes[3 * kMaxModes * 5];
    int nmodes;
};

// One CTA per element: f_c(x(alpha)) w_alpha detJ at every quadrature point
// into shared memory, then F_(a,c) = sum_alpha fq_c(alpha) Phi_a(alpha).
template <typename T>
__global__ void rhs_elements_kernel(const double *__restrict__ affine, T *__restrict__ ye, RhsParams P, Grid g)
{
    extern __shared__ double fq[];  // [3][Q^3]
    const int D = g.p + 1, D3 = D * D * D;
    const int Q = g.p + 2, Q3 = Q * Q * Q;
    for (int64_t e = blockIdx.x; e < g.ne; e += gridDim.x) {
        const double *A = affine + e * 12;
        double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
        for (int al = threadIdx.x; al < Q3; al += blockDim.x) {
            int qx = al % Q, qy = (al / Q) % Q, qz = al / (Q * Q);
            double xi[3] = {P.qx[qx], P.qx[qy], P.qx[qz]};
            double X[3];
            for (int i = 0; i < 3; ++i) X[i] = A[9 + i] + A[3 * i] * xi[0] + A[3 * i + 1] * xi[1] + A[3 * i + 2] * xi[2];
            double w = P.qw[qx] * P.qw[qy] * P.qw[qz] * det;
            for (int c = 0; c < 3; ++c) {
                double f = P.f0[c];
                for (int k = 0; k < P.nmodes; ++k) {
                    const double *md = P.modes + (c * P.nmodes + k) * 5;
                    f += md[0] * sin(md[1] * X[0] + md[2] * X[1] + md[3] * X[2] + md[4]);
                }
                fq[c * Q3 + al] = w * f;
            }
        }
        __syncthreads();
        for (int o = threadIdx.x; o < 3 * D3; o += blockDim.x) {
            int c = o / D3, a = o - c * D3;
            int ix = a % D, iy = (a / D) % D, iz = a / (D * D);
            double s = 0.0;
            for (int qz = 0; qz < Q; ++qz)
                for (int qy = 0; qy < Q; ++qy) {
                    double byz = P.B[iy * Q + qy] * P.B[iz * Q + qz];
                    const double *f = fq + c * Q3 + (qz * Q + qy) * Q;
                    double t = 0.0;
                    for (int qx = 0; qx < Q; ++qx) t += f[qx] * P.B[ix * Q + qx];
                    s += t * byz;
                }
            ye[(e * 3 + c) * D3 + a] = (T)s;
        }
        __syncthreads();
    }
}

template <typename T>
int launch_rhs_elements(const double *affine, T *ye, const Basis1D &b, const Grid &g, const double *f0,
                        int nmodes, const double *modes, cudaStream_t s)
{
    if (nmodes < 0 || nmodes > kMaxModes) return set_error(PA_EINVAL, "rhs: at most 16 modes per component");
    if (b.Q != b.p + 2) return set_error(PA_EINVAL, "rhs: q must be p + 2");
    RhsParams P{};
    for (int i = 0; i < b.D * b.Q; ++i) P.B[i] = b.B[i];
    for (int k = 0; k < b.Q; ++k) {
        P.qx[k] = b.qpts[k];
        P.qw[k] = b.qwts[k];
    }
    for (int c = 0; c < 3; ++c) P.f0[c] = f0 ? f0[c] : 0.0;
    P.nmodes = nmodes;
    for (int i = 0; i < 3 * nmodes * 5; ++i) P.modes[i] = modes[i];
    size_t smem = sizeof(double) * 3 * b.Q * b.Q * b.Q;
    int64_t nb = g.ne < (int64_t)152 * 32 ? g.ne : (int64_t)152 * 32;
    rhs_elements_kernel<T><<<(unsigned)nb, 128, smem, s>>>(affine, ye, P, g);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}
template int launch_rhs_elements<double>(const double *, double *, const Basis1D &, const Grid &, const double *, int,
                                         const double *, cudaStream_t);
template int launch_rhs_elements<float>(const double *, float *, const Basis1D &, const Grid &, const double *, int,
                                        const double *, cudaStream_t);

}  // namespace pa
