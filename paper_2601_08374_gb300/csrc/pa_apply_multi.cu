// Persistent apply of many operators of any degree (Sec. 4.2-4.5 for each
// operator; no counterpart in the paper, which applies one operator at a
// time): one element launch and one node-assembly launch for a whole list of
// operators, whatever their degrees and sizes.
//
// The element launch is a persistent grid (as many CTAs as fit on the SMs)
// whose CTAs walk the list of element tiles of all operators -- tile b is
// block b - cta_start[k] of operator k -- and run, per tile, the element
// body of that operator's degree: the flattened shared-memory body in FP64,
// the plane-fused body (p <= 4) or the register-tiled line body (p >= 5) in
// FP32, with the Z stage split over three lanes for the operators whose own
// launch shape uses the split form.  The 1D tables of every degree sit in
// constant memory.  The sums are those of the operator's own launch, so
// every result is bitwise the single apply's.  The assembly launch walks the
// node tiles of all operators the same way.
#include <algorithm>
#include <mutex>

#include "pa_apply.cuh"
#include "pa_apply_line.cuh"
#include "pa_apply_plane.cuh"

#ifndef PA_MULTI_MIN_BLOCKS_F32
#define PA_MULTI_MIN_BLOCKS_F32 1
#endif

namespace pa {

// 1D tables of every degree (q = p + 2), both precisions: filled once per
// device from the same construction as an operator's own tables.
__constant__ Tables<double> c_multi_tab64[kMaxP + 1];
__constant__ Tables<float> c_multi_tab32[kMaxP + 1];

namespace {

constexpr int kMaxDevices = 64;
bool g_tab_ready[kMaxDevices] = {};
std::mutex g_tab_mu;

int ensure_tables()
{
    int dev = 0;
    PA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(PA_EINVAL, "multi apply: device index out of range");
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (g_tab_ready[dev]) return PA_OK;
    static Tables<double> t64[kMaxP + 1];
    static Tables<float> t32[kMaxP + 1];
    for (int p = 1; p <= kMaxP; ++p) {
        Basis1D b;
        b.build(p, p + 2);
        fill_tables(b, t64[p]);
        fill_tables(b, t32[p]);
    }
    PA_CUDA_TRY(cudaMemcpyToSymbol(c_multi_tab64, t64, sizeof(t64)));
    PA_CUDA_TRY(cudaMemcpyToSymbol(c_multi_tab32, t32, sizeof(t32)));
    g_tab_ready[dev] = true;
    return PA_OK;
}

template <typename T>
__device__ __forceinline__ const Tables<T> &multi_tab(int p);
template <>
__device__ __forceinline__ const Tables<double> &multi_tab<double>(int p) { return c_multi_tab64[p]; }
template <>
__device__ __forceinline__ const Tables<float> &multi_tab<float>(int p) { return c_multi_tab32[p]; }

// One operator of a multi launch.
template <typename T>
struct MultiOp {
    const T *x;
    T *ye;
    const T *geo;
    const uint8_t *ess;
    Grid g;
    int epb;    // elements per tile
    int split;  // FP32: fused Z stage on three lanes per column
};


template <typename T>
struct MultiArgs {
    int count;
    int64_t cta_start[kMaxMulti + 1];  // prefix sum of tiles per operator
    MultiOp<T> op[kMaxMulti];
};

// Operator holding tile (or node) t: the last k with start[k] <= t.
__device__ __forceinline__ int find_op(const int64_t *start, int count, int64_t t)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// FP32 line bodies without the split Z stage need 185-255 registers at
// p = 7, 8: the multi kernel holds the split form only for those degrees
// (operators launched unsplit at p >= 7 are applied by the per-degree batch
// path), so that its register count stays that of the lower degrees.
template <typename T, int P>
constexpr bool multi_has_nonsplit()
{
    return sizeof(T) == 8 || P <= 6;
}

// The element body of degree P for one tile.
template <typename T, int P>
__device__ __forceinline__ void multi_tile(const ApplyArgs<T> &a, int epb, int64_t blk, int split)
{
    constexpr int D = P + 1, Q = P + 2;
    const Tables<T> &tab = multi_tab<T>(P);
    if constexpr (sizeof(T) == 8) {
        flat_body<T, D, Q>(a, tab, epb, blk);
    } else if constexpr (P <= 4) {
        if (split) plane_body<T, D, Q, true>(a, tab, epb, blk);
        else plane_body<T, D, Q, false>(a, tab, epb, blk);
    } else if constexpr (multi_has_nonsplit<T, P>()) {
        if (split) line_body<T, D, Q, true, true>(a, tab, epb, blk);
        else line_body<T, D, Q, true, false>(a, tab, epb, blk);
    } else {
        line_body<T, D, Q, true, true>(a, tab, epb, blk);
    }
}

// Threads per CTA and the minimum CTAs per SM the register allocation must
// allow (every degree's body shares one register count: the largest).
template <typename T>
constexpr int kMultiThreads = sizeof(T) == 8 ? 256 : 128;
template <typename T>
constexpr int kMultiMinBlocks = sizeof(T) == 8 ? 1 : PA_MULTI_MIN_BLOCKS_F32;

template <typename T>
__global__ void __launch_bounds__(kMultiThreads<T>, kMultiMinBlocks<T>) pa_apply_multi_kernel(MultiArgs<T> m)
{
    const int64_t total = m.cta_start[m.count];
    for (int64_t b = blockIdx.x; b < total; b += gridDim.x) {
        const int k = find_op(m.cta_start, m.count, b);
        const MultiOp<T> &o = m.op[k];
        ApplyArgs<T> a;
        a.x = o.x;
        a.ye = o.ye;
        a.geo = o.geo;
        a.ess = o.ess;
        a.skip = nullptr;
        a.g = o.g;
        const int64_t blk = b - m.cta_start[k];
        switch (o.g.p) {
#define PA_MULTI_CASE(P) \
    case P: multi_tile<T, P>(a, o.epb, blk, o.split); break;
            PA_MULTI_CASE(1) PA_MULTI_CASE(2) PA_MULTI_CASE(3) PA_MULTI_CASE(4)
            PA_MULTI_CASE(5) PA_MULTI_CASE(6) PA_MULTI_CASE(7) PA_MULTI_CASE(8)
#undef PA_MULTI_CASE
        default: break;
        }
        __syncthreads();  // the next tile reuses the shared memory
    }
}

// Shared memory of one tile of degree p with epb elements.
template <typename T>
size_t multi_tile_smem(int p, int epb, bool split)
{
    ApplyLaunch c;
    c.epb = epb;
    c.threads = 128;
    if (sizeof(T) == 8) c.variant = 0;
    else c.variant = p <= 4 ? (split ? 6 : 5) : (split ? 3 : 2);
    return apply_smem_bytes<T>(p, c);
}

}  // namespace

// Whether the multi launch gives an operator the bits of its own apply: its
// launch shape uses a body the multi kernel holds for its degree.
bool multi_eligible(const pa_op *op)
{
    if (op->d_cv || op->g.Nn >= ((int64_t)1 << 31)) return false;
    const int v = op->launch.variant;
    if (op->precision == PA_FP64) return v == 0;
    if (v == 3 || v == 6) return true;
    return (v == 2 || v == 5 || v == 7) && op->p <= 6;
}

template <typename T>
int apply_multi_group(pa_op *const *ops, const void *const *xs, void *const *ys, const std::vector<int> &idx,
                      cudaStream_t s)
{
    if (int rc = ensure_tables()) return rc;
    const int threads = kMultiThreads<T>;
    int dev = 0, nsm = 0;
    PA_CUDA_TRY(cudaGetDevice(&dev));
    PA_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    static bool smem_set[kMaxAttrDevices] = {};
    if (int rc = max_smem_once(pa_apply_multi_kernel<T>, smem_set)) return rc;
    // the operators of one degree next to each other in the tile list, the
    // highest degree first: the CTAs walk the list in step, so at any time
    // they run the bodies of one or two degrees (whose code then stays in
    // the instruction cache), and the longest tiles start first
    std::vector<int> order(idx);
    std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return ops[u]->p > ops[v]->p; });
    for (size_t c0 = 0; c0 < order.size(); c0 += kMaxMulti) {
        const size_t m = std::min(order.size() - c0, (size_t)kMaxMulti);
        MultiArgs<T> ma{};
        AssembleMulti<T> mb{};
        ma.count = mb.count = (int)m;
        ma.cta_start[0] = mb.node_start[0] = 0;
        size_t smem = 0;
        for (size_t j = 0; j < m; ++j) {
            pa_op *op = ops[order[c0 + j]];
            MultiOp<T> &o = ma.op[j];
            o.x = static_cast<const T *>(xs[order[c0 + j]]);
            o.ye = static_cast<T *>(op->d_ye);
            o.geo = static_cast<const T *>(op->d_geo);
            o.ess = op->d_ess;
            o.g = op->g;
            const int v = op->launch.variant;
            o.split = (sizeof(T) == 4 && (v == 3 || v == 6 || op->p >= 7)) ? 1 : 0;
            // the degree's default tile, made smaller for a small operator so
            // that its elements still spread over several tiles
            o.epb = default_apply_launch(op->p, op->precision).epb;
            if (op->g.ne < 4 * (int64_t)o.epb) o.epb = (int)std::max<int64_t>(1, op->g.ne / 4);
            smem = std::max(smem, multi_tile_smem<T>(op->p, o.epb, o.split != 0));
            ma.cta_start[j + 1] = ma.cta_start[j] + (op->g.ne + o.epb - 1) / o.epb;
            mb.ye[j] = o.ye;
            mb.y[j] = static_cast<T *>(ys[order[c0 + j]]);
            mb.x[j] = o.x;
            mb.ess[j] = op->d_ess;
            mb.g[j] = op->g;
            mb.node_start[j + 1] = mb.node_start[j] + op->g.Nn;
        }
        if (smem == 0 || smem > 227 * 1024) return set_error(PA_EINVAL, "multi apply: tile shared memory not admissible");
        int per_sm = 0;
        PA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pa_apply_multi_kernel<T>, threads, smem));
        if (per_sm < 1) return set_error(PA_EINVAL, "multi apply: no CTA fits on an SM");
        const int64_t tiles = ma.cta_start[m];
        const int64_t grid = std::min<int64_t>(tiles, (int64_t)per_sm * nsm);
        if (grid > 0) {
            pa_apply_multi_kernel<T><<<(unsigned)grid, threads, smem, s>>>(ma);
            PA_CUDA_TRY(cudaGetLastError());
        }
        if (int rc = launch_assemble_multi<T>(mb, s)) return rc;
    }
    return PA_OK;
}

template int apply_multi_group<double>(pa_op *const *, const void *const *, void *const *, const std::vector<int> &,
                                       cudaStream_t);
template int apply_multi_group<float>(pa_op *const *, const void *const *, void *const *, const std::vector<int> &,
                                      cudaStream_t);

}  // namespace pa
