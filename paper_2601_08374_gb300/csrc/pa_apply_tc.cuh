// Tensor-core variant of the fused element kernel for FP32 (variant 4):
// the six 1D contractions of the PA apply (Sec. 4.4, the forward X/Y/Z
// sweeps and the transposed Z/Y/X sweeps of Sec. 4.5) run on the 5th-gen
// tensor cores (tcgen05.mma kind::tf32, accumulators in TMEM), the gather,
// the pointwise Voigt stress (Eq. 7) and the layout changes between sweeps
// on the CUDA cores.
//
// A CTA takes E consecutive elements, E = floor(128 / Q^2), so that every
// sweep's lines fit one M = 128 tile: the lines of a sweep are the rows of
// the A operand, the contracted index its K, and the channels of a line
// (component c and the value / derivative channels) separate K slices of 8,
// each multiplied by its own 16 x 8 table (B, G or their weighted forms,
// zero-padded) into its own 16-column block of TMEM.  FP32 accuracy comes
// from three TF32 products per contraction, a_lo b_hi + a_hi b_lo + a_hi b_hi
// (a = a_hi + a_lo with a_hi the TF32 rounding of a).
//
//   X    rows (el, iz, iy)   slices c            K = ix   table [B | G]
//   Y    rows (el, iz, qx)   slices (c, u/v)      K = iy   [B | G] / [B]
//   Z    rows (el, qy, qx)   slices (c, k)        K = iz   [B] (k < 2) / [G]
//   pointwise per row: the 9 gradients at each qz -> 9 Q values
//   Z^T  rows (el, qy, qx)   slices (c, m)        K = qz   [Bw] / [Gw] (m = 2)
//   Y^T  rows (el, iz, qx)   slices (c, m)        K = qy   U0 = T0 Bw, U12 = T1 Gw + T2 Bw
//   X^T  rows (el, iz, iy)   slices (c, U0/U12)   K = qx   y = U0 Gw + U12 Bw
//
// Three threads per TMEM lane (384 threads; warps w, w + 4, w + 8 read the
// same lane quarter): thread part c handles displacement component c of its
// line (the pointwise stage: every third quadrature point).  After each
// sweep a thread reads its line's accumulators and writes the values, split
// into TF32 hi / lo, to the rows of the next sweep's A operand (a transpose
// through shared memory).  Operands are K-major without swizzle: core matrices of 8 rows x
// 16 bytes, LBO 128 B along K, SBO (K / 4) * 128 B along M.  Every wait on
// the tensor core is bounded (the operator's wait budget, then a drain of
// the MMAs in flight); on timeout the kernel flags a.err, frees its TMEM and
// returns.
#pragma once

#include <cstdint>

#include "pa_internal.h"

namespace pa {

namespace tc {

constexpr int kRows = 128;            // M of every MMA
constexpr int kSlices = 9;            // most K slices of a sweep
constexpr int kKT = kSlices * 8;      // K extent of the A buffer (floats)
constexpr int kSBO = (kKT / 4) * 128;  // bytes between 8-row groups of A
constexpr int kAbytes = (kRows / 8) * kSBO;  // one A part (hi or lo)
constexpr int kTab = 16 * 8;          // floats of one 16 x 8 table
constexpr int kNumTab = 5;            // [B|G], [B], [G], [Bw], [Gw]
constexpr int kTmemCols = 256;

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row, k) in a K-major, no-swizzle operand with SBO sbo
__host__ __device__ __forceinline__ int off(int r, int k, int sbo)
{
    return (r >> 3) * sbo + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint64_t desc(uint32_t start, uint32_t sbo)
{
    return (uint64_t)((start >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) |
           ((uint64_t)1 << 46);
}

// D f32, A and B tf32, K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtm),
                 "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ float tf32_hi(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// 16 columns of this thread's TMEM lane
__device__ __forceinline__ void ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// one column of this thread's TMEM lane
__device__ __forceinline__ float ld1(uint32_t taddr)
{
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    return __uint_as_float(r);
}

__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;"); }

// writes value v (split) at (row, k) of the A operand
__device__ __forceinline__ void put(unsigned char *Ahi, unsigned char *Alo, int r, int k, float v)
{
    const float h = tf32_hi(v);
    const int o = off(r, k, kSBO);
    *reinterpret_cast<float *>(Ahi + o) = h;
    *reinterpret_cast<float *>(Alo + o) = v - h;
}

}  // namespace tc

// Tables of variant 4 (kernel parameter): [B|G], [B], [G] with K = node
// index i and N = point index q; [Bw], [Gw] with K = q and N = i; each as
// TF32 hi and lo parts (FP32 values).
struct TcTables {
    float hi[tc::kNumTab][16][8];
    float lo[tc::kNumTab][16][8];
};

template <int D, int Q>
__device__ __forceinline__ void tc_issue(int sweep, uint32_t tmem, const unsigned char *Ahi, const unsigned char *Alo,
                                         const unsigned char *Thi, const unsigned char *Tlo)
{
    using namespace tc;
    // (A slice, table, TMEM block, first product into the block)
    int n = 0, sl[9], tb[9], blk[9], first[9];
    auto add = [&](int s, int t, int b, int f) {
        sl[n] = s;
        tb[n] = t;
        blk[n] = b;
        first[n] = f;
        ++n;
    };
    switch (sweep) {
    case 0:  // X
        for (int c = 0; c < 3; ++c) add(c, 0, c, 1);
        break;
    case 1:  // Y: u slices with [B|G] (d2, d1), v slices with [B] (d0)
        for (int c = 0; c < 3; ++c) {
            add(2 * c, 0, 2 * c, 1);
            add(2 * c + 1, 1, 2 * c + 1, 1);
        }
        break;
    case 2:  // Z
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 3; ++k) add(3 * c + k, k == 2 ? 2 : 1, 3 * c + k, 1);
        break;
    case 3:  // Z^T
        for (int c = 0; c < 3; ++c)
            for (int m = 0; m < 3; ++m) add(3 * c + m, m == 2 ? 4 : 3, 3 * c + m, 1);
        break;
    case 4:  // Y^T: U0 = T0 Bw, U12 = T1 Gw + T2 Bw
        for (int c = 0; c < 3; ++c) {
            add(3 * c, 3, 2 * c, 1);
            add(3 * c + 1, 4, 2 * c + 1, 1);
            add(3 * c + 2, 3, 2 * c + 1, 0);
        }
        break;
    default:  // X^T: y = U0 Gw + U12 Bw
        for (int c = 0; c < 3; ++c) {
            add(2 * c, 4, c, 1);
            add(2 * c + 1, 3, c, 0);
        }
        break;
    }
    const uint32_t ahi = saddr(Ahi), alo = saddr(Alo), thi = saddr(Thi), tlo = saddr(Tlo);
    for (int j = 0; j < n; ++j) {
        const uint32_t aoff = (uint32_t)sl[j] * 256u, toff = (uint32_t)tb[j] * (uint32_t)(kTab * 4);
        const uint32_t d = tmem + (uint32_t)blk[j] * 16u;
        const uint64_t Ah = desc(ahi + aoff, kSBO), Al = desc(alo + aoff, kSBO);
        const uint64_t Bh = desc(thi + toff, 256), Bl = desc(tlo + toff, 256);
        mma(d, Al, Bh, first[j] ? 0u : 1u);
        mma(d, Ah, Bl, 1u);
        mma(d, Ah, Bh, 1u);
    }
}

constexpr int kTcThreads = 384;

template <int D, int Q>
__global__ void __launch_bounds__(kTcThreads, 2) pa_apply_tc_kernel(ApplyArgs<float> a, TcTables tt, int64_t nbatch)
{
    using namespace tc;
    constexpr int E = kRows / (Q * Q);
    constexpr int D3 = D * D * D;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Ahi = smem, *Alo = smem + kAbytes;
    unsigned char *Thi = smem + 2 * kAbytes, *Tlo = Thi + kNumTab * kTab * 4;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(Tlo + kNumTab * kTab * 4);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & 127, part = tid >> 7;  // line (TMEM lane) and component
    const Grid &g = a.g;
    const int p = D - 1;
    const int64_t Nn = g.Nn, Mx = g.Mx, MxMy = (int64_t)g.Mx * g.My;

    // tables to their canonical layout; the A buffers zeroed (padding entries
    // must be finite: they meet zero table entries)
    for (int i = tid; i < kNumTab * 16 * 8; i += kTcThreads) {
        const int t = i / 128, r = (i / 8) % 16, k = i % 8;
        *reinterpret_cast<float *>(Thi + t * kTab * 4 + off(r, k, 256)) = tt.hi[t][r][k];
        *reinterpret_cast<float *>(Tlo + t * kTab * 4 + off(r, k, 256)) = tt.lo[t][r][k];
    }
    for (int i = tid; i < 2 * kAbytes / 16; i += kTcThreads)
        reinterpret_cast<float4 *>(smem)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    uint32_t phase = 0;
    bool ok = true;

    // one sweep: A written -> MMAs -> wait; false on timeout
    auto run = [&](int sweep) -> bool {
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            tc_issue<D, Q>(sweep, tmem, Ahi, Alo, Thi, Tlo);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(mbar)));
        }
        uint32_t done = 0;
        // the operator's wait budget (a.wait_cycles of SM clock)
        const long long t0 = clock64();
        while (!done && clock64() - t0 < a.wait_cycles)
            asm volatile("{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}"
                         : "=r"(done) : "r"(saddr(mbar)), "r"(phase));
        const bool late = !done;
        // past the budget the sweep counts as failed, but the MMAs in flight
        // must still finish before the TMEM they write is reused or freed:
        // drain with the fixed bound
        for (int it = 0; it < (1 << 24) && !done; ++it)
            asm volatile("{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}"
                         : "=r"(done) : "r"(saddr(mbar)), "r"(phase));
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // one decision for the whole CTA (every thread leaves or stays)
        return __syncthreads_or(late || !done) == 0;
    };

    for (int64_t b = blockIdx.x; b < nbatch && ok; b += gridDim.x) {
        if (a.skip && *a.skip) break;
        const int64_t e0 = b * E;
        const int ne = (int)((g.ne - e0) < E ? (g.ne - e0) : E);
        float v[16];

        // ---- gather: row (el, iz, iy), slice c = part, K = ix
        if (row < ne * D * D) {
            const int el = row / (D * D), iz = (row / D) % D, iy = row % D;
            const int64_t e = e0 + el, t = e / g.nx;
            const int ex = (int)(e - t * g.nx), ey = (int)(t % g.ny), ez = (int)(t / g.ny);
            const int64_t base = (int64_t)ex * p + Mx * ((int64_t)ey * p + iy) + MxMy * ((int64_t)ez * p + iz);
            const int c = part;
#pragma unroll
            for (int ix = 0; ix < D; ++ix) {
                const int64_t k = c * Nn + base + ix;
                const bool in = PA_INB(a.g, k, 3 * Nn);
                float xv = in ? a.x[k] : 0.f;
                if (in && a.ess && a.ess[k]) xv = 0.f;
                put(Ahi, Alo, row, 8 * c + ix, xv);
            }
        }
        if (!(ok = run(0))) break;
        // ---- X out: row (el, iz, iy); blocks c: u[qx] cols < Q, v[qx] cols Q..2Q-1
        //      -> Y rows (el, iz, qx), slices (c, u/v), K = iy
        {
            const bool act = row < ne * D * D;
            const int el = row / (D * D), iz = (row / D) % D, iy = row % D;
            const int c = part;
            ld16(lane_base + 16 * c, v);
            ld_wait();
            if (act)
#pragma unroll
                for (int qx = 0; qx < Q; ++qx) {
                    const int r = (el * D + iz) * Q + qx;
                    put(Ahi, Alo, r, 8 * (2 * c) + iy, v[qx]);
                    put(Ahi, Alo, r, 8 * (2 * c + 1) + iy, v[Q + qx]);
                }
        }
        if (!(ok = run(1))) break;
        // ---- Y out: row (el, iz, qx); block 2c: d2[qy] cols < Q, d1[qy] cols Q..; block 2c+1: d0[qy]
        //      -> Z rows (el, qy, qx), slices (c, k), K = iz
        {
            const bool act = row < ne * D * Q;
            const int el = row / (D * Q), iz = (row / Q) % D, qx = row % Q;
            const int c = part;
            float w[16];
            ld16(lane_base + 16 * (2 * c), v);
            ld16(lane_base + 16 * (2 * c + 1), w);
            ld_wait();
            if (act)
#pragma unroll
                for (int qy = 0; qy < Q; ++qy) {
                    const int r = (el * Q + qy) * Q + qx;
                    put(Ahi, Alo, r, 8 * (3 * c + 0) + iz, w[qy]);      // d0: d/dxi
                    put(Ahi, Alo, r, 8 * (3 * c + 1) + iz, v[Q + qy]);  // d1: d/deta
                    put(Ahi, Alo, r, 8 * (3 * c + 2) + iz, v[qy]);      // d2: interpolated
                }
        }
        if (!(ok = run(2))) break;
        // ---- Z out + pointwise: row (el, qy, qx); block 3c+k: gr[c][k] at qz (cols < Q)
        //      -> Z^T rows (el, qy, qx) (the same), slices (c, m), K = qz
        {
            const bool act = row < ne * Q * Q;
            const int el = act ? row / (Q * Q) : 0;
            const float *geo = a.geo + (e0 + el) * kGeoStride;
            float Ji[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) Ji[i] = act ? geo[i] : 0.f;
            const float cl = act ? geo[9] : 0.f, cm = act ? geo[10] : 0.f, m2 = cm + cm;
#pragma unroll 1
            for (int qz = part; qz < Q; qz += 3) {
                // the nine reference-gradient entries at this point (column qz of blocks 0..8)
                float gq[9];
#pragma unroll
                for (int s2 = 0; s2 < 9; ++s2) gq[s2] = ld1(lane_base + 16 * s2 + qz);
                ld_wait();
                if (act) {
                    float du[3][3];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            du[c][j] = fmaf(Ji[0 * 3 + j], gq[3 * c + 0],
                                            fmaf(Ji[1 * 3 + j], gq[3 * c + 1], Ji[2 * 3 + j] * gq[3 * c + 2]));
                    const float ld = cl * (du[0][0] + du[1][1] + du[2][2]);
                    float s3[3][3];
                    s3[0][0] = fmaf(m2, du[0][0], ld);
                    s3[1][1] = fmaf(m2, du[1][1], ld);
                    s3[2][2] = fmaf(m2, du[2][2], ld);
                    s3[0][1] = s3[1][0] = cm * (du[0][1] + du[1][0]);
                    s3[0][2] = s3[2][0] = cm * (du[0][2] + du[2][0]);
                    s3[1][2] = s3[2][1] = cm * (du[1][2] + du[2][1]);
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int m = 0; m < 3; ++m)
                            put(Ahi, Alo, row, 8 * (3 * c + m) + qz,
                                fmaf(s3[c][0], Ji[m * 3 + 0], fmaf(s3[c][1], Ji[m * 3 + 1], s3[c][2] * Ji[m * 3 + 2])));
                }
            }
        }
        if (!(ok = run(3))) break;
        // ---- Z^T out: row (el, qy, qx); block 3c+m: T[c][m][iz] (cols < D)
        //      -> Y^T rows (el, iz, qx), slices (c, m), K = qy
        {
            const bool act = row < ne * Q * Q;
            const int el = row / (Q * Q), qy = (row / Q) % Q, qx = row % Q;
#pragma unroll
            for (int s = 3 * part; s < 3 * part + 3; ++s) {
                ld16(lane_base + 16 * s, v);
                ld_wait();
                if (act)
#pragma unroll
                    for (int iz = 0; iz < D; ++iz) put(Ahi, Alo, (el * D + iz) * Q + qx, 8 * s + qy, v[iz]);
            }
        }
        if (!(ok = run(4))) break;
        // ---- Y^T out: row (el, iz, qx); block 2c: U0[iy], block 2c+1: U12[iy]
        //      -> X^T rows (el, iz, iy), slices (c, U0/U12), K = qx
        {
            const bool act = row < ne * D * Q;
            const int el = row / (D * Q), iz = (row / Q) % D, qx = row % Q;
#pragma unroll
            for (int s = 2 * part; s < 2 * part + 2; ++s) {
                ld16(lane_base + 16 * s, v);
                ld_wait();
                if (act)
#pragma unroll
                    for (int iy = 0; iy < D; ++iy) put(Ahi, Alo, (el * D + iz) * D + iy, 8 * s + qx, v[iy]);
            }
        }
        if (!(ok = run(5))) break;
        // ---- X^T out: row (el, iz, iy); block c: y[c][ix] -> E-vector
        {
            const bool act = row < ne * D * D;
            const int el = row / (D * D), iz = (row / D) % D, iy = row % D;
            const int c = part;
            ld16(lane_base + 16 * c, v);
            ld_wait();
            const int64_t ob = ((e0 + el) * 3 + c) * D3 + (iz * D + iy) * D;
            if (act && PA_INB(a.g, ob, g.ne * 3 * D3) && PA_INB(a.g, ob + D - 1, g.ne * 3 * D3)) {
                float *out = a.ye + ob;
#pragma unroll
                for (int ix = 0; ix < D; ++ix) out[ix] = v[ix];
            }
        }
    }
    if (!ok && tid == 0 && a.err) atomicOr(a.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// Shared memory of variant 4: two A parts, the tables, an mbarrier and the TMEM slot.
constexpr size_t tc_smem_bytes() { return 2 * (size_t)tc::kAbytes + 2 * (size_t)tc::kNumTab * tc::kTab * 4 + 16; }

// Elements per CTA of variant 4 (0: not instantiated for this degree).
constexpr int tc_elems(int D, int Q) { return (D <= 8 && Q <= 8) ? tc::kRows / (Q * Q) : 0; }

TcTables tc_tables(const Tables<float> &tab, int D, int Q);

template <int D, int Q>
int launch_tc(const ApplyArgs<float> &a, const TcTables &tt, cudaStream_t s)
{
    constexpr int E = tc::kRows / (Q * Q);
    const int64_t nbatch = (a.g.ne + E - 1) / E;
    if (nbatch <= 0) return PA_OK;
    auto kern = pa_apply_tc_kernel<D, Q>;
    static bool smem_set[kMaxAttrDevices] = {};
    if (int rc = max_smem_once(kern, smem_set, (int)tc_smem_bytes())) return rc;
    const int64_t grid = nbatch < 2 * 152 ? nbatch : 2 * 152;
    kern<<<(unsigned)grid, kTcThreads, tc_smem_bytes(), s>>>(a, tt, nbatch);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

}  // namespace pa
