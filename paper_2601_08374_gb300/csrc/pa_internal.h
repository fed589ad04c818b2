// Internal declarations of the PA elasticity library (not part of the ABI).
#pragma once

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "pa_elasticity.h"

namespace pa {

constexpr int kMaxP = 8;
constexpr int kMaxD = kMaxP + 1;
constexpr int kMaxQ = kMaxP + 2;

// ---------------------------------------------------------------- errors --
int set_error(int code, const std::string &msg);
int cuda_error(cudaError_t e, const char *what);

// A kernel's dynamic shared-memory limit raised once per device (the
// attribute belongs to the device the call is made on): done[] is the
// caller's per-kernel record, indexed by device.
constexpr int kMaxAttrDevices = 64;
template <typename K>
inline int max_smem_once(K kern, bool (&done)[kMaxAttrDevices], int bytes = 227 * 1024)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxAttrDevices) return set_error(PA_EINVAL, "device index out of range");
    if (!done[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
        done[dev] = true;
    }
    return PA_OK;
}

void clear_error();

// NVTX range for tools that record them (Nsight Systems and the like); the
// NVTX v3 header is header-only and costs a branch when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

#define PA_CUDA_TRY(call)                                       \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return ::pa::cuda_error(_e, #call); \
    } while (0)

// ------------------------------------------------------------ 1D rules --
// Gauss-Legendre points/weights on [0,1]; GLL nodes on [0,1]; Lagrange
// values/derivatives (product formula).  Host, double precision.
void gauss_legendre_01(int q, double *x, double *w);
void gll_nodes_01(int p, double *x);
void lagrange_product(int n, const double *nodes, int m, const double *pts, double *val, double *der);

// Reference tables of one (p, q): tab[i*Q + k] layout (dof i, point k).
struct Basis1D {
    int p = 0, D = 0, Q = 0;
    std::vector<double> nodes, qpts, qwts;
    std::vector<double> B, G;    // l_i(xi_k), l_i'(xi_k)
    std::vector<double> Bw, Gw;  // times the weight w_k (transposed sweeps)
    std::vector<double> Md, Cd, Kd;  // sum_k w B^2, w B G, w G^2 per dof i
    void build(int p, int q);
};

// Even row stride of the transposed tables.
constexpr int kTStride = (kMaxD + 1) & ~1;

// Kernel-parameter tables (passed by value; constant-bank operands).
template <typename T>
struct Tables {
    // 16-byte aligned: adjacent entries of an even index load as one pair
    alignas(16) T B[kMaxD * kMaxQ];
    alignas(16) T G[kMaxD * kMaxQ];
    alignas(16) T Bw[kMaxD * kMaxQ];
    alignas(16) T Gw[kMaxD * kMaxQ];
    // FP32 only: Bw and Gw transposed, [q * kTStride + i], zero past i = p,
    // so that the weights of nodes i, i + 1 (i even) at one point q load as
    // one aligned pair
    alignas(16) T BwT[sizeof(T) == 4 ? kMaxQ * kTStride : 1];
    alignas(16) T GwT[sizeof(T) == 4 ? kMaxQ * kTStride : 1];
};

template <typename T>
void fill_tables(const Basis1D &b, Tables<T> &t);

// Fill the transposed tables BwT, GwT (FP32) from Bw, Gw of degree D - 1;
// every table builder ends with this.
template <typename T>
inline void transpose_tables(Tables<T> &t, int D, int Q)
{
    constexpr int nT = (int)(sizeof(t.BwT) / sizeof(T));
    for (int k = 0; k < nT; ++k) t.BwT[k] = t.GwT[k] = T(0);
    if (nT < kMaxQ * kTStride) return;
    for (int i = 0; i < D; ++i)
        for (int q = 0; q < Q; ++q) {
            t.BwT[q * kTStride + i] = t.Bw[i * Q + q];
            t.GwT[q * kTStride + i] = t.Gw[i * Q + q];
        }
}

// Geometry record per element (12 values of the op's precision):
// J^-1 row-major (9), lambda*detJ, mu*detJ, detJ.
constexpr int kGeoStride = 12;
// UA geometry: J row-major per element.
constexpr int kUaStride = 9;

struct Grid {
    int nx, ny, nz, p;
    int Mx, My, Mz;
    int64_t ne, Nn;
    int *flags = nullptr;  // the operator's device status flags (bit 1: an index out of bounds, bounds build)
};

// Bounds-checking build (PA_BOUNDS_CHECK, `build.py --bounds`): every gather
// of x and every E-vector load or store checks its index against the
// array's length; an index outside it sets bit 1 of the grid's status flags
// (read by pa_op_check) and the access is skipped instead of made.  In the
// product build the check is the constant true and compiles away.
#ifdef PA_BOUNDS_CHECK
__device__ __forceinline__ bool pa_in_bounds(const Grid &g, int64_t i, int64_t n)
{
    if (i >= 0 && i < n) return true;
    if (g.flags) atomicOr(g.flags, 2);
    return false;
}
#define PA_INB(g, i, n) ::pa::pa_in_bounds((g), (int64_t)(i), (int64_t)(n))
#else
#define PA_INB(g, i, n) true
#endif

// Fills g for an nx*ny*nz mesh of degree p after checking every size the
// kernels index with: dimensions >= 1, at most 2^31 elements, node counts
// per direction (n p + 1) that fit an int, and at most 2^36 nodes (so byte
// counts of L-vectors, E-vectors and geometry records stay far from 64-bit
// overflow).  PA_EINVAL with a message naming `who` otherwise.
int make_grid(int nx, int ny, int nz, int p, Grid &g, const char *who);

// --------------------------------------------------------- apply launch --
constexpr int kMaxVariant = 7;
struct ApplyLaunch {
    int variant = 0;  // 0: flattened smem sweeps, 1: register-tiled lines, 2: lines + fused gather/store,
                      // 3: as 2 with the Z stage split over three lanes per column,
                      // 4: tensor-core contractions (FP32, p <= 6),
                      // 5: plane-fused sweeps (FP32, p <= 6), 6: as 5 with the Z stage split,
                      // 7: as 2 with the Z stage in two passes (FP32)
    int epb = 1;      // elements per CTA
    int threads = 256;
};

template <typename T>
struct ApplyArgs {
    const T *x;          // L-vector (3*Nn)
    T *ye;               // E-vector scratch [ne][3][D^3]
    const T *geo;        // [ne][kGeoStride]
    const uint8_t *ess;  // [3*Nn] or nullptr
    const int *skip;     // device flag: when non-null and set, the launch does nothing
    Grid g;
    const T *cvoigt = nullptr;   // anisotropic material: 6x6 Voigt matrices times detJ, upper triangle [ne][21]
    int *err = nullptr;          // device flag set by a kernel whose bounded wait on the tensor core ran out
    long long wait_cycles = 4000000000LL;  // that wait's budget in SM clock cycles (about 2 s)
    T *qvec = nullptr;         // ablation stages only: quadrature values [ne][3][3][Q^3]
    const T *ctensor = nullptr;  // ablation stages only: elasticity tensor per element [ne][81]
    // UA geometry (plane kernel): geo holds the 9 entries of each element's J
    // [ne][kUaStride]; the records are recomputed in the kernel with the
    // constant material (ua_lambda, ua_mu)
    int ua = 0;
    T ua_lambda = T(0), ua_mu = T(0);
};

template <typename T>
int launch_apply_elements(const ApplyArgs<T> &a, const Tables<T> &tab, const ApplyLaunch &cfg,
                          cudaStream_t s);

// Operators of one degree and precision applied by one launch.
constexpr int kMaxBatch = 24;
template <typename T>
struct BatchArgs {
    int count;
    int64_t cta_start[kMaxBatch + 1];  // prefix sum of CTAs per operator
    ApplyArgs<T> args[kMaxBatch];
};
template <typename T>
int launch_apply_batch(const BatchArgs<T> &b, int p, const Tables<T> &tab, const ApplyLaunch &cfg, cudaStream_t s);

template <typename T>
struct AssembleBatch {
    int count;
    int64_t node_start[kMaxBatch + 1];  // prefix sum of nodes per operator
    const T *ye[kMaxBatch];
    T *y[kMaxBatch];
    const T *x[kMaxBatch];
    const uint8_t *ess[kMaxBatch];
    Grid g[kMaxBatch];
};
template <typename T>
int launch_assemble_batch(const AssembleBatch<T> &b, cudaStream_t s);

// Operators of any degree in one persistent launch pair (pa_apply_multi.cu):
// the node sums of up to kMaxMulti operators in one assembly launch.
constexpr int kMaxMulti = 96;
template <typename T>
struct AssembleMulti {
    int count;
    int64_t node_start[kMaxMulti + 1];  // prefix sum of nodes per operator
    const T *ye[kMaxMulti];
    T *y[kMaxMulti];
    const T *x[kMaxMulti];
    const uint8_t *ess[kMaxMulti];
    Grid g[kMaxMulti];
};
template <typename T>
int launch_assemble_multi(const AssembleMulti<T> &b, cudaStream_t s);
// Whether the multi launch reproduces the operator's own apply bitwise.
bool multi_eligible(const pa_op *op);
// y_k = A_k x_k for the operators idx of one precision (all multi-eligible):
// one element launch and one assembly launch per kMaxMulti operators.
template <typename T>
int apply_multi_group(pa_op *const *ops, const void *const *xs, void *const *ys, const std::vector<int> &idx,
                      cudaStream_t s);
template <typename T>
size_t apply_smem_bytes(int p, const ApplyLaunch &cfg);
ApplyLaunch default_apply_launch(int p, int precision);

// E-vector -> L-vector sum (owner-computes per node, fixed order);
// constrained rows take xin (or `ess_value` when xin is null).
template <typename T>
int launch_assemble(const T *ye, T *y, const T *xin, const uint8_t *ess, T ess_value, bool accumulate,
                    const Grid &g, cudaStream_t s, const int *skip = nullptr);

// Neumann load of a constant traction on one box face, added to F
// (face = 2 * axis + side); m1 = integrals of the 1D basis functions.
template <typename T>
int launch_traction(const double *affine, T *F, const uint8_t *ess, const double *m1, int face, const double *t,
                    const Grid &g, cudaStream_t s);

// Closed-form PA diagonal per element into the E-vector.
template <typename T>
int launch_diag_elements(const T *geo, T *ye, const Basis1D &b, const Grid &g, cudaStream_t s, const T *cv = nullptr);

// Load vector per element into the E-vector.
template <typename T>
int launch_rhs_elements(const double *affine, T *ye, const Basis1D &b, const Grid &g, const double *f0,
                        int nmodes, const double *modes, cudaStream_t s);

// Apply with an optional device skip flag (used inside device-controlled
// loops); y = A x, or y += A x when accumulate.
int op_apply_async(pa_op *op, const void *x, void *y, bool accumulate, cudaStream_t s, const int *skip);

// y_k = A_k x_k for count operators (not validated): one element launch and
// one assembly launch per (precision, degree) and per kMaxBatch operators.
int apply_batch_async(pa_op *const *ops, const void *const *xs, void *const *ys, int count, cudaStream_t s);

// --------------------------------------------------- lockstep solving --
// Several GMG-PCG solvers (flexible-CG modes) advanced one CG step per tick,
// with the operator applies of all members batched per phase of the step
// (pa_solver.cu).  Members join (lockstep_add: the solve's start, graphs of
// its step) and leave (when converged or capped: true residual, x written)
// between ticks.  Solvers with equal lockstep_key share a lockstep.
struct Lockstep;
struct LockstepDone {
    void *tag = nullptr;
    int status = 0;
    std::string error;
    pa_solve_info info{};
};
int lockstep_create(Lockstep **out);
void lockstep_destroy(Lockstep *L);
int lockstep_add(Lockstep *L, pa_solver *s, const double *b, double *x, double rtol, int maxit, void *tag);
int lockstep_tick(Lockstep *L);
int lockstep_active(const Lockstep *L);
void lockstep_take_done(Lockstep *L, std::vector<LockstepDone> &out);
int lockstep_key(const pa_solver *s);
// Ends member `tag` between ticks with PA_ECANCELED (its LockstepDone is
// queued like a finished member's).
int lockstep_cancel(Lockstep *L, void *tag);
// The solve of s ends with PA_ECANCELED at its next CG step once *flag != 0
// (null: never).
void solver_set_cancel(pa_solver *s, const std::atomic<int> *flag);

}  // namespace pa

// ------------------------------------------------------------- handles --
struct pa_mesh {
    int nx, ny, nz;
    std::vector<double> affine;  // [ne][12]
};

struct pa_op {
    pa::Grid g{};
    int p = 0, q = 0, precision = PA_FP64;
    double lambda = 0, mu = 0;
    size_t elem = 8;  // bytes per scalar
    pa::Basis1D basis;
    pa::Tables<double> tab64{};
    pa::Tables<float> tab32{};
    pa::ApplyLaunch launch{};
    void *d_geo = nullptr;       // [ne][12] of the op's precision
    double *d_affine = nullptr;  // [ne][12] double (rhs only)
    uint8_t *d_ess = nullptr;    // [3*Nn] or null
    void *d_ye = nullptr;        // E-vector scratch
    void *d_xh = nullptr;        // device staging for apply_host
    void *d_yh = nullptr;
    std::vector<double> h_affine;  // host copy of the element maps (solver levels)
    std::vector<double> h_mat;     // per-element (lambda_e, mu_e), empty for the constant material
    std::vector<double> h_cv;      // per-element anisotropic 6x6 Voigt matrices [ne][36], empty if isotropic
    void *d_cv = nullptr;          // device copy: upper triangles times detJ [ne][21] in the op's precision
    int geometry_mode = 0;         // PA_GEOMETRY_STORED or PA_GEOMETRY_UA
    void *d_ua = nullptr;          // UA geometry: J per element [ne][9] in the op's precision
    int *d_err = nullptr;          // set when a tensor-core wait timed out (pa_op_check)
    long long wait_cycles = 4000000000LL;  // budget of those waits (pa_op_set_wait_limit)
    // ablation stages (pa_op_apply_stage), allocated on first use:
    // Q values [ne][9][Q^3], elasticity tensors [ne][81], dense basis-gradient
    // tables [3][D^3][Q^3] and weighted transposed [3][Q^3][D^3]
    void *d_abl[4] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<uint8_t> h_ess;    // host copy of the essential mask (may be empty)
    // measurement: 3 events per recorded apply
    bool prof_on = false;
    int prof_count = 0;
    std::vector<cudaEvent_t> prof_ev;
    int64_t ndofs() const { return 3 * g.Nn; }
};
