/*
 * pa_elasticity.h -- C ABI of the GB300 (sm_103a) matrix-free Partial
 * Assembly operator for high-order linear elasticity on affine hexahedra,
 * and of the p-multigrid preconditioned CG solver that it drives.
 *
 * Method: arXiv 2601.08374, "Shifting the Sweet Spot: High-Performance
 * Matrix-Free Method for High-Order Elasticity".
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - Mesh: structured nx*ny*nz grid of hexahedra, element e = ex + nx*(ey +
 *    ny*ez).  Each element is the image of the reference cell [0,1]^3 under
 *    its own affine map x = x0 + J xi (Sec. 4.4: J^-1 and det J are
 *    constant per element).
 *  - Space: H1 tensor-product Lagrange basis of degree p on the p+1
 *    Gauss-Lobatto-Legendre nodes per direction (Eq. 6; Sec. 5.1.4),
 *    integrated with q Gauss-Legendre points per direction (default
 *    q = p + 2, Sec. 5.1.4).
 *  - L-vector (all x, y, b, d arguments): component-major, 3*Nn entries with
 *    Nn = (nx p + 1)(ny p + 1)(nz p + 1); entry (c, g) at c*Nn + g with the
 *    global node g = gx + (nx p + 1)*(gy + (ny p + 1)*gz).
 *  - Precision: PA_FP64 vectors are double, PA_FP32 vectors are float.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  All apply/solve calls are asynchronous on that stream
 *    unless stated otherwise.
 *  - Memory: device pointers are owned by the caller.  Handles own their
 *    setup data and workspaces, allocated at create/setup time only; no
 *    apply allocates memory.
 *  - Errors: every function returns PA_OK (0) or a positive PA_E* code and
 *    never aborts; pa_last_error() returns a thread-local message for the
 *    last failure on the calling thread.
 */
#ifndef PA_ELASTICITY_H
#define PA_ELASTICITY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum pa_status {
    PA_OK = 0,
    PA_EINVAL = 1,     /* invalid argument (sizes, degree, null handle, det J <= 0) */
    PA_ENOMEM = 2,     /* device or host allocation failed                         */
    PA_ECUDA = 3,      /* a CUDA runtime call failed (message has the CUDA error)  */
    PA_ENOTCONV = 4,   /* solver reached its iteration cap                         */
    PA_EBREAKDOWN = 5, /* solver breakdown: p^T A p <= 0 or a NaN/Inf reduction    */
    PA_ETIMEOUT = 6,   /* a bounded device-side wait expired                       */
    PA_EBUSY = 7,      /* resource busy (e.g. server admission refused)            */
    PA_ECANCELED = 8   /* the request or solve was canceled (pa_server_cancel)    */
};

enum pa_precision { PA_FP64 = 0, PA_FP32 = 1 };

typedef struct pa_mesh pa_mesh;
typedef struct pa_op pa_op;
typedef struct pa_solver pa_solver;
typedef struct pa_server pa_server;

/* Message describing the last error on this thread ("" if none). */
const char *pa_last_error(void);

/* ABI version (major*10000 + minor*100 + patch). */
int pa_version(void);

/* Lame parameters from Young's modulus E > 0 and Poisson ratio -1 < nu < 1/2:
 * lambda = E nu / ((1+nu)(1-2nu)), mu = E / (2(1+nu)).  The operator takes
 * lambda and mu directly (Eq. 3); this helper is a convenience. */
int pa_lame(double E, double nu, double *lambda, double *mu);

/* ---------------------------------------------------------------- mesh -- */

/* Create a structured mesh (host-side description; copied).
 *   nx, ny, nz >= 1 : elements per direction.
 *   box    : host double[6] = {xlo, ylo, zlo, xhi, yhi, zhi}; used only when
 *            affine is NULL (then element maps are the uniform grid of box).
 *   affine : host double[n_e][12] or NULL: per element J (row-major 3x3,
 *            J[i][j] = d x_i / d xi_j) followed by x0[3].
 * Fails with PA_EINVAL if a dimension is < 1 or some det J <= 0. */
int pa_mesh_create(int nx, int ny, int nz, const double *box, const double *affine, pa_mesh **out);
int pa_mesh_destroy(pa_mesh *mesh);

/* ------------------------------------------------------------ operator -- */

/* Partial-assembly setup of the elasticity operator (Sec. 2.2.2 and 4.4: the stored
 * quadrature data D is J^-1 and w det J folded with lambda, mu per element).
 *   p in 1..8, q = 0 (meaning p + 2) or q = p + 2.
 *   lambda, mu : Lame parameters (mu > 0, lambda >= 0 expected).
 *   precision  : PA_FP64 or PA_FP32 (arithmetic and vector type).
 *   ess_mask   : host uint8[3*Nn] or NULL.  Non-zero entries are essential
 *                (Dirichlet) dofs: the operator becomes the constrained one,
 *                y = A z with z = x zeroed on essential dofs, then y = x there.
 * The mesh may be destroyed after this call. */
int pa_op_setup(const pa_mesh *mesh, int p, int q, double lambda, double mu, int precision,
                const uint8_t *ess_mask, pa_op **out);
int pa_op_destroy(pa_op *op);

/* Sizes: number of L-vector entries (3*Nn), elements, degree, precision. */
int pa_op_info(const pa_op *op, int64_t *ndofs, int64_t *nelem, int *p, int *precision);

/* y = A x  (Sec. 4.2-4.5: gather, sum-factorised gradient, Voigt stress,
 * transposed contraction, scatter).  x, y: device L-vectors of the op's
 * precision; they must not alias.  y is overwritten. */
int pa_op_apply(pa_op *op, const void *x, void *y, void *stream);

/* y += A x (the accumulating form of the apply, MFEM's AddMult; Sec.
 * 4.2-4.5 as pa_op_apply): the same computation as pa_op_apply with each node sum added to y instead of
 * stored; on essential dofs y += x (the constrained operator's identity
 * rows).  Same argument rules as pa_op_apply. */
int pa_op_apply_add(pa_op *op, const void *x, void *y, void *stream);

/* y_k = A_k x_k for k < count in few launches.  Operators of one precision
 * whose launch shape the persistent multi-operator kernels reproduce (FP64:
 * variant 0; FP32: variants 2 and 5 up to p = 6, variants 3 and 6 at any
 * degree; isotropic material) are applied by one element launch and one
 * assembly launch per 96 operators, whatever their degrees and sizes: a
 * persistent grid whose CTAs walk the element tiles of all of them, each
 * tile run by the body of its operator's degree.  Every result is bitwise
 * that operator's own apply.  Other operators are grouped by (precision,
 * degree), one launch pair per group of up to 24 (tensor-core shapes run as
 * the register-tiled line variant there, so their bits differ from their
 * own apply, within the FP32 tolerance); anisotropic ones and ones with UA
 * geometry are applied one by one.  No counterpart in the paper (it batches independent
 * applies of Sec. 4.2-4.5).  An operator may appear only once; x_k and y_k
 * must not alias. */
int pa_op_apply_batch(pa_op *const *ops, const void *const *xs, void *const *ys, int count, void *stream);

/* Same computation with host buffers (no counterpart in the paper, whose
 * operator works in host memory): copies x to the device, applies, and
 * copies y back, all on `stream`; returns after y is on the host.  Host
 * buffers should be pinned for full copy bandwidth. */
int pa_op_apply_host(pa_op *op, const void *x_host, void *y_host, void *stream);

/* Several operators applied from host buffers in one call, with the copies
 * overlapped with the applies: y_host[k] = A_k x_host[k] for k < count.
 * The inputs are copied to the device back to back on an internal stream;
 * operator k is applied on `stream` as soon as its input has landed, and its
 * result is copied back on a second internal stream while the following
 * operators compute.  Returns after every y_host[k] is on the host.  Each
 * operator may appear once (its staging vectors carry the copies); host
 * buffers should be pinned, otherwise the copies do not overlap.  Fails with
 * PA_EINVAL for null entries or a repeated operator. */
int pa_op_apply_host_batch(pa_op *const *ops, const void *const *x_host, void *const *y_host, int count,
                           void *stream);

/* d = diag(A) of the constrained operator (essential entries = 1), from the
 * closed form built on 1D sums of w B^2, w B G, w G^2 (Sec. 3.1: the
 * diagonal feeding the Chebyshev-Jacobi smoother).  d: device L-vector. */
int pa_op_diag(pa_op *op, void *d, void *stream);

/* Load vector of a body force (Eq. 5 right-hand side):
 *   F_(i,c) = sum_e sum_alpha w_alpha det J f_c(x(alpha)) Phi_i(alpha),
 *   f_c(x)  = f0[c] + sum_k amp sin(kx x + ky y + kz z + phase),
 * modes: host double[3][nmodes][5] = (amp, kx, ky, kz, phase) or NULL.
 * Essential entries are set to 0.  F: device L-vector of the op's precision. */
int pa_op_rhs(pa_op *op, const double *f0, int nmodes, const double *modes, void *F, void *stream);

/* Per-element material (the PA data D of Sec. 4.5 with lambda(alpha, e),
 * mu(alpha, e) constant on each element, e.g. the paper's two-material
 * beam): lambda_mu = host double[ne][2] (lambda_e, mu_e), element order
 * e = ex + nx (ey + ny ez); NULL restores the operator's constant (lambda,
 * mu).  Rewrites the element geometry records (lambda_e detJ, mu_e detJ) on
 * the device; solvers created afterwards build their coarse levels with the
 * same material.  Synchronous.  PA_EINVAL on non-finite values. */
int pa_op_set_material(pa_op *op, const double *lambda_mu);

/* Anisotropic material (Eq. 2 with a general elasticity tensor): cvoigt =
 * host double[ne][6][6], each a symmetric Voigt matrix in the order
 * [00, 11, 22, 01, 02, 12] acting on engineering strains, sigma_V = C_V
 * eps_V with eps_V = [e00, e11, e22, 2 e01, 2 e02, 2 e12]; it replaces the
 * Lame material (isotropic C_V is lambda in the upper-left 3x3 block plus
 * 2 mu on its diagonal and mu on the shear diagonal).  The element kernel
 * then runs in the flattened variant with a 6x6 product per quadrature
 * point; the diagonal, solver levels (coarse levels inherit the material;
 * the coarsest p = 1 level is solved by Jacobi-CG with operator applies)
 * and loads follow.  NULL restores the isotropic material.  Synchronous.
 * PA_EINVAL for non-finite or non-symmetric matrices.  The batched apply,
 * the ablation stages and the allocation-free apply take isotropic
 * operators only (anisotropic ones are applied one by one in a batch). */
int pa_op_set_anisotropic(pa_op *op, const double *cvoigt);

/* Adds the load of a constant traction t (host double[3]) on one face of
 * the box to F (device L-vector of the op's precision): the Neumann term of
 * the weak form, integral over the face of t . v (Eq. 1), with the op's
 * Gauss rule on each element face and the surface measure of the element's
 * affine map.  face = 2 * axis + side: 0 x = lo, 1 x = hi, 2 y = lo, 3 y = hi,
 * 4 z = lo, 5 z = hi.  Essential entries of F are set to 0.  Asynchronous on
 * `stream`. */
int pa_op_traction(pa_op *op, int face, const double *t, void *F, void *stream);

/* The paper's optimisation stack measured stage by stage (Table 8), y = A x
 * with the operator of pa_op_apply (same Dirichlet handling), FP64 only:
 *   stage 0: baseline -- two kernels with the quadrature values in HBM
 *            between them, dense O(p^6) contractions with the full 3D
 *            basis-gradient tables, stress by the full 81-term C_ijkl
 *            contraction;
 *   stage 1: + sum factorisation (1D sweeps, still two kernels, full C);
 *   stage 2: + Voigt notation (the structured stress of Eq. 7);
 *   stage 3: + fusion: the production apply (pa_op_apply; any precision).
 * Buffers of stages 0-2 (Q values, tensors, dense tables) are allocated on
 * first use and kept by the operator.  Asynchronous on `stream` except for
 * that first allocation.  PA_EINVAL for a stage outside 0..3 or stages 0-2
 * on an FP32 operator. */
int pa_op_apply_stage(pa_op *op, int stage, const void *x, void *y, void *stream);

/* Launch shape of the fused element kernel: variant 0 (flattened
 * shared-memory sweeps, one output per thread step), 1 (register-tiled 1D
 * lines), 2 (register-tiled lines whose X-sweep threads gather and whose
 * X^T-sweep threads store their own lines), 3 (as 2, with the fused Z
 * stage run by three lanes per quadrature column, one per displacement
 * component, exchanging gradient entries by warp shuffles: a third of the
 * registers) or 4 (FP32, p <= 6: the six 1D contractions on the tensor
 * cores, tcgen05.mma kind::tf32 with three TF32 products per contraction
 * for FP32 accuracy, accumulators in TMEM; one shape: 384 threads and
 * floor(128 / (p+2)^2) elements per CTA), 5 (FP32, p <= 6: plane-fused --
 * one thread per (element, component, z-plane) does the X and Y sweeps of
 * its plane in registers, one thread per quadrature column the fused Z
 * stage, one thread per plane the Y^T and X^T sweeps; two barriers per CTA
 * pass), 6 (FP32: as 5 with the Z stage on three lanes per column) or 7
 * (FP32: as 2 with the fused Z stage in two passes through shared memory,
 * half the registers per thread); variants 2, 5, 7 give the same bits, as
 * do 3 and 6; elements per CTA; threads per CTA (32..512, multiple of 32;
 * variants 1-3 and 5-7 at most 256; in FP64 variants 1 and 2 only for
 * p <= 4, variants 4-7 not at all).
 * pa_op_set_launch rejects shapes whose shared memory exceeds 227 KB.
 * pa_op_setup starts from a per-degree default shape; on a mesh with fewer
 * than 2 x 152 x (its elements per CTA) elements the elements per CTA drop
 * to max(1, n_e / 304), so that every SM gets two CTAs where it can. */
int pa_op_set_launch(pa_op *op, int variant, int elems_per_block, int threads);

/* Geometry data of the element kernel.  PA_GEOMETRY_STORED (the default):
 * the stored per-element record of the PA data D (J^-1, lambda detJ,
 * mu detJ, detJ; 12 values).  PA_GEOMETRY_UA: the unassembled evaluation
 * the paper contrasts with PA (Sec. 2, the operator chain: UA recomputes D
 * in every application): only the 9 entries of each element's J are kept
 * ([n_e][9] in the operator's precision, uploaded from the maps given at
 * mesh creation, owned by the operator), and the plane kernel recomputes
 * J^-1, detJ and the material factors per element at the start of each CTA
 * pass.  UA is available for FP32 operators with p <= 6 and the constant
 * isotropic material; it runs in variant 5 (setting UA moves the launch
 * shape to variant 5; pa_op_set_launch then rejects other variants), and
 * pa_op_set_material with a per-element material or pa_op_set_anisotropic
 * return PA_EINVAL while it is set.  Batched applies take UA operators one
 * by one.  The diagonal and the solver levels keep the stored records.
 * Synchronous (one host-to-device copy).  PA_EINVAL for another mode or an
 * operator that does not qualify. */
#define PA_GEOMETRY_STORED 0
#define PA_GEOMETRY_UA 1
int pa_op_set_geometry_mode(pa_op *op, int mode);
int pa_op_get_launch(const pa_op *op, int *variant, int *elems_per_block, int *threads);

/* Reports (and clears) the operator's device status since the last check:
 * PA_OK; PA_ETIMEOUT when a bounded tensor-core wait of an apply timed out
 * (variant 4; that result is not valid); PA_EINVAL when, in the
 * bounds-checking build of the library (build.py --bounds), a kernel met an
 * index outside its array and skipped the access.  Synchronous. */
int pa_op_check(pa_op *op);

/* Budget of the operator's bounded device waits (the tensor-core waits of
 * variant 4), in seconds of SM clock, 0 < seconds <= 60 (default about 2).
 * A wait that runs past it lets the MMAs in flight finish, marks the apply
 * invalid (pa_op_check then returns PA_ETIMEOUT) and ends the kernel; the
 * operator stays usable.  No counterpart in the paper: failure detection of
 * this library. */
int pa_op_set_wait_limit(pa_op *op, double seconds);

/* Autotuner: times every admissible (variant, elements per CTA, threads)
 * with CUDA events on `stream`, applying the operator to the op's own
 * staging vectors (filled with a fixed pattern), and keeps the fastest.
 * Synchronises `stream`. */
int pa_op_autotune(pa_op *op, void *stream);

/* Kernel timing for measurement.  While enabled, every apply records CUDA
 * events on its stream before the element kernel, between the element and
 * the assembly kernel, and after the assembly (at most 4096 applies are
 * kept; later ones are not recorded).  enable = 1 (re)starts the record,
 * enable = 0 stops recording.  pa_op_profile_read synchronises on the last
 * recorded event and returns the summed kernel times in milliseconds and the
 * number of recorded applies. */
int pa_op_profile(pa_op *op, int enable);
int pa_op_profile_read(pa_op *op, double *element_ms, double *assemble_ms, int64_t *applies);

/* Measured multiply-add rate of the CUDA cores in TFLOP/s (2 flops per
 * FMA) for PA_FP64 or PA_FP32 arithmetic: the ceiling of the element
 * kernels, which are bound by those units (Sec. 4: the operator's flops are
 * FMAs of the sum-factorised contractions).  precision = PA_FMA_FP32X2
 * measures FP32 on paired FMA instructions (two FP32 FMAs per instruction,
 * the form the FP32 element kernels use where they can), the same FMA work
 * in half the instructions.  Runs a probe kernel of independent FMA chains
 * over every SM on `stream` (best of five timed launches after one
 * warm-up), allocates and frees a small output buffer, synchronises.
 * PA_EINVAL for another precision.  No counterpart in the paper, which takes
 * its CPUs' peaks from a benchmark tool. */
#define PA_FMA_FP32X2 2
int pa_measure_fma_rate(int precision, double *tflops, void *stream);

/* p-transfer between two operators on the same mesh with degrees
 * pc = coarse->p < pf = fine->p (Sec. 3: polynomial interpolation between the
 * GLL spaces of p-levels).  prolong: xf = P xc evaluates the coarse field at
 * the fine nodes; restrict: rc = P^T rf (exact transpose).  FP64 device
 * L-vectors; no essential-dof masking is applied.  Both operators must be
 * FP64.  The same calls give the h-transfer when both operators are p = 1
 * and the fine mesh has twice the coarse element count in x, y and z (the
 * natural injection of the trilinear space under one uniform refinement:
 * fine node 2I takes coarse node I, an odd fine node the mean of its two
 * coarse neighbours along each axis). */
int pa_op_prolong(const pa_op *coarse, const pa_op *fine, const double *xc, double *xf, void *stream);
int pa_op_restrict(const pa_op *coarse, const pa_op *fine, const double *rf, double *rc, void *stream);

/* Operator apply that allocates no device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- plugins whose host framework owns all device memory through
 * its own pool, and latency-critical loops that must not block on the
 * implicit synchronisation of cudaMalloc/cudaFree.  It computes the same
 * y = A x as pa_op_setup + pa_op_apply, with everything passed in:
 *   nx, ny, nz, p, lambda, mu, precision : as for pa_mesh_create/pa_op_setup
 *                                          (q = p + 2);
 *   affine   : DEVICE double[n_e][12], per element J (row-major) then x0;
 *   ess_mask : DEVICE uint8[3*Nn] or NULL (constrained operator as above);
 *   x, y     : DEVICE L-vectors of `precision`, not aliased.
 * Scratch (geometry records and the element output vector,
 * 12 + 3 (p+1)^3 values per element, the geometry part rounded up to 256
 * bytes, plus 4 bytes) lives in one fixed
 * 64 MiB array in device memory that every GPU loading this library holds
 * until the process exits; meshes needing more are rejected with PA_EINVAL
 * and a message giving the required size.  Nothing in the scratch needs to
 * start at zero: every call overwrites what it reads.  All calls on a device
 * share that array, so calls that overlap on the GPU (other streams, other
 * host threads) race; serialise them.  The first call on a device looks up
 * the array's device address with that device current; make that first call
 * before any stream capture.  Asynchronous on `stream`; an element map with
 * det J <= 0 makes every entry of y NaN. */
int pa_apply_noalloc(int nx, int ny, int nz, int p, double lambda, double mu, int precision, const double *affine,
                     const uint8_t *ess_mask, const void *x, void *y, void *stream);

/* Assembled matrix of an FP64 p = 1 operator (Sec. 3.2: the coarsest level
 * is the one level that is assembled), as a 27-point nodal stencil without
 * essential-dof handling: vals is a DEVICE double array of 81 * 3Nn entries,
 * entry (row, k) at k * 3Nn + row, row = c*Nn + i, k = s*3 + d, where column
 * (d, j) with j = i + dx + Mx (dy + My dz), s = (dx+1) + 3(dy+1) + 9(dz+1);
 * entries whose neighbour lies outside the grid are 0.  The solver uses it
 * for its FP64 coarse CG. */
int pa_op_assemble_p1(const pa_op *op, double *vals, void *stream);

/* -------------------------------------------------------------- solver -- */

typedef struct pa_solve_info {
    int iterations;        /* outer iterations done                              */
    int status;            /* PA_OK, PA_ENOTCONV or PA_EBREAKDOWN                */
    double rel_residual;   /* true ||b - A x|| / ||b|| recomputed in FP64 at exit */
    double b_norm;         /* ||b||_2                                             */
    int inner_iterations;  /* mixed mode: total inner (FP32) iterations           */
    int refinements;       /* mixed mode: outer refinement steps                  */
    double lambda_max[8];  /* per level: power-iteration estimate of max eig(D^-1 A) */
    int coarse_iterations; /* coarse-level CG iterations summed over all V-cycles
                              (counted with graphs on, the default; 0 otherwise) */
    int tolerance_met;     /* 1 when the true residual rel_residual <= rtol, else 0.
                              PA_OK means the solver's own stopping test passed
                              (see pa_gmg_pcg_solve); near the FP64 rounding floor
                              that test can pass while the true residual is above
                              rtol, and this flag tells the two apart */
} pa_solve_info;

/* PA_SOLVE_FP64: everything in FP64.
 * PA_SOLVE_MIXED: FP64 iterative refinement (residual b - A x with the FP64
 *   operator) around an FP32 flexible CG preconditioned by an FP32 V-cycle.
 * PA_SOLVE_MIXED_FCG: FP64 flexible CG (FP64 apply, residual and dot
 *   products) preconditioned by an FP32 V-cycle (FP32 operators, smoothers,
 *   transfers); no restarts, so it keeps the FP64 iteration count.
 * In both mixed modes the coarse-level solve and every dot product are FP64. */
enum pa_solve_mode { PA_SOLVE_FP64 = 0, PA_SOLVE_MIXED = 1, PA_SOLVE_MIXED_FCG = 2 };

/* GMG-PCG solver on the p-hierarchy of `fine` (Sec. 3): levels
 * p_levels[0] = fine degree > p_levels[1] > ... > p_levels[nlev-1], all on the
 * fine mesh with the same essential dofs.  Chebyshev(cheb_order)-Jacobi
 * smoothing, V(1,1), lambda_max from 10 power iterations, interpolation
 * prolongation and its transpose as restriction, and an FP64 Jacobi-CG
 * coarse solve (coarse_rtol, coarse_maxit).  mode PA_SOLVE_MIXED builds FP32
 * copies of the operators and smoothers for an FP64 iterative-refinement
 * outer loop.  `fine` must be FP64 and must outlive the solver. */
int pa_solver_create(pa_op *fine, int nlev, const int *p_levels, int cheb_order, double coarse_rtol,
                     int coarse_maxit, int mode, pa_solver **out);

/* As pa_solver_create, with h_levels geometric levels appended below the
 * p-levels (Sec. 3: the hierarchy of r uniform refinements at p = 1, then
 * p-refinements).  Requires p_levels[nlev-1] = 1 when h_levels > 0 and
 * nlev + h_levels <= 8.  Each h-level is the p = 1 operator (matrix-free PA,
 * Chebyshev-Jacobi smoothed like the p-levels) on the mesh whose uniform
 * refinement is the level above: coarse element (I,J,K) merges fine elements
 * (2I+a, 2J+b, 2K+c), a, b, c in {0,1}, with x0 of child (0,0,0) and twice its
 * J.  Transfers between h-levels are the natural injection of the trilinear
 * space (prolongation) and its exact transpose (restriction).  A coarse dof
 * is essential when its interpolation reaches an essential fine dof.  The
 * coarsest level is solved as in pa_solver_create (assembled p = 1 matrix,
 * CG preconditioned by a Galerkin multigrid on that matrix).
 * Fails with PA_EINVAL if some h-level has an odd element count in any
 * direction, if some coarse element's eight children are not the eighths of
 * one affine map (to 1e-12 relative), or if the per-element material
 * (pa_op_set_material / pa_op_set_anisotropic) differs among them. */
int pa_solver_create_hp(pa_op *fine, int nlev, const int *p_levels, int h_levels, int cheb_order,
                        double coarse_rtol, int coarse_maxit, int mode, pa_solver **out);
int pa_solver_destroy(pa_solver *s);

/* Solver options:
 *  PA_SOLVER_OPT_GRAPHS (default 1): each CG step runs as one captured CUDA
 *    graph; 0: the same kernels are launched one by one.
 *  PA_SOLVER_OPT_PERSISTENT_COARSE (default 1): the FP64 coarse CG on the
 *    assembled p = 1 level runs as one cooperative kernel with bounded grid
 *    barriers (a barrier that waits more than ~2 s makes the solve return
 *    PA_ETIMEOUT); 0: one launch per kernel of every coarse iteration (a
 *    device-controlled graph loop when graphs are on).  Solvers that run
 *    concurrently on one GPU (the server) use 0.
 *  PA_SOLVER_OPT_COARSE_HMG (default 1): the coarse CG on the assembled
 *    p = 1 level is preconditioned by geometric h-multigrid on that level
 *    (structured coarsening, Galerkin stencils, Chebyshev-Jacobi smoothing,
 *    dense solve of the last level) -- the h-levels under the p-levels of the
 *    paper's hierarchy (Sec. 3); 0: Jacobi-preconditioned coarse CG.
 *  PA_SOLVER_OPT_CHEB_LOWER (default 0.05), PA_SOLVER_OPT_CHEB_UPPER
 *    (default 1.2): the Chebyshev smoother (Sec. 3.1) targets the interval
 *    [lower, upper] * lambda_max(D^-1 A) of each smoothed level, lambda_max
 *    its power-iteration estimate; 0 < lower < upper < 100.  Takes effect
 *    at the next solve.  (The upper factor covers the estimate's shortfall:
 *    ten power iterations fall 8-17 % below lambda_max on the measured
 *    problems, and an upper end below lambda_max makes the smoother amplify
 *    the top modes.)
 *  PA_SOLVER_OPT_CHEB_KIND (default 1): 1 -- the first-kind Chebyshev
 *    iteration on [lower, upper] * lambda_max (the paper's smoother, Sec.
 *    3.1); 4 -- the fourth-kind Chebyshev smoother on [0, upper *
 *    lambda_max] (Lottes 2023; no lower bound: after k steps the residual
 *    polynomial is W_k(1 - 2 lambda / (upper lambda_max)) / (2k + 1)).
 *    Same steps and kernels, other coefficients.  Takes effect at the next
 *    solve.  (Not in the paper: a smoother of this library.)
 *  PA_SOLVER_OPT_POWER_ITERS (default 10, Sec. 3.1): power iterations of
 *    the lambda_max estimates, 1..1000; setting it re-estimates every
 *    smoothed level at once (synchronous).
 *  PA_SOLVER_OPT_WAIT_LIMIT (seconds, default 2, at most 60): bound of every
 *    grid-barrier wait of the persistent coarse kernel.  A wait that runs
 *    past it ends the kernel and the solve returns PA_ETIMEOUT; the solver
 *    stays usable.  (No counterpart in the paper: failure detection of this
 *    library.)
 *  PA_SOLVER_OPT_INJECT_INNER_FAILURE (test hook, default 0): k > 0 makes the
 *    k-th inner solve of the next PA_SOLVE_MIXED solve report a breakdown
 *    without running (fault injection on the host); the solve then returns
 *    PA_EBREAKDOWN with info filled and x the last refined iterate.  One
 *    shot: the option returns to 0 when it fires.
 */
enum pa_solver_option {
    PA_SOLVER_OPT_GRAPHS = 1,
    PA_SOLVER_OPT_PERSISTENT_COARSE = 2,
    PA_SOLVER_OPT_COARSE_HMG = 3,
    PA_SOLVER_OPT_CHEB_LOWER = 4,
    PA_SOLVER_OPT_CHEB_UPPER = 5,
    PA_SOLVER_OPT_POWER_ITERS = 6,
    PA_SOLVER_OPT_WAIT_LIMIT = 7,
    PA_SOLVER_OPT_INJECT_INNER_FAILURE = 8,
    PA_SOLVER_OPT_CHEB_KIND = 9
};
int pa_solver_set_option(pa_solver *s, int option, double value);

/* Solve A x = b with the GMG-preconditioned CG of Sec. 3 (x: in = initial
 * guess, out = solution; device double L-vectors).  PA_SOLVE_FP64 and
 * PA_SOLVE_MIXED_FCG: the flexible CG stops when its recursively updated
 * residual satisfies ||r||_2 <= rtol ||b||_2 (the paper tests the
 * preconditioned norm; the relative residual is this library's reading).
 * PA_SOLVE_MIXED: iterative refinement stops when the FP64 residual b - A x
 * satisfies the same test, or when, within a factor 1e3 of the tolerance, a
 * refinement step no longer halves it (the FP64 rounding floor, of order
 * eps ||A|| ||x|| / ||b||, which for stiff bending problems can lie above
 * 1e-10).  info->rel_residual is always the true FP64 residual
 * ||b - A x|| / ||b|| recomputed at exit, and info->tolerance_met says
 * whether that true residual is within rtol (PA_OK alone does not).  maxit caps the outer CG
 * iterations (flexible-CG modes) or the total inner iterations (mixed).
 * Waits for `stream`, runs on the solver's own stream and returns when x is
 * written; returns PA_OK, PA_ENOTCONV or PA_EBREAKDOWN (info filled in every
 * case when non-NULL), PA_ETIMEOUT if a persistent coarse kernel's bounded
 * barrier gave up, PA_EINVAL for a non-finite b. */
int pa_gmg_pcg_solve(pa_solver *s, const double *b, double *x, double rtol, int maxit, pa_solve_info *info,
                     void *stream);

/* Solve count independent systems A_k x_k = b_k together (flexible-CG modes
 * PA_SOLVE_FP64 and PA_SOLVE_MIXED_FCG only, any hierarchies; each solver at
 * most once).  The solves advance in lockstep, one CG step per tick.  A step
 * is split at its operator applies (Sec. 4.2-4.5 on each level of the
 * V-cycle, Sec. 3) into phases; phase round j of a tick runs phase j of every
 * solve that has one and then the applies that end them as one batched
 * apply (pa_op_apply_batch: one persistent launch pair per precision for
 * any mix of degrees); a solve leaves the batch when it converges or
 * reaches maxit.  Every x_k, iteration count and residual is
 * bitwise that of pa_gmg_pcg_solve on the same solver.  b_k, x_k: device
 * double L-vectors (x_k in = initial guess, out = solution); infos: count
 * entries or NULL.  Waits for `stream`, returns when every x_k is written:
 * PA_OK when every solve converged, else the first failing solve's status
 * (each info has its own), PA_EINVAL for bad arguments, a mixed hierarchy or
 * the iterative-refinement mode. */
int pa_gmg_pcg_solve_batch(pa_solver *const *solvers, const double *const *b, double *const *x, int count,
                           double rtol, int maxit, pa_solve_info *infos, void *stream);

/* -------------------------------------------------------------- server -- */

/* Serving of many solves with continuous admission (no counterpart in the
 * paper's CPU study; it drives the same operator and solver).  Requests are
 * queued in arrival order; a request is admitted when one of `max_slots`
 * setup slots is free and its estimated device footprint fits in the memory
 * budget still available.  Its setup (mesh, operators on every level,
 * diagonals, eigenvalue estimates, load vector) runs on a worker thread and
 * CUDA stream of its own.  Then:
 *  - batch lane (flexible-CG modes PA_SOLVE_FP64 / PA_SOLVE_MIXED_FCG, at
 *    most PA_SERVER_OPT_BATCH_MAX_DOFS fine dofs): the request leaves its
 *    slot and joins the lockstep batch of its solve mode -- any degree and
 *    hierarchy depth -- whose stepper thread advances every member one CG
 *    step per tick with the operator applies of all members batched into
 *    one persistent launch pair per precision (see pa_gmg_pcg_solve_batch);
 *    members join and leave between ticks (continuous batching);
 *  - otherwise the worker solves it with pa_gmg_pcg_solve on the solver's
 *    stream, overlapping with everything else on the GPU.
 * Finished requests release their memory and the next queued ones are
 * admitted.  Solves are deterministic: a request gives the same bits alone
 * or in any mix, in either lane. */
#define PA_REQUEST_MAX_MODES 16

typedef struct pa_request {
    int nx, ny, nz;        /* elements per direction                              */
    double box[6];         /* xlo, ylo, zlo, xhi, yhi, zhi of the structured mesh */
    int p;                 /* degree 1..8; levels p, p/2, ..., 1                   */
    double E, nu;          /* material (Lame parameters via pa_lame)               */
    double f0[3];          /* constant body force                                 */
    int nmodes;            /* sine modes per component, <= PA_REQUEST_MAX_MODES    */
    double modes[3 * PA_REQUEST_MAX_MODES * 5]; /* [3][nmodes][5] (amp, kx, ky, kz, phase) */
    int clamp_x0;          /* non-zero: all dofs on the x = xlo face are essential */
    double rtol;           /* solve tolerance (see pa_gmg_pcg_solve)               */
    int maxit;             /* iteration cap                                        */
    int mode;              /* PA_SOLVE_FP64, PA_SOLVE_MIXED or PA_SOLVE_MIXED_FCG  */
    int keep_solution;     /* non-zero: keep x on the host for pa_server_wait      */
} pa_request;

typedef struct pa_request_timing {
    double latency_s;        /* submit to completion                      */
    double queue_s;          /* submit to admission                       */
    double setup_s;          /* operators, diagonals, eigenvalue estimates */
    double solve_s;          /* the solve (in either lane)                */
    int64_t footprint_bytes; /* admission estimate of device memory       */
    int batched;             /* 1: solved in the lockstep batch lane      */
    int levels;              /* multigrid levels of its solver, all told  */
    int h_levels;            /* of which h-levels (PA_SERVER_OPT_H_LEVELS) */
} pa_request_timing;

typedef struct pa_server_stats_t {
    int64_t queued, running, completed, used_bytes, peak_used_bytes;
    int64_t batched;          /* requests solved in the batch lane          */
    int64_t batch_ticks;      /* lockstep steps run (all batches)           */
    int64_t batch_member_ticks; /* sum over steps of the members stepped    */
    int64_t batch_max_members;  /* largest batch seen                       */
} pa_server_stats_t;

/* Server options (pa_server_set_option, before the first submit):
 *  PA_SERVER_OPT_BATCH (default 1): 0 turns the batch lane off (every
 *    request is solved by its worker).
 *  PA_SERVER_OPT_BATCH_MAX_DOFS (default 2,000,000): largest fine-level dof
 *    count that joins the batch lane (larger solves fill the GPU alone).
 *  PA_SERVER_OPT_BATCH_MAX_MEMBERS (default 64, at most 256): members per
 *    lockstep batch; further requests wait for a member to leave.
 *  PA_SERVER_OPT_H_LEVELS (default 1): each request's hierarchy gets h-levels
 *    below its p-levels (pa_solver_create_hp): the element counts are halved
 *    while all three are even, the p = 1 level above has more than 320
 *    dofs, and the hierarchy has at most 8 levels; 0: p-levels only. */
enum pa_server_option {
    PA_SERVER_OPT_BATCH = 1,
    PA_SERVER_OPT_BATCH_MAX_DOFS = 2,
    PA_SERVER_OPT_BATCH_MAX_MEMBERS = 3,
    PA_SERVER_OPT_H_LEVELS = 4
};
int pa_server_set_option(pa_server *s, int option, double value);

/* Uses the device current at creation; budget_bytes > 0; 1 <= max_slots <= 64. */
int pa_server_create(size_t budget_bytes, int max_slots, pa_server **out);
/* Copies *req and queues it; returns at once with a ticket.  A request whose
 * footprint exceeds the whole budget completes with PA_EBUSY. */
int pa_server_submit(pa_server *s, const pa_request *req, int64_t *ticket);
/* *done = 1 once the request has finished. */
int pa_server_poll(pa_server *s, int64_t ticket, int *done);
/* Blocks until the request finishes, then returns its solve status and
 * releases the ticket.  x_host (length x_len = 3 Nn, or NULL) receives the
 * solution if the request kept it; info and timing may be NULL. */
int pa_server_wait(pa_server *s, int64_t ticket, double *x_host, int64_t x_len, pa_solve_info *info,
                   pa_request_timing *timing);
/* Cancels a request: a queued one completes at once with PA_ECANCELED
 * (it held no memory); a running one ends with PA_ECANCELED at its next CG
 * step (solved by a worker) or before the next lockstep tick (batch lane),
 * and its memory is released; a finished one is left as it is.  The caller
 * still collects the ticket with pa_server_wait.  PA_OK, or PA_EINVAL for an
 * unknown ticket.  No counterpart in the paper (a serving control). */
int pa_server_cancel(pa_server *s, int64_t ticket);
int pa_server_stats(pa_server *s, pa_server_stats_t *out);
/* Finishes queued and running requests, then stops the workers. */
int pa_server_destroy(pa_server *s);

#ifdef __cplusplus
}
#endif
#endif /* PA_ELASTICITY_H */
