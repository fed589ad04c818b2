// Setup of the GMG-PCG solver (Sec. 3): the p- and h-level hierarchy, level
// operators and masks, assembled coarse stencils and their Galerkin
// products, the dense coarsest inverse, the power-iteration estimates of
// lambda_max that set the Chebyshev intervals (Sec. 3.1), the solver
// options and destruction.
#include "pa_solver_kernels.cuh"

namespace pa {


template <typename T>
int dalloc(pa_solver *s, T **ptr, int64_t n)
{
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(T) * (size_t)(n > 0 ? n : 1));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? set_error(PA_ENOMEM, "solver: device allocation")
                                                                 : cuda_error(e, "solver: cudaMalloc");
    s->allocs.push_back(p);
    *ptr = static_cast<T *>(p);
    return PA_OK;
}

// coarse essential mask: coarse dof j is essential when the coarse basis
// function j is non-zero at some essential fine dof (exact for essential sets
// made of whole element faces).
std::vector<uint8_t> coarse_mask(const std::vector<uint8_t> &fine, const Grid &gf, int pc, const Basis1D &bc,
                                 const Basis1D &bf)
{
    const int pf = gf.p;
    std::vector<double> val((size_t)(pc + 1) * (pf + 1)), der(val.size());
    lagrange_product(pc + 1, bc.nodes.data(), pf + 1, bf.nodes.data(), val.data(), der.data());
    const int Mxc = gf.nx * pc + 1, Myc = gf.ny * pc + 1, Mzc = gf.nz * pc + 1;
    const int64_t Nnc = (int64_t)Mxc * Myc * Mzc;
    std::vector<uint8_t> out((size_t)3 * Nnc, 0);
    auto owners = [&](int i, int n, int *cj) {
        int k = std::min(i / pf, n - 1), jl = i - k * pf, cnt = 0;
        for (int a = 0; a <= pc; ++a)
            if (std::fabs(val[a * (pf + 1) + jl]) > 1e-14) cj[cnt++] = k * pc + a;
        return cnt;
    };
    int cx[kMaxD + 1], cy[kMaxD + 1], cz[kMaxD + 1];
    for (int c = 0; c < 3; ++c)
        for (int64_t gn = 0; gn < gf.Nn; ++gn) {
            if (!fine[(size_t)c * gf.Nn + gn]) continue;
            int gx = (int)(gn % gf.Mx), gy = (int)((gn / gf.Mx) % gf.My), gz = (int)(gn / ((int64_t)gf.Mx * gf.My));
            int nxa = owners(gx, gf.nx, cx), nya = owners(gy, gf.ny, cy), nza = owners(gz, gf.nz, cz);
            for (int k = 0; k < nza; ++k)
                for (int j = 0; j < nya; ++j)
                    for (int i = 0; i < nxa; ++i)
                        out[(size_t)c * Nnc + cx[i] + (int64_t)Mxc * (cy[j] + (int64_t)Myc * cz[k])] = 1;
        }
    return out;
}

// Element data of one level's mesh: the fine operator's, or the mesh whose
// uniform refinement is the level above (Sec. 3: the h-levels of the
// hierarchy come from r uniform refinements of a coarse mesh).
struct LevelMesh {
    int nx = 0, ny = 0, nz = 0;
    std::vector<double> affine;  // [ne][12]: J row-major, x0
    std::vector<double> mat;     // [ne][2] (lambda_e, mu_e), or empty
    std::vector<double> cv;      // [ne][36] Voigt matrices, or empty
    double lambda = 0.0, mu = 0.0;
};

LevelMesh mesh_of(const pa_op *op)
{
    LevelMesh m;
    m.nx = op->g.nx;
    m.ny = op->g.ny;
    m.nz = op->g.nz;
    m.affine = op->h_affine;
    m.mat = op->h_mat;
    m.cv = op->h_cv;
    m.lambda = op->lambda;
    m.mu = op->mu;
    return m;
}

// Undo one uniform refinement: coarse element (I, J, K) is the union of the
// fine elements (2I + a, 2J + b, 2K + c), a, b, c in {0, 1}.  Its map is
// x0 = x0 of child (0,0,0), J = 2 J of that child.  Fails unless every
// dimension is even, every child's map is the matching eighth of that map
// (to rounding) and the children share one material.
int coarsen_mesh(const LevelMesh &f, LevelMesh &c)
{
    if ((f.nx & 1) || (f.ny & 1) || (f.nz & 1))
        return set_error(PA_EINVAL, "solver: h-coarsening needs even element counts in x, y and z");
    c = LevelMesh();
    c.nx = f.nx / 2;
    c.ny = f.ny / 2;
    c.nz = f.nz / 2;
    c.lambda = f.lambda;
    c.mu = f.mu;
    const int64_t nec = (int64_t)c.nx * c.ny * c.nz;
    c.affine.assign((size_t)nec * 12, 0.0);
    if (!f.mat.empty()) c.mat.assign((size_t)nec * 2, 0.0);
    if (!f.cv.empty()) c.cv.assign((size_t)nec * 36, 0.0);
    auto fe = [&](int ix, int iy, int iz) { return (int64_t)ix + (int64_t)f.nx * (iy + (int64_t)f.ny * iz); };
    for (int K = 0; K < c.nz; ++K)
        for (int J = 0; J < c.ny; ++J)
            for (int I = 0; I < c.nx; ++I) {
                const int64_t E = (int64_t)I + (int64_t)c.nx * (J + (int64_t)c.ny * K);
                const double *a0 = f.affine.data() + 12 * fe(2 * I, 2 * J, 2 * K);
                double *A = c.affine.data() + 12 * E;
                double scale = 0.0;
                for (int k = 0; k < 9; ++k) {
                    A[k] = 2.0 * a0[k];
                    scale = std::max(scale, std::fabs(A[k]));
                }
                for (int k = 0; k < 3; ++k) A[9 + k] = a0[9 + k];
                const double tol = 1e-12 * scale;
                for (int cc = 0; cc < 2; ++cc)
                    for (int bb = 0; bb < 2; ++bb)
                        for (int aa = 0; aa < 2; ++aa) {
                            const int64_t e = fe(2 * I + aa, 2 * J + bb, 2 * K + cc);
                            const double *ae = f.affine.data() + 12 * e;
                            const double off[3] = {0.5 * aa, 0.5 * bb, 0.5 * cc};
                            bool ok = true;
                            for (int k = 0; k < 9; ++k) ok = ok && std::fabs(ae[k] - 0.5 * A[k]) <= tol;
                            for (int i = 0; i < 3; ++i) {
                                const double x0 = A[9 + i] + A[3 * i] * off[0] + A[3 * i + 1] * off[1] + A[3 * i + 2] * off[2];
                                ok = ok && std::fabs(ae[9 + i] - x0) <= tol + 1e-12 * std::fabs(x0);
                            }
                            if (!ok) return set_error(PA_EINVAL, "solver: mesh is not a uniform refinement (h-coarsening)");
                            if (!f.mat.empty()) {
                                if (f.mat[2 * e] != f.mat[2 * fe(2 * I, 2 * J, 2 * K)] ||
                                    f.mat[2 * e + 1] != f.mat[2 * fe(2 * I, 2 * J, 2 * K) + 1])
                                    return set_error(PA_EINVAL, "solver: material varies inside a coarse element");
                            }
                            if (!f.cv.empty()) {
                                for (int k = 0; k < 36; ++k)
                                    if (f.cv[36 * e + k] != f.cv[36 * fe(2 * I, 2 * J, 2 * K) + k])
                                        return set_error(PA_EINVAL, "solver: material varies inside a coarse element");
                            }
                        }
                if (!f.mat.empty()) {
                    c.mat[2 * E] = f.mat[2 * fe(2 * I, 2 * J, 2 * K)];
                    c.mat[2 * E + 1] = f.mat[2 * fe(2 * I, 2 * J, 2 * K) + 1];
                }
                if (!f.cv.empty())
                    std::copy(f.cv.begin() + 36 * fe(2 * I, 2 * J, 2 * K), f.cv.begin() + 36 * fe(2 * I, 2 * J, 2 * K) + 36,
                              c.cv.begin() + 36 * E);
            }
    return PA_OK;
}

int make_level_op(const LevelMesh &lm, int p, int precision, const std::vector<uint8_t> &mask, pa_op **out)
{
    pa_mesh m;
    m.nx = lm.nx;
    m.ny = lm.ny;
    m.nz = lm.nz;
    m.affine = lm.affine;
    int rc = pa_op_setup(&m, p, 0, lm.lambda, lm.mu, precision, mask.empty() ? nullptr : mask.data(), out);
    if (rc == PA_OK && !lm.mat.empty()) rc = pa_op_set_material(*out, lm.mat.data());
    if (rc == PA_OK && !lm.cv.empty()) rc = pa_op_set_anisotropic(*out, lm.cv.data());
    if (rc && *out) {
        pa_op_destroy(*out);
        *out = nullptr;
    }
    return rc;
}

// blocking read of one device scalar
double read_scalar(pa_solver *s, int slot, cudaStream_t st)
{
    cudaMemcpyAsync(s->h_scal + slot, s->dev.scal + slot, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return s->h_scal[slot];
}

// Chebyshev centre and half-width of the interval [cheb_lo, cheb_hi] * lam,
// and the coefficients of the smoothing steps (d = cd d + cr Dinv (r - A e),
// e += d):
//   kind 1: the first-kind Chebyshev iteration on [a, b] (three-term
//     recurrence of Saad, Iterative Methods for Sparse Linear Systems,
//     Sec. 12.3): cr_0 = 1/theta, then rho_k = 1 / (2 sigma - rho_(k-1)),
//     cd_k = rho_k rho_(k-1), cr_k = 2 rho_k / delta, sigma = theta / delta;
//   kind 4: the fourth-kind Chebyshev smoother on [0, b] (Lottes, Optimal
//     polynomial smoothers for multigrid V-cycles, 2023): cr_0 = 4 / (3 b),
//     cd_k = (2k - 1) / (2k + 3), cr_k = (8k + 4) / ((2k + 3) b); after m
//     steps the residual polynomial is W_m(1 - 2 lambda / b) / (2m + 1), W_m
//     the fourth-kind Chebyshev polynomial, which needs no lower bound.
void cheb_interval(const pa_solver *s, double lam, double *theta, double *delta, ChebCoef *c)
{
    const double a = s->cheb_lo * lam, b = s->cheb_hi * lam;
    *theta = 0.5 * (a + b);
    *delta = 0.5 * (b - a);
    *c = ChebCoef{};
    if (s->cheb_kind == 4) {
        for (int k = 0; k < s->cheb_order && k < kMaxCheb; ++k) {
            c->cd[k] = k == 0 ? 0.0 : (2.0 * k - 1.0) / (2.0 * k + 3.0);
            c->cr[k] = k == 0 ? 4.0 / (3.0 * b) : (8.0 * k + 4.0) / ((2.0 * k + 3.0) * b);
        }
        return;
    }
    const double sigma = *theta / *delta;
    double rho_prev = 1.0 / sigma;
    for (int k = 0; k < s->cheb_order && k < kMaxCheb; ++k) {
        if (k == 0) {
            c->cd[k] = 0.0;
            c->cr[k] = 1.0 / *theta;
        } else {
            const double rho = 1.0 / (2.0 * sigma - rho_prev);
            c->cd[k] = rho * rho_prev;
            c->cr[k] = 2.0 * rho / *delta;
            rho_prev = rho;
        }
    }
}

// power iteration for lambda_max(D^-1 A) of level l (FP64), power_its (10 by
// default, Sec. 3.1) steps from a fixed pseudo-random start
int estimate_lmax(pa_solver *s, Level &L, cudaStream_t st)
{
    const int64_t n = L.n;
    k_random<<<blocks_for(n), 256, 0, st>>>(L.e, L.op->d_ess, n, 0x1234567ull + (uint64_t)L.p);
    double lam = 0.0;
    for (int it = 0; it < s->power_its; ++it) {
        k_norm2<double><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, L.e, n, P_DEN);
        int rc = op_apply_async(L.op, L.e, L.t, false, st, nullptr);
        if (rc) return rc;
        // d = Dinv (A e)   (k_cheb with a zero guess, cd = 0, cr = 1)
        k_cheb<double><<<blocks_for(n), 256, 0, st>>>(L.d, L.r, L.t, nullptr, L.dinv, 0.0, 1.0, 1, n);
        k_norm2<double><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, L.d, n, P_NUM);
        PA_CUDA_TRY(cudaMemcpyAsync(s->h_scal + P_NUM, s->dev.scal + P_NUM, 2 * sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
        PA_CUDA_TRY(cudaStreamSynchronize(st));
        const double num = s->h_scal[P_NUM], den = s->h_scal[P_DEN];
        if (!(den > 0.0) || !(num > 0.0) || !std::isfinite(num))
            return set_error(PA_EBREAKDOWN, "solver: power iteration broke down");
        lam = std::sqrt(num / den);
        k_scale_copy<double, double><<<blocks_for(n), 256, 0, st>>>(L.e, L.d, 1.0 / std::sqrt(num), n);
    }
    PA_CUDA_TRY(cudaGetLastError());
    L.lmax = lam;
    cheb_interval(s, lam, &L.theta, &L.delta, &L.cheb);
    return PA_OK;
}


// ------------------------------------------------------- h-hierarchy setup
int h_power_lmax(pa_solver *s, HLevel &H, cudaStream_t st)
{
    const int64_t n = H.n;
    k_random<<<blocks_for(n), 256, 0, st>>>(H.e, H.ess, n, 0x5151ull + (uint64_t)n);
    double lam = 0.0;
    for (int it = 0; it < s->power_its; ++it) {
        k_norm2<double><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, H.e, n, P_DEN);
        k_stencil_apply<<<row3_blocks(n), 128, 0, st>>>(H.vals, H.e, H.t, H.g);
        k_cheb<double><<<blocks_for(n), 256, 0, st>>>(H.d, H.r, H.t, nullptr, H.dinv, 0.0, 1.0, 1, n);
        k_norm2<double><<<red_blocks(n), kRedThreads, 0, st>>>(s->dev, H.d, n, P_NUM);
        PA_CUDA_TRY(cudaMemcpyAsync(s->h_scal + P_NUM, s->dev.scal + P_NUM, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        PA_CUDA_TRY(cudaStreamSynchronize(st));
        const double num = s->h_scal[P_NUM], den = s->h_scal[P_DEN];
        if (!(den > 0.0) || !(num > 0.0) || !std::isfinite(num)) return set_error(PA_EBREAKDOWN, "solver: h-level power iteration");
        lam = std::sqrt(num / den);
        k_scale_copy<double, double><<<blocks_for(n), 256, 0, st>>>(H.e, H.d, 1.0 / std::sqrt(num), n);
    }
    H.lmax = lam;
    cheb_interval(s, lam, &H.theta, &H.delta, &H.cheb);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

// Cholesky inverse of a small SPD matrix (host, in place on a copy).
bool spd_inverse(std::vector<double> &A, int n)
{
    std::vector<double> L((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(d > 0.0)) return false;
        const double ljj = std::sqrt(d);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double v = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = v / ljj;
        }
    }
    // inverse columns by forward/back substitution
    std::vector<double> col(n);
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= L[(size_t)i * n + k] * col[k];
            col[i] = v / L[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double v = col[i];
            for (int k = i + 1; k < n; ++k) v -= L[(size_t)k * n + i] * col[k];
            col[i] = v / L[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i) A[(size_t)i * n + c] = col[i];
    }
    return true;
}

// h-coarse essential mask: coarse dof j is essential when its interpolation
// reaches an essential fine dof (the 0/1 fine mask restricted); exact for
// essential sets made of whole faces.
std::vector<uint8_t> h_coarse_mask(const std::vector<uint8_t> &fm, const Grid &gf, const Grid &gc)
{
    std::vector<uint8_t> cm((size_t)3 * gc.Nn, 0);
    const int Mf[3] = {gf.Mx, gf.My, gf.Mz}, Mc[3] = {gc.Mx, gc.My, gc.Mz};
    for (int comp = 0; comp < 3; ++comp)
        for (int64_t i = 0; i < gf.Nn; ++i) {
            if (!fm[(size_t)(comp * gf.Nn + i)]) continue;
            const int f[3] = {(int)(i % gf.Mx), (int)((i / gf.Mx) % gf.My), (int)(i / ((int64_t)gf.Mx * gf.My))};
            int J[3][2], nJ[3];
            double w[3][2];
            for (int a = 0; a < 3; ++a) nJ[a] = h_parents(f[a], Mf[a], Mc[a], J[a], w[a]);
            for (int kz = 0; kz < nJ[2]; ++kz)
                for (int ky = 0; ky < nJ[1]; ++ky)
                    for (int kx = 0; kx < nJ[0]; ++kx)
                        cm[(size_t)(comp * gc.Nn + J[0][kx] + (int64_t)gc.Mx * (J[1][ky] + (int64_t)gc.My * J[2][kz]))] = 1;
        }
    return cm;
}

// Builds the h-hierarchy under the p = 1 level: Galerkin stencils, masks,
// diagonals, Chebyshev intervals, and a dense inverse on the coarsest level.
int build_h_levels(pa_solver *s, cudaStream_t st)
{
    Level &L = s->lv.back();
    if (!L.stencil) return PA_OK;
    const int64_t kMaxDense = 320;
    HLevel H0;
    H0.g = L.op->g;
    H0.n = L.n;
    H0.vals = L.stencil;
    H0.ess = L.op->d_ess;
    H0.dinv = L.dinv;
    s->hl.push_back(H0);
    while (true) {
        HLevel &F = s->hl.back();
        if (F.n <= kMaxDense) break;
        Grid c = F.g;
        c.Mx = h_coarse_size(F.g.Mx);
        c.My = h_coarse_size(F.g.My);
        c.Mz = h_coarse_size(F.g.Mz);
        if (c.Mx == F.g.Mx && c.My == F.g.My && c.Mz == F.g.Mz) break;
        c.nx = c.Mx - 1;
        c.ny = c.My - 1;
        c.nz = c.Mz - 1;
        c.p = 1;
        c.ne = (int64_t)c.nx * c.ny * c.nz;
        c.Nn = (int64_t)c.Mx * c.My * c.Mz;
        HLevel C;
        C.g = c;
        C.n = 3 * c.Nn;
        int rc;
        if ((rc = dalloc(s, &C.vals, 81 * C.n))) return rc;
        k_rap_stencil<<<blocks_for(C.n, 64), 64, 0, st>>>(F.vals, F.ess, F.g, C.vals, c);
        PA_CUDA_TRY(cudaGetLastError());
        if (F.ess) {
            // coarse essential dofs: those whose interpolation reaches an
            // essential fine dof (restrict the fine mask as a 0/1 field)
            std::vector<uint8_t> fm((size_t)F.n);
            PA_CUDA_TRY(cudaMemcpyAsync(fm.data(), F.ess, F.n, cudaMemcpyDeviceToHost, st));
            PA_CUDA_TRY(cudaStreamSynchronize(st));
            std::vector<uint8_t> cm = h_coarse_mask(fm, F.g, c);
            if ((rc = dalloc(s, &C.ess, C.n))) return rc;
            PA_CUDA_TRY(cudaMemcpyAsync(C.ess, cm.data(), C.n, cudaMemcpyHostToDevice, st));
            PA_CUDA_TRY(cudaStreamSynchronize(st));
        }
        if ((rc = dalloc(s, &C.dinv, C.n))) return rc;
        k_mask_stencil<<<blocks_for(C.n, 128), 128, 0, st>>>(C.vals, C.ess, c);
        PA_CUDA_TRY(cudaGetLastError());
        s->hl.push_back(C);
    }
    // work vectors, diagonals, Chebyshev intervals, coarsest inverse
    for (size_t k = 0; k < s->hl.size(); ++k) {
        HLevel &H = s->hl[k];
        int rc;
        // level 0 reads its right-hand side from the coarse CG residual in place
        if (k == 0) H.r = L.cr;
        else if ((rc = dalloc(s, &H.r, H.n))) return rc;
        if ((rc = dalloc(s, &H.e, H.n)) || (rc = dalloc(s, &H.e2, H.n)) || (rc = dalloc(s, &H.t, H.n)) ||
            (rc = dalloc(s, &H.d, H.n)) || (rc = dalloc(s, &H.xa, H.n)) || (rc = dalloc(s, &H.xb, H.n)))
            return rc;
        if (k > 0) {
            // diagonal = stencil centre entry (s = 13) of the own component; 1 on essential rows
            std::vector<double> cen((size_t)H.n);
            std::vector<uint8_t> em;
            for (int comp = 0; comp < 3; ++comp)
                PA_CUDA_TRY(cudaMemcpyAsync(cen.data() + comp * H.g.Nn, H.vals + (int64_t)(13 * 3 + comp) * H.n + comp * H.g.Nn,
                                            sizeof(double) * H.g.Nn, cudaMemcpyDeviceToHost, st));
            if (H.ess) {
                em.resize((size_t)H.n);
                PA_CUDA_TRY(cudaMemcpyAsync(em.data(), H.ess, H.n, cudaMemcpyDeviceToHost, st));
            }
            PA_CUDA_TRY(cudaStreamSynchronize(st));
            for (int64_t i = 0; i < H.n; ++i) cen[(size_t)i] = (H.ess && em[(size_t)i]) ? 1.0 : 1.0 / cen[(size_t)i];
            PA_CUDA_TRY(cudaMemcpyAsync(H.dinv, cen.data(), sizeof(double) * H.n, cudaMemcpyHostToDevice, st));
            PA_CUDA_TRY(cudaStreamSynchronize(st));
        }
        if (k + 1 < s->hl.size()) {
            if ((rc = h_power_lmax(s, H, st))) return rc;
        }
    }
    // dense inverse of the coarsest level (constrained: identity on essential dofs)
    HLevel &Hc = s->hl.back();
    if (Hc.n > 4 * kMaxDense) return set_error(PA_EINVAL, "solver: h-hierarchy coarsest level too large for a dense solve");
    const int n = (int)Hc.n;
    std::vector<double> V((size_t)81 * n);
    std::vector<uint8_t> em((size_t)n, 0);
    PA_CUDA_TRY(cudaMemcpyAsync(V.data(), Hc.vals, sizeof(double) * V.size(), cudaMemcpyDeviceToHost, st));
    if (Hc.ess) PA_CUDA_TRY(cudaMemcpyAsync(em.data(), Hc.ess, n, cudaMemcpyDeviceToHost, st));
    PA_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> A((size_t)n * n, 0.0);
    const Grid &g = Hc.g;
    for (int row = 0; row < n; ++row) {
        if (em[row]) {
            A[(size_t)row * n + row] = 1.0;
            continue;
        }
        const int c = (int)(row / g.Nn);
        const int64_t i = row - c * g.Nn;
        const int ix = (int)(i % g.Mx), iy = (int)((i / g.Mx) % g.My), iz = (int)(i / ((int64_t)g.Mx * g.My));
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (ix + dx < 0 || ix + dx >= g.Mx || iy + dy < 0 || iy + dy >= g.My || iz + dz < 0 || iz + dz >= g.Mz)
                        continue;
                    const int sidx = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                    const int64_t j = i + dx + (int64_t)g.Mx * (dy + (int64_t)g.My * dz);
                    for (int d = 0; d < 3; ++d) {
                        const int64_t col = d * g.Nn + j;
                        if (em[col]) continue;
                        A[(size_t)row * n + col] += V[(size_t)(sidx * 3 + d) * n + row];
                    }
                }
    }
    // symmetrise the rounding, then invert
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const double m = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
            A[(size_t)i * n + j] = A[(size_t)j * n + i] = m;
        }
    if (!spd_inverse(A, n)) return set_error(PA_EBREAKDOWN, "solver: coarsest h-level matrix is not SPD");
    int rc = dalloc(s, &Hc.Ainv, (int64_t)n * n);
    if (rc) return rc;
    PA_CUDA_TRY(cudaMemcpyAsync(Hc.Ainv, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice, st));
    PA_CUDA_TRY(cudaStreamSynchronize(st));
    return PA_OK;
}

}  // namespace pa

using namespace pa;

extern "C" {

int pa_solver_destroy(pa_solver *s)
{
    if (!s) return PA_OK;
    for (auto &L : s->lv) {
        if (L.own_op) pa_op_destroy(L.op);
        pa_op_destroy(L.op32);
    }
    for (StepGraphs *g : {&s->g64, &s->g32, &s->gmx}) {
        if (g->init) cudaGraphExecDestroy(g->init);
        if (g->iter) cudaGraphExecDestroy(g->iter);
    }
    if (s->stream) cudaStreamDestroy(s->stream);
    for (void *p : s->allocs) cudaFree(p);
    cudaFree(s->dev.scal);
    cudaFree(s->dev.flag);
    cudaFree(s->dev.partial);
    cudaFree(s->dev.counter);
    cudaFreeHost(s->h_scal);
    cudaFreeHost(s->h_flag);
    delete s;
    return PA_OK;
}

int pa_solver_create(pa_op *fine, int nlev, const int *p_levels, int cheb_order, double coarse_rtol, int coarse_maxit,
                     int mode, pa_solver **out)
{
    return pa_solver_create_hp(fine, nlev, p_levels, 0, cheb_order, coarse_rtol, coarse_maxit, mode, out);
}

int pa_solver_create_hp(pa_op *fine, int nlev, const int *p_levels, int h_levels, int cheb_order, double coarse_rtol,
                        int coarse_maxit, int mode, pa_solver **out)
{
    NvtxRange nvtx("pa_solver_create");
    if (!out) return set_error(PA_EINVAL, "pa_solver_create: null output");
    *out = nullptr;
    if (!fine || !p_levels || nlev < 1 || nlev > 8) return set_error(PA_EINVAL, "pa_solver_create: bad levels");
    if (h_levels < 0 || nlev + h_levels > 8) return set_error(PA_EINVAL, "pa_solver_create: at most 8 levels in all");
    if (h_levels > 0 && p_levels[nlev - 1] != 1)
        return set_error(PA_EINVAL, "pa_solver_create: h-levels need the last degree to be 1");
    if (fine->precision != PA_FP64) return set_error(PA_EINVAL, "pa_solver_create: fine operator must be FP64");
    if (p_levels[0] != fine->p) return set_error(PA_EINVAL, "pa_solver_create: p_levels[0] must be the fine degree");
    for (int l = 1; l < nlev; ++l)
        if (p_levels[l] >= p_levels[l - 1] || p_levels[l] < 1)
            return set_error(PA_EINVAL, "pa_solver_create: degrees must decrease");
    if (cheb_order < 1 || cheb_order > 8) return set_error(PA_EINVAL, "pa_solver_create: cheb_order in 1..8");
    if (coarse_maxit < 1 || !(coarse_rtol >= 0.0)) return set_error(PA_EINVAL, "pa_solver_create: bad coarse parameters");
    if (mode != PA_SOLVE_FP64 && mode != PA_SOLVE_MIXED && mode != PA_SOLVE_MIXED_FCG)
        return set_error(PA_EINVAL, "pa_solver_create: bad mode");
    const bool fp32_levels = mode != PA_SOLVE_FP64;

    pa_solver *s = new (std::nothrow) pa_solver;
    if (!s) return set_error(PA_ENOMEM, "pa_solver_create: host allocation");
    s->mode = mode;
    s->cheb_order = cheb_order;
    s->coarse_rtol = coarse_rtol;
    s->coarse_maxit = coarse_maxit;
    int rc = PA_OK;
#define TRY(x)                        \
    do {                              \
        rc = (x);                     \
        if (rc) {                     \
            pa_solver_destroy(s);     \
            return rc;                \
        }                             \
    } while (0)
#define TRYC(x) TRY(((x) == cudaSuccess) ? PA_OK : cuda_error(cudaGetLastError(), #x))
    TRYC(cudaMalloc((void **)&s->dev.scal, sizeof(double) * NSLOT));
    TRYC(cudaMalloc((void **)&s->dev.flag, sizeof(int) * NFLAG));
    TRYC(cudaMalloc((void **)&s->dev.partial, sizeof(double) * 3 * kRedBlocks));
    TRYC(cudaMalloc((void **)&s->dev.counter, sizeof(unsigned)));
    TRYC(cudaMemset(s->dev.counter, 0, sizeof(unsigned)));
    TRYC(cudaMemset(s->dev.flag, 0, sizeof(int) * NFLAG));
    TRYC(cudaMemset(s->dev.scal, 0, sizeof(double) * NSLOT));
    TRYC(cudaMallocHost((void **)&s->h_scal, sizeof(double) * NSLOT));
    TRYC(cudaMallocHost((void **)&s->h_flag, sizeof(int) * NFLAG));
    TRYC(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    TRY(dalloc(s, &s->bar, 2));
    TRY(dalloc(s, &s->coop_part, 9 * (int64_t)kRedBlocks));
    {
        int dev = 0, coop = 0, nsm = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_coop, 256, 0) == cudaSuccess)
            s->coop_blocks = std::min(kCoopBlocks, per_sm * nsm);
        int khz = 0;
        if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) == cudaSuccess && khz > 0) s->clock_khz = khz;
        s->wait_cycles = (long long)(2.0 * s->clock_khz * 1e3);
        cudaGetLastError();
    }

    const int ntot = nlev + h_levels;
    s->lv.resize(ntot);
    std::vector<uint8_t> mask = fine->h_ess;
    LevelMesh cur = mesh_of(fine);  // mesh of the level being built
    for (int l = 0; l < ntot; ++l) {
        Level &L = s->lv[l];
        L.p = l < nlev ? p_levels[l] : 1;
        if (l == 0) {
            L.op = fine;
        } else if (l < nlev) {
            // p-coarsening: same mesh, lower degree
            const pa_op *F = s->lv[l - 1].op;
            if (!mask.empty()) {
                Basis1D bc;
                bc.build(L.p, L.p + 2);
                mask = coarse_mask(mask, F->g, L.p, bc, F->basis);
            }
            TRY(make_level_op(cur, L.p, PA_FP64, mask, &L.op));
            L.own_op = true;
        } else {
            // h-coarsening: p = 1 on the mesh whose uniform refinement is the level above
            const pa_op *F = s->lv[l - 1].op;
            LevelMesh c;
            TRY(coarsen_mesh(cur, c));
            if (!mask.empty()) {
                Grid gc{};
                gc.nx = c.nx;
                gc.ny = c.ny;
                gc.nz = c.nz;
                gc.p = 1;
                gc.Mx = c.nx + 1;
                gc.My = c.ny + 1;
                gc.Mz = c.nz + 1;
                gc.ne = (int64_t)c.nx * c.ny * c.nz;
                gc.Nn = (int64_t)gc.Mx * gc.My * gc.Mz;
                mask = h_coarse_mask(mask, F->g, gc);
            }
            cur = std::move(c);
            TRY(make_level_op(cur, 1, PA_FP64, mask, &L.op));
            L.own_op = true;
            s->lv[l - 1].hdown = true;
        }
        L.n = L.op->ndofs();
        if (fp32_levels) TRY(make_level_op(cur, L.p, PA_FP32, L.op->h_ess, &L.op32));
    }
    const int nlev_all = ntot;
    cudaStream_t st = s->stream;
    for (int l = 0; l < nlev_all; ++l) {
        Level &L = s->lv[l];
        const int64_t n = L.n;
        TRY(dalloc(s, &L.dinv, n));
        TRY(dalloc(s, &L.r, n));
        TRY(dalloc(s, &L.e, n));
        TRY(dalloc(s, &L.t, n));
        TRY(dalloc(s, &L.d, n));
        TRY(pa_op_diag(L.op, L.t, st));
        k_recip<double><<<blocks_for(n), 256, 0, st>>>(L.dinv, L.t, n);
        if (l < nlev_all - 1) {
            TRY(dalloc(s, &L.xa, n));
            TRY(dalloc(s, &L.xb, n));
            if (!L.hdown) {
                const int pc = p_levels[l + 1];
                Basis1D bc;
                bc.build(pc, pc + 2);
                std::vector<double> val((size_t)(pc + 1) * (L.p + 1)), der(val.size());
                lagrange_product(pc + 1, bc.nodes.data(), L.p + 1, L.op->basis.nodes.data(), val.data(), der.data());
                for (size_t i = 0; i < val.size(); ++i) L.xt.L[i] = std::fabs(val[i]) < 1e-15 ? 0.0 : val[i];
            }
            TRY(estimate_lmax(s, L, st));
        } else {
            TRY(dalloc(s, &L.cx, n));
            TRY(dalloc(s, &L.cr, n));
            TRY(dalloc(s, &L.cp, n));
            TRY(dalloc(s, &L.cq, n));
            if (L.p == 1 && L.op->g.Nn < (1LL << 30) && L.op->h_cv.empty()) {
                // assemble the coarse matrix (same quadrature as the operator);
                // its kernels index nodes in 32 bits
                TRY(dalloc(s, &L.stencil, 81 * n));
                TRY(pa_op_assemble_p1(L.op, L.stencil, st));
                k_mask_stencil<<<blocks_for(n, 128), 128, 0, st>>>(L.stencil, L.op->d_ess, L.op->g);
            }
        }
        if (fp32_levels) {
            TRY(dalloc(s, &L.r32, n));
            TRY(dalloc(s, &L.e32, n));
            TRY(dalloc(s, &L.dinv32, n));
            TRY(dalloc(s, &L.t32, n));
            TRY(dalloc(s, &L.d32, n));
            TRY(dalloc(s, &L.xa32, n));
            TRY(dalloc(s, &L.xb32, n));
            k_scale_copy<double, float><<<blocks_for(n), 256, 0, st>>>(L.dinv32, L.dinv, 1.0, n);
            // one eager apply per FP32 operator before any graph capture
            TRY(op_apply_async(L.op32, L.dinv32, L.t32, false, st, nullptr));
        }
    }
    if (s->lv.back().stencil) TRY(build_h_levels(s, st));
    const int64_t n0 = s->lv[0].n;
    TRY(dalloc(s, &s->xin, n0));
    TRY(dalloc(s, &s->bin, n0));
    TRY(dalloc(s, &s->r, n0));
    TRY(dalloc(s, &s->z, n0));
    TRY(dalloc(s, &s->p, n0));
    TRY(dalloc(s, &s->q, n0));
    TRY(dalloc(s, &s->t, n0));
    if (mode == PA_SOLVE_MIXED) {
        TRY(dalloc(s, &s->r32, n0));
        TRY(dalloc(s, &s->z32, n0));
        TRY(dalloc(s, &s->p32, n0));
        TRY(dalloc(s, &s->q32, n0));
        TRY(dalloc(s, &s->x32, n0));
        TRY(dalloc(s, &s->b32, n0));
    }
    TRYC(cudaStreamSynchronize(st));
    TRYC(cudaGetLastError());
#undef TRY
#undef TRYC
    *out = s;
    clear_error();
    return PA_OK;
}

int pa_solver_set_option(pa_solver *s, int option, double value)
{
    if (!s) return set_error(PA_EINVAL, "pa_solver_set_option: null solver");
    switch (option) {
    case PA_SOLVER_OPT_GRAPHS:
    case PA_SOLVER_OPT_PERSISTENT_COARSE:
    case PA_SOLVER_OPT_COARSE_HMG: {
        // both change what the step graphs contain: drop any built graphs
        for (StepGraphs *g : {&s->g64, &s->g32, &s->gmx}) {
            if (g->init) cudaGraphExecDestroy(g->init);
            if (g->iter) cudaGraphExecDestroy(g->iter);
            g->init = g->iter = nullptr;
        }
        if (option == PA_SOLVER_OPT_GRAPHS) s->use_graphs = value != 0.0;
        else if (option == PA_SOLVER_OPT_PERSISTENT_COARSE) s->allow_coop = value != 0.0;
        else s->use_hmg = value != 0.0;
        return PA_OK;
    }
    case PA_SOLVER_OPT_CHEB_LOWER:
    case PA_SOLVER_OPT_CHEB_UPPER:
    case PA_SOLVER_OPT_CHEB_KIND:
    case PA_SOLVER_OPT_POWER_ITERS: {
        if (option == PA_SOLVER_OPT_CHEB_KIND) {
            if (value != 1.0 && value != 4.0) return set_error(PA_EINVAL, "pa_solver_set_option: Chebyshev kind 1 or 4");
        } else if (option == PA_SOLVER_OPT_POWER_ITERS) {
            if (!(value >= 1.0 && value <= 1000.0)) return set_error(PA_EINVAL, "pa_solver_set_option: power iterations in 1..1000");
        } else {
            const double lo = option == PA_SOLVER_OPT_CHEB_LOWER ? value : s->cheb_lo;
            const double hi = option == PA_SOLVER_OPT_CHEB_UPPER ? value : s->cheb_hi;
            if (!(lo > 0.0) || !(hi > lo) || !(hi < 100.0))
                return set_error(PA_EINVAL, "pa_solver_set_option: need 0 < lower < upper < 100 (fractions of lambda_max)");
        }
        // the step graphs hold the Chebyshev coefficients as kernel arguments
        for (StepGraphs *g : {&s->g64, &s->g32, &s->gmx}) {
            if (g->init) cudaGraphExecDestroy(g->init);
            if (g->iter) cudaGraphExecDestroy(g->iter);
            g->init = g->iter = nullptr;
        }
        if (option == PA_SOLVER_OPT_CHEB_LOWER) s->cheb_lo = value;
        else if (option == PA_SOLVER_OPT_CHEB_UPPER) s->cheb_hi = value;
        else if (option == PA_SOLVER_OPT_CHEB_KIND) s->cheb_kind = (int)value;
        else s->power_its = (int)value;
        cudaStream_t st = s->stream;
        // smoothed levels are the ones with an estimate (the assembled p = 1
        // level is solved, not smoothed; the last h-level is a dense solve)
        for (Level &L : s->lv) {
            if (!(L.lmax > 0.0)) continue;
            if (option == PA_SOLVER_OPT_POWER_ITERS) {
                if (int rc = estimate_lmax(s, L, st)) return rc;
            } else {
                cheb_interval(s, L.lmax, &L.theta, &L.delta, &L.cheb);
            }
        }
        for (HLevel &H : s->hl) {
            if (!(H.lmax > 0.0)) continue;
            if (option == PA_SOLVER_OPT_POWER_ITERS) {
                if (int rc = h_power_lmax(s, H, st)) return rc;
            } else {
                cheb_interval(s, H.lmax, &H.theta, &H.delta, &H.cheb);
            }
        }
        PA_CUDA_TRY(cudaStreamSynchronize(st));
        return PA_OK;
    }
    case PA_SOLVER_OPT_WAIT_LIMIT: {
        if (!(value > 0.0 && value <= 60.0)) return set_error(PA_EINVAL, "pa_solver_set_option: wait limit in (0, 60] s");
        // the limit is a kernel argument of the captured step graphs
        for (StepGraphs *g : {&s->g64, &s->g32, &s->gmx}) {
            if (g->init) cudaGraphExecDestroy(g->init);
            if (g->iter) cudaGraphExecDestroy(g->iter);
            g->init = g->iter = nullptr;
        }
        s->wait_cycles = std::max(1LL, (long long)(value * s->clock_khz * 1e3));
        return PA_OK;
    }
    case PA_SOLVER_OPT_INJECT_INNER_FAILURE:
        if (!(value >= 0.0 && value <= 1e6)) return set_error(PA_EINVAL, "pa_solver_set_option: inner-failure index >= 0");
        s->inject_inner_failure = (int)value;
        return PA_OK;
    default: return set_error(PA_EINVAL, "pa_solver_set_option: unknown option");
    }
}

}  // extern "C"
