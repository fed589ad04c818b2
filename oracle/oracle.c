/*
 * Plain FP64 CPU oracle for the high-order linear-elasticity operator of
 * "Shifting the Sweet Spot: High-Performance Matrix-Free Method for
 * High-Order Elasticity" (arXiv 2601.08374).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * (CUDA) path never calls it, and the two share no code, tables or headers.
 *
 * What it computes is the plain definition of the discrete operator, not
 * the paper's fast algorithm:
 *   a(u,v) = integral of sigma(u) : grad(v)                    (Sec. 2.1, Eq. 4)
 *   sigma  = lambda (div u) I + 2 mu eps(u),  eps = sym grad u (Eq. 3)
 *   A      = assembled Galerkin matrix of a(.,.) on the H1 space spanned by
 *            tensor-product GLL Lagrange polynomials of degree p (Eq. 5, 6),
 *            integrated with q Gauss-Legendre points per direction
 *            (Sec. 5.1.4: q = p + 2 by default).
 * The element matrix is formed from dense reference blocks
 *   S_mn[a][b] = sum_alpha w_alpha d_m Phi_a(alpha) d_n Phi_b(alpha)
 * built by a brute-force sum over all quadrature points with full 3D basis
 * tables (no sum factorisation), and from the element's constant inverse
 * Jacobian (affine elements, Sec. 4.4).
 *
 * Conventions (shared with the product only through the documented ABI,
 * never through code):
 *   reference cell [0,1]^3; element e = ex + nx*(ey + ny*ez);
 *   affine map x = x0 + J xi, per element 12 doubles: J row-major, then x0;
 *   local node a = ix + D*(iy + D*iz), D = p + 1;
 *   global node g = gx + Mx*(gy + My*gz), Mx = nx*p + 1, ...;
 *   L-vector component-major: value (c, g) at index c*Nn + g;
 *   element-local dof (c, a) at index c*D^3 + a.
 * Dirichlet handling (the constrained operator): z = x with essential
 * entries zeroed, y = A z, then y = x on essential entries.
 *
 * 1D rules use long double in the Newton iterations.  Large sums use double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long double ld;

/* ------------------------------------------------------------------------ */
/* Legendre polynomials by the three-term recurrence (textbook).             */
/* ------------------------------------------------------------------------ */
static void legendre(int n, ld t, ld *Pn, ld *Pnm1)
{
    ld p0 = 1.0L, p1 = t;
    if (n == 0) { *Pn = 1.0L; *Pnm1 = 0.0L; return; }
    for (int k = 1; k < n; ++k) {
        ld p2 = ((2.0L * k + 1.0L) * t * p1 - (ld)k * p0) / (ld)(k + 1);
        p0 = p1;
        p1 = p2;
    }
    *Pn = p1;
    *Pnm1 = p0;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Gauss-Legendre points and weights on [0,1], q >= 1.  Newton iteration on
 * P_q started from the usual cosine guesses.                                */
int orc_gauss01(int q, double *pts, double *wts)
{
    if (q < 1 || q > 64) return -1;
    double tmp[2 * 64];
    for (int k = 0; k < q; ++k) {
        ld t = cosl(3.14159265358979323846264338327950288L * (k + 0.75L) / (q + 0.5L));
        ld dP = 0.0L;
        for (int it = 0; it < 100; ++it) {
            ld Pn, Pm;
            legendre(q, t, &Pn, &Pm);
            dP = (ld)q * (t * Pn - Pm) / (t * t - 1.0L);
            ld dt = Pn / dP;
            t -= dt;
            if (fabsl(dt) < 1e-30L) break;
        }
        {
            ld Pn, Pm;
            legendre(q, t, &Pn, &Pm);
            dP = (ld)q * (t * Pn - Pm) / (t * t - 1.0L);
        }
        ld w = 2.0L / ((1.0L - t * t) * dP * dP);
        tmp[2 * k] = (double)((1.0L + t) / 2.0L);
        tmp[2 * k + 1] = (double)(w / 2.0L);
    }
    /* sort by point (pairs) */
    for (int i = 1; i < q; ++i)
        for (int j = i; j > 0 && tmp[2 * (j - 1)] > tmp[2 * j]; --j) {
            double a0 = tmp[2 * j], a1 = tmp[2 * j + 1];
            tmp[2 * j] = tmp[2 * (j - 1)];
            tmp[2 * j + 1] = tmp[2 * (j - 1) + 1];
            tmp[2 * (j - 1)] = a0;
            tmp[2 * (j - 1) + 1] = a1;
        }
    for (int k = 0; k < q; ++k) { pts[k] = tmp[2 * k]; wts[k] = tmp[2 * k + 1]; }
    return 0;
}

/* Gauss-Lobatto-Legendre nodes on [0,1]: the end points and the p-1 roots
 * of P'_p, found by Newton with P''_p from the Legendre equation.           */
int orc_gll01(int p, double *nodes)
{
    if (p < 1 || p > 63) return -1;
    nodes[0] = 0.0;
    nodes[p] = 1.0;
    double inner[64];
    for (int k = 1; k < p; ++k) {
        ld t = cosl(3.14159265358979323846264338327950288L * (ld)k / (ld)p);
        for (int it = 0; it < 100; ++it) {
            ld Pn, Pm;
            legendre(p, t, &Pn, &Pm);
            ld d1 = (ld)p * (t * Pn - Pm) / (t * t - 1.0L);
            ld d2 = (2.0L * t * d1 - (ld)p * (p + 1) * Pn) / (1.0L - t * t);
            ld dt = d1 / d2;
            t -= dt;
            if (fabsl(dt) < 1e-30L) break;
        }
        inner[k - 1] = (double)((1.0L + t) / 2.0L);
    }
    qsort(inner, (size_t)(p - 1), sizeof(double), cmp_double);
    for (int k = 1; k < p; ++k) nodes[k] = inner[k - 1];
    return 0;
}

/* Lagrange basis on n nodes, values and first derivatives at m points, by
 * the barycentric formula (Berrut & Trefethen 2004).  val[i*m + j] is
 * l_i(x_j), der[i*m + j] is l_i'(x_j).  Points that coincide with a node
 * use the differentiation-matrix form.                                      */
int orc_lagrange(int n, const double *nodes, int m, const double *x, double *val, double *der)
{
    if (n < 1 || n > 64) return -1;
    ld bw[64];
    for (int i = 0; i < n; ++i) {
        ld prod = 1.0L;
        for (int j = 0; j < n; ++j)
            if (j != i) prod *= ((ld)nodes[i] - (ld)nodes[j]);
        bw[i] = 1.0L / prod;
    }
    for (int j = 0; j < m; ++j) {
        ld xj = x[j];
        int hit = -1;
        for (int i = 0; i < n; ++i)
            if ((ld)nodes[i] == xj) hit = i;
        if (hit >= 0) {
            ld sum_off = 0.0L;
            for (int i = 0; i < n; ++i) {
                val[i * m + j] = (i == hit) ? 1.0 : 0.0;
                if (i != hit) {
                    ld d = (bw[i] / bw[hit]) / (xj - (ld)nodes[i]);
                    der[i * m + j] = (double)d;
                    sum_off += d;
                }
            }
            der[hit * m + j] = (double)(-sum_off);
            continue;
        }
        ld denom = 0.0L;
        for (int i = 0; i < n; ++i) denom += bw[i] / (xj - (ld)nodes[i]);
        for (int i = 0; i < n; ++i) {
            ld li = (bw[i] / (xj - (ld)nodes[i])) / denom;
            ld s = 0.0L;
            for (int k = 0; k < n; ++k)
                if (k != i) s += 1.0L / (xj - (ld)nodes[k]);
            val[i * m + j] = (double)li;
            der[i * m + j] = (double)(li * s);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Reference data for one (p, q).                                            */
/* ------------------------------------------------------------------------ */
typedef struct orc_ref {
    int p, q, D, Q, D3, Q3;
    double gll[64], gp[64], gw[64];
    double *B;   /* [D][Q] l_i(xi_q)   */
    double *G;   /* [D][Q] l_i'(xi_q)  */
    double *S;   /* [9][D3][D3], block (m,n) at (3m+n)*D3*D3 */
} orc_ref;

void orc_ref_destroy(orc_ref *r)
{
    if (!r) return;
    free(r->B);
    free(r->G);
    free(r->S);
    free(r);
}

orc_ref *orc_ref_create(int p, int q)
{
    if (p < 1 || p > 16) return NULL;
    if (q <= 0) q = p + 2;
    if (q > 32) return NULL;
    orc_ref *r = (orc_ref *)calloc(1, sizeof(orc_ref));
    if (!r) return NULL;
    r->p = p; r->q = q; r->D = p + 1; r->Q = q;
    r->D3 = r->D * r->D * r->D;
    r->Q3 = q * q * q;
    int D = r->D, Q = r->Q, D3 = r->D3, Q3 = r->Q3;
    orc_gll01(p, r->gll);
    orc_gauss01(q, r->gp, r->gw);
    r->B = (double *)malloc(sizeof(double) * D * Q);
    r->G = (double *)malloc(sizeof(double) * D * Q);
    r->S = (double *)calloc((size_t)9 * D3 * D3, sizeof(double));
    double *dphi = (double *)malloc(sizeof(double) * 3 * (size_t)Q3 * D3);
    double *w3 = (double *)malloc(sizeof(double) * Q3);
    if (!r->B || !r->G || !r->S || !dphi || !w3) {
        free(dphi); free(w3); orc_ref_destroy(r); return NULL;
    }
    orc_lagrange(D, r->gll, Q, r->gp, r->B, r->G);
    /* Full 3D tables of reference gradients (Eq. 6):
     * dphi[m][alpha][a] = d/dxi_m (l_ix l_iy l_iz) at alpha.               */
    for (int qz = 0; qz < Q; ++qz)
        for (int qy = 0; qy < Q; ++qy)
            for (int qx = 0; qx < Q; ++qx) {
                int al = qx + Q * (qy + Q * qz);
                w3[al] = r->gw[qx] * r->gw[qy] * r->gw[qz];
                for (int iz = 0; iz < D; ++iz)
                    for (int iy = 0; iy < D; ++iy)
                        for (int ix = 0; ix < D; ++ix) {
                            int a = ix + D * (iy + D * iz);
                            double bx = r->B[ix * Q + qx], by = r->B[iy * Q + qy], bz = r->B[iz * Q + qz];
                            double gx = r->G[ix * Q + qx], gy = r->G[iy * Q + qy], gz = r->G[iz * Q + qz];
                            dphi[(0 * (size_t)Q3 + al) * D3 + a] = gx * by * bz;
                            dphi[(1 * (size_t)Q3 + al) * D3 + a] = bx * gy * bz;
                            dphi[(2 * (size_t)Q3 + al) * D3 + a] = bx * by * gz;
                        }
            }
    /* S_mn[a][b] = sum over all Q^3 points of w * dphi_m[a] * dphi_n[b]. */
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int mn = 0; mn < 9; ++mn)
        for (int a = 0; a < D3; ++a) {
            int m = mn / 3, n = mn % 3;
            double *row = r->S + ((size_t)mn * D3 + a) * D3;
            for (int al = 0; al < Q3; ++al) {
                double t = w3[al] * dphi[((size_t)m * Q3 + al) * D3 + a];
                const double *dn = dphi + ((size_t)n * Q3 + al) * D3;
                for (int b = 0; b < D3; ++b) row[b] += t * dn[b];
            }
        }
    free(dphi);
    free(w3);
    return r;
}

void orc_ref_tables(const orc_ref *r, double *gll, double *gp, double *gw, double *B, double *G)
{
    if (gll) memcpy(gll, r->gll, sizeof(double) * r->D);
    if (gp) memcpy(gp, r->gp, sizeof(double) * r->Q);
    if (gw) memcpy(gw, r->gw, sizeof(double) * r->Q);
    if (B) memcpy(B, r->B, sizeof(double) * r->D * r->Q);
    if (G) memcpy(G, r->G, sizeof(double) * r->D * r->Q);
}

void orc_ref_blocks(const orc_ref *r, double *S)
{
    memcpy(S, r->S, sizeof(double) * 9 * (size_t)r->D3 * r->D3);
}

/* ------------------------------------------------------------------------ */
/* Element geometry and material coefficients.                               */
/* ------------------------------------------------------------------------ */

/* Inverse and determinant of a 3x3 row-major matrix (cofactor formula).    */
static double inv3(const double *J, double *Ji)
{
    double c00 = J[4] * J[8] - J[5] * J[7];
    double c01 = J[5] * J[6] - J[3] * J[8];
    double c02 = J[3] * J[7] - J[4] * J[6];
    double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
    double id = 1.0 / det;
    Ji[0] = c00 * id;
    Ji[1] = (J[2] * J[7] - J[1] * J[8]) * id;
    Ji[2] = (J[1] * J[5] - J[2] * J[4]) * id;
    Ji[3] = c01 * id;
    Ji[4] = (J[0] * J[8] - J[2] * J[6]) * id;
    Ji[5] = (J[2] * J[3] - J[0] * J[5]) * id;
    Ji[6] = c02 * id;
    Ji[7] = (J[1] * J[6] - J[0] * J[7]) * id;
    Ji[8] = (J[0] * J[4] - J[1] * J[3]) * id;
    return det;
}

/* Coefficients of the element matrix in terms of the reference blocks:
 *   K[(c,a),(b,d)] = sum_mn S_mn[a][b] * C[m][n][c][d]  with
 *   C = detJ * ( lambda Ji[m][c] Ji[n][d] + mu Ji[m][d] Ji[n][c]
 *                + mu delta_cd sum_k Ji[m][k] Ji[n][k] ),
 * which is sigma(phi_b e_d) : grad(phi_a e_c) with physical gradients
 * grad phi = J^{-T} grad_ref phi (Eq. 3, 4).                                */
int orc_element_coeff(const double *J, double lambda, double mu, double *C, double *detJ_out)
{
    double Ji[9];
    double det = inv3(J, Ji);
    if (!(det > 0.0)) return -1;
    for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) {
            double g = 0.0;
            for (int k = 0; k < 3; ++k) g += Ji[m * 3 + k] * Ji[n * 3 + k];
            for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d) {
                    double v = lambda * Ji[m * 3 + c] * Ji[n * 3 + d]
                             + mu * Ji[m * 3 + d] * Ji[n * 3 + c]
                             + (c == d ? mu * g : 0.0);
                    C[((m * 3 + n) * 3 + c) * 3 + d] = det * v;
                }
        }
    if (detJ_out) *detJ_out = det;
    return 0;
}

/* The same coefficients for a general (anisotropic) elasticity tensor
 * (Eq. 2), C4[((c*3 + j)*3 + d)*3 + l] = C_cjdl:
 *   C[m][n][c][d] = detJ sum_jl Ji[m][j] C_cjdl Ji[n][l],
 * i.e. sigma_cj = sum_dl C_cjdl du_d/dx_l tested with d phi_a / dx_j.       */
int orc_element_coeff_t(const double *J, const double *C4, double *C, double *detJ_out)
{
    double Ji[9];
    double det = inv3(J, Ji);
    if (!(det > 0.0)) return -1;
    for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n)
            for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d) {
                    double v = 0.0;
                    for (int j = 0; j < 3; ++j)
                        for (int l = 0; l < 3; ++l) v += Ji[m * 3 + j] * C4[((c * 3 + j) * 3 + d) * 3 + l] * Ji[n * 3 + l];
                    C[((m * 3 + n) * 3 + c) * 3 + d] = det * v;
                }
    if (detJ_out) *detJ_out = det;
    return 0;
}

/* Coefficients of element e: the per-element tensor (ctens[e], 81 values)
 * when given, else the per-element isotropic material, else the constants. */
static int element_coeff_of(int64_t e, const double *affine, double lambda, double mu, const double *mat,
                            const double *ctens, double *C)
{
    if (ctens) return orc_element_coeff_t(affine + 12 * e, ctens + 81 * e, C, NULL);
    const double le = mat ? mat[2 * e] : lambda, me = mat ? mat[2 * e + 1] : mu;
    return orc_element_coeff(affine + 12 * e, le, me, C, NULL);
}

/* Dense element matrix, row (c,a) = c*D3 + a, column (d,b) = d*D3 + b.     */
static void element_matrix_from(const orc_ref *r, const double *C, double *K);

int orc_element_matrix(const orc_ref *r, const double *J, double lambda, double mu, double *K)
{
    double C[81];
    if (orc_element_coeff(J, lambda, mu, C, NULL)) return -1;
    element_matrix_from(r, C, K);
    return 0;
}

/* Element matrix of an anisotropic tensor C4 (C_cjdl, 81 values).          */
int orc_element_matrix_t(const orc_ref *r, const double *J, const double *C4, double *K)
{
    double C[81];
    if (orc_element_coeff_t(J, C4, C, NULL)) return -1;
    element_matrix_from(r, C, K);
    return 0;
}

static void element_matrix_from(const orc_ref *r, const double *C, double *K)
{
    int D3 = r->D3, N = 3 * D3;
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < D3; ++a)
            for (int d = 0; d < 3; ++d)
                for (int b = 0; b < D3; ++b) {
                    double s = 0.0;
                    for (int mn = 0; mn < 9; ++mn)
                        s += r->S[((size_t)mn * D3 + a) * D3 + b] * C[(mn * 3 + c) * 3 + d];
                    K[(size_t)(c * D3 + a) * N + d * D3 + b] = s;
                }
}

/* ------------------------------------------------------------------------ */
/* Structured mesh helpers.                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz, p, D, Mx, My, Mz;
    int64_t Nn, ne;
} grid_t;

static grid_t make_grid(int nx, int ny, int nz, int p)
{
    grid_t g;
    g.nx = nx; g.ny = ny; g.nz = nz; g.p = p; g.D = p + 1;
    g.Mx = nx * p + 1; g.My = ny * p + 1; g.Mz = nz * p + 1;
    g.Nn = (int64_t)g.Mx * g.My * g.Mz;
    g.ne = (int64_t)nx * ny * nz;
    return g;
}

/* global node index of local node (ix,iy,iz) of element e */
static int64_t node_of(const grid_t *g, int64_t e, int ix, int iy, int iz)
{
    int ex = (int)(e % g->nx);
    int ey = (int)((e / g->nx) % g->ny);
    int ez = (int)(e / ((int64_t)g->nx * g->ny));
    int64_t gx = (int64_t)ex * g->p + ix, gy = (int64_t)ey * g->p + iy, gz = (int64_t)ez * g->p + iz;
    return gx + (int64_t)g->Mx * (gy + (int64_t)g->My * gz);
}

/* Element matrix action y_e = K_e x_e without storing K_e:
 *   v[mn][c][b] = sum_d C[m][n][c][d] x[d][b]
 *   y[c][a]     = sum_mn sum_b S_mn[a][b] v[mn][c][b]                      */
static void element_apply(const orc_ref *r, const double *C, const double *xe, double *ye, double *v)
{
    int D3 = r->D3;
    for (int mn = 0; mn < 9; ++mn)
        for (int c = 0; c < 3; ++c)
            for (int b = 0; b < D3; ++b) {
                double s = 0.0;
                for (int d = 0; d < 3; ++d) s += C[(mn * 3 + c) * 3 + d] * xe[d * D3 + b];
                v[((size_t)mn * 3 + c) * D3 + b] = s;
            }
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < D3; ++a) {
            double s = 0.0;
            for (int mn = 0; mn < 9; ++mn) {
                const double *Srow = r->S + ((size_t)mn * D3 + a) * D3;
                const double *vv = v + ((size_t)mn * 3 + c) * D3;
                for (int b = 0; b < D3; ++b) s += Srow[b] * vv[b];
            }
            ye[c * D3 + a] = s;
        }
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* y = A x for the whole mesh (constrained if ess != NULL).  Element results
 * are kept per element and summed node by node in a fixed order, so the
 * result does not depend on the thread count.                              */
/* mat: per-element material, (lambda_e, mu_e) at mat[2e], mat[2e+1], or
 * NULL for the constant (lambda, mu) -- the paper's PA data D holds the
 * material per quadrature point, lambda(alpha, e) and mu(alpha, e)
 * (Sec. 4.5); for material constant on each element that is this array.   */
int orc_apply_m(const orc_ref *r, int nx, int ny, int nz, const double *affine,
                double lambda, double mu, const double *mat, const double *ctens, const uint8_t *ess,
                const double *x, double *y, int nthreads);

int orc_apply(const orc_ref *r, int nx, int ny, int nz, const double *affine,
              double lambda, double mu, const uint8_t *ess, const double *x, double *y, int nthreads)
{
    return orc_apply_m(r, nx, ny, nz, affine, lambda, mu, NULL, NULL, ess, x, y, nthreads);
}

/* ctens: per-element anisotropic tensor [ne][81] (C_cjdl), or NULL.        */
int orc_apply_m(const orc_ref *r, int nx, int ny, int nz, const double *affine,
                double lambda, double mu, const double *mat, const double *ctens, const uint8_t *ess,
                const double *x, double *y, int nthreads)
{
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    grid_t g = make_grid(nx, ny, nz, r->p);
    int D = g.D, D3 = r->D3;
    double *ye_all = (double *)malloc(sizeof(double) * (size_t)g.ne * 3 * D3);
    if (!ye_all) return -2;
    int bad = 0;
    set_threads(nthreads);
#pragma omp parallel reduction(| : bad)
    {
        double *xe = (double *)malloc(sizeof(double) * 3 * D3);
        double *v = (double *)malloc(sizeof(double) * 27 * (size_t)D3);
        double C[81];
#pragma omp for schedule(dynamic, 16)
        for (int64_t e = 0; e < g.ne; ++e) {
            if (element_coeff_of(e, affine, lambda, mu, mat, ctens, C)) { bad = 1; continue; }
            for (int iz = 0; iz < D; ++iz)
                for (int iy = 0; iy < D; ++iy)
                    for (int ix = 0; ix < D; ++ix) {
                        int a = ix + D * (iy + D * iz);
                        int64_t gn = node_of(&g, e, ix, iy, iz);
                        for (int c = 0; c < 3; ++c) {
                            int64_t k = c * g.Nn + gn;
                            xe[c * D3 + a] = (ess && ess[k]) ? 0.0 : x[k];
                        }
                    }
            element_apply(r, C, xe, ye_all + (size_t)e * 3 * D3, v);
        }
        free(xe);
        free(v);
    }
    if (bad) { free(ye_all); return -3; }
    /* node-wise assembly: for each global node, the contributing elements
     * in increasing element order */
#pragma omp parallel for schedule(static)
    for (int64_t gz = 0; gz < g.Mz; ++gz)
        for (int64_t gy = 0; gy < g.My; ++gy)
            for (int64_t gx = 0; gx < g.Mx; ++gx) {
                int64_t gn = gx + g.Mx * (gy + g.My * gz);
                double acc[3] = {0.0, 0.0, 0.0};
                for (int dz = 1; dz >= 0; --dz)
                    for (int dy = 1; dy >= 0; --dy)
                        for (int dx = 1; dx >= 0; --dx) {
                            /* element whose local node (ix,iy,iz) is gn */
                            int64_t ex = gx / g.p - dx, ey = gy / g.p - dy, ez = gz / g.p - dz;
                            int ix = (int)(gx - (gx / g.p - dx) * g.p);
                            int iy = (int)(gy - (gy / g.p - dy) * g.p);
                            int iz = (int)(gz - (gz / g.p - dz) * g.p);
                            if (ex < 0 || ey < 0 || ez < 0 || ex >= g.nx || ey >= g.ny || ez >= g.nz) continue;
                            if (ix > g.p || iy > g.p || iz > g.p) continue;
                            int64_t e = ex + (int64_t)g.nx * (ey + (int64_t)g.ny * ez);
                            int a = ix + D * (iy + D * iz);
                            for (int c = 0; c < 3; ++c) acc[c] += ye_all[((size_t)e * 3 + c) * D3 + a];
                        }
                for (int c = 0; c < 3; ++c) {
                    int64_t k = c * g.Nn + gn;
                    y[k] = (ess && ess[k]) ? x[k] : acc[c];
                }
            }
    free(ye_all);
    return 0;
}

/* Selected entries of y = A x (rows are L-vector indices), computed one by
 * one from the rows of the contributing element matrices.                  */
int orc_apply_rows_m(const orc_ref *r, int nx, int ny, int nz, const double *affine,
                     double lambda, double mu, const double *mat, const double *ctens, const uint8_t *ess,
                     const double *x, int64_t nrows, const int64_t *rows, double *yrows, int nthreads);

int orc_apply_rows(const orc_ref *r, int nx, int ny, int nz, const double *affine,
                   double lambda, double mu, const uint8_t *ess, const double *x,
                   int64_t nrows, const int64_t *rows, double *yrows, int nthreads)
{
    return orc_apply_rows_m(r, nx, ny, nz, affine, lambda, mu, NULL, NULL, ess, x, nrows, rows, yrows, nthreads);
}

int orc_apply_rows_m(const orc_ref *r, int nx, int ny, int nz, const double *affine,
                     double lambda, double mu, const double *mat, const double *ctens, const uint8_t *ess,
                     const double *x, int64_t nrows, const int64_t *rows, double *yrows, int nthreads)
{
    grid_t g = make_grid(nx, ny, nz, r->p);
    int D = g.D, D3 = r->D3, p = g.p;
    int bad = 0;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8) reduction(| : bad)
    for (int64_t k = 0; k < nrows; ++k) {
        int64_t row = rows[k];
        if (row < 0 || row >= 3 * g.Nn) { bad = 1; continue; }
        int c = (int)(row / g.Nn);
        int64_t gn = row % g.Nn;
        if (ess && ess[row]) { yrows[k] = x[row]; continue; }
        int64_t gx = gn % g.Mx, gy = (gn / g.Mx) % g.My, gz = gn / ((int64_t)g.Mx * g.My);
        double acc = 0.0;
        for (int dz = 1; dz >= 0; --dz)
            for (int dy = 1; dy >= 0; --dy)
                for (int dx = 1; dx >= 0; --dx) {
                    int64_t ex = gx / p - dx, ey = gy / p - dy, ez = gz / p - dz;
                    if (ex < 0 || ey < 0 || ez < 0 || ex >= g.nx || ey >= g.ny || ez >= g.nz) continue;
                    int ix = (int)(gx - ex * p), iy = (int)(gy - ey * p), iz = (int)(gz - ez * p);
                    if (ix > p || iy > p || iz > p) continue;
                    int64_t e = ex + (int64_t)g.nx * (ey + (int64_t)g.ny * ez);
                    int a = ix + D * (iy + D * iz);
                    double C[81];
                    if (element_coeff_of(e, affine, lambda, mu, mat, ctens, C)) { bad = 1; continue; }
                    for (int bz = 0; bz < D; ++bz)
                        for (int by = 0; by < D; ++by)
                            for (int bx = 0; bx < D; ++bx) {
                                int b = bx + D * (by + D * bz);
                                int64_t gb = node_of(&g, e, bx, by, bz);
                                double xb[3];
                                for (int d = 0; d < 3; ++d) {
                                    int64_t kk = d * g.Nn + gb;
                                    xb[d] = (ess && ess[kk]) ? 0.0 : x[kk];
                                }
                                for (int mn = 0; mn < 9; ++mn) {
                                    double s = r->S[((size_t)mn * D3 + a) * D3 + b];
                                    const double *Cm = C + (mn * 3 + c) * 3;
                                    acc += s * (Cm[0] * xb[0] + Cm[1] * xb[1] + Cm[2] * xb[2]);
                                }
                            }
                }
        yrows[k] = acc;
    }
    return bad ? -3 : 0;
}

/* Diagonal of the (constrained) assembled matrix: sum over elements of the
 * element-matrix diagonal; essential entries are 1.                        */
int orc_diag_m(const orc_ref *r, int nx, int ny, int nz, const double *affine,
               double lambda, double mu, const double *mat, const double *ctens, const uint8_t *ess, double *dg,
               int nthreads);

int orc_diag(const orc_ref *r, int nx, int ny, int nz, const double *affine,
             double lambda, double mu, const uint8_t *ess, double *dg, int nthreads)
{
    return orc_diag_m(r, nx, ny, nz, affine, lambda, mu, NULL, NULL, ess, dg, nthreads);
}

int orc_diag_m(const orc_ref *r, int nx, int ny, int nz, const double *affine,
               double lambda, double mu, const double *mat, const double *ctens, const uint8_t *ess, double *dg,
               int nthreads)
{
    grid_t g = make_grid(nx, ny, nz, r->p);
    int D = g.D, D3 = r->D3, p = g.p;
    int bad = 0;
    set_threads(nthreads);
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t gn = 0; gn < g.Nn; ++gn) {
        int64_t gx = gn % g.Mx, gy = (gn / g.Mx) % g.My, gz = gn / ((int64_t)g.Mx * g.My);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int dz = 1; dz >= 0; --dz)
            for (int dy = 1; dy >= 0; --dy)
                for (int dx = 1; dx >= 0; --dx) {
                    int64_t ex = gx / p - dx, ey = gy / p - dy, ez = gz / p - dz;
                    if (ex < 0 || ey < 0 || ez < 0 || ex >= g.nx || ey >= g.ny || ez >= g.nz) continue;
                    int ix = (int)(gx - ex * p), iy = (int)(gy - ey * p), iz = (int)(gz - ez * p);
                    if (ix > p || iy > p || iz > p) continue;
                    int64_t e = ex + (int64_t)g.nx * (ey + (int64_t)g.ny * ez);
                    int a = ix + D * (iy + D * iz);
                    double C[81];
                    if (element_coeff_of(e, affine, lambda, mu, mat, ctens, C)) { bad = 1; continue; }
                    for (int c = 0; c < 3; ++c)
                        for (int mn = 0; mn < 9; ++mn)
                            acc[c] += r->S[((size_t)mn * D3 + a) * D3 + a] * C[(mn * 3 + c) * 3 + c];
                }
        for (int c = 0; c < 3; ++c) {
            int64_t k = c * g.Nn + gn;
            dg[k] = (ess && ess[k]) ? 1.0 : acc[c];
        }
    }
    return bad ? -3 : 0;
}

/* Load vector F_(i,c) = sum_e sum_alpha w_alpha detJ f_c(x(alpha)) Phi_i(alpha)
 * with f_c(x) = f0[c] + sum_k amp[c][k] sin(kx*x + ky*y + kz*z + phase),
 * mode k of component c stored as amp, kx, ky, kz, phase at
 * modes[(c*nmodes + k)*5 + 0..4].  Essential entries are 0.                 */
int orc_load(const orc_ref *r, int nx, int ny, int nz, const double *affine, const double *f0,
             int nmodes, const double *modes, const uint8_t *ess, double *F, int nthreads)
{
    grid_t g = make_grid(nx, ny, nz, r->p);
    int D = g.D, Q = r->Q, D3 = r->D3, Q3 = r->Q3;
    double *fe_all = (double *)malloc(sizeof(double) * (size_t)g.ne * 3 * D3);
    if (!fe_all) return -2;
    int bad = 0;
    set_threads(nthreads);
#pragma omp parallel reduction(| : bad)
    {
        double *fq = (double *)malloc(sizeof(double) * 3 * Q3);
#pragma omp for schedule(dynamic, 16)
        for (int64_t e = 0; e < g.ne; ++e) {
            const double *J = affine + 12 * e, *x0 = affine + 12 * e + 9;
            double Ji[9];
            double det = inv3(J, Ji);
            if (!(det > 0.0)) { bad = 1; continue; }
            for (int qz = 0; qz < Q; ++qz)
                for (int qy = 0; qy < Q; ++qy)
                    for (int qx = 0; qx < Q; ++qx) {
                        int al = qx + Q * (qy + Q * qz);
                        double xi[3] = {r->gp[qx], r->gp[qy], r->gp[qz]};
                        double X[3];
                        for (int i = 0; i < 3; ++i)
                            X[i] = x0[i] + J[3 * i] * xi[0] + J[3 * i + 1] * xi[1] + J[3 * i + 2] * xi[2];
                        double w = r->gw[qx] * r->gw[qy] * r->gw[qz] * det;
                        for (int c = 0; c < 3; ++c) {
                            double f = f0 ? f0[c] : 0.0;
                            for (int k = 0; k < nmodes; ++k) {
                                const double *md = modes + ((size_t)c * nmodes + k) * 5;
                                f += md[0] * sin(md[1] * X[0] + md[2] * X[1] + md[3] * X[2] + md[4]);
                            }
                            fq[c * Q3 + al] = w * f;
                        }
                    }
            double *fe = fe_all + (size_t)e * 3 * D3;
            for (int iz = 0; iz < D; ++iz)
                for (int iy = 0; iy < D; ++iy)
                    for (int ix = 0; ix < D; ++ix) {
                        int a = ix + D * (iy + D * iz);
                        double s[3] = {0.0, 0.0, 0.0};
                        for (int qz = 0; qz < Q; ++qz)
                            for (int qy = 0; qy < Q; ++qy)
                                for (int qx = 0; qx < Q; ++qx) {
                                    int al = qx + Q * (qy + Q * qz);
                                    double phi = r->B[ix * Q + qx] * r->B[iy * Q + qy] * r->B[iz * Q + qz];
                                    for (int c = 0; c < 3; ++c) s[c] += fq[c * Q3 + al] * phi;
                                }
                        for (int c = 0; c < 3; ++c) fe[c * D3 + a] = s[c];
                    }
        }
        free(fq);
    }
    if (bad) { free(fe_all); return -3; }
    int p = g.p;
#pragma omp parallel for schedule(static)
    for (int64_t gn = 0; gn < g.Nn; ++gn) {
        int64_t gx = gn % g.Mx, gy = (gn / g.Mx) % g.My, gz = gn / ((int64_t)g.Mx * g.My);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int dz = 1; dz >= 0; --dz)
            for (int dy = 1; dy >= 0; --dy)
                for (int dx = 1; dx >= 0; --dx) {
                    int64_t ex = gx / p - dx, ey = gy / p - dy, ez = gz / p - dz;
                    if (ex < 0 || ey < 0 || ez < 0 || ex >= g.nx || ey >= g.ny || ez >= g.nz) continue;
                    int ix = (int)(gx - ex * p), iy = (int)(gy - ey * p), iz = (int)(gz - ez * p);
                    if (ix > p || iy > p || iz > p) continue;
                    int64_t e = ex + (int64_t)g.nx * (ey + (int64_t)g.ny * ez);
                    int a = ix + D * (iy + D * iz);
                    for (int c = 0; c < 3; ++c) acc[c] += fe_all[((size_t)e * 3 + c) * D3 + a];
                }
        for (int c = 0; c < 3; ++c) {
            int64_t k = c * g.Nn + gn;
            F[k] = (ess && ess[k]) ? 0.0 : acc[c];
        }
    }
    free(fe_all);
    return 0;
}

/* Neumann load of a constant traction t on one face of the box (Eq. 1: the
 * boundary term integral over Gamma_N of t . v):
 *   F_(i,c) += sum over the boundary faces of the elements on that face of
 *              sum_(a,b) w_a w_b |dx/du x dx/dv| t_c Phi_i(face point),
 * face = 2 * axis + side (axis 0/1/2 = x/y/z, side 0 = low, 1 = high); the
 * face of an element is its reference face xi_axis = side, parametrised by
 * the two other reference coordinates (u, v) in increasing axis order, and
 * integrated with the q-point Gauss rule in each; the surface factor is the
 * norm of the cross product of the two corresponding columns of J.  The
 * basis is evaluated at the face points in full (no use of the nodal
 * property).  Contributions are added element by element in increasing
 * element order; essential entries are set to 0 afterwards.               */
int orc_traction(const orc_ref *r, int nx, int ny, int nz, const double *affine, int face, const double *t,
                 const uint8_t *ess, double *F)
{
    if (face < 0 || face > 5) return -1;
    grid_t g = make_grid(nx, ny, nz, r->p);
    const int D = g.D, Q = r->Q, D3 = r->D3;
    const int ax = face / 2, side = face % 2;
    const int bx = ax == 0 ? 1 : 0, cx = ax == 2 ? 1 : 2;  /* the two tangential axes, increasing */
    const int n3[3] = {nx, ny, nz};
    double side_pt = (double)side, lv[64], ld_[64];
    orc_lagrange(D, r->gll, 1, &side_pt, lv, ld_);      /* basis along the normal axis at the face */
    double *fe = (double *)malloc(sizeof(double) * 3 * D3);
    if (!fe) return -2;
    for (int64_t e = 0; e < g.ne; ++e) {
        const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
        const int64_t ei[3] = {ex, ey, ez};
        if (ei[ax] != (side ? n3[ax] - 1 : 0)) continue;
        const double *J = affine + 12 * e;
        /* columns b and c of J: dx/du and dx/dv */
        const double u[3] = {J[0 * 3 + bx], J[1 * 3 + bx], J[2 * 3 + bx]};
        const double v[3] = {J[0 * 3 + cx], J[1 * 3 + cx], J[2 * 3 + cx]};
        const double cr[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        const double ds = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        memset(fe, 0, sizeof(double) * 3 * D3);
        for (int iz = 0; iz < D; ++iz)
            for (int iy = 0; iy < D; ++iy)
                for (int ix = 0; ix < D; ++ix) {
                    const int il[3] = {ix, iy, iz};
                    double s = 0.0;
                    for (int qb = 0; qb < Q; ++qb)
                        for (int qa = 0; qa < Q; ++qa) {
                            double phi = lv[il[ax]] * r->B[il[bx] * Q + qa] * r->B[il[cx] * Q + qb];
                            s += r->gw[qa] * r->gw[qb] * ds * phi;
                        }
                    const int a = ix + D * (iy + D * iz);
                    for (int c = 0; c < 3; ++c) fe[c * D3 + a] = t[c] * s;
                }
        for (int iz = 0; iz < D; ++iz)
            for (int iy = 0; iy < D; ++iy)
                for (int ix = 0; ix < D; ++ix) {
                    const int a = ix + D * (iy + D * iz);
                    const int64_t gn = node_of(&g, e, ix, iy, iz);
                    for (int c = 0; c < 3; ++c) F[c * g.Nn + gn] += fe[c * D3 + a];
                }
    }
    free(fe);
    if (ess)
        for (int64_t k = 0; k < 3 * g.Nn; ++k)
            if (ess[k]) F[k] = 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* p-transfer between GLL spaces of degrees pc < pf on the same mesh:
 * prolongation evaluates the coarse field at the fine nodes (Sec. 3,
 * polynomial interpolation for p-levels); restriction is its transpose,
 * formed here by scattering each fine value with the same weights.         */
/* ------------------------------------------------------------------------ */
static int transfer(int pc, int pf, int nx, int ny, int nz, const double *in, double *out, int transpose)
{
    if (pc < 1 || pf < 1 || pc > 32 || pf > 32) return -1;
    grid_t gc = make_grid(nx, ny, nz, pc), gf = make_grid(nx, ny, nz, pf);
    double nc[64], nf[64];
    orc_gll01(pc, nc);
    orc_gll01(pf, nf);
    int Dc = pc + 1, Df = pf + 1;
    double *Lv = (double *)malloc(sizeof(double) * Dc * Df);
    double *Ld = (double *)malloc(sizeof(double) * Dc * Df);
    if (!Lv || !Ld) { free(Lv); free(Ld); return -2; }
    /* Lv[i*Df + j] = coarse basis i at fine node j */
    orc_lagrange(Dc, nc, Df, nf, Lv, Ld);
    if (transpose) memset(out, 0, sizeof(double) * 3 * gc.Nn);
    for (int64_t gn = 0; gn < gf.Nn; ++gn) {
        int64_t gx = gn % gf.Mx, gy = (gn / gf.Mx) % gf.My, gz = gn / ((int64_t)gf.Mx * gf.My);
        /* the element that holds this fine node (lowest index) */
        int64_t ex = gx / pf, ey = gy / pf, ez = gz / pf;
        if (ex >= nx) ex = nx - 1;
        if (ey >= ny) ey = ny - 1;
        if (ez >= nz) ez = nz - 1;
        int jx = (int)(gx - ex * pf), jy = (int)(gy - ey * pf), jz = (int)(gz - ez * pf);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int iz = 0; iz < Dc; ++iz)
            for (int iy = 0; iy < Dc; ++iy)
                for (int ix = 0; ix < Dc; ++ix) {
                    double w = Lv[ix * Df + jx] * Lv[iy * Df + jy] * Lv[iz * Df + jz];
                    if (w == 0.0) continue;
                    int64_t cn = (ex * pc + ix) + gc.Mx * ((ey * pc + iy) + (int64_t)gc.My * (ez * pc + iz));
                    for (int c = 0; c < 3; ++c) {
                        if (!transpose) acc[c] += w * in[c * gc.Nn + cn];
                        else out[c * gc.Nn + cn] += w * in[c * gf.Nn + gn];
                    }
                }
        if (!transpose)
            for (int c = 0; c < 3; ++c) out[c * gf.Nn + gn] = acc[c];
    }
    free(Lv);
    free(Ld);
    return 0;
}

int orc_prolong(int pc, int pf, int nx, int ny, int nz, const double *xc, double *xf)
{
    return transfer(pc, pf, nx, ny, nz, xc, xf, 0);
}

int orc_restrict(int pc, int pf, int nx, int ny, int nz, const double *rf, double *rc)
{
    return transfer(pc, pf, nx, ny, nz, rf, rc, 1);
}

/* Affine maps of the undistorted structured grid on the box [lo, hi]. */
int orc_box_affine(int nx, int ny, int nz, const double *lo, const double *hi, double *affine)
{
    double h[3] = {(hi[0] - lo[0]) / nx, (hi[1] - lo[1]) / ny, (hi[2] - lo[2]) / nz};
    for (int ez = 0; ez < nz; ++ez)
        for (int ey = 0; ey < ny; ++ey)
            for (int ex = 0; ex < nx; ++ex) {
                double *A = affine + 12 * ((size_t)ex + (size_t)nx * (ey + (size_t)ny * ez));
                memset(A, 0, sizeof(double) * 12);
                A[0] = h[0]; A[4] = h[1]; A[8] = h[2];
                A[9] = lo[0] + ex * h[0];
                A[10] = lo[1] + ey * h[1];
                A[11] = lo[2] + ez * h[2];
            }
    return 0;
}
