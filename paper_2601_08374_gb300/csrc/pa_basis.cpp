// Host construction of the 1D rules used by the PA operator (Sec. 4.4:
// 1D interpolation/derivative tables B(D1D,Q1D), G(D1D,Q1D); Sec. 5.1.4:
// p+1 GLL nodes and p+2 Gauss-Legendre points per direction).
//
// Nodes and points are eigenvalues of symmetric tridiagonal Jacobi matrices
// (Golub & Welsch 1969), located by Sturm-sequence bisection: Legendre for
// the Gauss points, Jacobi(1,1) for the interior GLL nodes.  Gauss weights
// come from w = 2 / ((1 - t^2) P_q'(t)^2).  Lagrange polynomials use the
// product formula.
#include <cmath>

#include "pa_internal.h"

namespace pa {
namespace {

// Number of eigenvalues < x of the symmetric tridiagonal matrix with zero
// diagonal and off-diagonal b[0..n-2] (LDL^T inertia).
int sturm_count(int n, const double *b, double x)
{
    int neg = 0;
    double d = -x;
    if (d < 0) ++neg;
    for (int i = 1; i < n; ++i) {
        double prev = (d == 0.0) ? 1e-300 : d;
        d = -x - b[i - 1] * b[i - 1] / prev;
        if (d < 0) ++neg;
    }
    return neg;
}

// All n eigenvalues (ascending) of that matrix; they lie in (-1, 1).
void tridiag_eigs(int n, const double *b, double *ev)
{
    for (int k = 0; k < n; ++k) {
        double lo = -1.0, hi = 1.0;
        for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid == lo || mid == hi) break;
            if (sturm_count(n, b, mid) > k) hi = mid;
            else lo = mid;
        }
        ev[k] = 0.5 * (lo + hi);
    }
}

// Legendre P_n(t) and P_n'(t).
void legendre_and_derivative(int n, double t, double &P, double &dP)
{
    double pm = 1.0, pc = t;
    if (n == 0) { P = 1.0; dP = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        double pn = ((2 * k - 1) * t * pc - (k - 1) * pm) / k;
        pm = pc;
        pc = pn;
    }
    P = pc;
    // n (P_{n-1} - t P_n) / (1 - t^2)
    dP = n * (pm - t * pc) / (1.0 - t * t);
}

}  // namespace

void gauss_legendre_01(int q, double *x, double *w)
{
    double b[kMaxQ + 8] = {}, t[kMaxQ + 8] = {};
    for (int k = 1; k < q; ++k) b[k - 1] = k / std::sqrt(4.0 * k * k - 1.0);
    tridiag_eigs(q, b, t);
    for (int k = 0; k < q; ++k) {
        double P, dP;
        // one Newton polish step on P_q
        legendre_and_derivative(q, t[k], P, dP);
        double tk = t[k] - P / dP;
        legendre_and_derivative(q, tk, P, dP);
        x[k] = 0.5 * (1.0 + tk);
        w[k] = 1.0 / ((1.0 - tk * tk) * dP * dP);  // (2 / (...)) / 2 on [0,1]
    }
}

void gll_nodes_01(int p, double *x)
{
    x[0] = 0.0;
    x[p] = 1.0;
    int n = p - 1;
    if (n <= 0) return;
    double b[kMaxD + 8] = {}, t[kMaxD + 8] = {};
    // Jacobi(1,1) recurrence: b_k^2 = k (k + 2) / ((2k + 1)(2k + 3))
    for (int k = 1; k < n; ++k) b[k - 1] = std::sqrt(k * (k + 2.0) / ((2.0 * k + 1.0) * (2.0 * k + 3.0)));
    tridiag_eigs(n, b, t);
    for (int k = 0; k < n; ++k) x[k + 1] = 0.5 * (1.0 + t[k]);
}

void lagrange_product(int n, const double *nodes, int m, const double *pts, double *val, double *der)
{
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < m; ++j) {
            double xv = pts[j];
            double v = 1.0;
            for (int k = 0; k < n; ++k)
                if (k != i) v *= (xv - nodes[k]) / (nodes[i] - nodes[k]);
            double d = 0.0;
            for (int l = 0; l < n; ++l) {
                if (l == i) continue;
                double prod = 1.0 / (nodes[i] - nodes[l]);
                for (int k = 0; k < n; ++k)
                    if (k != i && k != l) prod *= (xv - nodes[k]) / (nodes[i] - nodes[k]);
                d += prod;
            }
            val[i * m + j] = v;
            der[i * m + j] = d;
        }
    }
}

void Basis1D::build(int p_, int q_)
{
    p = p_;
    D = p + 1;
    Q = q_;
    nodes.assign(D, 0.0);
    qpts.assign(Q, 0.0);
    qwts.assign(Q, 0.0);
    gll_nodes_01(p, nodes.data());
    gauss_legendre_01(Q, qpts.data(), qwts.data());
    B.assign(D * Q, 0.0);
    G.assign(D * Q, 0.0);
    lagrange_product(D, nodes.data(), Q, qpts.data(), B.data(), G.data());
    Bw.resize(D * Q);
    Gw.resize(D * Q);
    Md.assign(D, 0.0);
    Cd.assign(D, 0.0);
    Kd.assign(D, 0.0);
    for (int i = 0; i < D; ++i)
        for (int k = 0; k < Q; ++k) {
            double b = B[i * Q + k], g = G[i * Q + k], w = qwts[k];
            Bw[i * Q + k] = b * w;
            Gw[i * Q + k] = g * w;
            Md[i] += w * b * b;
            Cd[i] += w * b * g;
            Kd[i] += w * g * g;
        }
}

template <typename T>
void fill_tables(const Basis1D &b, Tables<T> &t)
{
    for (int i = 0; i < kMaxD * kMaxQ; ++i) t.B[i] = t.G[i] = t.Bw[i] = t.Gw[i] = T(0);
    for (int i = 0; i < b.D * b.Q; ++i) {
        t.B[i] = T(b.B[i]);
        t.G[i] = T(b.G[i]);
        t.Bw[i] = T(b.Bw[i]);
        t.Gw[i] = T(b.Gw[i]);
    }
    transpose_tables(t, b.D, b.Q);
}
template void fill_tables<double>(const Basis1D &, Tables<double> &);
template void fill_tables<float>(const Basis1D &, Tables<float> &);

}  // namespace pa
