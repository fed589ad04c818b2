"""Exact-rational brute force of the elasticity stiffness matrix (p = 1, 2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

An independent cross-check of the FP64 oracle.  Nothing here uses Gauss
quadrature, barycentric formulas or the C library: the 1D Lagrange basis on
the rational GLL nodes ({0,1} for p=1, {0,1/2,1} for p=2) is expanded into
monomials with Fraction coefficients, every integral is done exactly
(int_0^1 x^k dx = 1/(k+1)), the inverse Jacobian is the exact cofactor
inverse, and each entry is the symmetric-gradient form of Eq. 4,
    a(u, v) = int lambda div(u) div(v) + 2 mu eps(u) : eps(v),
evaluated for u = phi_b e_d, v = phi_a e_c with physical gradients
grad phi = J^{-T} grad_ref phi.  Because the Gauss rule with p+2 points is
exact for these polynomial integrands on affine cells, this must agree with
the FP64 oracle to round-off.
"""
from __future__ import annotations

from fractions import Fraction as Fr
from itertools import product

GLL_RATIONAL = {1: [Fr(0), Fr(1)], 2: [Fr(0), Fr(1, 2), Fr(1)]}


def _pmul(a, b):
    out = [Fr(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] += x * y
    return out


def _pder(a):
    return [a[k] * k for k in range(1, len(a))] or [Fr(0)]


def _pint01(a):
    return sum((c / (k + 1) for k, c in enumerate(a)), Fr(0))


def lagrange_monomials(nodes):
    """Coefficients (ascending powers) of the Lagrange polynomials."""
    polys = []
    for i, xi in enumerate(nodes):
        poly = [Fr(1)]
        for j, xj in enumerate(nodes):
            if j != i:
                poly = _pmul(poly, [-xj / (xi - xj), Fr(1) / (xi - xj)])
        polys.append(poly)
    return polys


def one_d_integrals(p):
    """M[i][j] = int phi_i phi_j, Dm[i][j] = int phi_i' phi_j,
    K[i][j] = int phi_i' phi_j' on [0,1], exact."""
    phi = lagrange_monomials(GLL_RATIONAL[p])
    dphi = [_pder(f) for f in phi]
    n = p + 1
    M = [[_pint01(_pmul(phi[i], phi[j])) for j in range(n)] for i in range(n)]
    Dm = [[_pint01(_pmul(dphi[i], phi[j])) for j in range(n)] for i in range(n)]
    K = [[_pint01(_pmul(dphi[i], dphi[j])) for j in range(n)] for i in range(n)]
    return M, Dm, K


def ref_gradient_integrals(p):
    """R[m][n][a][b] = int_[0,1]^3 d_m Phi_a d_n Phi_b (Fubini over the
    tensor-product basis of Eq. 6)."""
    M, Dm, K = one_d_integrals(p)
    D = p + 1
    idx = [(ix, iy, iz) for iz in range(D) for iy in range(D) for ix in range(D)]

    def f1(i, j, da, db):
        if da and db:
            return K[i][j]
        if da:
            return Dm[i][j]
        if db:
            return Dm[j][i]
        return M[i][j]

    R = [[None] * 3 for _ in range(3)]
    for m in range(3):
        for n in range(3):
            blk = []
            for a in idx:
                row = []
                for b in idx:
                    v = Fr(1)
                    for k in range(3):
                        v *= f1(a[k], b[k], k == m, k == n)
                    row.append(v)
                blk.append(row)
            R[m][n] = blk
    return R


def inv3(J):
    (a, b, c), (d, e, f), (g, h, i) = J
    det = a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g)
    adj = [[e * i - f * h, c * h - b * i, b * f - c * e],
           [f * g - d * i, a * i - c * g, c * d - a * f],
           [d * h - e * g, b * g - a * h, a * e - b * d]]
    return [[adj[r][s] / det for s in range(3)] for r in range(3)], det


def element_matrix(p, J, lam, mu):
    """Exact element matrix (Fractions), rows/cols (c, a) -> c*D^3 + a."""
    J = [[Fr(v) for v in row] for row in J]
    lam, mu = Fr(lam), Fr(mu)
    Ji, det = inv3(J)
    if det <= 0:
        raise ValueError("detJ <= 0")
    R = ref_gradient_integrals(p)
    D3 = (p + 1) ** 3
    N = 3 * D3
    K = [[Fr(0)] * N for _ in range(N)]
    for a, b in product(range(D3), range(D3)):
        # P[j][k] = int d_j phi_b d_k phi_a dx (physical), 3x3
        P = [[det * sum(Ji[n][j] * Ji[m][k] * R[n][m][b][a] for n in range(3) for m in range(3))
              for k in range(3)] for j in range(3)]
        for c, d in product(range(3), range(3)):
            # div(phi_b e_d) div(phi_a e_c)
            val = lam * P[d][c]
            # eps(u)_ij = (delta_id d_j phi_b + delta_jd d_i phi_b)/2, eps(v) likewise
            ee = Fr(0)
            for i, j in product(range(3), range(3)):
                t = Fr(0)
                if i == d and i == c:
                    t += P[j][j]
                if i == d and j == c:
                    t += P[j][i]
                if j == d and i == c:
                    t += P[i][j]
                if j == d and j == c:
                    t += P[i][i]
                ee += t / 4
            val += 2 * mu * ee
            K[c * D3 + a][d * D3 + b] = val
    return K


def global_matrix(p, nx, J_list, lam, mu):
    """Exact assembled matrix of an nx*1*1 row of elements (component-major
    L-vector, node index x fastest), one exact J per element; lam and mu are
    numbers or one value per element."""
    D = p + 1
    D3 = D ** 3
    Mx, My = nx * p + 1, p + 1
    Nn = Mx * My * (p + 1)
    A = [[Fr(0)] * (3 * Nn) for _ in range(3 * Nn)]
    for e in range(nx):
        le = lam[e] if isinstance(lam, (list, tuple)) else lam
        me = mu[e] if isinstance(mu, (list, tuple)) else mu
        Ke = element_matrix(p, J_list[e], le, me)
        dofs = []
        for c in range(3):
            for a in range(D3):
                ix, iy, iz = a % D, (a // D) % D, a // (D * D)
                dofs.append(c * Nn + (e * p + ix) + Mx * (iy + My * iz))
        for r in range(3 * D3):
            for s in range(3 * D3):
                A[dofs[r]][dofs[s]] += Ke[r][s]
    return A
