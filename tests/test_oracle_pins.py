"""Pins of the FP64 CPU oracle against facts fixed by the mathematics and by
textbook special cases, not against the oracle itself.

Each test names what fixes the expected value: a textbook rule, an exact
rational brute force (oracle.exact), a library routine used as an
independent step (numpy's Gauss-Legendre rule and Legendre polynomials),
or an invariant of linear elasticity (symmetry, rigid-body kernel, patch
test, strain energy of a uniform strain, integration by parts).
"""
import math
from fractions import Fraction as Fr

import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

import oracle
from oracle import exact
import synthetic as syn


# --------------------------------------------------------------------------
# 1D rules
# --------------------------------------------------------------------------
def test_gauss_textbook_values():
    # Gauss(2), Gauss(3) on [0,1]: 1/2 -+ 1/(2 sqrt 3); 1/2 -+ sqrt(3/5)/2 with 5/18, 8/18, 5/18.
    x, w = oracle.gauss01(2)
    np.testing.assert_allclose(x, [0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [0.5, 0.5], rtol=0, atol=1e-15)
    x, w = oracle.gauss01(3)
    h = 0.5 * np.sqrt(3.0 / 5.0)
    np.testing.assert_allclose(x, [0.5 - h, 0.5, 0.5 + h], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [5 / 18, 8 / 18, 5 / 18], rtol=0, atol=1e-15)


@pytest.mark.parametrize("q", range(1, 13))
def test_gauss_matches_numpy_and_exactness(q):
    x, w = oracle.gauss01(q)
    t, v = npleg.leggauss(q)
    np.testing.assert_allclose(x, (t + 1) / 2, rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, v / 2, rtol=0, atol=2e-15)
    for k in range(2 * q):  # exact for degree <= 2q-1
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-14
    # and not beyond: the textbook error of the q-point rule on [0,1] for x^(2q)
    # is (q!)^4 / ((2q+1) ((2q)!)^2)
    err = 1.0 / (2 * q + 1) - np.dot(w, x ** (2 * q))
    theory = math.factorial(q) ** 4 / ((2 * q + 1) * math.factorial(2 * q) ** 2)
    if theory > 1e-11:
        assert abs(err - theory) <= 1e-3 * theory


def test_gll_textbook_values():
    np.testing.assert_allclose(oracle.gll01(1), [0, 1], atol=0)
    np.testing.assert_allclose(oracle.gll01(2), [0, 0.5, 1], atol=1e-16)
    s5 = np.sqrt(5) / 10
    np.testing.assert_allclose(oracle.gll01(3), [0, 0.5 - s5, 0.5 + s5, 1], atol=1e-15)
    s21 = np.sqrt(21) / 14
    np.testing.assert_allclose(oracle.gll01(4), [0, 0.5 - s21, 0.5, 0.5 + s21, 1], atol=1e-15)


@pytest.mark.parametrize("p", range(1, 11))
def test_gll_interior_nodes_are_roots_of_dP(p):
    x = oracle.gll01(p)
    assert x[0] == 0.0 and x[-1] == 1.0 and np.all(np.diff(x) > 0)
    dP = npleg.legder([0] * p + [1])
    if p > 1:
        assert np.max(np.abs(npleg.legval(2 * x[1:-1] - 1, dP))) < 1e-11 * p * p
    np.testing.assert_allclose(x, 1 - x[::-1], atol=1e-15)  # symmetric


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_lagrange_basis_properties(p):
    nodes = oracle.gll01(p)
    val, der = oracle.lagrange(nodes, nodes)
    np.testing.assert_allclose(val, np.eye(p + 1), atol=0)
    rng = np.random.default_rng(p)
    pts = rng.uniform(0, 1, 17)
    val, der = oracle.lagrange(nodes, pts)
    np.testing.assert_allclose(val.sum(0), 1.0, atol=1e-13)
    np.testing.assert_allclose(der.sum(0), 0.0, atol=1e-11)
    for deg in range(p + 1):  # reproduces polynomials and derivatives of degree <= p
        c = rng.normal(size=deg + 1)
        f = np.polynomial.Polynomial(c)
        for xs in (pts, nodes):
            v, d = oracle.lagrange(nodes, xs)
            np.testing.assert_allclose(f(nodes) @ v, f(xs), atol=1e-12)
            np.testing.assert_allclose(f(nodes) @ d, f.deriv()(xs), atol=1e-10)


# --------------------------------------------------------------------------
# Reference stiffness blocks S_mn
# --------------------------------------------------------------------------
def _numpy_1d_integrals(p):
    """int phi_i phi_j, int phi_i' phi_j, int phi_i' phi_j' on [0,1] with an
    independent construction: the Lagrange basis expanded in shifted Legendre
    polynomials (numpy.polynomial.legendre, Vandermonde solve on the GLL
    nodes) and integrated with numpy's 30-point Gauss rule."""
    nodes = oracle.gll01(p)
    coef = np.linalg.inv(npleg.legvander(2 * nodes - 1, p))  # column i: l_i in Legendre basis
    t, v = npleg.leggauss(30)
    w = v / 2
    P = npleg.legvander(t, p) @ coef
    dcoef = np.stack([2 * npleg.legder(coef[:, i]) for i in range(p + 1)], axis=1)
    dP = npleg.legvander(t, max(p - 1, 0))[:, :dcoef.shape[0]] @ dcoef
    M = P.T @ (w[:, None] * P)
    Dm = dP.T @ (w[:, None] * P)
    K = dP.T @ (w[:, None] * dP)
    return M, Dm, K


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8])
def test_ref_blocks_against_fubini(p):
    S = oracle.ref(p).blocks()
    M, Dm, K = _numpy_1d_integrals(p)
    D = p + 1
    mats = {(False, False): M, (True, False): Dm, (False, True): Dm.T, (True, True): K}
    for m in range(3):
        for n in range(3):
            # tensor index a = ix + D*(iy + D*iz) -> kron order (z, y, x)
            f = [mats[(k == m, k == n)] for k in range(3)]
            ref = np.kron(f[2], np.kron(f[1], f[0]))
            np.testing.assert_allclose(S[m, n], ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))
    np.testing.assert_allclose(S.sum(axis=3), 0.0, atol=1e-12)  # grad of a constant is 0
    for m in range(3):
        for n in range(3):
            np.testing.assert_allclose(S[m, n], S[n, m].T, atol=1e-14)


def test_ref_blocks_exact_rational_p2():
    S = oracle.ref(2).blocks()
    R = exact.ref_gradient_integrals(2)
    for m in range(3):
        for n in range(3):
            np.testing.assert_allclose(S[m, n], np.array(R[m][n], dtype=float), rtol=0, atol=2e-15)


# --------------------------------------------------------------------------
# Element matrix against the exact-rational brute force (p = 1, 2)
# --------------------------------------------------------------------------
J_RAT = [[Fr(1, 2), Fr(1, 10), Fr(0)], [Fr(-1, 8), Fr(1, 3), Fr(1, 7)], [Fr(1, 5), Fr(0), Fr(1)]]
J_RAT2 = [[Fr(2, 3), Fr(0), Fr(-1, 9)], [Fr(1, 4), Fr(3, 4), Fr(0)], [Fr(0), Fr(1, 6), Fr(1, 2)]]


@pytest.mark.parametrize("p", [1, 2])
def test_element_matrix_exact(p):
    lam, mu = Fr(3, 2), Fr(2, 3)
    Kx = np.array(exact.element_matrix(p, J_RAT, lam, mu), dtype=float)
    Ko = oracle.ref(p).element_matrix(np.array(J_RAT, dtype=float), float(lam), float(mu))
    assert np.max(np.abs(Ko - Kx)) <= 1e-13 * np.max(np.abs(Kx))
    np.testing.assert_allclose(Ko, Ko.T, atol=1e-13 * np.abs(Ko).max())


@pytest.mark.parametrize("p", [1, 2])
def test_global_two_element_exact(p):
    lam, mu = Fr(1, 1), Fr(5, 7)
    Ax = np.array(exact.global_matrix(p, 2, [J_RAT, J_RAT2], lam, mu), dtype=float)
    aff = np.zeros((2, 12))
    aff[0, :9] = np.array(J_RAT, dtype=float).reshape(9)
    aff[1, :9] = np.array(J_RAT2, dtype=float).reshape(9)
    Ao = oracle.assemble_dense(p, 2, 1, 1, aff, float(lam), float(mu))
    scale = np.abs(Ax).max()
    assert np.max(np.abs(Ao - Ax)) <= 1e-13 * scale
    x = np.random.default_rng(0).uniform(-1, 1, Ax.shape[0])
    y = oracle.apply(p, 2, 1, 1, aff, float(lam), float(mu), x)
    assert np.max(np.abs(y - Ax @ x)) <= 1e-13 * scale * np.abs(x).sum() / len(x) * 10


def test_trilinear_brick_is_textbook_p1():
    # For p = 1 on the unit cube with lambda = 0, mu = 1/2 the x-x block of
    # the stiffness equals the scalar Laplacian of the trilinear brick plus
    # the d_x d_x term:  K_xx = 1/2 (Lap + Dxx).  Both are products of the
    # 1D linear-element matrices  M = [[1/3,1/6],[1/6,1/3]],  K = [[1,-1],[-1,1]].
    M = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    Dxx = np.kron(M, np.kron(M, K1))
    Lap = Dxx + np.kron(M, np.kron(K1, M)) + np.kron(K1, np.kron(M, M))
    Ke = oracle.ref(1).element_matrix(np.eye(3), 0.0, 0.5)
    np.testing.assert_allclose(Ke[:8, :8], 0.5 * (Lap + Dxx), atol=1e-15)


# --------------------------------------------------------------------------
# Operator invariants on the global apply
# --------------------------------------------------------------------------
def _rand_mesh(n=2, seed=3):
    return syn.random_affine_cube(n, seed)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_symmetry_and_positivity(p):
    m = _rand_mesh()
    lam, mu = syn.lame(1.0, 0.3)
    N = m.n_dofs(p)
    rng = np.random.default_rng(p)
    x, y = rng.normal(size=N), rng.normal(size=N)
    Ax = oracle.apply(p, m.nx, m.ny, m.nz, m.affine, lam, mu, x)
    Ay = oracle.apply(p, m.nx, m.ny, m.nz, m.affine, lam, mu, y)
    assert abs(y @ Ax - x @ Ay) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(Ay)
    ess = syn.clamp_mask(m, p)
    xc = np.where(ess, 0.0, x)
    Axc = oracle.apply(p, m.nx, m.ny, m.nz, m.affine, lam, mu, xc, ess=ess)
    assert xc @ Axc > 0


@pytest.mark.parametrize("p", [1, 2, 4])
def test_translations_in_kernel_any_geometry(p):
    m = _rand_mesh(seed=7)
    lam, mu = syn.lame(1.0, 0.45)
    Nn = m.n_nodes(p)
    rng = np.random.default_rng(0)
    scale = np.abs(oracle.apply(p, m.nx, m.ny, m.nz, m.affine, lam, mu, rng.uniform(-1, 1, 3 * Nn))).max()
    for c in range(3):
        t = np.zeros(3 * Nn)
        t[c * Nn:(c + 1) * Nn] = 1.0
        y = oracle.apply(p, m.nx, m.ny, m.nz, m.affine, lam, mu, t)
        assert np.abs(y).max() <= 1e-12 * scale


M_GLOBAL = np.array([[1.3, 0.2, -0.1], [0.1, 0.9, 0.3], [-0.2, 0.15, 1.1]])


@pytest.mark.parametrize("p", [1, 2, 4])
def test_rotations_in_kernel_conforming(p):
    n = 2
    m = syn.globally_affine_mesh(n, n, n, M_GLOBAL, t=(0.3, -0.2, 0.5))
    X = oracle.node_coords_box(n, n, n, p) @ M_GLOBAL.T + np.array([0.3, -0.2, 0.5])
    lam, mu = syn.lame(2.0, 0.3)
    rng = np.random.default_rng(1)
    scale = np.abs(oracle.apply(p, n, n, n, m.affine, lam, mu, rng.uniform(-1, 1, 3 * len(X)))).max()
    for w in np.eye(3):
        u = np.cross(w, X)  # rigid rotation about axis w
        y = oracle.apply(p, n, n, n, m.affine, lam, mu, u.T.reshape(-1))
        assert np.abs(y).max() <= 1e-12 * scale


def _interior_rows(n, p):
    M1 = n * p + 1
    g = np.arange(M1)
    gz, gy, gx = np.meshgrid(g, g, g, indexing="ij")
    inner = ((gx > 0) & (gx < M1 - 1) & (gy > 0) & (gy < M1 - 1) & (gz > 0) & (gz < M1 - 1)).reshape(-1)
    return np.tile(inner, 3)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_patch_test_and_uniform_strain_energy(p):
    n = 3
    m = syn.globally_affine_mesh(n, n, n, M_GLOBAL, t=(0.1, 0.2, 0.3))
    X = oracle.node_coords_box(n, n, n, p) @ M_GLOBAL.T + np.array([0.1, 0.2, 0.3])
    lam, mu = syn.lame(1.0, 0.3)
    Gd = np.array([[0.3, -0.7, 0.2], [0.5, 0.1, -0.4], [0.25, 0.6, -0.2]])
    u = (X @ Gd.T + np.array([0.01, -0.02, 0.03])).T.reshape(-1)
    y = oracle.apply(p, n, n, n, m.affine, lam, mu, u)
    inner = _interior_rows(n, p)
    assert np.abs(y[inner]).max() <= 1e-12 * np.abs(y).max()
    eps = 0.5 * (Gd + Gd.T)
    vol = np.linalg.det(M_GLOBAL)
    energy = vol * (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps))
    assert abs(u @ y - energy) <= 1e-12 * energy


@pytest.mark.parametrize("p", [2, 3, 4])
def test_quadratic_field_integration_by_parts(p):
    # u_c = 1/2 x^T H_c x  =>  div sigma is constant and for interior dofs
    # (A u)_i = -int (div sigma) . phi_i  (no boundary term).
    n = 3
    m = syn.box_mesh(n, n, n, hi=(1.5, 1.0, 0.8))
    X = oracle.node_coords_box(n, n, n, p, hi=(1.5, 1.0, 0.8))
    lam, mu = 0.7, 0.4
    rng = np.random.default_rng(5)
    H = rng.normal(size=(3, 3, 3))
    H = 0.5 * (H + H.transpose(0, 2, 1))
    u = np.stack([0.5 * np.einsum("ni,ij,nj->n", X, H[c], X) for c in range(3)]).reshape(-1)
    # d_j u_i = H_i[j,k] x_k ; div sigma_i = lam d_i div u + mu sum_j (d_j d_j u_i + d_i d_j u_j)
    divsig = np.array([lam * sum(H[k][k][i] for k in range(3))
                       + mu * (np.trace(H[i]) + sum(H[j][i][j] for j in range(3))) for i in range(3)])
    y = oracle.apply(p, n, n, n, m.affine, lam, mu, u)
    F = oracle.load(p, n, n, n, m.affine, f0=-divsig)
    inner = _interior_rows(n, p)
    assert np.abs(y[inner] - F[inner]).max() <= 1e-11 * np.abs(y).max()


def test_linear_in_lame_and_scaling():
    p = 2
    m = _rand_mesh(seed=11)
    x = np.random.default_rng(2).normal(size=m.n_dofs(p))
    a = oracle.apply(p, 2, 2, 2, m.affine, 1.0, 0.0, x)
    b = oracle.apply(p, 2, 2, 2, m.affine, 0.0, 1.0, x)
    c = oracle.apply(p, 2, 2, 2, m.affine, 0.8, 0.3, x)
    np.testing.assert_allclose(c, 0.8 * a + 0.3 * b, atol=1e-12 * np.abs(c).max())
    # single element, J = s I: the stiffness scales like s^(d-2) = s
    one = np.zeros((1, 12))
    one[0, [0, 4, 8]] = 1.0
    two = one.copy()
    two[0, [0, 4, 8]] = 2.5
    x1 = np.random.default_rng(3).normal(size=3 * 27)
    y1 = oracle.apply(p, 1, 1, 1, one, 0.6, 0.9, x1)
    y2 = oracle.apply(p, 1, 1, 1, two, 0.6, 0.9, x1)
    np.testing.assert_allclose(y2, 2.5 * y1, atol=1e-13 * np.abs(y2).max())


# --------------------------------------------------------------------------
# Constraint, sampled rows, diagonal, load, transfers
# --------------------------------------------------------------------------
def test_constraint_semantics_and_rows():
    p = 3
    m = _rand_mesh(seed=4)
    lam, mu = syn.lame(1.0, 0.3)
    ess = syn.clamp_mask(m, p)
    x = syn.uniform_vector(m.n_dofs(p), 9)
    y = oracle.apply(p, 2, 2, 2, m.affine, lam, mu, x, ess=ess)
    e = ess.astype(bool)
    np.testing.assert_array_equal(y[e], x[e])
    x2 = x.copy()
    x2[e] = 123.0
    y2 = oracle.apply(p, 2, 2, 2, m.affine, lam, mu, x2, ess=ess)
    np.testing.assert_array_equal(y2[~e], y[~e])
    # matches the dense constrained matrix
    A = oracle.constrain_dense(oracle.assemble_dense(p, 2, 2, 2, m.affine, lam, mu), ess)
    np.testing.assert_allclose(y, A @ x, atol=1e-12 * np.abs(y).max())
    rows = np.random.default_rng(0).choice(len(x), 200, replace=False)
    yr = oracle.apply_rows(p, 2, 2, 2, m.affine, lam, mu, x, rows, ess=ess)
    np.testing.assert_allclose(yr, y[rows], atol=1e-12 * np.abs(y).max())


@pytest.mark.parametrize("p", [1, 2, 4])
def test_diag_equals_assembled_and_closed_form(p):
    m = syn.random_affine_cube(2, 21)
    lam, mu = syn.lame(3.0, 0.35)
    ess = syn.clamp_mask(m, p)
    d = oracle.diag(p, 2, 2, 2, m.affine, lam, mu, ess=ess)
    A = oracle.assemble_dense(p, 2, 2, 2, m.affine, lam, mu)
    e = ess.astype(bool)
    np.testing.assert_allclose(d[~e], np.diag(A)[~e], rtol=1e-13)
    assert np.all(d[e] == 1.0)
    # closed form from 1D sums (independent numpy tables):
    # diag_(i,c) = sum_e detJ sum_mn [(lam+mu) Ji_mc Ji_nc + mu sum_k Ji_mk Ji_nk] S^i_mn
    Mi, Ci, Ki = (np.diag(a) for a in _numpy_1d_integrals(p))
    D = p + 1
    Nn = m.n_nodes(p)
    dd = np.zeros(3 * Nn)
    Mx = 2 * p + 1
    for el in range(m.ne):
        J = m.affine[el, :9].reshape(3, 3)
        Ji, det = np.linalg.inv(J), np.linalg.det(J)
        ex, ey, ez = el % 2, (el // 2) % 2, el // 4
        for iz in range(D):
            for iy in range(D):
                for ix in range(D):
                    i3 = (ix, iy, iz)
                    S = np.empty((3, 3))
                    for mm in range(3):
                        for nn in range(3):
                            v = 1.0
                            for k in range(3):
                                if k == mm and k == nn:
                                    v *= Ki[i3[k]]
                                elif k == mm or k == nn:
                                    v *= Ci[i3[k]]
                                else:
                                    v *= Mi[i3[k]]
                            S[mm, nn] = v
                    g = (ex * p + ix) + Mx * ((ey * p + iy) + Mx * (ez * p + iz))
                    G = Ji @ Ji.T
                    for c in range(3):
                        coef = (lam + mu) * np.outer(Ji[:, c], Ji[:, c]) + mu * G
                        dd[c * Nn + g] += det * np.sum(coef * S)
    np.testing.assert_allclose(d[~e], dd[~e], rtol=1e-12)


def test_load_partition_of_unity():
    p = 3
    m = _rand_mesh(seed=8)
    f0 = np.array([0.5, -1.0, 2.0])
    F = oracle.load(p, 2, 2, 2, m.affine, f0=f0)
    Nn = m.n_nodes(p)
    vol = sum(np.linalg.det(m.affine[e, :9].reshape(3, 3)) for e in range(m.ne))
    for c in range(3):
        assert abs(F[c * Nn:(c + 1) * Nn].sum() - f0[c] * vol) <= 1e-13 * abs(f0[c] * vol)


def test_load_of_sine_modes_integrates_the_force():
    """A body force of sine modes f_c = amp sin(k . x + phi): the summed load
    of component c (the basis is a partition of unity) is the integral of
    f_c over the box, Im(amp e^{i phi} prod_d (e^{i k_d} - 1) / (i k_d)) on
    [0,1]^3, to the Gauss rule's error (q = 5 points per 0.25-wide
    element, |k| <= 2: far below the tolerance)."""
    p, n = 3, 4
    aff = oracle.box_affine(n, n, n)
    rng = np.random.default_rng(31)
    modes = np.zeros((3, 2, 5))
    modes[..., 0] = rng.uniform(-1, 1, (3, 2))
    modes[..., 1:4] = rng.uniform(0.5, 2.0, (3, 2, 3)) * rng.choice([-1.0, 1.0], (3, 2, 3))
    modes[..., 4] = rng.uniform(0, 2 * np.pi, (3, 2))
    F = oracle.load(p, n, n, n, aff, modes=modes)
    Nn = oracle.n_nodes(n, n, n, p)

    def integral(amp, kx, ky, kz, ph):
        prod = np.exp(1j * ph)
        for k in (kx, ky, kz):
            prod *= (np.exp(1j * k) - 1.0) / (1j * k)
        return amp * prod.imag

    for c in range(3):
        exact = sum(integral(*md) for md in modes[c])
        total = F[c * Nn:(c + 1) * Nn].sum()
        assert abs(total - exact) <= 1e-9 * max(1.0, abs(exact))
        # the check has teeth: a flipped phase or a dropped mode misses it
        flipped = sum(integral(md[0], md[1], md[2], md[3], -md[4]) for md in modes[c])
        assert abs(total - flipped) > 1e-2
        assert abs(total - integral(*modes[c][0])) > 1e-2


@pytest.mark.parametrize("pc,pf", [(1, 2), (2, 4), (4, 8), (1, 3)])
def test_transfer_adjoint_and_polynomial_exactness(pc, pf):
    n = 2
    rng = np.random.default_rng(pc * 10 + pf)
    u = rng.normal(size=3 * oracle.n_nodes(n, n, n, pc))
    v = rng.normal(size=3 * oracle.n_nodes(n, n, n, pf))
    Pu = oracle.prolong(pc, pf, n, n, n, u)
    Rv = oracle.restrict(pc, pf, n, n, n, v)
    assert abs(Pu @ v - u @ Rv) <= 1e-12 * np.linalg.norm(Pu) * np.linalg.norm(v)
    # a global polynomial of degree <= pc in each variable is interpolated exactly
    Xc = oracle.node_coords_box(n, n, n, pc)
    Xf = oracle.node_coords_box(n, n, n, pf)

    def field(X):
        x, y, z = X.T
        return np.stack([x ** pc * y + 0.3, (1 - z) ** pc * x, y ** pc - x * z]).reshape(-1)

    np.testing.assert_allclose(oracle.prolong(pc, pf, n, n, n, field(Xc)), field(Xf), atol=1e-13)


@pytest.mark.parametrize("nx,ny,nz", [(1, 1, 1), (2, 1, 3)])
def test_h_transfer_adjoint_and_trilinear_exactness(nx, ny, nz):
    """One uniform refinement at p = 1 (Sec. 3, h-levels): restriction is the
    exact transpose of prolongation, and a trilinear field on the coarse
    mesh is reproduced exactly at the fine nodes."""
    rng = np.random.default_rng(nx + 10 * ny + 100 * nz)
    u = rng.normal(size=3 * oracle.n_nodes(nx, ny, nz, 1))
    v = rng.normal(size=3 * oracle.n_nodes(2 * nx, 2 * ny, 2 * nz, 1))
    Pu = oracle.prolong_h(nx, ny, nz, u)
    Rv = oracle.restrict_h(nx, ny, nz, v)
    assert abs(Pu @ v - u @ Rv) <= 1e-13 * np.linalg.norm(Pu) * np.linalg.norm(v)
    hi = (2.0, 1.0, 3.0)
    Xc = oracle.node_coords_box(nx, ny, nz, 1, hi=hi)
    Xf = oracle.node_coords_box(2 * nx, 2 * ny, 2 * nz, 1, hi=hi)

    def field(X):
        x, y, z = X.T
        return np.stack([1 + x - 2 * y + 0.5 * x * y * z, x * y - z, 0.3 + y * z + x * z]).reshape(-1)

    np.testing.assert_allclose(oracle.prolong_h(nx, ny, nz, field(Xc)), field(Xf), atol=1e-14)
    # a field quadratic along x is not in the coarse space: interpolation
    # misses it at the odd fine nodes (the check above has teeth)
    q = np.concatenate([Xc[:, 0] ** 2] * 3)
    assert np.max(np.abs(oracle.prolong_h(nx, ny, nz, q) - np.concatenate([Xf[:, 0] ** 2] * 3))) > 1e-3


def test_h_coarse_operator_is_galerkin_product():
    """Nested trilinear spaces, exact Gauss quadrature and a material that
    is constant on each coarse element make the operator rediscretised on
    the coarse mesh equal to P^T A_fine P (the Galerkin product), on a
    globally affine (sheared) domain with two materials."""
    t = (0.3, -0.2, 0.5)
    mc = syn.globally_affine_mesh(2, 1, 2, M_GLOBAL, t=t)
    mf = syn.globally_affine_mesh(4, 2, 4, M_GLOBAL, t=t)
    mat_c = np.array([[3.0, 2.0], [0.5, 0.25], [1.0, 4.0], [2.0, 1.5]])
    ef = np.arange(mf.ne)
    parent = (ef % 4) // 2 + 2 * ((ef // 8) // 2)
    mat_f = mat_c[parent]
    Ac = oracle.assemble_dense(1, 2, 1, 2, mc.affine, 0.0, 0.0, mat=mat_c)
    Af = oracle.assemble_dense(1, 4, 2, 4, mf.affine, 0.0, 0.0, mat=mat_f)
    nc = Ac.shape[0]
    P = np.stack([oracle.prolong_h(2, 1, 2, np.eye(nc)[j]) for j in range(nc)], axis=1)
    G = P.T @ Af @ P
    assert np.max(np.abs(G - Ac)) <= 1e-12 * np.max(np.abs(Ac))
    # a material that is not constant per coarse element breaks the identity
    mat_bad = mat_f.copy()
    mat_bad[0] = [9.0, 9.0]
    Gb = P.T @ oracle.assemble_dense(1, 4, 2, 4, mf.affine, 0.0, 0.0, mat=mat_bad) @ P
    assert np.max(np.abs(Gb - Ac)) > 1e-3 * np.max(np.abs(Ac))


def test_dense_solve_residual():
    p = 2
    m = syn.box_mesh(2, 1, 1, hi=(2.0, 1.0, 1.0))
    lam, mu = syn.lame(1.0, 0.3)
    ess = syn.clamp_mask(m, p)
    b = oracle.load(p, 2, 1, 1, m.affine, f0=(0, 0, -1), ess=ess)
    x = oracle.solve_dense(p, 2, 1, 1, m.affine, lam, mu, b, ess)
    r = b - oracle.apply(p, 2, 1, 1, m.affine, lam, mu, x, ess=ess)
    assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(b)
    assert x[ess.astype(bool)].max() == 0.0


# --------------------------------------------------------------------------
# Per-element material (the PA data D with lambda(alpha, e), mu(alpha, e),
# Sec. 4.5, constant on each element) and the Neumann traction load (Eq. 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("p", [1, 2])
def test_per_element_material_exact(p):
    """Two elements with contrasting materials (a 50:1 contrast as in the
    paper's two-material beam) against the exact-rational brute force; pins
    that element e takes material e."""
    lam, mu = [Fr(50), Fr(1)], [Fr(50), Fr(1)]
    Ax = np.array(exact.global_matrix(p, 2, [J_RAT, J_RAT2], lam, mu), dtype=float)
    aff = np.zeros((2, 12))
    aff[0, :9] = np.array(J_RAT, dtype=float).reshape(9)
    aff[1, :9] = np.array(J_RAT2, dtype=float).reshape(9)
    mat = np.array([[50.0, 50.0], [1.0, 1.0]])
    x = np.random.default_rng(1).uniform(-1, 1, Ax.shape[0])
    y = oracle.apply(p, 2, 1, 1, aff, 0.0, 0.0, x, mat=mat)
    scale = np.abs(Ax).max()
    assert np.max(np.abs(y - Ax @ x)) <= 1e-12 * scale
    # the swapped assignment is a different operator
    y2 = oracle.apply(p, 2, 1, 1, aff, 0.0, 0.0, x, mat=mat[::-1].copy())
    assert np.max(np.abs(y2 - Ax @ x)) > 1e-3 * scale
    # diagonal and selected rows with the same material
    d = oracle.diag(p, 2, 1, 1, aff, 0.0, 0.0, mat=mat)
    assert np.max(np.abs(d - np.diag(Ax))) <= 1e-12 * scale
    rows = np.arange(0, Ax.shape[0], 5)
    yr = oracle.apply_rows(p, 2, 1, 1, aff, 0.0, 0.0, x, rows, mat=mat)
    assert np.max(np.abs(yr - (Ax @ x)[rows])) <= 1e-12 * scale


def test_uniform_material_array_is_the_constant_material():
    p, n = 3, 2
    m = syn.random_affine_cube(n, seed=11)
    x = syn.uniform_vector(m.n_dofs(p), seed=3)
    mat = np.tile([1.7, 0.6], (m.ne, 1))
    assert np.array_equal(oracle.apply(p, n, n, n, m.affine, 1.7, 0.6, x),
                          oracle.apply(p, n, n, n, m.affine, 0.0, 0.0, x, mat=mat))


@pytest.mark.parametrize("p", [1, 3, 4])
@pytest.mark.parametrize("face", [1, 4])
def test_traction_totals_are_the_surface_integrals(p, face):
    """Sum_i F_(i,c) = t_c |Gamma| (the basis sums to 1) and Sum_i F_(i,c)
    y_i = t_c * integral of y over the face (linear fields are reproduced), on
    a box [0,8] x [0,1] x [0,2] with uneven elements along the face."""
    nx, ny, nz = 3, 2, 2
    lo, hi = (0.0, 0.0, 0.0), (8.0, 1.0, 2.0)
    aff = oracle.box_affine(nx, ny, nz, lo, hi)
    t = np.array([0.3, -0.2, -1e-2])
    F = oracle.traction(p, nx, ny, nz, aff, face, t)
    X = oracle.node_coords_box(nx, ny, nz, p, lo, hi)
    Nn = X.shape[0]
    ax = face // 2
    others = [a for a in range(3) if a != ax]
    area = (hi[others[0]] - lo[others[0]]) * (hi[others[1]] - lo[others[1]])
    for c in range(3):
        Fc = F[c * Nn:(c + 1) * Nn]
        assert abs(Fc.sum() - t[c] * area) <= 1e-13 * area
        for a in others:  # first moments: centroid of the face along a
            centroid = 0.5 * (lo[a] + hi[a])
            assert abs((Fc * X[:, a]).sum() - t[c] * area * centroid) <= 1e-12 * area * hi[a]
        # only nodes on the face are loaded
        on_face = np.isclose(X[:, ax], hi[ax] if face % 2 else lo[ax])
        assert np.all(Fc[~on_face] == 0.0)


def test_traction_on_a_sheared_face_uses_the_surface_measure():
    """One element whose x = 1 face is mapped to a parallelogram: the total
    force is t times the parallelogram's area |u x v|."""
    J = np.array([[2.0, 0.0, 0.0], [0.3, 1.5, 0.0], [0.0, 0.4, 0.8]])
    aff = np.zeros((1, 12))
    aff[0, :9] = J.reshape(9)
    F = oracle.traction(2, 1, 1, 1, aff, 1, (0.0, 0.0, 1.0))
    area = np.linalg.norm(np.cross(J[:, 1], J[:, 2]))
    Nn = 27
    assert abs(F[2 * Nn:].sum() - area) <= 1e-14 * area


# --------------------------------------------------------------------------
# Anisotropic material (Eq. 2 with a general C_ijkl; a 6x6 Voigt matrix)
# --------------------------------------------------------------------------
def _iso_voigt(lam, mu):
    Cv = np.zeros((6, 6))
    Cv[:3, :3] = lam
    Cv[[0, 1, 2], [0, 1, 2]] = lam + 2 * mu
    Cv[[3, 4, 5], [3, 4, 5]] = mu
    return Cv


def _spd_voigt(seed):
    rng = np.random.default_rng(seed)
    L = rng.uniform(-1, 1, (6, 6))
    return L @ L.T + 2.0 * np.eye(6)


def test_isotropic_voigt_tensor_is_the_lame_operator():
    p, n = 2, 2
    m = syn.random_affine_cube(n, seed=21)
    x = syn.uniform_vector(m.n_dofs(p), seed=4)
    lam, mu = 1.3, 0.45
    ct = np.tile(oracle.voigt_to_tensor(_iso_voigt(lam, mu)), (m.ne, 1))
    y1 = oracle.apply(p, n, n, n, m.affine, lam, mu, x)
    y2 = oracle.apply(p, n, n, n, m.affine, 0.0, 0.0, x, ctens=ct)
    assert np.max(np.abs(y1 - y2)) <= 1e-13 * np.max(np.abs(y1))


@pytest.mark.parametrize("p", [1, 2])
def test_anisotropic_diagonal_is_the_dense_matrix_diagonal(p):
    """The anisotropic diagonal (closed form from 1D sums, per element
    tensor) equals the diagonal of the matrix assembled densely from the
    element matrices, constrained rows giving 1; with a Lame tensor it is
    the isotropic diagonal."""
    nx, ny, nz = 2, 1, 2
    m = syn.random_affine_cube(nx, seed=30 + p, ny=ny, nz=nz)
    ct = np.stack([oracle.voigt_to_tensor(_spd_voigt(200 + e)) for e in range(m.ne)])
    ess = syn.clamp_mask(m, p)
    d = oracle.diag(p, nx, ny, nz, m.affine, 0.0, 0.0, ess=ess, ctens=ct)
    A = oracle.constrain_dense(oracle.assemble_dense(p, nx, ny, nz, m.affine, 0.0, 0.0, ctens=ct), ess)
    assert np.max(np.abs(d - np.diag(A))) <= 1e-12 * np.max(np.abs(np.diag(A)))
    lam, mu = 0.9, 0.6
    ci = np.tile(oracle.voigt_to_tensor(_iso_voigt(lam, mu)), (m.ne, 1))
    di = oracle.diag(p, nx, ny, nz, m.affine, 0.0, 0.0, ctens=ci)
    dl = oracle.diag(p, nx, ny, nz, m.affine, lam, mu)
    assert np.max(np.abs(di - dl)) <= 1e-13 * np.max(np.abs(dl))


def test_anisotropic_operator_is_symmetric_and_kills_rigid_motions():
    p, n = 3, 2
    m = syn.globally_affine_mesh(n, n, n, M_GLOBAL, t=(0.3, -0.2, 0.5))
    ct = np.stack([oracle.voigt_to_tensor(_spd_voigt(100 + e)) for e in range(m.ne)])
    rng = np.random.default_rng(6)
    x, z = rng.uniform(-1, 1, (2, m.n_dofs(p)))
    Ax = oracle.apply(p, n, n, n, m.affine, 0.0, 0.0, x, ctens=ct)
    Az = oracle.apply(p, n, n, n, m.affine, 0.0, 0.0, z, ctens=ct)
    assert abs(z @ Ax - x @ Az) <= 1e-12 * np.abs(z) @ np.abs(Ax)
    assert x @ Ax > 0
    # translations and infinitesimal rotations u = w x X give zero strain
    X = oracle.node_coords_box(n, n, n, p) @ M_GLOBAL.T + np.array([0.3, -0.2, 0.5])
    Nn = X.shape[0]
    for w in np.eye(3):
        u = np.cross(w, X).T.reshape(-1)
        Au = oracle.apply(p, n, n, n, m.affine, 0.0, 0.0, u, ctens=ct)
        assert np.max(np.abs(Au)) <= 1e-11 * np.max(np.abs(Ax))
    t = np.concatenate([np.ones(Nn), np.zeros(2 * Nn)])
    assert np.max(np.abs(oracle.apply(p, n, n, n, m.affine, 0.0, 0.0, t, ctens=ct))) <= 1e-11 * np.max(np.abs(Ax))


@pytest.mark.parametrize("p", [1, 2])
def test_anisotropic_patch_test_energy(p):
    """u = G X linear: u^T A u = |Omega| eps_V . (C_V eps_V), eps_V with
    engineering shears, on a box [0,2] x [0,1] x [0,3]."""
    nx, ny, nz = 2, 2, 3
    lo, hi = (0.0, 0.0, 0.0), (2.0, 1.0, 3.0)
    aff = oracle.box_affine(nx, ny, nz, lo, hi)
    Cv = _spd_voigt(7)
    ct = np.tile(oracle.voigt_to_tensor(Cv), (nx * ny * nz, 1))
    G = np.random.default_rng(8).uniform(-1, 1, (3, 3))
    X = oracle.node_coords_box(nx, ny, nz, p, lo, hi)
    u = (X @ G.T).T.reshape(-1)
    e = np.array([G[0, 0], G[1, 1], G[2, 2], G[0, 1] + G[1, 0], G[0, 2] + G[2, 0], G[1, 2] + G[2, 1]])
    exact_energy = 6.0 * e @ Cv @ e
    energy = u @ oracle.apply(p, nx, ny, nz, aff, 0.0, 0.0, u, ctens=ct)
    assert abs(energy - exact_energy) <= 1e-12 * abs(exact_energy)


# --------------------------------------------------------------------------
# sparse assembly and the direct solve used to gate the GPU solves
# --------------------------------------------------------------------------
def test_sparse_assembly_equals_matrix_free_apply_and_dense_assembly():
    """The scipy assembly of the element matrices applied to a vector equals
    the element-by-element apply of oracle.c (a separate code path), and the
    dense assembly entry by entry, with per-element material."""
    p, (nx, ny, nz) = 3, (3, 2, 2)
    m = syn.random_affine_cube(nx, seed=41, ny=ny, nz=nz)
    mat = np.random.default_rng(4).uniform(0.5, 5.0, (m.ne, 2))
    A = oracle.assemble_sparse(p, nx, ny, nz, m.affine, 0.0, 0.0, mat=mat)
    x = syn.uniform_vector(m.n_dofs(p), seed=42)
    y = oracle.apply(p, nx, ny, nz, m.affine, 0.0, 0.0, x, mat=mat)
    assert np.max(np.abs(A @ x - y)) <= 1e-13 * np.max(np.abs(y))
    Ad = oracle.assemble_dense(p, nx, ny, nz, m.affine, 0.0, 0.0, mat=mat)
    assert np.max(np.abs(A.toarray() - Ad)) <= 1e-14 * np.max(np.abs(Ad))


@pytest.mark.parametrize("p", [1, 2, 4])
def test_direct_solve_recovers_a_linear_displacement(p):
    """Closed form: on a beam clamped at x = 0, the displacement u = (a x,
    b x, c x) has the uniform strain e_xx = a, e_xy = b/2, e_xz = c/2 and the
    constant stress s = lambda tr(e) I + 2 mu e; its load is the traction
    s n on the five free faces.  It lies in the finite-element space, so the
    solve of the constrained system with that load must return its nodal
    values (a dropped traction face, a wrong sign or a transposed stress
    index misses them by O(1))."""
    nx, ny, nz, hi = 4, 2, 1, (8.0, 1.0, 0.5)
    m = syn.box_mesh(nx, ny, nz, hi=hi)
    lam, mu = syn.lame(1.0, 0.3)
    a, b, c = 1e-2, -2e-2, 3e-2
    sxx, syy, szz, sxy, sxz = (lam + 2 * mu) * a, lam * a, lam * a, mu * b, mu * c
    faces = {1: (sxx, sxy, sxz), 2: (-sxy, -syy, 0.0), 3: (sxy, syy, 0.0), 4: (-sxz, 0.0, -szz),
             5: (sxz, 0.0, szz)}
    ess = syn.clamp_mask(m, p)
    F = sum(oracle.traction(p, nx, ny, nz, m.affine, f, t, ess=ess) for f, t in faces.items())
    x, res = oracle.solve_sparse(p, nx, ny, nz, m.affine, lam, mu, F, ess)
    X = oracle.node_coords_box(nx, ny, nz, p, hi=hi)[:, 0]
    u = np.concatenate([a * X, b * X, c * X])
    # residual at the FP64 floor; the nodal error grows along the clamped
    # beam with its condition number (2e-9 relative at p = 4), far below
    # the O(1) miss of a wrong load or operator
    assert res <= 1e-12
    assert np.max(np.abs(x - u)) <= 1e-8 * np.max(np.abs(u))
