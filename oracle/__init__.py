"""Plain FP64 CPU oracle of the high-order linear-elasticity operator
(arXiv 2601.08374, Sec. 2.1 Eq. 1-6 and Sec. 4.3-4.4 for what is computed).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA product path never calls it and shares no code with it.

The heavy lifting is in ``oracle.c`` (plain C, OpenMP over elements); this
module only marshals numpy arrays through ctypes.  ``oracle.exact`` holds an
exact-rational brute force of the element matrix for p = 1, 2.

Mesh convention: structured nx*ny*nz grid, element e = ex + nx*(ey + ny*ez),
one affine map per element given as 12 doubles (J row-major, then x0) with
x = x0 + J xi on the reference cell [0,1]^3.  L-vectors are component-major,
length 3*Nn with Nn = (nx p+1)(ny p+1)(nz p+1), node index x fastest.
"""
from __future__ import annotations

import ctypes
import functools
import os

import numpy as np

from . import build as _build

_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64p = ctypes.POINTER(ctypes.c_int64)


@functools.lru_cache(maxsize=None)
def _lib():
    path = _build.build()
    lib = ctypes.CDLL(path)
    lib.orc_gauss01.argtypes = [ctypes.c_int, _dp, _dp]
    lib.orc_gll01.argtypes = [ctypes.c_int, _dp]
    lib.orc_lagrange.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp]
    lib.orc_ref_create.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.orc_ref_create.restype = ctypes.c_void_p
    lib.orc_ref_destroy.argtypes = [ctypes.c_void_p]
    lib.orc_ref_tables.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp, _dp]
    lib.orc_ref_blocks.argtypes = [ctypes.c_void_p, _dp]
    lib.orc_element_coeff.argtypes = [_dp, ctypes.c_double, ctypes.c_double, _dp, _dp]
    lib.orc_element_matrix.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, ctypes.c_double, _dp]
    lib.orc_element_matrix_t.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
    common = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, _u8p]
    lib.orc_apply.argtypes = common + [_dp, _dp, ctypes.c_int]
    lib.orc_apply_rows.argtypes = common + [_dp, ctypes.c_int64, _i64p, _dp, ctypes.c_int]
    lib.orc_diag.argtypes = common + [_dp, ctypes.c_int]
    common_m = common[:7] + [_dp, _dp, _u8p]
    lib.orc_apply_m.argtypes = common_m + [_dp, _dp, ctypes.c_int]
    lib.orc_apply_rows_m.argtypes = common_m + [_dp, ctypes.c_int64, _i64p, _dp, ctypes.c_int]
    lib.orc_diag_m.argtypes = common_m + [_dp, ctypes.c_int]
    lib.orc_traction.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp,
                                 _u8p, _dp]
    lib.orc_load.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp,
                             ctypes.c_int, _dp, _u8p, _dp, ctypes.c_int]
    lib.orc_prolong.argtypes = [ctypes.c_int] * 5 + [_dp, _dp]
    lib.orc_restrict.argtypes = [ctypes.c_int] * 5 + [_dp, _dp]
    lib.orc_box_affine.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
    lib.orc_max_threads.restype = ctypes.c_int
    return lib


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _mask(ess):
    if ess is None:
        return None
    return np.ascontiguousarray(ess, dtype=np.uint8)


def max_threads() -> int:
    return int(_lib().orc_max_threads())


def gauss01(q: int):
    """Gauss-Legendre rule with q points on [0,1] (points ascending)."""
    pts, wts = np.zeros(q), np.zeros(q)
    if _lib().orc_gauss01(q, _d(pts), _d(wts)):
        raise ValueError("bad q")
    return pts, wts


def gll01(p: int):
    """The p+1 Gauss-Lobatto-Legendre nodes on [0,1]."""
    x = np.zeros(p + 1)
    if _lib().orc_gll01(p, _d(x)):
        raise ValueError("bad p")
    return x


def lagrange(nodes, x):
    """Barycentric Lagrange basis on ``nodes``: (val, der), each [n, m]."""
    nodes, x = _f64(nodes), _f64(np.atleast_1d(x))
    n, m = len(nodes), len(x)
    val, der = np.zeros((n, m)), np.zeros((n, m))
    if _lib().orc_lagrange(n, _d(nodes), m, _d(x), _d(val), _d(der)):
        raise ValueError("bad nodes")
    return val, der


class Ref:
    """Reference data for one (p, q): 1D rules, B/G tables, dense S_mn blocks."""

    def __init__(self, p: int, q: int = 0):
        self.p = p
        self.q = q if q > 0 else p + 2
        self.D = p + 1
        self.Q = self.q
        self._h = _lib().orc_ref_create(p, self.q)
        if not self._h:
            raise ValueError(f"unsupported p={p} q={q}")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib().orc_ref_destroy(h)
            self._h = None

    def tables(self):
        D, Q = self.D, self.Q
        gll, gp, gw = np.zeros(D), np.zeros(Q), np.zeros(Q)
        B, G = np.zeros((D, Q)), np.zeros((D, Q))
        _lib().orc_ref_tables(self._h, _d(gll), _d(gp), _d(gw), _d(B), _d(G))
        return dict(gll=gll, gp=gp, gw=gw, B=B, G=G)

    def blocks(self):
        D3 = self.D ** 3
        S = np.zeros((9, D3, D3))
        _lib().orc_ref_blocks(self._h, _d(S))
        return S.reshape(3, 3, D3, D3)

    def element_matrix(self, J, lam: float, mu: float):
        D3 = self.D ** 3
        K = np.zeros((3 * D3, 3 * D3))
        if _lib().orc_element_matrix(self._h, _d(_f64(J).reshape(9)), lam, mu, _d(K)):
            raise ValueError("detJ <= 0")
        return K

    def element_matrix_t(self, J, C4):
        """Element matrix of an anisotropic tensor C4 (81 values, C_cjdl)."""
        D3 = self.D ** 3
        K = np.zeros((3 * D3, 3 * D3))
        if _lib().orc_element_matrix_t(self._h, _d(_f64(J).reshape(9)), _d(_f64(C4).reshape(81)), _d(K)):
            raise ValueError("detJ <= 0")
        return K


@functools.lru_cache(maxsize=16)
def ref(p: int, q: int = 0) -> Ref:
    return Ref(p, q)


def element_coeff(J, lam, mu):
    C, det = np.zeros(81), np.zeros(1)
    if _lib().orc_element_coeff(_d(_f64(J).reshape(9)), lam, mu, _d(C), _d(det)):
        raise ValueError("detJ <= 0")
    return C.reshape(3, 3, 3, 3), float(det[0])


def n_nodes(nx, ny, nz, p):
    return (nx * p + 1) * (ny * p + 1) * (nz * p + 1)


def _check_mesh(nx, ny, nz, affine):
    affine = _f64(affine)
    if affine.shape != (nx * ny * nz, 12):
        raise ValueError("affine must be [n_e, 12]")
    return affine


def _material(mat, ne):
    """Per-element material [ne, 2] = (lambda_e, mu_e), or None."""
    if mat is None:
        return None
    mat = _f64(mat)
    if mat.shape != (ne, 2):
        raise ValueError("material must be [ne, 2] (lambda_e, mu_e)")
    return mat


def _tensor(ctens, ne):
    """Per-element anisotropic tensor [ne, 81] (C_cjdl), or None."""
    if ctens is None:
        return None
    ctens = _f64(ctens).reshape(ne, 81)
    return np.ascontiguousarray(ctens)


def voigt_to_tensor(Cv):
    """Full tensor C_ijkl (81, index ((i*3 + j)*3 + k)*3 + l) of a 6x6 Voigt
    matrix in the order [00, 11, 22, 01, 02, 12] with engineering shear
    strains (sigma_V = Cv eps_V, eps_V = [e00, e11, e22, 2 e01, 2 e02, 2 e12])."""
    Cv = _f64(Cv).reshape(6, 6)
    v = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]
    C = np.zeros(81)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C[((i * 3 + j) * 3 + k) * 3 + l] = Cv[v[i][j], v[k][l]]
    return C


def apply(p, nx, ny, nz, affine, lam, mu, x, ess=None, q=0, nthreads=0, mat=None, ctens=None):
    """y = A x (constrained operator when ``ess`` is given).  ``mat``: per
    element (lambda_e, mu_e) [ne, 2] in place of the constants lam, mu;
    ``ctens``: per-element anisotropic tensors [ne, 81] (takes precedence)."""
    r = ref(p, q)
    affine = _check_mesh(nx, ny, nz, affine)
    x = _f64(x)
    N = 3 * n_nodes(nx, ny, nz, p)
    if x.shape != (N,):
        raise ValueError("x has wrong length")
    y = np.zeros(N)
    m = _mask(ess)
    mt = _material(mat, nx * ny * nz)
    ct = _tensor(ctens, nx * ny * nz)
    rc = _lib().orc_apply_m(r._h, nx, ny, nz, _d(affine), lam, mu, _d(mt), _d(ct),
                            m.ctypes.data_as(_u8p) if m is not None else None, _d(x), _d(y), nthreads)
    if rc:
        raise RuntimeError(f"orc_apply failed ({rc})")
    return y


def apply_rows(p, nx, ny, nz, affine, lam, mu, x, rows, ess=None, q=0, nthreads=0, mat=None, ctens=None):
    """Selected entries (L-vector indices ``rows``) of y = A x."""
    r = ref(p, q)
    affine = _check_mesh(nx, ny, nz, affine)
    x = _f64(x)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros(len(rows))
    m = _mask(ess)
    mt = _material(mat, nx * ny * nz)
    ct = _tensor(ctens, nx * ny * nz)
    rc = _lib().orc_apply_rows_m(r._h, nx, ny, nz, _d(affine), lam, mu, _d(mt), _d(ct),
                                 m.ctypes.data_as(_u8p) if m is not None else None, _d(x),
                                 len(rows), rows.ctypes.data_as(_i64p), _d(out), nthreads)
    if rc:
        raise RuntimeError(f"orc_apply_rows failed ({rc})")
    return out


def diag(p, nx, ny, nz, affine, lam, mu, ess=None, q=0, nthreads=0, mat=None, ctens=None):
    r = ref(p, q)
    affine = _check_mesh(nx, ny, nz, affine)
    d = np.zeros(3 * n_nodes(nx, ny, nz, p))
    m = _mask(ess)
    mt = _material(mat, nx * ny * nz)
    ct = _tensor(ctens, nx * ny * nz)
    rc = _lib().orc_diag_m(r._h, nx, ny, nz, _d(affine), lam, mu, _d(mt), _d(ct),
                           m.ctypes.data_as(_u8p) if m is not None else None, _d(d), nthreads)
    if rc:
        raise RuntimeError(f"orc_diag failed ({rc})")
    return d


def load(p, nx, ny, nz, affine, f0=(0.0, 0.0, 0.0), modes=None, ess=None, q=0, nthreads=0):
    """Load vector of the body force f(x) = f0 + sum of sine modes.

    ``modes`` is [3, K, 5] with (amp, kx, ky, kz, phase) per mode."""
    r = ref(p, q)
    affine = _check_mesh(nx, ny, nz, affine)
    f0 = _f64(f0).reshape(3)
    if modes is None:
        modes = np.zeros((3, 0, 5))
    modes = _f64(modes)
    K = modes.shape[1]
    F = np.zeros(3 * n_nodes(nx, ny, nz, p))
    m = _mask(ess)
    rc = _lib().orc_load(r._h, nx, ny, nz, _d(affine), _d(f0), K, _d(modes.reshape(-1)) if K else None,
                         m.ctypes.data_as(_u8p) if m is not None else None, _d(F), nthreads)
    if rc:
        raise RuntimeError(f"orc_load failed ({rc})")
    return F


def traction(p, nx, ny, nz, affine, face, t, ess=None, q=0):
    """Load vector of a constant traction ``t`` (3,) on one face of the box:
    face = 2 * axis + side (axis x/y/z = 0/1/2, side 0 = low, 1 = high)."""
    r = ref(p, q)
    affine = _check_mesh(nx, ny, nz, affine)
    F = np.zeros(3 * n_nodes(nx, ny, nz, p))
    m = _mask(ess)
    rc = _lib().orc_traction(r._h, nx, ny, nz, _d(affine), int(face), _d(_f64(t).reshape(3)),
                             m.ctypes.data_as(_u8p) if m is not None else None, _d(F))
    if rc:
        raise RuntimeError(f"orc_traction failed ({rc})")
    return F


def prolong(pc, pf, nx, ny, nz, xc):
    xc = _f64(xc)
    xf = np.zeros(3 * n_nodes(nx, ny, nz, pf))
    if _lib().orc_prolong(pc, pf, nx, ny, nz, _d(xc), _d(xf)):
        raise RuntimeError("orc_prolong failed")
    return xf


def restrict(pc, pf, nx, ny, nz, rf):
    rf = _f64(rf)
    rc = np.zeros(3 * n_nodes(nx, ny, nz, pc))
    if _lib().orc_restrict(pc, pf, nx, ny, nz, _d(rf), _d(rc)):
        raise RuntimeError("orc_restrict failed")
    return rc


def _h_matrix_1d(n):
    """[2n+1, n+1] matrix of one uniform refinement of n linear elements:
    row i holds the coarse nodal basis (GLL p = 1, barycentric Lagrange)
    evaluated at fine node i, which lies at reference coordinate
    (i - 2E) / 2 of coarse element E = min(i // 2, n - 1)."""
    nodes = gll01(1)
    P = np.zeros((2 * n + 1, n + 1))
    for i in range(2 * n + 1):
        E = min(i // 2, n - 1)
        val, _ = lagrange(nodes, [(i - 2 * E) / 2.0])
        P[i, E:E + 2] = val[:, 0]
    return P


def prolong_h(nx, ny, nz, xc):
    """h-prolongation (Sec. 3, natural injection for h-refined levels): the
    p = 1 field on the nx*ny*nz coarse mesh evaluated at the nodes of its
    uniform refinement (2nx*2ny*2nz elements).  Component-major L-vectors."""
    Px, Py, Pz = _h_matrix_1d(nx), _h_matrix_1d(ny), _h_matrix_1d(nz)
    xc = _f64(xc).reshape(3, nz + 1, ny + 1, nx + 1)
    return np.einsum("ia,jb,kc,dcba->dkji", Px, Py, Pz, xc).reshape(-1)


def restrict_h(nx, ny, nz, rf):
    """Transpose of ``prolong_h`` (nx, ny, nz: the coarse element counts)."""
    Px, Py, Pz = _h_matrix_1d(nx), _h_matrix_1d(ny), _h_matrix_1d(nz)
    rf = _f64(rf).reshape(3, 2 * nz + 1, 2 * ny + 1, 2 * nx + 1)
    return np.einsum("ia,jb,kc,dkji->dcba", Px, Py, Pz, rf).reshape(-1)


def box_affine(nx, ny, nz, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    A = np.zeros((nx * ny * nz, 12))
    _lib().orc_box_affine(nx, ny, nz, _d(_f64(lo)), _d(_f64(hi)), _d(A))
    return A


def node_coords_box(nx, ny, nz, p, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Physical coordinates [Nn, 3] of the nodes of an undistorted box mesh."""
    g = gll01(p)
    axes = []
    for n, a, b in zip((nx, ny, nz), lo, hi):
        h = (b - a) / n
        c = [a + e * h + h * g[i] for e in range(n) for i in range(p)] + [b]
        axes.append(np.array(c))
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)


def assemble_dense(p, nx, ny, nz, affine, lam, mu, q=0, mat=None, ctens=None):
    """Global (unconstrained) stiffness matrix of a small mesh, assembled
    from the oracle's element matrices (``mat``: per-element material)."""
    r = ref(p, q)
    affine = _check_mesh(nx, ny, nz, affine)
    D = p + 1
    D3 = D ** 3
    Mx, My = nx * p + 1, ny * p + 1
    Nn = n_nodes(nx, ny, nz, p)
    A = np.zeros((3 * Nn, 3 * Nn))
    loc = np.arange(D3)
    ix, iy, iz = loc % D, (loc // D) % D, loc // (D * D)
    for e in range(nx * ny * nz):
        ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
        gn = (ex * p + ix) + Mx * ((ey * p + iy) + My * (ez * p + iz))
        dofs = np.concatenate([c * Nn + gn for c in range(3)])
        if ctens is not None:
            A[np.ix_(dofs, dofs)] += r.element_matrix_t(affine[e, :9], np.asarray(ctens, dtype=np.float64).reshape(-1, 81)[e])
            continue
        le, me = (lam, mu) if mat is None else (float(mat[e][0]), float(mat[e][1]))
        A[np.ix_(dofs, dofs)] += r.element_matrix(affine[e, :9], le, me)
    return A


def constrain_dense(A, ess):
    """Matrix of the constrained operator: ess rows/columns replaced by identity."""
    ess = np.asarray(ess, dtype=bool)
    Ac = A.copy()
    Ac[ess, :] = 0.0
    Ac[:, ess] = 0.0
    Ac[ess, ess] = 1.0
    return Ac


def solve_dense(p, nx, ny, nz, affine, lam, mu, b, ess, q=0, mat=None, ctens=None):
    """Direct FP64 solve of the constrained system (small meshes only)."""
    A = constrain_dense(assemble_dense(p, nx, ny, nz, affine, lam, mu, q, mat=mat, ctens=ctens), ess)
    return np.linalg.solve(A, _f64(b))


def assemble_sparse(p, nx, ny, nz, affine, lam, mu, q=0, mat=None):
    """Global (unconstrained) stiffness matrix as a scipy CSR matrix, summed
    from the oracle's element matrices (Eq. 3-5 element by element; the same
    sums as ``assemble_dense`` without the dense storage), for meshes whose
    matrix fits in host memory (config-size beams: ~65M entries)."""
    import scipy.sparse as sp
    r = ref(p, q)
    affine = _check_mesh(nx, ny, nz, affine)
    D = p + 1
    D3 = D ** 3
    Mx, My = nx * p + 1, ny * p + 1
    Nn = n_nodes(nx, ny, nz, p)
    loc = np.arange(D3)
    ix, iy, iz = loc % D, (loc // D) % D, loc // (D * D)
    ne = nx * ny * nz
    nloc = 3 * D3
    rows = np.empty((ne, nloc * nloc), dtype=np.int64)
    cols = np.empty((ne, nloc * nloc), dtype=np.int64)
    vals = np.empty((ne, nloc * nloc))
    for e in range(ne):
        ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
        gn = (ex * p + ix) + Mx * ((ey * p + iy) + My * (ez * p + iz))
        dofs = np.concatenate([c * Nn + gn for c in range(3)])
        le, me = (lam, mu) if mat is None else (float(mat[e][0]), float(mat[e][1]))
        vals[e] = r.element_matrix(affine[e, :9], le, me).reshape(-1)
        rows[e] = np.repeat(dofs, nloc)
        cols[e] = np.tile(dofs, nloc)
    A = sp.coo_matrix((vals.reshape(-1), (rows.reshape(-1), cols.reshape(-1))), shape=(3 * Nn, 3 * Nn)).tocsr()
    A.sum_duplicates()
    return A


def solve_sparse(p, nx, ny, nz, affine, lam, mu, b, ess, q=0, mat=None, refine=1):
    """FP64 solve of the constrained system A_c x = b (Sec. 2.1 with the
    essential rows and columns of the constrained operator replaced by the
    identity) by a sparse LU factorisation of the assembled matrix, then
    ``refine`` steps of iterative refinement whose residual b - A_c x is
    taken with the oracle's element-by-element apply.  Returns (x, relative
    residual ||b - A_c x|| / ||b||)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    A = assemble_sparse(p, nx, ny, nz, affine, lam, mu, q, mat=mat)
    essb = np.asarray(ess, dtype=bool)
    keep = sp.diags(np.where(essb, 0.0, 1.0))
    Ac = (keep @ A @ keep + sp.diags(essb.astype(np.float64))).tocsc()
    del A
    b = _f64(b)
    lu = spl.splu(Ac, permc_spec="MMD_AT_PLUS_A")
    del Ac
    x = lu.solve(b)
    for _ in range(refine + 1):
        res = b - apply(p, nx, ny, nz, affine, lam, mu, x, ess=ess, q=q, mat=mat)
        if _ == refine:
            break
        x = x + lu.solve(res)
    nb = np.linalg.norm(b)
    return x, (float(np.linalg.norm(res) / nb) if nb > 0 else 0.0)
