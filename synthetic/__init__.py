"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds input generation only (meshes, masks, vectors, material
draws).  It contains none of the operator's arithmetic, so both the CUDA
path and the CPU oracle can consume what it produces.

Mesh convention: structured nx*ny*nz grid, element e = ex + nx*(ey + ny*ez),
one affine map per element as 12 doubles (J row-major 3x3, then x0) with
x = x0 + J xi on the reference cell [0,1]^3.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def lame(E: float, nu: float):
    """Lame parameters from Young's modulus and Poisson's ratio."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


@dataclass
class Mesh:
    nx: int
    ny: int
    nz: int
    affine: np.ndarray  # [n_e, 12] float64

    @property
    def ne(self) -> int:
        return self.nx * self.ny * self.nz

    def n_nodes(self, p: int) -> int:
        return (self.nx * p + 1) * (self.ny * p + 1) * (self.nz * p + 1)

    def n_dofs(self, p: int) -> int:
        return 3 * self.n_nodes(p)


def box_mesh(nx, ny, nz, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> Mesh:
    """Undistorted structured grid on the box [lo, hi] (conforming)."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    h = (hi - lo) / np.array([nx, ny, nz], float)
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ex, ey, ez = ex.reshape(-1), ey.reshape(-1), ez.reshape(-1)
    A = np.zeros((nx * ny * nz, 12))
    A[:, 0], A[:, 4], A[:, 8] = h[0], h[1], h[2]
    A[:, 9] = lo[0] + ex * h[0]
    A[:, 10] = lo[1] + ey * h[1]
    A[:, 11] = lo[2] + ez * h[2]
    return Mesh(nx, ny, nz, A)


def globally_affine_mesh(nx, ny, nz, M, t=(0.0, 0.0, 0.0)) -> Mesh:
    """Box mesh on the unit cube pushed through one global affine map
    x -> M x + t (still conforming)."""
    M = np.asarray(M, float)
    base = box_mesh(nx, ny, nz)
    A = np.zeros_like(base.affine)
    for e in range(base.ne):
        J0 = base.affine[e, :9].reshape(3, 3)
        x0 = base.affine[e, 9:]
        A[e, :9] = (M @ J0).reshape(9)
        A[e, 9:] = M @ x0 + np.asarray(t, float)
    return Mesh(nx, ny, nz, A)


def random_affine_cube(n, seed, scale=(0.5, 2.0), shear=0.3, ny=None, nz=None) -> Mesh:
    """n^3 grid on the unit cube where every element gets its own random
    affine map J_e = h * diag(s) * (I + S): s ~ U[scale]^3 and the
    off-diagonal entries of S ~ U[-shear, shear].  x0 is the element's
    corner of the undistorted grid.  Neighbouring elements do not match
    geometrically; the assembled operator is still a sum of SPSD element
    matrices."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed)
    base = box_mesh(n, ny, nz)
    ne = base.ne
    h = np.array([1.0 / n, 1.0 / ny, 1.0 / nz])
    s = rng.uniform(scale[0], scale[1], size=(ne, 3))
    S = rng.uniform(-shear, shear, size=(ne, 3, 3))
    S[:, [0, 1, 2], [0, 1, 2]] = 0.0
    J = (h[None, :, None] * s[:, :, None]) * (np.eye(3)[None] + S)
    A = base.affine.copy()
    A[:, :9] = J.reshape(ne, 9)
    return Mesh(n, ny, nz, A)


def clamp_mask(mesh: Mesh, p: int, face: str = "x0") -> np.ndarray:
    """uint8 essential-dof mask (component-major L-vector) clamping all three
    components of every node on the given face of the structured grid."""
    Mx, My, Mz = mesh.nx * p + 1, mesh.ny * p + 1, mesh.nz * p + 1
    gz, gy, gx = np.meshgrid(np.arange(Mz), np.arange(My), np.arange(Mx), indexing="ij")
    sel = {"x0": gx == 0, "x1": gx == Mx - 1, "y0": gy == 0, "z0": gz == 0}[face].reshape(-1)
    return np.tile(sel, 3).astype(np.uint8)


def uniform_vector(n: int, seed: int, lo=-1.0, hi=1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=n)


def smooth_force_modes(seed: int, n_modes: int = 3, kmax: float = 3.0) -> np.ndarray:
    """[3, n_modes, 5] sine modes (amp, kx, ky, kz, phase) per component:
    f_c(x) = sum_k amp sin(kx x + ky y + kz z + phase), amp ~ U[-1, 1]."""
    rng = np.random.default_rng(seed)
    m = np.zeros((3, n_modes, 5))
    m[..., 0] = rng.uniform(-1.0, 1.0, size=(3, n_modes))
    m[..., 1:4] = rng.uniform(-kmax, kmax, size=(3, n_modes, 3)) * np.pi
    m[..., 4] = rng.uniform(0.0, 2.0 * np.pi, size=(3, n_modes))
    return m


def sweep_n(p: int, target_cube_root: float = 99.0) -> int:
    """Cube edge n for the ~3M-dof operator sweep: round(99/p), ties to even
    (p = 1, 2, 4, 6, 8 -> 99, 50, 25, 16, 12)."""
    return int(np.round(target_cube_root / p))


def mixed_n(p: int, target_dofs: float = 8e6) -> int:
    """Cube edge n for the ~8M-dof mixed-precision solves."""
    return int(np.round((np.cbrt(target_dofs / 3.0) - 1.0) / p))


SWEEP_P = (1, 2, 4, 6, 8)


def two_material(mesh: Mesh, split_x: float, inner=(50.0, 50.0), outer=(1.0, 1.0)):
    """Per-element material [ne, 2] (lambda_e, mu_e) of a two-material body:
    elements whose centre lies at x < split_x take ``inner``, the others
    ``outer`` (the paper's benchmark: lambda = mu = 50 and lambda = mu = 1, a
    50:1 stiffness contrast)."""
    A = mesh.affine
    centre_x = A[:, 9] + 0.5 * (A[:, 0] + A[:, 1] + A[:, 2])
    mat = np.empty((mesh.ne, 2))
    mat[centre_x < split_x] = inner
    mat[centre_x >= split_x] = outer
    return mat
