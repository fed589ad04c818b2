"""Python binding of the GB300 matrix-free PA elasticity library.

Thin ctypes marshalling over the C ABI declared in ``include/pa_elasticity.h``
(same function names).  Every step of the operator and the solver runs in the
library's CUDA kernels; this module only passes pointers, sizes and streams.
PyTorch provides device memory and streams.

Importing this package fails loudly if ``libpa_elasticity.so`` has not been
built (``python paper_2601_08374_gb300/build.py``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH

PA_OK, PA_EINVAL, PA_ENOMEM, PA_ECUDA, PA_ENOTCONV, PA_EBREAKDOWN, PA_ETIMEOUT, PA_EBUSY, PA_ECANCELED = range(9)
PA_FP64, PA_FP32 = 0, 1
PA_FMA_FP32X2 = 2  # pa_measure_fma_rate: FP32 on paired FMA instructions
PA_GEOMETRY_STORED, PA_GEOMETRY_UA = 0, 1
PA_SOLVE_FP64, PA_SOLVE_MIXED, PA_SOLVE_MIXED_FCG = 0, 1, 2

# PA_ELASTICITY_LIB selects another build of the same library (the tests'
# bounds-checking build); the default is the in-tree product build
_LIB_PATH = os.environ.get("PA_ELASTICITY_LIB", _LIB_PATH)
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with `python paper_2601_08374_gb300/build.py`")

lib = ctypes.CDLL(_LIB_PATH)

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)


class pa_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("b_norm", ctypes.c_double), ("inner_iterations", ctypes.c_int), ("refinements", ctypes.c_int),
                ("lambda_max", ctypes.c_double * 8), ("coarse_iterations", ctypes.c_int),
                ("tolerance_met", ctypes.c_int)]


PA_REQUEST_MAX_MODES = 16


class pa_request(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("box", ctypes.c_double * 6),
                ("p", ctypes.c_int), ("E", ctypes.c_double), ("nu", ctypes.c_double), ("f0", ctypes.c_double * 3),
                ("nmodes", ctypes.c_int), ("modes", ctypes.c_double * (3 * PA_REQUEST_MAX_MODES * 5)),
                ("clamp_x0", ctypes.c_int), ("rtol", ctypes.c_double), ("maxit", ctypes.c_int), ("mode", ctypes.c_int),
                ("keep_solution", ctypes.c_int)]


class pa_request_timing(ctypes.Structure):
    _fields_ = [("latency_s", ctypes.c_double), ("queue_s", ctypes.c_double), ("setup_s", ctypes.c_double),
                ("solve_s", ctypes.c_double), ("footprint_bytes", ctypes.c_int64), ("batched", ctypes.c_int),
                ("levels", ctypes.c_int), ("h_levels", ctypes.c_int)]


class pa_server_stats_t(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("running", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("used_bytes", ctypes.c_int64), ("peak_used_bytes", ctypes.c_int64), ("batched", ctypes.c_int64),
                ("batch_ticks", ctypes.c_int64), ("batch_member_ticks", ctypes.c_int64),
                ("batch_max_members", ctypes.c_int64)]


def _sig(name, args, res=ctypes.c_int):
    f = getattr(lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("pa_last_error", [], ctypes.c_char_p)
_sig("pa_version", [])
_sig("pa_lame", [ctypes.c_double, ctypes.c_double, _dp, _dp])
_sig("pa_mesh_create", [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.POINTER(_vp)])
_sig("pa_mesh_destroy", [_vp])
_sig("pa_op_setup", [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                     ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(_vp)])
_sig("pa_op_destroy", [_vp])
_sig("pa_op_info", [_vp, _i64p, _i64p, _ip, _ip])
_sig("pa_op_apply", [_vp, _vp, _vp, _vp])
_sig("pa_op_apply_add", [_vp, _vp, _vp, _vp])
_sig("pa_op_apply_host", [_vp, _vp, _vp, _vp])
_sig("pa_op_apply_host_batch", [_vp, _vp, _vp, ctypes.c_int, _vp])
_sig("pa_op_apply_batch", [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int, _vp])
_sig("pa_op_diag", [_vp, _vp, _vp])
_sig("pa_op_rhs", [_vp, _dp, ctypes.c_int, _dp, _vp, _vp])
_sig("pa_op_set_material", [_vp, _dp])
_sig("pa_op_set_anisotropic", [_vp, _dp])
_sig("pa_op_check", [_vp])
_sig("pa_op_set_wait_limit", [_vp, ctypes.c_double])
_sig("pa_op_apply_stage", [_vp, ctypes.c_int, _vp, _vp, _vp])
_sig("pa_op_traction", [_vp, ctypes.c_int, _dp, _vp, _vp])
_sig("pa_op_assemble_p1", [_vp, _vp, _vp])
_sig("pa_op_prolong", [_vp, _vp, _vp, _vp, _vp])
_sig("pa_op_restrict", [_vp, _vp, _vp, _vp, _vp])
_sig("pa_apply_noalloc", [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                          ctypes.c_int, _vp, _vp, _vp, _vp, _vp])
_sig("pa_measure_fma_rate", [ctypes.c_int, _dp, _vp])
_sig("pa_op_set_launch", [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int])
_sig("pa_op_set_geometry_mode", [_vp, ctypes.c_int])
_sig("pa_op_get_launch", [_vp, _ip, _ip, _ip])
_sig("pa_op_autotune", [_vp, _vp])
_sig("pa_op_profile", [_vp, ctypes.c_int])
_sig("pa_op_profile_read", [_vp, _dp, _dp, _i64p])
_sig("pa_server_create", [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_vp)])
_sig("pa_server_submit", [_vp, ctypes.POINTER(pa_request), _i64p])
_sig("pa_server_poll", [_vp, ctypes.c_int64, _ip])
_sig("pa_server_wait", [_vp, ctypes.c_int64, _dp, ctypes.c_int64, ctypes.POINTER(pa_solve_info),
                        ctypes.POINTER(pa_request_timing)])
_sig("pa_server_stats", [_vp, ctypes.POINTER(pa_server_stats_t)])
_sig("pa_server_cancel", [_vp, ctypes.c_int64])
_sig("pa_server_destroy", [_vp])
_sig("pa_server_set_option", [_vp, ctypes.c_int, ctypes.c_double])
if hasattr(lib, "pa_solver_create"):
    _sig("pa_solver_create", [_vp, ctypes.c_int, _ip, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                              ctypes.POINTER(_vp)])
    _sig("pa_solver_create_hp", [_vp, ctypes.c_int, _ip, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_int, ctypes.POINTER(_vp)])
    _sig("pa_solver_destroy", [_vp])
    _sig("pa_solver_set_option", [_vp, ctypes.c_int, ctypes.c_double])
    _sig("pa_gmg_pcg_solve", [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(pa_solve_info), _vp])
    _sig("pa_gmg_pcg_solve_batch", [_vp, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(pa_solve_info), _vp])


class PAError(RuntimeError):
    def __init__(self, code, where):
        msg = lib.pa_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


def _check(code, where):
    if code != PA_OK:
        raise PAError(code, where)
    return code


def _dptr(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(_dp)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _tptr(t):
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- C names --
def pa_version() -> int:
    return lib.pa_version()


def pa_lame(E: float, nu: float):
    lam, mu = ctypes.c_double(), ctypes.c_double()
    _check(lib.pa_lame(E, nu, ctypes.byref(lam), ctypes.byref(mu)), "pa_lame")
    return lam.value, mu.value


def pa_mesh_create(nx, ny, nz, box=None, affine=None):
    h = _vp()
    aff = None if affine is None else np.ascontiguousarray(affine, dtype=np.float64)
    if aff is not None and aff.shape != (nx * ny * nz, 12):
        raise ValueError("affine must be [n_e, 12]")
    bx = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
    _check(lib.pa_mesh_create(nx, ny, nz, _dptr(bx), _dptr(aff), ctypes.byref(h)), "pa_mesh_create")
    return h


def pa_mesh_destroy(h):
    lib.pa_mesh_destroy(h)


def pa_op_setup(mesh, p, q, lam, mu, precision, ess_mask=None):
    h = _vp()
    m = None
    if ess_mask is not None:
        m = np.ascontiguousarray(ess_mask, dtype=np.uint8)
    _check(lib.pa_op_setup(mesh, p, q, lam, mu, precision,
                           m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if m is not None else None,
                           ctypes.byref(h)), "pa_op_setup")
    return h


def pa_op_destroy(h):
    lib.pa_op_destroy(h)


def pa_op_info(op):
    n, ne, p, prec = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
    _check(lib.pa_op_info(op, ctypes.byref(n), ctypes.byref(ne), ctypes.byref(p), ctypes.byref(prec)), "pa_op_info")
    return n.value, ne.value, p.value, prec.value


def pa_op_apply(op, x, y, stream=None):
    _check(lib.pa_op_apply(op, _tptr(x), _tptr(y), _stream_ptr(stream)), "pa_op_apply")


def pa_op_apply_add(op, x, y, stream=None):
    """y += A x."""
    _check(lib.pa_op_apply_add(op, _tptr(x), _tptr(y), _stream_ptr(stream)), "pa_op_apply_add")


def pa_op_apply_batch(ops, xs, ys, stream=None):
    """One batched apply of several operators (lists of handles / tensors)."""
    n = len(ops)
    ha = (_vp * n)(*[o.value if isinstance(o, ctypes.c_void_p) else o for o in ops])
    xa = (_vp * n)(*[x.data_ptr() for x in xs])
    ya = (_vp * n)(*[y.data_ptr() for y in ys])
    _check(lib.pa_op_apply_batch(ha, xa, ya, n, _stream_ptr(stream)), "pa_op_apply_batch")


def pa_op_apply_host(op, x_host, y_host, stream=None):
    """x_host, y_host: CPU tensors (pinned for full bandwidth) or numpy arrays."""
    xp = ctypes.c_void_p(x_host.data_ptr() if hasattr(x_host, "data_ptr") else x_host.ctypes.data)
    yp = ctypes.c_void_p(y_host.data_ptr() if hasattr(y_host, "data_ptr") else y_host.ctypes.data)
    _check(lib.pa_op_apply_host(op, xp, yp, _stream_ptr(stream)), "pa_op_apply_host")


def _host_ptr(a):
    return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data


def pa_op_apply_host_batch(ops, xs_host, ys_host, stream=None):
    """Several operators from host buffers, copies overlapped with the applies."""
    n = len(ops)
    ha = (_vp * n)(*[o.value if isinstance(o, ctypes.c_void_p) else o for o in ops])
    xa = (_vp * n)(*[_host_ptr(x) for x in xs_host])
    ya = (_vp * n)(*[_host_ptr(y) for y in ys_host])
    _check(lib.pa_op_apply_host_batch(ha, xa, ya, n, _stream_ptr(stream)), "pa_op_apply_host_batch")


def pa_op_diag(op, d, stream=None):
    _check(lib.pa_op_diag(op, _tptr(d), _stream_ptr(stream)), "pa_op_diag")


def pa_op_rhs(op, F, f0=(0.0, 0.0, 0.0), modes=None, stream=None):
    f0 = np.ascontiguousarray(f0, dtype=np.float64).reshape(3)
    nm = 0
    md = None
    if modes is not None:
        md = np.ascontiguousarray(modes, dtype=np.float64)
        nm = md.shape[1]
    _check(lib.pa_op_rhs(op, _dptr(f0), nm, _dptr(md) if nm else None, _tptr(F), _stream_ptr(stream)), "pa_op_rhs")


def pa_op_assemble_p1(op, vals, stream=None):
    _check(lib.pa_op_assemble_p1(op, _tptr(vals), _stream_ptr(stream)), "pa_op_assemble_p1")


def pa_op_prolong(coarse, fine, xc, xf, stream=None):
    _check(lib.pa_op_prolong(coarse, fine, _tptr(xc), _tptr(xf), _stream_ptr(stream)), "pa_op_prolong")


def pa_op_restrict(coarse, fine, rf, rc, stream=None):
    _check(lib.pa_op_restrict(coarse, fine, _tptr(rf), _tptr(rc), _stream_ptr(stream)), "pa_op_restrict")


def _noalloc_arg(name, t, dtype, numel, shape=None):
    """Checks one tensor argument of pa_apply_noalloc (the C side has no
    handle to compare sizes against, so a wrong tensor would be read or
    written out of bounds on the device)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"pa_apply_noalloc: {name} must be a torch tensor")
    if t.dtype != dtype:
        raise ValueError(f"pa_apply_noalloc: {name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != shape:
        raise ValueError(f"pa_apply_noalloc: {name} must have shape {shape}, got {tuple(t.shape)}")
    if t.numel() != numel:
        raise ValueError(f"pa_apply_noalloc: {name} must have {numel} entries, got {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"pa_apply_noalloc: {name} must be contiguous")


def pa_apply_noalloc(nx, ny, nz, p, lam, mu, precision, affine, x, y, ess_mask=None, stream=None):
    """Allocation-free apply; affine [nx*ny*nz, 12] float64, x, y (L-vectors
    of ``precision``) and ess_mask (uint8, one entry per dof) are contiguous
    CUDA tensors.  Raises ValueError for a tensor of the wrong dtype, shape,
    layout or device before calling the library."""
    import torch
    if precision not in (PA_FP64, PA_FP32):
        raise ValueError("pa_apply_noalloc: precision must be PA_FP64 or PA_FP32")
    if min(nx, ny, nz) < 1 or not 1 <= p <= 8:
        raise ValueError("pa_apply_noalloc: need nx, ny, nz >= 1 and 1 <= p <= 8")
    ne = nx * ny * nz
    ndofs = 3 * (nx * p + 1) * (ny * p + 1) * (nz * p + 1)
    vt = torch.float64 if precision == PA_FP64 else torch.float32
    _noalloc_arg("affine", affine, torch.float64, 12 * ne, (ne, 12))
    _noalloc_arg("x", x, vt, ndofs)
    _noalloc_arg("y", y, vt, ndofs)
    if ess_mask is not None:
        _noalloc_arg("ess_mask", ess_mask, torch.uint8, ndofs)
    for name, t in (("affine", affine), ("x", x), ("y", y), ("ess_mask", ess_mask)):
        if t is not None and not t.is_cuda:
            raise ValueError(f"pa_apply_noalloc: {name} must be on a CUDA device")
    _check(lib.pa_apply_noalloc(nx, ny, nz, p, lam, mu, precision, _tptr(affine),
                                _tptr(ess_mask) if ess_mask is not None else None, _tptr(x), _tptr(y),
                                _stream_ptr(stream)), "pa_apply_noalloc")


def pa_op_apply_stage(op, stage, x, y, stream=None):
    """y = A x by one stage of the optimisation stack (0 baseline, 1 + sum
    factorisation, 2 + Voigt, 3 + fusion = the production apply)."""
    _check(lib.pa_op_apply_stage(op, int(stage), _tptr(x), _tptr(y), _stream_ptr(stream)), "pa_op_apply_stage")


def pa_op_set_material(op, mat):
    """Per-element material, [ne, 2] (lambda_e, mu_e); None restores the constant one."""
    if mat is None:
        _check(lib.pa_op_set_material(op, None), "pa_op_set_material")
        return
    m = np.ascontiguousarray(mat, dtype=np.float64)
    _check(lib.pa_op_set_material(op, m.ctypes.data_as(_dp)), "pa_op_set_material")


def pa_op_check(op):
    """Raises PAError(PA_ETIMEOUT) when a bounded tensor-core wait of an apply timed out."""
    _check(lib.pa_op_check(op), "pa_op_check")


def pa_op_set_wait_limit(op, seconds):
    """Budget (s) of the operator's bounded device waits (tensor-core variant)."""
    _check(lib.pa_op_set_wait_limit(op, float(seconds)), "pa_op_set_wait_limit")


def pa_op_set_anisotropic(op, cvoigt):
    """Per-element symmetric 6x6 Voigt matrices [ne, 6, 6]; None restores the isotropic material."""
    if cvoigt is None:
        _check(lib.pa_op_set_anisotropic(op, None), "pa_op_set_anisotropic")
        return
    c = np.ascontiguousarray(cvoigt, dtype=np.float64)
    _check(lib.pa_op_set_anisotropic(op, c.ctypes.data_as(_dp)), "pa_op_set_anisotropic")


def pa_op_traction(op, face, t, F, stream=None):
    tt = np.ascontiguousarray(t, dtype=np.float64).reshape(3)
    _check(lib.pa_op_traction(op, int(face), tt.ctypes.data_as(_dp), _tptr(F), _stream_ptr(stream)),
           "pa_op_traction")


def pa_measure_fma_rate(precision, stream=None):
    """Measured FMA rate of the CUDA cores (TFLOP/s) for PA_FP64 / PA_FP32,
    or FP32 on paired FMA instructions (PA_FMA_FP32X2)."""
    t = ctypes.c_double()
    _check(lib.pa_measure_fma_rate(precision, ctypes.byref(t), _stream_ptr(stream)), "pa_measure_fma_rate")
    return t.value


def pa_op_set_launch(op, variant, elems_per_block, threads):
    _check(lib.pa_op_set_launch(op, variant, elems_per_block, threads), "pa_op_set_launch")


def pa_op_set_geometry_mode(op, mode):
    """PA_GEOMETRY_STORED (stored per-element records) or PA_GEOMETRY_UA
    (J only; J^-1 and detJ recomputed in the FP32 plane kernel)."""
    _check(lib.pa_op_set_geometry_mode(op, mode), "pa_op_set_geometry_mode")


def pa_op_get_launch(op):
    v, e, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib.pa_op_get_launch(op, ctypes.byref(v), ctypes.byref(e), ctypes.byref(t)), "pa_op_get_launch")
    return v.value, e.value, t.value


def pa_op_autotune(op, stream=None):
    _check(lib.pa_op_autotune(op, _stream_ptr(stream)), "pa_op_autotune")
    return pa_op_get_launch(op)


def pa_op_profile(op, enable: bool):
    _check(lib.pa_op_profile(op, 1 if enable else 0), "pa_op_profile")


def pa_op_profile_read(op):
    """(element_ms, assemble_ms, applies) summed over the recorded applies."""
    te, ta, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(lib.pa_op_profile_read(op, ctypes.byref(te), ctypes.byref(ta), ctypes.byref(n)), "pa_op_profile_read")
    return te.value, ta.value, n.value


def pa_solver_create(op, p_levels, cheb_order=4, coarse_rtol=1e-4, coarse_maxit=300, mode=PA_SOLVE_FP64):
    h = _vp()
    lv = (ctypes.c_int * len(p_levels))(*p_levels)
    _check(lib.pa_solver_create(op, len(p_levels), lv, cheb_order, coarse_rtol, coarse_maxit, mode,
                                ctypes.byref(h)), "pa_solver_create")
    return h


def pa_solver_create_hp(op, p_levels, h_levels, cheb_order=4, coarse_rtol=1e-4, coarse_maxit=300,
                        mode=PA_SOLVE_FP64):
    """p-levels on the operator's mesh, then `h_levels` p = 1 levels on meshes
    coarsened by two per direction (uniform refinement undone)."""
    h = _vp()
    lv = (ctypes.c_int * len(p_levels))(*p_levels)
    _check(lib.pa_solver_create_hp(op, len(p_levels), lv, h_levels, cheb_order, coarse_rtol, coarse_maxit, mode,
                                   ctypes.byref(h)), "pa_solver_create_hp")
    return h


PA_SOLVER_OPT_GRAPHS = 1
PA_SOLVER_OPT_PERSISTENT_COARSE = 2
PA_SOLVER_OPT_COARSE_HMG = 3
PA_SOLVER_OPT_CHEB_LOWER = 4
PA_SOLVER_OPT_CHEB_UPPER = 5
PA_SOLVER_OPT_POWER_ITERS = 6
PA_SOLVER_OPT_WAIT_LIMIT = 7
PA_SOLVER_OPT_INJECT_INNER_FAILURE = 8
PA_SOLVER_OPT_CHEB_KIND = 9


def pa_solver_set_option(h, option, value):
    _check(lib.pa_solver_set_option(h, option, value), "pa_solver_set_option")


def pa_solver_destroy(h):
    lib.pa_solver_destroy(h)


def pa_gmg_pcg_solve(solver, b, x, rtol=1e-10, maxit=500, stream=None):
    info = pa_solve_info()
    code = lib.pa_gmg_pcg_solve(solver, _tptr(b), _tptr(x), rtol, maxit, ctypes.byref(info), _stream_ptr(stream))
    if code not in (PA_OK, PA_ENOTCONV, PA_EBREAKDOWN):
        raise PAError(code, "pa_gmg_pcg_solve")
    return code, info


def pa_gmg_pcg_solve_batch(solvers, bs, xs, rtol=1e-10, maxit=500, stream=None):
    """Lockstep solve of several systems with batched operator applies;
    returns (first status, [info per solve])."""
    n = len(solvers)
    ha = (_vp * n)(*[s.value if isinstance(s, ctypes.c_void_p) else s for s in solvers])
    ba = (_vp * n)(*[b.data_ptr() for b in bs])
    xa = (_vp * n)(*[x.data_ptr() for x in xs])
    infos = (pa_solve_info * max(n, 1))()
    code = lib.pa_gmg_pcg_solve_batch(ha, ba, xa, n, rtol, maxit, infos, _stream_ptr(stream))
    if code not in (PA_OK, PA_ENOTCONV, PA_EBREAKDOWN):
        raise PAError(code, "pa_gmg_pcg_solve_batch")
    return code, [infos[k] for k in range(n)]


def make_request(nx, ny, nz, box, p, E, nu, f0=(0.0, 0.0, 0.0), modes=None, clamp_x0=True, rtol=1e-10, maxit=1000,
                 mode=PA_SOLVE_MIXED, keep_solution=False):
    r = pa_request()
    r.nx, r.ny, r.nz, r.p, r.E, r.nu = nx, ny, nz, p, E, nu
    for i in range(6):
        r.box[i] = float(box[i])
    for i in range(3):
        r.f0[i] = float(f0[i])
    if modes is not None:
        m = np.ascontiguousarray(modes, dtype=np.float64)
        r.nmodes = m.shape[1]
        if r.nmodes > PA_REQUEST_MAX_MODES:
            raise ValueError("too many modes")
        flat = m.reshape(-1)
        for i, v in enumerate(flat):
            r.modes[i] = float(v)
    r.clamp_x0, r.rtol, r.maxit, r.mode, r.keep_solution = int(bool(clamp_x0)), rtol, maxit, mode, int(bool(keep_solution))
    return r


def pa_server_create(budget_bytes, max_slots):
    h = _vp()
    _check(lib.pa_server_create(int(budget_bytes), max_slots, ctypes.byref(h)), "pa_server_create")
    return h


def pa_server_submit(srv, req):
    t = ctypes.c_int64()
    _check(lib.pa_server_submit(srv, ctypes.byref(req), ctypes.byref(t)), "pa_server_submit")
    return t.value


def pa_server_poll(srv, ticket):
    d = ctypes.c_int()
    _check(lib.pa_server_poll(srv, ticket, ctypes.byref(d)), "pa_server_poll")
    return bool(d.value)


def pa_server_wait(srv, ticket, x_len=0):
    """Returns (status, info, timing, x or None)."""
    info, tm = pa_solve_info(), pa_request_timing()
    x = np.empty(x_len) if x_len else None
    code = lib.pa_server_wait(srv, ticket, x.ctypes.data_as(_dp) if x is not None else None, x_len,
                              ctypes.byref(info), ctypes.byref(tm))
    if code == PA_EINVAL:
        raise PAError(code, "pa_server_wait")
    return code, info, tm, x


PA_SERVER_OPT_BATCH = 1
PA_SERVER_OPT_BATCH_MAX_DOFS = 2
PA_SERVER_OPT_BATCH_MAX_MEMBERS = 3
PA_SERVER_OPT_H_LEVELS = 4


def pa_server_set_option(srv, option, value):
    _check(lib.pa_server_set_option(srv, option, float(value)), "pa_server_set_option")


def pa_server_cancel(srv, ticket):
    """Cancel a queued or running request (collect it with pa_server_wait)."""
    _check(lib.pa_server_cancel(srv, ticket), "pa_server_cancel")


def pa_server_stats(srv):
    st = pa_server_stats_t()
    _check(lib.pa_server_stats(srv, ctypes.byref(st)), "pa_server_stats")
    return st


def pa_server_destroy(srv):
    lib.pa_server_destroy(srv)


# ------------------------------------------------------- object wrappers --
class Operator:
    """Owns a mesh + operator handle; vectors are torch CUDA tensors."""

    def __init__(self, nx, ny, nz, affine, p, lam, mu, precision=PA_FP64, ess_mask=None, q=0, mat=None, cvoigt=None):
        import torch
        self._mesh = pa_mesh_create(nx, ny, nz, affine=affine)
        try:
            self.h = pa_op_setup(self._mesh, p, q, lam, mu, precision, ess_mask)
        finally:
            pa_mesh_destroy(self._mesh)
            self._mesh = None
        self.ndofs, self.nelem, self.p, self.precision = pa_op_info(self.h)
        self.dtype = torch.float64 if precision == PA_FP64 else torch.float32
        if mat is not None:
            pa_op_set_material(self.h, mat)
        if cvoigt is not None:
            pa_op_set_anisotropic(self.h, cvoigt)

    def close(self):
        if getattr(self, "h", None):
            pa_op_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        # at interpreter exit the module's globals may already be gone
        try:
            self.close()
        except Exception:
            pass

    def empty(self):
        import torch
        return torch.empty(self.ndofs, dtype=self.dtype, device="cuda")

    def apply(self, x, y=None, stream=None):
        if y is None:
            y = self.empty()
        pa_op_apply(self.h, x, y, stream)
        return y

    def diag(self, stream=None):
        d = self.empty()
        pa_op_diag(self.h, d, stream)
        return d

    def rhs(self, f0=(0.0, 0.0, 0.0), modes=None, stream=None, traction=None):
        """Load vector of the body force; ``traction`` = (face, t) adds a
        constant traction on one box face."""
        F = self.empty()
        pa_op_rhs(self.h, F, f0, modes, stream)
        if traction is not None:
            pa_op_traction(self.h, traction[0], traction[1], F, stream)
        return F
