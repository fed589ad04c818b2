"""The library built with every gather and E-vector access bounds-checked
(build.py --bounds; a kernel that meets an index outside its array records it
in the operator's status flags and skips the access, so nothing faults):
every element-kernel variant of both precisions, the batched and
multi-operator launches, the diagonal, the load and a small solve run on
single-element, thin and ragged meshes without a recorded violation, and
their results match the oracle.  This stands in for a memory checker, which
is not available on the GPUs these tests run on.  Runs in a child process
that loads the bounds-checking build."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MESHES = [(1, 1, 1), (2, 1, 1), (1, 3, 2), (3, 2, 1)]
TOL = {0: 1e-12, 1: 1e-5}


def _variants(p, prec):
    if prec == 0:
        return [0, 3] + ([1, 2] if p <= 4 else [])
    v = [0, 1, 2, 3, 6, 7]
    if p <= 6:
        v += [4, 5]
    return v


def _shape(v, p):
    if v == 4:
        return (4, 128 // (p + 2) ** 2, 384)
    return (v, 2, 128 if v != 0 else 256)


def _child():
    sys.path.insert(0, ROOT)
    import oracle
    import paper_2601_08374_gb300 as pa
    import synthetic as syn
    out = {"violations": [], "worst": {}, "runs": 0}
    ops, xs = [], []
    for p in range(1, 9):
        for prec in (0, 1):
            worst = 0.0
            for k, dims in enumerate(MESHES):
                m = syn.random_affine_cube(dims[0], seed=7000 + 10 * p + k, ny=dims[1], nz=dims[2])
                ess = syn.clamp_mask(m, p) if k % 2 else None
                op = pa.Operator(*dims, m.affine, p, 1.1, 0.7, precision=prec, ess_mask=ess)
                x = torch.tensor(syn.uniform_vector(op.ndofs, seed=k + p), dtype=op.dtype, device="cuda")
                yo = oracle.apply(p, *dims, m.affine, 1.1, 0.7, x.double().cpu().numpy(), ess=ess)
                for v in _variants(p, prec):
                    shape = _shape(v, p)
                    try:
                        pa.pa_op_set_launch(op.h, *shape)
                    except pa.PAError:  # two elements per CTA exceed the shared memory at high p
                        pa.pa_op_set_launch(op.h, shape[0], 1, shape[2])
                    y = op.apply(x).double().cpu().numpy()
                    try:
                        pa.pa_op_check(op.h)
                    except pa.PAError as e:
                        out["violations"].append([p, prec, list(dims), v, str(e)])
                    worst = max(worst, float(np.max(np.abs(y - yo)) / np.max(np.abs(yo))))
                    out["runs"] += 1
                pa.pa_op_set_launch(op.h, *((0, 1, 256) if prec == 0 else ((3, 1, 128) if p >= 7 else (5, 1, 128))))
                d = op.diag().double().cpu().numpy()
                do = oracle.diag(p, *dims, m.affine, 1.1, 0.7, ess=ess)
                worst = max(worst, float(np.max(np.abs(d - do)) / np.max(np.abs(do))))
                F = op.rhs(f0=(0.0, 0.0, -1.0)).double().cpu().numpy()
                Fo = oracle.load(p, *dims, m.affine, f0=(0.0, 0.0, -1.0), ess=ess)
                worst = max(worst, float(np.max(np.abs(F - Fo)) / np.max(np.abs(Fo))))
                try:
                    pa.pa_op_check(op.h)
                except pa.PAError as e:
                    out["violations"].append([p, prec, list(dims), "diag/rhs", str(e)])
                ops.append(op)
                xs.append(x)
            out["worst"][f"{p},{prec}"] = worst
    # every operator in one batched call (multi-operator and per-degree launches)
    ys = [torch.empty_like(x) for x in xs]
    pa.pa_op_apply_batch([o.h for o in ops], xs, ys)
    torch.cuda.synchronize()
    for o in ops:
        try:
            pa.pa_op_check(o.h)
        except pa.PAError as e:
            out["violations"].append(["batch", str(e)])
    # a small solve on each precision mode (level operators, transfers, assembly)
    m = syn.box_mesh(4, 2, 2, hi=(8.0, 1.0, 1.0))
    for mode in (0, 1, 2):
        op = pa.Operator(4, 2, 2, m.affine, 4, 1.0, 0.5, ess_mask=syn.clamp_mask(m, 4))
        b = op.rhs(f0=(0.0, 0.0, -1.0))
        s = pa.pa_solver_create_hp(op.h, [4, 2, 1], 1, 4, 1e-2, 10, mode)
        code, info = pa.pa_gmg_pcg_solve(s, b, torch.zeros_like(b), 1e-10, 300)
        out.setdefault("solves", []).append([mode, int(code), info.rel_residual])
        pa.pa_solver_destroy(s)
        try:
            pa.pa_op_check(op.h)
        except pa.PAError as e:
            out["violations"].append(["solve", mode, str(e)])
        op.close()
    for o in ops:
        o.close()
    print("RESULT " + json.dumps(out))


def test_bounds_checked_build_meets_no_out_of_range_index():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import importlib.util
    spec = importlib.util.spec_from_file_location("_pa_build", os.path.join(ROOT, "paper_2601_08374_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    lib = b.build(bounds=True)
    env = dict(os.environ, PA_ELASTICITY_LIB=lib)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--child"], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    assert res["violations"] == [], res["violations"][:5]
    assert res["runs"] > 300
    for key, worst in res["worst"].items():
        prec = int(key.split(",")[1])
        assert worst <= TOL[prec], (key, worst)
    for mode, code, rel in res["solves"]:
        assert code == 0 and rel <= 2e-9, (mode, code, rel)


if __name__ == "__main__" and "--child" in sys.argv:
    _child()
