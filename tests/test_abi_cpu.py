"""The C-ABI library loads on a machine without a GPU, exports every symbol that
include/dugks.h declares, and rejects invalid arguments before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1411_6121_gb300 import dugks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dugks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dugks_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert sorted(dugks.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol():
    lib = dugks.load()
    for name in _declared():
        assert hasattr(lib, name), name


def _create(**kw):
    lib = dugks.load()
    args = dict(dim=2, nx=8, ny=8, nz=1, dx=1.0, q=9, nu=0.1, dt=0.5, rt=1.0 / 3.0, bcs=None)
    args.update(kw)
    m = dugks.Mesh(args["dim"], args["nx"], args["ny"], args["nz"], args["dx"])
    keep = []
    for ax, fa in enumerate(args.get("faces") or []):
        if fa is not None:
            keep.append(np.ascontiguousarray(fa, dtype=np.float64))
            m.faces[ax] = keep[-1].ctypes.data_as(C.POINTER(C.c_double))
    f = dugks.Force()
    b = dugks.make_bcs(args["bcs"])
    o = dugks.Opts()
    lib.dugks_opts_default(C.byref(o))
    o.rt = args["rt"]
    o.model = args.get("model", 0)
    o.store = args.get("store", 0)
    h = C.c_void_p()
    rc = lib.dugks_create(C.byref(m), args["q"], args["nu"], args["dt"], C.byref(f), C.byref(b), C.byref(o), C.byref(h))
    return rc, h, lib.dugks_last_error(None).decode()


def test_cfl_violation_rejected():
    # Sec. 3: dt = a dx / sqrt(3RT); a > 1 is rejected before any device work
    rc, h, msg = _create(dt=1.01)
    assert rc == -2 and not h.value and "CFL" in msg


@pytest.mark.parametrize("kw", [dict(dim=4), dict(q=19), dict(dim=3, q=9, nz=4), dict(nx=0), dict(nu=-1.0),
                                dict(bcs=[(1, (0, 0, 0), 0.0), (0, (0, 0, 0), 0.0)]),
                                dict(nx=1, bcs=[(1, (0, 0, 0), 0.0), (1, (0, 0, 0), 0.0)]),
                                dict(bcs=[(4, (0, 0, 0), 0.0), (4, (0, 0, 0), 0.0)]), dict(model=2)])
def test_invalid_arguments_rejected(kw):
    rc, h, msg = _create(**kw)
    assert rc in (-1, -7) and not h.value and msg


_TANH8 = np.array([0.0, 0.3, 0.9, 2.0, 4.0, 6.0, 7.1, 7.7, 8.0])  # 8 cells, widths 0.3 .. 2


@pytest.mark.parametrize("kw,code", [
    # a non-uniform mesh (Sec. 3.4) takes F32 or F64 storage; its coordinates increase; a 2D
    # mesh has no z coordinates
    (dict(dim=3, q=19, nz=8, dt=0.1, store=1, faces=[None, None, _TANH8]), -7),
    (dict(dim=3, q=27, nz=8, dt=0.1, faces=[None, None, _TANH8[::-1].copy()]), -1),
    (dict(dt=0.1, faces=[None, None, _TANH8]), -1),
    (dict(store=1, dt=0.1, faces=[None, _TANH8]), -7),
    (dict(store=2, dt=0.1, faces=[_TANH8]), -7),
    (dict(dt=0.1, faces=[None, _TANH8[::-1].copy()]), -1),
    # the CFL condition takes the smallest width: 0.3 / sqrt(3 RT) = 0.3 (also along z)
    (dict(dt=0.31, faces=[None, _TANH8]), -2),
    (dict(dim=3, q=19, nz=8, dt=0.31, faces=[None, None, _TANH8]), -2),
])
def test_nonuniform_mesh_arguments_rejected(kw, code):
    rc, h, msg = _create(**kw)
    assert rc == code and not h.value and msg


def test_null_handle_calls_fail_cleanly():
    lib = dugks.load()
    assert lib.dugks_step(None, 1) == -1
    assert lib.dugks_init(None, None, None) == -1
    assert lib.dugks_sync(None, 0.1) == -1
    lib.dugks_destroy(None)


def test_header_constants_match_binding():
    src = open(os.path.join(ROOT, "include", "dugks.h")).read()
    consts = dict((k, int(v)) for k, v in re.findall(r"#define DUGKS_(BC_[A-Z_]+|STORE_[A-Z0-9_]+)\s+(-?\d+)", src))
    for name, value in consts.items():
        assert getattr(dugks, name) == value, name


def _batch_create(count=2, faces=None, store=0, model=0, dt=0.5, bc_type=None):
    lib = dugks.load()
    meshes = (dugks.Mesh * count)()
    nus = (C.c_double * count)()
    forces = (dugks.Force * count)()
    bcs = (dugks.Boundaries * count)()
    keep = []
    for i in range(count):
        meshes[i] = dugks.Mesh(2, 16, 8, 1, 1.0)
        nus[i] = 0.05
        bcs[i] = dugks.make_bcs([(0, (0, 0, 0), 0.0), (0, (0, 0, 0), 0.0),
                                 (bc_type if bc_type is not None else 1, (0, 0, 0), 0.0), (1, (0.05, 0, 0), 0.0)])
    if faces is not None:
        keep.append(np.ascontiguousarray(faces, dtype=np.float64))
        meshes[count - 1].faces[1] = keep[-1].ctypes.data_as(C.POINTER(C.c_double))
    o = dugks.Opts()
    lib.dugks_opts_default(C.byref(o))
    o.store, o.model = store, model
    h = C.c_void_p()
    rc = lib.dugks_batch_create(count, meshes, C.cast(nus, C.POINTER(C.c_double)), dt, forces, bcs, C.byref(o),
                                C.byref(h))
    return rc, h, lib.dugks_batch_last_error(None).decode()


@pytest.mark.parametrize("kw,code", [
    (dict(faces=np.linspace(0.0, 8.0, 9)), -7),   # graded meshes are not batched
    (dict(model=1), -7),                           # the batch runs the incompressible model
    (dict(store=3), -7),                           # F32/BF16/F16 storage only
    (dict(dt=1.01), -2),                           # CFL
    (dict(bc_type=0), -1),                         # a periodic face paired with a wall
    (dict(count=0), -1),
])
def test_batch_arguments_rejected(kw, code):
    rc, h, msg = _batch_create(**kw)
    assert rc == code and not h.value and msg


def test_product_package_never_imports_the_oracle():
    """The oracle is test infrastructure: no module of the package imports it (the CUDA path
    has no CPU fallback)."""
    import ast
    pkg = os.path.join(ROOT, "paper_1411_6121_gb300")
    for name in sorted(os.listdir(pkg)):
        if not name.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(pkg, name)).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            else:
                continue
            assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), (name, mods)


def test_missing_library_fails_loudly():
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-c",
                        "from paper_1411_6121_gb300 import dugks; dugks.load('/nonexistent/libdugks.so')"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0 and "OSError" in r.stderr
