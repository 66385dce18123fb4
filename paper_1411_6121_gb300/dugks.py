"""Thin Python binding of ``libdugks.so`` (the C ABI in ``include/dugks.h``).

Argument marshalling only: every step of the scheme runs in the library's CUDA kernels.
The entry points keep the C names (``dugks_create``, ``dugks_step``, ...); ``Sim`` wraps a
handle for convenience. PyTorch supplies streams and device buffers where a caller wants
device-resident outputs. Loading fails loudly when the library has not been built or no
CUDA device is present: there is no CPU fallback.
"""
import ctypes as C
import os

import numpy as np

from . import _build

DUGKS_OK = 0
ERRORS = {
    -1: "DUGKS_E_INVAL", -2: "DUGKS_E_CFL", -3: "DUGKS_E_NOMEM", -4: "DUGKS_E_CUDA",
    -5: "DUGKS_E_UNSTABLE", -6: "DUGKS_E_TIMEOUT", -7: "DUGKS_E_UNSUPPORTED",
}
D2Q9, D3Q19, D3Q27 = 9, 19, 27
STORE_F32, STORE_BF16, STORE_F16, STORE_F64 = 0, 1, 2, 3
BC_PERIODIC, BC_NEQ_VELOCITY, BC_NEQ_PRESSURE, BC_BOUNCE_BACK = 0, 1, 2, 3
MODEL_INCOMPRESSIBLE, MODEL_ORIGINAL = 0, 1

LIB_PATH = _build.LIB

# Every symbol declared in include/dugks.h (checked by the CPU test suite).
EXPORTS = [
    "dugks_opts_default", "dugks_create", "dugks_init", "dugks_step", "dugks_moments",
    "dugks_residual", "dugks_state_bytes", "dugks_get_state", "dugks_set_state",
    "dugks_get_clock", "dugks_set_clock", "dugks_set_force_field", "dugks_sync",
    "dugks_launch_count", "dugks_last_error", "dugks_destroy", "dugks_residual_static",
    "dugks_set_boundaries", "dugks_record", "dugks_adjoint", "dugks_adjoint_async", "dugks_adjoint_wall",
    "dugks_batch_create", "dugks_batch_init", "dugks_batch_step", "dugks_batch_moments", "dugks_batch_tune",
    "dugks_batch_sync", "dugks_batch_launch_count", "dugks_batch_last_error", "dugks_batch_destroy",
]


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64), ("dx", C.c_double),
                ("faces", C.POINTER(C.c_double) * 3)]


class FaceBC(C.Structure):
    _fields_ = [("type", C.c_int32), ("u", C.c_double * 3), ("p", C.c_double), ("p_amp", C.c_double)]


class Boundaries(C.Structure):
    _fields_ = [("face", FaceBC * 6)]


class Force(C.Structure):
    _fields_ = [("g", C.c_double * 3), ("omega", C.c_double), ("field", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("rt", C.c_double), ("rho0", C.c_double), ("store", C.c_int32), ("stream", C.c_void_p),
                ("use_graph", C.c_int32), ("tile_x", C.c_int32), ("tile_y", C.c_int32), ("kernel", C.c_int32),
                ("model", C.c_int32)]


class DugksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


_lib = None


def load(path=None):
    """Load ``libdugks.so`` (building it first if the sources are newer). Raises if the
    library cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path) or not _build.up_to_date():
        _build.build()
    lib = C.CDLL(path)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)
    lib.dugks_opts_default.argtypes = [C.POINTER(Opts)]
    lib.dugks_create.argtypes = [C.POINTER(Mesh), I32, C.c_double, C.c_double, C.POINTER(Force),
                                 C.POINTER(Boundaries), C.POINTER(Opts), C.POINTER(P)]
    lib.dugks_init.argtypes = [P, D, D]
    lib.dugks_step.argtypes = [P, I64]
    lib.dugks_moments.argtypes = [P, P, I32]
    lib.dugks_residual.argtypes = [P, D]
    lib.dugks_state_bytes.argtypes = [P, C.POINTER(C.c_size_t)]
    lib.dugks_get_state.argtypes = [P, P, C.c_size_t, I32]
    lib.dugks_set_state.argtypes = [P, P, C.c_size_t, I32]
    lib.dugks_get_clock.argtypes = [P, C.POINTER(C.c_int64), D]
    lib.dugks_set_clock.argtypes = [P, I64]
    lib.dugks_set_force_field.argtypes = [P, P]
    lib.dugks_sync.argtypes = [P, C.c_double]
    lib.dugks_launch_count.argtypes = [P]
    lib.dugks_launch_count.restype = I64
    lib.dugks_last_error.argtypes = [P]
    lib.dugks_last_error.restype = C.c_char_p
    lib.dugks_destroy.argtypes = [P]
    lib.dugks_destroy.restype = None
    lib.dugks_set_boundaries.argtypes = [P, C.POINTER(Boundaries)]
    lib.dugks_record.argtypes = [P, I64, I32]
    lib.dugks_adjoint.argtypes = [P, P, P, D, P]
    lib.dugks_adjoint_async.argtypes = [P, P, P, P]
    lib.dugks_adjoint_wall.argtypes = [P, D]
    lib.dugks_residual_static.argtypes = [I32, I32, P, I64, I64, I64, C.c_double, C.c_double, D, P, P, I32, D, P]
    lib.dugks_batch_create.argtypes = [I32, C.POINTER(Mesh), D, C.c_double, C.POINTER(Force), C.POINTER(Boundaries),
                                       C.POINTER(Opts), C.POINTER(P)]
    lib.dugks_batch_init.argtypes = [P, I32, D, D]
    lib.dugks_batch_step.argtypes = [P, I64]
    lib.dugks_batch_moments.argtypes = [P, I32, P, I32]
    lib.dugks_batch_tune.argtypes = [P, C.POINTER(I32), C.POINTER(I32)]
    lib.dugks_batch_sync.argtypes = [P]
    lib.dugks_batch_launch_count.argtypes = [P]
    lib.dugks_batch_launch_count.restype = I64
    lib.dugks_batch_last_error.argtypes = [P]
    lib.dugks_batch_last_error.restype = C.c_char_p
    lib.dugks_batch_destroy.argtypes = [P]
    lib.dugks_batch_destroy.restype = None
    _lib = lib
    return lib


def _check(rc, h=None):
    if rc != DUGKS_OK:
        msg = load().dugks_last_error(h).decode(errors="replace")
        raise DugksError(rc, msg)


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def make_bcs(bcs):
    """6 tuples (type, (ux, uy, uz), p[, p_amp]) in the order -x, +x, -y, +y, -z, +z
    (missing entries periodic; p_amp: amplitude of an oscillating wall pressure)."""
    b = Boundaries()
    bcs = list(bcs or [])
    bcs += [(BC_PERIODIC, (0.0, 0.0, 0.0), 0.0)] * (6 - len(bcs))
    for w, bc in enumerate(bcs[:6]):
        t, u, p = bc[:3]
        b.face[w].type = int(t)
        for a in range(3):
            b.face[w].u[a] = float(u[a]) if a < len(u) else 0.0
        b.face[w].p = float(p)
        b.face[w].p_amp = float(bc[3]) if len(bc) > 3 else 0.0
    return b


class Sim:
    """One simulation handle (see ``include/dugks.h``)."""

    def __init__(self, shape, q, nu, dt, dx=1.0, rt=1.0 / 3.0, rho0=1.0, g=(0.0, 0.0, 0.0), omega=0.0,
                 bcs=None, field=None, store=STORE_F32, stream=None, use_graph=True, tile=None, kernel=0,
                 model=MODEL_INCOMPRESSIBLE, faces=None):
        lib = load()
        self.lib = lib
        dim = len(shape)
        self.dim, self.q = dim, int(q)
        self.shape = tuple(int(s) for s in shape)
        self.ncell = int(np.prod(self.shape))
        m = Mesh(dim, self.shape[0], self.shape[1], self.shape[2] if dim == 3 else 1, float(dx))
        face_arrays = []  # non-uniform mesh: interface coordinates per axis (copied by create)
        for a, fa in enumerate(list(faces or [])[:3]):
            if fa is not None:
                arr = np.ascontiguousarray(fa, dtype=np.float64)
                face_arrays.append(arr)
                m.faces[a] = arr.ctypes.data_as(C.POINTER(C.c_double))
        f = Force()
        for a in range(3):
            f.g[a] = float(g[a]) if a < len(g) else 0.0
        f.omega = float(omega)
        self._field = field  # keep a reference: the handle reads it every step
        f.field = None if field is None else int(field.data_ptr())
        o = Opts()
        lib.dugks_opts_default(C.byref(o))
        o.rt, o.rho0, o.store = float(rt), float(rho0), int(store)
        o.stream = None if stream is None else int(stream)
        o.use_graph = 1 if use_graph else 0
        if tile:
            o.tile_x, o.tile_y = int(tile[0]), int(tile[1])
        o.kernel = int(kernel)
        o.model = int(model)
        self.bcs = make_bcs(bcs)
        h = C.c_void_p()
        rc = lib.dugks_create(C.byref(m), int(q), float(nu), float(dt), C.byref(f), C.byref(self.bcs), C.byref(o),
                              C.byref(h))
        _check(rc, None)
        self.h = h
        self.store = int(store)
        self.rt, self.rho0, self.dt = float(rt), float(rho0), float(dt)

    def close(self):
        if getattr(self, "h", None):
            self.lib.dugks_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def init(self, p=None, u=None):
        p = None if p is None else np.ascontiguousarray(p, dtype=np.float64).ravel()
        u = None if u is None else np.ascontiguousarray(u, dtype=np.float64).ravel()
        if p is not None:
            assert p.size == self.ncell
        if u is not None:
            assert u.size == self.dim * self.ncell
        _check(self.lib.dugks_init(self.h, _dp(p), _dp(u)), self.h)

    def step(self, n=1):
        _check(self.lib.dugks_step(self.h, int(n)), self.h)

    def moments(self, out=None):
        """Host numpy [dim+1][ncell] (p, u...) or, with a CUDA torch tensor ``out``, fills it."""
        if out is not None:
            _check(self.lib.dugks_moments(self.h, C.c_void_p(out.data_ptr()), 1), self.h)
            return out
        a = np.zeros((self.dim + 1, self.ncell), dtype=np.float32)
        _check(self.lib.dugks_moments(self.h, a.ctypes.data_as(C.c_void_p), 0), self.h)
        return a

    def residual(self):
        out = np.zeros(2 + self.dim)
        _check(self.lib.dugks_residual(self.h, _dp(out)), self.h)
        return out

    def state_bytes(self):
        n = C.c_size_t()
        _check(self.lib.dugks_state_bytes(self.h, C.byref(n)), self.h)
        return n.value

    def _dtype(self):
        return {STORE_F32: np.float32, STORE_BF16: np.uint16, STORE_F16: np.float16, STORE_F64: np.float64}[self.store]

    def get_state(self, out=None):
        """Raw stored deviation g~ = f~ - W rho0, [Q][ncell] in the storage type (bf16 as
        uint16 bit patterns on the host; f16 holds g~ * 2^12)."""
        nb = self.state_bytes()
        if out is not None:
            _check(self.lib.dugks_get_state(self.h, C.c_void_p(out.data_ptr()), nb, 1), self.h)
            return out
        a = np.zeros((self.q, self.ncell), dtype=self._dtype())
        _check(self.lib.dugks_get_state(self.h, a.ctypes.data_as(C.c_void_p), nb, 0), self.h)
        return a

    def set_state(self, a):
        nb = self.state_bytes()
        if hasattr(a, "data_ptr"):
            dev = 1 if a.is_cuda else 0
            _check(self.lib.dugks_set_state(self.h, C.c_void_p(a.data_ptr()), nb, dev), self.h)
            return
        a = np.ascontiguousarray(a, dtype=self._dtype())
        _check(self.lib.dugks_set_state(self.h, a.ctypes.data_as(C.c_void_p), nb, 0), self.h)

    def clock(self):
        s = C.c_int64()
        t = C.c_double()
        _check(self.lib.dugks_get_clock(self.h, C.byref(s), C.byref(t)), self.h)
        return s.value, t.value

    def set_clock(self, step):
        _check(self.lib.dugks_set_clock(self.h, int(step)), self.h)

    def set_force_field(self, field):
        self._field = field
        _check(self.lib.dugks_set_force_field(self.h, None if field is None else C.c_void_p(field.data_ptr())), self.h)

    def set_boundaries(self, bcs):
        """Replace wall velocities / pressures (same face types as at creation)."""
        b = make_bcs(bcs)
        _check(self.lib.dugks_set_boundaries(self.h, C.byref(b)), self.h)
        self.bcs = b

    def record(self, nsteps, every):
        """Run ``nsteps`` steps keeping a checkpoint every ``every`` steps (for ``adjoint``)."""
        _check(self.lib.dugks_record(self.h, int(nsteps), int(every)), self.h)

    def adjoint(self, dL_dmom, field_grad=True, state_grad=False):
        """Reverse sweep of the recorded rollout. ``dL_dmom``: CUDA float32 tensor
        [dim+1][ncell] (the gradient of the loss w.r.t. the final moments). Returns
        ``(dL/dfield CUDA [2][ncell] float32 or None, dL/du_wall numpy [6][3],
        dL/dstate0 CUDA [Q][ncell] or None)``."""
        import torch
        assert dL_dmom.is_cuda and dL_dmom.dtype == torch.float32 and dL_dmom.is_contiguous()
        assert dL_dmom.numel() == (self.dim + 1) * self.ncell
        dev = dL_dmom.device
        dfield = torch.empty((self.dim, self.ncell), dtype=torch.float32, device=dev) if field_grad else None
        dwall = np.zeros((6, 3), dtype=np.float64)
        dstate = None
        if state_grad:
            dt = torch.float64 if self.store == STORE_F64 else torch.float32
            dstate = torch.empty((self.q, self.ncell), dtype=dt, device=dev)
        rc = self.lib.dugks_adjoint(self.h, C.c_void_p(dL_dmom.data_ptr()),
                                    None if dfield is None else C.c_void_p(dfield.data_ptr()), _dp(dwall),
                                    None if dstate is None else C.c_void_p(dstate.data_ptr()))
        _check(rc, self.h)
        return dfield, dwall, dstate

    def adjoint_async(self, dL_dmom, dfield=None, dstate=None):
        """Enqueue the reverse sweep on the handle's stream and return (see
        ``dugks_adjoint_async``); ``dfield`` / ``dstate`` are CUDA tensors filled once the
        stream completes (``sync``)."""
        assert dL_dmom.is_cuda and dL_dmom.is_contiguous() and dL_dmom.numel() == (self.dim + 1) * self.ncell
        self._async_keep = (dL_dmom, dfield, dstate)  # kept alive until the next call
        rc = self.lib.dugks_adjoint_async(self.h, C.c_void_p(dL_dmom.data_ptr()),
                                          None if dfield is None else C.c_void_p(dfield.data_ptr()),
                                          None if dstate is None else C.c_void_p(dstate.data_ptr()))
        _check(rc, self.h)

    def adjoint_wall(self):
        """dL/du_wall [6][3] of the last adjoint (waits for the handle's stream)."""
        out = np.zeros((6, 3), dtype=np.float64)
        _check(self.lib.dugks_adjoint_wall(self.h, _dp(out)), self.h)
        return out

    def sync(self, timeout_s=0.0):
        _check(self.lib.dugks_sync(self.h, float(timeout_s)), self.h)

    def launch_count(self):
        return self.lib.dugks_launch_count(self.h)


class Batch:
    """Many independent D2Q9 instances advanced together (see ``dugks_batch_*``).

    ``instances``: list of dicts with ``shape`` (nx, ny), ``nu``, optional ``g``, ``omega``,
    ``field`` (CUDA float tensor [2][ncell]), ``bcs`` and ``dx``; shared ``dt``, ``rt``,
    ``rho0``, ``store``.
    """

    def __init__(self, instances, dt, rt=1.0 / 3.0, rho0=1.0, store=STORE_F32, stream=None, tile=None):
        lib = load()
        self.lib = lib
        n = len(instances)
        self.count = n
        meshes = (Mesh * n)()
        nus = (C.c_double * n)()
        forces = (Force * n)()
        bcs = (Boundaries * n)()
        self._fields = []
        self.shapes = []
        for i, ins in enumerate(instances):
            nx, ny = int(ins["shape"][0]), int(ins["shape"][1])
            self.shapes.append((nx, ny))
            meshes[i] = Mesh(2, nx, ny, 1, float(ins.get("dx", 1.0)))
            nus[i] = float(ins["nu"])
            g = ins.get("g", (0.0, 0.0, 0.0))
            for a in range(3):
                forces[i].g[a] = float(g[a]) if a < len(g) else 0.0
            forces[i].omega = float(ins.get("omega", 0.0))
            fld = ins.get("field")
            self._fields.append(fld)
            forces[i].field = None if fld is None else int(fld.data_ptr())
            bcs[i] = make_bcs(ins.get("bcs"))
        o = Opts()
        lib.dugks_opts_default(C.byref(o))
        o.rt, o.rho0, o.store = float(rt), float(rho0), int(store)
        o.stream = None if stream is None else int(stream)
        if tile:
            o.tile_x, o.tile_y = int(tile[0]), int(tile[1])
        h = C.c_void_p()
        rc = lib.dugks_batch_create(n, meshes, C.cast(nus, C.POINTER(C.c_double)), float(dt), forces, bcs,
                                    C.byref(o), C.byref(h))
        if rc != DUGKS_OK:
            raise DugksError(rc, lib.dugks_batch_last_error(None).decode(errors="replace"))
        self.h = h

    def _check(self, rc):
        if rc != DUGKS_OK:
            raise DugksError(rc, self.lib.dugks_batch_last_error(self.h).decode(errors="replace"))

    def close(self):
        if getattr(self, "h", None):
            self.lib.dugks_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def init(self, i, p=None, u=None):
        p = None if p is None else np.ascontiguousarray(p, dtype=np.float64).ravel()
        u = None if u is None else np.ascontiguousarray(u, dtype=np.float64).ravel()
        self._check(self.lib.dugks_batch_init(self.h, int(i), _dp(p), _dp(u)))

    def step(self, n=1):
        self._check(self.lib.dugks_batch_step(self.h, int(n)))

    def sync(self):
        self._check(self.lib.dugks_batch_sync(self.h))

    def moments(self, i):
        nx, ny = self.shapes[i]
        a = np.zeros((3, nx * ny), dtype=np.float32)
        self._check(self.lib.dugks_batch_moments(self.h, int(i), a.ctypes.data_as(C.c_void_p), 0))
        return a

    def tune(self):
        tx, ty = C.c_int32(), C.c_int32()
        self._check(self.lib.dugks_batch_tune(self.h, C.byref(tx), C.byref(ty)))
        return tx.value, ty.value

    def launch_count(self):
        return self.lib.dugks_batch_launch_count(self.h)
