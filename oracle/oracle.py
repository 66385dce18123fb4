"""ctypes wrapper of the FP64 CPU oracle (``dugks_oracle.c``).

TEST INFRASTRUCTURE. Marshals numpy arrays to the oracle's C functions; it adds no
arithmetic of the method. Arrays are direction-major / component-major with x fastest:
state ``[Q][ncell]``, moments ``[dim+1][ncell]`` (p, u_x, u_y[, u_z]).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

BC_PERIODIC = 0
BC_NEQ_VELOCITY = 1
BC_NEQ_PRESSURE = 2
BC_BOUNCE_BACK = 3


class OracleConfig(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("q", C.c_int),
        ("nx", C.c_int),
        ("ny", C.c_int),
        ("nz", C.c_int),
        ("dx", C.c_double),
        ("rt", C.c_double),
        ("rho0", C.c_double),
        ("nu", C.c_double),
        ("dt", C.c_double),
        ("g", C.c_double * 3),
        ("omega", C.c_double),
        ("bc_type", C.c_int * 6),
        ("bc_u", (C.c_double * 3) * 6),
        ("bc_p", C.c_double * 6),
        ("model", C.c_int),
        ("bc_p_amp", C.c_double * 6),
        ("faces", C.POINTER(C.c_double) * 3),
    ]


_LIBS = {}


def _lib(complex_step=False):
    name = "liboracle_cs.so" if complex_step else "liboracle.so"
    if name not in _LIBS:
        path = _build.lib_path(name)
        src = _build.SRC
        if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(src):
            _build.build()
        lib = C.CDLL(path)
        P, D, L, I = C.c_void_p, C.POINTER(C.c_double), C.c_long, C.c_int
        lib.oracle_create.restype = P
        lib.oracle_create.argtypes = [C.POINTER(OracleConfig)]
        lib.oracle_destroy.argtypes = [P]
        lib.oracle_lattice.argtypes = [P, C.POINTER(C.c_int), D]
        lib.oracle_set_field.argtypes = [P, D]
        lib.oracle_init.argtypes = [P, D, D]
        lib.oracle_step.argtypes = [P, L]
        lib.oracle_time.restype = C.c_double
        lib.oracle_time.argtypes = [P]
        lib.oracle_step_count.restype = L
        lib.oracle_step_count.argtypes = [P]
        lib.oracle_moments.argtypes = [P, D, D]
        lib.oracle_get_state.argtypes = [P, D, D]
        lib.oracle_set_state.argtypes = [P, D, D, C.c_double, L]
        lib.oracle_sums.argtypes = [P, D]
        lib.oracle_rel_change.restype = C.c_double
        lib.oracle_rel_change.argtypes = [D, D, L, I]
        lib.oracle_l2_error.restype = C.c_double
        lib.oracle_l2_error.argtypes = [D, D, L, I]
        if complex_step:
            lib.oracle_set_field_im.argtypes = [P, D]
            lib.oracle_set_wall_u_im.argtypes = [P, D]
        _LIBS[name] = lib
    return _LIBS[name]


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """One oracle simulation (FP64, CPU).

    Parameters mirror the paper's problem statement: a uniform mesh of ``shape`` cells
    with spacing ``dx``; lattice ``q`` (9, 19 or 27); ``rt`` = RT; ``rho0``; viscosity
    ``nu``; time step ``dt``; acceleration ``G(x, t) = (g + field(x)) cos(omega t)``;
    per-face boundaries ``bcs`` = 6 tuples ``(type, (ux, uy, uz), p)`` in the order
    -x, +x, -y, +y, -z, +z.
    """

    def __init__(self, shape, q, nu, dt, dx=1.0, rt=1.0 / 3.0, rho0=1.0, g=(0.0, 0.0, 0.0),
                 omega=0.0, bcs=None, field=None, complex_step=False, model=0, faces=None):
        dim = len(shape)
        nx, ny = int(shape[0]), int(shape[1])
        nz = int(shape[2]) if dim == 3 else 1
        cfg = OracleConfig()
        cfg.dim, cfg.q, cfg.nx, cfg.ny, cfg.nz = dim, int(q), nx, ny, nz
        cfg.dx, cfg.rt, cfg.rho0, cfg.nu, cfg.dt = dx, rt, rho0, nu, dt
        for a in range(3):
            cfg.g[a] = float(g[a]) if a < len(g) else 0.0
        cfg.omega = omega
        cfg.model = int(model)
        # non-uniform mesh: interface coordinates per axis (None: uniform spacing dx)
        self._faces = []
        for a, fa in enumerate(list(faces or [])[:3]):
            if fa is not None:
                arr = np.ascontiguousarray(fa, dtype=np.float64)
                self._faces.append(arr)
                cfg.faces[a] = arr.ctypes.data_as(C.POINTER(C.c_double))
        bcs = list(bcs or [])
        bcs += [(BC_PERIODIC, (0.0, 0.0, 0.0), 0.0)] * (6 - len(bcs))
        for w in range(6):
            t, u, p = bcs[w][:3]
            cfg.bc_type[w] = int(t)
            for a in range(3):
                cfg.bc_u[w][a] = float(u[a]) if a < len(u) else 0.0
            cfg.bc_p[w] = float(p)
            cfg.bc_p_amp[w] = float(bcs[w][3]) if len(bcs[w]) > 3 else 0.0
        self.lib = _lib(complex_step)
        self.complex_step = complex_step
        self.cfg = cfg
        self.h = self.lib.oracle_create(C.byref(cfg))
        if not self.h:
            raise ValueError("oracle: invalid configuration")
        self.dim, self.q = dim, int(q)
        self.shape = (nx, ny) if dim == 2 else (nx, ny, nz)
        self.ncell = nx * ny * nz
        self.set_field(field)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.oracle_destroy(h)
            self.h = None

    def lattice(self):
        e = np.zeros((self.q, 3), dtype=np.int32)
        W = np.zeros(self.q, dtype=np.float64)
        self.lib.oracle_lattice(self.h, e.ctypes.data_as(C.POINTER(C.c_int)), _dp(W))
        return e, W

    def set_field(self, field):
        f = _f64(field)
        if f is not None:
            assert f.size == self.dim * self.ncell
        self.lib.oracle_set_field(self.h, _dp(f))

    def init(self, p=None, u=None):
        p, u = _f64(p), _f64(u)
        if p is not None:
            assert p.size == self.ncell
        if u is not None:
            assert u.size == self.dim * self.ncell
        self.lib.oracle_init(self.h, _dp(p), _dp(u))

    def step(self, n=1):
        self.lib.oracle_step(self.h, int(n))

    @property
    def time(self):
        return self.lib.oracle_time(self.h)

    @property
    def steps(self):
        return self.lib.oracle_step_count(self.h)

    def moments(self, imag=False):
        out = np.zeros((self.dim + 1, self.ncell))
        im = np.zeros_like(out) if imag else None
        self.lib.oracle_moments(self.h, _dp(out), _dp(im))
        return (out, im) if imag else out

    def get_state(self, imag=False):
        re = np.zeros((self.q, self.ncell))
        im = np.zeros_like(re) if imag else None
        self.lib.oracle_get_state(self.h, _dp(re), _dp(im))
        return (re, im) if imag else re

    def set_state(self, re, im=None, t=None, step=None):
        re = _f64(re)
        im = _f64(im)
        assert re.size == self.q * self.ncell
        t = self.time if t is None else t
        step = self.steps if step is None else step
        self.lib.oracle_set_state(self.h, _dp(re), _dp(im), float(t), int(step))

    def sums(self):
        out = np.zeros(1 + self.dim)
        self.lib.oracle_sums(self.h, _dp(out))
        return out

    def set_field_im(self, im):
        self.lib.oracle_set_field_im(self.h, _dp(_f64(im)))

    def set_wall_u_im(self, im):
        self.lib.oracle_set_wall_u_im(self.h, _dp(_f64(im)))

    # Grid helpers (x fastest): views of a flat [ncell] array as (nz, ny, nx) / (ny, nx).
    def grid(self, a):
        a = np.asarray(a)
        return a.reshape(a.shape[:-1] + tuple(reversed(self.shape)))


def rel_change(u_new, u_old):
    """Steady-state criterion of Sec. 3.1 (relative L2 change of the velocity field)."""
    u_new, u_old = _f64(u_new), _f64(u_old)
    dim = u_new.shape[0]
    n = u_new[0].size
    return _lib().oracle_rel_change(_dp(u_new), _dp(u_old), n, dim)


def l2_error(phi, ref):
    """L2 relative global error E(phi) of Sec. 3.1; phi, ref shaped [ncomp][n]."""
    phi, ref = _f64(np.atleast_2d(phi)), _f64(np.atleast_2d(ref))
    return _lib().oracle_l2_error(_dp(phi), _dp(ref), phi[0].size, phi.shape[0])
