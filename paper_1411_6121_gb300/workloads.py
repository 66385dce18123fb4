"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the scheme: it only names the workloads (mesh sizes,
physical parameters in lattice units, boundary layouts) and draws seeded random fields.
Lattice units throughout: dx = 1, RT = 1/3 (so the particle speed sqrt(3RT) = 1), rho0 = 1,
dt = CFL * dx / sqrt(3RT) = 0.5.
"""
import math

import numpy as np

BC_PERIODIC = 0
BC_NEQ_VELOCITY = 1
BC_NEQ_PRESSURE = 2
BC_BOUNCE_BACK = 3

RT_LATTICE = 1.0 / 3.0
RHO0 = 1.0
CFL = 0.5


def dt_for(cfl=CFL, dx=1.0, rt=RT_LATTICE):
    """Time step from the CFL number of Sec. 3: dt = a dx / sqrt(3 RT)."""
    return cfl * dx / math.sqrt(3.0 * rt)


def periodic():
    return (BC_PERIODIC, (0.0, 0.0, 0.0), 0.0)


def wall(u=(0.0, 0.0, 0.0)):
    return (BC_NEQ_VELOCITY, tuple(float(a) for a in u) + (0.0,) * (3 - len(u)), 0.0)


def pressure(p, amp=0.0):
    """NEQ pressure condition p_w = p (+ amp cos(omega t) with the force's omega)."""
    if amp:
        return (BC_NEQ_PRESSURE, (0.0, 0.0, 0.0), float(p), float(amp))
    return (BC_NEQ_PRESSURE, (0.0, 0.0, 0.0), float(p))


def bounce_back(u=(0.0, 0.0, 0.0)):
    """Bounce-back wall (eq. (31)) moving with velocity u."""
    return (BC_BOUNCE_BACK, tuple(float(a) for a in u) + (0.0,) * (3 - len(u)), 0.0)


def channel_bcs(dim=2):
    """Periodic in x (and z in 3D), NEQ no-slip walls at y = 0 and y = H."""
    b = [periodic(), periodic(), wall(), wall()]
    b += [periodic(), periodic()] if dim == 3 else [periodic(), periodic()]
    return b


def cavity_bcs(dim, lid_u=0.1):
    """Lid-driven cavity: every face a NEQ velocity wall, the +y face moving along +x."""
    b = [wall(), wall(), wall(), wall((lid_u, 0.0, 0.0))]
    b += [wall(), wall()] if dim == 3 else [periodic(), periodic()]
    return b


def all_periodic():
    return [periodic()] * 6


# ---- named workloads -------------------------------------------------------------

def channel_8x32():
    """Force-driven channel: 8 x 32 cells, periodic x, NEQ walls, nu = 0.01, Gx = 1e-5."""
    return dict(shape=(8, 32), q=9, nu=0.01, dt=dt_for(), g=(1e-5, 0.0, 0.0),
                bcs=channel_bcs(2), rt=RT_LATTICE, rho0=RHO0)


def womersley_128x64(alpha=4.0, G0=1e-4, nu=0.2):
    """Force-driven Womersley channel: 128 x 64 cells, G(t) = G0 cos(omega t) with the
    Womersley number alpha = (H/2) sqrt(omega/nu)."""
    H = 64
    omega = nu * (2.0 * alpha / H) ** 2
    return dict(shape=(128, H), q=9, nu=nu, dt=dt_for(), g=(G0, 0.0, 0.0), omega=omega,
                bcs=channel_bcs(2), rt=RT_LATTICE, rho0=RHO0)


def cavity2d(n=1024, re=1000.0, lid_u=0.1):
    """2D lid-driven cavity, n x n cells, Re = U n / nu."""
    return dict(shape=(n, n), q=9, nu=lid_u * n / re, dt=dt_for(), bcs=cavity_bcs(2, lid_u),
                rt=RT_LATTICE, rho0=RHO0)


def cavity3d(n=256, re=1000.0, lid_u=0.1, q=19):
    """3D lid-driven cube, n^3 cells, lid (+y face) moving along +x, Re = U n / nu."""
    return dict(shape=(n, n, n), q=q, nu=lid_u * n / re, dt=dt_for(), bcs=cavity_bcs(3, lid_u),
                rt=RT_LATTICE, rho0=RHO0)


def batched_channels(count=64, seed=0x1411, u_max=0.05):
    """64 force-driven channels of uneven sizes: ny from {16, 32, 64, 128, 256}, nx = 2 ny,
    Re log-uniform in [10, 500], nu = u_max ny / Re, G = 8 nu u_max / ny^2."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        ny = int(rng.choice([16, 32, 64, 128, 256]))
        re = float(np.exp(rng.uniform(np.log(10.0), np.log(500.0))))
        nu = u_max * ny / re
        G = 8.0 * nu * u_max / ny ** 2
        out.append(dict(shape=(2 * ny, ny), q=9, nu=nu, dt=dt_for(), g=(G, 0.0, 0.0),
                        bcs=channel_bcs(2), rt=RT_LATTICE, rho0=RHO0, re=re))
    return out


def force_field(shape, G, seed, rel=0.1):
    """Per-cell acceleration field G (1 + rel N(0,1)) along x, zero along the other axes;
    layout [dim][ncell] with x fastest."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    f = np.zeros((len(shape), n))
    f[0] = G * (1.0 + rel * rng.standard_normal(n))
    return f


def random_state_fields(shape, seed, u_amp=0.05, p_amp=1e-3):
    """Smooth-plus-noise initial pressure and velocity fields (for parity tests that must
    exercise every term): returns p [ncell], u [dim][ncell], x fastest."""
    rng = np.random.default_rng(seed)
    dim = len(shape)
    grids = np.meshgrid(*[(np.arange(s) + 0.5) / s for s in reversed(shape)], indexing="ij")
    # grids[0] is the slowest axis; reverse so that coords[a] is axis a.
    coords = list(reversed(grids))
    n = int(np.prod(shape))
    u = np.zeros((dim, n))
    for a in range(dim):
        phase = rng.uniform(0, 2 * np.pi, size=dim)
        smooth = np.ones_like(coords[0])
        for b in range(dim):
            smooth = smooth * np.sin(2 * np.pi * coords[b] + phase[b])
        noise = rng.standard_normal(coords[0].shape)
        u[a] = (u_amp * (0.8 * smooth + 0.2 * noise)).ravel()
    p = (p_amp * rng.standard_normal(n))
    return p, u


def tanh_faces(n, length=1.0, k=2.5):
    """Interface coordinates of the paper's non-uniform mesh (Sec. 3.4): zeta_i = 0.5 +
    tanh(k (i/n - 0.5)) / (2 tanh(k/2)), i = 0 .. n, scaled to [0, length] (clustered at both
    ends; cell centres are the midpoints of their interfaces)."""
    import numpy as np
    i = np.arange(n + 1)
    return length * (0.5 + np.tanh(k * (i / n - 0.5)) / (2.0 * np.tanh(k / 2.0)))
