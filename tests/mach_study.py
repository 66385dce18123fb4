"""The compressibility study of Sec. 3.1 (test infrastructure): the force-driven periodic
flow on 32 x 32 cells with rho0 = 1, nu = 1e-2, dt = 1e-4 and CFL number 0.1, so that the
particle speed C = sqrt(3RT) = 0.1 dx / dt is fixed and the Mach number Ma = U / C is set by
the amplitude U = u0. Used by the oracle test (slow) and the CUDA test (FP64 path)."""
import numpy as np

from paper_1411_6121_gb300 import workloads as W
from tests import analytic as A


def golden():
    import os
    out = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "mach_sensitivity_periodic_flow.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def steady_error(ma, model, runner):
    """Steady L2 velocity error E(u) of the periodic flow at Mach number `ma` for `model`
    (0 incompressible, 1 original). runner(cfg, p, u, field) -> steady velocity [2][ncell]
    (reported u, which carries + G dt/2)."""
    N, nu, dt, cfl = 32, 1e-2, 1e-4, 0.1
    dx = 1.0 / N
    C = cfl * dx / dt
    x = A.cell_centres(N)
    X, Y = np.meshgrid(x, x)
    u, v, p, fx, fy = A.periodic_flow(X, Y, ma * C, 1.0, nu)
    ua = np.stack([u.ravel(), v.ravel()])
    force = np.stack([fx.ravel(), fy.ravel()])
    cfg = dict(shape=(N, N), q=9, nu=nu, dt=dt, dx=dx, rt=C * C / 3.0, bcs=W.all_periodic(), model=model)
    got = runner(cfg, p.ravel(), ua, force) - 0.5 * dt * force
    return float(np.sqrt(np.sum((got - ua) ** 2) / np.sum(ua ** 2)))


def check(err):
    """err(ma, model) -> E(u). Compares the study's three printed figures."""
    ref = golden()
    ma1 = ref["Ma_end"]
    e = {(m, ma): err(ma, m) for m in (0, 1) for ma in (ma1 / 8, ma1)}
    growth_c = 100 * (e[1, ma1] / e[1, ma1 / 8] - 1)
    growth_ic = 100 * (e[0, ma1] / e[0, ma1 / 8] - 1)
    below = 100 * (1 - e[0, ma1] / e[1, ma1])
    assert abs(growth_c - ref["growth_Ec_percent"]) < 2.0, (growth_c, e)
    assert abs(growth_ic - ref["growth_Eic_percent"]) < 0.5, (growth_ic, e)
    assert abs(below - ref["Eic_below_Ec_at_end_percent"]) < 1.5, (below, e)
    # at the smallest Mach number the two models nearly coincide
    assert abs(e[1, ma1 / 8] / e[0, ma1 / 8] - 1) < 1e-3, e
    return e
