"""The pressure-driven Womersley flow of Sec. 3.3 (test infrastructure): 2 x 1 channel of
40 x 20 cells, rho0 = 1, nu = 1e-3, dP/dx = G cos(omega t) with G = 1e-3 (NEQ pressure inlet
p_out - L_x G cos(omega t), outlet p_out = 0), bounce-back tube walls, CFL 0.5, RT = 16/3,
T = 100, alpha = 3.963; initialised from the analytic pressure and velocity, run until the
velocity changes by at most 1e-8 from one period to the next, then sampled at t = nT/8."""
import numpy as np

from paper_1411_6121_gb300 import workloads as W
from tests import analytic as A

LX, LY, NX, NY = 2.0, 1.0, 40, 20
NU, G, RT, PERIOD = 1e-3, 1e-3, 16.0 / 3.0, 100.0


def setup(alpha=None, g=G, model=0):
    """The case's configuration (alpha = 3.963 by default; another alpha sets nu at the same
    period), the exact (p, u) at time t and the steps per period."""
    dx = LX / NX
    c = np.sqrt(3 * RT)
    dt = 0.5 * dx / c
    omega = 2 * np.pi / PERIOD
    nu = NU if alpha is None else omega * (0.5 * LY / alpha) ** 2
    cfg = dict(shape=(NX, NY), q=9, nu=nu, dt=dt, dx=dx, rt=RT, omega=omega, model=model,
               bcs=[W.pressure(0.0, -LX * g), W.pressure(0.0), W.bounce_back(), W.bounce_back()])
    x = A.cell_centres(NX, LX)
    y = A.cell_centres(NY, LY)
    X, Y = np.meshgrid(x, y)  # [y][x]: ravel gives cell x + NX y

    def exact(t):
        p = -(LX - X) * g * np.cos(omega * t)
        u = A.womersley_real(Y, t, g, omega, nu, LY)
        return p.ravel(), np.stack([u.ravel(), np.zeros(X.size)])

    steps_per_period = int(round(PERIOD / dt))
    assert abs(steps_per_period * dt - PERIOD) < 1e-9
    return cfg, exact, steps_per_period


def errors(run_periods, sample):
    """run_periods(n): advance n periods, return the velocity [2][ncell]; sample(k): advance
    k steps, return (p, u). Returns (periods run, pressure error over the period, velocity
    error over the period), each error the L2 norm over the 8 phases relative to the exact."""
    cfg, exact, spp = setup()
    prev = None
    for n in range(1, 81):
        u = run_periods(1)
        if prev is not None and np.linalg.norm(u - prev) / np.linalg.norm(u) <= 1e-8:
            break
        prev = u
    dp = np.zeros(2)
    du = np.zeros(2)
    for m in range(8):
        p, u = sample(0 if m == 0 else spp // 8)
        pe, ue = exact(n * PERIOD + m * PERIOD / 8)
        dp += [np.sum((p - pe) ** 2), np.sum(pe ** 2)]
        du += [np.sum((u - ue) ** 2), np.sum(ue ** 2)]
    return n, float(np.sqrt(dp[0] / dp[1])), float(np.sqrt(du[0] / du[1]))


def phase_errors(run_periods, sample, exact, spp):
    """Run to the periodic state, then the L2 velocity error at each phase t = nT/8 and the
    largest |u| of the exact solution. Returns (E per phase, U_max)."""
    prev = None
    for n in range(1, 81):
        u = run_periods(1)
        if prev is not None and np.linalg.norm(u - prev) / np.linalg.norm(u) <= 1e-8:
            break
        prev = u
    E, umax = [], 0.0
    for m in range(8):
        _, u = sample(0 if m == 0 else spp // 8)
        _, ue = exact(n * PERIOD + m * PERIOD / 8)
        E.append(np.linalg.norm(u[0] - ue[0]) / np.linalg.norm(ue[0]))
        umax = max(umax, np.abs(ue[0]).max())
    return np.array(E), umax


def table2():
    import os
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "table2_womersley_models.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return rows
