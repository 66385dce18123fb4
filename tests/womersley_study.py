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


def setup():
    dx = LX / NX
    c = np.sqrt(3 * RT)
    dt = 0.5 * dx / c
    omega = 2 * np.pi / PERIOD
    cfg = dict(shape=(NX, NY), q=9, nu=NU, dt=dt, dx=dx, rt=RT, omega=omega,
               bcs=[W.pressure(0.0, -LX * G), W.pressure(0.0), W.bounce_back(), W.bounce_back()])
    x = A.cell_centres(NX, LX)
    y = A.cell_centres(NY, LY)
    X, Y = np.meshgrid(x, y)  # [y][x]: ravel gives cell x + NX y

    def exact(t):
        p = -(LX - X) * G * np.cos(omega * t)
        u = A.womersley_real(Y, t, G, omega, NU, LY)
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
