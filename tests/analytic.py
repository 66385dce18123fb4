"""Closed-form flow solutions the paper validates against (test infrastructure).

Each function states the passage it restates. These are solutions of the incompressible
Navier-Stokes equations, independent of the DUGKS scheme, and serve as pins for the
oracle and the CUDA path.
"""
import numpy as np


def cell_centres(n, length=1.0):
    """Cell-centre coordinates of a uniform cell-centred mesh of n cells on [0, length]."""
    return (np.arange(n) + 0.5) * (length / n)


def periodic_flow(x, y, u0, rho0, nu):
    """Force-driven periodic flow, Sec. 3.1 (eq. (35) and the body force after it):
    u = u0 sin2pix sin2piy, v = u0 cos2pix cos2piy,
    p = rho0 u0^2 (cos4pix - cos4piy)/4, F = 8 pi^2 nu (u, v)."""
    u = u0 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    v = u0 * np.cos(2 * np.pi * x) * np.cos(2 * np.pi * y)
    p = 0.25 * rho0 * u0 ** 2 * (np.cos(4 * np.pi * x) - np.cos(4 * np.pi * y))
    fx = 8 * np.pi ** 2 * nu * u
    fy = 8 * np.pi ** 2 * nu * v
    return u, v, p, fx, fy


def poiseuille(y, G, nu, H=1.0):
    """Plane Poiseuille flow, Sec. 3.2 (eq. (38)) for walls at y = 0 and y = H:
    u = G/(2 nu) y (H - y)."""
    return G / (2.0 * nu) * y * (H - y)


def womersley_complex(y, t, G, omega, nu, Ly):
    """Womersley velocity, Sec. 3.3 (eq. (39)), for the pressure gradient
    dP/dx = G cos(omega t): u = Re[ i G/omega (1 - cos(lam (2y/Ly - 1)) / cos(lam)) e^{i omega t} ].
    The printed definition of lambda is garbled; lam^2 = -i alpha^2 with alpha =
    (Ly/2) sqrt(omega/nu) is the reading that makes this solve u_t = -G cos(omega t) + nu u_yy
    with u = 0 at the walls (and it agrees with the real K-form below)."""
    alpha = 0.5 * Ly * np.sqrt(omega / nu)
    lam = alpha * (1 - 1j) / np.sqrt(2.0)
    prof = 1.0 - np.cos(lam * (2.0 * y / Ly - 1.0)) / np.cos(lam)
    return np.real(1j * G / omega * prof * np.exp(1j * omega * t))


def womersley_real(y, t, G, omega, nu, Ly):
    """Womersley velocity, real form of Sec. 3.3 (eq. (42) with K_r, K_i, K_a):
    u = G/omega [ -sin wt + (K_r sin wt + K_i cos wt)/K_a ], k = alpha/sqrt2,
    theta = k (2y/Ly - 1)."""
    alpha = 0.5 * Ly * np.sqrt(omega / nu)
    k = np.sqrt(2.0) * alpha / 2.0
    th = k * (2.0 * y / Ly - 1.0)
    Kr = np.cos(th) * np.cosh(th) * np.cos(k) * np.cosh(k) + np.sin(th) * np.sinh(th) * np.sin(k) * np.sinh(k)
    Ki = np.sin(th) * np.sinh(th) * np.cos(k) * np.cosh(k) - np.cos(th) * np.cosh(th) * np.sin(k) * np.sinh(k)
    Ka = (np.sin(k) * np.sinh(k)) ** 2 + (np.cos(k) * np.cosh(k)) ** 2
    wt = omega * t
    return G / omega * (-np.sin(wt) + (Kr * np.sin(wt) + Ki * np.cos(wt)) / Ka)


def womersley_forced(y, t, G0, omega, nu, Ly):
    """Womersley channel driven by a body force G(t) = G0 cos(omega t) instead of the
    pressure gradient: the momentum equation u_t = G(t) + nu u_yy is the paper's with
    dP/dx = -G0 cos(omega t), so the solution is the paper's with G -> -G0."""
    return womersley_real(y, t, -G0, omega, nu, Ly)


def kolmogorov(y, u0):
    """Steady Kolmogorov flow u = u0 sin(2 pi y) driven by F_x = 4 pi^2 nu u0 sin(2 pi y):
    the one-dimensional analogue of the periodic flow of Sec. 3.1."""
    return u0 * np.sin(2 * np.pi * y)


def couette(y, U, H):
    """Plane Couette flow between a wall at rest (y = 0) and one moving at U (y = H)."""
    return U * y / H
