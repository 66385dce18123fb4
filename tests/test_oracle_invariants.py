"""Pins of the oracle's whole time step (Appendix steps 1-10) by exact properties.

Every check is fixed by the mathematics of the scheme, not by re-running its formulas:
  * states that the paper's scheme must leave unchanged (rest, uniform flow, Couette);
  * symmetries (periodic translation, mirror);
  * conservation and the momentum/mass bookkeeping of the force term (eqs. (9), (17));
  * closed-form flows (Couette exactly; Poiseuille, Kolmogorov and Womersley closely).
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1411_6121_gb300 import workloads as W
from tests import analytic as A


def _bcs2(x="p", y="p"):
    m = {"p": [W.periodic(), W.periodic()], "w": [W.wall(), W.wall()]}
    return m[x] + m[y]


@pytest.mark.parametrize("q,shape", [(9, (6, 5)), (19, (4, 3, 5)), (27, (3, 4, 3))])
def test_rest_state_is_fixed(q, shape):
    bcs = W.cavity_bcs(len(shape), lid_u=0.0)
    o = Oracle(shape, q, nu=0.05, dt=0.5, bcs=bcs)
    o.init()
    f0 = o.get_state()
    o.step(7)
    assert np.abs(o.get_state() - f0).max() < 1e-15


@pytest.mark.parametrize("q,shape", [(9, (5, 7)), (19, (4, 5, 3)), (27, (3, 3, 4))])
def test_uniform_flow_is_fixed(q, shape):
    D = len(shape)
    U = np.array([0.03, -0.02, 0.01][:D])
    n = int(np.prod(shape))
    u = np.repeat(U[:, None], n, axis=1)
    o = Oracle(shape, q, nu=0.02, dt=0.5, bcs=W.all_periodic())
    o.init(u=u)
    f0 = o.get_state()
    o.step(9)
    assert np.abs(o.get_state() - f0).max() < 1e-15
    # the same uniform flow between NEQ velocity walls moving with it, and between NEQ
    # pressure boundaries at the reference pressure, is also unchanged.
    bw = [W.wall(tuple(U))] * (2 * D) + [W.periodic()] * (6 - 2 * D)
    o = Oracle(shape, q, nu=0.02, dt=0.5, bcs=bw)
    o.init(u=u)
    o.step(5)
    assert np.abs(o.get_state() - f0).max() < 1e-15
    bp = [W.pressure(0.0), W.pressure(0.0)] + [W.periodic()] * 4
    o = Oracle(shape, q, nu=0.02, dt=0.5, bcs=bp)
    o.init(u=u)
    o.step(5)
    assert np.abs(o.get_state() - f0).max() < 1e-15


@pytest.mark.parametrize("q,shape", [(9, (6, 5)), (19, (4, 5, 3))])
def test_periodic_translation_commutes(q, shape):
    D = len(shape)
    p, u = W.random_state_fields(shape, seed=3)
    field = W.force_field(shape, 1e-4, seed=4, rel=1.0)
    o = Oracle(shape, q, nu=0.03, dt=0.5, g=(1e-5, 2e-5, 0.0), field=field, bcs=W.all_periodic())
    o.init(p=p, u=u)
    f = o.get_state()
    shift = (2, 1, 1)[:D]
    rev = tuple(reversed(shape))

    def roll(a):
        a = a.reshape(a.shape[:-1] + rev)
        for ax in range(D):  # axis ax lives at position -1-ax of the reversed grid
            a = np.roll(a, shift[ax], axis=a.ndim - 1 - ax)
        return a.reshape(a.shape[: a.ndim - D] + (-1,))

    o.step(3)
    f_then_shift = roll(o.get_state())
    o2 = Oracle(shape, q, nu=0.03, dt=0.5, g=(1e-5, 2e-5, 0.0), field=roll(field), bcs=W.all_periodic())
    o2.set_state(roll(f), t=0.0, step=0)
    o2.step(3)
    assert np.array_equal(o2.get_state(), f_then_shift)


def test_channel_mirror_symmetry():
    """Reflection y -> H - y maps the channel onto itself (v -> -v): k <-> k with e_y flipped."""
    shape = (6, 8)
    p, u = W.random_state_fields(shape, seed=5)
    o = Oracle(shape, 9, nu=0.04, dt=0.5, g=(1e-5, 0, 0), bcs=W.channel_bcs())
    o.init(p=p, u=u)
    e, _ = o.lattice()
    flip = [int(np.where((e[:, 0] == e[k, 0]) & (e[:, 1] == -e[k, 1]))[0][0]) for k in range(9)]

    def mirror(f):
        g = f[flip].reshape(9, 8, 6)[:, ::-1, :]
        return g.reshape(9, -1)

    f0 = o.get_state()
    o.step(4)
    a = mirror(o.get_state())
    o2 = Oracle(shape, 9, nu=0.04, dt=0.5, g=(1e-5, 0, 0), bcs=W.channel_bcs())
    o2.set_state(mirror(f0), t=0.0, step=0)
    o2.step(4)
    assert np.abs(o2.get_state() - a).max() < 2e-15  # summation order differs


@pytest.mark.parametrize("q,shape", [(9, (7, 6)), (19, (4, 3, 5))])
def test_mass_conserved_periodic(q, shape):
    p, u = W.random_state_fields(shape, seed=7)
    o = Oracle(shape, q, nu=0.02, dt=0.5, bcs=W.all_periodic())
    o.init(p=p, u=u)
    m0 = o.sums()
    o.step(20)
    m1 = o.sums()
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-14
    # with G = 0 momentum is conserved too (the flux telescopes and Omega conserves it)
    assert np.abs(m1[1:] - m0[1:]).max() < 1e-14 * m0[0]


def test_force_bookkeeping_periodic():
    """With periodic boundaries the flux telescopes, so one step changes the totals only
    through the collision and force terms of eq. (17). Using sum_k xi_k S_k = rho G and
    sum_k S_k = G.u (rho0 - rho)/RT (both from eqs. (6) and (9)), per step
      dJ = sum_cells dt (rho0 dt + 2 tau rho) G / (2 tau + dt),   J = sum_k xi_k f~,
      dM = sum_cells 2 tau dt/(2 tau + dt) G.u (rho0 - rho)/RT,   M = sum_k f~."""
    shape = (6, 5)
    rt, rho0, nu, dt = 1.0 / 3.0, 1.0, 0.03, 0.5
    tau = nu / rt
    p, u = W.random_state_fields(shape, seed=11, u_amp=0.05, p_amp=0.01)
    field = W.force_field(shape, 1e-3, seed=12, rel=1.0)
    field[1] = 0.5e-3
    o = Oracle(shape, 9, nu=nu, dt=dt, rt=rt, rho0=rho0, field=field, bcs=W.all_periodic())
    o.init(p=p, u=u)
    for _ in range(3):
        m = o.moments()
        rho = rho0 + m[0] / rt
        uu = m[1:]
        s0 = o.sums()
        J0 = s0[1:] - rho0 * field.sum(1) * dt / 2      # sum xi f~ = rho0 u - rho0 G dt/2
        o.step(1)
        s1 = o.sums()
        J1 = s1[1:] - rho0 * field.sum(1) * dt / 2
        dJ = (dt * (rho0 * dt + 2 * tau * rho)[None, :] * field / (2 * tau + dt)).sum(1)
        dM = (2 * tau * dt / (2 * tau + dt) * (field * uu).sum(0) * (rho0 - rho) / rt).sum()
        assert np.abs((J1 - J0) - dJ).max() < 1e-15 * s0[0]
        assert abs((s1[0] - s0[0]) - dM) < 1e-15 * s0[0]


@pytest.mark.parametrize("q,shape,axis", [(9, (3, 8), 1), (19, (2, 6, 3), 1), (27, (2, 2, 6), 2)])
def test_couette_is_exact(q, shape, axis):
    """A linear shear profile between a wall at rest and a moving wall (NEQ velocity
    condition, eq. (32)) is a steady state of the scheme to rounding: the linear
    reconstruction and the linear ghost extrapolation are exact for it, and its
    non-equilibrium part is uniform, which the NEQ extrapolation copies exactly."""
    D = len(shape)
    U = 0.05
    bcs = [W.periodic()] * 6
    bcs[2 * axis] = W.wall()
    bcs[2 * axis + 1] = W.wall((U, 0.0, 0.0) if axis != 0 else (0.0, U, 0.0))
    o = Oracle(shape, q, nu=0.1, dt=0.5, bcs=bcs)
    coord = A.cell_centres(shape[axis], shape[axis])
    prof = A.couette(coord, U, shape[axis])
    rev = tuple(reversed(shape))
    grid = np.zeros(rev)
    sl = [None] * D
    sl[D - 1 - axis] = slice(None)
    grid = grid + prof[tuple(sl)]
    comp = 0 if axis != 0 else 1
    u = np.zeros((D, grid.size))
    u[comp] = grid.ravel()
    o.init(u=u)
    o.step(600)
    m = o.moments()
    assert np.abs(m[1 + comp] - grid.ravel()).max() < 1e-14
    assert np.abs(np.delete(m[1:], comp, axis=0)).max() < 1e-14
    assert np.abs(m[0]).max() < 1e-13


def test_poiseuille_parabola():
    """Sec. 3.2: the force-driven channel reaches u = G/(2 nu) y (H - y). In lattice units
    the mean free path sqrt(3RT) tau is 0.03 dx, so the kinetic slip is small; the
    steady profile agrees with the parabola to better than 1% (relative L2, Sec. 3.1)."""
    H, nu, G = 16, 0.05, 1e-5
    o = Oracle((2, H), 9, nu=nu, dt=0.5, g=(G, 0, 0), bcs=W.channel_bcs())
    y = A.cell_centres(H, H)
    ua = A.poiseuille(y, G, nu, H)
    u0 = np.zeros((2, 2 * H))
    u0[0] = np.repeat(ua, 2)
    o.init(u=u0)
    o.step(6000)
    ux = o.grid(o.moments()[1])[:, 0]
    err = np.sqrt(((ux - ua) ** 2).sum() / (ua ** 2).sum())
    assert err < 1e-2
    # the discrete profile is symmetric and the wall-normal velocity vanishes
    assert np.abs(ux - ux[::-1]).max() < 1e-15
    assert np.abs(o.moments()[2]).max() < 1e-15


def _kolmogorov_error(N, cfl=0.02, rt=5.0, nu=0.01, u0=1e-3):
    from oracle.oracle import rel_change
    dx = 1.0 / N
    dt = cfl * dx / np.sqrt(3 * rt)
    y = A.cell_centres(N)
    ua = A.kolmogorov(y, u0)
    field = np.zeros((2, N))
    field[0] = 4 * np.pi ** 2 * nu * ua
    o = Oracle((1, N), 9, nu=nu, dt=dt, dx=dx, rt=rt, field=field, bcs=W.all_periodic())
    u = np.zeros((2, N))
    u[0] = ua
    o.init(u=u)
    K = int(round(0.2 / (nu * 4 * np.pi ** 2) / dt))
    prev = o.moments()[1:]
    while True:
        o.step(K)
        cur = o.moments()[1:]
        if rel_change(cur, prev) < 1e-9:
            break
        prev = cur
    return np.sqrt(((cur[0] - ua) ** 2).sum() / (ua ** 2).sum())


def test_kolmogorov_second_order():
    """Steady forced shear flow (the one-dimensional analogue of Sec. 3.1's periodic
    flow) converges to its closed form at second order under mesh refinement (RT = 5 and
    nu = 0.01 as in Table 1; the mean free path 0.008 sets an error floor near 0.5% that
    the N = 16 -> 32 order starts to feel)."""
    e = [_kolmogorov_error(N) for N in (8, 16, 32)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert e[1] < 0.06
    assert abs(orders[0] - 2.0) < 0.1, (e, orders)
    assert abs(orders[1] - 2.0) < 0.25, (e, orders)


def _table1_run(N):
    rt, u0, rho0, nu, dt = 5.0, 0.1, 1.0, 0.01, 1e-4
    x = A.cell_centres(N)
    X, Y = np.meshgrid(x, x)
    u, v, p, fx, fy = A.periodic_flow(X, Y, u0, rho0, nu)
    o = Oracle((N, N), 9, nu=nu, dt=dt, dx=1.0 / N, rt=rt, rho0=rho0,
               field=np.stack([fx.ravel(), fy.ravel()]), bcs=W.all_periodic())
    o.init(p=p.ravel(), u=np.stack([u.ravel(), v.ravel()]))
    from oracle.oracle import l2_error, rel_change
    prev = o.moments()[1:]
    while True:  # steady criterion of Sec. 3.1
        o.step(1000)
        m = o.moments()
        if rel_change(m[1:], prev) <= 1e-6:
            break
        prev = m[1:]
    Eu = l2_error(m[1:], np.stack([u.ravel(), v.ravel()]))
    Ep = l2_error(m[0] - m[0].mean(), p.ravel())
    return Eu, Ep


def _table1():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_periodic_flow.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return {int(r[0]): (float(r[1]), float(r[3])) for r in rows}


def test_table1_convergence_order():
    """Table 1 (Sec. 3.1): the velocity error of the periodic flow falls at second order
    between N = 16 and N = 32 (paper: 2.015).

    The error constant is pinned by a closed form instead of the printed value. This run has
    dt = 1e-4 against tau = nu / RT = 2e-3, so h is tiny and the step-4 interface value is the
    plain mean of the two cells: the scheme then discretises the BGK equation with central
    differences, and the non-equilibrium part that carries the viscous stress is itself a
    central difference, so the viscous operator is the Laplacian of width 2 dx. For the mode
    sin(2 pi x) sin(2 pi y) it has the eigenvalue -2 sin^2(k dx) / dx^2 instead of -2 k^2
    (k = 2 pi), and the steady velocity balancing the force is too large by the factor
    (k dx)^2 / sin^2(k dx): E(u) = 5.30% at N = 16 and 1.30% at N = 32. The oracle must sit
    within 5% of that (it does to 2.5%). The printed constants (0.974%, 0.241%) are of the size
    of the compact Laplacian's (1.30%, 0.32%), which a step with h comparable to tau gives."""
    t = _table1()
    e16, p16 = _table1_run(16)
    e32, p32 = _table1_run(32)
    order_u = np.log2(e16 / e32)
    order_p = np.log2(p16 / p32)
    assert abs(order_u - 2.015) < 0.1, order_u
    assert abs(order_p - 2.027) < 0.25, order_p  # oracle: 1.86
    for n, e in ((16, e16), (32, e32)):
        kd = 2 * np.pi / n
        wide = kd ** 2 / np.sin(kd) ** 2 - 1.0
        assert abs(e / wide - 1.0) < 0.05, (n, e, wide)
    # the printed error at N = 16 is of the compact stencil's size (0.75 of it), far below the
    # wide stencil's
    kd = 2 * np.pi / 16
    compact = (kd / 2) ** 2 / np.sin(kd / 2) ** 2 - 1.0
    assert 0.5 * compact < t[16][0] < compact < 0.5 * e16


@pytest.mark.slow
def test_table1_n64():
    e32, _ = _table1_run(32)
    e64, _ = _table1_run(64)
    assert abs(np.log2(e32 / e64) - 2.0) < 0.3


def test_womersley_forms_agree():
    """The complex form (eq. (39), with the reading lam^2 = -i alpha^2) and the
    real K-form (eq. (42)) of Sec. 3.3 are the same function, and alpha = 3.963
    for the paper's nu = 1e-3, T = 100, Ly = 1."""
    Ly, nu, T = 1.0, 1e-3, 100.0
    omega = 2 * np.pi / T
    assert abs(0.5 * Ly * np.sqrt(omega / nu) - 3.963) < 5e-4
    y = np.linspace(0, 1, 41)
    for t in np.linspace(0, T, 9):
        a = A.womersley_complex(y, t, 1e-3, omega, nu, Ly)
        b = A.womersley_real(y, t, 1e-3, omega, nu, Ly)
        assert np.abs(a - b).max() < 1e-12
        assert abs(a[0]) < 1e-12 and abs(a[-1]) < 1e-12


def _womersley_error(H, nu=0.1, G0=1e-5, alpha=3.0, dt=0.5):
    omega = nu * (2 * alpha / H) ** 2
    period = 2 * np.pi / omega
    o = Oracle((1, H), 9, nu=nu, dt=dt, g=(G0, 0, 0), omega=omega, bcs=W.channel_bcs())
    y = A.cell_centres(H, H)
    u = np.zeros((2, H))
    u[0] = A.womersley_forced(y, 0.0, G0, omega, nu, H)
    o.init(u=u)
    o.step(int(round(3 * period / dt)))
    amp = max(np.linalg.norm(A.womersley_forced(y, t, G0, omega, nu, H)) for t in np.linspace(0, period, 33))
    errs = []
    for _ in range(8):  # the eight phases t = nT/8 of Sec. 3.3
        o.step(int(round(period / 8 / dt)))
        ua = A.womersley_forced(y, o.time, G0, omega, nu, H)
        errs.append(np.linalg.norm(o.moments()[1] - ua) / amp)
    return max(errs)


def test_womersley_forced_channel():
    """Force-driven Womersley flow (Sec. 3.3 with the pressure gradient supplied as a body
    force G0 cos(omega t), alpha = 3): after the start-up transient the oracle follows the
    closed form at every phase (L2 error over the channel relative to the profile's largest
    L2 norm over the period), and the error falls at second order from H = 16 to 32."""
    e16 = _womersley_error(16)
    e32 = _womersley_error(32)
    assert e16 < 0.03 and e32 < 0.008, (e16, e32)
    assert abs(np.log2(e16 / e32) - 2.0) < 0.2, (e16, e32)
