"""Pins of the bounce-back wall (Sec. 2.4, eq. (31)) in the oracle, by properties the equation
fixes exactly:
  * a bounce-back wall moving tangentially carries no mass. The incoming values are the
    outgoing ones plus 2 rho0 W_k xi_k.u_w / RT, whose xi_n moment cancels over the outgoing
    set, so a closed box keeps its mass to rounding (NEQ walls do not: the contrast keeps
    the check discriminating);
  * plane Couette flow between bounce-back walls is reproduced exactly (the sign and size of
    the wall term set the slope);
  * force-driven Poiseuille flow converges at second order (the paper's BB/NEQ comparison,
    Sec. 3.2), and bounce-back is the more accurate wall there, as the paper finds.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1411_6121_gb300 import workloads as W


def _box(dim, kind, lid):
    w = W.bounce_back if kind == "bb" else W.wall
    if dim == 2:
        return [w(), w(), w(), w((lid, 0.0))]
    return [w(), w(), w(), w((lid, 0.0, 0.0)), w(), w()]


@pytest.mark.parametrize("q,shape", [(9, (12, 10)), (19, (6, 5, 4)), (27, (5, 4, 4))])
def test_bounce_back_box_conserves_mass(q, shape):
    masses = {}
    for kind in ("bb", "neq"):
        o = Oracle(shape, q, nu=0.05, dt=0.5, bcs=_box(len(shape), kind, 0.1))
        o.init()
        m0 = o.moments()[0].sum()
        o.step(150)
        masses[kind] = abs(o.moments()[0].sum() - m0)
    ncell = int(np.prod(shape))
    # p = (rho - rho0) RT summed over the cells, relative to the total mass rho0 * ncell
    assert masses["bb"] / ncell < 1e-13, masses
    assert masses["neq"] / ncell > 1e-6, masses


@pytest.mark.parametrize("q", [9, 19, 27])
def test_bounce_back_couette_is_exact(q):
    ny, uw = 8, (0.05, 0.0, 0.02)
    if q == 9:
        shape, bcs = (4, ny), [W.periodic(), W.periodic(), W.bounce_back(), W.bounce_back(uw[:2])]
    else:
        shape = (3, ny, 3)
        bcs = [W.periodic(), W.periodic(), W.bounce_back(), W.bounce_back(uw), W.periodic(), W.periodic()]
    o = Oracle(shape, q, nu=0.2, dt=0.5, bcs=bcs)
    o.init()
    o.step(3000)
    m = o.moments()
    y = (np.arange(ny) + 0.5) / ny
    for a in range(len(shape)):
        u = m[1 + a].reshape(shape[::-1]).swapaxes(0, -1)  # [x][y](z)
        prof = u[0, :, 0] if q != 9 else u[0, :]
        assert np.abs(prof - uw[a] * y).max() < 1e-13, (a, np.abs(prof - uw[a] * y).max())


def _poiseuille_error(ny, wall):
    nu, umax = 0.1, 0.05
    G = 8 * nu * umax / ny ** 2
    o = Oracle((2, ny), 9, nu=nu, dt=0.5, g=(G, 0.0), bcs=[W.periodic(), W.periodic(), wall(), wall()])
    o.init()
    o.step(int(6 * ny * ny / nu))
    u = o.moments()[1].reshape(ny, 2)[:, 0] - 0.25 * G  # the reported u carries + G dt/2
    y = np.arange(ny) + 0.5
    ua = G / (2 * nu) * y * (ny - y)
    return np.linalg.norm(u - ua) / np.linalg.norm(ua)


def test_bounce_back_poiseuille_second_order():
    e8, e16 = _poiseuille_error(8, W.bounce_back), _poiseuille_error(16, W.bounce_back)
    order = np.log2(e8 / e16)
    assert 1.85 < order < 2.15, (e8, e16, order)
    # the paper finds bounce-back the more accurate of the two walls on this flow
    assert e8 < _poiseuille_error(8, W.wall)


@pytest.mark.slow
@pytest.mark.parametrize("rt", [5.0, 100.0 / 3.0])
def test_paper_poiseuille_bb_neq_close(rt):
    """Sec. 3.2's setting: unit square of 8 x 8 cells, rho0 = 1, Re = 10, G = 1e-3, dt = 1e-4,
    initialised from the analytic profile. The paper prints a largest BB/NEQ error
    difference of 0.16% (at 8 x 8) and does not state RT; at RT = 5 and 100/3 (its other
    cases' values) the two walls' errors are within 0.2% of each other."""
    G, Re, N = 1e-3, 10.0, 8
    nu = (G / (8 * Re)) ** 0.5
    y = (np.arange(N) + 0.5) / N
    ua = G / (2 * nu) * y * (1 - y)
    errs = []
    for wall in (W.bounce_back, W.wall):
        o = Oracle((2, N), 9, nu=nu, dt=1e-4, dx=1.0 / N, rt=rt, g=(G, 0.0),
                   bcs=[W.periodic(), W.periodic(), wall(), wall()])
        u0 = np.zeros((2, 2 * N))
        u0[0] = np.repeat(ua, 2)
        o.init(p=np.zeros(2 * N), u=u0)
        o.step(4_000_000)
        u = o.moments()[1].reshape(N, 2)[:, 0] - 0.5e-4 * G
        errs.append(np.linalg.norm(u - ua) / np.linalg.norm(ua))
    assert abs(errs[0] - errs[1]) < 2e-3, errs


@pytest.mark.slow
def test_womersley_pressure_driven_oracle():
    """Sec. 3.3's pressure-driven Womersley flow in the oracle: pressure errors over the
    period below the paper's 0.42% (several minutes of FP64 CPU time)."""
    from oracle.oracle import Oracle as Orc
    from tests import womersley_study as WS
    cfg, exact, spp = WS.setup()
    o = Orc(**cfg)
    o.init(*exact(0.0))

    def run_periods(n):
        o.step(n * spp)
        return o.moments()[1:]

    def sample(k):
        if k:
            o.step(k)
        m = o.moments()
        return m[0], m[1:]

    n, ep, eu = WS.errors(run_periods, sample)
    # pressure: the paper's bound (measured 0.244%); velocity: no printed figure, 2.03% measured
    assert ep < 0.0042 and eu < 0.03, (n, ep, eu)
