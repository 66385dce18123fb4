"""Degenerate mesh sizes through every kernel, element by element against the oracle: wall
axes of two cells (the smallest the NEQ condition allows: x_c is the other wall's
interface), periodic axes of one cell (every neighbour is the cell itself), and extents one
past a tile boundary (a tile of a single column or row)."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1411_6121_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = {
    "2d_2x2_cavity": dict(shape=(2, 2), q=9, nu=0.05, dt=0.5, bcs=W.cavity_bcs(2, 0.1)),
    "2d_1x3_channel": dict(shape=(1, 3), q=9, nu=0.05, dt=0.5, g=(1e-4, 0.0, 0.0), bcs=W.channel_bcs(2)),
    "2d_31x2_bb": dict(shape=(31, 2), q=9, nu=0.05, dt=0.5,
                       bcs=[W.bounce_back(), W.wall(), W.bounce_back(), W.bounce_back((0.05, 0.0))]),
    "2d_33x9_pressure": dict(shape=(33, 9), q=9, nu=0.05, dt=0.5,
                             bcs=[W.pressure(1e-3), W.pressure(-1e-3), W.wall(), W.wall()]),
    "3d_2x2x2_cavity19": dict(shape=(2, 2, 2), q=19, nu=0.05, dt=0.5, bcs=W.cavity_bcs(3, 0.1)),
    "3d_1x3x2_channel19": dict(shape=(1, 3, 2), q=19, nu=0.05, dt=0.5, g=(1e-4, 0.0, 0.0),
                               bcs=[W.periodic(), W.periodic(), W.wall(), W.wall((0.05, 0.0, 0.0)),
                                    W.wall(), W.wall()]),
    "3d_2x7x1_periodic_z19": dict(shape=(2, 7, 1), q=19, nu=0.05, dt=0.5,
                                  bcs=[W.wall(), W.wall((0.0, 0.05, 0.0)), W.periodic(), W.periodic(),
                                       W.periodic(), W.periodic()]),
    "3d_31x7x3_cavity27": dict(shape=(31, 7, 3), q=27, nu=0.05, dt=0.5, bcs=W.cavity_bcs(3, 0.1)),
    "3d_2x2x2_bb27": dict(shape=(2, 2, 2), q=27, nu=0.05, dt=0.5,
                          bcs=[W.bounce_back()] * 3 + [W.bounce_back((0.05, 0.0, 0.0))] + [W.bounce_back()] * 2),
}


def state_dev(o):
    e, Wt = o.lattice()
    return o.get_state() - Wt[:, None] * o.cfg.rho0


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("store,kernel", [(0, 0), (0, 1), (3, 1)])
def test_degenerate_sizes_elementwise(name, store, kernel):
    from paper_1411_6121_gb300 import dugks
    cfg = CASES[name]
    p, u = W.random_state_fields(cfg["shape"], seed=len(name) + 5, u_amp=0.03, p_amp=1e-3)
    o = Oracle(**cfg)
    o.init(p=p, u=u)
    o.step(10)
    s = dugks.Sim(store=store, kernel=kernel, **cfg)
    s.init(p=p, u=u)
    s.step(10)
    ref = state_dev(o)
    got = s.get_state().astype(np.float64)
    tol = 1e-11 if store == 3 else 2e-6
    assert np.abs(got - ref).max() < tol * np.abs(ref).max(), (np.abs(got - ref).max(), np.abs(ref).max())
