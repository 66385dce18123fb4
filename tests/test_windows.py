"""The window method of the full-size parity test, pinned on the CPU: with the oracle standing
in for the GPU on a cube small enough to step whole, one oracle step on each window gives,
on the compared cells, bitwise the whole-cube oracle's next state. It does so down to a
margin of one cell from an artificial side (one step of a cell reads its neighbours one cell
away; ghosts and x_c at true walls lie inside the window), and not at a margin of zero, so the
check is sharp and the margin of three used on the GPU is safe."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1411_6121_gb300 import workloads as W
from tests import windows as WD

N, WIN = 24, 11


@pytest.mark.parametrize("q", [19, 27])
def test_windows_reproduce_the_whole_cube(q):
    cfg = W.cavity3d(n=N, re=1000.0, lid_u=0.1, q=q)
    o = Oracle(**cfg)
    p, u = W.random_state_fields(cfg["shape"], seed=256, u_amp=0.03, p_amp=1e-3)
    o.init(p=p, u=u)
    o.step(3)
    f0 = o.get_state().reshape(q, N, N, N)
    o.step(1)
    f1 = o.get_state().reshape(q, N, N, N)
    short = 0.0
    for lo in WD.starts(N, WIN, np.random.default_rng(7)):
        zs, ys, xs = slice(lo[2], lo[2] + WIN), slice(lo[1], lo[1] + WIN), slice(lo[0], lo[0] + WIN)
        ow = Oracle((WIN, WIN, WIN), q, nu=cfg["nu"], dt=cfg["dt"], rt=cfg["rt"], rho0=cfg["rho0"],
                    bcs=WD.window_bcs(lo, WIN, N, cfg["bcs"]))
        ow.set_state(f0[:, zs, ys, xs].reshape(q, -1), t=3 * cfg["dt"], step=3)
        ow.step(1)
        ref = ow.get_state().reshape(q, WIN, WIN, WIN)
        want = f1[:, zs, ys, xs]
        sx, sy, sz = WD.compared(lo, WIN, N)
        assert np.array_equal(ref[:, sz, sy, sx], want[:, sz, sy, sx]), lo

        def grown(g):  # g cells closer to the artificial sides
            gs = [slice(max(0, sl.start - g), min(WIN, sl.stop + g)) for sl in (sx, sy, sz)]
            return np.abs(ref[:, gs[2], gs[1], gs[0]] - want[:, gs[2], gs[1], gs[0]]).max()

        assert grown(WD.MARGIN - 1) == 0.0, lo  # a margin of one cell is still exact
        short = max(short, grown(WD.MARGIN))    # a margin of zero is not
    assert short > 1e-6
