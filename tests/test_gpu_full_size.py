"""Parity at the benchmark's full size: the lid-driven cube of 256^3 cells through the
throughput kernel in the launch configuration the benchmark times, for each leg of the
benchmark (D3Q19 with FP32, BF16 and FP16 storage, D3Q27 with FP32). The oracle
cannot step 16.8 M cells, but one step of a cell reads only its neighbours (interface
reconstruction with tangential cross points; ghosts and x_c of a true wall lie inside a window
touching it; pinned on the CPU in test_windows.py). So the test
takes the GPU's state after a few steps and runs ONE oracle step on sampled windows of it:
  * windows at the domain's corners, edges, faces (with the true walls there) and inside;
  * on a window side that is not a domain boundary the oracle sees an artificial rest wall
    (or a periodic seam), so only cells at least three away from such sides are compared;
and compares those cells with the GPU's next state, element by element."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1411_6121_gb300 import workloads as W
from tests.windows import compared, starts, window_bcs

pytestmark = pytest.mark.gpu

N = 256
WIN = 11          # window edge (cells)


def _decode(a, store):
    """Stored values as float64 deviations (BF16: bit patterns; F16: g~ x 2^12)."""
    if store == 1:
        return (a.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    if store == 2:
        return a.astype(np.float64) / 4096.0
    return a.astype(np.float64)


# (velocity set, storage): the benchmark's main leg, its 16-bit legs and its D3Q27 leg.
# 16-bit results carry one stochastic rounding of the stored value: up to one unit in the
# last place, 2^-7 (BF16) or 2^-10 (FP16) of the value, on top of the FP32 arithmetic.
LEGS = [(19, 0, 0.0), (19, 1, 2.0 ** -7), (19, 2, 2.0 ** -10), (27, 0, 0.0)]
# Windows across z-chunk boundaries of the throughput kernels' launch: on 152 SMs the 256^3 cube
# runs in chunks of 52 planes (D3Q19: 9 x 43 tiles), so z = 52, 104, 156, 208 start a chunk,
# whose first interface takes the direct path and whose ring is filled anew. Each window below
# spans one of them by at least two planes on either side.
CHUNK_WINDOWS = [(122, 122, 47), (40, 200, 99), (200, 40, 151), (150, 150, 203)]


@pytest.mark.parametrize("q,store,ulp", LEGS)
def test_256_cube_sampled_windows(q, store, ulp):
    from paper_1411_6121_gb300 import dugks
    cfg = W.cavity3d(n=N, re=1000.0, lid_u=0.1, q=q)
    s = dugks.Sim(store=store, use_graph=False, **cfg)
    p, u = W.random_state_fields(cfg["shape"], seed=256, u_amp=0.03, p_amp=1e-3)
    s.init(p=p, u=u)
    del p, u
    s.step(3)
    g0 = _decode(s.get_state(), store).reshape(q, N, N, N)  # [Q][z][y][x]
    s.step(1)
    g1 = _decode(s.get_state(), store).reshape(q, N, N, N)
    s.close()
    o_tmp = Oracle((4, 4, 4), q, nu=cfg["nu"], dt=cfg["dt"])
    _, Wt = o_tmp.lattice()
    for lo in starts(N, WIN, np.random.default_rng(7)) + CHUNK_WINDOWS:
        zs, ys, xs = slice(lo[2], lo[2] + WIN), slice(lo[1], lo[1] + WIN), slice(lo[0], lo[0] + WIN)
        win0 = g0[:, zs, ys, xs]
        o = Oracle((WIN, WIN, WIN), q, nu=cfg["nu"], dt=cfg["dt"], rt=cfg["rt"], rho0=cfg["rho0"],
                   bcs=window_bcs(lo, WIN, N, cfg["bcs"]))
        o.set_state(win0.reshape(q, -1) + Wt[:, None] * cfg["rho0"], t=3 * cfg["dt"], step=3)
        o.step(1)
        ref = (o.get_state() - Wt[:, None] * cfg["rho0"]).reshape(q, WIN, WIN, WIN)
        sx, sy, sz = compared(lo, WIN, N)
        r = ref[:, sz, sy, sx]
        got = g1[:, zs, ys, xs][:, sz, sy, sx]
        scale = np.abs(g1).max()
        bound = 2e-6 * scale + ulp * np.abs(r)  # FP32 arithmetic + one stored rounding
        assert np.all(np.abs(got - r) <= bound), (lo, np.abs(got - r).max(), scale)
        # the step changed these cells far beyond the FP32 tolerance (the check is not vacuous)
        assert np.abs(r - win0[:, sz, sy, sx]).max() > 100 * 2e-6 * scale, lo


def test_batched_64_channels_full_workload():
    """The benchmark's batched leg at its full size (64 uneven channels, 3.04 M cells, per-cell
    fields, tuned tile, graph replay): three steps from rest, every instance's velocity against
    the oracle run on the whole instance."""
    import torch
    from paper_1411_6121_gb300 import dugks
    specs = W.batched_channels(64, seed=0x1411)
    ins, fields = [], []
    for i, sp in enumerate(specs):
        f64 = W.force_field(sp["shape"], sp["g"][0], seed=1000 + i, rel=0.1)
        fld = torch.tensor(f64, dtype=torch.float32, device="cuda")
        fields.append(fld.cpu().numpy().astype(np.float64))  # the FP32 values the GPU reads
        ins.append(dict(shape=sp["shape"], nu=sp["nu"], bcs=sp["bcs"], field=fld))
    b = dugks.Batch(ins, dt=specs[0]["dt"], stream=torch.cuda.Stream().cuda_stream)
    for i in range(len(ins)):
        b.init(i)
    b.tune()
    b.step(3)
    b.sync()
    worst = 0.0
    for i, sp in enumerate(specs):
        o = Oracle(sp["shape"], 9, nu=sp["nu"], dt=sp["dt"], bcs=sp["bcs"], field=fields[i])
        o.init()
        o.step(3)
        ref = o.moments()[1:]
        got = b.moments(i)[1:].astype(np.float64)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        worst = max(worst, err)
        assert err < 2e-6, (i, sp["shape"], err)
    b.close()
