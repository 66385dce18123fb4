"""Batched form: many independent D2Q9 instances in one persistent launch per step.

Each instance must evolve exactly as the same instance run alone through the
single-instance API (same kernel code per tile, so the results are bit-identical), and as
the FP64 oracle within the FP32 tolerance of the parity tests. The tile autotuner must leave
the batch's state and clock as it found them.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1411_6121_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _instances():
    import torch
    fld = torch.tensor(W.force_field((50, 26), 2e-5, seed=5, rel=0.5), dtype=torch.float32, device="cuda")
    return [
        dict(shape=(33, 17), nu=0.02, g=(1e-5, 0.0, 0.0), bcs=W.channel_bcs(2)),
        dict(shape=(64, 32), nu=0.05, g=(2e-5, 0.0, 0.0), bcs=W.channel_bcs(2)),
        dict(shape=(40, 21), nu=0.04, bcs=W.cavity_bcs(2, 0.08)),
        dict(shape=(32, 16), nu=0.03, bcs=[W.pressure(1e-3), W.pressure(-1e-3), W.wall(), W.wall()]),
        dict(shape=(50, 26), nu=0.06, g=(1e-5, 0.0, 0.0), omega=0.02, field=fld, bcs=W.channel_bcs(2)),
        dict(shape=(31, 18), nu=0.03, g=(1e-5, 0.0, 0.0),
             bcs=[W.periodic(), W.periodic(), W.bounce_back(), W.bounce_back((0.02, 0.0))]),
    ]


def _single(ins, steps, p, u, batch_tile):
    """The instance alone, through the single-instance API with the same tile body: the
    throughput kernel (batch tiles 30 x (rows - 2)) or the reference kernel."""
    from paper_1411_6121_gb300 import dugks
    kw = {k: v for k, v in ins.items()}
    tx, ty = batch_tile
    if tx == 30:
        s = dugks.Sim(q=9, dt=0.5, tile=(32, ty + 2), kernel=0, **kw)
    else:
        s = dugks.Sim(q=9, dt=0.5, tile=(16, 8) if (tx, ty) == (16, 8) else (32, 8), kernel=1, **kw)
    s.init(p=p, u=u)
    s.step(steps)
    m = s.moments()
    s.close()
    return m


@pytest.mark.parametrize("tile", [(30, 6), (30, 14), (30, 2), (32, 8), (64, 4)])
def test_batch_matches_single_instances_and_oracle(tile):
    from paper_1411_6121_gb300 import dugks
    ins = _instances()
    b = dugks.Batch(ins, dt=0.5, tile=tile)
    fields = []
    for i, d in enumerate(ins):
        p, u = W.random_state_fields(d["shape"], seed=10 + i, u_amp=0.02, p_amp=1e-4)
        fields.append((p, u))
        b.init(i, p=p, u=u)
    b.step(3)
    b.step(57)
    for i, d in enumerate(ins):
        got = b.moments(i)
        ref = _single(d, 60, *fields[i], tile)
        assert np.array_equal(got, ref), (tile, i)
    # three instances against the oracle (the last one has bounce-back walls)
    for i in (0, 3, 5):
        d = ins[i]
        o = Oracle(d["shape"], 9, nu=d["nu"], dt=0.5, g=d.get("g", (0, 0, 0)), bcs=d["bcs"])
        o.init(*fields[i])
        o.step(60)
        ref = o.moments()
        got = b.moments(i).astype(np.float64)
        err = np.linalg.norm(got[1:] - ref[1:]) / np.linalg.norm(ref[1:])
        assert err < 2e-6, (i, err)
    assert b.launch_count() == 60 * 2  # one launch per step plus the clock for omega != 0
    b.close()


def test_batch_tuner_restores_state():
    from paper_1411_6121_gb300 import dugks
    ins = _instances()[:4]
    b = dugks.Batch(ins, dt=0.5)
    for i in range(len(ins)):
        b.init(i, *W.random_state_fields(ins[i]["shape"], seed=20 + i, u_amp=0.02, p_amp=1e-4))
    b.step(10)
    before = [b.moments(i) for i in range(len(ins))]
    tx, ty = b.tune()
    assert (tx, ty) in [(30, 6), (30, 14), (30, 2), (32, 8), (16, 8), (32, 4), (64, 4)]
    after = [b.moments(i) for i in range(len(ins))]
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    # the tuned tile runs the same scheme
    b.step(20)
    for i in range(len(ins)):
        p, u = W.random_state_fields(ins[i]["shape"], seed=20 + i, u_amp=0.02, p_amp=1e-4)
        ref = _single(ins[i], 30, p, u, (tx, ty))
        got = b.moments(i)
        assert np.array_equal(got, ref), ((tx, ty), i)
    b.close()
