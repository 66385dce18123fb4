"""What storage precision alone costs, measured on the oracle (FP64 arithmetic) with its state
rounded after every step, stored as the deviation from the rest equilibrium like the CUDA path:
  * FP32: within 1e-7 of the exact oracle after 1000 steps (velocity, relative L2) on the
    channel, cavity and pressure-driven cases, so the 1e-6 bar is within reach of FP32 storage
    and a larger FP32 error comes from the arithmetic. The pressure, about 30 times smaller
    than the stored values, already moves by 1e-7 to 1e-6 (measured 4.6e-7 and 4.8e-7 on the
    cavity and the pressure-driven case): FP32 storage alone takes about half of a 1e-6
    pressure budget;
  * BF16: above 1e-3 even with stochastic rounding, so that bar is out of reach of the format."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1411_6121_gb300 import workloads as W

CASES = {
    "channel": dict(shape=(40, 21), q=9, nu=0.02, dt=0.5, g=(1e-5, 0.0, 0.0), bcs=W.channel_bcs(2)),
    "cavity": dict(shape=(45, 38), q=9, nu=0.05, dt=0.5, bcs=W.cavity_bcs(2, 0.1)),
    "pressure": dict(shape=(36, 19), q=9, nu=0.04, dt=0.5,
                     bcs=[W.pressure(1e-3), W.pressure(-1e-3), W.wall(), W.wall()]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp32_storage_rounding_alone(name):
    cfg = CASES[name]
    exact = Oracle(**cfg)
    exact.init()
    exact.step(1000)
    r = Oracle(**cfg)
    r.init()
    _, Wt = r.lattice()
    rest = Wt[:, None] * r.cfg.rho0
    for _ in range(1000):
        r.step(1)
        g = (r.get_state() - rest).astype(np.float32).astype(np.float64)
        r.set_state(g + rest)
    m, me = r.moments(), exact.moments()
    err = np.linalg.norm(m[1:] - me[1:]) / np.linalg.norm(me[1:])
    assert 0.0 < err < 1e-7, err
    if name != "channel":  # the force-driven channel from rest has p ~ 0
        ep = np.linalg.norm(m[0] - me[0]) / np.linalg.norm(me[0])
        assert 1e-7 < ep < 1e-6, ep


def _bf16(x, rng=None):
    """x rounded to bfloat16 (returned as float64): to nearest even, or stochastically (the
    discarded 16 bits compared with a uniform random 16-bit draw) when rng is given."""
    b = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    if rng is None:
        b = b + 0x7FFF + ((b >> 16) & 1)
    else:
        b = b + rng.integers(0, 1 << 16, size=b.shape, dtype=np.uint64)
    return ((b >> 16) << 16).astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("name", ["cavity", "channel"])
def test_bf16_storage_alone_exceeds_1e3(name):
    """BF16 storage (8 significant bits) alone, with the stochastic rounding the CUDA path
    uses, moves the velocity after 1000 steps by more than 1e-3 from the exact oracle (the
    GPU's BF16 2D cavity: 3.3e-3), so the 1e-3 bar is out of reach for that format whatever the
    arithmetic; rounding to nearest instead is several times worse still."""
    cfg = CASES[name]
    exact = Oracle(**cfg)
    exact.init()
    exact.step(1000)
    ue = exact.moments()[1:]
    errs = []
    for rng in (np.random.default_rng(1), None):
        r = Oracle(**cfg)
        r.init()
        _, Wt = r.lattice()
        rest = Wt[:, None] * r.cfg.rho0
        for _ in range(1000):
            r.step(1)
            r.set_state(_bf16(r.get_state() - rest, rng) + rest)
        errs.append(np.linalg.norm(r.moments()[1:] - ue) / np.linalg.norm(ue))
    sr, rne = errs
    assert 1e-3 < sr < 2e-2, sr
    assert rne > 5 * sr, (rne, sr)


@pytest.mark.slow
def test_fp32_storage_floor_at_steady_channel():
    """At a steady state FP32 storage costs far more than after 1000 steps: the stored deviation
    rounds the small non-equilibrium part that carries the viscous stress, and a steady state
    repeats those roundings at every step. The 8 x 32 channel (nu = 0.01, G = 1e-5, from rest,
    416,000 steps: the oracle's steady state at 1e-10) with its state rounded to FP32 every step
    settles 3.2e-4 from the exact steady profile (golden file of the exact one)."""
    import os
    cfg = W.channel_8x32()
    o = Oracle(cfg["shape"], 9, nu=cfg["nu"], dt=cfg["dt"], g=cfg["g"], bcs=cfg["bcs"])
    o.init()
    _, Wt = o.lattice()
    rest = Wt[:, None] * o.cfg.rho0
    gold = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "channel_8x32_oracle.txt")):
        if not line.startswith("#"):
            k, *v = line.split()
            gold[k] = v
    uo = np.array([float(v) for v in gold["u_x"]])
    for _ in range(int(gold["steps"][0])):
        o.step(1)
        o.set_state((o.get_state() - rest).astype(np.float32).astype(np.float64) + rest)
    ux = o.grid(o.moments()[1])[:, 0]
    err = np.linalg.norm(ux - uo) / np.linalg.norm(uo)
    assert 1e-4 < err < 1e-3, err  # measured 3.2e-4
