"""Writes channel_8x32_oracle.txt: the FP64 oracle on the force-driven channel of 8 x 32 cells
(periodic x, NEQ no-slip walls, nu = 0.01, G = 1e-5, CFL 0.5 in lattice units, from rest) run
to the steady criterion of Sec. 3.1 with K = 1000 and the tolerance 1e-10, with its steady
profile and its error against the parabola of Sec. 3.2. Calls only the oracle.

    python tests/golden/make_channel_8x32.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import Oracle  # noqa: E402
from oracle.oracle import rel_change  # noqa: E402
from paper_1411_6121_gb300 import workloads as W  # noqa: E402

H, NU, G = 32, 0.01, 1e-5


def main():
    cfg = W.channel_8x32()
    o = Oracle(cfg["shape"], cfg["q"], nu=cfg["nu"], dt=cfg["dt"], g=cfg["g"], bcs=cfg["bcs"])
    o.init()
    prev, n = o.moments()[1:], 0
    while True:
        o.step(1000)
        n += 1000
        m = o.moments()
        if rel_change(m[1:], prev) < 1e-10:
            break
        prev = m[1:]
    y = (np.arange(H) + 0.5)
    ua = G / (2 * NU) * y * (H - y)
    ux = o.grid(m[1])[:, 0]
    err = np.linalg.norm(ux - ua) / np.linalg.norm(ua)
    with open(os.path.join(HERE, "channel_8x32_oracle.txt"), "w") as f:
        f.write("# FP64 oracle, force-driven channel 8 x 32 (nu = 0.01, G = 1e-5, dt = 0.5, RT = 1/3), from rest,\n")
        f.write("# run to rel. velocity change < 1e-10 per 1000 steps (Sec. 3.1 criterion); written by\n")
        f.write("# tests/golden/make_channel_8x32.py (oracle only)\n")
        f.write("steps %d\n" % n)
        f.write("parabola_error %.9e\n" % err)
        f.write("u_x " + " ".join("%.12e" % v for v in ux) + "\n")


if __name__ == "__main__":
    main()
