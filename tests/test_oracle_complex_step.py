"""Pins of the oracle's complex-step build (its derivative, used to check the adjoint).

The complex-step build runs the same Appendix algorithm on double _Complex values; its
imaginary part must equal the derivative that central finite differences of the real
build approximate, and must be linear in the perturbation direction.
"""
import numpy as np

from oracle import Oracle
from paper_1411_6121_gb300 import workloads as W


def _setup(cs):
    shape = (4, 6)
    p, u = W.random_state_fields(shape, seed=21, u_amp=0.03, p_amp=1e-3)
    field = W.force_field(shape, 1e-4, seed=22, rel=0.5)
    bcs = [W.periodic(), W.periodic(), W.wall(), W.wall((0.02, 0.0, 0.0))]
    o = Oracle(shape, 9, nu=0.05, dt=0.5, bcs=bcs, field=field, complex_step=cs)
    o.init(p=p, u=u)
    return o, field


def test_complex_step_matches_central_differences():
    eps = 1e-20
    rng = np.random.default_rng(5)
    o, field = _setup(True)
    f0 = o.get_state()
    v = rng.standard_normal(f0.shape)
    vg = rng.standard_normal(field.shape)
    vw = np.zeros(18)
    vw[9] = 1.0  # +y wall, u_x
    o.set_state(f0, eps * v)
    o.set_field_im(eps * vg)
    o.set_wall_u_im(eps * vw)
    o.step(5)
    _, dm = o.moments(imag=True)
    jv = dm / eps
    # central differences on the real build
    h = 1e-6
    out = []
    for s in (+1, -1):
        r, _ = _setup(False)
        r.set_state(f0 + s * h * v)
        r.set_field(field + s * h * vg)
        bcs = [W.periodic(), W.periodic(), W.wall(), W.wall((0.02 + s * h, 0.0, 0.0))]
        r2 = Oracle((4, 6), 9, nu=0.05, dt=0.5, bcs=bcs, field=field + s * h * vg)
        r2.set_state(f0 + s * h * v, t=0.0, step=0)
        r2.step(5)
        out.append(r2.moments())
    fd = (out[0] - out[1]) / (2 * h)
    assert np.abs(jv - fd).max() < 1e-6 * np.abs(jv).max()
    # real part unaffected by the perturbation direction
    base, _ = _setup(False)
    base.step(5)
    m_cs, _ = o.moments(imag=True)
    assert np.abs(m_cs - base.moments()).max() < 1e-15


def test_complex_step_is_linear():
    eps = 1e-20
    rng = np.random.default_rng(6)
    res = []
    o, _ = _setup(True)
    f0 = o.get_state()
    v1 = rng.standard_normal(f0.shape)
    v2 = rng.standard_normal(f0.shape)
    for v in (v1, v2, 2.0 * v1 - 3.0 * v2):
        o2, _ = _setup(True)
        o2.set_state(f0, eps * v)
        o2.step(3)
        res.append(o2.moments(imag=True)[1] / eps)
    assert np.abs(res[2] - (2 * res[0] - 3 * res[1])).max() < 1e-12 * np.abs(res[2]).max()
