"""Pins of the oracle on a non-uniform mesh (Sec. 3.4's tanh mesh, reading R18), by what
the scheme fixes exactly:
  * a uniform mesh given by its interface coordinates takes the general formulas and must
    reproduce the uniform path bit for bit (every weight reduces to 1/2, every distance to dx);
  * plane Couette flow is linear, which the linear reconstruction on any mesh reproduces
    exactly (NEQ and bounce-back walls);
  * the interface fluxes telescope with the cells' interface areas, so a periodic box keeps
    its volume-weighted mass to rounding;
  * force-driven Poiseuille flow on the tanh mesh converges at second order;
  * the mesh of Sec. 3.4 runs from 0 to 1, symmetric, finest at the walls.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1411_6121_gb300 import workloads as W


def test_tanh_mesh_of_the_paper():
    z = W.tanh_faces(16)
    assert abs(z[0]) < 1e-15 and abs(z[-1] - 1.0) < 1e-15
    assert np.allclose(z + z[::-1], 1.0, atol=1e-15)
    dz = np.diff(z)
    assert dz[0] == dz.min() and dz[8] == dz.max() and dz[0] < 0.5 * dz[8]


def test_uniform_mesh_by_coordinates_is_bitwise_uniform():
    cfg = dict(shape=(12, 10), q=9, nu=0.05, dt=0.5, g=(1e-4, 2e-5, 0.0), bcs=W.cavity_bcs(2, 0.08))
    p, u = W.random_state_fields(cfg["shape"], seed=3, u_amp=0.03, p_amp=1e-3)
    a = Oracle(**cfg)
    a.init(p=p, u=u)
    a.step(30)
    b = Oracle(faces=[np.arange(13) * 1.0, np.arange(11) * 1.0], **cfg)
    b.init(p=p, u=u)
    b.step(30)
    assert np.array_equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("wall", [W.wall, W.bounce_back])
def test_couette_exact_on_tanh_mesh(wall):
    ny = 8
    yf = W.tanh_faces(ny, ny)
    dt = 0.5 * np.diff(yf).min()
    o = Oracle((4, ny), 9, nu=0.2, dt=dt, faces=[None, yf],
               bcs=[W.periodic(), W.periodic(), wall(), wall((0.05, 0.0))])
    o.init()
    o.step(int(3000 / dt))
    yc = 0.5 * (yf[1:] + yf[:-1])
    u = o.moments()[1].reshape(ny, 4)[:, 0]
    assert np.abs(u - 0.05 * yc / ny).max() < 1e-13


def test_mass_on_periodic_nonuniform_mesh():
    xf, yf = W.tanh_faces(10, 10), W.tanh_faces(9, 9)
    dt = 0.5 * min(np.diff(xf).min(), np.diff(yf).min())
    o = Oracle((10, 9), 9, nu=0.05, dt=dt, faces=[xf, yf], bcs=W.all_periodic())
    o.init(*W.random_state_fields((10, 9), seed=5, u_amp=0.03, p_amp=1e-3))
    vol = np.outer(np.diff(yf), np.diff(xf)).ravel()
    m0 = np.sum(o.moments()[0] * vol)
    o.step(100)
    assert abs(np.sum(o.moments()[0] * vol) - m0) / vol.sum() < 1e-13


def _poiseuille_tanh(ny, wall):
    nu, umax = 0.1, 0.05
    yf = W.tanh_faces(ny, ny)
    G = 8 * nu * umax / ny ** 2
    dt = 0.5 * np.diff(yf).min()
    o = Oracle((2, ny), 9, nu=nu, dt=dt, faces=[None, yf], g=(G, 0.0),
               bcs=[W.periodic(), W.periodic(), wall(), wall()])
    o.init()
    o.step(int(6 * ny * ny / nu / dt))
    yc = 0.5 * (yf[1:] + yf[:-1])
    u = o.moments()[1].reshape(ny, 2)[:, 0] - 0.5 * dt * G  # the reported u carries + G dt/2
    ua = G / (2 * nu) * yc * (ny - yc)
    return np.linalg.norm(u - ua) / np.linalg.norm(ua)


@pytest.mark.parametrize("wall", [W.wall, W.bounce_back])
def test_poiseuille_second_order_on_tanh_mesh(wall):
    e8, e16 = _poiseuille_tanh(8, wall), _poiseuille_tanh(16, wall)
    assert 1.85 < np.log2(e8 / e16) < 2.2, (e8, e16)


# ---- the same pins in 3D (the paper refines the cube of Sec. 3.5 with the same tanh law) ----

@pytest.mark.parametrize("q", [19, 27])
def test_uniform_mesh_by_coordinates_is_bitwise_uniform_3d(q):
    cfg = dict(shape=(8, 7, 6), q=q, nu=0.05, dt=0.5, g=(1e-4, 2e-5, -3e-5), bcs=W.cavity_bcs(3, 0.08))
    p, u = W.random_state_fields(cfg["shape"], seed=13, u_amp=0.03, p_amp=1e-3)
    a = Oracle(**cfg)
    a.init(p=p, u=u)
    a.step(10)
    b = Oracle(faces=[np.arange(9) * 1.0, np.arange(8) * 1.0, np.arange(7) * 1.0], **cfg)
    b.init(p=p, u=u)
    b.step(10)
    assert np.array_equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("wall", [W.wall, W.bounce_back])
@pytest.mark.parametrize("q", [19, 27])
def test_couette_exact_on_tanh_mesh_3d(q, wall):
    """Walls graded in y; the periodic z axis graded too (the flow does not vary along it, so
    its interpolations must reproduce constants); the wall moves along x and z."""
    ny, nz = 8, 4
    yf, zf = W.tanh_faces(ny, ny), W.tanh_faces(nz, nz)
    dt = 0.5 * min(np.diff(yf).min(), np.diff(zf).min())
    o = Oracle((3, ny, nz), q, nu=0.2, dt=dt, faces=[None, yf, zf],
               bcs=[W.periodic(), W.periodic(), wall(), wall((0.05, 0.0, 0.02)), W.periodic(), W.periodic()])
    o.init()
    o.step(int(3000 / dt))
    yc = 0.5 * (yf[1:] + yf[:-1])
    m = o.moments()
    ux = m[1].reshape(nz, ny, 3)
    uz = m[3].reshape(nz, ny, 3)
    assert np.abs(ux - (0.05 * yc / ny)[None, :, None]).max() < 1e-13
    assert np.abs(uz - (0.02 * yc / ny)[None, :, None]).max() < 1e-13
    assert np.abs(m[2]).max() < 1e-13


@pytest.mark.parametrize("q", [19, 27])
def test_mass_on_periodic_nonuniform_mesh_3d(q):
    xf, yf, zf = W.tanh_faces(6, 6), W.tanh_faces(5, 5), W.tanh_faces(4, 4)
    dt = 0.5 * min(np.diff(xf).min(), np.diff(yf).min(), np.diff(zf).min())
    o = Oracle((6, 5, 4), q, nu=0.05, dt=dt, faces=[xf, yf, zf], bcs=W.all_periodic())
    o.init(*W.random_state_fields((6, 5, 4), seed=9, u_amp=0.03, p_amp=1e-3))
    vol = (np.diff(zf)[:, None, None] * np.diff(yf)[None, :, None] * np.diff(xf)[None, None, :]).ravel()
    m0 = np.sum(o.moments()[0] * vol)
    o.step(60)
    assert abs(np.sum(o.moments()[0] * vol) - m0) / vol.sum() < 1e-13


def _poiseuille_tanh_3d(ny):
    nu, umax = 0.1, 0.05
    yf, zf = W.tanh_faces(ny, ny), W.tanh_faces(2, 2)
    G = 8 * nu * umax / ny ** 2
    dt = 0.5 * min(np.diff(yf).min(), np.diff(zf).min())
    o = Oracle((2, ny, 2), 19, nu=nu, dt=dt, faces=[None, yf, zf], g=(G, 0.0, 0.0),
               bcs=[W.periodic(), W.periodic(), W.wall(), W.wall(), W.periodic(), W.periodic()])
    o.init()
    o.step(int(6 * ny * ny / nu / dt))
    yc = 0.5 * (yf[1:] + yf[:-1])
    u = o.moments()[1].reshape(2, ny, 2)[0, :, 0] - 0.5 * dt * G  # the reported u carries + G dt/2
    ua = G / (2 * nu) * yc * (ny - yc)
    return np.linalg.norm(u - ua) / np.linalg.norm(ua)


def test_poiseuille_second_order_on_tanh_mesh_3d():
    e8, e16 = _poiseuille_tanh_3d(8), _poiseuille_tanh_3d(16)
    assert 1.85 < np.log2(e8 / e16) < 2.2, (e8, e16)
