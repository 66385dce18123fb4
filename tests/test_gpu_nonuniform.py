"""The CUDA path on a non-uniform 2D mesh (the tanh mesh of Sec. 3.4) against the oracle,
element by element, through the C ABI: cavity and channel walls (NEQ and bounce-back), a
pressure-driven channel, a periodic box with a force field, FP32 and FP64 storage, tiles
that leave a ragged tail."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1411_6121_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _sim(**kw):
    from paper_1411_6121_gb300 import dugks
    return dugks.Sim(**kw)


def state_dev(o):
    e, Wt = o.lattice()
    return o.get_state() - Wt[:, None] * o.cfg.rho0


def _dt(faces, dx=1.0):
    w = [np.diff(f).min() for f in faces if f is not None] + ([dx] if any(f is None for f in faces) else [])
    return 0.5 * min(w)


NX, NY = 45, 38
CASES = {
    # both axes on the tanh mesh, moving lid, NEQ walls
    "cavity": dict(shape=(NX, NY), faces=[W.tanh_faces(NX, NX), W.tanh_faces(NY, NY)],
                   bcs=W.cavity_bcs(2, 0.1)),
    # bounce-back box with a moving lid
    "bb_cavity": dict(shape=(NX, NY), faces=[W.tanh_faces(NX, NX), W.tanh_faces(NY, NY)],
                      bcs=[W.bounce_back(), W.bounce_back(), W.bounce_back(), W.bounce_back((0.1, 0.0))]),
    # channel: uniform periodic x, tanh y, body force
    "channel": dict(shape=(40, 21), faces=[None, W.tanh_faces(21, 21)], g=(1e-5, 0.0, 0.0),
                    bcs=W.channel_bcs(2)),
    # pressure inlet and outlet on the tanh x axis, bounce-back and NEQ walls in y
    "pressure": dict(shape=(36, 19), faces=[W.tanh_faces(36, 36), W.tanh_faces(19, 19)], omega=0.3,
                     bcs=[W.pressure(1e-3, 5e-4), W.pressure(-1e-3), W.bounce_back(), W.wall((0.02, 0.0))]),
    # periodic box, non-uniform in both axes, with a force field
    "periodic": dict(shape=(37, 29), faces=[W.tanh_faces(37, 37), W.tanh_faces(29, 29)],
                     g=(1e-5, -2e-5, 0.0), bcs=W.all_periodic()),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("store", [0, 3])
def test_nonuniform_state_elementwise(name, store):
    import torch
    case = dict(CASES[name])
    cfg = dict(q=9, nu=0.04, dt=_dt(case["faces"]), **case)
    p, u = W.random_state_fields(cfg["shape"], seed=sum(map(ord, name)) + 7, u_amp=0.03, p_amp=1e-3)
    field = None
    if name == "periodic":
        # the field is an FP32 input of the C ABI: both sides take the same rounded values
        field = 1e-5 * np.random.default_rng(11).standard_normal((2, cfg["shape"][0] * cfg["shape"][1]))
        field = field.astype(np.float32).astype(np.float64)
    o = Oracle(field=field, **cfg)
    o.init(p=p, u=u)
    o.step(20)
    tf = None if field is None else torch.tensor(field, dtype=torch.float32, device="cuda")
    s = _sim(field=tf, store=store, **cfg)
    s.init(p=p, u=u)
    s.step(20)
    ref = state_dev(o)
    got = s.get_state().astype(np.float64)
    scale = np.abs(ref).max()
    tol = 1e-11 if store == 3 else 2e-6
    assert np.abs(got - ref).max() < tol * scale, (np.abs(got - ref).max(), scale)
    # the uniform scheme on the same input differs far beyond the tolerance
    if store == 3:
        cfg_u = {k: v for k, v in cfg.items() if k != "faces"}
        ou = Oracle(field=field, **cfg_u)
        ou.init(p=p, u=u)
        ou.step(20)
        assert np.abs(state_dev(ou) - ref).max() > 1e3 * tol * scale


def test_nonuniform_tile_16x8_matches_32x8():
    case = CASES["cavity"]
    cfg = dict(q=9, nu=0.04, dt=_dt(case["faces"]), store=3, **case)
    p, u = W.random_state_fields(cfg["shape"], seed=5, u_amp=0.03, p_amp=1e-3)
    out = []
    for tile in [(32, 8), (16, 8)]:
        s = _sim(tile=tile, **cfg)
        s.init(p=p, u=u)
        s.step(10)
        out.append(s.get_state())
    assert np.array_equal(out[0], out[1])


def test_nonuniform_couette_exact_on_gpu():
    """Plane Couette flow is linear in y, which the scheme reproduces exactly on any mesh."""
    ny = 16
    yf = W.tanh_faces(ny, ny)
    dt = _dt([None, yf])
    s = _sim(shape=(8, ny), q=9, nu=0.2, dt=dt, faces=[None, yf], store=3,
             bcs=[W.periodic(), W.periodic(), W.wall(), W.wall((0.05, 0.0))])
    s.init()
    s.step(int(4000 / dt))
    yc = 0.5 * (yf[1:] + yf[:-1])
    u = s.moments()[1].reshape(ny, 8)[:, 0].astype(np.float64)
    assert np.abs(u - 0.05 * yc / ny).max() < 1e-7  # moments are FP32 output


@pytest.mark.parametrize("store", [0, 3])
def test_nonuniform_original_model(store):
    """The original DUGKS (eq. (5)) on the tanh mesh: the model switch and the mesh metrics
    together, against the oracle with both."""
    case = CASES["cavity"]
    cfg = dict(q=9, nu=0.04, dt=_dt(case["faces"]), **case)
    p, u = W.random_state_fields(cfg["shape"], seed=77, u_amp=0.08, p_amp=3e-3)
    o = Oracle(model=1, **cfg)
    o.init(p=p, u=u)
    o.step(15)
    s = _sim(store=store, model=1, **cfg)
    s.init(p=p, u=u)
    s.step(15)
    ref = state_dev(o)
    tol = 1e-11 if store == 3 else 2e-6
    assert np.abs(s.get_state().astype(np.float64) - ref).max() < tol * np.abs(ref).max()
    # the incompressible model gives a different state on the same input (about 1%)
    o0 = Oracle(**cfg)
    o0.init(p=p, u=u)
    o0.step(15)
    assert np.abs(state_dev(o0) - ref).max() > 100 * tol * np.abs(ref).max()


def test_nonuniform_handle_has_no_adjoint():
    from paper_1411_6121_gb300 import dugks
    case = CASES["channel"]
    s = _sim(q=9, nu=0.04, dt=_dt(case["faces"]), **case)
    s.init()
    with pytest.raises(dugks.DugksError) as e:
        s.record(10, 5)
    assert e.value.code == -7 and "uniform meshes only" in str(e.value)  # DUGKS_E_UNSUPPORTED


# ---- 3D: the cube of Sec. 3.5 on the same tanh law, D3Q19 and D3Q27 -----------------------

CASES_3D = {
    # graded on every axis, moving lid, NEQ walls on all six faces
    "cavity": dict(shape=(37, 21, 13), faces=[W.tanh_faces(37, 37), W.tanh_faces(21, 21), W.tanh_faces(13, 13)],
                   bcs=W.cavity_bcs(3, 0.1)),
    # bounce-back walls in x and y, NEQ velocity walls in z, one moving
    "bb_box": dict(shape=(34, 19, 11), faces=[W.tanh_faces(34, 34), None, W.tanh_faces(11, 11)],
                   bcs=[W.bounce_back(), W.bounce_back(), W.bounce_back(), W.bounce_back((0.1, 0.0, 0.02)),
                        W.wall(), W.wall((0.0, 0.03, 0.0))]),
    # pressure inlet and outlet along the graded x axis, NEQ walls in y, periodic graded z
    "pressure": dict(shape=(35, 10, 9), faces=[W.tanh_faces(35, 35), W.tanh_faces(10, 10), W.tanh_faces(9, 9)],
                     bcs=[W.pressure(1e-3), W.pressure(-1e-3), W.wall(), W.wall(), W.periodic(), W.periodic()]),
    # periodic box graded on every axis, with a force field
    "periodic": dict(shape=(33, 12, 10), faces=[W.tanh_faces(33, 33), W.tanh_faces(12, 12), W.tanh_faces(10, 10)],
                     g=(1e-5, -2e-5, 1e-5), bcs=W.all_periodic()),
}


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("name", sorted(CASES_3D))
@pytest.mark.parametrize("store", [0, 3])
def test_nonuniform_3d_state_elementwise(name, q, store):
    import torch
    case = dict(CASES_3D[name])
    cfg = dict(q=q, nu=0.04, dt=_dt(case["faces"]), **case)
    p, u = W.random_state_fields(cfg["shape"], seed=sum(map(ord, name)) + q, u_amp=0.03, p_amp=1e-3)
    field = None
    if name == "periodic":
        n = int(np.prod(cfg["shape"]))
        field = (1e-5 * np.random.default_rng(12).standard_normal((3, n))).astype(np.float32).astype(np.float64)
    o = Oracle(field=field, **cfg)
    o.init(p=p, u=u)
    o.step(8)
    tf = None if field is None else torch.tensor(field, dtype=torch.float32, device="cuda")
    s = _sim(field=tf, store=store, **cfg)
    s.init(p=p, u=u)
    s.step(8)
    ref = state_dev(o)
    got = s.get_state().astype(np.float64)
    scale = np.abs(ref).max()
    tol = 1e-11 if store == 3 else 2e-6
    assert np.abs(got - ref).max() < tol * scale, (np.abs(got - ref).max(), scale)
    if store == 3:  # the uniform scheme on the same input differs far beyond the tolerance
        cfg_u = {k: v for k, v in cfg.items() if k != "faces"}
        ou = Oracle(field=field, **cfg_u)
        ou.init(p=p, u=u)
        ou.step(8)
        assert np.abs(state_dev(ou) - ref).max() > 1e3 * tol * scale


def test_nonuniform_3d_couette_exact_on_gpu():
    """Couette flow between graded y walls moving along x and z, with a graded periodic z axis:
    linear in y to the FP32 output's rounding."""
    ny, nz = 12, 6
    yf, zf = W.tanh_faces(ny, ny), W.tanh_faces(nz, nz)
    dt = _dt([None, yf, zf])
    s = _sim(shape=(4, ny, nz), q=19, nu=0.2, dt=dt, faces=[None, yf, zf], store=3,
             bcs=[W.periodic(), W.periodic(), W.wall(), W.wall((0.05, 0.0, 0.02)), W.periodic(), W.periodic()])
    s.init()
    s.step(int(3000 / dt))
    yc = 0.5 * (yf[1:] + yf[:-1])
    m = s.moments().astype(np.float64)
    ux = m[1].reshape(nz, ny, 4)
    uz = m[3].reshape(nz, ny, 4)
    assert np.abs(ux - (0.05 * yc / ny)[None, :, None]).max() < 1e-7
    assert np.abs(uz - (0.02 * yc / ny)[None, :, None]).max() < 1e-7
