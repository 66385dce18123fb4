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
    """The original DUGKS (eq. feq) on the tanh mesh: the model switch and the mesh metrics
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
