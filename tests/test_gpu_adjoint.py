"""The adjoint (dugks_record / dugks_adjoint) against the FP64 oracle.

The loss is a weighted sum of the final moments, L = sum w . m(T) (any loss of the final
moments has this as its linearisation, with w = dL/dm). The library's reverse sweep gives
dL/dfield, dL/du_wall and dL/dstate0 through the transposed step. They are checked
  * exactly (to rounding) against the oracle's complex-step build, which carries the
    derivative of the Appendix algorithm along one input direction per run: every field
    component and wall-velocity component on a tiny grid, and random state directions;
  * against central finite differences of the real oracle (a second-order estimate;
    relative 1e-4), on sampled cells, for FP64 and FP32 storage;
  * for invariance under the checkpoint interval (bitwise: the recompute is deterministic).
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1411_6121_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EPS_CS = 1e-20  # complex-step size


def _torch():
    import torch
    return torch


def _sim(**kw):
    from paper_1411_6121_gb300 import dugks
    return dugks.Sim(**kw)


# tiny grids: every boundary kind of the adjoint (periodic seams, NEQ velocity walls with a
# moving lid, a pressure wall, bounce-back walls, corners), a field, a time-dependent G
CASES = {
    "channel_lid": dict(shape=(6, 5), q=9, nu=0.05, dt=0.5, g=(2e-5, 0.0, 0.0),
                        bcs=[W.periodic(), W.periodic(), W.wall(), W.wall((0.03, 0.0, 0.0))]),
    "cavity": dict(shape=(5, 6), q=9, nu=0.04, dt=0.5, bcs=W.cavity_bcs(2, 0.05)),
    "pressure_oscillating": dict(shape=(6, 4), q=9, nu=0.06, dt=0.5, g=(1e-4, -3e-5, 0.0), omega=0.07,
                                 bcs=[W.pressure(2e-3, 1.5e-3), W.pressure(-1e-3), W.wall((0.0, 0.01, 0.0)), W.wall()]),
    "periodic": dict(shape=(5, 4), q=9, nu=0.05, dt=0.5, g=(1e-5, 2e-5, 0.0), bcs=W.all_periodic()),
    # wide enough for interior cells and interfaces (the kernels' fast path) beside the
    # boundary ones
    "channel_wide": dict(shape=(12, 9), q=9, nu=0.05, dt=0.5, g=(2e-5, 0.0, 0.0), omega=0.05,
                         bcs=[W.periodic(), W.periodic(), W.wall(), W.wall((0.03, 0.0, 0.0))]),
    "periodic_wide": dict(shape=(10, 8), q=9, nu=0.04, dt=0.5, g=(1e-5, 2e-5, 0.0), bcs=W.all_periodic()),
    "cavity_wide": dict(shape=(9, 10), q=9, nu=0.04, dt=0.5,
                        bcs=[W.wall(), W.pressure(-1e-3), W.wall(), W.wall((0.05, 0.0, 0.0))]),
    # bounce-back walls (eq. (31)): a moving one, and beside NEQ walls
    "bb_channel": dict(shape=(6, 5), q=9, nu=0.05, dt=0.5, g=(2e-5, 0.0, 0.0),
                       bcs=[W.periodic(), W.periodic(), W.bounce_back(), W.bounce_back((0.03, 0.0, 0.0))]),
    "bb_cavity_wide": dict(shape=(9, 10), q=9, nu=0.04, dt=0.5, g=(1e-5, 0.0, 0.0),
                           bcs=[W.bounce_back((0.0, 0.01, 0.0)), W.bounce_back(), W.wall(),
                                W.bounce_back((0.05, 0.0, 0.0))]),
}
STEPS = 12


def _inputs(cfg, seed):
    shape = cfg["shape"]
    p, u = W.random_state_fields(shape, seed=seed, u_amp=0.03, p_amp=1e-3)
    rng = np.random.default_rng(seed + 1)
    field = 2e-4 * rng.standard_normal((2, int(np.prod(shape))))
    # dL/dm enters the library as float32: both sides use the same rounded weights
    w = rng.standard_normal((3, int(np.prod(shape)))).astype(np.float32).astype(np.float64)
    return p, u, field, w


def _gpu_grads(cfg, p, u, field, w, store, steps=STEPS, every=5):
    torch = _torch()
    tf = torch.tensor(field, dtype=torch.float32, device="cuda")
    s = _sim(field=tf, store=store, **cfg)
    s.init(p=p, u=u)
    s.record(steps, every)
    m = s.moments()
    wt = torch.tensor(w, dtype=torch.float32, device="cuda")
    dfield, dwall, dstate = s.adjoint(wt, field_grad=True, state_grad=True)
    return m, dfield.double().cpu().numpy(), dwall, dstate.double().cpu().numpy()


def _oracle_cs(cfg, p, u, field32, w, steps, field_dir=None, wall_dir=None, state_dir=None):
    """<w, d m(T)> along one input direction (complex step of the oracle)."""
    o = Oracle(field=field32, complex_step=True, **cfg)
    o.init(p=p, u=u)
    if state_dir is not None:
        o.set_state(o.get_state(), EPS_CS * state_dir, t=0.0, step=0)
    if field_dir is not None:
        o.set_field_im(EPS_CS * field_dir)
    if wall_dir is not None:
        o.set_wall_u_im(EPS_CS * wall_dir)
    o.step(steps)
    _, im = o.moments(imag=True)
    return float(np.sum(w * im) / EPS_CS)


@pytest.mark.parametrize("case", sorted(CASES))
def test_adjoint_equals_oracle_complex_step(case):
    cfg = CASES[case]
    p, u, field, w = _inputs(cfg, seed=101 + len(case))
    # the GPU reads the field as float32: give the oracle the same values
    field32 = field.astype(np.float32).astype(np.float64)
    _, dfield, dwall, dstate = _gpu_grads(cfg, p, u, field32, w, store=3)
    n = int(np.prod(cfg["shape"]))
    ref = np.zeros((2, n))
    for a in range(2):
        for c in range(n):
            d = np.zeros((2, n))
            d[a, c] = 1.0
            ref[a, c] = _oracle_cs(cfg, p, u, field32, w, STEPS, field_dir=d)
    scale = np.abs(ref).max()
    err = np.abs(dfield - ref).max() / scale
    # dL/dfield is converted to float32 at the end of the sweep
    assert err < 1e-6, "dL/dfield: max rel err %.3e (worst cell %s)" % (
        err, np.unravel_index(np.argmax(np.abs(dfield - ref)), ref.shape))
    # wall velocities: every velocity-wall face, tangential and normal component
    wref = np.zeros((6, 3))
    for f in range(4):
        if cfg["bcs"][f][0] not in (W.BC_NEQ_VELOCITY, W.BC_BOUNCE_BACK):
            continue
        for a in range(2):
            d = np.zeros(18)
            d[3 * f + a] = 1.0
            wref[f, a] = _oracle_cs(cfg, p, u, field32, w, STEPS, wall_dir=d)
    if np.abs(wref).max() > 0:
        werr = np.abs(dwall - wref).max() / np.abs(wref).max()
        assert werr < 1e-9, "dL/du_wall: rel err %.3e\n%s\n%s" % (werr, dwall, wref)
    else:
        assert np.all(dwall == 0.0)
    # initial state: random directions (dot-product test <dL/dg0, v> = d/de L(g0 + e v))
    rng = np.random.default_rng(7)
    for _ in range(3):
        v = rng.standard_normal(dstate.shape)
        r = _oracle_cs(cfg, p, u, field32, w, STEPS, state_dir=v)
        assert abs(np.sum(dstate * v) - r) <= 1e-9 * max(abs(r), np.abs(dstate).sum()), (np.sum(dstate * v), r)


def _loss_oracle(cfg, p, u, field, w, steps):
    o = Oracle(field=field, **cfg)
    o.init(p=p, u=u)
    o.step(steps)
    return float(np.sum(w * o.moments()))


@pytest.mark.parametrize("store", [3, 0])
@pytest.mark.parametrize("case", ["channel_lid", "pressure_oscillating"])
def test_adjoint_matches_central_differences(case, store):
    cfg = dict(CASES[case])
    cfg["shape"] = (13, 9)  # several cells between the walls
    steps = 40
    p, u, field, w = _inputs(cfg, seed=303)
    field32 = field.astype(np.float32).astype(np.float64)
    _, dfield, dwall, _ = _gpu_grads(cfg, p, u, field32, w, store=store, steps=steps, every=9)
    n = int(np.prod(cfg["shape"]))
    rng = np.random.default_rng(11)
    cells = rng.choice(n, size=4, replace=False)
    h = 1e-4
    scale = np.abs(dfield).max()
    for c in cells:
        for a in range(2):
            fp, fm = field32.copy(), field32.copy()
            fp[a, c] += h
            fm[a, c] -= h
            fd = (_loss_oracle(cfg, p, u, fp, w, steps) - _loss_oracle(cfg, p, u, fm, w, steps)) / (2 * h)
            assert abs(dfield[a, c] - fd) <= 1e-4 * max(abs(fd), 1e-2 * scale), (c, a, dfield[a, c], fd)


@pytest.mark.parametrize("store", [3, 0])
@pytest.mark.parametrize("case", ["cavity", "pressure_oscillating"])
def test_checkpoint_interval_does_not_change_the_gradient(case, store):
    """Bitwise the same gradients for every checkpoint interval. A segment's first reverse step
    recomputes its cells in a kernel of its own and the others in the previous step's cells
    kernel, so the intervals mix the two differently; with an oscillating G the two also take
    the force factor of each state's own time."""
    cfg = CASES[case]
    p, u, field, w = _inputs(cfg, seed=55)
    out = [_gpu_grads(cfg, p, u, field, w, store=store, steps=23, every=k) for k in (1, 5, 23, 100)]
    for o in out[1:]:
        assert np.array_equal(o[1], out[0][1])
        assert np.array_equal(o[2], out[0][2])
        assert np.array_equal(o[3], out[0][3])


def test_autograd_function_matches_direct_adjoint():
    torch = _torch()
    from paper_1411_6121_gb300 import autograd, dugks
    cfg = CASES["channel_lid"]
    p, u, field, w = _inputs(cfg, seed=77)
    s = dugks.Sim(store=dugks.STORE_F64, **cfg)
    s.init(p=p, u=u)
    g0 = s.get_state(out=torch.empty((9, s.ncell), dtype=torch.float64, device="cuda"))
    fld = torch.tensor(field, dtype=torch.float32, device="cuda", requires_grad=True)
    wall = torch.tensor([list(b[1]) for b in cfg["bcs"]] + [[0.0] * 3] * 2, dtype=torch.float64, requires_grad=True)
    st = g0.clone().requires_grad_(True)
    target = torch.zeros((3, s.ncell), dtype=torch.float32, device="cuda")
    m = autograd.rollout(s, fld, wall, STEPS, every=4, state0=st)
    loss = ((m[1:] - target[1:]) ** 2).sum()
    loss.backward()
    # the same through the raw calls
    s2 = dugks.Sim(field=torch.tensor(field, dtype=torch.float32, device="cuda"), store=dugks.STORE_F64, **cfg)
    s2.set_state(g0)
    s2.record(STEPS, 4)
    m2 = torch.empty((3, s2.ncell), dtype=torch.float32, device="cuda")
    s2.moments(m2)
    seed = torch.zeros_like(m2)
    seed[1:] = 2 * (m2[1:] - target[1:])
    df, dw, ds = s2.adjoint(seed, state_grad=True)
    assert torch.equal(fld.grad, df)
    assert np.array_equal(wall.grad.numpy(), dw)
    assert torch.equal(st.grad, ds)


def test_adjoint_error_codes():
    torch = _torch()
    from paper_1411_6121_gb300 import dugks
    cfg = CASES["cavity"]
    s = dugks.Sim(store=dugks.STORE_F32, **cfg)
    s.init()
    g = torch.zeros((3, s.ncell), dtype=torch.float32, device="cuda")
    with pytest.raises(dugks.DugksError) as e:
        s.adjoint(g)
    assert e.value.code == -1  # nothing recorded
    with pytest.raises(dugks.DugksError) as e:
        s.record(0, 5)
    assert e.value.code == -1
    b = dugks.Sim(store=dugks.STORE_BF16, **cfg)
    with pytest.raises(dugks.DugksError) as e:
        b.record(4, 2)
    assert e.value.code == -7
    c3 = dugks.Sim(shape=(8, 8, 8), q=19, nu=0.05, dt=0.5, bcs=W.cavity_bcs(3, 0.05))
    with pytest.raises(dugks.DugksError) as e:
        c3.record(4, 2)
    assert e.value.code == -7
    with pytest.raises(dugks.DugksError) as e:
        s.set_boundaries(W.all_periodic())  # face types may not change
    assert e.value.code == -1


def _host_u(state, cfg, field, steps):
    """u(T) in FP64 from an FP64 state (eq. (27)), for finite differences that
    must not be limited by the float32 moments output."""
    o = Oracle(**cfg)
    e, _ = o.lattice()
    c = np.sqrt(3.0 * cfg.get("rt", 1.0 / 3.0))
    rho0 = cfg.get("rho0", 1.0)
    g = np.asarray(cfg.get("g", (0.0, 0.0, 0.0)))[:2, None]
    return c / rho0 * (e[:, :2].T.astype(np.float64) @ state) + (g + field) * 0.5 * cfg["dt"]


def test_long_rollout_fp32_adjoint_on_uneven_channels():
    """Channels of uneven size and Re, loss ||u(T) - u_target||^2 over 2000 steps with a
    checkpoint every 100 steps, FP32: the gradient at 4 cells per instance agrees with
    central differences of the FP64 forward within 1e-4 relative."""
    torch = _torch()
    from paper_1411_6121_gb300 import dugks
    insts = W.batched_channels(64)
    pick = sorted(range(64), key=lambda i: insts[i]["shape"][1])
    pick = [pick[0], pick[20], pick[45], pick[63]]
    steps, every = 2000, 100
    for idx in pick:
        ins = dict(insts[idx])
        ins.pop("re")
        n = int(np.prod(ins["shape"]))
        rng = np.random.default_rng(1000 + idx)
        field = (ins["g"][0] * 0.3 * rng.standard_normal((2, n))).astype(np.float32).astype(np.float64)
        ut = 0.5 * W.random_state_fields(ins["shape"], seed=idx, u_amp=0.05)[1].reshape(2, n)

        def u_fp64(fld):
            s = dugks.Sim(field=torch.tensor(fld, dtype=torch.float32, device="cuda"), store=dugks.STORE_F64, **ins)
            s.init()
            s.step(steps)
            return _host_u(s.get_state(), ins, fld, steps)

        s = dugks.Sim(field=torch.tensor(field, dtype=torch.float32, device="cuda"), store=dugks.STORE_F32, **ins)
        s.init()
        s.record(steps, every)
        m = s.moments()
        seed = np.zeros((3, n), dtype=np.float32)
        seed[1:] = 2 * (m[1:] - ut)
        df, _, _ = s.adjoint(torch.tensor(seed, device="cuda"))
        df = df.double().cpu().numpy()
        cells = rng.choice(n, size=4, replace=False)
        h = 1e-2 * abs(ins["g"][0])
        for c in cells:
            fp, fm = field.copy(), field.copy()
            fp[0, c] = np.float32(field[0, c] + h)
            fm[0, c] = np.float32(field[0, c] - h)
            lp = np.sum((u_fp64(fp) - ut) ** 2)
            lm = np.sum((u_fp64(fm) - ut) ** 2)
            fd = (lp - lm) / (fp[0, c] - fm[0, c])
            assert abs(df[0, c] - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(df[0]).max()), (idx, c, df[0, c], fd)


def test_async_adjoint_on_two_streams_matches_sync():
    """dugks_adjoint_async on two handles in flight together gives bitwise the results of
    the synchronous call; dugks_adjoint_wall returns the same wall gradient."""
    torch = _torch()
    from paper_1411_6121_gb300 import dugks
    cfg = CASES["channel_wide"]
    p, u, field, w = _inputs(cfg, seed=91)
    tf = torch.tensor(field, dtype=torch.float32, device="cuda")
    wt = torch.tensor(w, dtype=torch.float32, device="cuda")
    ref = dugks.Sim(field=tf, store=0, **cfg)
    ref.init(p=p, u=u)
    ref.record(40, 7)
    dref, wref, _ = ref.adjoint(wt)
    sims, outs = [], []
    for _ in range(2):
        s = dugks.Sim(field=tf, store=0, stream=torch.cuda.Stream().cuda_stream, **cfg)
        s.init(p=p, u=u)
        s.record(40, 7)
        sims.append(s)
    for s in sims:
        o = torch.empty_like(dref)
        s.adjoint_async(wt, dfield=o)
        outs.append(o)
    for s, o in zip(sims, outs):
        s.sync()
        assert torch.equal(o, dref)
        assert np.array_equal(s.adjoint_wall(), wref)


def test_segment_graphs_reused_only_while_valid():
    """Segment graphs survive across adjoint calls and records of the same length. A second
    record + adjoint on the same handle, and one after the acceleration field was replaced
    (a new pointer baked into the old graphs), give bitwise the results of fresh handles."""
    torch = _torch()
    from paper_1411_6121_gb300 import dugks
    cfg = dict(CASES["channel_wide"], omega=0.0)  # graphs need a time-independent force
    p, u, field, w = _inputs(cfg, seed=17)
    tf = torch.tensor(field, dtype=torch.float32, device="cuda")
    tf2 = torch.tensor(1.5 * field, dtype=torch.float32, device="cuda")
    wt = torch.tensor(w, dtype=torch.float32, device="cuda")

    def fresh(fld):
        s = dugks.Sim(field=fld, store=0, **cfg)
        s.init(p=p, u=u)
        s.record(40, 7)  # 6 segments: captured as graphs
        return s.adjoint(wt)

    d1, w1, _ = fresh(tf)
    d2, w2, _ = fresh(tf2)
    s = dugks.Sim(field=tf, store=0, **cfg)
    for _ in range(2):  # the second pass replays the graphs of the first
        s.init(p=p, u=u)
        s.record(40, 7)
        d, wg, _ = s.adjoint(wt)
        assert torch.equal(d, d1) and np.array_equal(wg, w1)
    s.set_force_field(tf2)
    s.init(p=p, u=u)
    s.record(40, 7)
    d, wg, _ = s.adjoint(wt)
    assert torch.equal(d, d2) and np.array_equal(wg, w2)
    assert not torch.equal(d1, d2)
