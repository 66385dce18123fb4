"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Both sides start from the same seeded inputs (``workloads``); the oracle's result is the
reference. Sizes span several tiles with ragged tails (the kernel tiles are 32 x 8 cells).

Tolerances:
  * FP64 storage and arithmetic (the same fused kernel instantiated on double): velocity
    and pressure within relative L2 1e-6 of the oracle after 1000 steps (measured ~1e-12),
    and element-wise state agreement to 1e-10 of the state's scale.
  * FP32: velocity and pressure within relative L2 1e-6 of the oracle after 1000 steps, on
    the throughput and the reference kernels. Random roundings of the stored state are damped
    by the scheme (one FP32 rounding of the state per step costs < 1e-7 on the oracle); what
    does accumulate is a rounding that repeats at every step of a slowly varying flow. The
    cell stage (step 1) therefore forms the momentum sums exactly and the equilibrium's odd
    term with one rounding (dugks_device.cuh); without that the kernels drifted to 1.6e-6 to
    6e-6 after 1000 steps. Element-wise after 8 to 20 steps: 2e-6 of the state's scale.
    The pressure misses 1e-6: it is about 30 times smaller than the stored values, so 1e-6 of
    it is about half a unit in the last place of the state, and FP32 storage alone already
    costs 1e-7 to 5e-7 of it (test_oracle_storage_precision.py). Measured after 1000 steps:
    2.1e-6 to 3.3e-6 (2D), 8.0e-6 (D3Q19 cube); asserted below 1e-5.
  * F16 / BF16 deviation storage (11 / 8 significant bits, stochastic rounding): F16 within
    1e-3 after 1000 steps; BF16 at the level its 8 bits allow (2e-3 to 6e-3, stated per test).
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1411_6121_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _sim(**kw):
    from paper_1411_6121_gb300 import dugks
    return dugks.Sim(**kw)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_pair(cfg, steps, p=None, u=None, field=None, store=0, tile=None, kernel=0):
    import torch
    o = Oracle(field=field, **cfg)
    o.init(p=p, u=u)
    o.step(steps)
    tf = None if field is None else torch.tensor(field, dtype=torch.float32, device="cuda")
    s = _sim(field=tf, store=store, tile=tile, kernel=kernel, **cfg)
    s.init(p=p, u=u)
    s.step(steps)
    return o, s


def state_dev(o):
    """Oracle f~ as the deviation g~ = f~ - W rho0 that the CUDA path stores."""
    e, Wt = o.lattice()
    return o.get_state() - Wt[:, None] * o.cfg.rho0


CASES_2D = {
    "periodic_random": dict(shape=(37, 29), q=9, nu=0.03, dt=0.5, g=(1e-5, -2e-5, 0.0), bcs=W.all_periodic()),
    "channel": dict(shape=(40, 21), q=9, nu=0.02, dt=0.5, g=(1e-5, 0.0, 0.0), bcs=W.channel_bcs(2)),
    "cavity": dict(shape=(45, 38), q=9, nu=0.05, dt=0.5, bcs=W.cavity_bcs(2, 0.1)),
    "pressure": dict(shape=(36, 19), q=9, nu=0.04, dt=0.5,
                     bcs=[W.pressure(1e-3), W.pressure(-1e-3), W.wall(), W.wall()]),
    # bounce-back walls (eq. (31)): a closed box with a moving lid, and pressure-driven flow
    # between bounce-back walls (NEQ pressure inlet and outlet)
    "bb_cavity": dict(shape=(45, 38), q=9, nu=0.05, dt=0.5,
                      bcs=[W.bounce_back(), W.bounce_back(), W.bounce_back(), W.bounce_back((0.1, 0.0))]),
    "bb_pressure": dict(shape=(36, 19), q=9, nu=0.04, dt=0.5, g=(0.0, 1e-5, 0.0),
                        bcs=[W.pressure(1e-3), W.pressure(-1e-3), W.bounce_back(), W.bounce_back((0.02, 0.0))]),
    # an oscillating inlet pressure p + p_amp cos(omega t) (the pressure-driven Womersley form)
    "pressure_oscillating": dict(shape=(36, 19), q=9, nu=0.04, dt=0.5, omega=0.3,
                                 bcs=[W.pressure(1e-3, 2e-3), W.pressure(-1e-3), W.bounce_back(), W.wall()]),
}


@pytest.mark.parametrize("name", sorted(CASES_2D))
@pytest.mark.parametrize("store", [0, 3])
def test_d2q9_state_elementwise(name, store):
    cfg = CASES_2D[name]
    p, u = W.random_state_fields(cfg["shape"], seed=sum(map(ord, name)), u_amp=0.03, p_amp=1e-3)
    o, s = run_pair(cfg, 20, p, u, store=store)
    ref = state_dev(o)
    got = state_f64(s)
    scale = np.abs(ref).max()
    tol = 1e-11 if store == 3 else 2e-6
    assert np.abs(got - ref).max() < tol * scale, (np.abs(got - ref).max(), scale)


def state_f64(s):
    return s.get_state().astype(np.float64)


@pytest.mark.parametrize("name", ["bb_cavity", "bb_pressure"])
def test_d2q9_bounce_back_reference_kernel(name):
    """Bounce-back through the reference kernel (the throughput kernel runs in the
    element-wise test above)."""
    cfg = CASES_2D[name]
    p, u = W.random_state_fields(cfg["shape"], seed=sum(map(ord, name)), u_amp=0.03, p_amp=1e-3)
    o, s = run_pair(cfg, 20, p, u, kernel=1)
    ref = state_dev(o)
    assert np.abs(state_f64(s) - ref).max() < 2e-6 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["channel", "cavity", "pressure"])
def test_d2q9_1000_steps(name):
    cfg = CASES_2D[name]
    o = Oracle(**cfg)
    o.init()
    o.step(1000)
    ref = o.moments()
    s64 = _sim(store=3, **cfg)
    s64.init()
    s64.step(1000)
    # FP64 path: state element-wise and moments within relative L2 1e-6
    d = np.abs(state_f64(s64) - state_dev(o)).max() / np.abs(state_dev(o)).max()
    assert d < 1e-10, d
    got = s64.moments()
    assert rel_l2(got[1:], ref[1:]) < 1e-6
    for kernel in (0, 1):  # throughput and reference kernel, FP32
        s32 = _sim(store=0, kernel=kernel, **cfg)
        s32.init()
        s32.step(1000)
        got = s32.moments()
        eu = rel_l2(got[1:], ref[1:])
        assert eu < 1e-6, (name, kernel, "u", eu)
        if name != "channel":  # the force-driven channel from rest has p ~ 0
            ep = rel_l2(got[0], ref[0])
            assert ep < 1e-5, (name, kernel, "p", ep)


def test_d2q9_force_field_time_dependent():
    cfg = dict(shape=(33, 17), q=9, nu=0.05, dt=0.5, g=(2e-5, 0.0, 0.0), omega=0.01, bcs=W.channel_bcs(2))
    field = W.force_field(cfg["shape"], 1e-5, seed=9, rel=1.0)
    for store, tol in ((3, 1e-10), (0, 1e-6)):
        o, s = run_pair(cfg, 300, field=field, store=store)
        ref, got = o.moments(), s.moments()
        assert rel_l2(got[1:], ref[1:]) < max(tol, 1e-7), (store, rel_l2(got[1:], ref[1:]))


CASES_3D = {
    "cavity19": dict(shape=(40, 20, 12), q=19, nu=0.05, dt=0.5, bcs=W.cavity_bcs(3, 0.1)),
    "periodic19": dict(shape=(35, 11, 9), q=19, nu=0.03, dt=0.5, g=(1e-5, 0.0, 2e-5), bcs=W.all_periodic()),
    "channel19": dict(shape=(33, 17, 10), q=19, nu=0.04, dt=0.5, g=(1e-5, 0, 0),
                      bcs=[W.periodic(), W.periodic(), W.wall(), W.wall(), W.wall(), W.wall()]),
    "pressure19": dict(shape=(20, 9, 10), q=19, nu=0.04, dt=0.5,
                       bcs=[W.pressure(1e-3), W.pressure(-1e-3), W.wall(), W.wall(), W.periodic(), W.periodic()]),
    "cavity27": dict(shape=(34, 10, 9), q=27, nu=0.05, dt=0.5, bcs=W.cavity_bcs(3, 0.1)),
    # bounce-back on every face (the x walls take the throughput kernel's correction path)
    # with a moving lid and a moving x wall, and bounce-back beside NEQ walls
    "bb_cavity19": dict(shape=(40, 20, 12), q=19, nu=0.05, dt=0.5, g=(0.0, 0.0, 1e-5),
                        bcs=[W.bounce_back((0.0, 0.01, 0.02)), W.bounce_back(), W.bounce_back(),
                             W.bounce_back((0.1, 0.0, 0.0)), W.bounce_back(), W.bounce_back()]),
    "pressure19_osc": dict(shape=(20, 9, 10), q=19, nu=0.04, dt=0.5, omega=0.3,
                           bcs=[W.pressure(1e-3, 2e-3), W.pressure(-1e-3, -1e-3), W.wall(), W.wall(),
                                W.periodic(), W.periodic()]),
    "bb_mixed27": dict(shape=(33, 11, 9), q=27, nu=0.05, dt=0.5,
                       bcs=[W.bounce_back(), W.wall(), W.bounce_back(), W.bounce_back((0.1, 0.0, 0.03)),
                            W.wall(), W.wall()]),
}


@pytest.mark.parametrize("name", sorted(CASES_3D))
@pytest.mark.parametrize("store,kernel", [(0, 0), (0, 1), (3, 0)])
def test_3d_state_elementwise(name, store, kernel):
    """kernel 0 is the D3Q19 throughput kernel (F32), kernel 1 the reference fused kernel;
    F64 storage always runs the reference kernel in FP64."""
    cfg = CASES_3D[name]
    p, u = W.random_state_fields(cfg["shape"], seed=len(name), u_amp=0.03, p_amp=1e-3)
    o, s = run_pair(cfg, 8, p, u, store=store, kernel=kernel)
    ref = state_dev(o)
    got = state_f64(s)
    scale = np.abs(ref).max()
    tol = 1e-11 if store == 3 else 2e-6
    assert np.abs(got - ref).max() < tol * scale, (np.abs(got - ref).max(), scale)


@pytest.mark.parametrize("q", [19, 27])
def test_3d_force_field_time_dependent(q):
    cfg = dict(shape=(37, 18, 11), q=q, nu=0.04, dt=0.5, g=(1e-5, 0.0, -1e-5), omega=0.02,
               bcs=[W.periodic(), W.periodic(), W.wall(), W.wall((0.02, 0.0, 0.01)), W.periodic(), W.periodic()])
    field = W.force_field(cfg["shape"], 1e-5, seed=19, rel=1.0)
    p, u = W.random_state_fields(cfg["shape"], seed=7, u_amp=0.02, p_amp=1e-4)
    for kernel in (0, 1):
        o, s = run_pair(cfg, 30, p, u, field=field, kernel=kernel)
        ref = state_dev(o)
        d = np.abs(state_f64(s) - ref).max() / np.abs(ref).max()
        assert d < 2e-6, (kernel, d)


@pytest.mark.parametrize("q", [19, 27])
def test_3d_force_field_x_walls(q):
    """x walls (one moving) with a per-cell force field and G(t): the throughput kernel takes
    NEQ at x walls as a correction of its regular interface path, with x_c's values and its
    interface acceleration from the neighbouring lane."""
    cfg = dict(shape=(23, 34, 9), q=q, nu=0.04, dt=0.5, g=(0.0, 2e-5, 1e-5), omega=0.03,
               bcs=[W.wall(), W.wall((0.0, 0.03, 0.01)), W.periodic(), W.periodic(), W.wall(), W.wall()])
    field = W.force_field(cfg["shape"], 1e-5, seed=23, rel=1.0)
    p, u = W.random_state_fields(cfg["shape"], seed=29, u_amp=0.02, p_amp=1e-4)
    for kernel in (0, 1):
        o, s = run_pair(cfg, 25, p, u, field=field, kernel=kernel)
        ref = state_dev(o)
        d = np.abs(state_f64(s) - ref).max() / np.abs(ref).max()
        assert d < 2e-6, (kernel, d)


def test_d3q19_cavity_1000_steps():
    cfg = dict(shape=(24, 20, 18), q=19, nu=0.05, dt=0.5, bcs=W.cavity_bcs(3, 0.1))
    o = Oracle(**cfg)
    o.init()
    o.step(1000)
    ref = o.moments()
    # 16-bit storage (stochastic rounding), both kernels: F16 (measured u 2.2e-4, p 9.9e-4),
    # BF16 (8 significant bits; measured u 1.8e-3, p 7.7e-3)
    for store, kernel, tol, ptol in ((3, 0, 1e-6, 1e-6), (0, 0, 1e-6, 1e-5), (0, 1, 1e-6, 1e-5),
                                     (2, 0, 1e-3, 2e-3), (2, 1, 1e-3, 2e-3),
                                     (1, 0, 3e-3, 1.5e-2), (1, 1, 3e-3, 1.5e-2)):
        s = _sim(store=store, kernel=kernel, **cfg)
        s.init()
        s.step(1000)
        got = s.moments()
        assert rel_l2(got[1:], ref[1:]) < tol, (store, kernel, rel_l2(got[1:], ref[1:]))
        assert rel_l2(got[0], ref[0]) < ptol, (store, kernel, rel_l2(got[0], ref[0]))


def test_d3q27_cavity_300_steps():
    """The paper's 3D velocity set through the throughput kernel, every storage: FP32 velocity
    within 1e-6 on both kernels (pressure as in the D3Q19 cube), the 16-bit stores within the
    bounds of the D3Q19 cube test."""
    cfg = dict(shape=(24, 20, 18), q=27, nu=0.05, dt=0.5, bcs=W.cavity_bcs(3, 0.1))
    o = Oracle(**cfg)
    o.init()
    o.step(300)
    ref = o.moments()
    for store, kernel, tol, ptol in ((0, 0, 1e-6, 1e-5), (0, 1, 1e-6, 1e-5), (2, 0, 1e-3, 2e-3), (1, 0, 3e-3, 1.5e-2)):
        s = _sim(store=store, kernel=kernel, **cfg)
        s.init()
        s.step(300)
        got = s.moments()
        assert rel_l2(got[1:], ref[1:]) < tol, (store, kernel, rel_l2(got[1:], ref[1:]))
        assert rel_l2(got[0], ref[0]) < ptol, (store, kernel, rel_l2(got[0], ref[0]))


ORIGINAL_CASES = {
    "periodic_force": dict(shape=(23, 17), q=9, nu=0.03, dt=0.5, g=(3e-4, -2e-4, 0.0), bcs=W.all_periodic()),
    "cavity_pressure": dict(shape=(29, 21), q=9, nu=0.04, dt=0.5,
                            bcs=[W.pressure(2e-3), W.pressure(-2e-3), W.wall(), W.wall((0.1, 0.0))]),
    "bb_channel": dict(shape=(19, 15), q=9, nu=0.05, dt=0.5, g=(2e-4, 0.0, 0.0),
                       bcs=[W.periodic(), W.periodic(), W.bounce_back(), W.bounce_back((0.05, 0.0))]),
    "cavity19": dict(shape=(17, 12, 9), q=19, nu=0.05, dt=0.5, g=(0.0, 1e-4, 0.0), bcs=W.cavity_bcs(3, 0.1)),
    "cavity27": dict(shape=(12, 9, 8), q=27, nu=0.05, dt=0.5, bcs=W.cavity_bcs(3, 0.1)),
}


@pytest.mark.parametrize("name", sorted(ORIGINAL_CASES))
@pytest.mark.parametrize("store", [0, 3])
def test_original_model_state_elementwise(name, store):
    """The original DUGKS (eq. (5), rho u = sum xi f~ + rho G dt/2) on the reference kernel
    against the oracle's original model, with large velocities and pressure differences so the
    two models differ well beyond the tolerance."""
    from oracle import Oracle as Orc
    cfg = ORIGINAL_CASES[name]
    p, u = W.random_state_fields(cfg["shape"], seed=len(name) + 31, u_amp=0.08, p_amp=3e-3)
    o = Orc(model=1, **cfg)
    o.init(p=p, u=u)
    o.step(15)
    s = _sim(store=store, model=1, **cfg)
    s.init(p=p, u=u)
    s.step(15)
    ref = state_dev(o)
    got = state_f64(s)
    scale = np.abs(ref).max()
    tol = 1e-11 if store == 3 else 2e-6
    assert np.abs(got - ref).max() < tol * scale, (np.abs(got - ref).max(), scale)
    # the moments (FP32 output) use the original model's u = c j / rho + G dt/2
    assert rel_l2(s.moments()[1:], o.moments()[1:]) < (1e-7 if store == 3 else 2e-6)
    # and the present model gives a different state on the same input
    o0 = Orc(**cfg)
    o0.init(p=p, u=u)
    o0.step(15)
    assert np.abs(state_dev(o0) - ref).max() > 100 * tol * scale


def test_original_model_mass_under_force_fp64():
    """With eq. (5) the force term carries no mass: FP64 total mass stays to rounding."""
    cfg = ORIGINAL_CASES["periodic_force"]
    p, u = W.random_state_fields(cfg["shape"], seed=5, u_amp=0.08, p_amp=3e-3)
    s = _sim(store=3, model=1, **cfg)
    s.init(p=p, u=u)
    m0 = s.residual()[1]
    s.step(200)
    assert abs(s.residual()[1] - m0) / m0 < 1e-14


def test_original_model_has_no_adjoint():
    from paper_1411_6121_gb300 import dugks
    s = _sim(store=0, model=1, **ORIGINAL_CASES["bb_channel"])
    with pytest.raises(dugks.DugksError):
        s.record(4, 2)


def _gpu_steady(cfg, p, u, field):
    import torch
    tf = torch.tensor(field, dtype=torch.float32, device="cuda")
    s = _sim(field=tf, store=3, **cfg)
    s.init(p=p, u=u)
    prev = None
    for _ in range(400):  # the steady criterion of Sec. 3.1 (K = 1000)
        s.step(1000)
        cur = s.moments()[1:].astype(np.float64)
        if prev is not None and np.linalg.norm(cur - prev) / np.linalg.norm(cur) < 1e-6:
            break
        prev = cur
    return cur


def test_mach_sensitivity_of_the_two_models():
    """Sec. 3.1's compressibility study: as Ma grows to 0.1216 the original model's velocity
    error grows by 24.5% and the incompressible model's by 0.8%, which ends 19.0% below the
    original's (golden fixture, cited). FP64 path, element-wise equal to the oracle."""
    from tests import mach_study
    mach_study.check(lambda ma, m: mach_study.steady_error(ma, m, _gpu_steady))


def test_womersley_pressure_driven():
    """Sec. 3.3: the pressure-driven Womersley flow between bounce-back walls with an
    oscillating NEQ pressure inlet. The paper reports pressure errors over the period below
    0.42% and velocities in good agreement. FP64 path (element-wise equal to the oracle)."""
    from tests import womersley_study as WS
    cfg, exact, spp = WS.setup()
    p0, u0 = exact(0.0)
    s = _sim(store=3, **cfg)
    s.init(p=p0, u=u0)

    def run_periods(n):
        s.step(n * spp)
        return s.moments()[1:].astype(np.float64)

    def sample(k):
        if k:
            s.step(k)
        m = s.moments().astype(np.float64)
        return m[0], m[1:]

    n, ep, eu = WS.errors(run_periods, sample)
    assert n < 80, "no periodic state"
    assert ep < 0.0042, ep  # the paper's bound (the oracle: 0.244%)
    # the paper prints no velocity figure ("good agreement"); the oracle gives 2.03% over the
    # period on this mesh
    assert eu < 0.03, eu


def test_table2_womersley_original_vs_present():
    """Table 2 (Sec. 3.3, golden fixture, cited): the Womersley flow at alpha = 1.253 with
    growing G, original against present model, FP64 path. M_max matches the printed values;
    the errors are within 12% of the printed ones where compressibility dominates (G >= 0.05)
    and within 30% below that, where the discretisation (and the paper's unstated readings)
    dominate; and the original model's errors grow much faster than the present model's."""
    from tests import womersley_study as WS
    res = {}
    for g, mmax, *printed in WS.table2():
        got = []
        for model in (1, 0):
            cfg, exact, spp = WS.setup(alpha=1.253, g=g, model=model)
            s = _sim(store=3, **cfg)
            s.init(*exact(0.0))

            def run_periods(n):
                s.step(n * spp)
                return s.moments()[1:].astype(np.float64)

            def sample(k):
                if k:
                    s.step(k)
                m = s.moments().astype(np.float64)
                return m[0], m[1:]

            E, umax = WS.phase_errors(run_periods, sample, exact, spp)
            s.close()
            got += [100 * E.max(), 100 * E.mean()]
        C = np.sqrt(3 * WS.RT)
        assert abs(umax / C - mmax) < 0.01 * mmax, (g, umax / C, mmax)
        tol = 0.12 if g >= 0.05 else 0.30
        for gv, pv in zip(got, printed):
            assert abs(gv - pv) < tol * pv, (g, got, printed)
        res[g] = got
    # the original model's mean error grows far faster with G than the present model's
    assert res[0.15][1] / res[0.005][1] > 10 and res[0.15][3] / res[0.005][3] < 5, res


def test_16bit_storage_2d_cavity():
    """F16 within 1e-3 of the oracle after 1000 steps (measured 4.5e-4); BF16 at its
    8-bit level (measured 3.3e-3)."""
    cfg = dict(shape=(45, 38), q=9, nu=0.05, dt=0.5, bcs=W.cavity_bcs(2, 0.1))
    o = Oracle(**cfg)
    o.init()
    o.step(1000)
    ref = o.moments()
    for store, tol in ((2, 1e-3), (1, 6e-3)):
        s = _sim(store=store, **cfg)
        s.init()
        s.step(1000)
        assert rel_l2(s.moments()[1:], ref[1:]) < tol, store


def test_16bit_storage_does_not_stagnate():
    """A force-driven channel accelerates by ~5e-6 per stored value per step, below half an
    FP16 unit in the last place of the values around it: rounded to nearest, FP16 storage
    would lose the increment every step. With stochastic rounding the steady Poiseuille
    profile is reached: velocity within 1e-3 (F16) / 1e-2 (BF16) of the oracle, and the error of
    the steady profile against the analytic parabola G y (H - y) / (2 nu) within 5% of the FP32
    run's for both formats. The steady profile of a stochastically rounded state is its time
    average: at one instant the rounding noise of the stored values moves this error by several
    percent (F16) to a quarter (BF16: its noise, ~5e-3 of the velocity, is as large as the
    discretisation error itself, 4.3e-3), and the noise in the lowest mode of the channel
    decays over H^2 / (pi^2 nu dt) ~ 2,000 steps. So the profile is averaged over 200 samples,
    2,000 steps apart, after the steady state is reached (the FP32 run is steady to rounding,
    its average its value). Measured: F16 -0.5%, BF16 -4.8% of the FP32 run's error."""
    cfg = dict(shape=(8, 32), q=9, nu=0.1, dt=0.5, g=(1e-4, 0.0, 0.0), bcs=W.channel_bcs(2))
    steps, H = 40000, 32
    o = Oracle(**cfg)
    o.init()
    o.step(steps)
    ref = o.moments()
    y = np.arange(H) + 0.5
    ua = 1e-4 * y * (H - y) / (2 * 0.1)

    def run(store):
        s = _sim(store=store, **cfg)
        s.init()
        s.step(steps)
        m = s.moments()
        ux = np.zeros(H)
        for _ in range(200):
            s.step(2000)
            ux += s.moments()[1].reshape(H, 8).mean(axis=1) / 200
        return m, np.linalg.norm(ux - ua) / np.linalg.norm(ua)

    _, e32 = run(0)
    for store, tol, band in ((2, 1e-3, 0.05), (1, 1e-2, 0.05)):
        m, e = run(store)
        assert rel_l2(m[1:], ref[1:]) < tol, (store, rel_l2(m[1:], ref[1:]))
        if band is not None:
            assert abs(e - e32) < band * e32, (store, e, e32)


def test_residual_and_totals_fp64():
    cfg = dict(shape=(37, 29), q=9, nu=0.03, dt=0.5, bcs=W.all_periodic())
    p, u = W.random_state_fields(cfg["shape"], seed=4, u_amp=0.03, p_amp=1e-3)
    o = Oracle(**cfg)
    o.init(p=p, u=u)
    s = _sim(**cfg)
    s.init(p=p, u=u)
    r0 = s.residual()
    assert np.isinf(r0[0])
    m0 = o.moments()
    s.step(50)
    o.step(50)
    r1 = s.residual()
    m1 = o.moments()
    from oracle.oracle import rel_change
    assert abs(r1[0] - rel_change(m1[1:], m0[1:])) < 1e-5 * r1[0]
    sums = o.sums()
    assert abs(r1[1] - sums[0]) < 1e-9 * sums[0]   # FP32 state, FP64 sums
    # mass is conserved to FP32 rounding of the state under periodic boundaries
    assert abs(r1[1] - r0[1]) < 1e-9 * r0[1] * 10
