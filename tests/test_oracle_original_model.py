"""Pins of the original DUGKS (the comparison model of Sec. 2.1-2.2: eq. (5) with
rho u = sum xi f~ + rho G dt/2) in the oracle, by what the equations fix exactly:
  * eq. (5)'s moments: sum f_eq = rho, sum xi f_eq = rho u, sum xi xi f_eq = rho RT I + rho u u;
  * with eq. (5) the force term of eq. (9) has zero mass, sum_k S_k = G.(rho u - u rho)/RT = 0,
    so a periodic box keeps its mass to rounding under any force. The incompressible model's S
    does not sum to zero when rho != rho0, which keeps the check discriminating;
  * at rho = rho0 the two equilibria coincide, so a uniform flow of density rho0 is a fixed
    point of both.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1411_6121_gb300 import workloads as W


@pytest.mark.parametrize("q", [9, 19, 27])
def test_original_equilibrium_moments(q):
    rng = np.random.default_rng(100 + q)
    D = 2 if q == 9 else 3
    shape = (5, 4) if D == 2 else (3, 2, 2)
    rt, rho0 = 0.7, 1.3
    o = Oracle(shape, q, nu=0.1, dt=0.5, rt=rt, rho0=rho0, model=1)
    n = o.ncell
    p = rng.normal(0, 0.05, n)
    u = rng.normal(0, 0.1, (D, n))
    o.init(p=p, u=u)
    f = o.get_state()
    e, Wt = o.lattice()
    xi = np.sqrt(3 * rt) * e[:, :D].astype(float)
    rho = rho0 + p / rt
    assert np.abs(f.sum(0) - rho).max() < 1e-14
    assert np.abs(np.einsum("ka,kn->an", xi, f) - rho * u).max() < 1e-14
    m2 = np.einsum("ka,kb,kn->abn", xi, xi, f)
    ref = rho[None, None, :] * (rt * np.eye(D)[:, :, None] + np.einsum("an,bn->abn", u, u))
    assert np.abs(m2 - ref).max() < 1e-13
    # the velocity reported back is the one given (rho u / rho)
    assert np.abs(o.moments()[1:] - u).max() < 1e-14


@pytest.mark.parametrize("q,shape", [(9, (12, 10)), (19, (5, 4, 4))])
def test_original_model_conserves_mass_under_force(q, shape):
    D = len(shape)
    g = (2e-3, -1e-3, 1.5e-3)[:D] + (0.0,) * (3 - D)
    field = W.force_field(shape, 1e-3, seed=3, rel=1.0)
    p, u = W.random_state_fields(shape, seed=4, u_amp=0.05, p_amp=2e-3)
    drift = {}
    for model in (0, 1):
        o = Oracle(shape, q, nu=0.05, dt=0.5, g=g, field=field, omega=0.05, bcs=W.all_periodic(), model=model)
        o.init(p=p, u=u)
        m0 = o.moments()[0].sum()
        o.step(60)
        drift[model] = abs(o.moments()[0].sum() - m0)
    n = int(np.prod(shape))
    assert drift[1] / n < 1e-14, drift
    assert drift[0] / n > 1e-9, drift


@pytest.mark.parametrize("q,shape", [(9, (6, 5)), (19, (4, 3, 3))])
def test_uniform_flow_of_rho0_is_fixed_in_both_models(q, shape):
    D = len(shape)
    n = int(np.prod(shape))
    u = np.zeros((D, n))
    u[0], u[1] = 0.04, -0.03
    states = []
    for model in (0, 1):
        o = Oracle(shape, q, nu=0.05, dt=0.5, bcs=W.all_periodic(), model=model)
        o.init(u=u)
        f0 = o.get_state()
        o.step(9)
        assert np.abs(o.get_state() - f0).max() < 1e-15
        states.append(f0)
    assert np.abs(states[0] - states[1]).max() < 1e-16


@pytest.mark.slow
def test_mach_sensitivity_oracle():
    """Sec. 3.1's compressibility study in the oracle (golden fixture, cited): about four
    minutes of FP64 CPU time."""
    from oracle.oracle import rel_change
    from tests import mach_study

    def run(cfg, p, u, field):
        o = Oracle(field=field, **cfg)
        o.init(p=p, u=u)
        prev = o.moments()[1:]
        while True:
            o.step(1000)
            cur = o.moments()[1:]
            if rel_change(cur, prev) <= 1e-6:
                return cur
            prev = cur

    mach_study.check(lambda ma, m: mach_study.steady_error(ma, m, run))
