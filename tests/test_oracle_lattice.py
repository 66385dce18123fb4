"""Pins of the oracle's velocity sets and equilibrium (Sec. 2.1, eq. (6); Sec. 2.3).

The checks are exact moment identities of Gauss-Hermite quadrature and of the He-Luo
equilibrium, derived independently of the oracle's code: a dropped term, a wrong sign or a
wrong weight in either fails one of them.
"""
import itertools

import numpy as np
import pytest

from oracle import Oracle


def _lat(q):
    shape = (3, 3) if q == 9 else (3, 3, 3)
    o = Oracle(shape, q, nu=0.1, dt=0.5)
    e, W = o.lattice()
    return o, e[:, : len(shape)].astype(float), W


@pytest.mark.parametrize("q", [9, 19, 27])
def test_quadrature_moments(q):
    o, e, W = _lat(q)
    D = e.shape[1]
    assert len(W) == q
    assert abs(W.sum() - 1.0) < 1e-15
    assert np.abs((W[:, None] * e).sum(0)).max() < 1e-15
    # sum W e_a e_b = delta_ab / 3  (xi = sqrt(3RT) e  ->  sum W xi xi = RT I)
    m2 = np.einsum("k,ka,kb->ab", W, e, e)
    assert np.abs(m2 - np.eye(D) / 3.0).max() < 1e-15
    m3 = np.einsum("k,ka,kb,kc->abc", W, e, e, e)
    assert np.abs(m3).max() < 1e-15
    # fourth moment isotropy: sum W e_a e_b e_c e_d = (d_ab d_cd + d_ac d_bd + d_ad d_bc)/9
    m4 = np.einsum("k,ka,kb,kc,kd->abcd", W, e, e, e, e)
    I = np.eye(D)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I) + np.einsum("ad,bc->abcd", I, I)) / 9.0
    assert np.abs(m4 - iso).max() < 1e-15


def test_paper_index_order_and_weights():
    """Sec. 2.3 prints the D2Q9 set x-major with W = 4/9 (i = 5), 1/9 (i = 2,4,6,8),
    1/36 (i = 1,3,7,9), and the D3Q27 set with W = 8/27 at i = 14 and 1/216 at the corners."""
    _, e, W = _lat(9)
    ex = [-1, -1, -1, 0, 0, 0, 1, 1, 1]
    ey = [-1, 0, 1, -1, 0, 1, -1, 0, 1]
    assert list(e[:, 0]) == ex and list(e[:, 1]) == ey
    w = {1: 1 / 36, 2: 1 / 9, 3: 1 / 36, 4: 1 / 9, 5: 4 / 9, 6: 1 / 9, 7: 1 / 36, 8: 1 / 9, 9: 1 / 36}
    assert np.allclose(W, [w[i] for i in range(1, 10)], rtol=0, atol=1e-16)
    _, e27, W27 = _lat(27)
    assert W27[13] == pytest.approx(8 / 27, abs=1e-16)
    for i in (1, 3, 7, 9, 19, 21, 25, 27):
        assert W27[i - 1] == pytest.approx(1 / 216, abs=1e-17)
    for i in (5, 11, 13, 15, 17, 23):
        assert W27[i - 1] == pytest.approx(2 / 27, abs=1e-16)
    assert list(map(tuple, e27.astype(int))) == list(itertools.product([-1, 0, 1], repeat=3))
    # D3Q19 is D3Q27 without the 8 corners, same order.
    _, e19, W19 = _lat(19)
    corners = {(a, b, c) for a, b, c in itertools.product([-1, 1], repeat=3)}
    assert list(map(tuple, e19.astype(int))) == [v for v in itertools.product([-1, 0, 1], repeat=3) if v not in corners]


@pytest.mark.parametrize("q", [9, 19, 27])
def test_equilibrium_moments(q):
    """eq. (6): sum f_eq = rho, sum xi f_eq = rho0 u, sum xi xi f_eq = rho RT I + rho0 u u."""
    rng = np.random.default_rng(q)
    D = 2 if q == 9 else 3
    shape = (5, 4) if D == 2 else (3, 2, 2)
    rt, rho0 = 0.7, 1.3
    o = Oracle(shape, q, nu=0.1, dt=0.5, rt=rt, rho0=rho0)
    n = o.ncell
    p = rng.normal(0, 0.05, n)
    u = rng.normal(0, 0.1, (D, n))
    o.init(p=p, u=u)
    f = o.get_state()                       # f~ = f_eq(rho0 + p/RT, u), reading R7
    e, W = o.lattice()
    xi = np.sqrt(3 * rt) * e[:, :D].astype(float)
    rho = rho0 + p / rt
    assert np.abs(f.sum(0) - rho).max() < 1e-14
    assert np.abs(np.einsum("ka,kn->an", xi, f) - rho0 * u).max() < 1e-14
    m2 = np.einsum("ka,kb,kn->abn", xi, xi, f)
    ref = rho[None, None, :] * rt * np.eye(D)[:, :, None] + rho0 * np.einsum("an,bn->abn", u, u)
    assert np.abs(m2 - ref).max() < 1e-13
    # the incompressible form differs from the original eq. (5): rho enters only the
    # zeroth-order term, so f_eq(rho, 0) = W rho and the velocity part is rho-independent.
    o.init(p=p, u=np.zeros((D, n)))
    f0 = o.get_state()
    assert np.abs(f0 - W[:, None] * rho[None, :]).max() < 1e-15
