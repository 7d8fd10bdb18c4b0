"""Pins of the oracle's equilibria and collision.

* Eq. 14 equilibria equal the moments of the 2D Maxwellian (R = 1) computed by
  Gauss-Hermite quadrature of the continuous moment polynomials 5a-5p, for
  k not in {12, 15, 16}; those three are zero (text after Eq. 14).
* The collision conserves rho, j, e exactly (Sec. II: conserved moments).
* f^eq of a state returns the state; a uniform equilibrium is a fixed point.
* Brute force: one step on a 1 x 1 periodic grid is a pure collision, written
  here with scalar loops and the formulas, not with the oracle's matrices.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import lattice, scheme


def _maxwellian_moments(rho, u, v, T, n=24):
    x, w = np.polynomial.hermite_e.hermegauss(n)   # weight exp(-x^2/2)
    w = w / math.sqrt(2.0 * math.pi)
    VX = u + math.sqrt(T) * x[:, None]
    VY = v + math.sqrt(T) * x[None, :]
    WW = w[:, None] * w[None, :]
    return np.array([rho * (WW * r).sum() for r in lattice.moment_rows(VX, VY)])


@pytest.mark.parametrize("seed", range(5))
def test_equilibria_are_maxwellian_moments(seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 5)
    u, v = rng.uniform(-3, 3, 2)
    T = rng.uniform(0.1, 5)
    meq = scheme.moment_equilibria(*scheme.conserved_from_state(rho, u, v, T))
    ref = _maxwellian_moments(rho, u, v, T)
    for k in range(16):
        if k + 1 in (12, 15, 16):
            assert meq[k] == 0.0
        else:
            assert abs(meq[k] - ref[k]) <= 1e-10 * max(1.0, abs(ref[k])), k + 1


def test_feq_returns_state():
    rng = np.random.default_rng(7)
    rho = rng.uniform(0.1, 10, 50)
    u = rng.uniform(-2, 2, 50)
    v = rng.uniform(-2, 2, 50)
    T = rng.uniform(0.1, 10, 50)
    f = scheme.equilibrium_populations(rho, u, v, T)
    r2, u2, v2, T2 = scheme.macroscopic(f)
    np.testing.assert_allclose(r2, rho, rtol=1e-13)
    np.testing.assert_allclose(u2, u, atol=1e-12)
    np.testing.assert_allclose(v2, v, atol=1e-12)
    np.testing.assert_allclose(T2, T, rtol=1e-11)


def test_collision_conserves():
    rng = np.random.default_rng(3)
    w = W.random_state(9, 7, seed=3, smooth=False)
    f = scheme.init_populations(*w.fields())
    f = f * (1.0 + 0.05 * rng.standard_normal(f.shape))  # off equilibrium
    df = scheme.collision(f, w.s, 1e-5)
    m = scheme.moments(df)
    scale = np.abs(scheme.moments(np.abs(f)))[:4].max()
    assert np.abs(m[:4]).max() < 1e-14 * scale
    # and it does change the non-conserved moments
    assert np.abs(m[4:]).max() > 1e-8


def test_uniform_equilibrium_is_fixed_point():
    for bc in ((("periodic", None),) * 4,
               (("eq", (1.3, 0.2, -0.1, 0.9)),) * 4):
        w = W.random_state(6, 5, seed=1, bc=bc)
        rho, u, v, T = (np.full((5, 6), x) for x in (1.3, 0.2, -0.1, 0.9))
        f = scheme.init_populations(rho, u, v, T)
        g = scheme.step(f, w.cfg())
        assert np.abs(g - f).max() < 1e-14 * np.abs(f).max()


def _scalar_collision(fl, s, dt):
    """Independent restatement with Python scalars: moments from formulas
    5a-5p, equilibria 14a-14i, relaxation, and back-mapping by solving
    M x = dm with scalar Gaussian elimination."""
    r2 = math.sqrt(2.0)
    vel = ([(1, 0), (0, 1), (-1, 0), (0, -1)]
           + [(6 * a, 6 * b) for a, b in [(1, 0), (0, 1), (-1, 0), (0, -1)]]
           + [(r2 * a, r2 * b) for a, b in [(1, 1), (-1, 1), (-1, -1), (1, -1)]]
           + [(3 / r2 * a, 3 / r2 * b) for a, b in [(1, 1), (-1, 1), (-1, -1), (1, -1)]])
    rows = []
    for vx, vy in vel:
        q = vx * vx + vy * vy
        rows.append([1, vx, vy, q / 2, vx * vx - vy * vy, vx * vy, vx * q / 2, vy * q / 2,
                     vx * (vx * vx - 3 * vy * vy), vy * (3 * vx * vx - vy * vy), q * q / 4,
                     vx ** 4 - 6 * vx * vx * vy * vy + vy ** 4, q * (vx * vx - vy * vy),
                     q * vx * vy, vx * (vx * vx - 3 * vy * vy) * q, vy * (3 * vx * vx - vy * vy) * q])
    Mt = [[rows[i][k] for i in range(16)] for k in range(16)]  # M[k][i]
    m = [sum(Mt[k][i] * fl[i] for i in range(16)) for k in range(16)]
    rho, jx, jy, e = m[0], m[1], m[2], m[3]
    P = e - (jx * jx + jy * jy) / (2 * rho)
    A = 6 * rho * e - 2 * jx * jx - 2 * jy * jy
    meq = [rho, jx, jy, e, (jx * jx - jy * jy) / rho, jx * jy / rho, (e + P) * jx / rho,
           (e + P) * jy / rho, (jx * jx - 3 * jy * jy) * jx / rho ** 2,
           (3 * jx * jx - jy * jy) * jy / rho ** 2,
           2 * e * e / rho - (jx * jx + jy * jy) ** 2 / (4 * rho ** 3), 0.0,
           A * (jx * jx - jy * jy) / rho ** 3, A * jx * jy / rho ** 3, 0.0, 0.0]
    dm = [-dt * s[k] * (m[k] - meq[k]) for k in range(16)]
    # solve M x = dm
    a = [Mt[k][:] + [dm[k]] for k in range(16)]
    for c in range(16):
        p = max(range(c, 16), key=lambda r: abs(a[r][c]))
        a[c], a[p] = a[p], a[c]
        for r in range(16):
            if r != c:
                fac = a[r][c] / a[c][c]
                a[r] = [x - fac * y for x, y in zip(a[r], a[c])]
    return [a[k][16] / a[k][k] for k in range(16)]


def test_single_node_step_is_pure_collision_brute_force():
    w = W.random_state(1, 1, seed=11)
    f = scheme.init_populations(*w.fields())
    rng = np.random.default_rng(11)
    f = f * (1.0 + 0.1 * rng.standard_normal(f.shape))
    g = scheme.step(f, w.cfg())
    dfl = _scalar_collision([float(x) for x in f[:, 0, 0]], w.s, w.dt)
    np.testing.assert_allclose(g[:, 0, 0] - f[:, 0, 0], dfl, rtol=1e-9,
                               atol=1e-13 * np.abs(f).max())
