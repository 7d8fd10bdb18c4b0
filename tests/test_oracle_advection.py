"""Pins of the oracle's space/time discretisation (Eq. A.1) and ghost nodes.

* Pure advection (S_hat = 0) of a Fourier mode multiplies it by the
  Lax-Wendroff amplification 1 - i c sin(k dx) - c^2 (1 - cos(k dx)),
  c = v dt / dx -- the advective part of the von Neumann matrix G of Sec. IV.
  This catches a wrong sign, a missing 1/2, a swapped neighbour or a missing
  second-difference term.
* On a periodic grid the advection telescopes: the grid sum of every
  population is unchanged (S_hat = 0), and with collision the grid totals of
  rho, j, e are unchanged.
* Corner ghosts are never read (they are NaN in the oracle).
* Ghost states of the reflecting, extrapolating and wall sides.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lattice, scheme


def _cfg(nx, ny, dx, dy, dt, s, bc=None):
    return {"nx": nx, "ny": ny, "dx": dx, "dy": dy, "dt": dt, "s": s,
            "bc": bc or (("periodic", None),) * 4}


@pytest.mark.parametrize("i", [0, 1, 4, 5, 8, 11, 12, 15])
@pytest.mark.parametrize("mode", [1, 3])
def test_fourier_amplification(i, mode):
    nx = ny = 16
    dx, dy, dt = 0.01, 0.013, 4e-4
    v, _, _ = lattice.matrices()
    base = scheme.init_populations(*(np.full((ny, nx), x) for x in (1.0, 0.1, 0.05, 1.0)))
    X = np.arange(nx)[None, :]
    Y = np.arange(ny)[:, None]
    kx, ky = 2 * np.pi * mode / nx, 2 * np.pi * (mode + 1) / ny
    phase = kx * X + ky * Y
    eps = 1e-3
    f = base.copy()
    f[i] = f[i] + eps * np.cos(phase)
    g = scheme.step(f, _cfg(nx, ny, dx, dy, dt, (0.0,) * 16))
    cx = v[i, 0] * dt / dx
    cy = v[i, 1] * dt / dy
    G = (1 - 1j * cx * np.sin(kx) - cx * cx * (1 - np.cos(kx))
         - 1j * cy * np.sin(ky) - cy * cy * (1 - np.cos(ky)))
    expect = base[i] + eps * np.real(G * np.exp(1j * phase))
    np.testing.assert_allclose(g[i], expect, rtol=0, atol=1e-15 * 50)
    others = [k for k in range(16) if k != i]
    np.testing.assert_allclose(g[others], base[others], rtol=0, atol=1e-14)


def test_periodic_advection_conserves_each_population():
    w = W.random_state(13, 11, seed=5, smooth=False)
    f = scheme.init_populations(*w.fields())
    g = scheme.step(f, _cfg(13, 11, 0.01, 0.02, 2e-4, (0.0,) * 16))
    np.testing.assert_allclose(g.sum(axis=(1, 2)), f.sum(axis=(1, 2)), rtol=1e-13)
    assert np.abs(g - f).max() > 1e-4


def test_periodic_step_conserves_totals():
    w = W.random_state(12, 10, seed=6, smooth=False)
    f = scheme.init_populations(*w.fields())
    t0 = scheme.conserved_totals(f, w.dx, w.dy)
    for _ in range(20):
        f = scheme.step(f, w.cfg())
    t1 = scheme.conserved_totals(f, w.dx, w.dy)
    np.testing.assert_allclose(t1, t0, rtol=1e-13, atol=1e-15)


def test_corners_are_never_read():
    bc = (("eq", (1.0, 0.1, 0.0, 1.0)), ("extrap", None),
          ("reflect", None), ("wall", (1.0, 0.3, 0.0, 1.2)))
    w = W.random_state(7, 6, seed=2, bc=bc)
    f = scheme.init_populations(*w.fields())
    g = scheme.padded(f, w.bc)
    assert np.isnan(g[:, 0, 0]).all() and np.isnan(g[:, -1, -1]).all()
    out = scheme.step(f, w.cfg())
    assert np.isfinite(out).all()


def test_ghost_states():
    w = W.random_state(5, 4, seed=9)
    f = scheme.init_populations(*w.fields())
    rho, u, v, T = scheme.macroscopic(f)
    # reflecting bottom: (rho, u, -v, T) of row 0
    gl = scheme._ghost_line(f, "y-", ("reflect", None))
    r, uu, vv, TT = scheme.macroscopic(gl)
    np.testing.assert_allclose(np.stack([r, uu, vv, TT]),
                               np.stack([rho[0], u[0], -v[0], T[0]]), rtol=1e-12, atol=1e-13)
    # reflecting right side: (rho, -u, v, T) of the last column
    gl = scheme._ghost_line(f, "x+", ("reflect", None))
    np.testing.assert_allclose(scheme.macroscopic(gl)[1], -u[:, -1], atol=1e-13)
    # extrapolation on the left side: 2 q(col 0) - q(col 1)
    gl = scheme._ghost_line(f, "x-", ("extrap", None))
    got = np.stack(scheme.macroscopic(gl))
    want = np.stack([2 * q[:, 0] - q[:, 1] for q in (rho, u, v, T)])
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12)
    # moving wall on the top: rho of the last row, prescribed u, v, T
    gl = scheme._ghost_line(f, "y+", ("wall", (9.9, 0.25, -0.1, 1.5)))
    got = np.stack(scheme.macroscopic(gl))
    want = np.stack([rho[-1], np.full(5, 0.25), np.full(5, -0.1), np.full(5, 1.5)])
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_outflow_ghost_agrees_with_reflect_and_extrap_where_they_coincide():
    """Zero-gradient outflow (reading R20) against the two other kinds built
    from the adjacent node: equal to the reflecting ghost where the normal
    velocity is zero, and to the extrapolating one where the first two
    interior lines are equal."""
    w = W.random_state(6, 5, seed=31)
    rho, u, v, T = (np.array(a, dtype=np.float64) for a in w.fields())
    v[0, :] = 0.0                                  # no normal velocity on row 0
    f = scheme.init_populations(rho, u, v, T)
    np.testing.assert_allclose(scheme._ghost_line(f, "y-", ("outflow", None)),
                               scheme._ghost_line(f, "y-", ("reflect", None)), rtol=0, atol=1e-14)
    rho2, u2, v2, T2 = (a.copy() for a in (rho, u, v, T))
    for q in (rho2, u2, v2, T2):
        q[:, 1] = q[:, 0]                          # columns 0 and 1 equal
    f2 = scheme.init_populations(rho2, u2, v2, T2)
    np.testing.assert_allclose(scheme._ghost_line(f2, "x-", ("outflow", None)),
                               scheme._ghost_line(f2, "x-", ("extrap", None)), rtol=1e-12, atol=1e-13)


def test_uniform_state_is_fixed_with_outflow_sides():
    n = (7, 5)
    st = (1.3, 0.2, -0.1, 0.8)
    f = scheme.init_populations(*(np.full(n[::-1], x) for x in st))
    bc = (("outflow", None),) * 4
    w = W.random_state(n[0], n[1], seed=1, bc=bc)
    out = scheme.step(f, w.cfg())
    np.testing.assert_allclose(out, f, rtol=1e-12, atol=1e-13)


def test_extrapolation_falls_back_when_unphysical():
    rho = np.array([[0.2, 1.0]])
    T = np.array([[1.0, 1.0]])
    z = np.zeros((1, 2))
    f = scheme.init_populations(rho, z, z, T)
    gl = scheme._ghost_line(f, "x-", ("extrap", None))   # 2*0.2 - 1.0 < 0
    np.testing.assert_allclose(scheme.macroscopic(gl)[0], [0.2], rtol=1e-13)


def test_one_step_matches_formula_at_a_boundary_node():
    """Direct evaluation of Eq. A.1 at node (0, 0) of a small grid with a
    Dirichlet left side and a reflecting bottom, from the definitions."""
    bc = (("eq", (1.1, 0.2, 0.0, 0.9)), ("extrap", None), ("reflect", None),
          ("eq", (0.9, 0.1, -0.1, 1.1)))
    w = W.random_state(4, 3, seed=21, bc=bc)
    f = scheme.init_populations(*w.fields())
    out = scheme.step(f, w.cfg())
    v, _, _ = lattice.matrices()
    west = scheme.equilibrium_populations(*(np.array([x]) for x in (1.1, 0.2, 0.0, 0.9)))[:, 0]
    r, uu, vv, TT = (q[0, 0] for q in scheme.macroscopic(f))
    south = scheme.equilibrium_populations(*(np.array([x]) for x in (r, uu, -vv, TT)))[:, 0]
    c = f[:, 0, 0]
    e = f[:, 0, 1]
    n = f[:, 1, 0]
    adv = (v[:, 0] * (e - west) / (2 * w.dx) + v[:, 1] * (n - south) / (2 * w.dy)
           - v[:, 0] ** 2 * w.dt * (e - 2 * c + west) / (2 * w.dx ** 2)
           - v[:, 1] ** 2 * w.dt * (n - 2 * c + south) / (2 * w.dy ** 2))
    want = c - w.dt * adv + scheme.collision(f, w.s, w.dt)[:, 0, 0]
    np.testing.assert_allclose(out[:, 0, 0], want, rtol=1e-13, atol=1e-15)
