"""Pins of the Sec. IV amplification matrix G in ``oracle/stability.py``.

* With S_hat = 0 (no collision) G is diagonal and its entries are the
  Lax-Wendroff factors 1 - i C sin(theta) - C^2 (1 - cos theta) per axis, of
  modulus |omega|^2 = 1 - C^2 (1 - C^2) (1 - cos theta)^2 in 1D (closed form).
* At k = 0 the eigenvalues are 1 four times (the conserved moments) and
  1 - dt s_k for the twelve others: in the moment basis S_hat (I - J) is block
  triangular with a zero block for the conserved rows.
* G F is the linear part of one step of ``scheme.step``: on a periodic grid a
  perturbation eps Re(F e^{i k.x}) of a uniform equilibrium state maps to
  eps Re((G F) e^{i k.x}) (central difference in eps through the nonlinear
  scheme; brute force). Dropping the collision term from G, or flipping the
  sign of its advective part, fails this check.
* The complex-step derivative of the Eq. 14 equilibria agrees with central
  finite differences.
"""
import numpy as np
import pytest

from oracle import scheme, stability
from oracle.lattice import matrices

STATE = (1.3, 0.2, -0.1, 0.9)


def _rates(seed):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(1e2), np.log(1e4), 16))


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.1, np.pi / 2, 2.9, np.pi])
def test_no_collision_gives_lax_wendroff_factors(theta):
    dx, dt = 2e-3, 1e-4
    G = stability.amplification_matrix(STATE, np.zeros(16), dx, dx, dt, theta / dx, 0.0)
    assert np.count_nonzero(G - np.diag(np.diag(G))) == 0
    vel, _, _ = matrices()
    C = vel[:, 0] * dt / dx
    lw = 1.0 - 1j * C * np.sin(theta) - C ** 2 * (1.0 - np.cos(theta))
    np.testing.assert_allclose(np.diag(G), lw, rtol=0, atol=1e-15)
    mod2 = 1.0 - C ** 2 * (1.0 - C ** 2) * (1.0 - np.cos(theta)) ** 2
    np.testing.assert_allclose(np.abs(np.diag(G)) ** 2, mod2, rtol=0, atol=1e-14)


def test_no_collision_2d_factor_is_sum_of_axes():
    dx, dy, dt, tx, ty = 2e-3, 3e-3, 1e-4, 0.7, 2.2
    G = stability.amplification_matrix(STATE, np.zeros(16), dx, dy, dt, tx / dx, ty / dy)
    vel, _, _ = matrices()
    cx, cy = vel[:, 0] * dt / dx, vel[:, 1] * dt / dy
    lw = (1.0 - 1j * cx * np.sin(tx) - cx ** 2 * (1 - np.cos(tx))
          - 1j * cy * np.sin(ty) - cy ** 2 * (1 - np.cos(ty)))
    np.testing.assert_allclose(np.diag(G), lw, rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_zero_wave_number_spectrum(seed):
    s = _rates(seed)
    dt = 1e-4
    G = stability.amplification_matrix(STATE, s, 2e-3, 2e-3, dt, 0.0, 0.0)
    w = np.sort_complex(stability.eigenvalues(G))
    expect = np.sort_complex(np.concatenate([np.ones(4), 1.0 - dt * s[4:]]).astype(complex))
    np.testing.assert_allclose(w, expect, rtol=0, atol=1e-12)


def _linear_part(G_fn, seed):
    nx, ny, dx, dy, dt = 8, 4, 0.01, 0.02, 1e-4
    s = _rates(seed)
    kx, ky = 2 * np.pi * 3 / (nx * dx), 2 * np.pi * 1 / (ny * dy)
    rng = np.random.default_rng(100 + seed)
    F = rng.normal(size=16) + 1j * rng.normal(size=16)
    f0 = scheme.equilibrium_populations(*[np.full((ny, nx), q) for q in STATE])
    x = np.arange(nx)[None, :] * dx
    y = np.arange(ny)[:, None] * dy
    phase = np.exp(1j * (kx * x + ky * y))
    eps = 1e-6 * np.abs(f0).max()
    pert = eps * np.real(F[:, None, None] * phase[None])
    per = ("periodic", None)
    cfg = {"dx": dx, "dy": dy, "dt": dt, "s": s, "bc": (per, per, per, per)}
    lin = (scheme.step(f0 + pert, cfg) - scheme.step(f0 - pert, cfg)) / 2.0
    G = G_fn(STATE, s, dx, dy, dt, kx, ky)
    want = eps * np.real((G @ F)[:, None, None] * phase[None])
    return float(np.abs(lin - want).max() / np.abs(want).max())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_G_is_the_linear_part_of_one_scheme_step(seed):
    assert _linear_part(stability.amplification_matrix, seed) < 1e-8


def test_linearisation_pin_catches_planted_mistakes():
    def no_collision(state, s, *a):
        return stability.amplification_matrix(state, np.zeros(16), *a)

    def flipped_advection(state, s, dx, dy, dt, kx, ky):
        return stability.amplification_matrix(state, s, dx, dy, dt, -kx, -ky)

    assert _linear_part(no_collision, 0) > 1e-4
    assert _linear_part(flipped_advection, 0) > 1e-4


def test_complex_step_jacobian_matches_finite_differences():
    J = stability.equilibrium_jacobian(*STATE)
    c = np.array(scheme.conserved_from_state(*STATE))
    h = 1e-6
    for q in range(4):
        cp, cm = c.copy(), c.copy()
        cp[q] += h
        cm[q] -= h
        fd = (scheme.moment_equilibria(*cp) - scheme.moment_equilibria(*cm)) / (2 * h)
        np.testing.assert_allclose(J[:, q], fd, rtol=1e-7, atol=1e-8)
    np.testing.assert_array_equal(J[:4], np.eye(4))  # conserved rows
