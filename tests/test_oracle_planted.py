"""The pins catch plausible mistakes: each test plants one mistake in a copy of
the oracle's arithmetic (on the CPU, by monkeypatching) and checks that the
corresponding pin then fails."""
import numpy as np
import pytest

from oracle import lattice, scheme
import test_oracle_advection as adv
import test_oracle_collision as col
import test_oracle_lattice as lat


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_sign_error_in_one_moment_row_breaks_eq9(golden_dir, monkeypatch):
    real = lattice.moment_rows

    def bad(vx, vy):
        rows = real(vx, vy)
        rows[9] = -rows[9]          # m_10 with the wrong sign
        return rows
    monkeypatch.setattr(lattice, "moment_rows", bad)
    monkeypatch.setattr(lattice, "_CACHE", {})
    _fails(lat.test_flux_matrices_reproduce_eq9, golden_dir, 0)
    _fails(lat.test_matrix_matches_printed, golden_dir)


def test_transposed_inverse_breaks_conservation(monkeypatch):
    v, M, Minv = lattice.matrices()
    monkeypatch.setattr(lattice, "_CACHE", {"m": (v, M, Minv.T.copy())})
    _fails(col.test_collision_conserves)


def test_wrong_equilibrium_breaks_maxwellian_pin(monkeypatch):
    real = scheme.moment_equilibria

    def bad(rho, jx, jy, e):
        out = real(rho, jx, jy, e).copy()
        out[6] = e * jx / rho        # f7^eq without the pressure term
        return out
    monkeypatch.setattr(scheme, "moment_equilibria", bad)
    _fails(col.test_equilibria_are_maxwellian_moments, 0)


def test_dropped_second_difference_breaks_fourier_pin(monkeypatch):
    def bad(g, dx, dy, dt):
        v, _, _ = lattice.matrices()
        vx = v[:, 0].reshape(16, 1, 1)
        vy = v[:, 1].reshape(16, 1, 1)
        return (vx * (g[:, 1:-1, 2:] - g[:, 1:-1, :-2]) / (2 * dx)
                + vy * (g[:, 2:, 1:-1] - g[:, :-2, 1:-1]) / (2 * dy))
    monkeypatch.setattr(scheme, "advection", bad)
    _fails(adv.test_fourier_amplification, 4, 1)


def test_swapped_neighbours_break_fourier_pin(monkeypatch):
    real = scheme.advection

    def bad(g, dx, dy, dt):
        return real(g[:, :, ::-1], dx, dy, dt)[:, :, ::-1]
    monkeypatch.setattr(scheme, "advection", bad)
    _fails(adv.test_fourier_amplification, 4, 1)
