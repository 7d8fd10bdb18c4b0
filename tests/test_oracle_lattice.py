"""Pins of the oracle's lattice and moment space against what the paper prints.

* M from formulas 5a-5p == the printed matrix (Sec. III.A), entry by entry.
* M^-1 is a two-sided inverse.
* E_alpha = M diag(v_alpha) M^-1 reproduces every flux coefficient of
  Eq. 9a-9p (both directions), which the paper derived from M and Eq. 4 --
  a transposed, mis-signed or mis-scaled entry anywhere in M or M^-1 breaks it.
"""
import math
import os

import numpy as np
import pytest

from oracle import lattice


def _printed_matrix(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "moment_matrix_printed.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([eval(tok, {"__builtins__": {}}, {"s2": math.sqrt(2.0)})
                         for tok in line.split()])
    return np.array(rows, dtype=np.float64)


def _eq9(golden_dir):
    out = {}
    with open(os.path.join(golden_dir, "flux_eq9.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, xs, ys = (part.strip() for part in line.split("|"))
            vecs = []
            for terms in (xs, ys):
                vec = np.zeros(16)
                for t in terms.split():
                    c, m = t.split("*m")
                    vec[int(m) - 1] += float(c)
                vecs.append(vec)
            out[int(k)] = vecs
    return out


def test_matrix_matches_printed(golden_dir):
    P = _printed_matrix(golden_dir)
    assert P.shape == (16, 16)
    M = lattice.moment_matrix()
    np.testing.assert_allclose(M, P, rtol=0, atol=1e-12 * np.abs(P).max())


def test_velocity_order_fixed_by_rows_2_3(golden_dir):
    P = _printed_matrix(golden_dir)
    v = lattice.velocities()
    np.testing.assert_allclose(v[:, 0], P[1], atol=1e-14)
    np.testing.assert_allclose(v[:, 1], P[2], atol=1e-14)
    speeds = np.hypot(v[:, 0], v[:, 1])
    np.testing.assert_allclose(speeds, [1] * 4 + [6] * 4 + [2] * 4 + [3] * 4)


def test_inverse_two_sided():
    _, M, Minv = lattice.matrices()
    I = np.eye(16)
    assert np.abs(M @ Minv - I).max() < 1e-13
    assert np.abs(Minv @ M - I).max() < 1e-13
    # matches an independent LAPACK inverse to rounding
    ref = np.linalg.inv(M)
    assert np.abs(Minv - ref).max() < 1e-12 * np.abs(ref).max()


def test_structure_counts():
    _, M, Minv = lattice.matrices()
    assert (np.abs(M) > 0).sum() == 192
    assert (np.abs(Minv) > 1e-13).sum() == 192


@pytest.mark.parametrize("axis", [0, 1])
def test_flux_matrices_reproduce_eq9(golden_dir, axis):
    v, M, Minv = lattice.matrices()
    E = M @ np.diag(v[:, axis]) @ Minv
    eq9 = _eq9(golden_dir)
    assert sorted(eq9) == list(range(1, 17))
    for k in range(1, 17):
        np.testing.assert_allclose(E[k - 1], eq9[k][axis], rtol=0, atol=1e-9,
                                   err_msg="Eq. 9 row %d, axis %d" % (k, axis))
