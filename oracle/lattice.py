"""D2V16 lattice and moment space (Sec. III.A of the paper).

Test infrastructure only (see ``oracle/__init__``).

* ``velocities()``      -- Eq. 4: four groups of four velocities.
* ``moment_matrix()``   -- Eqs. 5a-5p evaluated on Eq. 4; the paper prints the
                           result (Sec. III.A, the 16 rows m_1..m_16).
* ``inverse_matrix()``  -- M^-1 (Sec. II: f = M^-1 f_hat), Gauss-Jordan with
                           partial pivoting in extended precision.

Reading of Eq. 4's ordering: "cyc" lists the axis groups as (1,0), (0,1),
(-1,0), (0,-1) (times 1 and times 6) and the diagonal groups as (+,+), (-,+),
(-,-), (+,-) (times sqrt2 and 3/sqrt2). The printed rows m_2 and m_3 fix this
order uniquely, and a test compares the whole printed matrix.
"""
import numpy as np

Q = 16  # number of discrete velocities


def velocities():
    """Eq. 4: (v_ix, v_iy) for i = 1..16, returned as a (16, 2) float64 array
    (row i-1 holds velocity i)."""
    axis = [(1.0, 0.0), (0.0, 1.0), (-1.0, 0.0), (0.0, -1.0)]
    diag = [(1.0, 1.0), (-1.0, 1.0), (-1.0, -1.0), (1.0, -1.0)]
    v = []
    for (x, y) in axis:                      # i = 1..4: cyc (+-1, 0)
        v.append((x, y))
    for (x, y) in axis:                      # i = 5..8: cyc (+-6, 0)
        v.append((6.0 * x, 6.0 * y))
    r2 = np.sqrt(2.0)
    for (x, y) in diag:                      # i = 9..12: sqrt2 (+-1, +-1)
        v.append((r2 * x, r2 * y))
    c = 3.0 / np.sqrt(2.0)
    for (x, y) in diag:                      # i = 13..16: 3/sqrt2 (+-1, +-1)
        v.append((c * x, c * y))
    return np.array(v, dtype=np.float64)


def moment_rows(vx, vy):
    """Eqs. 5a-5p: the 16 polynomial moments of a velocity (vx, vy).

    Works elementwise on arrays, so it also gives the continuous moments
    m_k(v) used to take Maxwellian moments by quadrature in the tests.
    Returns a list of 16 arrays (k = 1..16 at index k-1).
    """
    v2 = vx * vx + vy * vy
    return [
        np.ones_like(vx),                                  # 5a
        vx,                                                # 5b
        vy,                                                # 5c
        v2 / 2.0,                                          # 5d
        vx * vx - vy * vy,                                 # 5e
        vx * vy,                                           # 5f
        vx * v2 / 2.0,                                     # 5g
        vy * v2 / 2.0,                                     # 5h
        vx * (vx * vx - 3.0 * vy * vy),                    # 5i
        vy * (3.0 * vx * vx - vy * vy),                    # 5j
        v2 * v2 / 4.0,                                     # 5k
        vx ** 4 - 6.0 * vx * vx * vy * vy + vy ** 4,       # 5l
        v2 * (vx * vx - vy * vy),                          # 5m
        v2 * vx * vy,                                      # 5n
        vx * (vx * vx - 3.0 * vy * vy) * v2,               # 5o
        vy * (3.0 * vx * vx - vy * vy) * v2,               # 5p
    ]


def moment_matrix():
    """M with m_ki = (Eq. 5k-th formula)(v_i); shape (16, 16), float64."""
    v = velocities()
    rows = moment_rows(v[:, 0], v[:, 1])
    return np.array([np.asarray(r, dtype=np.float64) for r in rows])


def inverse_matrix(M=None):
    """M^-1 by Gauss-Jordan elimination with partial pivoting, carried out in
    numpy's extended precision (``np.longdouble``) and rounded to float64.

    Sec. II defines f = M^-1 f_hat; the paper does not print M^-1. This is a
    plain textbook elimination written out with loops (16 x 16 is small).
    """
    if M is None:
        M = moment_matrix()
    n = M.shape[0]
    a = [[np.longdouble(M[i, j]) for j in range(n)] +
         [np.longdouble(1.0 if i == j else 0.0) for j in range(n)]
         for i in range(n)]
    for col in range(n):
        piv = max(range(col, n), key=lambda r: abs(a[r][col]))
        if a[piv][col] == 0:
            raise ValueError("singular moment matrix")
        a[col], a[piv] = a[piv], a[col]
        p = a[col][col]
        a[col] = [x / p for x in a[col]]
        for r in range(n):
            if r != col and a[r][col] != 0:
                fac = a[r][col]
                a[r] = [x - fac * y for x, y in zip(a[r], a[col])]
    return np.array([[float(a[i][n + j]) for j in range(n)] for i in range(n)],
                    dtype=np.float64)


_CACHE = {}


def matrices():
    """(v, M, Minv) computed once per process."""
    if "m" not in _CACHE:
        M = moment_matrix()
        _CACHE["m"] = (velocities(), M, inverse_matrix(M))
    return _CACHE["m"]
