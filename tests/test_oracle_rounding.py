"""The oracle's own FP64 rounding error, measured against an extended-precision
(numpy longdouble) run of the same algorithm on a supersonic shock-reflection
problem, grows roughly linearly with the step count, at under 1e-14 per step
for rho, u, v, the populations, and T relative to max(e/rho). This is what
sets the FP64 parity tolerance of the GPU tests (harness.fp64_tol): two
correct FP64 evaluations in different operation orders differ by about the
sum of their rounding errors."""
import numpy as np
import pytest

import workloads as W
from oracle import lattice, scheme
from harness import field_errors


def _extended_matrices():
    ld = np.longdouble
    r2 = np.sqrt(ld(2))
    ax = [(1, 0), (0, 1), (-1, 0), (0, -1)]
    dg = [(1, 1), (-1, 1), (-1, -1), (1, -1)]
    v = np.array([(ld(a), ld(b)) for a, b in ax] + [(6 * ld(a), 6 * ld(b)) for a, b in ax]
                 + [(r2 * a, r2 * b) for a, b in dg] + [(3 / r2 * a, 3 / r2 * b) for a, b in dg])
    M = np.array(lattice.moment_rows(v[:, 0], v[:, 1]), dtype=ld)
    n = 16
    a = [list(M[i]) + [ld(1.0 if i == j else 0.0) for j in range(n)] for i in range(n)]
    for c in range(n):
        p = max(range(c, n), key=lambda r: abs(a[r][c]))
        a[c], a[p] = a[p], a[c]
        a[c] = [x / a[c][c] for x in a[c]]
        for r in range(n):
            if r != c and a[r][c] != 0:
                fac = a[r][c]
                a[r] = [x - fac * y for x, y in zip(a[r], a[c])]
    return v, M, np.array([row[n:] for row in a], dtype=ld)


@pytest.mark.slow
@pytest.mark.skipif(np.finfo(np.longdouble).eps > 1e-18, reason="needs extended long double")
def test_fp64_rounding_growth_against_extended_precision(monkeypatch):
    w = W.regular_reflection(nx=90, ny=30, dx=1e-3 * 600 / 90, dt=2e-6 * 600 / 90)
    ext = _extended_matrices()
    f64 = scheme.init_populations(*w.fields())
    monkeypatch.setattr(lattice, "_CACHE", {"m": ext})
    cfg = dict(w.cfg())
    cfg_ld = dict(cfg, dt=np.longdouble(cfg["dt"]), dx=np.longdouble(cfg["dx"]),
                  dy=np.longdouble(cfg["dy"]), s=np.array(cfg["s"], dtype=np.longdouble))
    fl = scheme.init_populations(*[np.asarray(a, dtype=np.longdouble) for a in w.fields()])
    monkeypatch.setattr(lattice, "_CACHE", {})
    done = 0
    for n in (10, 40, 100):
        for _ in range(n - done):
            f64 = scheme.step(f64, cfg)
            monkeypatch.setattr(lattice, "_CACHE", {"m": ext})
            fl = scheme.step(fl, cfg_ld)
            monkeypatch.setattr(lattice, "_CACHE", {})
        done = n
        monkeypatch.setattr(lattice, "_CACHE", {"m": ext})
        ref = dict(zip(("rho", "u", "v", "T"), (np.asarray(q, dtype=np.float64) for q in scheme.macroscopic(fl))))
        monkeypatch.setattr(lattice, "_CACHE", {})
        got = dict(zip(("rho", "u", "v", "T"), scheme.macroscopic(f64)))
        err = field_errors(got, ref)
        perr = float(np.abs(f64 - fl).max() / np.abs(fl).max())
        assert max(err.values()) < 1e-14 * n and perr < 1e-14 * n, (n, err, perr)
        assert max(err.values()) > 1e-17 * n     # the two runs do differ
