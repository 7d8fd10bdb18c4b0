"""Two time steps per launch (lbm_set_fused_steps(ctx, 2), FP32 grids).

The fused kernel computes each node with the one-step arithmetic, the ring of
intermediate nodes around a tile in unpaired FP32, so it must agree with
single FP32 steps to FP32 rounding and with the FP64 oracle within the FP32
bounds of test_gpu_parity_fp32.py (both comparisons take the case's bar: on
the shock cases last-bit differences grow as they do against FP64). The cases cover what is special to it:
periodic wraps in x and y on grids that are not multiples of the tile
(nx = 70, ny = 19; ny = 4 < the tile height), a one-node-deep grid in each
direction, every boundary kind (Dirichlet, reflecting, extrapolating,
outflow, wall, and split sides that move with time), odd step counts (a
final single step), graph-captured runs (>= 64 steps), the audit log and the
watchdog.
"""
import math

import numpy as np
import pytest

import workloads as W
from harness import field_errors, oracle_run

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def bound(n):
    return 30 * U32 * math.sqrt(max(n, 1)) + 3e-6


def run(w, nsteps, fused, audit_every=0, chunks=None):
    from paper_0908_3749_gb300 import lbm
    cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, "fp32", audit_every)
    ctx = lbm.lbm_create(cfg)
    try:
        lbm.lbm_set_init(ctx, *[np.ascontiguousarray(a, dtype=np.float64) for a in w.fields()])
        if fused:
            lbm.lbm_set_fused_steps(ctx, 2)
        for n in (chunks or [nsteps]):
            lbm.lbm_step(ctx, n)
        out = {k: np.empty((w.ny, w.nx)) for k in ("rho", "u", "v", "T")}
        lbm.lbm_moments(ctx, out["rho"], out["u"], out["v"], out["T"])
        f = np.empty((16, w.ny, w.nx), dtype=np.float32)
        steps = lbm.lbm_get_populations(ctx, f)
        status = lbm.lbm_status(ctx)
        log = lbm.lbm_audit_log(ctx) if audit_every else None
    finally:
        lbm.lbm_destroy(ctx)
    return out, f.astype(np.float64), status, steps, log


BCS = {
    "mixed": (("eq", (1.0, 0.3, 0.0, 1.0)), ("extrap", None), ("reflect", None),
              ("eq", (1.2, 0.25, -0.1, 1.1))),
    "outflow_wall": (("outflow", None), ("extrap", None), ("wall", (1.0, -0.1, 0.0, 1.0)),
                     ("wall", (1.0, 0.2, 0.0, 1.1))),
    "periodic_x": (("periodic", None), ("periodic", None), ("reflect", None), ("extrap", None)),
    "periodic_y": (("outflow", None), ("eq", (1.1, 0.1, 0.0, 0.9)), ("periodic", None),
                   ("periodic", None)),
}

CASES = [
    ("periodic_70x19", lambda: W.random_state(70, 19, seed=70, smooth=True), 101, None),
    ("mixed_64x17", lambda: W.random_state(64, 17, seed=9, smooth=True, bc=BCS["mixed"]), 100, None),
    ("outflow_wall_45x23", lambda: W.random_state(45, 23, seed=4, smooth=True, bc=BCS["outflow_wall"]),
     66, None),
    ("periodic_x_one_row", lambda: W.random_state(37, 1, seed=5, smooth=True, bc=BCS["periodic_x"]),
     30, None),
    ("periodic_y_one_column", lambda: W.random_state(1, 29, seed=6, smooth=True, bc=BCS["periodic_y"]),
     30, None),
    ("sod_ny4", lambda: W.sod_config1("stable", ny=4), 1000, None),
    ("reflection", lambda: W.regular_reflection(), 40, 2e-4),
    ("mach_split", lambda: W.mach_reflection(nx=96, ny=48, dx=0.003, foot=24), 31, 2e-4),
]


@pytest.mark.parametrize("name,make,nsteps,tol", CASES, ids=[c[0] for c in CASES])
def test_fused_against_oracle_and_single_steps(name, make, nsteps, tol):
    w = make()
    got, f, status, steps, _ = run(w, nsteps, fused=True)
    one, f1, status1, _, _ = run(w, nsteps, fused=False)
    ref, _ = oracle_run(w, nsteps)
    assert steps == nsteps and status[0] == 0 and status[1] == -1
    err = max(field_errors(got, ref).values())
    diff = float(np.abs(f - f1).max() / np.abs(f1).max())
    tol = bound(nsteps) if tol is None else tol
    print("fused %s n=%d: vs oracle %.3g (bar %.3g), vs single steps %.3g" % (name, nsteps, err, tol, diff))
    assert err <= tol
    assert diff <= tol      # with a shock on the grid, last-bit differences grow as against FP64


def test_fused_audits_and_levels_match_single_steps():
    w = W.random_state(64, 40, seed=12, smooth=True, bc=BCS["mixed"])
    _, _, _, steps, log = run(w, 131, fused=True, audit_every=10, chunks=[3, 64, 1, 63])
    _, _, _, steps1, log1 = run(w, 131, fused=False, audit_every=10)
    assert steps == steps1 == 131
    tot, lv = log
    tot1, lv1 = log1
    assert lv == lv1 == list(range(0, 131, 10))
    t, t1 = np.array(tot), np.array(tot1)
    assert np.array_equal(t[0], t1[0])            # level 0: the same input
    np.testing.assert_allclose(t, t1, rtol=1e-6, atol=1e-9)


def test_fused_with_audit_every_step_takes_single_steps():
    w = W.random_state(40, 16, seed=3, smooth=True, bc=BCS["mixed"])
    a = run(w, 12, fused=True, audit_every=1)
    b = run(w, 12, fused=False, audit_every=1)
    assert np.array_equal(a[1], b[1]) and a[4] == b[4]


def test_fused_watchdog_level_matches_single_steps():
    """Sod with every rate 1e5 (the paper's literal Sod rates) turns
    unphysical after about a thousand steps; both modes report the same first
    bad level."""
    w = W.sod_config1("literal", ny=4)
    _, _, st, _, _ = run(w, 1400, fused=True)
    _, _, st1, _, _ = run(w, 1400, fused=False)
    print("first bad level: fused %d, single %d" % (st[1], st1[1]))
    assert st1[1] > 0 and abs(st[1] - st1[1]) <= 1


def test_set_fused_steps_validation():
    from paper_0908_3749_gb300 import lbm
    w = W.random_state(40, 16, seed=3)
    for prec, ok in (("fp32", True), ("fp64", False), ("tc_tf32x3", False)):
        cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, prec, 0)
        ctx = lbm.lbm_create(cfg)
        try:
            assert lbm.lbm_fused_steps(ctx) == 1
            if ok:
                lbm.lbm_set_fused_steps(ctx, 2)
                assert lbm.lbm_fused_steps(ctx) == 2
                with pytest.raises(lbm.LBMError) as ei:
                    lbm.lbm_set_fused_steps(ctx, 3)
                assert ei.value.code == lbm.LBM_ERR_INVALID
            else:
                with pytest.raises(lbm.LBMError) as ei:
                    lbm.lbm_set_fused_steps(ctx, 2)
                assert ei.value.code == lbm.LBM_ERR_UNSUPPORTED
        finally:
            lbm.lbm_destroy(ctx)
