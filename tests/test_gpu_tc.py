"""GPU tests of the tensor-core step (precision LBM_TC_TF32X3): the two
16 x 16 moment transforms run as tcgen05 MMAs (A in tensor memory, two nodes
per thread, 32 x 8 node tiles) with the 3xTF32 split (a_hi b_hi + a_hi b_lo
+ a_lo b_hi, FP32 accumulation).

Bar against the FP64 oracle: the same bound as the FP32 step (the dropped
a_lo b_lo term and the product's reading of a_lo to 19 bits are each below
2^-21 relative, a few units of FP32 rounding): relative
L-infinity <= 30 u sqrt(n) + 3e-6 for smooth flows, u = 2^-24. The audit and
the watchdog run through the same epilogue as the other precisions.
"""
import math

import numpy as np
import pytest

import workloads as W
from harness import field_errors, gpu_run, oracle_run, pop_error

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def bound(n):
    return 30 * U32 * math.sqrt(max(n, 1)) + 3e-6


@pytest.mark.parametrize("nx,ny,nsteps", [(1, 1, 3), (33, 9, 20), (70, 19, 100), (129, 13, 50)])
def test_tc_periodic_matches_oracle(nx, ny, nsteps):
    w = W.random_state(nx, ny, seed=nx + 7 * ny, smooth=nx * ny > 20)
    got, f, status = gpu_run(w, nsteps, "tc_tf32x3")
    ref, fref = oracle_run(w, nsteps)
    err = field_errors(got, ref)
    print("tc", nx, ny, nsteps, err, pop_error(f, fref))
    assert max(err.values()) <= bound(nsteps), err
    assert status[0] == 0


def test_tc_boundaries_match_oracle():
    bc = (("eq", (1.0, 0.3, 0.0, 1.0)), ("extrap", None), ("reflect", None),
          ("eq", (1.2, 0.25, -0.1, 1.1)))
    w = W.random_state(64, 17, seed=9, smooth=True, bc=bc)
    got, f, status = gpu_run(w, 100, "tc_tf32x3")
    ref, _ = oracle_run(w, 100)
    err = field_errors(got, ref)
    assert max(err.values()) <= bound(100), err


def test_tc_close_to_fp32_path_on_bubble():
    w = W.shock_bubble(nx=256, ny=128, radius=16)
    a, fa, sa = gpu_run(w, 200, "tc_tf32x3")
    b, fb, sb = gpu_run(w, 200, "fp32")
    c, fc, sc = gpu_run(w, 200, "fp64")
    e_tc = field_errors(a, c)
    e_32 = field_errors(b, c)
    print("bubble 256x128, 200 steps: tc vs fp64", e_tc, "fp32 vs fp64", e_32)
    assert sa[0] == sb[0] == sc[0] == 0
    assert max(e_tc.values()) < 10 * max(max(e_32.values()), 1e-6)


def test_tc_audit_conserves_on_periodic_grid():
    from paper_0908_3749_gb300 import lbm
    w = W.random_state(96, 40, seed=4, smooth=True)
    cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, "tc_tf32x3", 10)
    ctx = lbm.lbm_create(cfg)
    try:
        lbm.lbm_set_init(ctx, *[np.ascontiguousarray(a) for a in w.fields()])
        lbm.lbm_step(ctx, 200)       # graph batches and single launches
        log, steps = lbm.lbm_audit_log(ctx)
        assert steps == list(range(0, 200, 10))
        t = np.array(log)
        drift = np.abs(t - t[0]).max(axis=0) / np.abs(t[0]).max()
        assert drift.max() < 2e-5, drift
        rc, bad, _ = lbm.lbm_status(ctx)
        assert rc == 0 and bad == -1
    finally:
        lbm.lbm_destroy(ctx)


def _planted_nan_run(precision, node):
    """One step from a state with one non-finite population: the first bad
    step and the nodes whose output is not finite."""
    from paper_0908_3749_gb300 import lbm
    w = W.random_state(64, 16, seed=21, smooth=True)
    cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, precision, 0)
    ctx = lbm.lbm_create(cfg)
    try:
        lbm.lbm_set_init(ctx, *[np.ascontiguousarray(a) for a in w.fields()])
        lbm.lbm_step(ctx, 5)
        f = np.empty((16, w.ny, w.nx), dtype=np.float32)
        step = lbm.lbm_get_populations(ctx, f)
        f[8, node[1], node[0]] = np.nan   # a diagonal population: x and y neighbours
        lbm.lbm_set_populations(ctx, f, step)
        lbm.lbm_step(ctx, 1)
        rc, bad, _ = lbm.lbm_status(ctx)
        out = np.empty_like(f)
        lbm.lbm_get_populations(ctx, out)
    finally:
        lbm.lbm_destroy(ctx)
    return step, rc, bad, set(zip(*np.nonzero(~np.isfinite(out).all(axis=0))))


def test_tc_planted_nan_reaches_the_partner_node_and_the_watchdog():
    """The two nodes of a thread (rows y and y + 4 of a 32 x 8 tile) share an
    MMA row: a non-finite population of one makes the other's update
    non-finite in the same step (zero coefficients times NaN). The watchdog
    reports the step that holds the NaN, as the FP32 step does; the
    non-finite outputs are the NaN node, its four stencil neighbours and, in
    the tensor-core form only, the partner node."""
    from paper_0908_3749_gb300 import lbm
    node = (10, 2)                       # (x, y): tile row 2, partner row 6
    s32, rc32, bad32, nf32 = _planted_nan_run("fp32", node)
    stc, rctc, badtc, nftc = _planted_nan_run("tc_tf32x3", node)
    assert rc32 == rctc == lbm.LBM_ERR_NONFINITE
    assert bad32 == badtc == s32 == stc, (bad32, badtc, s32)
    x, y = node
    stencil = {(y, x), (y, x - 1), (y, x + 1), (y - 1, x), (y + 1, x)}
    assert nf32 == stencil, nf32
    assert nftc == stencil | {(y + 4, x)}, nftc
