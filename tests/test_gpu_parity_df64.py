"""The double-word step (LBM_DF64) against the FP64 oracle through the C ABI.

LBM_DF64 keeps every population as an unevaluated pair h + l of FP32 numbers
and does every operation of the step with error-free FP32 transformations
(TwoSum, FMA-based TwoProd): a rounding error of about 2^-48 of the operands
per operation where FP64 has 2^-53. Its bar (harness.df64_tol) is the FP64
bar scaled by 2^-48 / 2^-53 = 32 (3.2e-11 relative L-infinity per field and
for the populations up to 100 steps, 3.2e-13 per step beyond), or, where the
populations are large against rho (kappa = max sum_i |f_i| / rho), the
storage bound 16 kappa 2^-48 per step, whichever is larger. The tests print
the measured errors next to the bar.
"""
import numpy as np
import pytest

import workloads as W
from harness import (cancellation, df64_tol, field_errors, gpu_run, oracle_run, pop_error,
                     read_populations)
from test_gpu_parity_fp64 import BC_SETS

pytestmark = pytest.mark.gpu


def _kappa(w):
    """kappa of the initial state (the oracle's equilibrium populations)."""
    from oracle import scheme
    return cancellation(scheme.init_populations(*w.fields()))


def _check(w, nsteps, tol=None):
    got, f, status = gpu_run(w, nsteps, "df64")
    ref, fref = oracle_run(w, nsteps)
    tol = df64_tol(nsteps, _kappa(w)) if tol is None else tol
    err = field_errors(got, ref)
    perr = pop_error(f, fref)
    print("\n%s n=%d df64: fields %s pop %.2e (bar %.1e)"
          % (w.name, nsteps, {k: "%.2e" % v for k, v in err.items()}, perr, tol))
    assert status[0] == 0
    assert max(err.values()) <= tol and perr <= tol, (w.name, nsteps, err, perr)
    return err, perr


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 1), (1, 5), (5, 3), (33, 9), (70, 19), (100, 37)])
@pytest.mark.parametrize("nsteps", [1, 10])
def test_periodic_random(nx, ny, nsteps):
    w = W.random_state(nx, ny, seed=nx * 100 + ny, smooth=(nx * ny > 20))
    _check(w, nsteps)


@pytest.mark.parametrize("bcs", range(len(BC_SETS)))
@pytest.mark.parametrize("nx,ny", [(2, 2), (37, 11), (64, 17)])
def test_boundary_kinds(bcs, nx, ny):
    w = W.random_state(nx, ny, seed=7 + bcs, bc=BC_SETS[bcs], smooth=True)
    _check(w, 12)


def test_boundaries_one_node_deep():
    bc = (("extrap", None), ("reflect", None), ("wall", (1.0, 0.1, 0.0, 1.0)), ("extrap", None))
    for nx, ny in ((1, 6), (6, 1), (1, 1)):
        _check(W.random_state(nx, ny, seed=3, bc=bc), 5)


@pytest.mark.parametrize("nsteps", [1, 10, 100])
def test_regular_reflection_full_size(nsteps):
    _check(W.regular_reflection(), nsteps)


def test_sod_config1_stable_full_run():
    w = W.sod_config1("stable", ny=4)
    _check(w, w.nsteps)


def test_mach_reflection_split_sides_40_steps():
    _check(W.mach_reflection(), 40)


def test_watchdog_first_bad_step_matches_oracle():
    """The literal Sod configuration blows up near level 1120; the
    double-word run reaches it within five levels of the oracle (its state
    differs from the FP64 one by about 1e-11 when the instability starts to
    grow, and the growth amplifies that difference)."""
    from oracle import scheme
    from paper_0908_3749_gb300.lbm import LBM_ERR_NONFINITE
    w = W.sod_config1("literal", ny=4)
    _, bad_ref = scheme.run(scheme.init_populations(*w.fields()), w.cfg(), 1500, check_every=1)
    _, _, (rc, bad, negT) = gpu_run(w, 1500, "df64")
    assert rc == LBM_ERR_NONFINITE
    assert bad_ref is not None and abs(bad - bad_ref) <= 5, (bad, bad_ref)


def test_launch_shapes_checkpoint_and_audit():
    """Every launch shape gives bitwise the same populations; a checkpoint
    restores the run bitwise; the audit totals match the oracle's totals of
    the same populations."""
    from oracle import scheme
    from paper_0908_3749_gb300 import lbm
    w = W.random_state(150, 45, seed=21, smooth=False,
                       bc=(("extrap", None), ("eq", (1.1, 0.2, 0.0, 0.9)), ("reflect", None),
                           ("outflow", None)))
    cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, "df64", 5)
    results = []
    for blocks in (0, 8, 25, 59):
        ctx = lbm.lbm_create(cfg)
        try:
            lbm.lbm_set_init(ctx, *[np.ascontiguousarray(a) for a in w.fields()])
            lbm.lbm_set_step_blocks(ctx, blocks)
            lbm.lbm_step(ctx, 30)
            raw = np.empty((16, w.ny, w.nx, 2), dtype=np.float32)
            lbm.lbm_get_populations(ctx, raw)
            results.append(raw)
            if blocks == 0:
                tot = np.array(lbm.lbm_audit(ctx))
                f = read_populations(lbm, ctx, w, "df64")
                ref = scheme.conserved_totals(f, w.dx, w.dy)
                np.testing.assert_allclose(tot, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
                # checkpoint: 30 more steps from a restored copy equal 30 more in place
                lbm.lbm_step(ctx, 30)
                a = np.empty_like(raw)
                lbm.lbm_get_populations(ctx, a)
                lbm.lbm_set_populations(ctx, raw, 30)
                lbm.lbm_step(ctx, 30)
                b = np.empty_like(raw)
                lbm.lbm_get_populations(ctx, b)
                assert np.array_equal(a, b)
                assert lbm.lbm_step_count(ctx) == 60
        finally:
            lbm.lbm_destroy(ctx)
    for r in results[1:]:
        assert np.array_equal(r, results[0])


def test_bubble_full_size_one_step_in_bench_launch():
    """The 2048 x 1024 shock bubble, one step in the autotuned launch the
    benchmark uses, every node against the oracle."""
    from oracle import scheme
    from paper_0908_3749_gb300 import lbm
    w = W.shock_bubble()
    cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, "df64", 0)
    ctx = lbm.lbm_create(cfg)
    try:
        lbm.lbm_set_init(ctx, *[np.ascontiguousarray(a) for a in w.fields()])
        lbm.lbm_autotune(ctx, 5)
        lbm.lbm_step(ctx, 1)
        f = read_populations(lbm, ctx, w, "df64")
    finally:
        lbm.lbm_destroy(ctx)
    f0 = scheme.init_populations(*w.fields())
    fref = scheme.step(f0, w.cfg())
    err = pop_error(f, fref)
    bar = df64_tol(1, cancellation(f0))
    print("\nbubble 2048x1024 df64: one-step population error %.2e (bar %.1e)" % (err, bar))
    assert err <= bar


def test_error_growth_curve():
    """Per-field error of the double-word step against the oracle at levels
    1, 10, 100, 1000 (600 x 200 reflection) and to 10 000 (stable Sod)."""
    from test_gpu_error_growth import _curve
    for w, levels in ((W.sod_config1("stable", ny=4), [1, 10, 100, 1000, 10000]),
                      (W.regular_reflection(), [1, 10, 100, 1000])):
        kappa = _kappa(w)
        for level, err in _curve(w, levels, "df64"):
            assert max(err.values()) <= df64_tol(level, kappa), (w.name, level, err, kappa)
