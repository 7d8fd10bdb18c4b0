"""Shared helpers of the tests: run a workload on the GPU through the C ABI and
on the oracle, and compare fields the way the parity bar defines it.

Relative L-infinity per field: max |a - b| / max |b| for rho; the two
velocity components share the maximum speed of the reference as denominator
(a pointwise relative error is meaningless where u = 0); T is recovered as
e/rho - |u|^2/2, a difference of two terms, so its error is taken relative to
the larger of them, max(e/rho) = max(T + |u|^2/2) of the reference;
populations use the largest reference population.

FP64 tolerance: 1e-12 for runs of up to 100 steps, 1e-14 per step beyond:
the oracle's own FP64 rounding, measured against an extended-precision run of
the same algorithm, grows about linearly with the step count at roughly this
rate (tests/test_oracle_rounding.py), so no FP64 evaluation in a different
operation order can stay within a fixed 1e-12 over thousands of steps.
"""
import numpy as np

import workloads as W


def gpu_run(w, nsteps, precision="fp64", audit_every=0, chunks=None, stream=None):
    """Runs ``nsteps`` steps of workload ``w`` through the C ABI. Returns
    (fields dict, populations (16, ny, nx) float64, status tuple, ctx-free)."""
    from paper_0908_3749_gb300 import lbm
    cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, precision, audit_every)
    ctx = lbm.lbm_create(cfg, stream)
    try:
        lbm.lbm_set_init(ctx, *[np.ascontiguousarray(a, dtype=np.float64) for a in w.fields()])
        for n in (chunks or [nsteps]):
            lbm.lbm_step(ctx, n)
        out = {k: np.empty((w.ny, w.nx)) for k in ("rho", "u", "v", "T")}
        lbm.lbm_moments(ctx, out["rho"], out["u"], out["v"], out["T"])
        f = read_populations(lbm, ctx, w, precision)
        status = lbm.lbm_status(ctx)
    finally:
        lbm.lbm_destroy(ctx)
    return out, f, status


def read_populations(lbm, ctx, w, precision):
    """The context's populations as float64 (16, ny, nx); a double-word
    checkpoint (precision "df64") holds a float pair (h, l) per population."""
    if precision == "df64":
        f = np.empty((16, w.ny, w.nx, 2), dtype=np.float32)
        lbm.lbm_get_populations(ctx, f)
        return f[..., 0].astype(np.float64) + f[..., 1].astype(np.float64)
    es = lbm.lbm_element_size(ctx)
    f = np.empty((16, w.ny, w.nx), dtype=np.float64 if es == 8 else np.float32)
    lbm.lbm_get_populations(ctx, f)
    return f.astype(np.float64)


def oracle_run(w, nsteps):
    from oracle import scheme
    f = scheme.init_populations(*w.fields())
    f, _ = scheme.run(f, w.cfg(), nsteps)
    rho, u, v, T = scheme.macroscopic(f)
    return {"rho": rho, "u": u, "v": v, "T": T}, f


def field_errors(got, ref):
    speed2 = ref["u"] ** 2 + ref["v"] ** 2
    speed = np.sqrt(speed2).max()
    speed = speed if speed > 0 else 1.0
    escale = np.abs(ref["T"] + 0.5 * speed2).max()
    return {
        "rho": float(np.abs(got["rho"] - ref["rho"]).max() / np.abs(ref["rho"]).max()),
        "u": float(np.abs(got["u"] - ref["u"]).max() / speed),
        "v": float(np.abs(got["v"] - ref["v"]).max() / speed),
        "T": float(np.abs(got["T"] - ref["T"]).max() / escale),
    }


def fp64_tol(nsteps):
    return max(1e-12, 1e-14 * nsteps)


# Unit roundoff of double-word arithmetic over that of FP64: 2^-48 / 2^-53.
DW_OVER_FP64 = 32.0


def df64_tol(nsteps, kappa=1.0):
    """Bar of the double-word step (LBM_DF64) against the FP64 oracle, the
    larger of two terms:
      32 x fp64_tol(n): the FP64 bar scaled by the ratio of the unit
        roundoffs, 2^-48 / 2^-53 (each double-word operation rounds at about
        2^-48 of its operands where FP64 rounds at 2^-53);
      16 kappa 2^-48 n: the storage of the 16 populations, each rounded to
        the double-word format (48-bit significand) at every step at up to
        2^-48 of its size, kappa rho at most. Where the state is nearly
        steady and the relaxation slow, that rounding repeats from step to
        step and adds up linearly, in the conserved totals too (measured: a
        uniform Mach-2.9 flow with the MRT rates of Sec. V.B.a drifts by
        about 1e-12 per step, kappa = 103, while FP64 storage, 32 times
        finer, drifts about a thousand times less); kappa = max over nodes of
        sum_i |f_i| / rho (harness.cancellation)."""
    return max(DW_OVER_FP64 * fp64_tol(nsteps), 16.0 * kappa * 2.0 ** -48 * nsteps)


def cancellation(f):
    """kappa = max over nodes of sum_i |f_i| / rho: how much the moment sums
    cancel. States far outside the lattice speeds (flow speed or sound speed
    several times the largest |v_i| = 6) have large equilibrium populations
    of both signs, and a rounding difference between two evaluation orders
    of the same FP64 scheme grows with kappa (measured: ~1e-14 kappa per
    field over 150 steps)."""
    return float((np.abs(f).sum(axis=0) / np.abs(f.sum(axis=0))).max())


def fp64_tol_conditioned(nsteps, kappa):
    """fp64_tol, held for kappa up to ~100 (the parity states and the shock
    reflection), scaled by kappa / 50 beyond."""
    return fp64_tol(nsteps) * max(1.0, kappa / 50.0)


def l1_errors(got, ref):
    """Sec. V.A's E = sum |num - exa| / sum |exa| per field."""
    return {k: float(np.abs(got[k] - ref[k]).sum() / max(np.abs(ref[k]).sum(), 1e-300))
            for k in ("rho", "u", "v", "T")}


def pop_error(f, fref):
    return float(np.abs(f - fref).max() / np.abs(fref).max())


__all__ = ["gpu_run", "oracle_run", "field_errors", "pop_error", "fp64_tol", "l1_errors", "W",
           "cancellation", "fp64_tol_conditioned", "df64_tol", "read_populations"]
