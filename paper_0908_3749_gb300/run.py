"""Command-line runner: one of the synthetic workloads stepped through the C ABI.

    python -m paper_0908_3749_gb300.run --workload reflection --precision fp32 --steps 100
    python -m paper_0908_3749_gb300.run --workload tubes --steps 20 --autotune 5
    python -m paper_0908_3749_gb300.run --workload vn --nx 4096 --steps 1

Prints one JSON line with the step count, the watchdog status, the
conservation totals and the ranges of rho, u, v, T. Nothing is timed; it is
the plain driver for quick checks and for profiler runs of a single kernel
(every launch of the step is one time step, in order). Run from the
repository root (the workload generators live in ``workloads.py`` there).
"""
import argparse
import json

import numpy as np

from . import lbm

WORKLOADS = ("reflection", "bubble", "sod", "couette", "random", "mach", "heavy_bubble",
             "tubes", "vn")


def make_workload(name, nx=None, ny=None):
    import workloads as W
    if name == "reflection":
        return W.regular_reflection(nx=nx or 600, ny=ny or 200)
    if name == "bubble":
        return W.shock_bubble(nx=nx or 2048, ny=ny or 1024)
    if name == "sod":
        return W.sod_config1()
    if name == "couette":
        return W.couette()
    if name == "mach":
        return W.mach_reflection()
    if name == "heavy_bubble":
        return W.heavy_bubble(nx=nx or 2048, ny=ny or 1024)
    return W.random_state(nx or 256, ny or 128, seed=0)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", choices=WORKLOADS, default="reflection")
    ap.add_argument("--nx", type=int, default=None)
    ap.add_argument("--ny", type=int, default=None)
    ap.add_argument("--precision", choices=("fp64", "df64", "fp32", "fp32_dwmom", "tc_tf32x3"), default="fp32")
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--audit-every", type=int, default=0)
    ap.add_argument("--blocks", type=int, default=0,
                    help="step launch blocks (0: one per tile); see lbm_set_step_blocks")
    ap.add_argument("--fused", type=int, default=1, choices=(1, 2),
                    help="time steps per FP32 launch (lbm_set_fused_steps)")
    ap.add_argument("--autotune", type=int, default=0,
                    help="if > 0, choose the launch shape with lbm_autotune(launches)")
    args = ap.parse_args(argv)
    if args.workload == "tubes":
        return run_tubes(args)
    if args.workload == "vn":
        return run_vn(args)

    w = make_workload(args.workload, args.nx, args.ny)
    cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, args.precision,
                          args.audit_every)
    ctx = lbm.lbm_create(cfg)
    try:
        lbm.lbm_set_init(ctx, *[np.ascontiguousarray(a) for a in w.fields()])
        if args.blocks and args.precision != "tc_tf32x3":
            lbm.lbm_set_step_blocks(ctx, args.blocks)
        if args.autotune > 0:
            lbm.lbm_autotune(ctx, args.autotune)
        if args.fused == 2:
            lbm.lbm_set_fused_steps(ctx, 2)
        lbm.lbm_step(ctx, args.steps)
        rc, bad, neg = lbm.lbm_status(ctx)
        m = [np.empty((w.ny, w.nx)) for _ in range(4)]
        lbm.lbm_moments(ctx, *m)
        out = {"workload": args.workload, "nx": w.nx, "ny": w.ny, "precision": args.precision,
               "steps": lbm.lbm_step_count(ctx), "step_blocks": lbm.lbm_step_blocks(ctx),
               "status": rc, "first_bad_step": bad, "first_negT_step": neg,
               "totals": lbm.lbm_audit(ctx),
               "ranges": {k: [float(np.nanmin(a)), float(np.nanmax(a))]
                          for k, a in zip(("rho", "u", "v", "T"), m)}}
    finally:
        lbm.lbm_destroy(ctx)
    print(json.dumps(out))
    return 0 if rc == lbm.LBM_OK else 1


def run_tubes(args):
    """The seeded tube batch (``--nx`` tubes, default 4096) in one persistent
    launch per ``lbm_batch_step`` call of ``--steps`` steps."""
    import workloads as W
    B = W.tube_batch(ntubes=args.nx or 4096)
    nt = len(B["nx"])
    b = lbm.lbm_batch_create(B["nx"], B["dx"], B["dt"], B["s"], B["left"], B["right"])
    try:
        lbm.lbm_batch_set_init(b, *W.tube_fields(B))
        if args.autotune > 0:
            lbm.lbm_batch_autotune(b, args.autotune, None)
        lbm.lbm_batch_step(b, args.steps)
        rc, bad, nbad, to = lbm.lbm_batch_status(b, nt)
        out = {"workload": "tubes", "tubes": nt, "nodes": lbm.lbm_batch_total_nodes(b),
               "steps": lbm.lbm_batch_step_count(b), "tiling": list(lbm.lbm_batch_get_tiling(b)),
               "status": rc, "unstable_tubes": nbad, "timeout": to}
    finally:
        lbm.lbm_batch_destroy(b)
    print(json.dumps(out))
    return 0 if rc == lbm.LBM_OK and to == 0 else 1


def run_vn(args):
    """Stability sweep of the Sec. IV example (workloads.vn_example): MRT and
    SRT rates, ``--nx`` wave numbers k dx in [0, pi] along x (default 4096),
    ``--steps`` repetitions of the sweep (one eigenvalue launch each)."""
    import workloads as W
    ex = W.vn_example(nk=args.nx or 4096)
    cases = lbm.vn_cases(ex["states"], ex["rates"])
    for _ in range(max(1, args.steps)):
        radius, _, nf = lbm.lbm_vn_spectrum(cases, ex["k"], ex["dx"], ex["dy"], ex["dt"],
                                            want_omega=False)
    out = {"workload": "vn", "cases": ex["names"], "nk": int(ex["k"].shape[0]),
           "max_radius": [float(r.max()) for r in radius], "nonconverged": nf}
    print(json.dumps(out))
    return 0 if nf == 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
