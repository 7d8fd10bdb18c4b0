"""Learned coarse-grid corrector: data generation, training and evaluation.

Orchestration only: every field, restriction, forward and backward pass and
optimiser update runs in the CUDA kernels behind ``include/lbm.h`` and
``include/lbm_cnn.h``; this module moves device pointers between them.

Data: for each seeded problem (a callable ``make(seed, n, dt)`` returning a
workload with ``nx, ny, dx, dy, dt, s, bc`` and initial fields), a fine run
on an (r n) x (r n) grid with dt / r and a coarse run on n x n with dt, both
to the same end time, through the FP32 step. The fine result restricted by r
(block means of rho, j, e) is the target of the coarse result. Problems whose
fine or coarse run trips the watchdog are skipped and counted.
"""
import math
import time

import numpy as np

from . import lbm


def run_fields(w, nsteps, precision="fp32", stream=None):
    """Runs workload ``w`` for ``nsteps`` and returns (fields, ok): fields a
    CUDA float64 tensor [4][ny][nx] (rho, u, v, T); ok is False when the
    watchdog tripped or the final state is not finite with rho > 0 and
    T > 0 everywhere (the network takes log rho and log T)."""
    import torch
    cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, precision, 0)
    ctx = lbm.lbm_create(cfg, stream)
    try:
        dev = [torch.as_tensor(np.ascontiguousarray(a), device="cuda") for a in
               (w.rho, w.u, w.v, w.T)]
        lbm.lbm_set_init(ctx, *dev)
        lbm.lbm_step(ctx, nsteps)
        out = torch.empty((4, w.ny, w.nx), dtype=torch.float64, device="cuda")
        lbm.lbm_moments(ctx, out[0], out[1], out[2], out[3])
        rc, bad, _ = lbm.lbm_status(ctx)
    finally:
        lbm.lbm_destroy(ctx)
    ok = (rc == lbm.LBM_OK and bad < 0 and bool(torch.isfinite(out).all())
          and bool((out[0] > 0).all()) and bool((out[3] > 0).all()))
    return out, ok


def make_pairs(make, seeds, n, ratio, t_end, dt=1e-5, stream=None):
    """(pairs, skipped, timing): pairs of (coarse, target) CUDA tensors."""
    import torch
    pairs, skipped = [], 0
    t_fine = t_coarse = 0.0
    nc = int(round(t_end / dt))
    nf = nc * ratio
    for seed in seeds:
        wf = make(seed, n * ratio, dt / ratio)
        wc = make(seed, n, dt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fine, ok_f = run_fields(wf, nf, stream=stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        coarse, ok_c = run_fields(wc, nc, stream=stream)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        t_fine += t1 - t0
        t_coarse += t2 - t1
        if not (ok_f and ok_c):
            skipped += 1
            continue
        target = torch.empty((4, n, n), dtype=torch.float64, device="cuda")
        lbm.lbm_restrict(fine, ratio, target)
        if not (bool((target[3] > 0).all()) and bool(torch.isfinite(target).all())):
            skipped += 1
            continue
        pairs.append((coarse, target))
    torch.cuda.synchronize()
    used = max(len(seeds), 1)
    return pairs, skipped, {"fine_s_per_problem": t_fine / used,
                            "coarse_s_per_problem": t_coarse / used}


def init_params(seed):
    """He-normal weights (biases zero) from a seeded generator; the last
    layer starts at zero so the untrained corrector is the identity."""
    rng = np.random.default_rng(seed)
    parts = []
    ch = lbm.CNN_CHANNELS
    for l in range(len(ch) - 1):
        cin, cout = ch[l], ch[l + 1]
        if l == len(ch) - 2:
            w = np.zeros((3, 3, cin, cout))
        else:
            w = rng.standard_normal((3, 3, cin, cout)) * math.sqrt(2.0 / (9 * cin))
        parts += [w.reshape(-1), np.zeros(cout)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == lbm.CNN_NPARAMS
    return p


def train(pairs, epochs=20, lr=1e-3, seed=0, stream=None, log_every=0, loss="l1"):
    """Trains a fresh network on ``pairs``; returns (handle, losses). The
    loss is "l1" (mean absolute feature error, the measure the evaluation
    reports) or "mse"; the network's output scale is the RMS correction
    (restricted fine minus coarse) of each feature over the pairs. The
    caller owns the handle (lbm.lbm_cnn_destroy)."""
    H, W = pairs[0][0].shape[1:]
    net = lbm.lbm_cnn_create(H, W, stream)
    lbm.lbm_cnn_set_params(net, init_params(seed))
    lbm.lbm_cnn_set_adam(net, lr)
    lbm.lbm_cnn_set_loss(net, loss)
    # Corrections in units of the training data's RMS correction per feature.
    ms = np.zeros(4)
    for c, t in pairs:
        ms += np.square(lbm.lbm_cnn_residual_rms(net, c, t))
    scale = np.sqrt(ms / len(pairs))
    lbm.lbm_cnn_set_output_scale(net, np.where(scale > 0, scale, 1.0))
    rng = np.random.default_rng(seed + 1)
    losses = []
    for ep in range(epochs):
        tot = 0.0
        for k in rng.permutation(len(pairs)):
            tot += lbm.lbm_cnn_train_step(net, pairs[k][0], pairs[k][1])
        losses.append(tot / len(pairs))
        if not math.isfinite(losses[-1]):
            raise FloatingPointError("training loss is not finite at epoch %d" % ep)
        if log_every and ep % log_every == 0:
            print("epoch %d loss %.4g" % (ep, losses[-1]))
    return net, losses


def rel_l1(a, b):
    """Sec. V.A's E per field: sum |a - b| / sum |b| over the grid."""
    return [float((a[k] - b[k]).abs().sum() / b[k].abs().sum()) for k in range(4)]


def rel_l2(a, b):
    """Per field: sqrt(sum (a - b)^2 / sum b^2) over the grid."""
    return [float(((a[k] - b[k]) ** 2).sum().sqrt() / (b[k] ** 2).sum().sqrt()) for k in range(4)]


def evaluate(net, pairs, mass_tol=1e-2):
    """Mean relative L1 error per field (rho, u, v, T) of the plain coarse
    fields and of the corrected ones against the restricted fine fields, the
    number of fallbacks, and the inference time per problem."""
    import torch
    plain, corr, plain2, corr2, fallbacks, t_inf = [], [], [], [], 0, 0.0
    for coarse, target in pairs:
        out = torch.empty_like(coarse)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fb = lbm.lbm_cnn_correct(net, coarse, out, mass_tol)
        torch.cuda.synchronize()
        t_inf += time.perf_counter() - t0
        fallbacks += int(fb)
        plain.append(rel_l1(coarse, target))
        corr.append(rel_l1(out, target))
        plain2.append(rel_l2(coarse, target))
        corr2.append(rel_l2(out, target))
    n = max(len(pairs), 1)
    return {"plain": np.mean(plain, axis=0).tolist(), "corrected": np.mean(corr, axis=0).tolist(),
            "plain_l2": np.mean(plain2, axis=0).tolist(),
            "corrected_l2": np.mean(corr2, axis=0).tolist(),
            "fallbacks": fallbacks, "inference_s_per_problem": t_inf / n}


def main(argv=None):
    """Full-size evaluation: trains on seeded quadrant problems and reports,
    on held-out seeds, the error of the plain and of the corrected coarse run
    against the restricted fine run, and the wall time of the fine run
    against the coarse run plus inference. One JSON line.

        python -m paper_0908_3749_gb300.corrector --n 512 --ratio 4 --t-end 0.02
    """
    import argparse
    import json

    import workloads as W
    ap = argparse.ArgumentParser(description="learned coarse-grid corrector: train and evaluate")
    ap.add_argument("--n", type=int, default=512, help="coarse grid n x n")
    ap.add_argument("--ratio", type=int, default=4, help="fine / coarse resolution")
    ap.add_argument("--t-end", type=float, default=0.02)
    ap.add_argument("--dt", type=float, default=1e-5, help="coarse time step (fine: dt / ratio)")
    ap.add_argument("--train", type=int, default=64, help="training seeds 1 .. train")
    ap.add_argument("--test", type=int, default=8, help="held-out seeds 10001 .. 10000 + test")
    ap.add_argument("--epochs", type=int, default=150)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--loss", choices=("l1", "mse"), default="mse")
    args = ap.parse_args(argv)

    t0 = time.perf_counter()
    train_pairs, skipped_tr, tm_tr = make_pairs(W.corrector_quadrant, range(1, args.train + 1),
                                                args.n, args.ratio, args.t_end, args.dt)
    test_pairs, skipped_te, tm_te = make_pairs(W.corrector_quadrant,
                                               range(10001, 10001 + args.test),
                                               args.n, args.ratio, args.t_end, args.dt)
    t1 = time.perf_counter()
    if not train_pairs or not test_pairs:
        raise SystemExit("every problem was rejected")
    net, losses = train(train_pairs, epochs=args.epochs, lr=args.lr, seed=0, loss=args.loss)
    t2 = time.perf_counter()
    try:
        res = evaluate(net, test_pairs)
    finally:
        lbm.lbm_cnn_destroy(net)
    coarse_s = tm_te["coarse_s_per_problem"]
    fine_s = tm_te["fine_s_per_problem"]
    out = {
        "workload": "2D Riemann quadrants, coarse %dx%d, fine %dx%d, t_end %g"
                    % (args.n, args.n, args.n * args.ratio, args.n * args.ratio, args.t_end),
        "train_problems": len(train_pairs), "train_rejected": skipped_tr,
        "test_problems": len(test_pairs), "test_rejected": skipped_te,
        "rel_l1_plain": dict(zip(("rho", "u", "v", "T"), res["plain"])),
        "rel_l1_corrected": dict(zip(("rho", "u", "v", "T"), res["corrected"])),
        "rel_l2_plain": dict(zip(("rho", "u", "v", "T"), res["plain_l2"])),
        "rel_l2_corrected": dict(zip(("rho", "u", "v", "T"), res["corrected_l2"])),
        "fallbacks": res["fallbacks"],
        "fine_run_s": fine_s, "coarse_run_s": coarse_s,
        "inference_s": res["inference_s_per_problem"],
        "speedup_vs_fine": fine_s / (coarse_s + res["inference_s_per_problem"]),
        "loss": args.loss, "loss_first_last": [losses[0], losses[-1]], "epochs": args.epochs,
        "data_s": t1 - t0, "train_s": t2 - t1,
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
