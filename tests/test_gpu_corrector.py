"""GPU tests of the learned coarse-grid corrector (include/lbm_cnn.h).

* Loss and every parameter gradient of the GPU network (an FP32 first layer
  on the FP32 features, then BF16 tensor-core convolutions and weight
  gradients with FP32 accumulation) against the FP64 CPU reference (oracle/cnn.py) run with the
  same BF16 rounding of the later layers' parameters, the stored activations
  and the stored output gradients:
  what is left is FP32-vs-FP64 accumulation order, so the bar is a relative
  L2 error of 2e-3 per gradient. Against the unrounded FP64 network the loss
  agrees within 1e-2 (BF16 keeps 8 significant bits; the rounded output
  gradients, propagated back through five layers, move the first layer's
  weight gradient by several percent, which the rounded reference reproduces).
* Restriction against the CPU reference.
* Training lowers the loss; on held-out quadrant problems the corrected
  coarse fields are closer to the restricted fine run than the plain coarse
  fields (what the network gains over the method without it).
"""
import numpy as np
import pytest

import workloads as W
from oracle import cnn

pytestmark = pytest.mark.gpu


_bf16 = cnn.bf16


def _unpack(p):
    from paper_0908_3749_gb300 import lbm
    ch = lbm.CNN_CHANNELS
    out, o = [], 0
    for l in range(len(ch) - 1):
        nw = 9 * ch[l] * ch[l + 1]
        out.append((p[o:o + nw].reshape(3, 3, ch[l], ch[l + 1]), p[o + nw:o + nw + ch[l + 1]]))
        o += nw + ch[l + 1]
    return out


def _fields(rng, H, W):
    rho = np.exp(rng.uniform(-1, 1, (H, W)))
    T = np.exp(rng.uniform(-1, 1, (H, W)))
    u, v = rng.uniform(-0.8, 0.8, (2, H, W))
    return np.stack([rho, u, v, T])


@pytest.mark.parametrize("loss_kind,H,W", [("mse", 7, 5), ("mse", 13, 11), ("l1", 13, 11),
                                            ("mse", 257, 203)])
def test_gradients_match_cpu_reference(loss_kind, H, W):
    """7 x 5: one partial 64-pixel chunk of the tensor-core weight gradients;
    13 x 11: three chunks, the last one ragged; 257 x 203: 816 chunks, so
    that some CTAs of the persistent grid (4 per SM) accumulate two chunks in
    tensor memory."""
    import torch
    from paper_0908_3749_gb300 import lbm, corrector
    rng = np.random.default_rng(0)
    params = corrector.init_params(3)
    last = _unpack(params)[-1][0]
    last[...] = rng.standard_normal(last.shape) * 0.05      # non-zero last layer
    coarse, target = _fields(rng, H, W), _fields(rng, H, W)
    scale = (0.5, 2.0, 1.0, 0.25)
    net = lbm.lbm_cnn_create(H, W)
    try:
        lbm.lbm_cnn_set_params(net, params)
        lbm.lbm_cnn_set_output_scale(net, scale)
        lbm.lbm_cnn_set_loss(net, loss_kind)
        loss, g = lbm.lbm_cnn_loss_grad(net, torch.tensor(coarse, device="cuda"),
                                        torch.tensor(target, device="cuda"))
        rms = lbm.lbm_cnn_residual_rms(net, torch.tensor(coarse, device="cuda"),
                                       torch.tensor(target, device="cuda"))
    finally:
        lbm.lbm_cnn_destroy(net)
    # first layer: FP32 features and FP32 weights; later layers: BF16 weights
    ref_params = [(w.astype(np.float64) if l == 0 else _bf16(w), b.astype(np.float64))
                  for l, (w, b) in enumerate(_unpack(params))]
    xf = cnn.features(*coarse).astype(np.float32).astype(np.float64)
    x = xf
    t = cnn.features(*target).astype(np.float32).astype(np.float64)
    exact_loss, _ = cnn.loss_and_grads(x, t, ref_params, x_res=xf, scale=scale, loss=loss_kind)
    rloss, rgrads = cnn.loss_and_grads(x, t, ref_params, x_res=xf, store=cnn.bf16, scale=scale,
                                       loss=loss_kind)
    np.testing.assert_allclose(rms, np.sqrt(((t - xf) ** 2).mean(axis=(0, 1))), rtol=1e-12)
    assert abs(loss - exact_loss) <= 1e-2 * exact_loss, (loss, exact_loss)
    assert abs(loss - rloss) <= 1e-5 * rloss, (loss, rloss)
    errs = []
    for l, (gw, gb) in enumerate(_unpack(g.astype(np.float64))):
        for got, ref in ((gw, rgrads[l][0]), (gb, rgrads[l][1])):
            errs.append(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30))
    print("gradient relative L2 errors vs the rounded reference", errs)
    assert max(errs) < 2e-3, errs


def test_restriction_matches_cpu_reference():
    import torch
    from paper_0908_3749_gb300 import lbm
    rng = np.random.default_rng(1)
    f = _fields(rng, 16, 12)
    out = torch.empty((4, 4, 3), dtype=torch.float64, device="cuda")
    lbm.lbm_restrict(torch.tensor(f, device="cuda"), 4, out)
    torch.cuda.synchronize()
    ref = cnn.restrict(*f, 4)
    for k in range(4):
        np.testing.assert_allclose(out[k].cpu().numpy(), ref[k], rtol=1e-13, atol=1e-14)


def test_training_gains_over_plain_coarse_on_held_out_problems():
    from paper_0908_3749_gb300 import corrector, lbm
    n, ratio, t_end = 32, 4, 0.02
    # Problems on which the scheme itself goes unstable (the watchdog trips in
    # the fine or the coarse run) are rejected and counted.
    train_pairs, skipped_tr, _ = corrector.make_pairs(W.corrector_quadrant, range(1, 65), n, ratio, t_end)
    test_pairs, skipped_te, _ = corrector.make_pairs(W.corrector_quadrant, range(10001, 10017), n, ratio, t_end)
    print("rejected", skipped_tr, "of 64 training and", skipped_te, "of 16 held-out problems")
    assert len(train_pairs) >= 24 and len(test_pairs) >= 6, (skipped_tr, skipped_te)
    net, losses = corrector.train(train_pairs, epochs=60, lr=2e-3, seed=0)
    try:
        assert losses[-1] < 0.5 * losses[0], losses[::5]
        res = corrector.evaluate(net, test_pairs)
    finally:
        lbm.lbm_cnn_destroy(net)
    print("plain", res["plain"], "corrected", res["corrected"], "fallbacks", res["fallbacks"])
    assert np.mean(res["corrected"]) < np.mean(res["plain"]), res


def test_training_gains_at_full_scale():
    """The learned part at its configuration's scale: 512 x 512 coarse runs
    against 4x finer (2048 x 2048) runs restricted by 4, t_end 0.02; trained
    on the GPU (own forward / backward / Adam kernels, MSE loss, 150 epochs)
    on seeded quadrant problems 1 .. 64 and evaluated on held-out problems
    10001 .. 10008. The corrected coarse fields must be closer to the fine
    run than the plain coarse fields on every field, in L1 and in L2, with a
    mean L1 gain of at least 1.3x (measured 1.8-2.8x per field)."""
    from paper_0908_3749_gb300 import corrector, lbm
    n, ratio, t_end = 512, 4, 0.02
    train_pairs, skipped_tr, _ = corrector.make_pairs(W.corrector_quadrant, range(1, 65), n, ratio,
                                                      t_end)
    test_pairs, skipped_te, tm = corrector.make_pairs(W.corrector_quadrant, range(10001, 10009), n,
                                                      ratio, t_end)
    assert len(train_pairs) >= 48 and len(test_pairs) >= 6, (skipped_tr, skipped_te)
    net, losses = corrector.train(train_pairs, epochs=150, lr=2e-3, seed=0, loss="mse")
    try:
        res = corrector.evaluate(net, test_pairs)
    finally:
        lbm.lbm_cnn_destroy(net)
    gain = np.array(res["plain"]) / np.array(res["corrected"])
    print("\n512/2048: rejected %d + %d; L1 plain %s corrected %s (gain %s); L2 plain %s corrected %s;"
          " fine %.3f s, coarse %.3f s, inference %.4f s per problem; fallbacks %d"
          % (skipped_tr, skipped_te, np.round(res["plain"], 5), np.round(res["corrected"], 5),
             np.round(gain, 2), np.round(res["plain_l2"], 5), np.round(res["corrected_l2"], 5),
             tm["fine_s_per_problem"], tm["coarse_s_per_problem"], res["inference_s_per_problem"],
             res["fallbacks"]))
    assert all(c < p for c, p in zip(res["corrected"], res["plain"])), res
    assert all(c < p for c, p in zip(res["corrected_l2"], res["plain_l2"])), res
    assert gain.mean() >= 1.3, gain
