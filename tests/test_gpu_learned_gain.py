"""What the trained proposal network gains over the method without it.

The network is trained on the GPU by the library's own forward, backward and
Adam kernels, on patterns the method generates (the 128 x 128 map generator:
BCC master, random orientations over SO(3), PC jitter, Poisson noise at
50-500 counts), 1,562 steps of 256 (two passes over 200,000 orientations,
fresh noise per pass).  On 1,000 held-out patterns the learned path
(8 proposals scored by the correlation peak, refinement, full-search
fallback below a threshold calibrated on 1,000 other patterns) must:
  * evaluate at most 5 % of the (pattern, template) correlations of the full
    4,065-template search (8 per pattern plus the library for each fallback);
  * fall back on at most 5 % of the patterns (an untrained network, the
    method without a useful proposal, falls back on more than half);
  * hold the mean misorientation at or below 0.5 deg, at least 98 % of the
    patterns within 1 deg, and the median within 0.05 deg of the full search
    + refinement on the same patterns (the threshold admits up to 0.5 % of
    wrong matches, which move the mean, not the median)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def px():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_11313_gb300 as px
    px.load()
    return px


def _noisy(clean, pcs, peak, gen):
    """Poisson(peak (0.6 background hump at the PC + 0.4 clean scaled to [0, 1]))."""
    P, H, W = clean.shape
    lo, hi = clean.amin(dim=(1, 2), keepdim=True), clean.amax(dim=(1, 2), keepdim=True)
    ih = (clean - lo) / (hi - lo).clamp_min(1e-30)
    ry = torch.arange(H, device=clean.device, dtype=torch.float32) + 0.5
    rx = torch.arange(W, device=clean.device, dtype=torch.float32) + 0.5
    cy, cx = (pcs[:, 1] * H).float().view(P, 1, 1), (pcs[:, 0] * W).float().view(P, 1, 1)
    hump = torch.exp(-((ry.view(1, H, 1) - cy) ** 2 + (rx.view(1, 1, W) - cx) ** 2) / (2 * (0.35 * W) ** 2))
    return torch.poisson(peak.float().view(P, 1, 1) * (0.6 * hump + 0.4 * ih), generator=gen)


def _generate(px, ctx, master, geom, q, pcs, peak, gen):
    return _noisy(px.xcf_project(ctx, master, q.contiguous(), geom, pcs=pcs.contiguous()), pcs, peak, gen)


def _tau(px, ctx, net, lib, pats, pcs, truth):
    """Lowest refined peak above which at most 0.5 % of the calibration
    patterns are off by more than 1 deg (the learned path without fallback)."""
    q, pk, _, _ = px.xcf_index_learned(ctx, net, lib, pats, pcs=pcs, tau=float("-inf"))
    mis = px.xcf_disorientation(ctx, q, truth)
    order = torch.argsort(pk, descending=True)
    wrong = (mis[order] > 1.0).double().cumsum(0) / torch.arange(1, len(order) + 1, device=pk.device)
    ok = torch.nonzero(wrong <= 0.005).flatten()
    return float(pk[order][ok.max()]) if ok.numel() else float("inf")


def test_trained_network_gains_over_the_full_search(px):
    dev = torch.device("cuda")
    wl = synth.config_learned_128(seed=31, n_train=200000, n_test=1000, n_cal=1000)
    n, k = wl["n"], wl["k"]
    geom = px.geometry(n, n, wl["pc"])
    ctx = px.Context(max_iter=wl["max_iter"], tol_deg=1e-3)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    master, libq = d(wl["master"]), d(wl["lib_q"])
    gen = torch.Generator(device=dev)
    gen.manual_seed(32)
    lib = px.xcf_build_library(ctx, master, libq, geom)
    T = lib.T
    tq, tpc, tpk = d(wl["test_q"]), d(wl["test_pcs"]), d(wl["test_peak"])
    cq, cpc, cpk = d(wl["cal_q"]), d(wl["cal_pcs"]), d(wl["cal_peak"])
    pats = _generate(px, ctx, master, geom, tq, tpc, tpk, gen)
    cpats = _generate(px, ctx, master, geom, cq, cpc, cpk, gen)
    P = pats.shape[0]

    # the method without a useful proposal: the untrained network
    net0 = px.xcf_net_create(ctx, k, d(synth.cnn_init_params(k, 33)))
    net0.set_bf16(True)
    tau0 = _tau(px, ctx, net0, lib, cpats, cpc, cq)
    _, _, _, fb0 = px.xcf_index_learned(ctx, net0, lib, pats, pcs=tpc, tau=tau0)
    net0.close()

    # training on the GPU: forward, backward and Adam kernels of the library
    net = px.xcf_net_create(ctx, k, d(synth.cnn_init_params(k, 33)))
    trq, trpc, trpk = d(wl["train_q"]), d(wl["train_pcs"]), d(wl["train_peak"])
    B, per_epoch = 256, len(wl["train_q"]) // 256
    steps = 2 * per_epoch
    for i in range(steps):
        sl = slice((i % per_epoch) * B, (i % per_epoch + 1) * B)
        imgs = _generate(px, ctx, master, geom, trq[sl], trpc[sl], trpk[sl], gen)
        px.xcf_net_loss_grad(ctx, net, imgs, trq[sl].contiguous(), geom)
        px.xcf_net_adam(ctx, net, lr=float(2e-3 * 0.5 * (1.0 + np.cos(np.pi * i / steps))))
    net.set_bf16(True)
    tau = _tau(px, ctx, net, lib, cpats, cpc, cq)
    q, pk, it, fb = px.xcf_index_learned(ctx, net, lib, pats, pcs=tpc, tau=tau)
    full = px.xcf_index_refine(ctx, lib, pats, pcs=tpc)
    torch.cuda.synchronize()

    mis = px.xcf_disorientation(ctx, q, tq).cpu().numpy()
    mis_full = px.xcf_disorientation(ctx, full["quats"], tq).cpu().numpy()
    n_fb, n_fb0 = int(fb.sum()), int(fb0.sum())
    pairs_learned = P * k + n_fb * T
    pairs_full = P * T
    print(f"fallbacks {n_fb}/{P} (untrained {n_fb0}/{P}), pairs {pairs_learned} vs {pairs_full} "
          f"({pairs_learned / pairs_full:.4f}), mean {mis.mean():.3f} vs {mis_full.mean():.3f} deg, tau {tau:.3f}")
    assert n_fb0 > 0.5 * P
    assert n_fb <= 0.05 * P
    assert pairs_learned <= 0.05 * pairs_full
    assert mis.mean() <= 0.5 and np.median(mis) <= np.median(mis_full) + 0.05
    assert (mis < 1.0).mean() >= 0.98
    lib.close()
    net.close()
    ctx.close()
