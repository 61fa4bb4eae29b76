"""Proposal network on the GPU against the FP64 oracle: forward outputs,
loss, gradient, Adam step and proposals on identical seeded inputs; then the
learned indexing path (proposal scoring, refinement, fallback to the full
search) against the plain search + refinement.

Tolerances: the FP32 network against FP64 -- outputs 2e-4 of their scale,
the gradient 1e-3 in relative L2 norm per parameter block (FP32 sums over up
to 2 x 10^5 products, split-K atomics), Adam 1e-5 relative."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
K = 8


@pytest.fixture(scope="module")
def px():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_11313_gb300 as px
    px.load()
    return px


@pytest.fixture(scope="module")
def ctx(px):
    c = px.Context()
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _images(B, seed, side=128):
    rng = np.random.default_rng(seed)
    x = rng.gamma(2.0, 20.0, size=(B, side, side)).astype(np.float32)
    x += np.linspace(0, 30, side, dtype=np.float32)[None, None, :]
    return x


def _quats(B, seed):
    return synth.random_quaternions(B, seed)


def _blocks(k):
    ch = synth.CNN_CHANNELS
    out, o = [], 0
    for l in range(5):
        for n in (ch[l + 1] * ch[l] * 9, ch[l + 1]):
            out.append((o, o + n))
            o += n
    for n in (256 * 128, 256, 6 * k * 256, 6 * k):
        out.append((o, o + n))
        o += n
    return out


def test_param_count(px, orc):
    assert px.xcf_net_num_params(K) == orc.cnn_num_params(K)
    assert px.xcf_net_num_params(0) == -1


def test_forward_matches_oracle(px, ctx, orc):
    p = synth.cnn_init_params(K, 3)
    x = _images(5, 1)
    x[2] = 7.0                                   # constant: standardised to zeros
    net = px.xcf_net_create(ctx, K, dev(p))
    out = px.xcf_net_forward(ctx, net, dev(x)).cpu().numpy()
    ref = orc.cnn_forward(p, x, K)
    assert np.abs(out - ref).max() <= 2e-4 * np.abs(ref).max()
    net.close()


def test_bf16_forward_matches_oracle_bf16_form(px, ctx, orc):
    """BF16 inference: convolutions 2..5 on the tensor cores.  Against the
    oracle's BF16 form (the same operands rounded to BF16, FP64 accumulation)
    only the accumulation order differs, apart from rare operands that sit on
    a BF16 rounding boundary after an FP32 (not FP64) previous layer: 2e-3 of
    the output scale.  Against the FP32 forward: the BF16 rounding itself."""
    p = synth.cnn_init_params(K, 5)
    x = _images(37, 4)                           # ragged against the 128-row tiles
    x[3] = 2.0                                   # constant image
    net = px.xcf_net_create(ctx, K, dev(p))
    net.set_bf16(True)
    out = px.xcf_net_forward(ctx, net, dev(x)).cpu().numpy()
    ref = orc.cnn_forward_bf16(p, x, K)
    scale = np.abs(ref).max()
    assert np.abs(out - ref).max() <= 2e-3 * scale, np.abs(out - ref).max() / scale
    assert np.abs(out - orc.cnn_forward(p, x, K)).max() <= 3e-2 * scale
    # the proposals follow the same forward; FP32 again when switched off
    q = px.xcf_propose(ctx, net, dev(x[:4])).cpu().numpy()
    np.testing.assert_allclose(np.linalg.norm(q, axis=-1), 1.0, atol=1e-9)
    net.set_bf16(False)
    out32 = px.xcf_net_forward(ctx, net, dev(x)).cpu().numpy()
    assert np.abs(out32 - orc.cnn_forward(p, x, K)).max() <= 2e-4 * scale
    net.close()


def test_bf16_forward_many_tiles_sampled(px, ctx, orc):
    """The BF16 form on 1,100 patterns: two network passes (1,024 + 76), tens
    of tiles per CTA in every tensor-core convolution (so both accumulator
    buffers and every ring stage wrap many times), ragged last tiles; sampled
    rows against the oracle's BF16 form at the same 2e-3 of the output scale."""
    p = synth.cnn_init_params(K, 6)
    x = _images(1100, 7)
    net = px.xcf_net_create(ctx, K, dev(p))
    net.set_bf16(True)
    out = px.xcf_net_forward(ctx, net, dev(x)).cpu().numpy()
    idx = np.array([0, 1, 2, 127, 128, 511, 700, 1022, 1023, 1024, 1025, 1062, 1098, 1099])
    ref = orc.cnn_forward_bf16(p, x[idx], K)
    scale = np.abs(ref).max()
    assert np.abs(out[idx] - ref).max() <= 2e-3 * scale, np.abs(out[idx] - ref).max() / scale
    assert np.isfinite(out).all()
    net.close()


def test_forward_reads_the_centred_crop(px, ctx, orc):
    W, H, pc = 160, 140, (0.5, 0.5, 0.6)
    p = synth.cnn_init_params(K, 4)
    x = _images(3, 2, side=160)[:, :H, :W].copy()
    net = px.xcf_net_create(ctx, K, dev(p))
    out = px.xcf_net_forward(ctx, net, dev(x), px.geometry(W, H, pc)).cpu().numpy()
    n, ox, oy, _ = orc.crop(W, H, pc, 128)
    assert n == 128
    ref = orc.cnn_forward(p, x[:, oy:oy + n, ox:ox + n], K)
    assert np.abs(out - ref).max() <= 2e-4 * np.abs(ref).max()
    with pytest.raises(px.XcfError):
        px.xcf_net_forward(ctx, net, dev(_images(1, 3, side=100)), px.geometry(100, 100, pc))
    net.close()


def test_loss_and_gradient_match_oracle(px, ctx, orc):
    p = synth.cnn_init_params(K, 5)
    x, q = _images(6, 4), _quats(6, 5)
    net = px.xcf_net_create(ctx, K, dev(p))
    loss, grad, win = px.xcf_net_loss_grad(ctx, net, dev(x), dev(q), want_grad=True, want_winners=True)
    rloss, rgrad, rwin = orc.cnn_loss_grad(p, x, q, K)
    assert abs(float(loss) - rloss) <= 1e-5 * abs(rloss)
    assert np.array_equal(win.cpu().numpy(), rwin)
    g = grad.cpu().numpy().astype(np.float64)
    for a, b in _blocks(K):
        ref = rgrad[a:b]
        err = np.linalg.norm(g[a:b] - ref) / max(np.linalg.norm(ref), 1e-30)
        assert err < 1e-3, (a, b, err)
    net.close()


def test_adam_step_matches_oracle(px, ctx, orc):
    p = synth.cnn_init_params(K, 6)
    x, q = _images(4, 6), _quats(4, 7)
    net = px.xcf_net_create(ctx, K, dev(p))
    _, grad, _ = px.xcf_net_loss_grad(ctx, net, dev(x), dev(q), want_grad=True)
    g = grad.cpu().numpy().astype(np.float64)
    px.xcf_net_adam(ctx, net, lr=1e-3)
    p1 = net.params().cpu().numpy().astype(np.float64)
    ref, m, v = p.astype(np.float64), np.zeros(len(p)), np.zeros(len(p))
    orc.adam(ref, g, m, v, 1, lr=1e-3)
    np.testing.assert_allclose(p1, ref, rtol=1e-5, atol=1e-7)
    # second step on the same batch: state carried over
    _, grad2, _ = px.xcf_net_loss_grad(ctx, net, dev(x), dev(q), want_grad=True)
    px.xcf_net_adam(ctx, net, lr=1e-3)
    orc.adam(ref, grad2.cpu().numpy().astype(np.float64), m, v, 2, lr=1e-3)
    np.testing.assert_allclose(net.params().cpu().numpy(), ref, rtol=1e-5, atol=1e-7)
    net.close()


def test_training_is_reproducible(px, ctx):
    """The gradients are summed in a fixed order (split partials and bias
    partials reduced in index order, no atomics), so the same initial
    parameters and batches give bit-identical parameters after several Adam
    steps, on a batch large enough for the weight gradients to be split."""
    p = synth.cnn_init_params(K, 12)
    batches = [(_images(64, 20 + i), _quats(64, 30 + i)) for i in range(3)]
    runs = []
    for _ in range(2):
        net = px.xcf_net_create(ctx, K, dev(p))
        for x, q in batches:
            px.xcf_net_loss_grad(ctx, net, dev(x), dev(q))
            px.xcf_net_adam(ctx, net, lr=1e-3)
        torch.cuda.synchronize()
        runs.append(net.params().cpu().clone())
        net.close()
    assert torch.equal(runs[0], runs[1])
    assert not torch.equal(runs[0], torch.from_numpy(p))


def test_proposals_match_oracle(px, ctx, orc):
    p = synth.cnn_init_params(K, 7)
    x = _images(4, 8)
    net = px.xcf_net_create(ctx, K, dev(p))
    got = px.xcf_propose(ctx, net, dev(x)).cpu().numpy()
    ref = orc.cnn_proposals(orc.cnn_forward(p, x, K), K)
    d = np.minimum(np.abs(got - ref).max(axis=2), np.abs(got + ref).max(axis=2))   # q and -q
    assert d.max() < 1e-3
    np.testing.assert_allclose(np.linalg.norm(got, axis=2), 1.0, atol=1e-12)
    net.close()


def test_training_lowers_the_loss(px, ctx):
    """Adam on projected patterns of a few orientations: the loss falls."""
    master = dev(synth.master_pattern("bcc", 512))
    g = px.geometry(128, 128, (0.5, 0.5, 0.6))
    centres = _quats(4, 11)
    torch.manual_seed(0)
    net = px.xcf_net_create(ctx, K, dev(synth.cnn_init_params(K, 8)))
    losses = []
    for step in range(60):
        idx = np.random.default_rng(step).integers(0, 4, 64)
        q = dev(synth.perturb(centres[idx], 3.0, 100 + step))
        imgs = px.xcf_project(ctx, master, q, g)
        loss, _, _ = px.xcf_net_loss_grad(ctx, net, imgs, q, g)
        px.xcf_net_adam(ctx, net, lr=1e-3)
        losses.append(float(loss))
    assert np.mean(losses[-10:]) < 0.7 * np.mean(losses[:5]), losses
    net.close()


# --------------------------------------------------------- learned indexing
@pytest.fixture(scope="module")
def learned_case(px, ctx):
    master = dev(synth.master_pattern("bcc", 512))
    g = px.geometry(128, 128, (0.5, 0.5, 0.6))
    lq = dev(synth.so3_grid_cubic_fz(10.0))
    lib = px.xcf_build_library(ctx, master, lq, g)
    q0 = synth.random_quaternions(1, 21)[0]
    truth = dev(synth.perturb(np.repeat(q0[None], 24, axis=0), 2.0, 22))
    pcs = dev(synth.jittered_pcs(24, 23))
    clean = px.xcf_project(ctx, master, truth, g, pcs=pcs)
    pats = (clean * 80 + 20 + torch.randn(clean.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(3)) * 2)
    pats[5] = 3.0                                               # degenerate
    yield dict(master=master, g=g, lib=lib, lq=lq, q0=q0, truth=truth, pcs=pcs, pats=pats.contiguous())
    lib.close()


def test_learned_all_fallback_equals_full_search(px, ctx, learned_case):
    c = learned_case
    net = px.xcf_net_create(ctx, K, dev(synth.cnn_init_params(K, 9)))
    q, pk, it, fb = px.xcf_index_learned(ctx, net, c["lib"], c["pats"], pcs=c["pcs"], tau=float("inf"))
    ref = px.xcf_index_refine(ctx, c["lib"], c["pats"], pcs=c["pcs"])
    okn = np.ones(24, bool)
    okn[5] = False
    ok = torch.from_numpy(okn).cuda()
    fbn = fb.cpu().numpy()
    assert np.all(fbn[okn] == 1) and fbn[5] == 0
    assert torch.equal(q[ok], ref["quats"][ok]) and torch.equal(pk[ok], ref["rpeak"][ok])
    assert torch.equal(it[ok], ref["iters"][ok])
    net.close()


def test_learned_exact_proposal_needs_no_fallback(px, ctx, learned_case, orc):
    """Weights zero, output bias encoding the map's mean orientation in head 3:
    every pattern is proposed that orientation, refinement converges to the
    truth, no fallback happens."""
    c = learned_case
    n = px.xcf_net_num_params(K)
    p = np.zeros(n, np.float32)
    R = orc.quat_to_matrix(c["q0"])
    b = np.random.default_rng(1).normal(size=6 * K).astype(np.float32)
    b[18:24] = np.r_[R[:, 0], R[:, 1]]
    p[n - 6 * K:] = b
    net = px.xcf_net_create(ctx, K, dev(p))
    prop = px.xcf_propose(ctx, net, c["pats"], c["g"]).cpu().numpy()
    assert np.allclose(np.abs(np.sum(prop[:, 3] * c["q0"], axis=1)), 1.0, atol=1e-6)
    q, pk, it, fb = px.xcf_index_learned(ctx, net, c["lib"], c["pats"], pcs=c["pcs"], tau=0.2)
    fbn = fb.cpu().numpy()
    assert fbn.sum() == 0
    mis = px.xcf_disorientation(ctx, q, c["truth"]).cpu().numpy()
    ok = np.arange(24) != 5
    assert np.mean(mis[ok]) < 0.5 and float(pk[5]) == 0.0
    net.close()

