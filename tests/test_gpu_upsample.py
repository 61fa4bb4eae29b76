"""Up-sampled correlation peak (the paper's peak up-sampling, reading: the
correlation's Fourier series on a +-1 px grid of step 1/U) on the GPU against
the FP64 oracle: same template, peak to 1e-4, shift to the grid step (a grid
point may flip only on a near-tie of the FP32 and FP64 values)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
PC0 = (0.5, 0.5, 0.6)


@pytest.fixture(scope="module")
def px():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_11313_gb300 as px
    px.load()
    return px


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,U", [(64, 10), (128, 20), (256, 8)])
def test_index_upsampled_matches_oracle(px, orc, n, U):
    master = synth.master_pattern("bcc", 512)
    lq = synth.random_quaternions(6, 60 + n)
    timgs = orc.project_many(master, lq, PC0, n).astype(np.float32)
    rng = np.random.default_rng(n)
    src = np.arange(5) % 6
    truth = synth.perturb(lq[src], 1.5, 61 + n)
    pimgs = (orc.project_many(master, truth, (0.507, 0.493, 0.6), n) * 80 + 10
             + rng.normal(0, 2, (5, n, n))).astype(np.float32)
    ctx0, ctx = px.Context(), px.Context(upsample=U)
    g = px.geometry(n, n, PC0)
    lib = px.xcf_build_library_images(ctx, dev(timgs), dev(lq), g)
    b0, p0, s0 = (t.cpu().numpy() for t in px.xcf_index(ctx0, lib, dev(pimgs)))
    b, pk, sh = (t.cpu().numpy() for t in px.xcf_index(ctx, lib, dev(pimgs)))
    np.testing.assert_array_equal(b, b0)                  # the search is unchanged
    St, _, _ = orc.prep_many(timgs)
    Sp, _, _ = orc.prep_many(pimgs)
    for i in range(5):
        opk, (odx, ody) = orc.pair_upsampled(St[b[i]], Sp[i], U)
        assert abs(pk[i] - opk) <= 1e-4 * abs(opk), (i, pk[i], opk)
        assert abs(sh[i, 0] - odx) <= 1.0 / U + 1e-4 and abs(sh[i, 1] - ody) <= 1.0 / U + 1e-4, (i, sh[i], odx, ody)
        assert pk[i] >= p0[i] - 1e-5                     # the grid contains the integer peak
    lib.close()
    ctx.close()
    ctx0.close()


def test_refine_upsampled_matches_oracle(px, orc):
    n, P, U = 128, 6, 10
    master = synth.master_pattern("bcc", 1024)
    truth = synth.random_quaternions(P, 70)
    seeds = synth.perturb(truth, 3.0, 71)
    pcs = synth.jittered_pcs(P, 72)
    pats = orc.project_many(master, truth, pcs, n).astype(np.float32)
    ctx = px.Context(max_iter=4, upsample=U)
    lib = px.xcf_build_library(ctx, dev(master), dev(seeds[:2]), px.geometry(n, n, PC0))
    q, pk, it = px.xcf_refine(ctx, lib, dev(pats), dev(seeds), pcs=dev(pcs))
    oq, opk, oit = orc.refine_many(master, pats, seeds, pcs, max_it=4, tol_deg=1e-3,
                                   opts=orc.default_opts(n, upsample=U))
    mis = orc.disorientation(q.cpu().numpy(), oq)
    assert mis.max() < 0.02, mis
    assert orc.disorientation(q.cpu().numpy(), truth).mean() < 0.1
    lib.close()
    ctx.close()
