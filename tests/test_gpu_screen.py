"""Precision form: BF16 zero-shift screen on the tensor cores (top-k), FP32
FFT rescore of the candidates, refinement.  Compared with the oracle's
screen on BF16-rounded inputs (FP64 accumulation), its search restricted to
the same candidates, and the ground truth."""
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


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _oracle_topk(S, k):
    """(cand, score) by score descending, index ascending."""
    order = np.lexsort((np.broadcast_to(np.arange(S.shape[1]), S.shape), -S), axis=1)[:, :k]
    return order, np.take_along_axis(S, order, axis=1)


def _tol(K, s):
    """Tensor-core FP32 accumulation is not round-to-nearest: over the K/16
    accumulations of a K-long dot product of unit vectors (every partial sum
    is at most 1 by Cauchy-Schwarz) the score drifts down by up to about
    1e-8 K (measured: 3.8e-5 at K = 4,096, 8.7e-5 at 16,384, 1.1e-4 at
    65,536)."""
    return 1e-5 + 1e-8 * K + 0 * np.abs(s)


def _check_topk(cand, score, S_ref, k, K):
    oc, os_ = _oracle_topk(S_ref, k)
    for p in range(S_ref.shape[0]):
        got = set(cand[p].tolist())
        want = set(oc[p].tolist())
        kth = os_[p, -1]
        for t in got ^ want:     # differences only among near-ties at the k-th score
            assert abs(S_ref[p, t] - kth) <= 2 * _tol(K, kth), (p, t, S_ref[p, t], kth)
        # every reported score is the BF16 product sum of its template
        ref = S_ref[p, cand[p]]
        assert np.all(np.abs(score[p] - ref) <= _tol(K, ref)), (p, score[p] - ref)
        assert np.all(np.diff(score[p]) <= 0)


def _images_case(orc, n, T, P, seed):
    master = synth.master_pattern("bcc", 512)
    lq = synth.random_quaternions(T, seed)
    timgs = orc.project_many(master, lq, PC0, n).astype(np.float32)
    tq = synth.perturb(lq[np.arange(P) * 3 % T], 2.0, seed + 1)
    pimgs = synth.add_noise(orc.project_many(master, tq, PC0, n), np.broadcast_to(np.asarray(PC0), (P, 3)),
                            300.0, seed + 2)
    return lq, timgs, pimgs


def test_screen_single_tile(px, orc):
    """Smallest case first: one 128 x 256 tile, four K-blocks."""
    n, T, P, k = 16, 7, 5, 4
    rng = np.random.default_rng(0)
    timgs = rng.standard_normal((T, n, n)).astype(np.float32)
    pimgs = (timgs[[1, 3, 5, 0, 2]] + 0.5 * rng.standard_normal((P, n, n))).astype(np.float32)
    ctx = px.Context()
    lib = px.xcf.xcf_build_library_ex(ctx, dev(synth.random_quaternions(T, 1)), px.geometry(n, n),
                                      images=dev(timgs), flags=px.xcf.XCF_LIB_SCREEN)
    cand, score = (host(t) for t in px.xcf.xcf_screen_topk(ctx, lib, dev(pimgs), k))
    _, yt, _ = orc.prep_many(timgs, want_spatial=True)
    _, yp, _ = orc.prep_many(pimgs, want_spatial=True)
    _check_topk(cand, score, orc.screen(yp, yt, bf16=True), k, n * n)
    assert cand[:, 0].tolist() == [1, 3, 5, 0, 2]
    lib.close()
    ctx.close()


@pytest.mark.parametrize("n,T,P,k", [(64, 300, 20, 32), (128, 520, 130, 16), (256, 37, 3, 8)])
def test_screen_matches_oracle(px, orc, n, T, P, k):
    lq, timgs, pimgs = _images_case(orc, n, T, P, 100 + n)
    ctx = px.Context()
    lib = px.xcf.xcf_build_library_ex(ctx, dev(lq), px.geometry(n, n, PC0), images=dev(timgs),
                                      flags=px.xcf.XCF_LIB_SCREEN)
    cand, score = (host(t) for t in px.xcf.xcf_screen_topk(ctx, lib, dev(pimgs), k))
    _, yt, _ = orc.prep_many(timgs, want_spatial=True)
    _, yp, _ = orc.prep_many(pimgs, want_spatial=True)
    _check_topk(cand, score, orc.screen(yp, yt, bf16=True), k, n * n)
    lib.close()
    ctx.close()


def test_screen_from_master_and_fewer_templates_than_k(px, orc):
    n, T, P, k = 64, 5, 3, 8
    master = synth.master_pattern("diamond", 512)
    lq = synth.random_quaternions(T, 7)
    ctx = px.Context()
    lib = px.xcf.xcf_build_library_ex(ctx, dev(lq), px.geometry(n, n, PC0), master=dev(master),
                                      flags=px.xcf.XCF_LIB_SCREEN)
    pimgs = orc.project_many(master, lq[[4, 0, 2]], PC0, n).astype(np.float32)
    cand, score = (host(t) for t in px.xcf.xcf_screen_topk(ctx, lib, dev(pimgs), k))
    assert cand[:, 0].tolist() == [4, 0, 2] and np.all(cand[:, T:] == -1)
    assert np.all(score[:, 0] > 0.99)
    lib.close()
    ctx.close()


def test_rescore_matches_oracle(px, orc):
    n, T, P, k = 128, 80, 6, 8
    lq, timgs, pimgs = _images_case(orc, n, T, P, 7)
    rng = np.random.default_rng(3)
    cand = np.stack([rng.choice(T, k, replace=False) for _ in range(P)]).astype(np.int32)
    cand[:, 0] = np.arange(P) * 3 % T                     # the true template is always a candidate
    cand[1, -1] = -1                                       # an empty slot
    ctx = px.Context()
    lib = px.xcf_build_library_images(ctx, dev(timgs), dev(lq), px.geometry(n, n, PC0))
    best, peak, shift = (host(t) for t in px.xcf.xcf_rescore(ctx, lib, dev(pimgs), dev(cand)))
    St, _, _ = orc.prep_many(timgs)
    Sp, _, deg = orc.prep_many(pimgs)
    _, _, _, allp = orc.index(St, Sp, deg, want_all=True)
    for p in range(P):
        valid = cand[p][cand[p] >= 0]
        vals = allp[p, valid]
        ob = valid[np.lexsort((valid, -vals))][0]
        if best[p] != ob:
            assert abs(allp[p, best[p]] - allp[p, ob]) <= 2e-5 * abs(allp[p, ob])
        np.testing.assert_allclose(peak[p], allp[p, best[p]], rtol=1e-4)
    lib.close()
    ctx.close()


def test_precision_form_end_to_end(px, orc):
    """Screen top-32 -> FP32 rescore -> refinement on a noisy map sample with
    the ~4,000-template library: the rescore finds the full search's template
    for most patterns (the zero-shift screen is blind to shifts, so a template
    that only wins after a translation can fall outside the top 32) and the
    refined orientations meet the 0.5 deg accuracy bar."""
    n, P = 128, 48
    master = synth.master_pattern("bcc", 1024)
    lq = synth.so3_grid_cubic_fz(5.35)
    truth = synth.smooth_orientation_map(6, 8, 11)
    pcs = synth.jittered_pcs(P, 12)
    pimgs = synth.add_noise(orc.project_many(master, truth, pcs, n), pcs, 200.0, 13)
    ctx = px.Context(max_iter=10)
    lib = px.xcf.xcf_build_library_ex(ctx, dev(lq), px.geometry(n, n, PC0), master=dev(master),
                                      flags=px.xcf.XCF_LIB_SCREEN)
    cand, _ = px.xcf.xcf_screen_topk(ctx, lib, dev(pimgs), 32)
    best, peak, _ = px.xcf.xcf_rescore(ctx, lib, dev(pimgs), cand)
    fbest, fpeak, _ = px.xcf_index(ctx, lib, dev(pimgs))
    seeds = dev(lq[host(best)])
    q, _, _ = px.xcf_refine(ctx, lib, dev(pimgs), seeds, pcs=dev(pcs))
    b, fb = host(best), host(fbest)
    assert np.mean(b == fb) >= 0.8, np.mean(b == fb)
    mis = orc.disorientation(host(q), truth)
    assert mis.mean() <= 0.5, mis.mean()
    lib.close()
    ctx.close()


@pytest.mark.parametrize("n,P,k", [(128, 40, 16), (256, 9, 8)])
def test_fused_precision_equals_the_three_calls(px, n, P, k):
    """xcf_index_precision (one pre-processing per chunk) returns exactly what
    screen_topk -> rescore -> refine_best return, including degenerate input."""
    master = synth.master_pattern("bcc", 512)
    lq = synth.so3_grid_cubic_fz(12.0)
    truth = synth.random_quaternions(P, 31 + n)
    pcs = synth.jittered_pcs(P, 32)
    ctx = px.Context(max_iter=3)
    g = px.geometry(n, n, PC0)
    lib = px.xcf.xcf_build_library_ex(ctx, dev(lq), g, master=dev(master), flags=px.xcf.XCF_LIB_SCREEN)
    pats = px.xcf_project(ctx, dev(master), dev(truth), g, pcs=dev(pcs)) * 90 + 15
    pats[3] = 1.0                                            # degenerate
    pats = pats.contiguous()
    b, q, pk, it = px.xcf_index_precision(ctx, lib, pats, pcs=dev(pcs), k=k)
    cand, _ = px.xcf.xcf_screen_topk(ctx, lib, pats, k)
    best, _, _ = px.xcf.xcf_rescore(ctx, lib, pats, cand)
    q2, pk2, it2 = px.xcf.xcf_refine_best(ctx, lib, pats, best, pcs=dev(pcs))
    torch.cuda.synchronize()
    assert torch.equal(b, best) and int(b[3]) == -1
    assert torch.equal(q, q2) and torch.equal(pk, pk2) and torch.equal(it, it2)
    lib.close()
    ctx.close()
