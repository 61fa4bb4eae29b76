"""Native 96 x 96, 160 x 160 and 200 x 200 detectors (option native_sizes:
mixed-radix 3 x 32 and 5 x 32 register line transforms with two images per
pre-processing CTA at 96 and 160; at 200 one template per pass through the
real-output transform, 8 x 5 x 5 and 4 x 5 x 5 Stockham line passes) against
the oracle, whose lines of those lengths are direct DFTs: pre-processing
(spectra, spatial images, degeneracy, cropping), all-pairs correlation peaks,
library search, candidate-list rescore, the up-sampled peak and the
refinement."""
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


@pytest.fixture(scope="module")
def nctx(px):
    c = px.Context(native_sizes=1)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("n", [96, 160, 200])
def test_native_prep_matches_oracle(px, nctx, orc, n):
    rng = np.random.default_rng(n)
    imgs = (rng.standard_normal((5, n, n)) * 3 + 7).astype(np.float32)   # odd count: a lone last image
    imgs[3] = 2.0                                                          # degenerate: constant
    g = px.geometry(n, n)
    spec, spat, deg = px.xcf_prep(nctx, dev(imgs), g, want_spatial=True)
    S, y, odeg = orc.prep_many(imgs, want_spatial=True)
    assert host(deg).tolist() == odeg.tolist() == [0, 0, 0, 1, 0]
    np.testing.assert_allclose(host(spec), S[:, :, : n // 2 + 1], rtol=0, atol=2e-6)
    np.testing.assert_allclose(host(spat), y, rtol=0, atol=2e-6)


def test_native_crop_of_a_rectangular_detector(px, nctx, orc):
    rng = np.random.default_rng(9)
    W, H = 200, 180
    imgs = rng.standard_normal((3, H, W)).astype(np.float32)
    g = px.geometry(W, H, (0.45, 0.52, 0.6))
    n, ox, oy, _ = orc.crop(W, H, (0.45, 0.52, 0.6), native=True)
    assert (n, ox, oy) == (160, 20, 10)
    spec, _, _ = px.xcf_prep(nctx, dev(imgs), g)
    assert spec.shape[1] == 160
    S, _, _ = orc.prep_many(imgs[:, oy:oy + n, ox:ox + n])
    np.testing.assert_allclose(host(spec), S[:, :, : n // 2 + 1], rtol=0, atol=2e-6)
    # a 240 x 210 detector keeps a 200 px square
    W, H = 240, 210
    imgs = rng.standard_normal((2, H, W)).astype(np.float32)
    g = px.geometry(W, H, (0.5, 0.48, 0.6))
    n, ox, oy, _ = orc.crop(W, H, (0.5, 0.48, 0.6), native=True)
    assert (n, ox, oy) == (200, 20, 5) and px.xcf_crop(g, native=True)[:3] == (200, 20, 5)
    spec, spat, _ = px.xcf_prep(nctx, dev(imgs), g, want_spatial=True)
    S, y, _ = orc.prep_many(imgs[:, oy:oy + n, ox:ox + n], want_spatial=True)
    np.testing.assert_allclose(host(spec), S[:, :, : n // 2 + 1], rtol=0, atol=2e-6)
    np.testing.assert_allclose(host(spat), y, rtol=0, atol=2e-6)


def _patterns(orc, master, lib_q, idx, n, seed, pc=PC0, peak=300.0, perturb_deg=2.0):
    q = synth.perturb(lib_q[idx], perturb_deg, seed)
    clean = orc.project_many(master, q, pc, n)
    return synth.add_noise(clean, np.broadcast_to(np.asarray(pc), (len(idx), 3)), peak, seed + 1), q


@pytest.mark.parametrize("n,T,P", [(96, 23, 5), (160, 9, 3), (200, 7, 3)])
def test_native_search_matches_oracle(px, nctx, orc, n, T, P):
    master = synth.master_pattern("bcc", 512)
    lq = synth.random_quaternions(T, 60 + n)
    timgs = orc.project_many(master, lq, PC0, n).astype(np.float32)
    pimgs, _ = _patterns(orc, master, lq, np.arange(P) * 3 % T, n, 70 + n)
    pimgs = np.concatenate([pimgs, np.full((1, n, n), 4.0, np.float32)])   # + a degenerate one
    g = px.geometry(n, n, PC0)
    lib = px.xcf_build_library_images(nctx, dev(timgs), dev(lq), g)
    peaks = host(px.xcf_correlate_all(nctx, lib, dev(pimgs)))
    best, peak, shift = (host(t) for t in px.xcf_index(nctx, lib, dev(pimgs)))
    St, _, _ = orc.prep_many(timgs)
    Sp, _, deg = orc.prep_many(pimgs)
    ob, opk, osh, allp = orc.index(St, Sp, deg, want_all=True)
    np.testing.assert_allclose(peaks, allp, rtol=1e-4, atol=1e-6)
    for p in range(P):
        assert best[p] == ob[p] or abs(allp[p, best[p]] - opk[p]) <= 2e-5 * abs(opk[p])
    same = best == ob
    np.testing.assert_allclose(peak[same], opk[same], rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(shift[same], osh[same], atol=2e-3)
    assert best[-1] == -1 and peak[-1] == 0.0
    # the candidate-list search (the rescore) over every template in a shuffled order finds the same best
    cand = np.stack([np.random.default_rng(p).permutation(T) for p in range(P + 1)]).astype(np.int32)
    cand[0, -1] = -1                                   # an empty slot is skipped
    rb, rpk, rsh = (host(t) for t in px.xcf_rescore(nctx, lib, dev(pimgs), dev(cand)))
    for p in range(P):
        allowed = [t for t in cand[p] if t >= 0]
        ob_p = max(allowed, key=lambda t: (allp[p, t], -t))
        assert rb[p] == ob_p or abs(allp[p, rb[p]] - allp[p, ob_p]) <= 2e-5 * abs(allp[p, ob_p])
    lib.close()


@pytest.mark.parametrize("n", [96, 200])
def test_native_upsampled_peak_matches_oracle(px, orc, n):
    U = 5
    ctx = px.Context(native_sizes=1, upsample=U)
    master = synth.master_pattern("bcc", 512)
    lq = synth.random_quaternions(6, 81)
    timgs = orc.project_many(master, lq, PC0, n).astype(np.float32)
    pimgs, _ = _patterns(orc, master, lq, np.array([1, 4, 5]), n, 82)
    lib = px.xcf_build_library_images(ctx, dev(timgs), dev(lq), px.geometry(n, n, PC0))
    best, peak, shift = (host(t) for t in px.xcf_index(ctx, lib, dev(pimgs)))
    St, _, _ = orc.prep_many(timgs)
    Sp, _, _ = orc.prep_many(pimgs)
    for p in range(3):
        opk, (odx, ody) = orc.pair_upsampled(St[best[p]], Sp[p], U)
        assert abs(peak[p] - opk) <= 1e-4 * abs(opk), (p, peak[p], opk)
        assert abs(shift[p, 0] - odx) <= 1.0 / U + 1e-4 and abs(shift[p, 1] - ody) <= 1.0 / U + 1e-4
    lib.close()
    ctx.close()


@pytest.mark.parametrize("n,P", [(96, 6), (160, 3), (200, 3)])
def test_native_refine_matches_oracle(px, orc, n, P):
    master = synth.master_pattern("bcc", 1024)
    seeds = synth.random_quaternions(P, 90 + n)
    truth = synth.perturb(seeds, 3.0, 91 + n)
    pcs = synth.jittered_pcs(P, 92 + n)
    clean = np.stack([orc.project(master, truth[i], pcs[i], n) for i in range(P)])
    pats = synth.add_noise(clean, pcs, 200.0, 93 + n)
    c = px.Context(max_iter=3, tol_deg=0.0, native_sizes=1)
    lib = px.xcf_build_library(c, dev(master), dev(seeds[:2]), px.geometry(n, n, PC0))
    q, pk, it = (host(t) for t in px.xcf_refine(c, lib, dev(pats), dev(seeds), pcs=dev(pcs)))
    oq, opk, oit = orc.refine_many(master, pats, seeds, pcs, max_it=3, tol_deg=0.0)
    assert it.tolist() == oit.tolist() == [3] * P
    assert orc.disorientation(q, oq).max() < 0.01
    np.testing.assert_allclose(pk, opk, rtol=1e-3)
    assert orc.disorientation(q, truth).mean() < 1.0
    # the NDP needs 2^k sides
    with pytest.raises(px.XcfError):
        px.xcf.xcf_build_library_ex(c, dev(seeds), px.geometry(n, n, PC0), master=dev(master),
                                    flags=px.XCF_LIB_NDP)
    lib.close()
    c.close()


def test_native_maps_batch_matches_oracle(px, orc):
    """One xcf_index_maps call over native 96 / 160 maps, a 2^k map and a
    native 200 px map (the cluster-free 200 kernel in the same stream) against
    the oracle's search of each map."""
    master = synth.master_pattern("bcc", 512)
    c = px.Context(native_sizes=1)
    batch, oracle_in = [], []
    for i, (W, T, P) in enumerate(((96, 11, 4), (160, 7, 3), (128, 9, 3), (200, 5, 2))):
        n, ox, oy, pcc = orc.crop(W, W, PC0, native=True)
        lq = synth.random_quaternions(T, 200 + i)
        q = synth.perturb(lq[np.arange(P) % T], 2.0, 210 + i)
        timgs = orc.project_many(master, lq, pcc, n).astype(np.float32)
        pimgs = synth.add_noise(orc.project_many(master, q, pcc, n), np.broadcast_to(pcc, (P, 3)), 300.0, 220 + i)
        tfull = np.zeros((T, W, W), np.float32)
        pfull = np.zeros((P, W, W), np.float32)
        tfull[:, oy:oy + n, ox:ox + n] = timgs
        pfull[:, oy:oy + n, ox:ox + n] = pimgs
        lib = px.xcf_build_library_images(c, dev(tfull), dev(lq), px.geometry(W, W, PC0))
        batch.append((lib, dev(pfull)))
        oracle_in.append((timgs, pimgs))
    assert [lib.N for lib, _ in batch] == [96, 160, 128, 200]
    outs = px.xcf_index_maps(c, batch)
    for (best, peak, shift), (timgs, pimgs), (lib, _) in zip(outs, oracle_in, batch):
        best, peak, shift = host(best), host(peak), host(shift)
        St, _, _ = orc.prep_many(timgs)
        Sp, _, deg = orc.prep_many(pimgs)
        ob, opk, osh, allp = orc.index(St, Sp, deg, want_all=True)
        for p in range(len(ob)):
            assert best[p] == ob[p] or abs(allp[p, best[p]] - opk[p]) <= 2e-5 * abs(opk[p])
        same = best == ob
        np.testing.assert_allclose(peak[same], opk[same], rtol=1e-4, atol=1e-6)
        np.testing.assert_allclose(shift[same], osh[same], atol=2e-3)
        lib.close()
    c.close()
