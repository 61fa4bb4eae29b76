"""Normalised dot product (Eq. 1) dictionary indexing and the peak-width
experiment of the sampling-frequency section (Figs. 3, 4) on the GPU, against
the oracle: BF16 tensor-core NDP scores against the oracle's on BF16-rounded
operands, the FP32 rescore against the FP64 NDP, the rotation scan's curves
and FWHMs against the oracle's, and the paper's accuracy experiment (100
random patterns, NDP at 2.5 deg / FFT at 7.5 deg, two refinements; Fig. 8)."""

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

PC0 = (0.5, 0.5, 0.6)
PC_SCAN = (0.5, 0.3, 0.6)


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


def _tol(K):
    """BF16-operand scores: FP32 tensor-core accumulation of K products of
    unit vectors drifts by up to about 1e-8 K (as for the XCF screen)."""
    return 1e-5 + 1e-8 * K


def _bg(orc, imgs, sigma):
    """Oracle background correction of each image (sigma as the option)."""
    return np.stack([orc.ndp_background(im, sigma) for im in imgs])


def _ndp_vectors(orc, imgs, n):
    """Oracle contrast-normalised crops scaled by 1/n (unit vectors)."""
    return np.stack([orc.ndp_normalise(im)[0].ravel() / n for im in imgs])


def _case(orc, n, T, P, seed):
    """Oracle projections on an n x n screen: T random library orientations,
    P noisy patterns 1 deg away from library entries."""
    master = synth.master_pattern("bcc", 512)
    lq = synth.random_quaternions(T, seed)
    timgs = orc.project_many(master, lq, PC0, n)
    tq = synth.perturb(lq[np.arange(P) * 7 % T], 1.0, seed + 1)
    pimgs = synth.add_noise(orc.project_many(master, tq, PC0, n), np.broadcast_to(np.asarray(PC0), (P, 3)),
                            300.0, seed + 2)
    return master, lq, timgs.astype(np.float32), pimgs.astype(np.float32)


@pytest.mark.parametrize("n,T,P,k,sigma", [(64, 300, 37, 8, 0.0), (128, 500, 21, 4, 0.0), (64, 300, 37, 8, -1.0),
                                           (16, 60, 9, 4, 0.0), (32, 80, 11, 3, 2.5)])
def test_ndp_index_matches_oracle(px, orc, n, T, P, k, sigma):
    master, lq, timgs, pimgs = _case(orc, n, T, P, seed=n)
    pimgs[P - 1] = 3.0                                  # a constant (degenerate) pattern
    ctx = px.Context(ndp_bg_sigma=sigma)
    g = px.geometry(n, n, PC0)
    lib = px.xcf.xcf_build_library_ex(ctx, dev(lq), g, images=dev(timgs),
                                      flags=px.XCF_LIB_NDP | px.XCF_LIB_NO_SPECTRA)
    best, ndp, cand, cs = px.xcf_index_ndp(ctx, lib, dev(pimgs), k=k, want_cand=True)
    best, ndp, cand, cs = host(best), host(ndp), host(cand), host(cs)
    # background correction (or none with sigma < 0), then Eq. 1
    timgs, pimgs = _bg(orc, timgs, sigma), _bg(orc, pimgs, sigma)
    vt, vp = _ndp_vectors(orc, timgs, n), _ndp_vectors(orc, pimgs, n)
    S_bf = orc.screen(vp, vt, bf16=True)
    S = vp @ vt.T                                        # Eq. 1, FP64
    K = n * n
    for p in range(P - 1):
        # candidates: the BF16 top-k (ties only at the k-th score), scores descending
        order = np.lexsort((np.arange(T), -S_bf[p]))[:k]
        kth = S_bf[p, order[-1]]
        for t in set(cand[p].tolist()) ^ set(order.tolist()):
            assert abs(S_bf[p, t] - kth) <= 2 * _tol(K), (p, t)
        np.testing.assert_allclose(cs[p], S_bf[p, cand[p]], atol=_tol(K))
        assert np.all(np.diff(cs[p]) <= 0)
        # FP32 rescore: the candidates' best by the FP64 NDP, and its value
        sc = S[p, cand[p]]
        assert best[p] in cand[p]
        assert S[p, best[p]] >= sc.max() - 2e-6, (p, best[p], sc)
        assert ndp[p] == pytest.approx(S[p, best[p]], abs=2e-6)
        # Eq. 1 directly on the images
        assert ndp[p] == pytest.approx(orc.ndp(pimgs[p], timgs[best[p]]), abs=2e-6)
    assert best[P - 1] == -1 and ndp[P - 1] == 0.0
    # the oracle's dictionary indexing agrees wherever its winner is a candidate
    ob, osc, _ = orc.ndp_index(pimgs, timgs)
    for p in range(P - 1):
        if ob[p] in cand[p]:
            assert best[p] == ob[p] or abs(S[p, best[p]] - osc[p]) <= 2e-6
    # an NDP-only library refuses the FFT search
    with pytest.raises(px.XcfError) as e:
        px.xcf_index(ctx, lib, dev(pimgs.astype(np.float32)))
    assert e.value.code == -1
    lib.close()
    ctx.close()


def test_ndp_cropped_detector_and_master_library(px, orc):
    """An 80 x 72 detector (crop 64 at offsets (8, 4)): the library projected
    from the master equals the one made from the detector images, and both
    agree with the oracle on the background-corrected crops."""
    W, H, T, P = 80, 72, 120, 9
    master = synth.master_pattern("bcc", 512)
    lq = synth.random_quaternions(T, 3)
    ctx = px.Context()
    g = px.geometry(W, H, PC0)
    n, ox, oy, _ = orc.crop(W, H, PC0)
    assert (n, ox, oy) == (64, 8, 4)
    full_t = px.xcf_project(ctx, dev(master), dev(lq), g)
    tq = synth.perturb(lq[:P], 1.0, 4)
    pats = px.xcf_project(ctx, dev(master), dev(tq), g)
    lib_m = px.xcf.xcf_build_library_ex(ctx, dev(lq), g, master=dev(master), flags=px.XCF_LIB_NDP)
    lib_i = px.xcf.xcf_build_library_ex(ctx, dev(lq), g, master=dev(master), images=full_t,
                                        flags=px.XCF_LIB_NDP)
    bm, nm = px.xcf_index_ndp(ctx, lib_m, pats, k=4)
    bi, ni = px.xcf_index_ndp(ctx, lib_i, pats, k=4)
    assert torch.equal(bm, bi) and torch.equal(nm, ni)
    crops_t = _bg(orc, host(full_t)[:, oy:oy + n, ox:ox + n], 0.0)
    crops_p = _bg(orc, host(pats)[:, oy:oy + n, ox:ox + n], 0.0)
    ob, osc, _ = orc.ndp_index(crops_p, crops_t)
    bm, nm = host(bm), host(nm)
    for p in range(P):
        assert nm[p] == pytest.approx(orc.ndp(crops_p[p], crops_t[bm[p]]), abs=2e-6)
        assert bm[p] == ob[p] or osc[p] - nm[p] <= 2e-6
    # a library with both forms serves the FFT search too
    b, pk, sh = px.xcf_index(ctx, lib_m, pats)
    assert host(b).min() >= 0
    lib_m.close()
    lib_i.close()
    ctx.close()


def test_ndp_empty_and_arguments(px):
    ctx = px.Context()
    g = px.geometry(64, 64, PC0)
    master = dev(synth.master_pattern("bcc", 256))
    lq = dev(synth.random_quaternions(5, 1))
    lib = px.xcf.xcf_build_library_ex(ctx, lq, g, master=master, flags=px.XCF_LIB_NDP)
    b, s = px.xcf_index_ndp(ctx, lib, torch.empty((0, 64, 64), device="cuda"))
    assert b.numel() == 0
    with pytest.raises(px.XcfError):
        px.xcf_index_ndp(ctx, lib, torch.zeros((2, 64, 64), device="cuda"), k=65)
    plain = px.xcf_build_library(ctx, master, lq, g)
    with pytest.raises(px.XcfError):
        px.xcf_index_ndp(ctx, plain, torch.zeros((2, 64, 64), device="cuda"))
    with pytest.raises(px.XcfError):
        px.xcf_rotation_scan(ctx, master, g, dev(np.array([1.0, 0, 0, 0])), 0, 1.0)
    plain.close()
    lib.close()
    ctx.close()


@pytest.mark.parametrize("n,upsample,pc_test", [(64, 0, None), (128, 0, (0.51, 0.29, 0.6)), (256, 0, None),
                                                (64, 5, (0.5, 0.3, 0.62))])
def test_rotation_scan_matches_oracle(px, orc, n, upsample, pc_test):
    master = synth.master_pattern("bcc", 1024)
    q = synth.random_quaternions(1, 20 + n)[0]
    h, step = 8, 1.5
    ctx = px.Context(upsample=upsample)
    g = px.geometry(n, n, PC_SCAN)
    nd, xc, fw = px.xcf_rotation_scan(ctx, dev(master), g, dev(q), h, step,
                                      pc_test=dev(np.asarray(pc_test)) if pc_test else None)
    nd, xc, fw = host(nd), host(xc), host(fw)
    ond, oxc = orc.rotation_scan(master, q, PC_SCAN, n, h, step, pc_test=pc_test,
                                 opts=orc.default_opts(n, upsample=upsample))
    np.testing.assert_allclose(nd, ond, atol=2e-5)
    np.testing.assert_allclose(xc, oxc, rtol=2e-4, atol=2e-5)
    for r, curves in enumerate((nd, xc)):
        for a in range(3):
            # the device's FWHM is the oracle's rule applied to the device curve
            assert fw[r, a] == pytest.approx(orc.fwhm(curves[a].astype(np.float64), step), abs=1e-4)
            wo = orc.fwhm((ond, oxc)[r][a], step)
            if wo > 0 and fw[r, a] > 0:
                assert fw[r, a] == pytest.approx(wo, abs=0.02)
    if pc_test is None:
        np.testing.assert_allclose(nd[:, h], 1.0, atol=2e-6)
        np.testing.assert_allclose(xc[:, h], 1.0, atol=2e-5)
    ctx.close()


def test_rotation_scan_paper_claims(px):
    """On the device: the FFT peak is wider than the NDP peak about every
    axis; the NDP is narrowest about x or y (sampling-frequency section)."""
    master = dev(synth.master_pattern("bcc", 1024))
    ctx = px.Context()
    g = px.geometry(128, 128, PC_SCAN)
    for seed in (5, 6, 7):
        q = dev(synth.random_quaternions(1, seed)[0])
        _, _, fw = px.xcf_rotation_scan(ctx, master, g, q, 90, 0.5)
        fw = host(fw)
        assert np.all(fw[0] > 0), fw
        assert np.all((fw[1] == -1) | (fw[1] > fw[0])), fw
        assert min(fw[0, 0], fw[0, 1]) < fw[0, 2], fw
    ctx.close()


def test_accuracy_fig8_ndp_and_fft(px):
    """100 random orientations, 128 x 128, NDP at 2.5 deg (39,784 templates)
    and FFT at 7.5 deg, two refinement iterations each: both reach the
    paper's accuracy (better than about 0.1-0.2 deg)."""
    master = dev(synth.master_pattern("bcc", 1024))
    truth = dev(synth.random_quaternions(100, 77))
    g = px.geometry(128, 128, PC0)
    ctx = px.Context(max_iter=2, tol_deg=1e-3)
    pats = px.xcf_project(ctx, master, truth, g)
    res = {}
    for name, sf in (("ndp", 2.5), ("fft", 7.5)):
        lq = dev(synth.so3_grid_cubic_fz(sf))
        if name == "ndp":
            lib = px.xcf.xcf_build_library_ex(ctx, lq, g, master=master,
                                              flags=px.XCF_LIB_NDP | px.XCF_LIB_NO_SPECTRA)
            best, _ = px.xcf_index_ndp(ctx, lib, pats, k=4)
        else:
            lib = px.xcf_build_library(ctx, master, lq, g)
            best, _, _ = px.xcf_index(ctx, lib, pats)
        q, _, _ = px.xcf_refine_best(ctx, lib, pats, best)
        res[name] = (host(px.xcf_disorientation(ctx, lq[best.long()].contiguous(), truth)),
                     host(px.xcf_disorientation(ctx, q, truth)))
        lib.close()
    ctx.close()
    lib_ndp, ref_ndp = res["ndp"]
    lib_fft, ref_fft = res["fft"]
    # the library match is bounded by the sampling (half the cell diagonal)
    assert np.median(lib_ndp) < 2.5 and np.median(lib_fft) < 7.5, (np.median(lib_ndp), np.median(lib_fft))
    for ref in (ref_ndp, ref_fft):
        assert np.median(ref) < 0.2 and np.mean(ref < 0.5) >= 0.9, (np.median(ref), np.mean(ref < 0.5))
