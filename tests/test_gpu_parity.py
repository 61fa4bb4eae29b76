"""CUDA path against the FP64 oracle, element by element, on identical seeded
inputs (through the C ABI).  Tolerances: spectra and images to a few 1e-6 of
their scale (FP32 transforms), correlation peaks to 1e-4 relative, indices
bit-exact outside documented ties (oracle peaks within 2e-5 relative), refined
orientations to 0.01 deg."""
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
def ctx(px):
    c = px.Context()
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _check_index(orc_best, orc_peak, orc_all, best, peak, rel_tie=2e-5):
    """Bit-exact template index, or a documented tie in the oracle's peaks."""
    for p in range(len(orc_best)):
        if best[p] == orc_best[p]:
            continue
        assert orc_best[p] >= 0 and best[p] >= 0, (p, best[p], orc_best[p])
        a, b = orc_all[p, orc_best[p]], orc_all[p, best[p]]
        assert abs(a - b) <= rel_tie * abs(a), (p, best[p], orc_best[p], a, b)


# ---------------------------------------------------------------- prep
@pytest.mark.parametrize("n", [16, 32, 64, 128, 256])
def test_prep_matches_oracle(px, ctx, orc, n):
    rng = np.random.default_rng(n)
    imgs = (rng.standard_normal((5, n, n)) * 3 + 7).astype(np.float32)
    imgs[3] = 2.0                                       # degenerate: constant
    g = px.geometry(n, n)
    spec, spat, deg = px.xcf_prep(ctx, dev(imgs), g, want_spatial=True)
    S, y, odeg = orc.prep_many(imgs, want_spatial=True)
    assert host(deg).tolist() == odeg.tolist() == [0, 0, 0, 1, 0]
    np.testing.assert_allclose(host(spec), S[:, :, : n // 2 + 1], rtol=0, atol=2e-6)
    np.testing.assert_allclose(host(spat), y, rtol=0, atol=2e-6)


def test_prep_crops_rectangular_detector(px, ctx, orc):
    rng = np.random.default_rng(3)
    W, H = 150, 140
    imgs = rng.standard_normal((3, H, W)).astype(np.float32)
    g = px.geometry(W, H, (0.45, 0.52, 0.6))
    n, ox, oy, _ = px.xcf_crop(g)
    assert (n, ox, oy) == (128, 11, 6)
    spec, _, _ = px.xcf_prep(ctx, dev(imgs), g)
    S, _, _ = orc.prep_many(imgs[:, oy:oy + n, ox:ox + n])
    np.testing.assert_allclose(host(spec), S[:, :, : n // 2 + 1], rtol=0, atol=2e-6)


def test_prep_window_off(px, orc):
    c = px.Context(window=0, sigma_hp=3.0, sigma_lp=10.0)
    rng = np.random.default_rng(4)
    imgs = rng.standard_normal((2, 64, 64)).astype(np.float32)
    spec, _, _ = px.xcf_prep(c, dev(imgs), px.geometry(64, 64))
    S, _, _ = orc.prep_many(imgs, orc.default_opts(64, window=0, sigma_hp=3.0, sigma_lp=10.0))
    np.testing.assert_allclose(host(spec), S[:, :, :33], rtol=0, atol=2e-6)
    c.close()


# ---------------------------------------------------------- projection
def _proj_check(out, ref, master):
    rng_v = float(master.max() - master.min())
    err = np.abs(out - ref)
    assert err.max() < 2e-3 * rng_v, err.max()
    assert np.quantile(err, 0.99) < 1e-4 * rng_v, np.quantile(err, 0.99)


@pytest.mark.parametrize("n,pc", [(64, PC0), (128, (0.43, 0.56, 0.65))])
def test_project_matches_oracle(px, ctx, orc, n, pc):
    m = synth.master_pattern("bcc", 1024)
    q = synth.random_quaternions(6, 3)
    out = px.xcf_project(ctx, dev(m), dev(q), px.geometry(n, n, pc))
    _proj_check(host(out), orc.project_many(m, q, pc, n), m)


def test_project_per_pattern_pc_and_rectangle(px, ctx, orc):
    m = synth.master_pattern("diamond", 1024)
    q = synth.random_quaternions(4, 8)
    pcs = synth.jittered_pcs(4, 9, jitter=0.02)
    W, H = 160, 120
    g = px.geometry(W, H, PC0)
    out = host(px.xcf_project(ctx, dev(m), dev(q), g, pcs=dev(pcs)))
    n, ox, oy, _ = px.xcf_crop(g)
    for i in range(4):
        _, _, _, pcc = orc.crop(W, H, pcs[i], cap=256)
        ref = orc.project(m, q[i], pcc, n)
        _proj_check(out[i, oy:oy + n, ox:ox + n], ref, m)


# ---------------------------------------------------------- library search
def _patterns(orc, master, lib_q, idx, n, seed, pc=PC0, peak=300.0, perturb_deg=2.0):
    q = synth.perturb(lib_q[idx], perturb_deg, seed)
    pcs = np.broadcast_to(np.asarray(pc), (len(idx), 3))
    clean = orc.project_many(master, q, pc, n)
    return synth.add_noise(clean, pcs, peak, seed + 1), q


@pytest.mark.parametrize("n,T,P", [(16, 5, 3), (32, 9, 2), (64, 37, 5), (128, 41, 4), (128, 3, 1),
                                   (128, 1, 2), (128, 200, 3), (256, 7, 2)])
def test_correlate_all_matches_oracle(px, ctx, orc, n, T, P):
    master = synth.master_pattern("bcc", 512)
    lq = synth.random_quaternions(T, 10 + T)
    timgs = orc.project_many(master, lq, PC0, n).astype(np.float32)
    pimgs, _ = _patterns(orc, master, lq, np.arange(P) % T, n, 20 + P)
    pimgs = np.concatenate([pimgs, np.full((1, n, n), 5.0, np.float32)])   # + a degenerate one
    g = px.geometry(n, n, PC0)
    lib = px.xcf_build_library_images(ctx, dev(timgs), dev(lq), g)
    peaks = host(px.xcf_correlate_all(ctx, lib, dev(pimgs)))
    St, _, _ = orc.prep_many(timgs)
    Sp, _, deg = orc.prep_many(pimgs)
    _, _, _, allp = orc.index(St, Sp, deg, want_all=True)
    np.testing.assert_allclose(peaks, allp, rtol=1e-4, atol=1e-6)
    assert np.all(peaks <= 1.0 + 1e-5)
    lib.close()


@pytest.mark.parametrize("n,T,P", [(64, 50, 9), (128, 60, 12), (256, 12, 3)])
def test_index_matches_oracle(px, ctx, orc, n, T, P):
    master = synth.master_pattern("bcc", 1024)
    lq = synth.random_quaternions(T, 40 + n)
    timgs = orc.project_many(master, lq, PC0, n).astype(np.float32)
    pimgs, _ = _patterns(orc, master, lq, np.arange(P) * 5 % T, n, 50 + n, pc=(0.51, 0.49, 0.6))
    pimgs = np.concatenate([pimgs, np.zeros((1, n, n), np.float32)])
    g = px.geometry(n, n, PC0)
    lib = px.xcf_build_library_images(ctx, dev(timgs), dev(lq), g)
    best, peak, shift = (host(t) for t in px.xcf_index(ctx, lib, dev(pimgs)))
    St, _, _ = orc.prep_many(timgs)
    Sp, _, deg = orc.prep_many(pimgs)
    ob, opk, osh, allp = orc.index(St, Sp, deg, want_all=True)
    _check_index(ob, opk, allp, best, peak)
    same = best == ob
    np.testing.assert_allclose(peak[same], opk[same], rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(shift[same], osh[same], atol=2e-3)
    assert best[-1] == -1 and peak[-1] == 0.0 and np.all(shift[-1] == 0)
    lib.close()


@pytest.mark.parametrize("n,W,H", [(64, 64, 64), (128, 150, 140)])
def test_index_per_pattern_pcs_matches_oracle(px, ctx, orc, n, W, H):
    """Per-pattern pattern centres (a map whose centre drifts): indices and
    peaks are the library-centre search's, the shift is reported relative to
    the template at the pattern's own centre; against the oracle at the
    stated bounds, on a cropped rectangular detector too."""
    P, T = 10, 40
    master = synth.master_pattern("bcc", 1024)
    lq = synth.random_quaternions(T, 300 + n)
    g = px.geometry(W, H, PC0)
    cn, ox, oy, pcc = orc.crop(W, H, PC0)
    assert cn == n
    timgs = np.zeros((T, H, W), np.float32)
    timgs[:, oy:oy + n, ox:ox + n] = orc.project_many(master, lq, pcc, n)
    pcs = synth.jittered_pcs(P, 301 + n, jitter=0.03)
    q = synth.perturb(lq[np.arange(P) * 3 % T], 1.5, 302)
    full = np.zeros((P, H, W), np.float32)
    for i in range(P):
        _, _, _, pci = orc.crop(W, H, pcs[i])
        full[i, oy:oy + n, ox:ox + n] = orc.project(master, q[i], pci, n)
    pimgs = synth.add_noise(full, pcs, 300.0, 303)
    lib = px.xcf_build_library_images(ctx, dev(timgs), dev(lq), g)
    best, peak, shift = (host(t) for t in px.xcf_index(ctx, lib, dev(pimgs), pcs=dev(pcs)))
    b0, p0, s0 = (host(t) for t in px.xcf_index(ctx, lib, dev(pimgs)))
    St, _, _ = orc.prep_many(timgs[:, oy:oy + n, ox:ox + n])
    Sp, _, deg = orc.prep_many(pimgs[:, oy:oy + n, ox:ox + n])
    ob, opk, osh, allp = orc.index(St, Sp, deg, want_all=True, pcs=pcs, geom=(W, H, PC0[0], PC0[1]))
    _check_index(ob, opk, allp, best, peak)
    same = best == ob
    np.testing.assert_allclose(peak[same], opk[same], rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(shift[same], osh[same], atol=2e-3)
    # the centres change only the shift, by the translation they produce
    assert np.array_equal(best, b0) and np.array_equal(peak, p0)
    move = np.stack([(pcs[:, 0] - PC0[0]) * W, (pcs[:, 1] - PC0[1]) * H], axis=1)
    np.testing.assert_allclose(s0 - shift, move, atol=1e-4)
    lib.close()


def test_build_library_matches_oracle_spectra(px, ctx, orc):
    n = 128
    master = synth.master_pattern("bcc", 1024)
    lq = synth.random_quaternions(7, 77)
    lib = px.xcf_build_library(ctx, dev(master), dev(lq), px.geometry(n, n, PC0))
    got = host(lib.spectra())
    St, _, _ = orc.prep_many(orc.project_many(master, lq, PC0, n))
    ref = St[:, :, : n // 2 + 1]
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() < 2e-4 * scale
    lib.close()


@pytest.mark.parametrize("n,W,H", [(64, 64, 64), (128, 150, 140), (256, 256, 256)])
def test_library_projection_inside_prep_equals_two_kernels(px, ctx, n, W, H):
    """The library build projects its templates inside the pre-processing
    kernel (sides up to 128) or with the projection kernel first (256): the
    spectra are bit-identical to xcf_project followed by xcf_prep, including
    on a detector larger than its crop."""
    master = synth.master_pattern("bcc", 512)
    lq = synth.random_quaternions(5, 9)
    g = px.geometry(W, H, PC0)
    assert px.xcf_crop(g)[0] == n
    lib = px.xcf_build_library(ctx, dev(master), dev(lq), g)
    imgs = px.xcf_project(ctx, dev(master), dev(lq), g)
    spec, _, degen = px.xcf_prep(ctx, imgs, g)
    assert torch.equal(lib.spectra(), spec) and int(degen.sum()) == 0
    lib.close()


def test_index_chunks_and_empty(px, orc):
    """More patterns than one device pass holds (ragged tail), and P = 0."""
    c = px.Context()
    n, P = 16, 16384 + 37
    rng = np.random.default_rng(5)
    timgs = rng.standard_normal((3, n, n)).astype(np.float32)
    src = rng.integers(0, 3, size=P)
    shifts = rng.integers(-4, 5, size=(P, 2))
    pimgs = np.stack([np.roll(timgs[s], tuple(d), axis=(0, 1)) for s, d in zip(src, shifts)])
    g = px.geometry(n, n)
    lib = px.xcf_build_library_images(c, dev(timgs), dev(synth.random_quaternions(3, 1)), g)
    best, peak, _ = (host(t) for t in px.xcf_index(c, lib, dev(pimgs)))
    St, _, _ = orc.prep_many(timgs)
    sel = np.r_[0:5, P - 40:P]
    Sp, _, deg = orc.prep_many(pimgs[sel])
    ob, opk, _, allp = orc.index(St, Sp, deg, want_all=True)
    _check_index(ob, opk, allp, best[sel], peak[sel])
    np.testing.assert_allclose(peak[sel], opk, rtol=1e-4)
    e = px.xcf_index(c, lib, torch.empty((0, n, n), dtype=torch.float32, device="cuda"))
    assert all(t.numel() == 0 for t in e)
    lib.close()
    c.close()


def _config1_inputs(orc):
    """The 64 x 64 parity configuration: diamond-cubic master on a
    2 x 1024^2 grid, 300 random templates, 16 random test patterns with
    Poisson noise (peak 200) plus background, seed 0."""
    n = 64
    master = synth.master_pattern("diamond", 1024)
    lq = synth.random_quaternions(300, 0)
    tq = synth.random_quaternions(16, 1)
    pcs = np.broadcast_to(np.asarray(PC0), (16, 3))
    pimgs = synth.add_noise(orc.project_many(master, tq, PC0, n), pcs, 200.0, 2)
    return n, master, lq, pimgs


def test_config1_parity_same_templates(px, ctx, orc):
    """The search itself at the parity configuration, at the stated bounds:
    both sides correlate the same FP32 template images (the oracle's FP64
    projection rounded to FP32), so only the FP32 transforms differ.  Indices
    bit-exact outside ties (oracle peaks within 2e-5 relative), peaks 1e-4
    relative, shifts 2e-3 px; every per-template peak 1e-4 relative."""
    n, master, lq, pimgs = _config1_inputs(orc)
    timgs = orc.project_many(master, lq, PC0, n).astype(np.float32)
    g = px.geometry(n, n, PC0)
    lib = px.xcf_build_library_images(ctx, dev(timgs), dev(lq), g, master=dev(master))
    best, peak, shift = (host(t) for t in px.xcf_index(ctx, lib, dev(pimgs)))
    allg = host(px.xcf_correlate_all(ctx, lib, dev(pimgs)))
    St, _, _ = orc.prep_many(timgs)
    Sp, _, deg = orc.prep_many(pimgs)
    ob, opk, osh, allp = orc.index(St, Sp, deg, want_all=True)
    _check_index(ob, opk, allp, best, peak, rel_tie=2e-5)
    same = best == ob
    assert same.sum() >= 15
    np.testing.assert_allclose(peak[same], opk[same], rtol=1e-4)
    np.testing.assert_allclose(shift[same], osh[same], atol=2e-3)
    np.testing.assert_allclose(allg, allp, rtol=1e-4, atol=1e-6)
    lib.close()


def test_config1_parity(px, ctx, orc):
    """End to end at the parity configuration: the GPU library comes from the
    GPU's own FP32 projection, the oracle's from its FP64 projection, so the
    comparison carries the projection's FP32 error (up to ~1e-3 of the
    master's range at single pixels near band edges) into the correlation.
    Bounds: ties 1e-4 relative, peaks 2e-4 relative, shifts 5e-3 px."""
    n = 64
    master = synth.master_pattern("diamond", 1024)
    lq = synth.random_quaternions(300, 0)
    tq = synth.random_quaternions(16, 1)
    pcs = np.broadcast_to(np.asarray(PC0), (16, 3))
    pimgs = synth.add_noise(orc.project_many(master, tq, PC0, n), pcs, 200.0, 2)
    lib = px.xcf_build_library(ctx, dev(master), dev(lq), px.geometry(n, n, PC0))
    best, peak, shift = (host(t) for t in px.xcf_index(ctx, lib, dev(pimgs)))
    St, _, _ = orc.prep_many(orc.project_many(master, lq, PC0, n))
    Sp, _, deg = orc.prep_many(pimgs)
    ob, opk, osh, allp = orc.index(St, Sp, deg, want_all=True)
    _check_index(ob, opk, allp, best, peak, rel_tie=1e-4)
    same = best == ob
    np.testing.assert_allclose(peak[same], opk[same], rtol=2e-4)
    np.testing.assert_allclose(shift[same], osh[same], atol=5e-3)
    lib.close()


# ------------------------------------------------------------ refinement
@pytest.mark.parametrize("noise,n,P,windows", [(None, 128, 8, 0), (150.0, 128, 8, 0), (150.0, 256, 4, 0),
                                               (150.0, 128, 8, 1), (150.0, 64, 8, 3), (150.0, 32, 6, 8)])
def test_refine_matches_oracle(px, orc, noise, n, P, windows):
    master = synth.master_pattern("bcc", 1024)
    seeds = synth.random_quaternions(P, 90)
    truth = synth.perturb(seeds, 4.0, 91)
    pcs = synth.jittered_pcs(P, 92)
    clean = np.stack([orc.project(master, truth[i], pcs[i], n) for i in range(P)])
    pats = clean.astype(np.float32) if noise is None else synth.add_noise(clean, pcs, noise, 93)
    c = px.Context(max_iter=4, tol_deg=0.0, lp_windows=windows)
    lib = px.xcf_build_library(c, dev(master), dev(seeds[:2]), px.geometry(n, n, PC0))
    q, pk, it = (host(t) for t in px.xcf_refine(c, lib, dev(pats), dev(seeds), pcs=dev(pcs)))
    # log-polar windows: 0 selects four (at most the N/4 radii)
    oq, opk, oit = orc.refine_many(master, pats, seeds, pcs, max_it=4, tol_deg=0.0,
                                   opts=orc.default_opts(n, lp_windows=min(windows or 4, n // 4)))
    assert it.tolist() == oit.tolist() == [4] * P
    d = orc.disorientation(q, oq)
    assert d.max() < 0.01, d
    np.testing.assert_allclose(pk, opk, rtol=1e-3)
    if noise is None:
        assert orc.disorientation(q, truth).max() < 0.01
    lib.close()
    c.close()


def test_refine_converges_and_stops(px, orc):
    n, P = 64, 6
    master = synth.master_pattern("diamond", 1024)
    seeds = synth.random_quaternions(P, 95)
    truth = synth.perturb(seeds, 3.0, 96)
    pats = orc.project_many(master, truth, PC0, n).astype(np.float32)
    pats[2] = 1.0                                     # degenerate: not refined
    c = px.Context(max_iter=12, tol_deg=1e-3)
    lib = px.xcf_build_library(c, dev(master), dev(seeds[:1]), px.geometry(n, n, PC0))
    q, pk, it = (host(t) for t in px.xcf_refine(c, lib, dev(pats), dev(seeds)))
    ok = np.arange(P) != 2
    assert it[2] == 0 and np.allclose(q[2], seeds[2])
    assert np.all(it[ok] < 12) and np.all(it[ok] >= 2)
    assert orc.disorientation(q[ok], truth[ok]).max() < 0.02
    lib.close()
    c.close()


def test_disorientation_matches_oracle(px, ctx, orc):
    qa = synth.random_quaternions(500, 1)
    qb = synth.perturb(qa, 20.0, 2)
    qb[:100] = synth.random_quaternions(100, 3)
    d = host(px.xcf_disorientation(ctx, dev(qa), dev(qb)))
    np.testing.assert_allclose(d, orc.disorientation(qa, qb), atol=1e-6)


def test_host_pipeline_matches_device_path(px, orc):
    n, T, P = 64, 30, 50
    master = synth.master_pattern("bcc", 512)
    lq = synth.random_quaternions(T, 60)
    pimgs, _ = _patterns(orc, master, lq, np.arange(P) % T, n, 61)
    pcs = synth.jittered_pcs(P, 62)
    c = px.Context(max_iter=3)
    lib = px.xcf_build_library(c, dev(master), dev(lq), px.geometry(n, n, PC0))
    out = px.xcf_index_refine_host(c, lib, torch.from_numpy(pimgs).pin_memory(),
                                   pcs=torch.from_numpy(pcs), chunk=16)
    best, peak, shift = (host(t) for t in px.xcf_index(c, lib, dev(pimgs), pcs=dev(pcs)))
    seeds = dev(lq[np.maximum(best, 0)])
    q, rpk, it = (host(t) for t in px.xcf_refine(c, lib, dev(pimgs), seeds, pcs=dev(pcs)))
    assert np.array_equal(out["best"].numpy(), best)
    assert np.array_equal(out["peak"].numpy(), peak)
    assert np.array_equal(out["shift"].numpy(), shift)
    assert np.array_equal(out["quats"].numpy(), q)
    assert np.array_equal(out["iters"].numpy(), it)
    lib.close()
    c.close()


def test_errors_are_reported(px, ctx):
    with pytest.raises(px.XcfError) as e:               # below the smallest 2^n crop
        px.xcf_prep(ctx, torch.zeros((1, 12, 40), device="cuda"), px.geometry(40, 12))
    assert e.value.code == px.xcf.XCF_ERR_SIZE
    lib = px.xcf_build_library_images(ctx, torch.rand((2, 64, 64), device="cuda"),
                                      torch.from_numpy(synth.random_quaternions(2, 0)).cuda(), px.geometry(64, 64))
    with pytest.raises(px.XcfError) as e:               # no master pattern: nothing to re-project
        px.xcf_refine(ctx, lib, torch.rand((1, 64, 64), device="cuda"),
                      torch.from_numpy(synth.random_quaternions(1, 1)).cuda())
    assert e.value.code == px.xcf.XCF_ERR_ARG
    lib.close()
    with pytest.raises(TypeError):
        px.xcf_prep(ctx, torch.zeros((1, 64, 64), dtype=torch.float64, device="cuda"), px.geometry(64, 64))


@pytest.mark.parametrize("n", [64, 128, 256])
def test_pattern_at_library_orientation_returns_that_template(px, ctx, n):
    """A noise-free pattern simulated at a library orientation (same geometry)
    returns that template with a correlation peak of 1 at zero shift."""
    master = dev(synth.master_pattern("bcc", 512))
    lq = synth.so3_grid_cubic_fz(14.0 if n == 256 else 10.0)
    g = px.geometry(n, n, PC0)
    lib = px.xcf_build_library(ctx, master, dev(lq), g)
    pick = np.array([0, 7, len(lq) // 2, len(lq) - 1])
    pats = px.xcf_project(ctx, master, dev(lq[pick]), g)
    best, peak, shift = (host(t) for t in px.xcf_index(ctx, lib, pats))
    np.testing.assert_array_equal(best, pick)
    np.testing.assert_allclose(peak, 1.0, atol=2e-5)
    np.testing.assert_allclose(shift, 0.0, atol=1e-3)
    lib.close()


def test_bicubic_projection_matches_oracle(px, orc):
    """Projection with the bicubic master lookup (Keys, a = -1/2) against the oracle."""
    n, P = 64, 5
    master = synth.master_pattern("bcc", 256)
    q = synth.random_quaternions(P, 81)
    pcs = synth.jittered_pcs(P, 82)
    ctx = px.Context(master_interp=1)
    got = px.xcf_project(ctx, dev(master), dev(q), px.geometry(n, n, PC0), pcs=dev(pcs)).cpu().numpy()
    ref = orc.project_many(master, q, pcs, n, interp=1)
    lin = orc.project_many(master, q, pcs, n, interp=0)
    _proj_check(got, ref, master)                         # FP32 ray and Lambert maths, as for bilinear
    assert np.abs(got - lin).max() > 1e-3 * float(master.max() - master.min())   # the option is in effect
    ctx.close()


def test_scratch_limit_gives_oom_and_context_survives(px):
    """A cap on the context's scratch turns a too-large call into XCF_ERR_OOM
    before any allocation; the same context then serves calls that fit."""
    n = 64
    ctx = px.Context()
    lq = synth.random_quaternions(4, 91)
    master = dev(synth.master_pattern("bcc", 128))
    lib = px.xcf_build_library(ctx, master, dev(lq), px.geometry(n, n, PC0))
    pats = px.xcf_project(ctx, master, dev(lq), px.geometry(n, n, PC0))
    best, _, _ = px.xcf_index(ctx, lib, pats)             # the small call's scratch is now held
    used = px.xcf_scratch_bytes(ctx)
    px.xcf_set_scratch_limit(ctx, used + 1024)
    big = pats.repeat(2000, 1, 1).contiguous()           # needs far more scratch
    with pytest.raises(px.XcfError) as e:
        px.xcf_index(ctx, lib, big)
    assert e.value.code == -3 and px.xcf_scratch_bytes(ctx) <= used + 1024
    best, peak, _ = px.xcf_index(ctx, lib, pats)          # fits in what is held
    assert torch.equal(best.cpu(), torch.arange(4, dtype=torch.int32))
    px.xcf_set_scratch_limit(ctx, 0)                      # lifted: the large call now runs
    best, _, _ = px.xcf_index(ctx, lib, big)
    assert torch.equal(best[:4].cpu(), torch.arange(4, dtype=torch.int32))
    lib.close()
    ctx.close()
