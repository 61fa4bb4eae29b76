"""Multi-map search (one persistent launch over every map up to 160 x 160 of
a batch, 256 x 256 maps on the cluster kernel in the same stream; Fig. 1 B-C
per map) against the per-map search and the FP64 oracle.

Each map's detector is cropped to its 2^n square (FFT section): 40 -> 32,
96 x 80 -> 64, 160 x 140 and 200 x 200 -> 128, 256 -> 256.  With each side
pinned to the search body its per-map kernel runs, best index, peak and shift
must equal xcf_index bit for bit; every body the queue has is checked against
the oracle; and the autotuner's choice is one of them, with results equal to
the per-map search up to ties."""
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


@pytest.fixture(scope="module")
def master():
    return torch.from_numpy(synth.master_pattern("bcc", 512)).cuda()


# (width, height, pattern centre, templates, patterns, seed)
MAPS = [
    (40, 40, (0.5, 0.5, 0.6), 9, 11, 1),
    (96, 80, (0.48, 0.52, 0.62), 20, 30, 2),
    (160, 140, (0.5, 0.45, 0.58), 64, 40, 3),
    (200, 200, (0.52, 0.5, 0.6), 33, 17, 4),
    (256, 256, (0.5, 0.5, 0.6), 6, 5, 5),
]


def _make_map(px, ctx, master, W, H, pc, T, P, seed):
    g = px.geometry(W, H, pc)
    lq = torch.from_numpy(synth.random_quaternions(T, 100 + seed)).cuda()
    lib = px.xcf_build_library(ctx, master, lq, g)
    src = torch.from_numpy(np.arange(P) * 7 % T).cuda()
    q = torch.from_numpy(synth.perturb(lq[src].cpu().numpy(), 2.0, 200 + seed)).cuda()
    clean = px.xcf_project(ctx, master, q, g)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    pats = (clean * 50 + 10 + torch.randn(clean.shape, device="cuda", generator=gen) * 3).contiguous()
    pats[-1] = 4.0   # a degenerate (constant) pattern
    lib.quats_dev = lq
    return g, lib, pats


@pytest.fixture(scope="module")
def maps(px, master):
    ctx = px.Context()
    out = [_make_map(px, ctx, master, *m) for m in MAPS]
    yield ctx, out
    for _, lib, _ in out:
        lib.close()
    ctx.close()


def _per_map(px, ctx, lib, pats):
    return [t.clone() for t in px.xcf_index(ctx, lib, pats)]


def _pin_per_map_bodies(px, ctx, ms):
    """Each (side, library) of the batch on the body of its per-map kernel."""
    for _, lib, _ in ms:
        if lib.N == 256:
            continue
        body = (px.XCF_BODY_ROUNDS if lib.N == 128 else px.XCF_BODY_OCT if lib.N == 64 else
                px.XCF_BODY_SMEM if lib.N < 64 else px.XCF_BODY_REG)
        px.xcf_maps_set_tuning(ctx, lib.N, lib.T, body, max(1, (lib.T + 1) // 8))


def _oracle_check(px, ctx, master, orc, g, lib, pats, best, peak, shift):
    n, ox, oy, _ = orc.crop(g.width, g.height, (g.pcx, g.pcy, g.pcz))
    timgs = px.xcf_project(ctx, master, lib.quats_dev, g).cpu().numpy()[:, oy:oy + n, ox:ox + n]
    St, _, _ = orc.prep_many(timgs)
    Sp, _, deg = orc.prep_many(pats.cpu().numpy()[:, oy:oy + n, ox:ox + n])
    ob, opk, osh, allp = orc.index(St, Sp, deg, want_all=True)
    assert deg[-1] == 1 and best[-1] == -1
    for i in range(len(ob)):
        if best[i] != ob[i]:   # only where the oracle's peaks tie
            assert abs(allp[i, ob[i]] - allp[i, best[i]]) <= 2e-5 * abs(allp[i, ob[i]])
    same = best == ob
    assert same.sum() >= len(ob) - 1
    np.testing.assert_allclose(peak[same], opk[same], rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(shift[same], osh[same], atol=2e-3)


def _assert_same(a, b):
    for x, y in zip(a, b):
        torch.cuda.synchronize()
        assert torch.equal(x, y), (x, y)


def test_maps_equal_per_map_search(px, maps):
    ctx, ms = maps
    _pin_per_map_bodies(px, ctx, ms)
    outs = px.xcf_index_maps(ctx, [(lib, pats) for _, lib, pats in ms])
    for (g, lib, pats), o in zip(ms, outs):
        _assert_same(o, _per_map(px, ctx, lib, pats))
        assert int(o[0][-1]) == -1 and float(o[1][-1]) == 0.0


def test_maps_smallest_against_oracle(px, maps, master, orc):
    ctx, ms = maps
    g, lib, pats = ms[0]
    best, peak, shift = (t.cpu().numpy() for t in px.xcf_index_maps(ctx, [(lib, pats)])[0])
    _oracle_check(px, ctx, master, orc, g, lib, pats, best, peak, shift)


@pytest.mark.parametrize("which,body,groups", [(0, 2, 1), (0, 2, 4), (1, 0, 1), (1, 0, 2), (1, 0, 4), (1, 2, 1),
                                               (1, 2, 4), (1, 3, 1), (1, 3, 2), (1, 3, 4), (2, 0, 1), (2, 1, 1),
                                               (3, 1, 1)])
def test_maps_every_body_against_oracle(px, maps, master, orc, which, body, groups):
    """Each search body the queue has for a side (32: radix-2 in shared
    memory; 64: warp lines, radix-2 in shared memory or 8 x 8 transforms on
    eight-lane groups; 128: warp lines or three register rounds), on whole CTAs or on 2 / 4 groups of warps per CTA
    where it fits, at two granularities, against the oracle at the stated
    bounds."""
    ctx, ms = maps
    g, lib, pats = ms[which]
    for pairs in (max(1, (lib.T + 1) // 2), 3):
        c = px.Context()
        px.xcf_maps_set_tuning(c, lib.N, lib.T, body, pairs, groups)
        assert px.xcf_maps_get_tuning(c, lib.N, lib.T) == (body, groups, min(pairs, (lib.T + 1) // 2))
        best, peak, shift = (t.cpu().numpy() for t in px.xcf_index_maps(c, [(lib, pats)])[0])
        _oracle_check(px, c, master, orc, g, lib, pats, best, peak, shift)
        c.close()


def test_maps_autotuner_choice(px, maps):
    """An unpinned context times the candidate bodies and granularities on the
    first call and records one that serves each side; the results equal the
    per-map search up to the bodies' rounding (ties within 2e-5 relative)."""
    _, ms = maps
    ctx = px.Context()
    outs = px.xcf_index_maps(ctx, [(lib, pats) for _, lib, pats in ms])
    serves = {16: {2}, 32: {2}, 64: {0, 2, 3}, 96: {0}, 128: {0, 1}, 160: {0}}
    for (g, lib, pats), o in zip(ms, outs):
        ref = _per_map(px, ctx, lib, pats)
        if lib.N == 256:
            assert px.xcf_maps_get_tuning(ctx, lib.N, lib.T) is None
            _assert_same(o, ref)
            continue
        body, groups, pairs = px.xcf_maps_get_tuning(ctx, lib.N, lib.T)
        assert body in serves[lib.N] and groups in (1, 2, 4) and 1 <= pairs <= (lib.T + 1) // 2
        assert groups == 1 or lib.N <= 96
        allp = px.xcf_correlate_all(ctx, lib, pats).cpu().numpy()
        b, rb = o[0].cpu().numpy(), ref[0].cpu().numpy()
        for i in np.nonzero(b != rb)[0]:
            assert abs(allp[i, b[i]] - allp[i, rb[i]]) <= 2e-5 * abs(allp[i, rb[i]])
        same = torch.from_numpy(b == rb).cuda()
        assert torch.equal(o[1][same], ref[1][same]) and torch.equal(o[2][same], ref[2][same])
    ctx.close()


def test_maps_order_and_subsets(px, maps):
    """Reversed order, a repeated map and a single map give the same outputs."""
    ctx, ms = maps
    _pin_per_map_bodies(px, ctx, ms)
    sel = [ms[4], ms[1], ms[1], ms[0]]
    outs = px.xcf_index_maps(ctx, [(lib, pats) for _, lib, pats in sel])
    for (g, lib, pats), o in zip(sel, outs):
        _assert_same(o, _per_map(px, ctx, lib, pats))
    assert px.xcf_index_maps(ctx, []) == []


def test_maps_graph_replay_follows_new_data(px, maps):
    ctx, ms = maps
    _pin_per_map_bodies(px, ctx, ms)
    batch = [(lib, pats.clone()) for _, lib, pats in ms]
    outs = px.xcf_index_maps(ctx, batch, graph=True)
    for (lib, pats), o in zip(batch, outs):
        _assert_same(o, _per_map(px, ctx, lib, pats))
    px.xcf_profile_enable(ctx, True)
    px.xcf_profile_read(ctx, reset=True)
    for it in range(2):
        for (lib, pats), (_, _, src) in zip(batch, ms):   # new data, same buffers
            pats.copy_(torch.roll(src, shifts=(it + 1, -it - 2), dims=(1, 2)))
        outs2 = px.xcf_index_maps(ctx, batch, outs=outs, graph=True)
        assert outs2 is outs
        for (lib, pats), o in zip(batch, outs):
            _assert_same(o, _per_map(px, ctx, lib, pats))
    prof = px.xcf_profile_read(ctx, reset=True)
    px.xcf_profile_enable(ctx, False)
    # two replays (per replay: one prep per map, the queue kernel for every map up to 160 x 160 and
    # one cluster search per 256 x 256 map) and 2 x len(batch) per-map searches
    nm = len(batch)
    n_other = sum(px.xcf_crop(lib.geom)[0] == 256 for lib, _ in batch)
    assert prof["search"][1] == 2 * (1 + n_other) + 2 * nm
    assert prof["prep"][1] == 2 * nm + 2 * nm


def test_maps_tuning_rejects_what_does_not_fit(px):
    c = px.Context()
    for N, body, groups in ((128, 1, 2), (128, 0, 2), (160, 0, 2), (96, 0, 4), (256, 0, 1), (96, 1, 1), (160, 2, 1),
                            (64, 0, 3), (96, 3, 1), (128, 3, 1), (32, 3, 1), (64, 4, 1)):
        with pytest.raises(px.XcfError):
            px.xcf_maps_set_tuning(c, N, 100, body, 10, groups)
    assert px.xcf_maps_get_tuning(c, 96, 100) is None
    px.xcf_maps_set_tuning(c, 96, 100, 0, 10, 2)
    assert px.xcf_maps_get_tuning(c, 96, 100) == (0, 2, 10)
    px.xcf_maps_set_tuning(c, 96, 100, 0, 1000, 1)          # pairs clamped to the library's 50
    assert px.xcf_maps_get_tuning(c, 96, 100) == (0, 1, 50)
    c.close()


def test_maps_errors(px, maps):
    import ctypes as C
    ctx, ms = maps
    _, lib, pats = ms[0]
    L = px.load()
    assert L.xcf_index_maps(ctx.handle, None, 1, 0, None) != 0          # no descriptors
    d = (px.xcf.xcf_map_desc * 1)()
    d[0] = px.xcf.xcf_map_desc(lib.handle, pats.data_ptr(), pats.shape[0], None, None, None)
    assert L.xcf_index_maps(ctx.handle, C.cast(d, C.c_void_p), 1, 0, None) != 0   # no outputs
    best, peak, shift = _per_map(px, ctx, lib, pats)
    d[0] = px.xcf.xcf_map_desc(lib.handle, pats.data_ptr(), pats.shape[0], best.data_ptr(), peak.data_ptr(),
                               shift.data_ptr())
    assert L.xcf_index_maps(ctx.handle, C.cast(d, C.c_void_p), 1, 4, None) != 0   # unknown flag
    assert L.xcf_index_maps(ctx.handle, C.cast(d, C.c_void_p), -1, 0, None) != 0  # negative count
    assert L.xcf_index_maps(ctx.handle, C.cast(d, C.c_void_p), 0, 0, None) == 0   # nothing to do
