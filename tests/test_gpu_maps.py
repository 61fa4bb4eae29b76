"""Multi-map search (one persistent launch over the 128 x 128 maps of a batch,
the other sides in their own kernels of the same stream; Fig. 1 B-C per map)
against the per-map search and the FP64 oracle.

Each map's detector is cropped to its 2^n square (FFT section): 40 -> 32,
96 x 80 -> 64, 160 x 140 and 200 x 200 -> 128, 256 -> 256.  The multi-map
launch runs the same search bodies as the per-map kernels, so best index,
peak and shift must equal xcf_index bit for bit; the smallest map is also
checked against the oracle."""
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


def _assert_same(a, b):
    for x, y in zip(a, b):
        torch.cuda.synchronize()
        assert torch.equal(x, y), (x, y)


def test_maps_equal_per_map_search(px, maps):
    ctx, ms = maps
    outs = px.xcf_index_maps(ctx, [(lib, pats) for _, lib, pats in ms])
    for (g, lib, pats), o in zip(ms, outs):
        _assert_same(o, _per_map(px, ctx, lib, pats))
        assert int(o[0][-1]) == -1 and float(o[1][-1]) == 0.0


def test_maps_smallest_against_oracle(px, maps, master, orc):
    ctx, ms = maps
    g, lib, pats = ms[0]
    best, peak, shift = (t.cpu().numpy() for t in px.xcf_index_maps(ctx, [(lib, pats)])[0])
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


def test_maps_order_and_subsets(px, maps):
    """Reversed order, a repeated map and a single map give the same outputs."""
    ctx, ms = maps
    sel = [ms[4], ms[1], ms[1], ms[0]]
    outs = px.xcf_index_maps(ctx, [(lib, pats) for _, lib, pats in sel])
    for (g, lib, pats), o in zip(sel, outs):
        _assert_same(o, _per_map(px, ctx, lib, pats))
    assert px.xcf_index_maps(ctx, []) == []


def test_maps_graph_replay_follows_new_data(px, maps):
    ctx, ms = maps
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
    # two replays (per replay: one prep per map, the queue kernel for the 128 x 128 maps and one
    # search kernel per other map) and 2 x len(batch) per-map searches
    nm = len(batch)
    n_other = sum(px.xcf_crop(lib.geom)[0] != 128 for lib, _ in batch)
    assert prof["search"][1] == 2 * (1 + n_other) + 2 * nm
    assert prof["prep"][1] == 2 * nm + 2 * nm


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
