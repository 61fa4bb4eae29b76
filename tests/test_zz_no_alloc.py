"""xcf_index_noalloc: the library search for callers that cannot allocate
device memory (their memory belongs to another allocator, or their loop
cannot take the synchronisation of cudaMalloc / cudaFree).  It must give the
results of xcf_index, call after call, from its fixed scratch array, and
refuse sizes that do not fit.  Collected last on purpose (file name)."""
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


def _inputs(n, T, P, seed):
    rng = np.random.default_rng(seed)
    timgs = synth.random_images(T, n, n, seed)
    src = rng.integers(0, T, size=P)
    pats = np.stack([np.roll(timgs[s], tuple(rng.integers(-6, 7, size=2)), axis=(0, 1)) for s in src])
    pats = pats + 0.3 * rng.standard_normal(pats.shape).astype(np.float32)
    return timgs, pats.astype(np.float32)


def _compare(ref, got):
    rb, rp, rs = (t.cpu().numpy() for t in ref)
    gb, gp, gs = (t.cpu().numpy() for t in got)
    assert np.array_equal(rb, gb)
    np.testing.assert_allclose(gp, rp, rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(gs, rs, atol=2e-3)


def test_first_call_commits_at_most_the_array(px):
    """The first call on the device loads the module holding the fixed array
    (CUDA loads modules lazily) and so commits the array there; it may take
    no more than the array plus a small slack for the module itself.  Every
    other kernel of the call is loaded beforehand by an ordinary xcf_index."""
    n, T, P = 64, 5, 8
    timgs, pats = _inputs(n, T, P, 7)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = px.Context()
    lib = px.xcf_build_library_images(ctx, dev(timgs), dev(synth.random_quaternions(T, 8)), px.geometry(n, n))
    pd = dev(pats)
    ref = px.xcf_index(ctx, lib, pd)
    out = (torch.empty(P, dtype=torch.int32, device="cuda"), torch.empty(P, device="cuda"),
           torch.empty((P, 2), device="cuda"))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    px.xcf_index_noalloc(ctx, lib, pd, *out)
    torch.cuda.synchronize()
    taken = free0 - torch.cuda.mem_get_info()[0]
    assert taken <= px.xcf.XCF_NOALLOC_SCRATCH_BYTES + (8 << 20), taken
    _compare(ref, out)
    lib.close()
    ctx.close()


@pytest.mark.parametrize("n", [128, 64, 96, 160, 256])
def test_noalloc_matches_index_on_consecutive_calls(px, n):
    T = 37
    timgs, pats1 = _inputs(n, T, 40, 1)
    _, pats2 = _inputs(n, T, 9, 2)
    pats2[3] = 1.5                                   # a pattern with no signal
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx_ref = px.Context(native_sizes=int(n in (96, 160)))
    g = px.geometry(n, n)
    lib = px.xcf_build_library_images(ctx_ref, dev(timgs), dev(synth.random_quaternions(T, 3)), g)
    ref1 = px.xcf_index(ctx_ref, lib, dev(pats1))
    ref2 = px.xcf_index(ctx_ref, lib, dev(pats2))
    torch.cuda.synchronize()

    ctx = px.Context()                               # a context whose own scratch stays empty
    outs = []
    for pats in (pats1, pats2, pats1):
        P = pats.shape[0]
        out = (torch.empty(P, dtype=torch.int32, device="cuda"), torch.empty(P, device="cuda"),
               torch.empty((P, 2), device="cuda"))
        px.xcf_index_noalloc(ctx, lib, dev(pats), *out)
        torch.cuda.synchronize()
        outs.append(out)
    _compare(ref1, outs[0])
    _compare(ref2, outs[1])
    _compare(ref1, outs[2])
    assert outs[1][0][3].item() == -1 and outs[1][1][3].item() == 0.0

    # after the first call (the one-time address look-up), calls allocate nothing
    free0 = torch.cuda.mem_get_info()[0]
    P = pats1.shape[0]
    out = (torch.empty(P, dtype=torch.int32, device="cuda"), torch.empty(P, device="cuda"),
           torch.empty((P, 2), device="cuda"))
    pd = dev(pats1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    px.xcf_index_noalloc(ctx, lib, pd, *out)
    px.xcf_index_noalloc(ctx, lib, pd, *out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    _compare(ref1, out)
    lib.close()
    ctx.close()
    ctx_ref.close()


def test_noalloc_rejects_oversize(px):
    n = 128
    pmax = px.xcf.xcf_noalloc_max_patterns(n)
    assert pmax == 252
    assert px.xcf.xcf_noalloc_max_patterns(256) == 63 and px.xcf.xcf_noalloc_max_patterns(64) == 992
    assert px.xcf.xcf_noalloc_max_patterns(96) > 0 and px.xcf.xcf_noalloc_max_patterns(160) > 0
    assert px.xcf.xcf_noalloc_max_patterns(100) == 0 and px.xcf.xcf_noalloc_max_patterns(512) == 0
    timgs, _ = _inputs(n, 3, 1, 4)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = px.Context()
    lib = px.xcf_build_library_images(ctx, dev(timgs), dev(synth.random_quaternions(3, 5)), px.geometry(n, n))
    P = pmax + 1
    pats = torch.zeros((P, n, n), device="cuda")
    out = (torch.empty(P, dtype=torch.int32, device="cuda"), torch.empty(P, device="cuda"),
           torch.empty((P, 2), device="cuda"))
    with pytest.raises(px.XcfError) as e:
        px.xcf_index_noalloc(ctx, lib, pats, *out)
    assert e.value.code == px.xcf.XCF_ERR_SIZE and str(pmax) in str(e.value)
    lib.close()
    ctx.close()
