"""Full-size workload in the launch configuration bench.py times (10,000
patterns of 128 x 128 against the 4,065-template library, refinement to
convergence): sampled outputs against the oracle one by one, and the
properties that must hold everywhere."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def run(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_11313_gb300 as px
    wl = synth.config_map_128(seed=0)
    n, P = wl["n"], len(wl["truth_q"])
    clean = orc.project_many(wl["master"], wl["truth_q"][:P], wl["pcs"][:P], n)
    pats = synth.add_noise(clean, wl["pcs"], wl["peak"], wl["noise_seed"])
    del clean
    ctx = px.Context(max_iter=wl["max_iter"], tol_deg=1e-3)
    geom = px.geometry(n, n, wl["pc"])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    lib = px.xcf_build_library(ctx, dev(wl["master"]), dev(wl["lib_q"]), geom)
    out = px.xcf_index_refine(ctx, lib, dev(pats), pcs=dev(wl["pcs"]))
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    lib.close()
    ctx.close()
    return wl, pats, res


def test_properties_everywhere(orc, run):
    wl, pats, r = run
    T = len(wl["lib_q"])
    assert np.all((r["best"] >= 0) & (r["best"] < T))
    assert np.all(r["peak"] <= 1.0 + 1e-5) and np.all(r["peak"] > 0)
    assert np.all(np.abs(r["shift"]) <= 64)
    assert np.all((r["iters"] >= 1) & (r["iters"] <= wl["max_iter"]))
    mis = orc.disorientation(r["quats"], wl["truth_q"])
    assert mis.mean() <= 0.5, mis.mean()


def test_sampled_patterns_match_oracle(orc, run):
    wl, pats, r = run
    n = wl["n"]
    sel = np.array([0, 1, 4321, 5000, 7777, 9999])
    St, _, _ = orc.prep_many(orc.project_many(wl["master"], wl["lib_q"], wl["pc"], n))
    Sp, _, deg = orc.prep_many(pats[sel])
    # the map's per-pattern centres: shifts relative to each pattern's own centre
    ob, opk, osh, allp = orc.index(St, Sp, deg, want_all=True, pcs=wl["pcs"][sel], geom=(n, n, *wl["pc"][:2]))
    del St
    best = r["best"][sel]
    for i, p in enumerate(sel):
        if best[i] != ob[i]:
            a, b = allp[i, ob[i]], allp[i, best[i]]
            assert abs(a - b) <= 2e-5 * abs(a), (p, best[i], ob[i], a, b)
    same = best == ob
    np.testing.assert_allclose(r["peak"][sel][same], opk[same], rtol=1e-4)
    np.testing.assert_allclose(r["shift"][sel][same], osh[same], atol=2e-3)
    seeds = wl["lib_q"][best]
    oq, opk2, oit = orc.refine_many(wl["master"], pats[sel], seeds, wl["pcs"][sel],
                                    max_it=wl["max_iter"], tol_deg=1e-3)
    d = orc.disorientation(r["quats"][sel], oq)
    assert d.max() < 0.01, d
    assert np.all(np.abs(r["iters"][sel] - oit) <= 1)
