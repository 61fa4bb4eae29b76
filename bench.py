#!/usr/bin/env python
"""Throughput of the GB300 refined template-matching EBSD indexer.

Workload (synthetic, seeded): BCC master pattern on a 2 x 1024^2 Lambert grid,
128 x 128 detector, 4,065-orientation cubic-fundamental-zone library
(S^2 x S^1 grid, 5.35 deg), a 100 x 100 map (10,000 patterns) of smoothly
varying orientations with +-2 deg jitter, PC jittered by +-0.005, Poisson noise
at 100 counts plus background.  One step = build the library (projection +
pre-processing of every template), search every pattern against every
template (FFT cross-correlation, best template, sub-pixel shift) and refine
every pattern to convergence (at most 10 iterations) -- all through the C ABI
on device-resident inputs.  The metric is patterns per second; the mean
misorientation of the refined orientations against the ground truth is
reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank indexes its own map (weak scaling, no data
exchange); rank 0 prints one JSON line.  --impl reference times the FP64 CPU
oracle on the host cores instead (bounded samples of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "patterns indexed/s at <=0.5 deg mean misorientation vs plain FP32 XCF; % roofline"
UNIT = "patterns/s"
FLOPS_PER_PAIR_128 = 2.5 * 128 * 128 * 14 + 6 * 128 * 65   # inverse real FFT + conj-multiply


# ------------------------------------------------------------ multi-rank timing
def max_over_ranks(elapsed, dist, device):
    """The job's time: every rank's elapsed time (any unit), all-reduced by
    MAX (the slowest rank); unchanged on one rank."""
    if not dist:
        return elapsed
    import torch
    t = torch.tensor([float(elapsed)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, world, elapsed_ms):
    """Whole-job throughput: the units every rank processed in `steps` steps
    (weak scaling: the same count per rank), over the job's time."""
    return units_per_rank_step * steps * world / (elapsed_ms / 1e3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--map", type=int, default=100, help="map side (patterns = map^2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="plain form: skip the precision / learned / batched sub-records of the line")
    ap.add_argument("--form-steps", type=int, default=3, help="timed steps of each sub-record form")
    ap.add_argument("--cpu-sample", type=int, default=0, help="patterns in the CPU sample (0: auto)")
    ap.add_argument("--form", default="plain",
                    choices=["plain", "precision", "batched", "learned", "ndp", "fwhm", "so3", "net"],
                    help="plain: full FP32 XCF search + refinement of the 128^2 map; precision: BF16 "
                         "tensor-core screen top-32 + FP32 rescore + refinement at 256^2; batched: eight maps "
                         "with different detectors in one persistent graph-captured search; learned: CNN proposals "
                         "+ correlation score + refinement with full-search fallback; ndp: normalised dot product "
                         "(Eq. 1) over the 2.5 deg library on the tensor cores + FP32 rescore + refinement of the "
                         "same 128^2 map; fwhm: the peak-width experiments of Figs. 3-4 (rotation scans about the "
                         "detector axes, NDP and FFT, against screen size and PC error); so3: the SO(3) sampling "
                         "study of Fig. 2 (library generation and nearest-neighbour disorientations); net: the proposal "
                         "network's forward alone on 128^2 images (--patterns, default 100,000)")
    ap.add_argument("--patterns", type=int, default=0,
                    help="precision form: patterns per GPU (0: 50,000); net form: images per GPU (0: 100,000)")
    ap.add_argument("--scale", type=float, default=1.0, help="batched form: scale of every map's pattern count")
    ap.add_argument("--native", action="store_true",
                    help="batched form: native crop rule (96 and 160 px detectors used whole, 200 -> 160)")
    ap.add_argument("--upsample", type=int, default=0,
                    help="plain form: 0 = 3-point parabolic peak; U in [2, 20] = up-sampled peak (grid step 1/U px)")
    ap.add_argument("--train", type=int, default=200000, help="learned form: training patterns")
    ap.add_argument("--batch", type=int, default=256, help="learned form: training batch")
    ap.add_argument("--epochs", type=int, default=2, help="learned form: passes over the training set")
    ap.add_argument("--lr", type=float, default=1e-3, help="learned form: peak learning rate")
    ap.add_argument("--net-fp32", action="store_true",
                    help="learned form: FP32 network inference (default: BF16 tensor-core convolutions 2..5)")
    ap.add_argument("--sigma-hp", type=float, default=0.0,
                    help="fwhm form: high-pass sigma of the FFT path, cycles/image (0: the library default)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def clocks_start(gpu_index: int):
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    try:
        p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={CLOCK_Q}",
                              "--format=csv,noheader,nounits", "-lms", "200"], stdout=f,
                             stderr=subprocess.DEVNULL)
    except OSError:
        p = None
    return p, f.name


def clocks_stop(handle):
    p, path = handle
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    rows = []
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), hw=parts[5], hwt=parts[6],
                             swt=parts[7], swp=parts[8]))
        except ValueError:
            continue
    os.unlink(path)
    if not rows:
        return None
    reasons = set()
    for r in rows:
        for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                        ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
            if r[k].lower().startswith("active"):
                reasons.add(name)
    return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
            "reasons": sorted(reasons), "samples": len(rows)}


# --------------------------------------------------------------- cpu side
def cpu_oracle_rate(wl, pats: np.ndarray, sample: int):
    """Time the FP64 oracle (as it stands) on `sample` patterns of the workload:
    library build (amortised over the whole map) + full search + refinement."""
    import oracle
    threads = oracle.num_threads()
    n, pc = wl["n"], wl["pc"]
    t0 = time.perf_counter()
    St, _, _ = oracle.prep_many(oracle.project_many(wl["master"], wl["lib_q"], pc, n))
    t_lib = time.perf_counter() - t0
    sel = np.arange(sample)
    t0 = time.perf_counter()
    Sp, _, deg = oracle.prep_many(pats[sel])
    best, _, _, _ = oracle.index(St, Sp, deg)
    seeds = wl["lib_q"][np.maximum(best, 0)]
    oracle.refine_many(wl["master"], pats[sel], seeds, wl["pcs"][sel], max_it=wl["max_iter"], tol_deg=1e-3)
    t_s = time.perf_counter() - t0
    P = len(wl["truth_q"])
    per_pattern = t_s / sample + t_lib / P
    return 1.0 / per_pattern, threads, t_lib, t_s


def _roofline_traffic(meta_name: str, sources):
    """DRAM bytes per launch of a kernel from the committed ncu summary, if it
    was taken on the current source of that kernel (sha256 over `sources`)."""
    import hashlib
    meta = os.path.join(ROOT, "profiles", meta_name)
    if not os.path.exists(meta):
        return None
    m = json.load(open(meta))
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(ROOT, "paper_1807_11313_gb300", "csrc", f), "rb").read())
    if m.get("source_sha256") != h.hexdigest():
        return None
    return m.get("bytes_per_launch_full")


SEARCH128_SOURCES = ("search128.cuh", "k_search128.cu")


def _l2_note(pattern_bytes, lib_bytes, what):
    big = pattern_bytes > L2_BYTES or lib_bytes > L2_BYTES
    return (f"{'inputs larger than L2' if big else 'inputs NOT larger than L2'} "
            f"({pattern_bytes / 1e6:.0f} MB patterns, {lib_bytes / 1e6:.0f} MB {what}; L2 129 MB)")


L2_BYTES = 129e6


def peaks_file():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(p)) if os.path.exists(p) else None


# ------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    wl = synth.config_map_128(seed=0, ny=args.map, nx=args.map)
    n, P = wl["n"], len(wl["truth_q"])
    threads = oracle.num_threads()
    sample = args.cpu_sample or max(threads, 8)
    t0 = time.perf_counter()
    St, _, _ = oracle.prep_many(oracle.project_many(wl["master"], wl["lib_q"], wl["pc"], n))
    t_lib = time.perf_counter() - t0
    times = []
    for s in range(args.warmup + args.steps):
        sel = (np.arange(sample) + s * sample) % P
        clean = oracle.project_many(wl["master"], wl["truth_q"][sel], wl["pc"], n)
        pats = synth.add_noise(clean, wl["pcs"][sel], wl["peak"], wl["noise_seed"] + s)
        t0 = time.perf_counter()
        Sp, _, deg = oracle.prep_many(pats)
        best, _, _, _ = oracle.index(St, Sp, deg)
        oracle.refine_many(wl["master"], pats, wl["lib_q"][np.maximum(best, 0)], wl["pcs"][sel],
                           max_it=wl["max_iter"], tol_deg=1e-3)
        dt = time.perf_counter() - t0 + t_lib * sample / P
        if s >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = sample / (ms / 1e3)
    samp = (f"{sample} patterns per step of the {P}-pattern map: full {len(wl['lib_q'])}-template search + "
            f"refinement (<= {wl['max_iter']} iterations); library build ({t_lib:.1f} s) amortised over {P}")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "patterns_per_step": sample, "detector": n,
                       "templates": len(wl["lib_q"])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": samp},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------- precision form
def _noisy_on_device(torch, clean, pcs, peak, gen):
    """Poisson(peak (0.6 hump + 0.4 clean scaled to [0, 1])) on the device
    (input generation only, outside the timed region)."""
    P, H, W = clean.shape
    lo = clean.amin(dim=(1, 2), keepdim=True)
    hi = clean.amax(dim=(1, 2), keepdim=True)
    ih = (clean - lo) / (hi - lo).clamp_min(1e-30)
    ry = torch.arange(H, device=clean.device, dtype=torch.float32) + 0.5
    rx = torch.arange(W, device=clean.device, dtype=torch.float32) + 0.5
    cy = (pcs[:, 1] * H).float().view(P, 1, 1)
    cx = (pcs[:, 0] * W).float().view(P, 1, 1)
    hump = torch.exp(-((ry.view(1, H, 1) - cy) ** 2 + (rx.view(1, 1, W) - cx) ** 2) / (2 * (0.35 * W) ** 2))
    lam = peak.float().view(P, 1, 1) * (0.6 * hump + 0.4 * ih)
    return torch.poisson(lam, generator=gen)


def cpu_precision_rate(wl, pats, pcs, P_total, t_sub=256):
    """The FP64 oracle on a bounded sample of the precision workload: the
    library build and the screen on t_sub evenly spaced templates (both
    linear in the template count, scaled to the whole library), then for each
    sample pattern its top-k candidates of that screen rescored by the XCF
    (one pattern per call, timed on one core and divided by the core count:
    patterns are independent) and the refinement (max_iter iterations)."""
    import oracle
    n, T, k = wl["n"], len(wl["lib_q"]), wl["k"]
    threads = oracle.num_threads()
    sub = np.linspace(0, T - 1, min(T, t_sub)).astype(np.int64)
    t0 = time.perf_counter()
    St, yt, _ = oracle.prep_many(oracle.project_many(wl["master"], wl["lib_q"][sub], wl["pc"], n), want_spatial=True)
    t_lib = (time.perf_counter() - t0) * T / len(sub)
    t0 = time.perf_counter()
    Sp, yp, deg = oracle.prep_many(pats, want_spatial=True)
    t_prep = time.perf_counter() - t0
    t0 = time.perf_counter()
    sc = oracle.screen(yp, yt, bf16=True)
    t_screen = (time.perf_counter() - t0) * T / len(sub)
    kk = min(k, len(sub))
    cand = np.argsort(-sc, axis=1, kind="stable")[:, :kk]
    t0 = time.perf_counter()
    best = np.array([cand[p][max(0, int(oracle.index(St[cand[p]], Sp[p:p + 1], deg[p:p + 1])[0][0]))]
                     for p in range(len(pats))])
    t_rescore = (time.perf_counter() - t0) / threads
    t0 = time.perf_counter()
    oracle.refine_many(wl["master"], pats, wl["lib_q"][sub][best], pcs, max_it=wl["max_iter"], tol_deg=1e-3)
    t_refine = time.perf_counter() - t0
    S = len(pats)
    per = t_lib / P_total + (t_prep + t_screen + t_rescore + t_refine) / S
    sample = (f"{S} of the {P_total} patterns: pre-processing, BF16-rounded screen against {len(sub)} of the {T} "
              f"templates scaled to {T} ({t_screen:.1f} s), top-{kk} XCF rescore ({t_rescore:.1f} s, one core / "
              f"{threads}), refinement ({t_refine:.1f} s); library build of {len(sub)} templates scaled to {T} "
              f"({t_lib:.0f} s) amortised over {P_total}")
    return {"value": 1.0 / per, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}


def run_precision(args, px, torch, dev, rank, world, local, dist, emit=True):
    P = args.patterns or 50000
    wl = synth.config_precision_256(seed=rank, P=P)
    n, T, k = wl["n"], len(wl["lib_q"]), wl["k"]
    geom = px.geometry(n, n, wl["pc"])
    ctx = px.Context(max_iter=wl["max_iter"], tol_deg=1e-3)
    master_d = torch.from_numpy(np.ascontiguousarray(wl["master"])).to(dev)
    libq_d = torch.from_numpy(wl["lib_q"]).to(dev)
    truth_d = torch.from_numpy(wl["truth_q"]).to(dev)
    pcs_d = torch.from_numpy(wl["pcs"]).to(dev)
    peak_d = torch.from_numpy(wl["peak"]).to(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(wl["noise_seed"])
    pats_d = torch.empty((P, n, n), device=dev)
    for c0 in range(0, P, 4096):
        c1 = min(P, c0 + 4096)
        clean = px.xcf_project(ctx, master_d, truth_d[c0:c1].contiguous(), geom, pcs=pcs_d[c0:c1].contiguous())
        pats_d[c0:c1] = _noisy_on_device(torch, clean, pcs_d[c0:c1], peak_d[c0:c1], gen)
    del clean
    outq = (torch.empty((P, 4), dtype=torch.float64, device=dev), torch.empty(P, device=dev),
            torch.empty(P, dtype=torch.int32, device=dev))
    res = {}

    best_d = torch.empty(P, dtype=torch.int32, device=dev)

    def step():
        lib = px.xcf.xcf_build_library_ex(ctx, libq_d, geom, master=master_d, flags=px.xcf.XCF_LIB_SCREEN)
        # screen top-k, FP32 rescore and refinement with one pre-processing of the patterns
        px.xcf_index_precision(ctx, lib, pats_d, pcs=pcs_d, k=k, out=(best_d, outq[0], outq[1], outq[2]))
        res["best"] = best_d
        lib.close()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    mis = px.xcf_disorientation(ctx, outq[0], truth_d)
    lib_mis = px.xcf_disorientation(ctx, libq_d[res["best"].clamp(min=0).long()].contiguous(), truth_d)
    accuracy = {"mean_misorientation_deg": float(mis.mean()), "median_misorientation_deg": float(mis.median()),
                "frac_below_1deg": float((mis < 1.0).double().mean()),
                "library_match_mean_deg": float(lib_mis.mean()), "iters_mean": float(outq[2].double().mean())}
    px.xcf_profile_read(ctx, reset=True)
    px.xcf_profile_enable(ctx, True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks_start(local)
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    torch.cuda.synchronize()
    clocks = clocks_stop(clk)
    elapsed_ms = ev0.elapsed_time(ev1)
    elapsed_ms = max_over_ranks(elapsed_ms, dist, dev)
    px.xcf_profile_enable(ctx, False)
    prof = px.xcf_profile_read(ctx, reset=True)
    pk = peaks_file() or {}
    tensor_peak = pk.get("bf16_tflops_sustained") or 1700.0
    s_ms, s_n = prof["screen"]
    flops_step = 2.0 * P * T * n * n
    achieved = flops_step * args.steps / (s_ms / 1e3) / 1e12
    screen_roof = {"bound": "tensor", "achieved": achieved, "peak": tensor_peak, "unit": "TFLOP/s",
                   "frac": achieved / tensor_peak, "traffic": None, "kernel": "k_screen_tc",
                   "peak_basis": "measured sustained cuBLAS BF16 (MEASURED_PEAKS.json)" if pk else "fallback",
                   "screen_ms_per_launch": s_ms / max(s_n, 1), "launches_per_step": s_n / args.steps}
    # the dominant stage: the FP32 FFT rescore of the k candidates (k_search_c256, candidate-list mode)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = pk.get("sm_max_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
    fp32_peak = sms * 128 * 2 * sm_max * 1e6 / 1e12
    r_ms = prof["search"][0] / args.steps
    r_ach = P * k * flops_per_pair(n) / (r_ms / 1e3) / 1e12
    stages = {kk: v[0] / args.steps for kk, v in prof.items()}
    roofline = {"bound": "alu", "achieved": r_ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": r_ach / fp32_peak,
                "traffic": None, "kernel": "k_search_c256w (rescore of the top-k candidates)",
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                "stage_share": r_ms / max(sum(stages.values()), 1e-9),
                "stage_ms_per_step": stages, "secondary": {"screen": screen_roof}}
    value = whole_job_rate(P, args.steps, world, elapsed_ms)
    e2e = None
    if not args.no_e2e:
        pats_h = pats_d.cpu().pin_memory()
        pcs_h = pcs_d.cpu().pin_memory()
        hout = (torch.empty(P, dtype=torch.int32, pin_memory=True), torch.empty((P, 4), dtype=torch.float64,
                pin_memory=True), torch.empty(P, pin_memory=True), torch.empty(P, dtype=torch.int32, pin_memory=True))

        def e2e_step():
            pats_d.copy_(pats_h, non_blocking=True)
            pcs_d.copy_(pcs_h, non_blocking=True)
            step()
            for h, o in zip(hout, (best_d, outq[0], outq[1], outq[2])):
                h.copy_(o, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": whole_job_rate(P, args.steps, world, dt * 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(pats_h.numel() * 4 + pcs_h.numel() * 8),
               "d2h_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hout)),
               "note": "patterns and PCs copied in from pinned host memory, outputs copied out, library built "
                       "on the device from the resident master, every step"}
        del pats_h
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        S = args.cpu_sample or oracle.num_threads()
        cpu = cpu_precision_rate(wl, pats_d[:S].cpu().numpy(), wl["pcs"][:S], P)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16 screen + f32 xcf", "data": "synthetic",
                "config": {"workload": wl["name"], "form": "precision", "detector": n, "templates": T,
                           "patterns_per_gpu": P, "top_k": k, "max_iter": wl["max_iter"],
                           "parallelism": f"replicas x{world}",
                           "l2": _l2_note(pats_d.numel() * 4, T * n * n * 2, "BF16 templates")},
                "accuracy": accuracy, "gpu_launches": int(sum(v[1] for v in prof.values())), "clocks": clocks,
                "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu}
        if emit:
            print(json.dumps(line), flush=True)
    else:
        line = None
    ctx.close()
    return line


# --------------------------------------------------------------- ndp form
def run_ndp(args, px, torch, dev, rank, world, local, dist):
    """NDP dictionary indexing (Eq. 1) of the plain form's map against the
    2.5 deg library, then the same refinement."""
    wl = synth.config_ndp_128(seed=rank, ny=args.map, nx=args.map)
    n, P, T, k = wl["n"], len(wl["truth_q"]), len(wl["lib_q"]), wl["k"]
    geom = px.geometry(n, n, wl["pc"])
    ctx = px.Context(max_iter=wl["max_iter"], tol_deg=1e-3)
    master_d = torch.from_numpy(np.ascontiguousarray(wl["master"])).to(dev)
    libq_d = torch.from_numpy(wl["lib_q"]).to(dev)
    truth_d = torch.from_numpy(wl["truth_q"]).to(dev)
    pcs_d = torch.from_numpy(wl["pcs"]).to(dev)
    clean = px.xcf_project(ctx, master_d, truth_d, geom, pcs=pcs_d).cpu().numpy()
    pats_d = torch.from_numpy(synth.add_noise(clean, wl["pcs"], wl["peak"], wl["noise_seed"])).to(dev)
    del clean
    outq = (torch.empty((P, 4), dtype=torch.float64, device=dev), torch.empty(P, device=dev),
            torch.empty(P, dtype=torch.int32, device=dev))
    res = {}

    def step():
        lib = px.xcf.xcf_build_library_ex(ctx, libq_d, geom, master=master_d,
                                          flags=px.XCF_LIB_NDP | px.XCF_LIB_NO_SPECTRA)
        best, ndp = px.xcf_index_ndp(ctx, lib, pats_d, k=k)
        px.xcf_refine_best(ctx, lib, pats_d, best, pcs=pcs_d, out=outq)
        res["best"], res["ndp"] = best, ndp
        lib.close()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    mis = px.xcf_disorientation(ctx, outq[0], truth_d)
    lib_mis = px.xcf_disorientation(ctx, libq_d[res["best"].clamp(min=0).long()].contiguous(), truth_d)
    accuracy = {"mean_misorientation_deg": float(mis.mean()), "median_misorientation_deg": float(mis.median()),
                "frac_below_1deg": float((mis < 1.0).double().mean()),
                "library_match_mean_deg": float(lib_mis.mean()), "iters_mean": float(outq[2].double().mean()),
                "ndp_mean": float(res["ndp"].mean())}
    px.xcf_profile_read(ctx, reset=True)
    px.xcf_profile_enable(ctx, True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks_start(local)
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    torch.cuda.synchronize()
    clocks = clocks_stop(clk)
    elapsed_ms = ev0.elapsed_time(ev1)
    elapsed_ms = max_over_ranks(elapsed_ms, dist, dev)
    px.xcf_profile_enable(ctx, False)
    prof = px.xcf_profile_read(ctx, reset=True)
    pk = peaks_file() or {}
    tensor_peak = pk.get("bf16_tflops_sustained") or 1700.0
    s_ms, s_n = prof["screen"]
    flops_step = 2.0 * P * T * n * n
    achieved = flops_step * args.steps / (s_ms / 1e3) / 1e12
    roofline = {"bound": "tensor", "achieved": achieved, "peak": tensor_peak, "unit": "TFLOP/s",
                "frac": achieved / tensor_peak, "traffic": None, "kernel": "k_screen_tc (NDP operands)",
                "peak_basis": "measured sustained cuBLAS BF16 (MEASURED_PEAKS.json)" if pk else "fallback",
                "screen_ms_per_launch": s_ms / max(s_n, 1), "launches_per_step": s_n / args.steps,
                "stage_ms_per_step": {kk: v[0] / args.steps for kk, v in prof.items()}}
    value = whole_job_rate(P, args.steps, world, elapsed_ms)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16 ndp + f32 rescore / refinement",
                "data": "synthetic",
                "config": {"workload": wl["name"], "form": "ndp", "detector": n, "templates": T,
                           "patterns_per_gpu": P, "top_k": k, "max_iter": wl["max_iter"],
                           "parallelism": f"replicas x{world}",
                           "l2": _l2_note(pats_d.numel() * 4, T * n * n * 6, "FP32 + BF16 NDP templates")},
                "accuracy": accuracy, "gpu_launches": int(sum(v[1] for v in prof.values())), "clocks": clocks,
                "roofline": roofline, "e2e": None, "cpu_baseline": None}
        print(json.dumps(line), flush=True)
    ctx.close()


# -------------------------------------------------------------- fwhm form
FWHM_SIDES = (16, 32, 64, 128, 256)
FWHM_DPC = (-0.04, -0.02, 0.0, 0.02, 0.04)


def run_fwhm(args, px, torch, dev, rank, world, local, dist):
    """Figs. 3-4: rotation scans (+-45 deg in 0.5 deg steps about detector x,
    y, z) of a reference pattern at PC (0.5, 0.3, 0.6), NDP and FFT, for every
    screen side, and at 128 x 128 for PC errors along x, y and z; FWHMs
    averaged over four reference orientations.  One step = the whole sweep."""
    pc0 = (0.5, 0.3, 0.6)
    h, step_deg = 90, 0.5
    master = torch.from_numpy(np.ascontiguousarray(synth.master_pattern("bcc", 1024))).to(dev)
    qs = torch.from_numpy(synth.random_quaternions(4, 100 + rank)).to(dev)
    ctx = px.Context(sigma_hp=args.sigma_hp) if args.sigma_hp > 0 else px.Context()
    cases = [(n, None) for n in FWHM_SIDES]
    cases += [(128, (ax, d)) for ax in range(3) for d in FWHM_DPC if d != 0.0]
    pct = {}
    for n, e in cases:
        if e is not None:
            pc = list(pc0)
            pc[e[0]] += e[1]
            pct[e] = torch.tensor(pc, dtype=torch.float64, device=dev)
    out = {}

    def step():
        for n, e in cases:
            g = px.geometry(n, n, pc0)
            fws = []
            for i in range(qs.shape[0]):
                _, _, fw = px.xcf_rotation_scan(ctx, master, g, qs[i].contiguous(), h, step_deg,
                                                pc_test=pct[e] if e is not None else None)
                fws.append(fw)
            out[(n, e)] = torch.stack(fws)

    for _ in range(args.warmup):
        step()
    px.xcf_profile_read(ctx, reset=True)
    px.xcf_profile_enable(ctx, True)
    torch.cuda.synchronize()
    clk = clocks_start(local)
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    torch.cuda.synchronize()
    clocks = clocks_stop(clk)
    elapsed_ms = ev0.elapsed_time(ev1)
    px.xcf_profile_enable(ctx, False)
    prof = px.xcf_profile_read(ctx, reset=True)

    def summary(fw):
        """FWHM per (method, axis) for each reference orientation (-1: wider than the scan)"""
        f = fw.cpu().numpy()
        return {f"{m}_{ax}": [round(float(v), 1) for v in f[:, r, a]]
                for r, m in enumerate(("ndp", "fft")) for a, ax in enumerate("xyz")}

    table = {"screen_side": {str(n): summary(out[(n, None)]) for n in FWHM_SIDES},
             "pc_error_128": {f"d{'xyz'[a]}={d:+.2f}": summary(out[(128, (a, d))])
                              for a in range(3) for d in FWHM_DPC if d != 0.0}}
    images = sum((1 + 3 * (2 * h + 1)) * qs.shape[0] for _ in cases)
    if rank == 0:
        line = {"metric": "rotation-scan test patterns/s (FWHM experiments of Figs. 3-4)",
                "value": images * args.steps / (elapsed_ms / 1e3), "unit": "patterns/s", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"fwhm_scan_h{h}_step{step_deg}_pc{pc0}", "form": "fwhm",
                           "sigma_hp": ctx.options.sigma_hp,
                           "scans_per_step": len(cases) * qs.shape[0], "patterns_per_scan": 1 + 3 * (2 * h + 1)},
                "fwhm_deg": table, "gpu_launches": int(sum(v[1] for v in prof.values())), "clocks": clocks,
                "stage_ms_per_step": {kk: v[0] / args.steps for kk, v in prof.items()},
                "roofline": None, "e2e": None, "cpu_baseline": None}
        print(json.dumps(line), flush=True)
    ctx.close()


# --------------------------------------------------------------- net form
def run_net(args, px, torch, dev, rank, world, local, dist):
    """The proposal network's forward pass alone (the learned form's stage
    `net`): standardisation, five convolutions, pool, two fc layers on
    synthetic 128 x 128 images with seeded random weights.  One step = the
    forward of every image; BF16 tensor-core convolutions 2-5 unless --net-fp32."""
    n = args.patterns or 100000
    g = torch.Generator(device=dev).manual_seed(11 + rank)
    imgs = torch.rand((n, 128, 128), generator=g, device=dev, dtype=torch.float32)
    ctx = px.Context()
    net = px.xcf_net_create(ctx, 8, torch.from_numpy(synth.cnn_init_params(8, 3)).to(dev))
    net.set_bf16(not args.net_fp32)
    for _ in range(args.warmup):
        out = px.xcf_net_forward(ctx, net, imgs)
    px.xcf_profile_read(ctx, reset=True)
    px.xcf_profile_enable(ctx, True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks_start(local)
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        out = px.xcf_net_forward(ctx, net, imgs)
    ev1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clocks_stop(clk)
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    px.xcf_profile_enable(ctx, False)
    prof = px.xcf_profile_read(ctx, reset=True)
    pk = peaks_file()
    if args.net_fp32:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_max = (pk or {}).get("sm_max_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
        peak, bound, basis = sms * 128 * 2 * sm_max * 1e6 / 1e12, "alu", "152 SMs x 128 FP32 lanes x 2 x clock"
        kern = "proposal network forward (k_gemm, FP32)"
    else:
        peak, bound = (pk or {}).get("bf16_tflops_sustained") or 1700.0, "tensor"
        basis = "measured sustained cuBLAS BF16 (MEASURED_PEAKS.json)" if pk else "fallback"
        kern = "proposal network forward (convolution 1 direct FP32 -> BF16; 2-5 k_conv_tc implicit GEMM, tcgen05 BF16)"
    achieved = CNN_FORWARD_FLOPS * n * args.steps / (elapsed_ms / 1e3) / 1e12
    if rank == 0:
        line = {"metric": "proposal network forward images/s", "value": whole_job_rate(n, args.steps, world, elapsed_ms),
                "unit": "images/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.net_fp32 else "bf16 convolutions 2-5 + f32",
                "data": "synthetic",
                "config": {"workload": f"net128_k8_B{n}", "form": "net", "images_per_gpu": n,
                           "parallelism": f"replicas x{world}",
                           "l2": f"inputs larger than L2 ({n * 128 * 128 * 4 / 1e6:.0f} MB images; L2 129 MB)"},
                "checksum": float(out.double().abs().sum()),
                "gpu_launches": int(sum(v[1] for v in prof.values())), "clocks": clocks,
                "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": None, "kernel": kern, "peak_basis": basis},
                "stage_ms_per_step": {kk: v[0] / args.steps for kk, v in prof.items()},
                "e2e": None, "cpu_baseline": None}
        print(json.dumps(line), flush=True)
    net.close()
    ctx.close()


# --------------------------------------------------------------- so3 form
SO3_STEPS = (10.0, 7.5, 5.0, 3.5, 2.5)


def run_so3(args, px, torch, dev, rank, world, local, dist):
    """Fig. 2: for each sampling frequency, generate the library (S^2 x S^1
    grid in the cubic zone, symmetry copies dropped), every member's
    disorientation to its nearest other member (max / mean / median / mode
    of the distribution) and the coverage of 100,000 random orientations.
    One step = the whole sweep."""
    ctx = px.Context()
    rnd = torch.from_numpy(synth.random_quaternions(100000, 300 + rank)).to(dev)
    res = {}

    def step():
        for sf in SO3_STEPS:
            g = px.xcf_so3_grid(ctx, sf)
            nn, _ = px.xcf_nearest_disorientation(ctx, g)
            cov, _ = px.xcf_nearest_disorientation(ctx, rnd, g)
            res[sf] = (g.shape[0], nn, cov)

    for _ in range(args.warmup):
        step()
    px.xcf_profile_read(ctx, reset=True)
    px.xcf_profile_enable(ctx, True)
    torch.cuda.synchronize()
    clk = clocks_start(local)
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    torch.cuda.synchronize()
    clocks = clocks_stop(clk)
    elapsed_ms = ev0.elapsed_time(ev1)
    px.xcf_profile_enable(ctx, False)
    prof = px.xcf_profile_read(ctx, reset=True)
    table, pairs = {}, 0
    for sf, (T, nn, cov) in res.items():
        a = nn.cpu().numpy()
        h, e = np.histogram(a, bins=np.arange(0.0, sf + 0.5, 0.1))
        c = cov.cpu().numpy()
        table[str(sf)] = {"orientations": int(T), "nn_max": round(float(a.max()), 3),
                          "nn_mean": round(float(a.mean()), 3), "nn_median": round(float(np.median(a)), 3),
                          "nn_mode_bin": round(float(e[h.argmax()]), 1),
                          "nn_frac_below_0.9sf": round(float(np.mean(a < 0.9 * sf)), 3),
                          "cover_max": round(float(c.max()), 3), "cover_mean": round(float(c.mean()), 3)}
        pairs += T * T + rnd.shape[0] * T
    if rank == 0:
        line = {"metric": "orientation pairs compared/s (SO(3) sampling study of Fig. 2)",
                "value": pairs * args.steps / (elapsed_ms / 1e3), "unit": "pairs/s", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 rank + f64 angle",
                "data": "synthetic",
                "config": {"workload": "so3_study_" + "_".join(str(x) for x in SO3_STEPS), "form": "so3",
                           "random_orientations": int(rnd.shape[0])},
                "so3": table, "gpu_launches": int(sum(v[1] for v in prof.values())), "clocks": clocks,
                "stage_ms_per_step": {kk: v[0] / args.steps for kk, v in prof.items()},
                "roofline": None, "e2e": None, "cpu_baseline": None}
        print(json.dumps(line), flush=True)
    ctx.close()


# ----------------------------------------------------------- batched form
def flops_per_pair(n: int) -> float:
    """Inverse real FFT of one n x n surface + conj-multiply of a half spectrum."""
    import math
    return 2.5 * n * n * math.log2(n * n) + 6 * n * (n // 2 + 1)


def cpu_batched_rate(wl, pats_list, crop_ns, native=False, t_sub=256):
    """The FP64 oracle on a bounded sample of the batched workload: per map,
    the library build and the search (pre-processing, every pair's surface,
    best template, sub-pixel peak) against t_sub evenly spaced templates of its
    library (both linear in the template count, scaled to the whole library),
    on one sample pattern per core; the maps' times are added."""
    import oracle
    threads = oracle.num_threads()
    total, P_all, parts = 0.0, 0, []
    for m, pats, n in zip(wl["maps"], pats_list, crop_ns):
        T, P = len(m["lib_q"]), len(m["truth_q"])
        W, H = m["W"], m["H"]
        _, ox, oy, pcc = oracle.crop(W, H, wl["pc"], native=native)
        sub = np.linspace(0, T - 1, min(T, t_sub)).astype(np.int64)
        t0 = time.perf_counter()
        St, _, _ = oracle.prep_many(oracle.project_many(wl["master"], m["lib_q"][sub], pcc, n))
        t_lib = (time.perf_counter() - t0) * T / len(sub)
        S = min(threads, len(pats))
        t0 = time.perf_counter()
        Sp, _, deg = oracle.prep_many(pats[:S, oy:oy + n, ox:ox + n])
        oracle.index(St, Sp, deg)
        t_s = (time.perf_counter() - t0) * T / len(sub)
        total += t_lib + P * t_s / S
        P_all += P
        parts.append(f"{W}px/{n} T{T} P{P}: lib {t_lib:.1f} s, {P * t_s / S:.1f} s search")
    sample = (f"per map, {threads} sample patterns searched against {t_sub} evenly spaced templates and the "
              f"library build of those templates, both scaled to the whole library: " + "; ".join(parts))
    return {"value": P_all / total, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}


def run_batched(args, px, torch, dev, rank, world, local, dist, emit=True):
    wl = synth.config_batched(seed=rank, scale=args.scale)
    ctx = px.Context(native_sizes=int(args.native))
    master_d = torch.from_numpy(np.ascontiguousarray(wl["master"])).to(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(wl["noise_seed"])
    batch, truths, libqs, hosts, ns, flops = [], [], [], [], [], 0.0
    for m in wl["maps"]:
        g = px.geometry(m["W"], m["H"], wl["pc"])
        libq = torch.from_numpy(m["lib_q"]).to(dev)
        lib = px.xcf_build_library(ctx, master_d, libq, g)
        truth = torch.from_numpy(m["truth_q"]).to(dev)
        pcs = torch.from_numpy(m["pcs"]).to(dev)
        peak = torch.from_numpy(m["peak"]).to(dev)
        P = truth.shape[0]
        pats = torch.empty((P, m["H"], m["W"]), device=dev)
        for c0 in range(0, P, 2048):
            c1 = min(P, c0 + 2048)
            clean = px.xcf_project(ctx, master_d, truth[c0:c1].contiguous(), g, pcs=pcs[c0:c1].contiguous())
            pats[c0:c1] = _noisy_on_device(torch, clean, pcs[c0:c1], peak[c0:c1], gen)
        batch.append((lib, pats))
        truths.append(truth)
        libqs.append(libq)
        n = px.xcf_crop(g, native=args.native)[0]
        ns.append(n)
        flops += P * lib.T * flops_per_pair(n)   # every (pattern, template) pair
    P_all = sum(p.shape[0] for _, p in batch)
    outs = px.xcf_index_maps(ctx, batch, graph=True)          # first call: tune + capture
    for _ in range(args.warmup):
        px.xcf_index_maps(ctx, batch, outs=outs, graph=True)
    torch.cuda.synchronize()
    lib_mis = torch.cat([px.xcf_disorientation(ctx, libq[o[0].clamp(min=0).long()].contiguous(), t)
                         for libq, o, t in zip(libqs, outs, truths)])
    accuracy = {"library_match_mean_deg": float(lib_mis.mean()),
                "library_match_median_deg": float(lib_mis.median()),
                "frac_below_library_step": float(sum(
                    (px.xcf_disorientation(ctx, libq[o[0].clamp(min=0).long()].contiguous(), t) < m["step"])
                    .double().sum() for libq, o, t, m in zip(libqs, outs, truths, wl["maps"])) / P_all)}

    def timed(fn):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ms = max_over_ranks(ms, dist, dev)
        return ms

    px.xcf_profile_read(ctx, reset=True)
    px.xcf_profile_enable(ctx, True)
    clk = clocks_start(local)
    time.sleep(0.3)
    elapsed_ms = timed(lambda: px.xcf_index_maps(ctx, batch, outs=outs, graph=True))
    clocks = clocks_stop(clk)
    prof = px.xcf_profile_read(ctx, reset=True)
    launches = int(sum(v[1] for v in prof.values()))
    # the same maps one after another through the per-map entry point, for comparison
    seq_ms = timed(lambda: [px.xcf_index(ctx, lib, pats) for lib, pats in batch])
    px.xcf_profile_read(ctx, reset=True)
    # the search kernel alone (uncaptured calls time each stage)
    for _ in range(2):
        px.xcf_index_maps(ctx, batch, outs=outs)
    torch.cuda.synchronize()
    prof2 = px.xcf_profile_read(ctx, reset=True)
    px.xcf_profile_enable(ctx, False)
    # one call launches the queue kernel (128 x 128 maps) and one search kernel
    # per map of another side: the stage time per call covers all of them
    search_ms_call = prof2["search"][0] / 2
    # per-map search time through the per-map entry point (its own kernel per side)
    by_side = {}
    for (lib, pats), n in zip(batch, ns):
        px.xcf_profile_enable(ctx, True)
        px.xcf_index(ctx, lib, pats)
        torch.cuda.synchronize()
        ms_map = px.xcf_profile_read(ctx, reset=True)["search"][0]
        px.xcf_profile_enable(ctx, False)
        d = by_side.setdefault(str(n), {"ms": 0.0, "tflop": 0.0})
        d["ms"] += ms_map
        d["tflop"] += pats.shape[0] * lib.T * flops_per_pair(n) / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    pk = peaks_file()
    sm_max = (pk or {}).get("sm_max_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
    fp32_peak = sms * 128 * 2 * sm_max * 1e6 / 1e12
    for d in by_side.values():
        d["achieved_tflops"] = d["tflop"] / (d["ms"] / 1e3)
        d["frac"] = d["achieved_tflops"] / fp32_peak
    achieved = flops / (search_ms_call / 1e3) / 1e12
    kernels = {16: "k_search_maps", 32: "k_search_maps", 64: "k_search_maps", 96: "k_search_maps",
               128: "k_search_maps", 160: "k_search_maps", 200: "k_search_n200", 256: "k_search_c256w"}
    body_names = {0: "warp lines (R x 32)", 1: "three rounds (16x8 | 4x32)", 2: "radix-2 in shared memory",
                  3: "eight-lane groups (8 x 8)"}
    tuning = {}
    for (lib, _), n in zip(batch, ns):
        t = px.xcf_maps_get_tuning(ctx, n, lib.T)
        if t is not None:
            tuning[f"{n}px_T{lib.T}"] = {"body": body_names.get(t[0], t[0]), "patterns_per_cta": t[1],
                                         "pairs_per_item": t[2], "pairs_total": (lib.T + 1) // 2}
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": None,
                "kernel": "search stage of one call: " + " + ".join(sorted({kernels[n] for n in ns})),
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                "search_ms_per_call": search_ms_call,
                "autotuned": tuning,
                "by_side_per_map_calls": by_side,
                "stage_ms_per_step_uncaptured": {k: v[0] / 2 for k, v in prof2.items()}}
    e2e = None
    if not args.no_e2e:
        hp = [p.cpu().pin_memory() for _, p in batch]
        ho = [tuple(torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in o) for o in outs]

        def e2e_step():
            for (lib, pats), h in zip(batch, hp):
                pats.copy_(h, non_blocking=True)
            px.xcf_index_maps(ctx, batch, outs=outs, graph=True)
            for o, h in zip(outs, ho):
                for a, b in zip(h, o):
                    a.copy_(b, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": whole_job_rate(P_all, args.steps, world, dt * 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(h.numel() * 4 for h in hp)),
               "d2h_bytes_per_step": int(sum(a.numel() * a.element_size() for h in ho for a in h))}
    value = whole_job_rate(P_all, args.steps, world, elapsed_ms)
    if rank == 0:
        line = {"metric": "patterns indexed/s (batched maps: prep + search + peak per map)", "value": value,
                "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl["name"] + ("_native" if args.native else ""), "form": "batched",
                           "crop_rule": "native (16..256 incl. 96, 160)" if args.native else "2^k",
                           "maps": len(batch),
                           "detectors": [[m["W"], m["H"]] for m in wl["maps"]], "crop": ns,
                           "templates": [lib.T for lib, _ in batch], "patterns": [p.shape[0] for _, p in batch],
                           "graph": True, "libraries": "resident (built before the timed region)",
                           "parallelism": f"replicas x{world}",
                           "l2": _l2_note(sum(p.numel() * 4 for _, p in batch),
                                          sum(lib.T * n * (n // 2 + 1) * 8 for (lib, _), n in zip(batch, ns)),
                                          "library spectra")},
                "sequential_ms_per_step": seq_ms / args.steps,
                "accuracy": accuracy, "gpu_launches": launches, "clocks": clocks, "roofline": roofline,
                "e2e": e2e, "cpu_baseline": None}
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            S = oracle.num_threads()
            line["cpu_baseline"] = cpu_batched_rate(wl, [p[:S].cpu().numpy() for _, p in batch], ns, args.native)
        if emit:
            print(json.dumps(line), flush=True)
    else:
        line = None
    for lib, _ in batch:
        lib.close()
    ctx.close()
    return line


# ----------------------------------------------------------- learned form
def _generate(px, torch, ctx, master_d, geom, q, pcs, peak, gen, chunk=4096):
    """Noisy patterns [P, n, n] on the device from orientations / PCs / peaks (input generation)."""
    P = q.shape[0]
    out = torch.empty((P, geom.height, geom.width), device=q.device)
    for c0 in range(0, P, chunk):
        c1 = min(P, c0 + chunk)
        clean = px.xcf_project(ctx, master_d, q[c0:c1].contiguous(), geom, pcs=pcs[c0:c1].contiguous())
        out[c0:c1] = _noisy_on_device(torch, clean, pcs[c0:c1], peak[c0:c1], gen)
    return out


# forward multiply-adds of the proposal network per pattern x 2: five 3 x 3
# stride-2 convolutions (1-32-64-64-128-128 channels, outputs 64^2 .. 4^2) and two fc layers
CNN_FORWARD_FLOPS = 2.0 * (sum(co * ci * 9 * s * s for ci, co, s in
                               ((1, 32, 64), (32, 64, 32), (64, 64, 16), (64, 128, 8), (128, 128, 4)))
                           + 256 * 128 + 48 * 256)


def cpu_learned_rate(wl, params, pats, pcs, fb_frac, P_total, tau):
    """The FP64 oracle on a bounded sample of the learned workload: the
    network's forward pass (BF16 form, the trained parameters) on the
    standardised centred crops, the k proposals projected, pre-processed and
    correlated with the pattern, refinement from the best proposal; patterns
    whose refined peak stays below tau take the full search + refinement,
    counted at the GPU run's fallback fraction and timed on two patterns
    (library build amortised over the map)."""
    import oracle
    n, k = wl["n"], wl["k"]
    threads = oracle.num_threads()
    S = len(pats)
    t0 = time.perf_counter()
    x = np.stack([oracle.cnn_standardise(p) for p in pats])
    props = oracle.cnn_proposals(oracle.cnn_forward_bf16(params, x, k), k)
    t_net = time.perf_counter() - t0
    t0 = time.perf_counter()
    Sp, _, deg = oracle.prep_many(pats)
    tm = oracle.project_many(wl["master"], props.reshape(-1, 4), np.repeat(pcs, k, axis=0), n)
    St, _, _ = oracle.prep_many(tm)
    seeds = np.empty((S, 4))
    for p in range(S):
        b = oracle.index(St[p * k:(p + 1) * k], Sp[p:p + 1], deg[p:p + 1])[0][0]
        seeds[p] = props[p, max(0, int(b))]
    t_score = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.refine_many(wl["master"], pats, seeds, pcs, max_it=wl["max_iter"], tol_deg=1e-3)
    t_refine = time.perf_counter() - t0
    t0 = time.perf_counter()
    Sl, _, _ = oracle.prep_many(oracle.project_many(wl["master"], wl["lib_q"], wl["pc"], n))
    t_lib = time.perf_counter() - t0
    t0 = time.perf_counter()
    b, _, _, _ = oracle.index(Sl, Sp[:2], deg[:2])
    oracle.refine_many(wl["master"], pats[:2], wl["lib_q"][np.maximum(b, 0)], pcs[:2], max_it=wl["max_iter"],
                       tol_deg=1e-3)
    t_full = (time.perf_counter() - t0) / 2 * min(2, threads) / threads
    per = (t_net + t_score + t_refine) / S + fb_frac * t_full + t_lib / P_total
    sample = (f"{S} of the {P_total} test patterns: network forward ({t_net:.1f} s), {k} proposals projected, "
              f"pre-processed and correlated ({t_score:.1f} s), refinement ({t_refine:.1f} s); the full-search "
              f"fallback at the GPU run's fraction {fb_frac:.4f}, timed on 2 patterns; library build ({t_lib:.1f} s) "
              f"amortised over {P_total}; training not included (set-up)")
    return {"value": 1.0 / per, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}


def run_learned(args, px, torch, dev, rank, world, local, dist, emit=True):
    n_test = args.patterns or 100000
    wl = synth.config_learned_128(seed=rank, n_train=args.train, n_test=n_test)
    n, k = wl["n"], wl["k"]
    geom = px.geometry(n, n, wl["pc"])
    ctx = px.Context(max_iter=wl["max_iter"], tol_deg=1e-3)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    master_d, libq_d = d(wl["master"]), d(wl["lib_q"])
    gen = torch.Generator(device=dev)
    gen.manual_seed(wl["noise_seed"])
    # ---- training (setup, outside the timed region): passes over the generated training set
    # (fresh Poisson noise each pass)
    net = px.xcf_net_create(ctx, k, d(synth.cnn_init_params(k, rank)))
    trq, trpc, trpk = d(wl["train_q"]), d(wl["train_pcs"]), d(wl["train_peak"])
    B, n_train = args.batch, len(wl["train_q"])
    per_epoch = max(1, n_train // B)
    steps = per_epoch * args.epochs
    t0 = time.perf_counter()
    losses = []
    for i in range(steps):
        j = i % per_epoch
        sl = slice(j * B, (j + 1) * B)
        imgs = _generate(px, torch, ctx, master_d, geom, trq[sl], trpc[sl], trpk[sl], gen)
        loss, _, _ = px.xcf_net_loss_grad(ctx, net, imgs, trq[sl].contiguous(), geom)
        lr = args.lr * 0.5 * (1.0 + np.cos(np.pi * i / steps))          # cosine schedule
        px.xcf_net_adam(ctx, net, lr=float(lr))
        if i % 50 == 0 or i == steps - 1:
            losses.append(float(loss))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # inference precision of the network (training above ran in FP32)
    net.set_bf16(not args.net_fp32)
    # ---- test set, resident on the device
    teq, tepc, tepk = d(wl["test_q"]), d(wl["test_pcs"]), d(wl["test_peak"])
    pats = _generate(px, torch, ctx, master_d, geom, teq, tepc, tepk, gen)
    lib = px.xcf_build_library(ctx, master_d, libq_d, geom)
    # ---- fallback threshold from separate calibration patterns: the learned path without
    # fallback; tau = the lowest refined peak above which at most 0.5 % of patterns are off by > 1 deg
    caq, capc, capk = d(wl["cal_q"]), d(wl["cal_pcs"]), d(wl["cal_peak"])
    cpats = _generate(px, torch, ctx, master_d, geom, caq, capc, capk, gen)
    cq, cpk, _, _ = px.xcf_index_learned(ctx, net, lib, cpats, pcs=capc, tau=float("-inf"))
    cmis = px.xcf_disorientation(ctx, cq, caq)
    order = torch.argsort(cpk, descending=True)
    wrong = (cmis[order] > 1.0).double().cumsum(0) / torch.arange(1, len(order) + 1, device=dev)
    okpos = torch.nonzero(wrong <= 0.005).flatten()
    tau = float(cpk[order][okpos.max()]) if okpos.numel() else float("inf")
    cal_accept = float((okpos.max() + 1) / len(order)) if okpos.numel() else 0.0
    ncal = min(2000, n_test)
    outs = (torch.empty((n_test, 4), dtype=torch.float64, device=dev), torch.empty(n_test, device=dev),
            torch.empty(n_test, dtype=torch.int32, device=dev), torch.empty(n_test, dtype=torch.int32, device=dev))

    def step():
        px.xcf_index_learned(ctx, net, lib, pats, pcs=tepc, tau=tau, out=outs)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    px.xcf_profile_read(ctx, reset=True)
    px.xcf_profile_enable(ctx, True)
    if dist:
        dist.barrier()
    clk = clocks_start(local)
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clocks = clocks_stop(clk)
    elapsed_ms = e0.elapsed_time(e1)
    px.xcf_profile_enable(ctx, False)
    prof = px.xcf_profile_read(ctx, reset=True)
    elapsed_ms = max_over_ranks(elapsed_ms, dist, dev)
    mis = px.xcf_disorientation(ctx, outs[0], teq)
    fb = outs[3].double()
    # ---- ablation: the plain full search + refinement on the same test set, and the raw proposals
    e0.record()
    full = px.xcf_index_refine(ctx, lib, pats, pcs=tepc)
    e1.record()
    torch.cuda.synchronize()
    full_ms = e0.elapsed_time(e1)
    mis_full = px.xcf_disorientation(ctx, full["quats"], teq)
    prop = px.xcf_propose(ctx, net, pats[:ncal].contiguous(), geom)
    best_prop = torch.stack([px.xcf_disorientation(ctx, prop[:, h].contiguous(), teq[:ncal].contiguous())
                             for h in range(k)]).min(dim=0).values
    value = whole_job_rate(n_test, args.steps, world, elapsed_ms)
    pk = peaks_file()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = (pk or {}).get("sm_max_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
    fp32_peak = sms * 128 * 2 * sm_max * 1e6 / 1e12
    net_ms, net_n = prof["net"]
    net_flops = CNN_FORWARD_FLOPS * n_test * args.steps
    if args.net_fp32:
        net_peak, bound, kern, basis = fp32_peak, "alu", "proposal network forward (k_gemm, FP32)", "FP32 ALU"
    else:
        net_peak = (pk or {}).get("bf16_tflops_sustained") or 1700.0
        bound, kern = "tensor", "proposal network forward (convolution 1 direct FP32 -> BF16; 2-5 k_conv_tc implicit GEMM, tcgen05 BF16)"
        basis = "measured sustained cuBLAS BF16 (MEASURED_PEAKS.json)" if pk else "fallback"
    roofline = {"bound": bound, "achieved": net_flops / (net_ms / 1e3) / 1e12 if net_ms else None, "peak": net_peak,
                "unit": "TFLOP/s", "kernel": kern, "peak_basis": basis, "traffic": None,
                "stage_ms_per_step": {kk: v[0] / args.steps for kk, v in prof.items()}}
    roofline["frac"] = roofline["achieved"] / net_peak if roofline["achieved"] else None
    net_roof = roofline
    # the dominant stage: pre-processing (k_prep_real).  Timed alone on the step's own test patterns (spectra
    # and filtered images, as the learned path takes them); algorithmic bytes: the image in, the half spectrum
    # and the filtered image out
    stages = {kk: v[0] / args.steps for kk, v in prof.items()}
    px.xcf_prep(ctx, pats, geom, want_spatial=True)            # warm-up (output buffers)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(3):
        px.xcf_prep(ctx, pats, geom, want_spatial=True)
    e1.record()
    torch.cuda.synchronize()
    prep_ms = e0.elapsed_time(e1) / 3
    prep_bytes = n_test * (4 * n * n + 8 * n * (n // 2 + 1) + 4 * n * n)
    hbm = (pk or {}).get("hbm_gbs") or 6800.0
    roofline = {"bound": "hbm", "achieved": prep_bytes / (prep_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                "traffic": None, "kernel": "k_prep_real (pre-processing: crop, statistics, window, FFT, band-pass, "
                "norm, filtered image)", "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)" if pk else
                "fallback", "timed": f"alone on the {n_test} test patterns, {prep_ms:.2f} ms per launch",
                "stage_share": stages.get("prep", 0.0) / max(sum(stages.values()), 1e-9),
                "stage_ms_per_step": stages, "secondary": {"network": net_roof}}
    roofline["frac"] = roofline["achieved"] / hbm
    e2e = None
    if not args.no_e2e:
        pats_h = pats.cpu().pin_memory()
        pcs_h = tepc.cpu().pin_memory()
        hout = tuple(torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in outs)

        def e2e_step():
            pats.copy_(pats_h, non_blocking=True)
            tepc.copy_(pcs_h, non_blocking=True)
            step()
            for h, o in zip(hout, outs):
                h.copy_(o, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": whole_job_rate(n_test, args.steps, world, dt * 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(pats_h.numel() * 4 + pcs_h.numel() * 8),
               "d2h_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hout)),
               "note": "test patterns and PCs copied in from pinned host memory, outputs copied out, every step"}
        del pats_h
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        S = args.cpu_sample or oracle.num_threads()
        cpu = cpu_learned_rate(wl, net.params().cpu().numpy(), pats[:S].cpu().numpy(), wl["test_pcs"][:S],
                               float(fb.mean()), n_test, tau)
    if rank == 0:
        line = {"metric": "patterns indexed/s (learned proposals + correlation score + refinement, full-search fallback)",
                "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.net_fp32 else "bf16 network + f32 xcf",
                "data": "synthetic",
                "config": {"workload": wl["name"], "form": "learned", "detector": n, "templates": lib.T, "heads": k,
                           "network_inference": "fp32" if args.net_fp32 else "bf16", "train_patterns": n_train, "epochs": args.epochs, "batch": B, "test_patterns": n_test,
                           "tau": tau, "calibration_patterns": len(wl["cal_q"]),
                           "calibration_accepted_fraction": cal_accept,
                           "parallelism": f"replicas x{world}",
                           "l2": _l2_note(pats.numel() * 4, lib.T * n * (n // 2 + 1) * 8, "library spectra")},
                "training": {"seconds": t_train, "steps": steps, "loss_trace": losses},
                "accuracy": {"mean_misorientation_deg": float(mis.mean()),
                             "median_misorientation_deg": float(mis.median()),
                             "frac_below_1deg": float((mis < 1.0).double().mean()),
                             "fallback_fraction": float(fb.mean())},
                "ablation": {"full_search_patterns_per_s": n_test / (full_ms / 1e3),
                             "full_search_mean_misorientation_deg": float(mis_full.mean()),
                             "full_search_frac_below_1deg": float((mis_full < 1.0).double().mean()),
                             "best_proposal_median_deg": float(best_prop.median()),
                             "best_proposal_frac_below_5deg": float((best_prop < 5.0).double().mean()),
                             "speedup_vs_full_search": value / (n_test / (full_ms / 1e3))},
                "gpu_launches": int(sum(v[1] for v in prof.values())), "clocks": clocks, "roofline": roofline,
                "e2e": e2e, "cpu_baseline": cpu}
        if emit:
            print(json.dumps(line), flush=True)
    else:
        line = None
    lib.close()
    net.close()
    ctx.close()
    return line


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import paper_1807_11313_gb300 as px
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    if args.form in ("precision", "batched", "learned", "ndp", "fwhm", "so3", "net"):
        fn = {"precision": run_precision, "batched": run_batched, "learned": run_learned, "ndp": run_ndp,
              "fwhm": run_fwhm, "so3": run_so3, "net": run_net}[args.form]
        fn(args, px, torch, dev, rank, world, local, dist)
        if dist:
            dist.destroy_process_group()
        return

    # ---- inputs (each rank its own map: weak scaling)
    wl = synth.config_map_128(seed=rank, ny=args.map, nx=args.map)
    n, P, T = wl["n"], len(wl["truth_q"]), len(wl["lib_q"])
    geom = px.geometry(n, n, wl["pc"])
    ctx = px.Context(max_iter=wl["max_iter"], tol_deg=1e-3, upsample=args.upsample)
    master_d = torch.from_numpy(np.ascontiguousarray(wl["master"])).to(dev)
    libq_d = torch.from_numpy(wl["lib_q"]).to(dev)
    truth_d = torch.from_numpy(wl["truth_q"]).to(dev)
    pcs_d = torch.from_numpy(wl["pcs"]).to(dev)
    clean = px.xcf_project(ctx, master_d, truth_d, geom, pcs=pcs_d).cpu().numpy()
    pats_np = synth.add_noise(clean, wl["pcs"], wl["peak"], wl["noise_seed"])
    del clean
    pats_d = torch.from_numpy(pats_np).to(dev)
    out = dict(best=torch.empty(P, dtype=torch.int32, device=dev), peak=torch.empty(P, device=dev),
               shift=torch.empty((P, 2), device=dev), quats=torch.empty((P, 4), dtype=torch.float64, device=dev),
               rpeak=torch.empty(P, device=dev), iters=torch.empty(P, dtype=torch.int32, device=dev))

    def step():
        lib = px.xcf_build_library(ctx, master_d, libq_d, geom)
        px.xcf_index_refine(ctx, lib, pats_d, pcs=pcs_d, out=out)
        lib.close()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    mis = px.xcf_disorientation(ctx, out["quats"], truth_d)
    best_np = out["best"].cpu().numpy()
    lib_mis = px.xcf_disorientation(ctx, libq_d[out["best"].clamp(min=0).long()].contiguous(), truth_d)
    accuracy = {"mean_misorientation_deg": float(mis.mean()), "median_misorientation_deg": float(mis.median()),
                "frac_below_1deg": float((mis < 1.0).double().mean()),
                "library_match_mean_deg": float(lib_mis.mean()), "iters_mean": float(out["iters"].double().mean()),
                "degenerate": int((best_np < 0).sum())}

    # ---- timed region
    px.xcf_profile_read(ctx, reset=True)
    px.xcf_profile_enable(ctx, True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks_start(local)
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    torch.cuda.synchronize()
    clocks = clocks_stop(clk)
    if dist:
        dist.barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    elapsed_ms = max_over_ranks(elapsed_ms, dist, dev)
    px.xcf_profile_enable(ctx, False)
    prof = px.xcf_profile_read(ctx, reset=True)
    launches = int(sum(v[1] for v in prof.values()))
    value = whole_job_rate(P, args.steps, world, elapsed_ms)

    # ---- roofline of the dominant kernel (the all-pairs search)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    pk = peaks_file()
    sm_max = (pk or {}).get("sm_max_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
    fp32_peak = sms * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s, FMA = 2 flops
    s_ms, s_n = prof["search"]
    per_launch_ms = s_ms / max(s_n, 1)
    flops_launch = P * T * FLOPS_PER_PAIR_128                 # one launch covers the whole map
    achieved = flops_launch / (per_launch_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak,
                "traffic": _roofline_traffic("search128_traffic.json", SEARCH128_SOURCES),
                "kernel": "k_search128", "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                "search_ms_per_launch": per_launch_ms,
                "stage_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()}}
    fma_tflops, _ = px.xcf_fp32_fma_rate(ctx)                 # measured FMA rate, beside the derived peak
    roofline["fma_probe_tflops"] = fma_tflops
    roofline["frac_of_fma_probe"] = achieved / fma_tflops

    # ---- end to end through the host-memory entry point
    e2e = None
    if not args.no_e2e:
        pats_h = torch.from_numpy(pats_np).pin_memory()
        pcs_h = torch.from_numpy(wl["pcs"]).pin_memory()
        master_h = torch.from_numpy(np.ascontiguousarray(wl["master"])).pin_memory()
        libq_h = torch.from_numpy(wl["lib_q"]).pin_memory()
        hout = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in out.items()}

        def e2e_step():
            m = master_h.to(dev, non_blocking=True)
            q = libq_h.to(dev, non_blocking=True)
            lib = px.xcf_build_library(ctx, m, q, geom)
            px.xcf_index_refine_host(ctx, lib, pats_h, pcs=pcs_h, out=hout)
            lib.close()

        e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, dist, dev)
        h2d = pats_h.numel() * 4 + pcs_h.numel() * 8 + master_h.numel() * 4 + libq_h.numel() * 8
        d2h = sum(v.numel() * v.element_size() for v in hout.values())
        e2e = {"value": whole_job_rate(P, args.steps, world, dt * 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    # ---- CPU oracle baseline (rank 0, one GPU only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        sample = args.cpu_sample or max(2 * oracle.num_threads(), 16)
        rate, threads, t_lib, t_s = cpu_oracle_rate(wl, pats_np, sample)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": (f"{sample} of the {P} patterns: full {T}-template search + refinement "
                          f"(<= {wl['max_iter']} iterations) in {t_s:.1f} s; library build ({t_lib:.1f} s) "
                          f"amortised over {P}")}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl["name"], "detector": n, "templates": T, "patterns_per_gpu": P,
                           "max_iter": wl["max_iter"], "parallelism": f"replicas x{world}",
                           "subpixel": f"up-sampled, step 1/{args.upsample} px" if args.upsample else "3-point parabola",
                           "l2": _l2_note(pats_d.numel() * 4, T * n * (n // 2 + 1) * 8, "library spectra")},
                "accuracy": accuracy, "gpu_launches": launches, "clocks": clocks, "roofline": roofline,
                "e2e": e2e, "cpu_baseline": cpu}
    if world == 1 and not args.no_forms:
        del pats_d, out
        ctx.close()
        torch.cuda.empty_cache()
        line["forms"] = run_forms(args, px, torch, dev, rank, world, local, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


FORM_KEYS = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config", "accuracy", "ablation",
             "training", "sequential_ms_per_step", "gpu_launches", "clocks", "roofline", "e2e", "cpu_baseline")


def run_forms(args, px, torch, dev, rank, world, local, dist):
    """The other forms of the indexer, each on its own workload, measured in
    the same run as the plain form (one GPU): each a sub-record with its
    throughput, the roofline of the stage that dominates its step, an end to
    end number (host buffers, copies in the timed region) and the oracle on
    a bounded sample."""
    forms = {}
    for name, fn in (("precision", run_precision), ("batched", run_batched), ("learned", run_learned)):
        sub = argparse.Namespace(**vars(args))
        sub.form, sub.steps, sub.warmup = name, max(1, args.form_steps), max(3, min(args.warmup, 3))
        sub.patterns, sub.scale, sub.native, sub.upsample, sub.cpu_sample = 0, 1.0, False, 0, 0
        t0 = time.perf_counter()
        rec = fn(sub, px, torch, dev, rank, world, local, dist, emit=False)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        if rec is not None:
            rec = {k: rec[k] for k in FORM_KEYS if k in rec}
            rec["wall_s"] = time.perf_counter() - t0
            forms[name] = rec
    return forms


if __name__ == "__main__":
    main()
