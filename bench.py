#!/usr/bin/env python
"""Dependence-volume benchmark: one reference vertex against every vertex of a
250 x 352 x 20 grid (1.76M vertices) of a 1000-member synthetic ensemble shaped
like the paper's CSEns data (Sec. 6.1, Table 1 workload).

One step = one exact dependence volume for one reference vertex: the Pearson
volume (Eq. 1) and the KSG mutual-information volume (k = 8), both through the
C ABI of libndf.so, inputs resident in HBM.  ``e2e`` repeats the step through
the same ABI from pinned host memory: ensemble upload + statistics + both
volumes + copies of both volumes back to the host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun every rank computes its own reference vertices on its own copy
of the ensemble (weak scaling, no data-path collective); rank 0 prints one JSON
line with the max-over-ranks time.  ``--impl reference`` times the CPU oracle
on the host cores instead (rank 0 only), on a bounded sample of vertices.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

K_NN = 8
# DRAM bytes per launch of the KSG kernels at the full 250x352x20 volume, from a
# one-level slab capture (ncu dram__bytes_read.sum + dram__bytes_write.sum for
# 88,000 vertices) scaled by the vertices processed (x20): the kernels stream each
# query column and its sorted copy once (algorithmic 14.08 GB + 7 MB output).
KSG_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on the "
                      "250x352x1 slab (88,000 vertices, profiles/), x20 vertices")
KSG_PRUNED_TRAFFIC_PER_VOLUME = (705.641e6 + 4.142e6) * 20
KSG_BRUTE_TRAFFIC_PER_VOLUME = (705.845e6 + 4.089e6) * 20
KSG_BLOCK_TRAFFIC_PER_VOLUME = (705.26e6 + 3.64e6) * 20
KSG_LANES_TRAFFIC_PER_VOLUME = (704.32e6 + 3.37e6) * 20
KSG_SEARCHES = {  # name: (ndf constant name, kernel at k = 8, DRAM bytes per volume)
    "pruned": ("NDF_KSG_PRUNED", "ksg_pruned_kernel<9>", KSG_PRUNED_TRAFFIC_PER_VOLUME),
    "block": ("NDF_KSG_BLOCK", "ksg_block_kernel<9>", KSG_BLOCK_TRAFFIC_PER_VOLUME),
    "lanes": ("NDF_KSG_LANES", "ksg_lane_kernel<9>", KSG_LANES_TRAFFIC_PER_VOLUME),
}
METRIC = "ms per 1.76M-voxel dependence volume (Pearson + KSG MI k=8, M=1000)"


def workload_name(recipe):
    return (f"csens-like ensemble {recipe.X}x{recipe.Y}x{recipe.Z} (N={recipe.N:,}), "
            f"M={recipe.M} FP32 members, one reference per volume")


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def build_everything():
    import oracle
    import synth
    from paper_2307_02203_gb300 import build

    synth.build()
    oracle.build()
    build.build()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)),
                "bf16_tflops": float(d.get("bf16_tflops", 1900.0)), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "bf16_tflops": 1900.0, "source": "fallback"}


def make_field(recipe, pinned, nthreads):
    import torch

    import synth

    shape = (recipe.M, recipe.Z, recipe.Y, recipe.X)
    if pinned:
        t = torch.empty(shape, dtype=torch.float32, pin_memory=True)
        arr = t.numpy()
        synth.generate(recipe, out=arr, nthreads=nthreads)
        return t, arr
    arr = synth.generate(recipe, nthreads=nthreads)
    return None, arr


def cpu_baseline(field, recipe, ref, seconds_target, seed, nthreads=0, k=K_NN):
    """Times the oracle (nthreads host cores, 0 = all) on a bounded seeded vertex
    sample and extrapolates to ms per full volume (the full volume when the
    sample covers the grid)."""
    import oracle
    import synth

    cores = oracle.threads(nthreads)
    probe = synth.sample_vertices(recipe, max(2 * cores, 32), seed=seed + 1)
    t0 = time.perf_counter()
    oracle.ksg_volume(field, field, ref, k, verts=probe, nthreads=nthreads)
    oracle.pearson_volume(field, field, ref, verts=probe, nthreads=nthreads)
    per_vertex = (time.perf_counter() - t0) / len(probe)
    count = int(max(len(probe), min(recipe.N, seconds_target / max(per_vertex, 1e-9))))
    verts = synth.sample_vertices(recipe, count, seed=seed)
    t0 = time.perf_counter()
    oracle.pearson_volume(field, field, ref, verts=verts, nthreads=nthreads)
    tp = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.ksg_volume(field, field, ref, k, verts=verts, nthreads=nthreads)
    tk = time.perf_counter() - t0
    scale = recipe.N / count
    ms = (tp + tk) * scale * 1e3
    sample = (f"Pearson + KSG at {count} seeded vertices of {recipe.N}, time x {scale:.1f} "
              f"(extrapolated)" if count < recipe.N else f"Pearson + KSG, full volume of {recipe.N}")
    return {"value": ms, "unit": "ms per volume", "cores": cores, "kind": "oracle",
            "sample": sample, "pearson_ms": tp * scale * 1e3, "ksg_ms": tk * scale * 1e3}


def cpu_baseline_grid(field, recipe, ref, seconds_target):
    """The oracle on all host cores and on one core, for the tiny workload (16x16x4,
    M = 100, k = 4: full volume) and for the benchmark's workload (k = 8, bounded
    samples, extrapolated); host CPU model stated."""
    import synth

    tiny = synth.generate(synth.TINY)
    tref = synth.vertex_index(*synth.TINY_REF, synth.TINY)
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    import oracle

    all_n = oracle.threads(0)  # the oracle's current thread count (all host cores)
    grid = {"cpu_model": model, "nproc": os.cpu_count()}
    try:
        for name, fld, rec, r, secs, k in (
                ("tiny_16x16x4_m100_k4", tiny, synth.TINY, tref, 1.0, 4),
                ("bench_workload_k8", field, recipe, ref, seconds_target / 3, K_NN)):
            grid[name] = {}
            for cores in (all_n, 1):
                d = cpu_baseline(fld, rec, r, secs, seed=11, nthreads=cores, k=k)
                grid[name]["one_core" if cores == 1 else "all_cores"] = {
                    "ms_per_volume": d["value"], "cores": d["cores"], "sample": d["sample"]}
                oracle.threads(all_n)
    finally:
        oracle.threads(all_n)
    return grid


def measure_pearson_batch(ndf, ctx, fid, field, recipe, stream, rank, R=64, reps=3):
    """Times ndf_pearson_batch for R references per precision (the standardised
    copies are built by an untimed first call) and states the error of each
    precision against the FP64 oracle on a seeded vertex sample."""
    import torch

    import oracle
    import synth

    N, M = recipe.N, recipe.M
    rng = np.random.default_rng(4242 + rank)
    refs = [int(r) for r in rng.integers(0, N, size=R)]
    out = torch.empty((R, N), dtype=torch.float32, device="cuda")
    verts = synth.sample_vertices(recipe, 512, seed=99)
    want = np.stack([oracle.pearson_volume(field, field, r, verts=verts) for r in refs])
    res = {"refs": R}
    for name, code in (("tf32", ndf.NDF_PREC_TF32), ("bf16x3", ndf.NDF_PREC_BF16X3),
                       ("fp32", ndf.NDF_PREC_FP32)):
        ndf.ndf_pearson_batch(ctx, fid, fid, refs, code, out)  # builds the copy, warms up
        ndf.ndf_synchronize(ctx)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            ndf.ndf_pearson_batch(ctx, fid, fid, refs, code, out)
        ev1.record(stream)
        ndf.ndf_synchronize(ctx)
        ms = ev0.elapsed_time(ev1) / reps
        got = out[:, torch.from_numpy(verts).cuda()].cpu().numpy().astype(np.float64)
        err = np.abs(got - want)
        kp = (M + 63) // 64 * 64
        zbytes = {"tf32": 4, "bf16x3": 4, "fp32": None}[name]
        entry = {"ms": ms, "ms_per_volume": ms / R, "max_abs_err_vs_fp64": float(err.max()),
                 "mean_abs_err_vs_fp64": float(err.mean())}
        if zbytes:
            gb = (N * kp * zbytes + R * N * 4) / (ms * 1e-3) / 1e9
            entry["hbm_gbs"] = gb
            entry["flops_tflops"] = 2.0 * R * N * kp * (3 if name == "bf16x3" else 1) / (
                ms * 1e-3) / 1e12
        res[name] = entry
    return res


def error_refs(N, count, seed=777):
    """The seeded reference vertices of the learned part's error statement."""
    rng = np.random.default_rng(seed)
    return [int(r) for r in rng.integers(0, N, size=count)]


def measure_ksg_batch(ndf, ctx, fid, recipe, stream, refs, out):
    """len(refs) KSG volumes (k = 8) in one persistent launch (the context's search;
    one work counter over all (reference, vertex) pairs), first eagerly, then the
    same launch captured in a CUDA graph on the context's stream and replayed (device-
    resident reference indices, so the call enqueues no host copy).  out: [R][N]
    device tensor; holds the replay's volumes afterwards."""
    import torch

    N = recipe.N
    R = len(refs)
    d_refs = torch.tensor(refs, dtype=torch.int64, device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ndf.ndf_synchronize(ctx)
    e0.record(stream)
    ndf.ndf_mi_ksg_batch(ctx, fid, fid, d_refs, K_NN, out)
    e1.record(stream)
    ndf.ndf_synchronize(ctx)
    ms = e0.elapsed_time(e1)
    res = {"refs": R, "ms": ms, "ms_per_volume": ms / R, "mi_pairs_per_s": R * N / (ms * 1e-3)}
    eager = out[:2].clone()
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
            ndf.ndf_mi_ksg_batch(ctx, fid, fid, d_refs, K_NN, out)
        out[:2].fill_(float("nan"))
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            g.replay()
            e1.record(stream)
        ndf.ndf_synchronize(ctx)
        torch.cuda.synchronize()
        gms = e0.elapsed_time(e1)
        res["graph"] = {"ms": gms, "ms_per_volume": gms / R,
                        "equals_eager": bool(torch.equal(out[:2], eager))}
        del g
    except Exception as exc:  # noqa: BLE001 -- reported in the line, the eager figure stands
        res["graph"] = {"error": str(exc)[:200]}
    return res


def measure_render(ndf, ctx, model, refs, recipe, stream, W=1024, H=1024):
    """Decode one reference volume and ray-march it (DVR, iso-surface, and the
    difference of two reference fields) into a 1024x1024 RGBA buffer on the
    device; CUDA-event times per image, and decode + render together."""
    import torch

    N = recipe.N
    vol = torch.empty(N, dtype=torch.float32, device="cuda")
    vol2 = torch.empty(N, dtype=torch.float32, device="cuda")
    img = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    tf = [[0.0, 0.0, 0.5, 0.0], [0.1, 0.3, 0.9, 0.5], [0.9, 0.9, 0.9, 0.2], [1.0, 0.5, 0.0, 3.0],
          [0.8, 0.0, 0.0, 12.0]]
    cam = dict(eye=(2.2, 1.6, 2.6), target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fov_y_deg=32.0,
               width=W, height=H, step=2.0 / 512, tf=tf)
    X, Y, Z = recipe.X, recipe.Y, recipe.Z
    modes = {"dvr": dict(mode=ndf.NDF_RENDER_DVR, vmin=-1.0, vmax=1.0),
             "iso": dict(mode=ndf.NDF_RENDER_ISO, vmin=-1.0, vmax=1.0, iso=0.5)}
    ndf.ndf_infer(model, refs[0], vol)
    ndf.ndf_infer(model, refs[1], vol2)
    for kw in modes.values():  # warm-up
        ndf.ndf_render_volume(ctx, vol, None, X, Y, Z, img, **cam, **kw)
    ndf.ndf_synchronize(ctx)
    res = {"width": W, "height": H, "step": cam["step"]}
    for name, kw in modes.items():
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ndf.ndf_infer(model, refs[2], vol)
        e1.record(stream)
        ndf.ndf_render_volume(ctx, vol, None, X, Y, Z, img, **cam, **kw)
        e2.record(stream)
        ndf.ndf_synchronize(ctx)
        res[f"{name}_render_ms"] = e1.elapsed_time(e2)
        res[f"{name}_decode_plus_render_ms"] = e0.elapsed_time(e2)
    e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    e0.record(stream)
    ndf.ndf_render_volume(ctx, vol, vol2, X, Y, Z, img, **cam, **modes["dvr"])
    e1.record(stream)
    ndf.ndf_synchronize(ctx)
    res["difference_dvr_render_ms"] = e0.elapsed_time(e1)
    return res


def measure_sampler(ndf, ctx, fid, stream):
    """Continuous-position training samples (uniform random positions, trilinear
    member columns, paired estimators): triples per second for each measure."""
    import torch

    res = {}
    for name, measure, k, n in (("pearson", ndf.NDF_MEASURE_PEARSON, 0, 1 << 20),
                                ("mi", ndf.NDF_MEASURE_MI_KSG, K_NN, 1 << 17)):
        pr = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        pq = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        t = torch.empty(n, dtype=torch.float32, device="cuda")
        ndf.ndf_sample_triples(ctx, fid, fid, measure, k, 4096, 1, pr, pq, t)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ndf.ndf_sample_triples(ctx, fid, fid, measure, k, n, 2, pr, pq, t)
        e1.record(stream)
        ndf.ndf_synchronize(ctx)
        ms = e0.elapsed_time(e1)
        res[name] = {"triples": n, "ms": ms, "triples_per_s": n / (ms * 1e-3)}
    return res


def measure_hash_ndf(ndf, ctx, fid, recipe, stream, args, grid_only=False, n_freq=None,
                     merge=None, paper_recipe=False, act=None, enc_layers=None):
    """The paper's architecture (hash grid, Fourier features, SnakeAlt MLPs, product
    merge) trained on continuous samples renewed every pass (Pearson, self field);
    decode time per volume and MAE against the exact estimator, beside the best
    constant volume's.  grid_only: the ablation without encoder MLPs (Sec. 6.4);
    merge: another merge operator (Sec. 4.1); paper_recipe: the training recipe of
    Sec. 4.3 run to its end (batch 1000, learning rate 3e-4, 200 passes of 10^6
    fresh pairs, x0.1 after 5 passes without improvement, stop after 2 decays)
    instead of the bench's time-boxed one."""
    import torch

    N = recipe.N
    arch = ndf.ndf_hash_arch_default()
    if grid_only:
        arch.enc_layers = 0
    if n_freq is not None:
        arch.n_freq = n_freq
    if merge is not None:
        arch.merge = merge
    if act is not None:
        arch.act = act
    if enc_layers is not None:
        arch.enc_layers = enc_layers
    cfg = ndf.ndf_train_cfg_default()
    cfg.n_triples = 1 << 19
    cfg.batch = 1 << 13
    cfg.lr = 1e-3
    cfg.max_decays = 100
    cfg.time_budget_s = float(args.ndf_seconds)
    if paper_recipe:
        cfg.n_triples = 1000000
        cfg.batch = 1000
        cfg.lr = 3e-4
        cfg.max_passes = 200
        cfg.patience = 5
        cfg.max_decays = 2
        cfg.time_budget_s = 0.0
    # warm-up: the first training steps of a process load the kernels
    warm = ndf.ndf_hash_model_create(ctx, arch, ndf.NDF_MEASURE_PEARSON, False, 1, recipe.X, recipe.Y,
                                     recipe.Z)
    wp = torch.rand((cfg.batch, 3), device="cuda") * 2 - 1
    for _ in range(10):
        ndf.ndf_hash_model_step(warm, wp, wp, wp[:, 0].contiguous(), 1e-3, True)
    ndf.ndf_hash_model_free(warm)
    t0 = time.perf_counter()
    model = ndf.ndf_hash_train(ctx, fid, fid, ndf.NDF_MEASURE_PEARSON, 0, arch, cfg)
    ndf.ndf_synchronize(ctx)
    wall = time.perf_counter() - t0
    info = ndf.ndf_hash_model_info(model)
    rng = np.random.default_rng(778)
    refs = [int(r) for r in rng.integers(0, N, size=8)]
    dec = torch.empty((len(refs), N), dtype=torch.float32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        ndf.ndf_synchronize(ctx)
        e0.record(stream)
        fn()
        e1.record(stream)
        ndf.ndf_synchronize(ctx)
        return e0.elapsed_time(e1)

    def one_per_call():
        for i, r in enumerate(refs):
            ndf.ndf_hash_infer(model, r, dec[i])

    def batched():
        ndf.ndf_hash_infer_batch(model, refs, dec)

    exact = torch.empty((len(refs), N), dtype=torch.float32, device="cuda")
    ndf.ndf_pearson_batch(ctx, fid, fid, refs, ndf.NDF_PREC_FP32, exact)
    decode = {}
    vols = {}
    tc = ndf.ndf_hash_get_decode(model) == ndf.NDF_HASH_DECODE_TC
    paths = [("fp32", ndf.NDF_HASH_DECODE_FP32, False)]
    if tc:
        paths += [("tc", ndf.NDF_HASH_DECODE_TC, False)]
        if arch.enc_layers > 0 and arch.dec_layers >= 2:  # the query-latent cache needs both
            paths += [("tc_cached", ndf.NDF_HASH_DECODE_TC, True)]
    for name, mode, cache in paths:
        ndf.ndf_hash_set_decode(model, mode, cache)
        first = timed(lambda: ndf.ndf_hash_infer(model, refs[0], dec[0]))  # warm-up (builds a cache)
        d = {"ms_per_volume": timed(one_per_call) / len(refs)}
        if mode == ndf.NDF_HASH_DECODE_TC:
            d["ms_per_volume_batched"] = timed(batched) / len(refs)
        if cache:
            d["first_call_ms_with_query_encoding"] = first
        err = (dec - exact).abs()
        d["mae"] = float(err.mean())
        d["max_err_mean_over_refs"] = float(err.amax(dim=1).mean())
        vols[name] = dec.clone()
        decode[name] = d
    if tc:
        diff = (vols["tc"] - vols["fp32"]).abs()
        decode["tc"]["vs_fp32_mean_abs"] = float(diff.mean())
        decode["tc"]["vs_fp32_max_abs"] = float(diff.max())
        if "tc_cached" in vols:
            decode["tc_cached"]["equals_tc"] = bool(torch.equal(vols["tc_cached"], vols["tc"]))
        # tensor-core roofline: algorithmic flops of the dense layers per volume
        # multiply-adds per vertex: encoder (din -> c, then c -> c), decoder hidden
        # layers (latent -> c, then c -> c), output layer (c -> 1)
        din = 3 + 6 * arch.n_freq + arch.levels * arch.feat
        c = arch.width
        lat = c if arch.enc_layers else din
        enc_mac = din * c + (arch.enc_layers - 1) * c * c if arch.enc_layers else 0
        dec_mac = lat * c + (arch.dec_layers - 2) * c * c if arch.dec_layers >= 2 else 0
        out_mac = c if arch.dec_layers >= 2 else lat
        flop_full = 2.0 * N * (enc_mac + dec_mac + out_mac)
        flop_cached = 2.0 * N * (dec_mac + out_mac)
        peaks = load_peaks()
        peak = peaks["bf16_tflops"]
        for name, fl, key in (("tc", flop_full, "ms_per_volume_batched"),
                              ("tc_cached", flop_cached, "ms_per_volume_batched")):
            if name not in decode:
                continue
            ach = fl / (decode[name][key] * 1e-3) / 1e12
            decode[name]["tensor_tflops"] = ach
            decode[name]["tensor_frac_of_bf16_peak"] = ach / peak
            decode[name]["peak_source"] = peaks["source"]
            decode[name]["algorithmic_gflop_per_volume"] = fl / 1e9
    ndf.ndf_hash_set_decode(model, ndf.NDF_HASH_DECODE_TC if tc else ndf.NDF_HASH_DECODE_FP32)
    ex = exact.reshape(-1)
    idx = torch.randint(0, ex.numel(), (1 << 20,), device="cuda",
                        generator=torch.Generator(device="cuda").manual_seed(3))
    smp = ex[idx]
    const_mae = float((smp - smp.median()).abs().mean())
    res = {"arch": {n: getattr(arch, n) for n, _ in arch._fields_}, "const_mae": const_mae,
           "recipe": "Sec. 4.3 (batch 1000, lr 3e-4, 200 x 1e6 pairs, plateau x0.1)"
           if paper_recipe else "time-boxed (--ndf-seconds)",
           "params": ndf.ndf_hash_model_param_count(model), "triples_per_pass": int(cfg.n_triples),
           "batch": int(cfg.batch), "passes": info["passes"], "adam_steps": info["adam_steps"],
           "train_seconds": info["train_seconds"], "sample_seconds": info["gen_seconds"],
           "train_steps_per_s": info["adam_steps"] / max(info["train_seconds"], 1e-9),
           "train_wall_s": wall, "last_pass_l1": info["last_loss"],
           "decode_ms_per_volume": decode["tc" if tc else "fp32"]["ms_per_volume"],
           "mae": decode["tc" if tc else "fp32"]["mae"], "decode": decode,
           "error_refs": len(refs)}
    ndf.ndf_hash_model_free(model)
    return res


def error_statement(ndf, ctx, model, fa, fb, measure, refs, N, stream, cached=None, chunk=64):
    """Decoded volumes of `model` for every reference in refs against the exact
    estimator on the same GPU, in chunks of `chunk` references (the exact volumes of a
    chunk from one batched call; `cached` may hold the first chunk's).  Decoding is
    timed one reference per launch and 16 per launch.  Reports the MAE over all
    vertices of all volumes, the max error per volume, and the MAE of the best
    constant volume (the median of the exact values) beside it, both of the latter
    from a seeded subsample of 2^18 values per chunk."""
    import torch

    exact = torch.empty((chunk, N), dtype=torch.float32, device="cuda")
    dec = torch.empty((chunk, N), dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    for _ in range(3):  # warm-up of both decode paths
        ndf.ndf_infer(model, refs[0], dec[0])
        ndf.ndf_infer_batch(model, refs[:16], dec[:16])
    ndf.ndf_synchronize(ctx)
    abs_sum, n_vals, max_per_ref, ms_one, ms_16, samples = 0.0, 0, [], 0.0, 0.0, []
    net_samples = []
    for c0 in range(0, len(refs), chunk):
        rs = refs[c0:c0 + chunk]
        R = len(rs)
        if cached is not None and c0 == 0:
            exact[:R].copy_(cached[:R])
        elif measure == ndf.NDF_MEASURE_PEARSON:
            ndf.ndf_pearson_batch(ctx, fa, fb, rs, ndf.NDF_PREC_FP32, exact[:R])
        else:
            ndf.ndf_mi_ksg_batch(ctx, fa, fb, rs, K_NN, exact[:R])
        ndf.ndf_synchronize(ctx)
        e0.record(stream)
        for i, r in enumerate(rs):
            ndf.ndf_infer(model, r, dec[i])
        e1.record(stream)
        for b0 in range(0, R, 16):
            ndf.ndf_infer_batch(model, rs[b0:b0 + 16], dec[b0:b0 + 16])
        e2.record(stream)
        ndf.ndf_synchronize(ctx)
        ms_one += e0.elapsed_time(e1)
        ms_16 += e1.elapsed_time(e2)
        err = (dec[:R] - exact[:R]).abs()
        abs_sum += float(err.double().sum())
        n_vals += R * N
        max_per_ref += err.amax(dim=1).tolist()
        idx = torch.randint(0, R * N, (1 << 18,), generator=gen, device="cuda")
        samples.append(exact[:R].reshape(-1)[idx])
        net_samples.append(dec[:R].reshape(-1)[idx])
    s = torch.cat(samples)
    med = s.median()
    return {"error_refs": len(refs), "mae": abs_sum / n_vals,
            "max_err_mean_over_refs": float(np.mean(max_per_ref)), "max_err": float(max(max_per_ref)),
            "const_value": float(med), "const_mae": float((s - med).abs().mean()),
            "mae_on_const_sample": float((torch.cat(net_samples) - s).abs().mean()),
            "exact_mean_abs_value": float(s.abs().mean()),
            "decode_ms_per_volume_1ref": ms_one / len(refs),
            "decode_ms_per_volume_16refs": ms_16 / len(refs)}


def train_step_bytes(param_count, grid_params):
    """Algorithmic HBM bytes of one Adam step: the gradient zeroed (4 per parameter),
    FP32 master, gradient and both moments read (16), master and moments written
    (12), the grid's BF16 copy written (2 per grid parameter)."""
    return 32.0 * param_count + 2.0 * grid_params


def measure_ndf(ndf, ctx, fid, recipe, stream, args, exact_ms, fid_b=None, mi_first_chunk=None):
    """Learned part: trains a Pearson and a KSG-MI network on the loaded field
    (targets from the GPU estimators), then states the error of the decoded volumes
    against the exact estimator over --ndf-err-refs seeded references (one and 16
    per decode launch), with the best constant volume's error beside it and the
    exact method's time on the same GPU.  With a second field, the same for
    cross-field networks (reference in field A, query in field B).
    mi_first_chunk: exact A->A MI volumes of the first 64 error references, if
    already computed (the batched KSG measurement)."""
    N = recipe.N
    out = {}
    refs = error_refs(N, args.ndf_err_refs)
    runs = [("pearson", ndf.NDF_MEASURE_PEARSON, 0, args.ndf_triples, fid, fid),
            ("mi", ndf.NDF_MEASURE_MI_KSG, K_NN, args.ndf_mi_triples, fid, fid)]
    if fid_b is not None:
        runs += [("pearson_cross", ndf.NDF_MEASURE_PEARSON, 0, args.ndf_triples, fid, fid_b),
                 ("mi_cross", ndf.NDF_MEASURE_MI_KSG, K_NN, args.ndf_mi_triples, fid, fid_b)]
    for name, measure, k, triples, fa, fb in runs:
        cfg = ndf.ndf_train_cfg_default()
        cfg.res[:] = [int(v) for v in args.ndf_res.split(",")]
        cfg.n_triples = int(triples)
        cfg.time_budget_s = float(args.ndf_seconds)
        t0 = time.perf_counter()
        model = ndf.ndf_train(ctx, fa, fb, measure, k, cfg)
        ndf.ndf_synchronize(ctx)
        wall = time.perf_counter() - t0
        info = ndf.ndf_model_info(model)
        render = measure_render(ndf, ctx, model, refs, recipe, stream) if name == "pearson" else None
        cached = mi_first_chunk if name == "mi" else None
        err = error_statement(ndf, ctx, model, fa, fb, measure, refs, N, stream, cached=cached)
        exact = exact_ms[name.split("_")[0]]
        peaks = load_peaks()
        # a10 roofline: the network's multiply-adds per (vertex, reference) -- three
        # 128 x 128 layers (the first on the 128-wide merged input) and the 128-input
        # output -- against the measured BF16 peak
        flop = 2.0 * N * (3 * 128 * 128 + 128)
        tfl = flop / (err["decode_ms_per_volume_16refs"] * 1e-3) / 1e12
        decode_roofline = {"bound": "tensor", "kernel": "infer_tc_kernel", "achieved": tfl,
                           "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                           "frac": tfl / peaks["bf16_tflops"], "flop_per_volume": flop,
                           "peak_source": peaks["source"]}
        # a9 roofline: the Adam step's algorithmic bytes (train_step_bytes) over the
        # whole step's time
        step_ms = 1e3 * max(info["train_seconds"], 1e-9) / max(info["adam_steps"], 1)
        step_bytes = train_step_bytes(info["param_count"], info["grid_params"])
        gbs = step_bytes / (step_ms * 1e-3) / 1e9
        train_roofline = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                          "frac": gbs / peaks["hbm_gbs"], "bytes_per_step": step_bytes,
                          "ms_per_step": step_ms, "peak_source": peaks["source"]}
        out[name] = {
            "triples": info["n_triples"], "triples_per_s": info["n_triples"] / max(info["gen_seconds"], 1e-9),
            "train_seconds": info["train_seconds"], "adam_steps": info["adam_steps"],
            "train_steps_per_s": info["adam_steps"] / max(info["train_seconds"], 1e-9),
            "passes": info["passes"], "last_pass_l1": info["last_loss"], "batch": int(cfg.batch),
            "train_wall_s": wall,
            "network_bytes": info["network_bytes"], "training_bytes": info["training_bytes"],
            "exact_ms_per_volume": exact,
            "speedup_vs_exact_16refs": exact / err["decode_ms_per_volume_16refs"],
            "fields": "A->B" if fb != fa else "A->A", **err,
            "decode_roofline": decode_roofline, "train_roofline": train_roofline,
        }
        if render is not None:
            out[name]["render"] = render
        ndf.ndf_model_free(model)
    return out


def rank_references(N, count, rank):
    """Reference vertices of one rank: an independent seeded stream per rank, so
    that every rank computes its own volumes (weak scaling, no data-path
    collective)."""
    rng = np.random.default_rng(20230705 + rank)
    return [int(r) for r in rng.integers(0, N, size=count)]


def max_over_ranks(values, world, device):
    """Element-wise maximum of per-rank timings: the slowest rank sets the job time."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_ms_per_volume(total_ms, steps, world):
    """Whole-job time per volume: the max-over-ranks time of the timed region over
    the volumes all ranks processed."""
    return total_ms / (steps * world)


def slab_bounds(Z, world):
    """Contiguous z-ranges [z0, z1) of the ranks' slabs: sizes differ by at most one
    level (a rank gets an empty slab only when there are more ranks than levels)."""
    base, extra = divmod(Z, world)
    out, z = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


def slab_owner(ref, plane, bounds):
    """Rank whose slab holds the flat vertex ref (plane = X * Y vertices per level)."""
    z = ref // plane
    for r, (z0, z1) in enumerate(bounds):
        if z0 <= z < z1:
            return r
    raise ValueError(f"vertex {ref} outside the slabs")


def slab_step(ref, plane, bounds, rank, column_of, broadcast, compute):
    """One reference over a grid split into z-slabs.  The owner of the reference
    vertex reads its member column from its own slab (local index ref - z0 * plane)
    and broadcasts it (the one exchange: M floats); every rank then computes the
    volumes of its own slab against that column.  Returns compute's result."""
    owner = slab_owner(ref, plane, bounds)
    col = column_of(ref - bounds[owner][0] * plane) if rank == owner else None
    col = broadcast(col, owner)
    return compute(col)


def torch_broadcast(M, device, world):
    """broadcast(col, owner) for slab_step over torch.distributed (M float32); the
    identity for a single rank."""
    import torch
    import torch.distributed as dist

    def bc(col, owner):
        if world == 1:
            return col
        t = col if col is not None else torch.empty(M, dtype=torch.float32, device=device)
        dist.broadcast(t, src=owner)
        return t
    return bc


def run_slabs(args, recipe, world, rank, local_rank):
    """Strong scaling over z-slabs: every rank holds one slab of the grid (its share
    of the members' values and statistics); per reference the rank whose slab holds
    the reference vertex broadcasts its member column (NCCL, M floats) and every rank
    computes its slab's Pearson and KSG volumes against it.  value = the job's time
    per volume (max over ranks), scaling "strong"."""
    import torch
    import torch.distributed as dist

    from paper_2307_02203_gb300 import ndf

    nthreads = max(1, (os.cpu_count() or 1) // max(1, env_int("LOCAL_WORLD_SIZE", world)))
    _, field = make_field(recipe, pinned=False, nthreads=nthreads)
    M, Z, Y, X = field.shape
    plane, N = X * Y, recipe.N
    bounds = slab_bounds(Z, world)
    z0, z1 = bounds[rank]
    Zs = z1 - z0
    Ns = Zs * plane
    slab_t = None
    if Zs:
        slab_t = torch.empty((M, Zs, Y, X), dtype=torch.float32, pin_memory=True)
        slab_t.numpy()[:] = field[:, z0:z1]
    del field
    stream = torch.cuda.Stream()
    ctx = ndf.ndf_create(local_rank, stream.cuda_stream)
    ndf.ndf_set_ksg_algorithm(ctx, getattr(ndf, KSG_SEARCHES[args.ksg_search][0]))
    if args.ksg_schedule:
        ndf.ndf_ksg_set_schedule(ctx, *args.ksg_schedule)
    fid = ndf.ndf_load_ensemble(ctx, slab_t, M, Zs, Y, X) if Zs else None
    out_r = torch.empty(max(Ns, 1), dtype=torch.float32, device="cuda")
    out_mi = torch.empty(max(Ns, 1), dtype=torch.float32, device="cuda")
    col = torch.empty(M, dtype=torch.float32, device="cuda")
    bc = torch_broadcast(M, "cuda", world)
    refs = rank_references(N, args.warmup + args.steps, 0)  # one reference stream per job
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    cur = {"i": None}

    def column_of(v_local):
        ndf.ndf_field_column(ctx, fid, v_local, col)
        return col

    def compute(c):
        i = cur["i"]
        if i is not None:
            ev[i][0].record(stream)
        if fid is not None:
            ndf.ndf_pearson_column(ctx, c, fid, out_r)
        if i is not None:
            ev[i][1].record(stream)
        if fid is not None:
            ndf.ndf_mi_ksg_column(ctx, c, fid, K_NN, out_mi)
        if i is not None:
            ev[i][2].record(stream)

    def step(ref):
        with torch.cuda.stream(stream):
            slab_step(ref, plane, bounds, rank, column_of, bc, compute)

    for i in range(args.warmup):
        step(refs[i])
    ndf.ndf_synchronize(ctx)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    launches0 = ndf.ndf_launch_count(ctx)
    with ClockSampler(local_rank) as clk:
        barrier()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            cur["i"] = i
            step(refs[args.warmup + i])
        cur["i"] = None
        t_end.record(stream)
        barrier()
    launches = ndf.ndf_launch_count(ctx) - launches0
    total_ms = t_start.elapsed_time(t_end)
    pearson_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    ksg_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    total_ms, pearson_ms, ksg_ms = max_over_ranks([total_ms, pearson_ms, ksg_ms], world, "cuda")
    ms_per_volume = total_ms / args.steps  # every step is one volume of the whole job

    # end to end: each rank uploads its slab from pinned host memory, then the
    # column exchange and both slab volumes into pinned host buffers
    host_r = torch.empty(max(Ns, 1), dtype=torch.float32, pin_memory=True)
    host_mi = torch.empty(max(Ns, 1), dtype=torch.float32, pin_memory=True)
    e2e_steps = max(1, min(args.e2e_steps, args.steps))

    def e2e_volume(ref):
        nonlocal fid
        fid_keep = fid
        fid = ndf.ndf_load_ensemble(ctx, slab_t, M, Zs, Y, X) if Zs else None

        def compute_host(c):
            if fid is not None:
                ndf.ndf_pearson_column(ctx, c, fid, host_r)
                ndf.ndf_mi_ksg_column(ctx, c, fid, K_NN, host_mi)
        with torch.cuda.stream(stream):
            slab_step(ref, plane, bounds, rank, column_of, bc, compute_host)
        if fid is not None:
            ndf.ndf_free_ensemble(ctx, fid)
        fid = fid_keep

    e2e_volume(refs[0])
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        e2e_volume(refs[args.warmup + i])
    barrier()
    e2e_ms = max_over_ranks([(time.perf_counter() - t0) * 1e3], world, "cuda")[0] / e2e_steps

    peaks = load_peaks()
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    peak = sms * 64 / 2 * peaks["sm_max_mhz"] * 1e6 / 1e9
    rank_evals = float(max(b[1] - b[0] for b in bounds) * plane) * M * (M - 1)
    achieved = rank_evals / (ksg_ms * 1e-3) / 1e9
    if rank == 0:
        line = {
            "metric": METRIC, "value": ms_per_volume, "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_volume,
            "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(recipe), "M": M, "grid_xyz": [X, Y, Z], "k": K_NN,
                       "parallelism": f"zslabs{world}", "slabs_z": bounds,
                       "exchange": "one M-float reference column per volume (NCCL broadcast)",
                       "l2": "inputs larger than L2 (each slab read once per volume)"},
            "pearson_ms": pearson_ms, "ksg_ms": ksg_ms, "mi_pairs_per_s": N / (ms_per_volume * 1e-3),
            "ksg_search": args.ksg_search,
            "roofline": {"bound": "alu", "kernel": KSG_SEARCHES[args.ksg_search][1],
                         "achieved": achieved, "peak": peak, "unit": "Gdist/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_source": f"{peaks['source']} max SM clock",
                         "algorithmic_evals_per_launch": rank_evals},
            "e2e": {"value": e2e_ms, "unit": "ms", "call": "ndf_load_ensemble (slab) + "
                    "ndf_field_column + broadcast + ndf_pearson_column + ndf_mi_ksg_column",
                    "h2d_bytes_per_step": int(M * N * 4), "d2h_bytes_per_step": int(2 * N * 4)},
            "gpu_launches": int(launches), "clocks": clk.summary(), "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)
    if fid is not None:
        ndf.ndf_free_ensemble(ctx, fid)
    ndf.ndf_destroy(ctx)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_reference(args, recipe):
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    _, field = make_field(recipe, pinned=False, nthreads=0)
    rng = np.random.default_rng(20230705)
    refs = rng.integers(0, recipe.N, size=args.steps + args.warmup)
    per_step = max(5.0, 60.0 / max(args.steps, 1))
    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        info = cpu_baseline(field, recipe, int(refs[i]), per_step if i >= args.warmup else 2.0,
                            seed=1000 + i)
        if i >= args.warmup:
            vals.append(info["value"])
    v = float(np.mean(vals))
    line = {"metric": METRIC, "value": v, "unit": "ms", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": workload_name(recipe), "k": K_NN},
            "cpu_baseline": {"kind": "oracle", "cores": info["cores"], "sample": info["sample"],
                             "value": v, "unit": "ms"},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


CASES = ("hash-decode", "dense-decode", "pearson-gemm", "ksg", "train-step", "load-device",
         "hash-train-step")


def run_case(args, recipe):
    """One kernel path timed on its own (CUDA events around --repeat calls after
    --warmup calls), for ncu captures and sweeps; prints one JSON line with the
    case's figures.  Not the benchmark line.

      hash-decode   the paper's NDF architecture (seeded parameters, non-zero output
                    layer) decoded over the workload's grid, --decode-mode tc|cached|fp32,
                    --case-refs references per call
      dense-decode  the dense-grid NDF (seeded initialisation) decoded on tcgen05,
                    --case-refs references per call
      pearson-gemm  batched Pearson of --case-refs references on the loaded workload
                    (--precision tf32|bf16x3|fp32)
      ksg           one KSG volume (k = 8) of the loaded workload, --ksg-search
      train-step    dense-NDF Adam steps at batch --case-batch (seeded pairs)
      load-device   ndf_load_ensemble of the workload's field from device memory (the
                    copy, statistics and sorted columns), then ndf_free_ensemble
      hash-train-step  Adam steps of the paper's network (default architecture, Pearson)
                    at batch --case-batch (seeded continuous positions and targets)
    """
    import torch

    import synth
    from paper_2307_02203_gb300 import build
    build.build()
    from paper_2307_02203_gb300 import ndf

    X, Y, Z, N = recipe.X, recipe.Y, recipe.Z, recipe.N
    stream = torch.cuda.Stream()
    ctx = ndf.ndf_create(0, stream.cuda_stream)
    R = max(1, args.case_refs)
    rng = np.random.default_rng(2)
    fid = None
    if args.case in ("pearson-gemm", "ksg"):
        synth.build()
        field = synth.generate(recipe)
        fid = ndf.ndf_load_ensemble(ctx, field, recipe.M, Z, Y, X)
        del field
    elif args.case == "load-device":
        synth.build()
        field_dev = torch.from_numpy(synth.generate(recipe)).cuda()
    out = torch.empty((R, N), dtype=torch.float32, device="cuda")
    info = {}
    free = []
    if args.case == "hash-decode":
        arch = ndf.ndf_hash_arch_default()
        m = ndf.ndf_hash_model_create(ctx, arch, ndf.NDF_MEASURE_PEARSON, False, 1, X, Y, Z)
        p = np.empty(ndf.ndf_hash_model_param_count(m), np.float32)
        ndf.ndf_hash_model_get_params(m, p)
        p[-129:-1] = np.random.default_rng(1).uniform(-0.3, 0.3, 128)  # output layer (0 at init)
        ndf.ndf_hash_model_set_params(m, p)
        mode = {"tc": (ndf.NDF_HASH_DECODE_TC, False), "cached": (ndf.NDF_HASH_DECODE_TC, True),
                "fp32": (ndf.NDF_HASH_DECODE_FP32, False)}[args.decode_mode]
        ndf.ndf_hash_set_decode(m, *mode)
        free.append(lambda: ndf.ndf_hash_model_free(m))
        info["decode_mode"] = args.decode_mode

        def call():
            refs = [int(r) for r in rng.integers(0, N, size=R)]
            if R == 1:
                ndf.ndf_hash_infer(m, refs[0], out[0])
            else:
                ndf.ndf_hash_infer_batch(m, refs, out)
    elif args.case == "dense-decode":
        res = [int(v) for v in args.ndf_res.split(",")]
        m = ndf.ndf_model_create(ctx, res, ndf.NDF_MEASURE_PEARSON, 1, X, Y, Z)
        free.append(lambda: ndf.ndf_model_free(m))

        def call():
            refs = [int(r) for r in rng.integers(0, N, size=R)]
            if R == 1:
                ndf.ndf_infer(m, refs[0], out[0])
            else:
                ndf.ndf_infer_batch(m, refs, out)
    elif args.case == "pearson-gemm":
        prec = {"tf32": ndf.NDF_PREC_TF32, "bf16x3": ndf.NDF_PREC_BF16X3,
                "fp32": ndf.NDF_PREC_FP32}[args.precision]
        info["precision"] = args.precision
        refs = [int(r) for r in rng.integers(0, N, size=R)]

        def call():
            ndf.ndf_pearson_batch(ctx, fid, fid, refs, prec, out)
    elif args.case == "ksg":
        ndf.ndf_set_ksg_algorithm(ctx, getattr(ndf, KSG_SEARCHES[args.ksg_search][0]))
        if args.ksg_schedule:
            ndf.ndf_ksg_set_schedule(ctx, *args.ksg_schedule)
            info["schedule"] = args.ksg_schedule
        info["search"] = args.ksg_search

        def call():
            ndf.ndf_mi_ksg(ctx, fid, fid, int(rng.integers(0, N)), K_NN, out[0])
    elif args.case == "hash-train-step":
        m = ndf.ndf_hash_model_create(ctx, ndf.ndf_hash_arch_default(), ndf.NDF_MEASURE_PEARSON,
                                      False, 1, X, Y, Z)
        free.append(lambda: ndf.ndf_hash_model_free(m))
        B = args.case_batch
        g = torch.Generator(device="cuda").manual_seed(1)
        pr = torch.rand((B, 3), device="cuda", generator=g) * 2 - 1
        pq = torch.rand((B, 3), device="cuda", generator=g) * 2 - 1
        tgt = torch.rand(B, device="cuda", generator=g) * 2 - 1
        info["batch"] = B
        R = 1

        def call():
            ndf.ndf_hash_model_step(m, pr, pq, tgt, 1e-3, True)
    elif args.case == "load-device":
        info["field_bytes"] = 4 * recipe.M * N
        R = 1

        def call():
            ndf.ndf_free_ensemble(ctx, ndf.ndf_load_ensemble(ctx, field_dev, recipe.M, Z, Y, X))
    else:  # train-step
        res = [int(v) for v in args.ndf_res.split(",")]
        m = ndf.ndf_model_create(ctx, res, ndf.NDF_MEASURE_PEARSON, 1, X, Y, Z)
        free.append(lambda: ndf.ndf_model_free(m))
        B = args.case_batch
        pr = torch.rand((B, 3), device="cuda") * 2 - 1
        pq = torch.rand((B, 3), device="cuda") * 2 - 1
        tgt = torch.rand(B, device="cuda") * 2 - 1
        info["batch"] = B
        R = 1

        def call():
            ndf.ndf_model_step(m, pr, pq, tgt, 3e-4, True)

    for _ in range(args.warmup):
        call()
    ndf.ndf_synchronize(ctx)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.repeat):
        call()
    e1.record(stream)
    ndf.ndf_synchronize(ctx)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.repeat
    if args.case == "train-step":
        mi = ndf.ndf_model_info(m)
        step_bytes = train_step_bytes(mi["param_count"], mi["grid_params"])
        info["step_bytes"] = step_bytes
        info["hbm_frac"] = step_bytes / (ms * 1e-3) / 1e9 / load_peaks()["hbm_gbs"]
    line = {"case": args.case, "workload": workload_name(recipe), "grid_xyz": [X, Y, Z],
            "refs_per_call": R, "ms_per_call": ms, "ms_per_volume": ms / R, **info}
    print(json.dumps(line), flush=True)
    for fn in free:
        fn()
    if fid is not None:
        ndf.ndf_free_ensemble(ctx, fid)
    ndf.ndf_destroy(ctx)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-grid", type=int, default=1,
                    help="also time the oracle on one core and on the tiny workload")
    ap.add_argument("--batch", type=int, default=1, help="also time 64-reference Pearson GEMMs")
    ap.add_argument("--ksg-batch", type=int, default=1,
                    help="also time a 64-reference KSG launch (eager and graph-replayed)")
    ap.add_argument("--ksg-autotune", type=int, default=1,
                    help="pick the exact search and its schedule with ndf_ksg_autotune_search")
    ap.add_argument("--ksg-search", choices=sorted(KSG_SEARCHES), default="lanes",
                    help="exact KSG search of the timed step")
    ap.add_argument("--brute-steps", type=int, default=1,
                    help="volumes timed with the brute-force KSG search (same results)")
    ap.add_argument("--ndf", type=int, default=1, help="also train and time the neural field")
    ap.add_argument("--ndf-seconds", type=float, default=25.0, help="training budget per network")
    ap.add_argument("--ndf-hash", type=int, default=1,
                    help="also train the paper's hash-grid architecture (continuous samples)")
    ap.add_argument("--ndf-hash-variants", type=int, default=0,
                    help="also train the ablations of the hash-grid architecture: the sum, "
                         "|difference| and concatenation merges, ReLU encoders, two-layer "
                         "encoders, L = 4, grid-only")
    ap.add_argument("--ndf-hash-recipe", type=int, default=0,
                    help="also train the hash-grid network with the paper's full recipe (minutes)")
    ap.add_argument("--ndf-cross", type=int, default=1,
                    help="also train cross-field networks (reference in A, query in a second field B)")
    ap.add_argument("--ndf-triples", type=int, default=1 << 26, help="Pearson training triples")
    ap.add_argument("--ndf-mi-triples", type=int, default=1 << 26, help="KSG-MI training triples")
    ap.add_argument("--ndf-err-refs", type=int, default=256,
                    help="references of the learned part's error statement (exact volumes each)")
    ap.add_argument("--ndf-res", default="32,64,128,256",
                    help="dense grid points per axis of the 4 levels (smaller only for profiling)")
    ap.add_argument("--workload", choices=["csens", "csens-slab", "tiny"], default="csens",
                    help="csens: 250x352x20, M=1000 (the benchmark); csens-slab: one vertical "
                         "level of it (profiling); tiny: 16x16x4, M=100 (checks)")
    ap.add_argument("--ksg-schedule", type=int, nargs=2, default=None, metavar=("SWITCH_MIN", "EVERY"),
                    help="lane-refill search schedule (default: the library's or the autotuner's)")
    ap.add_argument("--parallel", choices=["replicas", "slabs"], default=None,
                    help="several GPUs: replicas (every rank its own references on its own copy, "
                         "weak scaling) or slabs (the grid split into z-slabs, one reference "
                         "column broadcast per volume, strong scaling; the default for N > 1)")
    ap.add_argument("--case", choices=CASES, default=None,
                    help="time one kernel path on its own (profiling; prints its own JSON line)")
    ap.add_argument("--case-refs", type=int, default=1, help="--case: references per call")
    ap.add_argument("--case-batch", type=int, default=1 << 18, help="--case train-step: batch")
    ap.add_argument("--repeat", type=int, default=10, help="--case: timed calls")
    ap.add_argument("--decode-mode", choices=["tc", "cached", "fp32"], default="tc",
                    help="--case hash-decode: decoder")
    ap.add_argument("--precision", choices=["tf32", "bf16x3", "fp32"], default="tf32",
                    help="--case pearson-gemm: precision")
    ap.add_argument("--grid", type=int, nargs=3, default=None, metavar=("X", "Y", "Z"),
                    help="--case: grid of the decode cases (default: the workload's)")
    args = ap.parse_args()

    import synth

    global METRIC
    recipe = {"csens": synth.CSENS, "tiny": synth.TINY,
              "csens-slab": synth.scaled(synth.CSENS, Z=1)}[args.workload]
    if args.workload != "csens":
        METRIC = f"ms per {recipe.N}-voxel dependence volume (Pearson + KSG MI k=8, M={recipe.M})"
    if args.impl == "reference":
        return run_reference(args, recipe)
    if args.case:
        if args.grid:
            recipe = synth.scaled(recipe, X=args.grid[0], Y=args.grid[1], Z=args.grid[2])
        return run_case(args, recipe)

    import torch
    import torch.distributed as dist

    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.parallel is None:
        args.parallel = "slabs" if world > 1 else "replicas"
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local_rank)
    build_everything()
    from paper_2307_02203_gb300 import ndf

    if args.parallel == "slabs":
        return run_slabs(args, recipe, world, rank, local_rank)

    nthreads = max(1, (os.cpu_count() or 1) // max(1, env_int("LOCAL_WORLD_SIZE", world)))
    field_t, field = make_field(recipe, pinned=True, nthreads=nthreads)
    stream = torch.cuda.Stream()
    ctx = ndf.ndf_create(local_rank, stream.cuda_stream)
    M, Z, Y, X = field.shape
    N = recipe.N
    fid = ndf.ndf_load_ensemble(ctx, field_t, M, Z, Y, X)
    refs = rank_references(N, args.warmup + args.steps, rank)
    out_r = torch.empty(N, dtype=torch.float32, device="cuda")
    out_mi = torch.empty(N, dtype=torch.float32, device="cuda")

    search = getattr(ndf, KSG_SEARCHES[args.ksg_search][0])
    ndf.ndf_set_ksg_algorithm(ctx, search)
    if args.ksg_schedule:
        ndf.ndf_ksg_set_schedule(ctx, *args.ksg_schedule)
    tuned = None
    if args.ksg_autotune:
        t0 = time.perf_counter()
        alg, sw, every = ndf.ndf_ksg_autotune_search(ctx, fid, fid, K_NN)
        args.ksg_search = next(n for n, v in KSG_SEARCHES.items() if getattr(ndf, v[0]) == alg)
        search = alg
        tuned = {"search": args.ksg_search, "switch_min": sw, "every": every,
                 "seconds": time.perf_counter() - t0}

    def step(ref):
        ndf.ndf_pearson(ctx, fid, fid, ref, out_r)
        ndf.ndf_mi_ksg(ctx, fid, fid, ref, K_NN, out_mi)

    for i in range(args.warmup):
        step(refs[i])
    ndf.ndf_synchronize(ctx)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    launches0 = ndf.ndf_launch_count(ctx)
    with ClockSampler(local_rank) as clk:
        barrier()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            ref = refs[args.warmup + i]
            ev[i][0].record(stream)
            ndf.ndf_pearson(ctx, fid, fid, ref, out_r)
            ev[i][1].record(stream)
            ndf.ndf_mi_ksg(ctx, fid, fid, ref, K_NN, out_mi)
            ev[i][2].record(stream)
        t_end.record(stream)
        barrier()
    launches = ndf.ndf_launch_count(ctx) - launches0
    total_ms = t_start.elapsed_time(t_end)
    pearson_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    ksg_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    total_ms, pearson_ms, ksg_ms = max_over_ranks([total_ms, pearson_ms, ksg_ms], world, "cuda")
    ms_per_volume = job_ms_per_volume(total_ms, args.steps, world)

    # ---- distance evaluations of the timed search on the same references (counted
    # in a separate, untimed pass); the brute-force search and the other exact
    # search timed beside it
    nb = max(1, min(args.brute_steps, args.steps))
    ndf.ndf_set_ksg_algorithm(ctx, search, True)
    for i in range(nb):
        ndf.ndf_mi_ksg(ctx, fid, fid, refs[args.warmup + i], K_NN, out_mi)
    search_evals = ndf.ndf_ksg_take_eval_count(ctx) / nb

    def time_search(code):
        ndf.ndf_set_ksg_algorithm(ctx, code, False)
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for i in range(nb):
            ndf.ndf_mi_ksg(ctx, fid, fid, refs[args.warmup + i], K_NN, out_mi)
        b1.record(stream)
        ndf.ndf_synchronize(ctx)
        return b0.elapsed_time(b1) / nb

    ksg_brute_ms = time_search(ndf.NDF_KSG_BRUTE)
    others = {name: {"kernel": KSG_SEARCHES[name][1],
                     "ms": time_search(getattr(ndf, KSG_SEARCHES[name][0]))}
              for name in sorted(KSG_SEARCHES) if name != args.ksg_search}
    ndf.ndf_set_ksg_algorithm(ctx, search, False)
    # KSG algorithm 2 (non-strict counts within the k-NN set's marginal extents): one
    # volume per reference, after a warm-up call
    ndf.ndf_mi_ksg2(ctx, fid, fid, refs[args.warmup], K_NN, out_mi)
    b0 = torch.cuda.Event(enable_timing=True)
    b1 = torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    for i in range(nb):
        ndf.ndf_mi_ksg2(ctx, fid, fid, refs[args.warmup + i], K_NN, out_mi)
    b1.record(stream)
    ndf.ndf_synchronize(ctx)
    ksg2_ms = b0.elapsed_time(b1) / nb
    # ---- device-resident load: copy, statistics and column sorts of a field already in
    # device memory (the second of two loads; the first fills the allocation cache)
    field_dev = field_t.to("cuda")
    load_device_ms = None
    for _ in range(2):
        ndf.ndf_synchronize(ctx)
        b0.record(stream)
        fid_dev = ndf.ndf_load_ensemble(ctx, field_dev, M, Z, Y, X)
        b1.record(stream)
        ndf.ndf_synchronize(ctx)
        load_device_ms = b0.elapsed_time(b1)
        ndf.ndf_free_ensemble(ctx, fid_dev)
    del field_dev
    # ---- batched KSG: 16 references in one launch
    ksg_batch, mi_first_chunk = None, None
    if args.ksg_batch:
        # 64 references in one persistent launch, eager and graph-replayed; they are the
        # first 64 references of the learned part's error statement, whose exact A->A MI
        # volumes they provide
        refs64 = error_refs(N, 64)
        mi_first_chunk = torch.empty((64, N), dtype=torch.float32, device="cuda")
        ksg_batch = measure_ksg_batch(ndf, ctx, fid, recipe, stream, refs64, mi_first_chunk)

    # ---- batched multi-reference Pearson (64 references per call) per precision
    batch = measure_pearson_batch(ndf, ctx, fid, field, recipe, stream, rank) if args.batch else None

    # ---- learned part: train, decode, error against the exact estimators
    fid_b = None
    if args.ndf and args.ndf_cross:
        recipe_b = synth.scaled(synth.CSENS_B, M=recipe.M, Z=recipe.Z, Y=recipe.Y, X=recipe.X)
        _, field_b = make_field(recipe_b, pinned=False, nthreads=nthreads)
        fid_b = ndf.ndf_load_ensemble(ctx, field_b, M, Z, Y, X)
        del field_b
    ndf_res = measure_ndf(ndf, ctx, fid, recipe, stream, args,
                          {"pearson": pearson_ms, "mi": ksg_ms}, fid_b,
                          mi_first_chunk=mi_first_chunk) if args.ndf else None
    mi_first_chunk = None
    if fid_b is not None:
        ndf.ndf_free_ensemble(ctx, fid_b)
        ndf.ndf_trim_cache(ctx)
    if ndf_res is not None:
        ndf_res["continuous_sampler"] = measure_sampler(ndf, ctx, fid, stream)
    if args.ndf_hash or args.ndf_hash_variants or args.ndf_hash_recipe:
        ndf_res = {} if ndf_res is None else ndf_res
        if args.ndf_hash:
            ndf_res["hash_grid_pearson"] = measure_hash_ndf(ndf, ctx, fid, recipe, stream, args)
        if args.ndf_hash_recipe:
            ndf_res["hash_grid_pearson_paper_recipe"] = measure_hash_ndf(
                ndf, ctx, fid, recipe, stream, args, paper_recipe=True)
        if args.ndf_hash_variants:
            for name, code in (("sum", ndf.NDF_MERGE_SUM), ("absdiff", ndf.NDF_MERGE_ABSDIFF),
                               ("concat", ndf.NDF_MERGE_CONCAT)):
                ndf_res[f"hash_grid_pearson_merge_{name}"] = measure_hash_ndf(
                    ndf, ctx, fid, recipe, stream, args, merge=code)
            ndf_res["hash_grid_pearson_relu"] = measure_hash_ndf(ndf, ctx, fid, recipe, stream, args,
                                                                 act=ndf.NDF_ACT_RELU)
            ndf_res["hash_grid_pearson_enc2"] = measure_hash_ndf(ndf, ctx, fid, recipe, stream, args,
                                                                 enc_layers=2)
            ndf_res["hash_grid_pearson_L4"] = measure_hash_ndf(ndf, ctx, fid, recipe, stream, args,
                                                               n_freq=4)
            ndf_res["hash_grid_only_pearson"] = measure_hash_ndf(ndf, ctx, fid, recipe, stream,
                                                                 args, grid_only=True)

    # ---- end to end through the ABI with host buffers (upload + stats + both volumes + D2H)
    host_r = torch.empty(N, dtype=torch.float32, pin_memory=True)
    host_mi = torch.empty(N, dtype=torch.float32, pin_memory=True)
    e2e_steps = max(1, min(args.e2e_steps, args.steps))

    def e2e_volume(ref):  # one call: upload pipelined with the statistics, sorts and search
        fid2 = ndf.ndf_load_and_compute(ctx, field_t, M, Z, Y, X, ref, K_NN, host_r, host_mi)
        ndf.ndf_free_ensemble(ctx, fid2)

    def e2e_volume_sequential(ref):  # load, then each volume
        fid2 = ndf.ndf_load_ensemble(ctx, field_t, M, Z, Y, X)
        ndf.ndf_pearson(ctx, fid2, fid2, ref, host_r)
        ndf.ndf_mi_ksg(ctx, fid2, fid2, ref, K_NN, host_mi)
        ndf.ndf_free_ensemble(ctx, fid2)

    # the host link the end-to-end number depends on, sampled by one plain copy of the
    # pinned field just before each timed call (it is shared with the machine's other
    # GPUs, and its rate changes within seconds)
    h2d_dev = torch.empty(field_t.shape, dtype=torch.float32, device="cuda")

    def link_gbs():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d_dev.copy_(field_t, non_blocking=True)
        torch.cuda.synchronize()
        return field.nbytes / (time.perf_counter() - t0) / 1e9

    def time_e2e(fn):
        fn(refs[0])  # warm-up: first-touch of the second field's device pages
        calls_ms, links = [], []
        for i in range(e2e_steps):
            links.append(link_gbs())
            barrier()
            t0 = time.perf_counter()
            fn(refs[args.warmup + i])
            barrier()
            calls_ms.append((time.perf_counter() - t0) * 1e3)
        ms = max_over_ranks([sum(calls_ms)], world, "cuda")[0]
        return job_ms_per_volume(ms, e2e_steps, world), calls_ms, links

    e2e_per_volume, e2e_calls_ms, e2e_links = time_e2e(e2e_volume)
    e2e_sequential, _, _ = time_e2e(e2e_volume_sequential)
    h2d_gbs = [link_gbs() for _ in range(2)]
    del h2d_dev

    # ---- roofline of the dominant kernel (KSG: ALU-bound distance evaluations)
    peaks = load_peaks()
    props = torch.cuda.get_device_properties(local_rank)
    sms = props.multi_processor_count
    brute_evals = float(N) * M * (M - 1)  # every member pair of every vertex
    # peak: 64 ALU-pipe lanes per SM per clock, 2 ALU instructions per evaluation
    # (the abs-max distance and its threshold compare), at the maximum SM clock.
    # Algorithmic work: the estimator's M (M - 1) distance evaluations per vertex; the
    # exact searches skip most of them (evaluations performed are reported beside).
    peak = sms * 64 / 2 * peaks["sm_max_mhz"] * 1e6 / 1e9
    achieved = brute_evals / (ksg_ms * 1e-3) / 1e9  # algorithmic Gdist/s
    performed = search_evals / (ksg_ms * 1e-3) / 1e9  # Gdist/s actually evaluated
    brute_achieved = brute_evals / (ksg_brute_ms * 1e-3) / 1e9
    pearson_gbs = (4.0 * M * N + 4.0 * N + 16.0 * N) / (pearson_ms * 1e-3) / 1e9

    result = None
    if rank == 0:
        clocks = clk.summary()
        cpu = cpu_baseline(field, recipe, refs[args.warmup], args.cpu_seconds, seed=7) \
            if world == 1 else None
        if cpu is not None and args.cpu_grid:
            cpu["grid"] = cpu_baseline_grid(field, recipe, refs[args.warmup], args.cpu_seconds)
        result = {
            "metric": METRIC, "value": ms_per_volume, "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(recipe), "M": M, "grid_xyz": [X, Y, Z], "k": K_NN,
                       "refs_per_rank": args.steps, "parallelism": f"replicas{world}",
                       "ksg_autotune": tuned,
                       "l2": "inputs larger than L2 (7.04 GB field, read once per volume)"},
            "pearson_ms": pearson_ms, "ksg_ms": ksg_ms,
            "mi_pairs_per_s": N / (ksg_ms * 1e-3),
            "pearson_hbm_gbs": pearson_gbs,
            "pearson_hbm_frac": pearson_gbs / peaks["hbm_gbs"],
            "ksg_search": args.ksg_search,
            "roofline": {"bound": "alu", "kernel": KSG_SEARCHES[args.ksg_search][1],
                         "achieved": achieved, "peak": peak, "unit": "Gdist/s",
                         "frac": achieved / peak, "traffic": KSG_SEARCHES[args.ksg_search][2],
                         "traffic_source": KSG_TRAFFIC_SOURCE,
                         "peak_source": f"{peaks['source']} max SM clock",
                         "algorithmic_evals_per_volume": brute_evals,
                         "evals_performed_per_volume": search_evals,
                         "performed_gdist_s": performed, "performed_frac": performed / peak},
            "ksg_brute_force": {"ms": ksg_brute_ms, "kernel": "ksg_volume_kernel<9>",
                                "roofline": {"bound": "alu", "achieved": brute_achieved,
                                             "peak": peak, "unit": "Gdist/s",
                                             "frac": brute_achieved / peak,
                                             "traffic": KSG_BRUTE_TRAFFIC_PER_VOLUME,
                                             "evals_per_volume": brute_evals},
                                "speedup_of_timed_search": ksg_brute_ms / ksg_ms},
            "ksg_other_searches": others,
            "ksg2_ms": ksg2_ms,
            "load_device_ms": load_device_ms,
            "ksg_batch64": ksg_batch,
            "e2e": {"value": e2e_per_volume, "unit": "ms", "call": "ndf_load_and_compute",
                    "sequential_calls_ms": e2e_sequential,
                    "per_call_ms": e2e_calls_ms,
                    "host_link_gbs_before_call": e2e_links,
                    "host_link_gbs": max(h2d_gbs + e2e_links),
                    "host_link_note": "one pinned-host to device copy of the field, this box: before each timed call and twice after",
                    "h2d_bytes_per_step": int(field.nbytes),
                    "d2h_bytes_per_step": int(2 * N * 4)},
            "gpu_launches": int(launches),
            "pearson_batch64": batch,
            "ndf": ndf_res,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(result), flush=True)
    ndf.ndf_destroy(ctx)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
