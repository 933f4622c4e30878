#!/usr/bin/env python
"""Benchmark of GMP features + position gradients on GB300.

One step = the whole hot path on one batch of synthetic input resident in
HBM: exact neighbor images (binning, FP32 pre-screen, FP64-exact cutoff
decision), per-center MCSH moments and rotation-invariant features, and the
vector-Jacobian product of a fixed upstream gradient (forces), all through
the C ABI (gmp_featurize_vjp).  Default workload: the 262,144-atom FCC alloy
slab (orders 0-6, 16 sigmas, cutoff 8 A).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU
oracle on the host cores instead (bounded sample of centers per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "atom-features/sec (features + grads)"
UNIT = "atom-features/s"


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.lines = []
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(self.idx), "-lms", "200"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ work model
def work_model(w, pairs: int):
    """Algorithmic work per step (forward + VJP), per neighbor pair:
    EX2 = n_sigma K, FMA_fwd = n_sigma K (1 + n_l) + n_sigma C + 2C
    (C = Cartesian MCSH components of the requested orders), the VJP costing
    2.5x the forward FMAs and one more set of exps (recompute)."""
    orders = [l for l in w.orders if l >= 0]
    n_l = len(orders)
    C = sum((l + 1) * (l + 2) // 2 for l in orders)
    ns = len(w.sigmas)
    # mean primitives per neighbor, weighted by species frequency
    counts = np.bincount(w.species, minlength=w.n_elements)
    K = float(np.dot(counts, w.n_gauss) / counts.sum())
    fma_fwd = ns * K * (1 + n_l) + ns * C + 2 * C
    ex2 = 2 * ns * K * pairs
    return {"fma_per_pair_fwd": fma_fwd, "flop_fwd": 2.0 * fma_fwd * pairs,
            "flop_bwd": 2.0 * 2.5 * fma_fwd * pairs, "flop_step": 2.0 * 3.5 * fma_fwd * pairs, "ex2_step": ex2}


# DRAM bytes per neighbor pair of the forward and backward kernels, from one
# ncu capture of fcc_slab32k (same instantiation as the default workload;
# dram__bytes_read.sum + dram__bytes_write.sum over its 4,585,082 pairs),
# scaled by the pairs of the run.  Update with the ncu summaries whenever
# the kernels change.
TRAFFIC_PER_PAIR = {"forward": (147.334656e6 + 79.260672e6) / 4585082,
                    "backward": (272.902656e6 + 6.698496e6) / 4585082}


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2303_12980_gb300 import build as B, dist_util, synth
    B.build()
    from paper_2303_12980_gb300.binding import GMPFeaturizer

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = synth.workload(args.workload)
    # A batch of many structures is split across ranks by structure (no
    # data exchange; strong scaling of the fixed batch); a single structure
    # runs as one replica per rank (weak scaling).
    sharded = world > 1 and w.n_struct >= world
    if sharded:
        s0, s1 = dist_util.shard_structures(w.atom_off, rank, world)
        w = dist_util.slice_workload(w, s0, s1)
    N, F_ = w.n_atoms, w.n_features
    Fz = GMPFeaturizer.from_workload(w, device=local_rank)
    pos = torch.from_numpy(w.positions).to(dev)
    sp = torch.from_numpy(w.species).to(dev)
    g_np = synth.upstream_gradient(N, F_, seed=2024 + rank)
    g = torch.from_numpy(g_np).to(dev)
    feat = torch.empty((N, F_), dtype=torch.float32, device=dev)
    gp = torch.empty((N, 3), dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step():
        if args.call == "grad":  # dense Jacobian (diagnostics and profiling of that kernel)
            Fz.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc)
        elif args.call == "features":
            Fz.featurize(pos, sp, w.atom_off, w.cells, w.pbc, out=feat)
        else:
            Fz.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, g, out=(feat, gp))

    tuning = Fz.tune(pos, sp, w.atom_off, w.cells, w.pbc, reps=2) if not args.no_tune else None
    try:  # FP32 FMA / packed-FMA / ex2 throughput at the present clocks (before the timed region)
        from paper_2303_12980_gb300.binding import probe_peaks
        measured = probe_peaks(local_rank)
    except Exception as exc:  # diagnostics only
        measured = {"error": str(exc)}
    contraction = None
    if args.probes:  # the moment and adjoint contractions, FP32 (as run) against tensor-core versions
        from paper_2303_12980_gb300.binding import probe_backward_contraction, probe_contraction
        contraction = {}
        for name, fn in (("forward_moments", probe_contraction), ("backward_adjoints", probe_backward_contraction)):
            try:
                contraction[name] = fn(local_rank)
            except Exception as exc:  # diagnostics only
                contraction[name] = {"error": str(exc)}

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    noff, _, _ = Fz.neighbors(pos, sp, w.atom_off, w.cells, w.pbc)
    pairs = int(noff[-1].item())
    wm = work_model(w, pairs)

    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    Fz.profile(True)
    launches0 = Fz.kernel_launches
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = Fz.kernel_launches - launches0
    prof = Fz.profile_read()
    Fz.profile(False)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_max, units = dist_util.reduce_timing(ms, args.steps * N * F_, device=dev)
    value = units / (ms_max * 1e-3)

    # roofline of the dominant kernel, timed live by CUDA events on the
    # launching stream inside the library (one forward and one backward
    # launch per step for a <= 16-sigma probe set)
    stage = {k: (v[0] / v[1] if v[1] else None) for k, v in prof.items()}
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sm_count * 128 * 2 * 2070e6 / 1e12   # FP32 FMA lanes x 2 FLOP x max SM clock
    kern = {"forward": {"ms": stage["features"], "algorithmic_flop": wm["flop_fwd"]},
            "backward": {"ms": stage["backward"], "algorithmic_flop": wm["flop_bwd"]}}
    for v in kern.values():
        v["tflops"] = v["algorithmic_flop"] / (v["ms"] * 1e-3) / 1e12 if v["ms"] else None
        v["frac"] = v["tflops"] / peak if v["tflops"] else None
    dom = max(kern, key=lambda k: kern[k]["ms"] or 0.0)
    achieved = kern[dom]["tflops"]
    ex2_kernel = wm["ex2_step"] / 2  # each of the forward and backward kernels evaluates n_sigma K exps per pair
    if "fp32_fma_tflops" in measured and achieved:
        measured["frac_of_fp32_fma"] = achieved / measured["fp32_fma_tflops"]
        measured["frac_of_fp32_fma2"] = achieved / measured["fp32_fma2_tflops"]
        for k, v in kern.items():
            if v["ms"]:
                v["ex2_tops"] = ex2_kernel / (v["ms"] * 1e-3) / 1e12
                v["frac_of_ex2"] = v["ex2_tops"] / measured["ex2_tops"]

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e and args.call == "vjp":
        pos_h = torch.from_numpy(w.positions).pin_memory()
        sp_h = torch.from_numpy(w.species).pin_memory()
        g_h = torch.from_numpy(g_np).pin_memory()
        feat_h = torch.empty((N, F_), dtype=torch.float32).pin_memory()
        gp_h = torch.empty((N, 3), dtype=torch.float32).pin_memory()
        Fz.featurize_vjp(pos_h, sp_h, w.atom_off, w.cells, w.pbc, g_h, out=(feat_h, gp_h))
        ke = max(3, args.steps // 2)
        t0 = time.perf_counter()
        for _ in range(ke):
            Fz.featurize_vjp(pos_h, sp_h, w.atom_off, w.cells, w.pbc, g_h, out=(feat_h, gp_h))
        te = (time.perf_counter() - t0) / ke
        te_max, e_units = dist_util.reduce_timing(te * 1e3, N * F_, device=dev)
        e2e = {"value": e_units / (te_max * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(N * 3 * 8 + N * 4 + N * F_ * 4),
               "d2h_bytes_per_step": int(N * F_ * 4 + N * 3 * 4)}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "atoms": N, "structures": w.n_struct, "features": F_,
                   "orders": w.orders, "n_sigmas": len(w.sigmas), "cutoff": w.cutoff, "pairs": pairs,
                   "step": {"vjp": "neighbors + features + VJP (forces), gmp_featurize_vjp",
                            "grad": "neighbors + features + dense Jacobian, gmp_featurize_grad",
                            "features": "neighbors + features, gmp_featurize"}[args.call],
                   "l2": "256 MB buffer written between timed steps (outside the step events)",
                   "parallelism": (f"dp{world}, structures sharded" if sharded else f"replicas{world}")
                   if world > 1 else "single"},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": {"bound": "alu", "kernel": "k_jacobian" if (args.call == "grad" and dom == "backward") else f"k_{dom}",
                     "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                     "traffic": (TRAFFIC_PER_PAIR[dom] * pairs
                                 if dom in TRAFFIC_PER_PAIR and args.call == "vjp" else None),
                     "peak_basis": f"{sm_count} SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz (derived)",
                     "kernels": kern, "ex2_per_step": wm["ex2_step"], "measured_peaks": measured,
                     "contraction_probe": contraction, "stage_ms": stage},
        "wall_s_timed": wall,
        "tuning": tuning,
    }
    if rank == 0 and args.batched:
        out["batched"] = batched_comparison(args)
    if rank == 0 and not args.no_cpu_baseline and args.call == "vjp":
        out["cpu_baseline"], acc = cpu_baseline(w, feat, gp, g_np, budget_s=args.cpu_budget)
        out["accuracy"] = acc
    return out


def batched_comparison(args):
    """10,000 uneven structures (batched10k, features + VJP): one batched
    call, its CUDA-graph replay, and the plain one-structure-per-call loop,
    same kernels and accuracy."""
    import torch
    from paper_2303_12980_gb300 import synth
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    w = synth.workload("batched10k")
    dev = torch.device("cuda")
    pos = torch.from_numpy(w.positions).to(dev)
    sp = torch.from_numpy(w.species).to(dev)
    g = torch.from_numpy(synth.upstream_gradient(w.n_atoms, w.n_features, seed=7)).to(dev)
    feat = torch.empty((w.n_atoms, w.n_features), device=dev)
    gp = torch.empty((w.n_atoms, 3), device=dev)
    units = w.n_atoms * w.n_features
    s = torch.cuda.Stream()
    res = {"workload": "batched10k", "structures": w.n_struct, "atoms": w.n_atoms}
    with torch.cuda.stream(s):
        Fz = GMPFeaturizer.from_workload(w)
        res["tuning"] = Fz.tune(pos, sp, w.atom_off, w.cells, w.pbc, reps=2)
        for mode in ("eager", "graph"):
            Fz.set_graph(mode == "graph")
            for _ in range(3):
                Fz.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, g, out=(feat, gp))
            s.synchronize()
            t0 = time.perf_counter()
            for _ in range(5):
                Fz.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, g, out=(feat, gp))
            s.synchronize()
            dt = (time.perf_counter() - t0) / 5
            res[mode] = {"ms": dt * 1e3, "value": units / dt}
        Fz.set_graph(False)
        off = w.atom_off
        t0 = time.perf_counter()
        for k in range(w.n_struct):
            a, b = int(off[k]), int(off[k + 1])
            Fz.featurize_vjp(pos[a:b], sp[a:b], np.array([0, b - a]), w.cells[k:k + 1], w.pbc[k:k + 1],
                             g[a:b], out=(feat[a:b], gp[a:b]))
        s.synchronize()
        dt = time.perf_counter() - t0
        res["per_structure"] = {"ms": dt * 1e3, "value": units / dt,
                                "note": "one gmp_featurize_vjp call per structure (plain path)"}
    res["unit"] = UNIT
    return res


# ------------------------------------------------------------------ all workloads
CONFIG_TABLE = [
    ("random64_box", "features"),
    ("fcc4096", "features"),
    ("batched10k", "features"),
    ("fcc4096", "jacobian"),
    ("fcc_slab262k", "vjp"),
]


def run_configs(args):
    """Every workload of the baseline table: the optimised path (autotuned
    shapes, CUDA-graph replay where the call supports it) against the plain
    path (default shapes, eager; one call per structure for a batch), the
    ALU-roofline fraction of the dominant kernel, the FP64 oracle on the
    host cores and the accuracy of a sampled subset against it."""
    import torch
    from oracle import oracle as O
    from paper_2303_12980_gb300 import build as B, synth
    B.build()
    O.build()
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    dev = torch.device("cuda")
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sm_count * 128 * 2 * 2070e6 / 1e12
    rows = []
    s = torch.cuda.Stream()
    for idx, (name, mode) in enumerate(CONFIG_TABLE):
        w = synth.workload(name)
        N, F_ = w.n_atoms, w.n_features
        pos = torch.from_numpy(w.positions).to(dev)
        sp = torch.from_numpy(w.species).to(dev)
        g_np = synth.upstream_gradient(N, F_, seed=31)
        g = torch.from_numpy(g_np).to(dev)
        feat = torch.empty((N, F_), device=dev)
        gp = torch.empty((N, 3), device=dev)
        units = N * F_

        def call(Fz, a=0, b=N, k0=0, k1=None):
            k1 = w.n_struct if k1 is None else k1
            off = np.asarray(w.atom_off[k0:k1 + 1]) - w.atom_off[k0]
            args_ = (pos[a:b], sp[a:b], off, w.cells[k0:k1], w.pbc[k0:k1])
            if mode == "features":
                return Fz.featurize(*args_, out=feat[a:b])
            if mode == "vjp":
                return Fz.featurize_vjp(*args_, g[a:b], out=(feat[a:b], gp[a:b]))
            return Fz.featurize_grad(*args_)

        def timed(fn, reps):
            for _ in range(3):
                fn()
            s.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                fn()
            e1.record(s)
            s.synchronize()
            return e0.elapsed_time(e1) / reps

        row = {"config": idx, "workload": name, "mode": mode, "atoms": N, "structures": w.n_struct,
               "features": F_}
        with torch.cuda.stream(s):
            plain = GMPFeaturizer.from_workload(w)
            if w.n_struct > 1:
                off = w.atom_off
                ms_plain = timed(lambda: [call(plain, int(off[k]), int(off[k + 1]), k, k + 1)
                                          for k in range(w.n_struct)], 1)
                row["plain"] = {"path": "one call per structure, default shapes, eager"}
            else:
                ms_plain = timed(lambda: call(plain), 5)
                row["plain"] = {"path": "default shapes, eager"}
            row["plain"].update(ms=ms_plain, value=units / (ms_plain * 1e-3))
            Fz = GMPFeaturizer.from_workload(w)
            Fz.tune(pos, sp, w.atom_off, w.cells, w.pbc, reps=2)
            graph = mode != "jacobian"
            Fz.set_graph(graph)
            ms_opt = timed(lambda: call(Fz), 5)
            Fz.set_graph(False)
            Fz.profile(True)
            Fz.profile_read()
            out = call(Fz)
            s.synchronize()
            prof = Fz.profile_read()
            Fz.profile(False)
            noff, _, _ = Fz.neighbors(pos, sp, w.atom_off, w.cells, w.pbc)
            s.synchronize()
        pairs = int(noff[-1].item())
        wm = work_model(w, pairs)
        stage = {k: (v[0] / v[1] if v[1] else None) for k, v in prof.items()}
        row["optimised"] = {"path": "autotuned" + (", CUDA-graph replay" if graph else ", eager"),
                            "ms": ms_opt, "value": units / (ms_opt * 1e-3), "stage_ms": stage}
        if mode == "vjp":
            kern, flop, ms_k = "k_backward", wm["flop_bwd"], stage["backward"]
        elif mode == "jacobian":
            kern, flop, ms_k = "k_jacobian", wm["flop_bwd"], stage["backward"]
        else:
            kern, flop, ms_k = "k_forward", wm["flop_fwd"], stage["features"]
        tfl = flop / (ms_k * 1e-3) / 1e12 if ms_k else None
        row["roofline"] = {"kernel": kern, "achieved_tflops": tfl, "peak_tflops": peak,
                           "frac": tfl / peak if tfl else None, "pairs": pairs}
        # oracle: a bounded sample of centers on the host cores
        c = synth.subset_centers(N, 8, seed=11)
        fn = O.features if mode == "features" else O.jacobian_rows
        t0 = time.perf_counter()
        fn(w, c)
        dt = time.perf_counter() - t0
        n = int(max(8, min(N, 8 * args.cpu_budget / 5.0 / max(dt, 1e-3))))
        c = synth.subset_centers(N, n, seed=11)
        t0 = time.perf_counter()
        f_ref, f_abs = O.features(w, c, want_abs=True)
        if mode != "features":
            ooff, oj, ojac, oabs = O.jacobian_rows(w, c, want_abs=True)
        dt = time.perf_counter() - t0
        row["oracle"] = {"value": n * F_ / dt, "cores": O.num_threads(), "centers": n,
                         "work": "FP64 features" + ("" if mode == "features" else " + d(features)/d(positions) rows")}
        fgpu = (out[0] if mode == "jacobian" else feat).cpu().numpy()[c]
        err = np.abs(fgpu - f_ref) / np.maximum(np.maximum(np.abs(f_ref), 1e-6 * f_abs), 2.0 ** -126)
        acc = {"features_max_rel_err": float(err.max())}
        if mode == "jacobian":
            joff, jj, jac = (t.cpu().numpy() for t in out[1:])
            worst = 0.0
            for t, i in enumerate(c):
                a, b = joff[i], joff[i + 1]
                num = np.linalg.norm(jac[a:b].astype(np.float64) - ojac[ooff[t]:ooff[t + 1]], axis=-1)
                den = np.maximum(np.maximum(np.linalg.norm(ojac[ooff[t]:ooff[t + 1]], axis=-1),
                                            5e-3 * oabs[ooff[t]:ooff[t + 1]]), 2.0 ** -126)
                worst = max(worst, float((num / den).max()))
            acc["grad_max_rel_err"] = worst
        elif mode == "vjp":
            atoms = synth.subset_centers(N, 4, seed=12)
            gref, gscale = O.vjp_atoms(w, g_np, atoms, want_abs=True)
            acc["grad_max_rel_err"] = float(np.max(np.linalg.norm(gp.cpu().numpy()[atoms] - gref, axis=1)
                                                   / np.maximum(np.linalg.norm(gref, axis=1), 1e-3 * gscale)))
        row["accuracy"] = acc
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    return {"configs": rows, "unit": UNIT, "peak_basis": f"{sm_count} SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz"}


def _oracle_sample(w, centers):
    from oracle import oracle as O
    t0 = time.perf_counter()
    O.jacobian_rows(w, centers)
    return time.perf_counter() - t0


def cpu_baseline(w, feat_dev, gp_dev, g_np, budget_s=15.0):
    """The FP64 oracle (features + full position derivatives of sampled
    centers) timed on the host cores; the same sample checks accuracy."""
    from oracle import oracle as O
    from paper_2303_12980_gb300 import synth
    O.build()
    n = 16
    c = synth.subset_centers(w.n_atoms, n, seed=11)
    dt = _oracle_sample(w, c)
    n = int(max(16, min(4096, n * budget_s / max(dt, 1e-3))))
    c = synth.subset_centers(w.n_atoms, n, seed=11)
    t0 = time.perf_counter()
    f_ref, f_abs = O.features(w, c, want_abs=True)
    O.jacobian_rows(w, c)
    dt = time.perf_counter() - t0
    base = {"value": n * w.n_features / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{n} random centers of {w.name}: FP64 features + d(features)/d(positions) rows"}
    f = feat_dev.cpu().numpy()[c]
    err = np.abs(f - f_ref) / np.maximum(np.abs(f_ref), 1e-6 * f_abs)
    ferr = float(np.max(err))
    # per feature group: the (order, sigma) columns, order-major; order -1 has one column
    col_err = err.max(axis=0)
    by_order, worst, c0 = {}, (None, None, -1.0), 0
    for l in w.orders:
        nc = 1 if l < 0 else len(w.sigmas)
        e = col_err[c0:c0 + nc]
        by_order[str(l)] = float(e.max())
        k = int(np.argmax(e))
        if e[k] > worst[2]:
            worst = (int(l), None if l < 0 else float(w.sigmas[k]), float(e[k]))
        c0 += nc
    atoms = synth.subset_centers(w.n_atoms, 4, seed=12)
    gref, gscale = O.vjp_atoms(w, g_np, atoms, want_abs=True)
    gerr = float(np.max(np.linalg.norm(gp_dev.cpu().numpy()[atoms] - gref, axis=1)
                        / np.maximum(np.linalg.norm(gref, axis=1), 1e-3 * gscale)))
    acc = {"features_max_rel_err": ferr, "grad_max_rel_err": gerr,
           "features_max_rel_err_by_order": by_order,
           "worst_group": {"order": worst[0], "sigma": worst[1], "rel_err": worst[2]},
           "sample": f"{n} centers (features), 4 atoms (VJP)",
           "floors": "features: max(|f|, 1e-6 F_abs); grads: max(|g|, 1e-3 G_abs)"}
    return base, acc


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The FP64 CPU oracle on the host cores, each step a bounded sample of
    centers of the same workload (features + position derivatives)."""
    from oracle import oracle as O
    from paper_2303_12980_gb300 import synth
    O.build()
    w = synth.workload(args.workload)
    c0 = synth.subset_centers(w.n_atoms, 8, seed=21)
    dt = _oracle_sample(w, c0)
    per = int(max(8, min(2048, 8 * args.ref_step_s / max(dt, 1e-3))))
    times = []
    for k in range(args.warmup + args.steps):
        c = synth.subset_centers(w.n_atoms, per, seed=100 + k)
        t = _oracle_sample(w, c)
        if k >= args.warmup:
            times.append(t)
    ms = 1e3 * sum(times) / len(times)
    value = per * w.n_features / (ms * 1e-3)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "atoms": w.n_atoms, "features": w.n_features,
                   "step": f"{per} random centers: FP64 features + d(features)/d(positions)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{per} random centers per step of {w.name}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fcc_slab262k")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--batched", action="store_true",
                    help="add the 10,000-structure batched / graph / per-structure comparison")
    ap.add_argument("--ref-step-s", type=float, default=4.0)
    ap.add_argument("--call", default="vjp", choices=["vjp", "grad", "features"],
                    help="the timed call (default: features + VJP, the headline step)")
    ap.add_argument("--probes", action="store_true",
                    help="also run the contraction probe (packed FP32 against tensor-core versions) before the timed region")
    ap.add_argument("--configs", action="store_true",
                    help="measure every workload of the baseline table (one JSON object) instead")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if args.configs:
        if rank == 0:
            print(json.dumps(run_configs(args)), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
