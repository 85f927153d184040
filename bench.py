#!/usr/bin/env python
"""Benchmark of the AICA pair-force step on GB300.

A step is one MD step of the method's per-timestep hot path on one batch of
synthetic input resident in HBM: bin the molecules into the mesh cells, then
evaluate LJ forces, energy and virial over the AICA pair set (same-cell, DIL
and real-referred pairs).  The interaction lists are built once beforehand,
as in the paper (App. A); their build time is reported under "setup".
Steps are replayed from a CUDA graph; L2 is flushed (256 MiB memset) before
every timed step, outside the step's CUDA events.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead.
Multi-GPU (torchrun): every rank runs an independent replica (weak scaling);
the value is the sum of pairs over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LJ pair interactions/s within rc (FP32 vs FP64 on same GB300) at stated force error"
UNIT = "pairs/s"
FLOPS_EVAL, FLOPS_WITHIN = 8, 32     # the method's work: flops per AICA-evaluated pair (distance test)
                                     # and per pair within rc (force, energy, virial)
FLOPS64_EVAL, FLOPS64_WITHIN = 14, 35  # FP64 path: (x_k - x_l) - n.L and r^2 unfused; pair body
BIN_BYTES = 84                       # binning: pos 24 + species 4 + previous cell 4 read; cell, order,
                                     # inverse 4 each + float4 16 + FP64 copy 24 written, per molecule
FORCE_TOL = {"fp32": 1e-5, "fp64": 1e-12}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None, help="timed steps (default: 200 on c5, 1000 otherwise)")
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default="c5", help="workload (default c5, the largest single-GPU configuration)")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--fp64-steps", type=int, default=0, help="timed FP64 steps (default steps/10)")
    p.add_argument("--no-extras", action="store_true", help="skip FP64, e2e, accuracy and CPU legs")
    p.add_argument("--study", choices=["cost", "vertex", "nve", "wedge", "adjoint"], default=None,
                   help="instead of the step: the cost-versus-mesh-size study of §2.4 (cost) or the "
                        "vertex-vertex list criterion of §2.2 against the minimum distance (vertex), or the "
                        "paper's verification run of §3 on two meshes (nve), or rotational periodicity through "
                        "general referring transforms (wedge), or the adjoint alone on --config (adjoint)")
    return p.parse_args()


# ------------------------------------------------------------------ distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(backend):
    import torch.distributed as dist
    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend)
    return dist if ws > 1 else None


def aggregate(dist, pairs, ms, device=None):
    """Whole-job value: units of all ranks over the slowest rank's time."""
    import torch
    if dist is None:
        return pairs, ms
    t = torch.tensor([float(pairs), float(ms)], dtype=torch.float64, device=device)
    s = t.clone()
    dist.all_reduce(s[:1], op=dist.ReduceOp.SUM)
    dist.all_reduce(t[1:], op=dist.ReduceOp.MAX)
    return s[0].item(), t[1].item()


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampler for the GPU in use (started before, stopped after)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import numpy as np
    import torch

    global synth
    from paper_cs_0702131_gb300 import synth
    from paper_cs_0702131_gb300.aica import Mesh, aica_last_launch_count

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init("nccl")

    cfg = synth.make(args.config, args.seed + rank)
    n = len(cfg["pos"])
    t0 = time.perf_counter()
    mesh = Mesh(cfg["mesh"], cfg["box"])
    t_create = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mesh.build_lists(cfg["rc"], cfg["skin"])
    t_build = time.perf_counter() - t0
    # two position sets a small MD step apart (0.01 sigma, random directions);
    # consecutive steps alternate between them, so binning re-locates molecules
    rng = np.random.default_rng(args.seed + 1000 + rank)
    posB = synth.random_displacement(cfg["pos"], 0.01, rng, cfg["box"]["L"], cfg["box"]["periodic"])
    pos_sets = [torch.tensor(cfg["pos"], dtype=torch.float64, device=dev),
                torch.tensor(posB, dtype=torch.float64, device=dev)]
    pos = pos_sets[0]
    sp = torch.tensor(cfg["species"], dtype=torch.int32, device=dev)
    # a displaced molecule that left the meshed region (an open boundary or a
    # removed post) keeps its original position in the second set
    mesh.set_deferred(True)
    cB, _, _ = mesh.bin(pos_sets[1], sp)
    out_of_mesh = cB < 0
    pos_sets[1][out_of_mesh] = pos_sets[0][out_of_mesh]
    clear_flags(mesh)
    mesh.set_deferred(False)
    eps, sig = cfg["eps"], cfg["sigma"]
    F32 = torch.empty((n, 3), dtype=torch.float32, device=dev)
    F64 = torch.empty((n, 3), dtype=torch.float64, device=dev)
    evs = [torch.empty(7, dtype=torch.float64, device=dev) for _ in range(2)]
    cnts = [torch.empty(6, dtype=torch.int64, device=dev) for _ in range(2)]
    ev, cnt = evs[0], cnts[0]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    launches = {}

    def step(prec, j=0):
        mesh.bin(pos_sets[j], sp, outputs=False)
        lb = aica_last_launch_count(mesh.h)
        mesh.forces(eps, sig, prec, out=F32 if prec == "fp32" else F64, ev=evs[j], counts=cnts[j])
        launches[prec] = lb + aica_last_launch_count(mesh.h)

    # the timed step computes what the method outputs (forces, energy, virial,
    # pairs within rc); the count of AICA-evaluated pairs (a diagnostic for the
    # flop model, an extra pass over the cell schedule) is taken untimed below
    mesh.set_option("count_evaluated", 0)
    # eager warm-up with checks, then one graph per (precision, position set)
    step("fp32")
    mesh.check()
    step("fp32", 1)
    mesh.check()
    mesh.set_deferred(True)
    graphs = {}
    bin_only = lambda j: mesh.bin(pos_sets[j], sp, outputs=False)
    for prec in ("fp32", "fp64", "bin"):
        fn = bin_only if prec == "bin" else (lambda j, prec=prec: step(prec, j))
        for j in range(2):
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                for _ in range(max(3, args.warmup)):
                    fn(j)
            torch.cuda.current_stream().wait_stream(s)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                fn(j)
            graphs[prec, j] = g
    torch.cuda.synchronize()

    def timed(prec, K, W):
        for i in range(W):
            flush.zero_()
            graphs[prec, i % 2].replay()
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(K):
            flush.zero_()
            e0[i].record()
            graphs[prec, (W + i) % 2].replay()
            e1[i].record()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return [a.elapsed_time(b) for a, b in zip(e0, e1)]

    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    clocks = Clocks(f"GPU-{uuid}" if uuid is not None else str(local))
    clocks.start()
    time.sleep(0.3)
    t_main = timed("fp32", args.steps, args.warmup)
    cAB = [c.cpu().numpy() for c in cnts]
    mesh.set_option("count_evaluated", 1)
    mesh.set_deferred(False)
    mesh.bin(pos_sets[0], sp, outputs=False)
    mesh.forces(eps, sig, "fp32", out=F32, ev=evs[0], counts=cnts[0])
    counts = cnts[0].cpu().numpy()
    assert (counts[3:] == cAB[0][3:]).all(), "within-rc counts differ between calls"
    refined = int(mesh.get_option("refined"))
    mesh.set_option("count_evaluated", 0)
    mesh.set_deferred(True)
    ev_main = evs[0].cpu().numpy()
    stats = mesh.last_stats()

    # pair-kernel duration with CUDA events on its launching stream (eager steps)
    mesh.set_kernel_timing(True)
    kms = []
    for i in range(min(args.steps, 300)):
        flush.zero_()
        step("fp32")
        if (i + 1) % 50 == 0:
            kms += [float(x) for x in mesh.take_kernel_times()]
    kms += [float(x) for x in mesh.take_kernel_times()]
    mesh.set_kernel_timing(False)
    t_bin = timed("bin", max(3, min(args.steps, 200)), 3)
    fp64 = None
    if not args.no_extras:
        K64 = args.fp64_steps or max(3, args.steps // 10)
        t64 = timed("fp64", K64, 3)
        c64AB = [c.cpu().numpy() for c in cnts]
        mesh.set_kernel_timing(True)
        for i in range(10):
            flush.zero_()
            step("fp64")
        kms64 = [float(x) for x in mesh.take_kernel_times()]
        mesh.set_kernel_timing(False)
        stats64 = mesh.last_stats()
    time.sleep(0.2)
    clk = clocks.stop()
    mesh.check()

    unique = lambda c: int(c[3] + c[4] + c[5])
    pairs = (unique(cAB[0]) + unique(cAB[1])) / 2.0      # steps alternate between the two sets
    ms = statistics.mean(t_main)
    tot_pairs, ms_max = aggregate(dist, pairs, ms, dev)
    value = tot_pairs / (ms_max * 1e-3)
    if fp64 is None and not args.no_extras:
        pairs64 = (unique(c64AB[0]) + unique(c64AB[1])) / 2.0
        ms64 = statistics.mean(t64)
        tp64, ms64_max = aggregate(dist, pairs64, ms64, dev)
        fp64 = {"value": tp64 / (ms64_max * 1e-3), "ms_per_step": ms64_max, "steps": len(t64),
                "pairs_equal_fp32": bool(all((c64AB[j][3:] == cAB[j][3:]).all() for j in range(2)))}
        if rank == 0:
            from paper_cs_0702131_gb300.aica import aica_probe_fma_rate
            peak64 = aica_probe_fma_rate(True, 20000) / 1e12
            k64 = statistics.mean(kms64)
            w64 = int(c64AB[0][3] + c64AB[0][4] + c64AB[0][5])
            fl64 = FLOPS64_EVAL * int(stats64[0]) + FLOPS64_WITHIN * w64
            fp64["roofline"] = {"kernel": "pair_fwd64", "bound": "alu", "achieved": round(fl64 / (k64 * 1e-3) / 1e12, 4),
                                "peak": round(peak64, 4), "unit": "TFLOP/s",
                                "frac": round(fl64 / (k64 * 1e-3) / 1e12 / peak64, 4), "kernel_ms": round(k64, 4),
                                "peak_basis": "measured FP64 FMA rate of this GPU (aica_probe_fma_rate)",
                                "flop_model": (f"{FLOPS64_EVAL} per FP64 distance test ({int(stats64[0])}) + "
                                               f"{FLOPS64_WITHIN} per within-rc pair; FP32 sphere tests not counted")}

    out = None
    if rank == 0:
        props = torch.cuda.get_device_properties(dev)
        peaks = measured_peaks()
        sm_max = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
        evals = int(counts[0] + counts[1] + counts[2])
        within_evals = int(counts[3] + counts[4] + counts[5])
        tests, culls = int(stats[0]), int(stats[1])
        # the method's work per launch: every pair of every scheduled cell pair gets a
        # distance test (§2.3's loops), every pair within rc the force body
        flops = FLOPS_EVAL * evals + FLOPS_WITHIN * within_evals
        kmean = statistics.mean(kms)
        achieved = flops / (kmean * 1e-3) / 1e12
        peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
        kname = "pair_fwd32c" if mesh.get_option("cluster_path") else "pair_fwd32"
        roof = {"kernel": kname, "bound": "alu", "achieved": round(achieved, 3),
                "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "traffic": None, "kernel_ms": round(kmean, 5), "launches_timed": len(kms),
                "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz",
                "flops_per_launch": flops,
                "flop_model": (f"{FLOPS_EVAL} per AICA-evaluated pair ({evals}: every pair of every scheduled cell "
                               f"pair) + {FLOPS_WITHIN} per pair within rc ({within_evals})"),
                "work_done": {"pair_tests": tests, "culling_tests": culls,
                              "note": "distance tests the kernel actually performed after culling, and its "
                                      "bounding-box / sphere culling tests; not counted as the method's flops"}}
        if clk and clk.get("sm_mhz"):
            roof["frac_at_sampled_clock"] = round(achieved / (peak * clk["sm_mhz"] / sm_max), 4)
        from paper_cs_0702131_gb300.aica import aica_probe_fma_rate
        peak_fma = aica_probe_fma_rate(False, 1 << 20) / 1e12
        roof["peak_measured_fma"] = round(peak_fma, 2)
        roof["frac_of_measured_fma"] = round(achieved / peak_fma, 4)
        tb = statistics.mean(t_bin)
        hbm = peaks.get("hbm_gbs") or 6800.0
        binning = {"ms_per_step": round(tb, 4), "bytes_per_molecule": BIN_BYTES,
                   "achieved_GBps": round(n * BIN_BYTES / (tb * 1e-3) / 1e9, 1), "peak_GBps": hbm,
                   "frac": round(n * BIN_BYTES / (tb * 1e-3) / 1e9 / hbm, 4),
                   "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)" if peaks.get("hbm_gbs")
                   else "fallback 6.8 TB/s",
                   "note": "whole binning stage (point location with previous-cell hints, counting sort, gather, "
                           "spheres), CUDA graph, L2 flushed, position sets alternating"}
        # DRAM bytes per launch of this kernel from the committed ncu summary
        # (dram__bytes_read.sum + dram__bytes_write.sum), if one exists for it
        prof = os.path.join(ROOT, "profiles", f"{kname}_{args.config}.md")
        if os.path.exists(prof):
            for line in open(prof):
                if line.startswith("| traffic_bytes_per_launch |"):
                    roof["traffic"] = int(line.split("|")[2].strip())
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": synth.CONFIGS[args.config]["doc"], "name": cfg["name"], "n_molecules": n,
                          "n_cells": cfg["mesh"]["n_cells"], "rc": cfg["rc"], "skin": cfg["skin"],
                          "step": ("bin molecules + LJ forces/energy/virial (FP32 pairs, FP64 sums), CUDA graph; "
                        "steps alternate between two position sets 0.01 sigma apart"),
                          "l2": "flushed before every timed step (256 MiB memset outside the step events)",
                          "parallelism": f"replicas x{ws}"},
               "pairs_per_step": {"within_rc": pairs, "aica_evaluated": evals,
                                  "aica_efficiency": round(within_evals / max(evals, 1), 4),
                                  "pair_tests_after_culling": tests, "sphere_tests": culls,
                                  "counts": [int(x) for x in counts],
                                  "count_names": ["eval_same", "eval_dil", "eval_ref", "within_same",
                                                  "within_dil", "within_ref"]},
               "energy_per_molecule": ev_main[0] / n,
               "fp32_refined_molecules": refined,
               "precision": ("pair arithmetic FP32 (separations rounded once); energy and virial sums and the "
                             "cut-off decisions within 1e-5 rc^2 of rc in FP64; molecules whose FP32 force the "
                             "error bound cannot certify to 1e-5 of max(|F_ic|, ||F_i||) recomputed in "
                             f"double-single arithmetic ({refined} of {n} here), inside the timed step"),
               "gpu_launches": int(launches["fp32"]) * args.steps,
               "launches_per_step": int(launches["fp32"]),
               "roofline": roof, "binning": binning, "clocks": clk,
               "setup": {"mesh_create_s": round(t_create, 3), "build_lists_s": round(t_build, 4)}}
        if fp64:
            out["fp64"] = fp64
            out["speedup_fp32_vs_fp64"] = round(value / fp64["value"], 2)
    if not args.no_extras and rank == 0:
        out["rebuild"] = rebuild_and_rebin(cfg, mesh, pos_sets[0], sp, dev)
        mesh.bin(pos_sets[0], sp, outputs=False)      # the oracle sees the first set
        out["force_error"] = accuracy(cfg, mesh, eps, sig, F32, F64, dev)
        out["e2e"] = e2e(args, cfg, mesh, flush, dev)
        out["adjoint"] = adjoint_timing(cfg, mesh, flush, dev, pairs)
        if ws == 1:
            out["cpu_baseline"] = cpu_baseline(cfg)
            out["cpu_cell_list"] = cpu_cell_list(cfg)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    mesh.close()
    return out


def rebuild_and_rebin(cfg, mesh, pos, sp, dev):
    """Interaction-list rebuild (the mesh is static, so the lists do not
    change; timed as the workload asks) and re-binning after every molecule
    moved 0.5 sigma in a random direction (previous cells as the hint)."""
    import numpy as np
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mesh.build_lists(cfg["rc"], cfg["skin"])
    t_build = time.perf_counter() - t0
    rng = np.random.default_rng(4242)
    far = synth.random_displacement(cfg["pos"], 0.5, rng, cfg["box"]["L"], cfg["box"]["periodic"])
    far_d = torch.tensor(far, dtype=torch.float64, device=dev)
    mesh.set_deferred(True)
    cells, _, _ = mesh.bin(far_d, sp)
    keep = cells < 0                      # left the meshed region: keep the original position
    far_d[keep] = pos[keep]
    clear_flags(mesh)
    res = {"build_lists_s": round(t_build, 4)}
    for name, hint_from in (("rebin_0.5sigma_ms", pos), ("bin_from_scratch_like_ms", None)):
        ms = []
        for _ in range(5):
            mesh.bin(hint_from if hint_from is not None else far_d, sp, outputs=False)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            mesh.bin(far_d, sp, outputs=False)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        res[name] = round(statistics.median(ms), 4)
    mesh.check()
    mesh.set_deferred(False)
    res["note"] = ("rebin: previous cells from the undisplaced molecules; second figure: re-binning the same "
                   "displaced molecules (previous cells exact)")
    return res


def accuracy(cfg, mesh, eps, sig, F32, F64, dev, n_sample=4096):
    """Force error on seeded sampled molecules vs the FP64 oracle, per
    component: the stated tolerance |dF_ic| <= tol * max(|F_ic|, ||F_i||)
    (1e-5 FP32, 1e-12 FP64), and the same error relative to sum_l |f_kl|
    (the condition scale of the sum) as a second figure."""
    import numpy as np
    import torch
    import oracle
    rng = np.random.default_rng(123)
    idx = np.sort(rng.choice(len(cfg["pos"]), min(n_sample, len(cfg["pos"])), replace=False))
    ref = oracle.lj(cfg["pos"], cfg["species"], cfg["eps"], cfg["sigma"], cfg["rc"], cfg["box"], idx=idx)
    Fr = ref["F"]
    norm = np.maximum(np.abs(Fr), np.linalg.norm(Fr, axis=1)[:, None])
    res = {}
    for prec, F in (("fp32", F32), ("fp64", F64)):
        mesh.forces(eps, sig, prec, out=F)
        torch.cuda.synchronize()
        Fg = F.double().cpu().numpy()[idx]
        d = np.abs(Fg - Fr)
        e_norm = d / np.maximum(norm, 1e-300)
        e_abs = d / np.maximum(ref["Fabs"], 1e-300)[:, None]
        res[prec] = {"max_rel_to_norm_F": float(e_norm.max()), "p999_rel_to_norm_F": float(np.quantile(e_norm, 0.999)),
                     "tolerance": FORCE_TOL[prec], "within_tolerance": bool(e_norm.max() <= FORCE_TOL[prec]),
                     "max_rel_to_sum_abs_f": float(e_abs.max()),
                     "p999_rel_to_sum_abs_f": float(np.quantile(e_abs, 0.999))}
    res["normalisation"] = "|dF_ic| / max(|F_ic|, ||F_i||_2) (the stated tolerance); also / sum_l |f_kl|"
    res["sample"] = f"{len(idx)} seeded molecules, oracle all-pairs FP64"
    return res


def adjoint_timing(cfg, mesh, flush, dev, pairs):
    """The adjoint (aica_forces_backward: position gradient, i.e. a Hessian-
    vector product, and per-species eps/sigma gradients) for a seeded random
    dL/dF, timed eagerly with CUDA events, L2 flushed before each call."""
    import numpy as np
    import torch
    n = len(cfg["pos"])
    v = torch.tensor(np.random.default_rng(77).normal(size=(n, 3)), device=dev)
    res = {}
    for prec, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        g = v.to(dt)
        for _ in range(2):
            mesh.forces_backward(cfg["eps"], cfg["sigma"], g, prec)
        ms = []
        mesh.set_kernel_timing(True)
        for _ in range(10):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            mesh.forces_backward(cfg["eps"], cfg["sigma"], g, prec)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        kms = [float(x) for x in mesh.take_kernel_times()]
        mesh.set_kernel_timing(False)
        t = statistics.median(ms)
        res[prec] = {"ms": round(t, 4), "pairs_per_s": pairs / (t * 1e-3),
                     "kernel_ms": round(statistics.median(kms), 4) if kms else None}
    res["note"] = ("one backward call (gather of dL/dF, pair kernel recomputing every pair term, scatter); "
                   "kernel_ms: the adjoint pair kernel alone; binning of the current positions not included")
    return res


def clear_flags(mesh):
    """Read and clear the deferred error flags of a binning that was expected
    to find molecules outside the mesh."""
    from paper_cs_0702131_gb300.aica import AicaError
    try:
        mesh.check()
    except AicaError as e:
        if e.name != "AICA_ERR_OUTSIDE_MESH":
            raise


def e2e(args, cfg, mesh, flush, dev):
    """Through the public API with host buffers: H2D of positions and species
    from pinned memory, bin + forces, D2H of forces and energy/virial.  Error
    checks are deferred (one aica_check_status after the timed steps), as a
    pipelined MD loop would run them."""
    import torch
    n = len(cfg["pos"])
    pos_h = torch.tensor(cfg["pos"], dtype=torch.float64).pin_memory()
    sp_h = torch.tensor(cfg["species"], dtype=torch.int32).pin_memory()
    F_h = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    ev_h = torch.empty(7, dtype=torch.float64).pin_memory()
    pos_d = torch.empty_like(pos_h, device=dev)
    sp_d = torch.empty_like(sp_h, device=dev)
    F = torch.empty((n, 3), dtype=torch.float32, device=dev)
    ev = torch.empty(7, dtype=torch.float64, device=dev)
    cnt = torch.empty(6, dtype=torch.int64, device=dev)
    K = max(3, min(args.steps, 200))

    def one():
        pos_d.copy_(pos_h, non_blocking=True)
        sp_d.copy_(sp_h, non_blocking=True)
        mesh.bin(pos_d, sp_d, outputs=False)
        mesh.forces(cfg["eps"], cfg["sigma"], "fp32", out=F, ev=ev, counts=cnt)
        F_h.copy_(F, non_blocking=True)
        ev_h.copy_(ev, non_blocking=True)

    deferred = mesh.deferred
    mesh.set_deferred(True)
    for _ in range(3):
        one()
    torch.cuda.synchronize()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    for i in range(K):
        flush.zero_()
        e0[i].record()
        one()
        e1[i].record()
    torch.cuda.synchronize()
    mesh.check()
    mesh.set_deferred(deferred)
    ms = statistics.mean(a.elapsed_time(b) for a, b in zip(e0, e1))
    c = cnt.cpu().numpy()
    pairs = int(c[3] + c[4] + c[5])
    return {"value": pairs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": K,
            "h2d_bytes_per_step": int(pos_h.numel() * 8 + sp_h.numel() * 4),
            "d2h_bytes_per_step": int(F_h.numel() * 4 + ev_h.numel() * 8)}


def cpu_baseline(cfg, budget_s=10.0):
    """The FP64 all-pairs oracle on the host cores over a bounded sample of
    molecules; each sampled molecule's row is a full O(N) pass."""
    import numpy as np
    import oracle
    n = len(cfg["pos"])
    rng = np.random.default_rng(321)
    probe = np.sort(rng.choice(n, min(n, 64), replace=False))
    t0 = time.perf_counter()
    oracle.lj(cfg["pos"], cfg["species"], cfg["eps"], cfg["sigma"], cfg["rc"], cfg["box"], idx=probe)
    per = (time.perf_counter() - t0) / len(probe)
    m = int(min(n, max(64, budget_s / max(per, 1e-9))))
    idx = np.sort(rng.choice(n, m, replace=False))
    t0 = time.perf_counter()
    r = oracle.lj(cfg["pos"], cfg["species"], cfg["eps"], cfg["sigma"], cfg["rc"], cfg["box"], idx=idx)
    t = time.perf_counter() - t0
    # each physical pair appears in two rows of the full job: unique pairs/s = row pairs / 2 / time
    return {"value": r["row_pairs"] / 2.0 / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{m} of {n} molecules, each a full all-pairs row (FP64, OpenMP); {t:.2f} s",
            "seconds": round(t, 3)}


def cpu_cell_list(cfg):
    """The textbook cubic-cell algorithm (§2.1) in FP64 on the host cores over
    the whole workload: the practical CPU baseline (not the timed reference)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.lj_cells(cfg["pos"], cfg["species"], cfg["eps"], cfg["sigma"], cfg["rc"], cfg["box"])
    t = time.perf_counter() - t0
    return {"value": r["pairs"] / t, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "cubic-cell algorithm of the paper's §2.1, FP64, OpenMP (oracle library)",
            "sample": f"all {len(cfg['pos'])} molecules, one evaluation", "seconds": round(t, 3)}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    import numpy as np
    import oracle
    from paper_cs_0702131_gb300 import synth
    cfg = synth.make(args.config, args.seed)
    n = len(cfg["pos"])
    rng = np.random.default_rng(99)
    probe = np.sort(rng.choice(n, min(n, 32), replace=False))
    t0 = time.perf_counter()
    oracle.lj(cfg["pos"], cfg["species"], cfg["eps"], cfg["sigma"], cfg["rc"], cfg["box"], idx=probe)
    per = (time.perf_counter() - t0) / len(probe)
    budget = 150.0 / max(1, args.steps + args.warmup)          # whole run in about 2.5 minutes
    m = int(min(n, max(8, budget / max(per, 1e-9))))
    times, cnts = [], []
    for i in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(n, m, replace=False))
        t0 = time.perf_counter()
        r = oracle.lj(cfg["pos"], cfg["species"], cfg["eps"], cfg["sigma"], cfg["rc"], cfg["box"], idx=idx)
        t = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(t)
            cnts.append(r["row_pairs"])
    t = sum(times)
    value = sum(cnts) / 2.0 / t
    ms_step = t / len(times) * 1e3
    sample = f"{m} of {n} molecules per step, each a full all-pairs row (FP64, OpenMP)"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": synth.CONFIGS[args.config]["doc"], "name": cfg["name"], "n_molecules": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def n_c(x):
    """§2.4: cubes of a uniform cubic mesh with a corner within x = rc/w of a
    corner of the central cube, the central cube included (exact count)."""
    k = int(np.ceil(x)) + 1
    r = np.arange(-k, k + 1)
    I, J, K = np.meshgrid(r, r, r, indexing="ij")
    g = lambda t: np.maximum(np.abs(t) - 1, 0)
    return int(((g(I) ** 2 + g(J) ** 2 + g(K) ** 2) < x * x).sum())


def _pairs_and_kernel(mesh, cfg, pos, sp, prec="fp32", reps=20):
    import torch
    mesh.bin(pos, sp, outputs=False)
    F, ev, cnt = mesh.forces(cfg["eps"], cfg["sigma"], prec)
    mesh.set_kernel_timing(True)
    for _ in range(reps):
        mesh.forces(cfg["eps"], cfg["sigma"], prec)
    kms = [float(x) for x in mesh.take_kernel_times()]
    mesh.set_kernel_timing(False)
    torch.cuda.synchronize()
    return F, ev.cpu().numpy(), cnt.cpu().numpy(), statistics.median(kms)


def nve_study(args, steps=2000, dt=0.005, every=20):
    """§3 verification run: 27 000 LJ molecules from a simple cubic lattice at
    120 K (T* = 120 / 119.8), no thermostat, velocity Verlet; the same start on
    jittered hexahedra and on Kuhn tetrahedra, FP64 and FP32 pairs."""
    import torch
    from paper_cs_0702131_gb300 import synth
    from paper_cs_0702131_gb300.aica import Mesh, aica_kinetic
    dev = torch.device("cuda", 0)
    rho, nsc, rc, T = 0.8, 30, 2.5, 120.0 / 119.8
    a = (1.0 / rho) ** (1.0 / 3.0)
    L = nsc * a
    box = dict(L=np.array([L, L, L]), periodic=np.array([1, 1, 1], np.int32))
    g = (np.arange(nsc) + 0.5) * a
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos0 = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    n = len(pos0)
    rng = np.random.default_rng(args.seed + 120)
    v0 = rng.normal(size=(n, 3))
    v0 -= v0.mean(0)
    v0 *= np.sqrt(3.0 * (n - 1) * T / (v0 * v0).sum())
    eps, sig, mass = np.array([1.0]), np.array([1.0]), [1.0]
    meshes = {"hex 12^3 jittered": synth.hex_mesh((12, 12, 12), (0, 0, 0), (L, L, L), 0.15, np.random.default_rng(1)),
              "tet 10^3 x 6 Kuhn": synth.hex_mesh((10, 10, 10), (0, 0, 0), (L, L, L), 0.15, np.random.default_rng(2),
                                                 tets=True)}
    runs = {}
    for prec in ("fp64", "fp32"):
        for name, mesh_d in meshes.items():
            m = Mesh(mesh_d, box)
            m.build_lists(rc, 1e-3)
            pos = torch.tensor(pos0, dtype=torch.float64, device=dev)
            vel = torch.tensor(v0, dtype=torch.float64, device=dev)
            sp = torch.zeros(n, dtype=torch.int32, device=dev)
            m.bin(pos, sp, outputs=False)
            F, ev, _ = m.forces(eps, sig, prec, shift=True)
            kin = torch.empty(4, dtype=torch.float64, device=dev)
            aica_kinetic(mass, sp, vel, kin)
            rec = [(0, kin[0].item() / n, ev[0].item() / n, *kin[1:].tolist())]
            m.set_deferred(True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in range(1, steps + 1):
                m.verlet_step(eps, sig, mass, dt, pos, vel, sp, F, prec=prec, ev=ev, kin=kin, shift=True)
                if i % every == 0:
                    rec.append((i, kin[0].item() / n, ev[0].item() / n, *kin[1:].tolist()))
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            m.check()
            m.close()
            rec = np.array(rec)
            te = rec[:, 1] + rec[:, 2]
            runs[(prec, name)] = rec
            rows_ = {"precision": prec, "mesh": name, "cells": mesh_d["n_cells"],
                     "KE_PE_TE_per_molecule_start": [round(rec[0, 1], 6), round(rec[0, 2], 6), round(te[0], 6)],
                     "KE_PE_TE_per_molecule_end": [round(rec[-1, 1], 6), round(rec[-1, 2], 6), round(te[-1], 6)],
                     "TE_max_rel_drift": float(np.abs(te - te[0]).max() / abs(te[0])),
                     "momentum_max_abs": float(np.abs(rec[:, 3:]).max()),
                     "steps_per_s": steps / wall}
            runs[(prec, name, "row")] = rows_
    rows = [v for k, v in runs.items() if len(k) == 3]
    names = list(meshes)
    same = {}
    for prec in ("fp64", "fp32"):
        a_, b_ = runs[(prec, names[0])], runs[(prec, names[1])]
        ta, tb = a_[:, 1] + a_[:, 2], b_[:, 1] + b_[:, 2]
        d = np.abs(ta - tb) / np.abs(ta)
        same[prec] = {"TE_rel_difference_between_meshes_at_step": {int(a_[j, 0]): float(d[j])
                                                                   for j in range(0, len(d), len(d) // 10)}}
    return {"study": "nve", "what": ("27 000 LJ molecules, simple cubic start at rho* = 0.8, T = 120 K (T* = "
                                      f"{T:.4f}), rc = 2.5, dt = {dt} (reduced), {steps} steps, no thermostat, "
                                      "velocity Verlet (aica_verlet_step), energy-shifted potential"),
            "rows": rows, "mesh_independence": same}


def wedge_study(args, steps=100):
    """Rotational periodicity (§2.2.2): a quarter annulus with the quarter
    turn and the z shift as referring transforms; pairs within rc per second
    of bin + forces (FP32 and FP64), against the oracle's sum over images on
    sampled molecules."""
    import torch
    import oracle
    from oracle import transforms as T
    from paper_cs_0702131_gb300 import synth
    from paper_cs_0702131_gb300.aica import Mesh
    dev = torch.device("cuda", 0)
    c = synth.wedge(args.seed, r0=20.0, r1=100.0, nz_sc=20, nr=32, ntheta=48, nz=8)
    n = len(c["pos"])
    m = Mesh(c["mesh"], c["box"])
    m.set_transforms(c["transforms"])
    t0 = time.perf_counter()
    m.build_lists(c["rc"], c["skin"])
    t_build = time.perf_counter() - t0
    pos = torch.tensor(c["pos"], dtype=torch.float64, device=dev)
    sp = torch.tensor(c["species"], dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = {"study": "wedge", "molecules": n, "cells": c["mesh"]["n_cells"], "build_lists_s": round(t_build, 3),
           "referred_cells": int(len(m.lists()["ref_src"]))}
    idx = np.sort(np.random.default_rng(5).choice(n, 64, replace=False))
    pos_s = c["pos"]
    for prec in ("fp32", "fp64"):
        m.bin(pos, sp, outputs=False)
        F, ev, cnt = m.forces(c["eps"], c["sigma"], prec)
        k = cnt.cpu().numpy()
        pairs = int(k[3] + k[4]) + int(k[5]) / 2.0
        ms = []
        for _ in range(steps if prec == "fp32" else max(5, steps // 10)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            m.bin(pos, sp, outputs=False)
            m.forces(c["eps"], c["sigma"], prec, out=F, ev=ev, counts=cnt)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = statistics.median(ms)
        out[prec] = {"pairs_per_s": pairs / (t * 1e-3), "ms_per_step": round(t, 4), "pairs_within_rc": pairs}
    # sampled rows of the oracle's image sum (all molecules as partners, closure of depth 6)
    xf = T.closure(c["transforms"], 6)
    ref = oracle.lj_images(pos_s, c["species"], c["eps"], c["sigma"], c["rc"], xf, idx=idx)
    for prec in ("fp32", "fp64"):
        F, _, _ = m.forces(c["eps"], c["sigma"], prec)
        err = np.abs(F.double().cpu().numpy()[idx] - ref["F"]) / ref["Fabs"][:, None]
        out[prec]["max_rel_to_sum_abs_f"] = float(err.max())
    m.close()
    return out


def run_study(args):
    """Studies of the paper's analysis on this GPU (one JSON line)."""
    import numpy as np
    import torch
    from paper_cs_0702131_gb300 import synth
    from paper_cs_0702131_gb300.aica import Mesh
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    rows = []
    if args.study == "cost":
        # uniform cubic meshes over one FCC fluid: evaluated / within-rc pairs
        # against V_AICA / V_ideal = N_c(rc/w) w^3 / (4/3 pi rc^3) (§2.4)
        rc, nf = 2.5, 24
        rng = np.random.default_rng(args.seed)
        a = synth.A_FCC_08
        L = nf * a
        box = dict(L=np.array([L, L, L]), periodic=np.array([1, 1, 1], np.int32))
        posn = synth.wrap(synth.jitter(synth.fcc_sites(nf, nf, nf, a), 0.05, rng), box["L"], box["periodic"])
        cfg = dict(eps=np.array([1.0]), sigma=np.array([1.0]))
        pos = torch.tensor(posn, dtype=torch.float64, device=dev)
        sp = torch.zeros(len(posn), dtype=torch.int32, device=dev)
        for nh in (16, 20, 27, 33, 41, 55, 66):
            w = L / nh
            mesh = Mesh(synth.hex_mesh((nh,) * 3, (0, 0, 0), (L, L, L), 0.0, np.random.default_rng(0)), box)
            mesh.build_lists(rc, 0.0)
            _, ev, c, kms = _pairs_and_kernel(mesh, cfg, pos, sp)
            within = int(c[3] + c[4] + c[5])
            evaluated = int(c[0] + c[1] + c[2])
            v_aica = n_c(rc / w) * w ** 3 / (4.0 / 3.0 * np.pi * rc ** 3)
            rows.append({"w_over_rc": round(w / rc, 4), "cells": nh ** 3, "N_c": n_c(rc / w),
                         "evaluated_over_within": round(evaluated / within, 4),
                         "V_AICA_over_V_ideal": round(v_aica, 4),
                         "pair_tests_over_within": round(int(mesh.last_stats()[0]) / within, 4),
                         "kernel_ms": round(kms, 4), "ns_per_pair": round(kms * 1e6 / within, 4)})
            mesh.close()
        out = {"study": "cost", "what": ("evaluated/within-rc pairs on uniform cubic meshes vs V_AICA/V_ideal "
                                          "(§2.4); CCA would be 27 rc^3 / V_ideal = 6.45"),
               "molecules": len(posn), "rc": rc, "rows": rows}
    elif args.study == "nve":
        out = nve_study(args)
    elif args.study == "wedge":
        out = wedge_study(args)
    elif args.study == "adjoint":
        cfg = synth.make(args.config, args.seed)
        mesh = Mesh(cfg["mesh"], cfg["box"])
        mesh.build_lists(cfg["rc"], cfg["skin"])
        pos = torch.tensor(cfg["pos"], dtype=torch.float64, device=dev)
        sp = torch.tensor(cfg["species"], dtype=torch.int32, device=dev)
        mesh.bin(pos, sp)
        _, _, cnt = mesh.forces(cfg["eps"], cfg["sigma"], "fp32")
        pairs = int(cnt[3:6].sum().item())
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        out = {"study": "adjoint", "config": args.config, "molecules": len(cfg["pos"]), "pairs_within_rc": pairs,
               "adjoint": adjoint_timing(cfg, mesh, flush, dev, pairs)}
    else:
        # the paper's vertex-vertex criterion against the minimum distance on
        # jittered meshes: pairs within rc it misses, and the error they make
        for name in ("t0", "c1", "c4", "c2"):
            cfg = synth.make(name, args.seed)
            pos = torch.tensor(cfg["pos"], dtype=torch.float64, device=dev)
            sp = torch.tensor(cfg["species"], dtype=torch.int32, device=dev)
            mesh = Mesh(cfg["mesh"], cfg["box"])
            mesh.build_lists(cfg["rc"], 0.0)
            F0, ev0, c0, k0 = _pairs_and_kernel(mesh, cfg, pos, sp, "fp64", reps=3)
            F0 = F0.cpu().numpy()
            within0 = int(c0[3] + c0[4] + c0[5])
            scale = np.abs(F0).max()
            for skin in (0.0, 0.1, 0.25, 0.5):
                mesh.build_lists(cfg["rc"], skin, criterion="vertex")
                F, ev, c, _ = _pairs_and_kernel(mesh, cfg, pos, sp, "fp64", reps=3)
                within = int(c[3] + c[4] + c[5])
                rows.append({"config": name, "cells": cfg["mesh"]["n_cells"], "skin": skin,
                             "pairs_within_rc": within0, "missed_pairs": within0 - within,
                             "missed_fraction": (within0 - within) / within0,
                             "evaluated_vertex_over_min_distance": round(int(c[0] + c[1] + c[2]) /
                                                                         int(c0[0] + c0[1] + c0[2]), 4),
                             "max_force_error_rel_max_force": float(np.abs(F.cpu().numpy() - F0).max() / scale),
                             "energy_error_rel": float(abs(ev[0] - ev0[0]) / abs(ev0[0]))})
            mesh.close()
        out = {"study": "vertex", "what": ("vertex-vertex DIL criterion (§2.2, App. A.1) vs exact minimum "
                                            "distance, FP64 path, rc as configured"), "rows": rows}
    return out


def main():
    args = parse()
    if args.steps is None:
        args.steps = 200 if args.config == "c5" else 1000
    if args.study:
        out = run_study(args)
    else:
        out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out, default=lambda o: o.item() if hasattr(o, "item") else str(o)), flush=True)


if __name__ == "__main__":
    main()
