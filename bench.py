#!/usr/bin/env python
"""Benchmark of the multi-pocket docking hot path on GB300 (one process per GPU).

One step = the whole path over the multi-pocket workload: a 5,000-atom synthetic receptor with
10 carved pockets (radius 6-10 A, 24 A boxes at 0.375 A spacing), one 30-atom ligand with 6
torsions, 1,000 chains x 2,000 MC steps per pocket, top-9 poses per pocket merged and ranked:
receptor typing + binning + grid maps, batched MC/RILC-BFGS search, selection and merge.
value = docked ligand-pocket pairs per second (all ranks). Extra figures: score+gradient
evaluations per second, the plain one-launch-per-pocket path on a sample, the score
microbenchmark (65,536 poses), the search kernel's roofline, and the FP64 CPU oracle.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) the job is N ligands x the 10 pockets (10 pairs per GPU: weak scaling), split
into equal pocket-major runs of pairs (shard.plan_pairs) that keep the unsplit job's random streams;
each rank builds only its pockets' maps, and the ranked poses are gathered and merged on rank 0.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import pvsynth as S  # noqa: E402

METRIC = "docked ligand-pocket pairs/sec and score+grad evals/sec at 1 GB300, batched vs plain"
UNIT = "pairs/s"
WORKLOAD = ("multi-pocket: 5,000-atom receptor, 10 pockets (r 6-10 A, 24 A boxes, 0.375 A), "
            "1 ligand 30 atoms / 6 torsions, 1,000 chains x 2,000 MC steps per pocket, top-9 merged")
CHAINS, STEPS, TOP_K = 1000, 2000, 9
# FP32 operations of one (grid node, receptor atom within 8 A, ligand type) term evaluation of the
# map build: surface distance 2, two Gaussians 8 (with their exponentials), repulsion 3,
# hydrophobic and H-bond ramps 4, accumulation 1
GRID_FLOPS_PER_TERM = 18
L2_FLUSH_BYTES = 512 << 20


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ------------------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------- workload --
def workload(seed: int):
    w = S.multipocket(seed=seed, chains=CHAINS, steps=STEPS)
    return w.receptors[0], w.boxes[0], w.ligands[0]


# Sources of what the multi-pocket bench launches (grid build, search, top-k, merge) and of the
# host code that shapes those launches; the stored profiles are valid while these are unchanged.
DOCK_SOURCES = ("pv_api.cu", "pv_chain.cuh", "pv_device.cuh", "pv_grid.cu", "pv_internal.h",
                "pv_layout.h", "pv_ligand.cpp", "pv_ligand.h", "pv_search.cu", "pv_search_packed.cu",
                "pv_stage.cuh", "pv_terms.h", "pv_thread.cuh", "pv_warp.cuh")


def _code_only(text: str, hash_comment: str) -> str:
    """The source without its comments (C/C++ `//` and `/* */`, or the given line-comment marker
    for Python) and with runs of whitespace collapsed; string and character literals are kept."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":                                    # a literal: copied through its closing quote
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith(hash_comment, i):
            while i < n and text[i] != "\n":
                i += 1
        elif hash_comment == "//" and text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash() -> str:
    """Hash of the code (comments and layout left out) of the dock path's sources and of the build
    script (its compiler flags shape the code): a stored profile stays valid while none of them
    changes."""
    d = os.path.join(ROOT, "paper_2506_20043_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(DOCK_SOURCES):
        h.update(_code_only(open(os.path.join(d, f), encoding="utf-8").read(), "//").encode())
    h.update(_code_only(open(os.path.join(ROOT, "paper_2506_20043_gb300", "build.py"), encoding="utf-8").read(),
                        "#").encode())
    return h.hexdigest()[:16]


def stored_grid_profile():
    """DRAM bytes (read + write) of one map build of the ten boxes, from the committed ncu summary of
    grid_kernel, if it was taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "grid_kernel_multipocket.md")
    if not os.path.exists(p):
        return None
    import re
    txt = open(p).read()
    m_hash = re.search(r"kernel source hash at capture:\s*`?([0-9a-f]{16})", txt, re.I)
    m_tr = re.search(r"dram bytes per launch:\s*([0-9.eE+]+)", txt)
    if not m_hash or m_hash.group(1) != kernel_source_hash() or not m_tr:
        return None
    return float(m_tr.group(1))


def stored_profile():
    """Figures of the committed ncu summary of the search kernel, if it was taken on the current
    kernel sources (else {}): 'traffic' = DRAM bytes (read + write) of one launch of the bench's
    shape (16 step blocks, each sweeping the pockets' maps once; captured at 400 steps, which
    makes the same sweeps), 'inst' = warp instructions per evaluation."""
    p = os.path.join(ROOT, "profiles", "search_round_kernel_multipocket.md")
    if not os.path.exists(p):
        return {}
    txt = open(p).read()
    import re
    m_hash = re.search(r"kernel source hash at capture:\s*`?([0-9a-f]{16})", txt, re.I)
    if not m_hash or m_hash.group(1) != kernel_source_hash():
        return {}
    out = {}
    m_tr = re.search(r"dram bytes per launch:\s*([0-9.eE+]+)", txt)
    m_in = re.search(r"warp instructions per evaluation:\s*([0-9.eE+]+)", txt)
    if m_tr:
        out["traffic"] = float(m_tr.group(1))
    if m_in:
        out["inst"] = float(m_in.group(1))
    return out


# ------------------------------------------------------------------------------ our arm --
def run_ours(args):
    import torch
    import torch.distributed as dist
    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    import paper_2506_20043_gb300 as pv
    pv.build()
    from paper_2506_20043_gb300 import api, shard

    ctx = api.Context(local)
    stream = ctx.stream
    rec, boxes, lig_src = workload(seed=0)
    # the job: `world` ligands x the 10 pockets, split into equal runs of the pocket-major pair list
    # (shard.plan_pairs), each pair keeping its random stream of the unsplit job; at N = 1 that is
    # the headline workload (1 ligand x 10 pockets) docked in one call
    job_ligs = [lig_src] + [S.ligand_centered(S.make_ligand(30, 6, 1000 + i)) for i in range(1, world)]
    run = shard.plan_pairs(list(range(len(boxes))), len(job_ligs), world)[rank]
    my_pockets = sorted({p for _, p, _ in run})              # this rank builds only these maps
    local_pocket = {p: i for i, p in enumerate(my_pockets)}
    my_ligs = sorted({l for l, _, _ in run})
    local_lig = {l: i for i, l in enumerate(my_ligs)}
    ligs = [ctx.ligand(job_ligs[l]) for l in my_ligs]
    lig = ligs[0]
    types = sorted(set(int(t) for l in ligs for t in l.xs_types.tolist()))
    dev_rec = S.Receptor(torch.tensor(rec.xyz, dtype=torch.float32, device="cuda"),
                         torch.tensor(rec.element, device="cuda"), torch.tensor(rec.donor, device="cuda"),
                         torch.tensor(rec.acceptor, device="cuda"))
    my_boxes = [boxes[p] for p in my_pockets]
    pair_lig = [local_lig[l] for l, _, _ in run]
    pair_pocket = [local_pocket[p] for _, p, _ in run]
    params = api.DockParams(chains=CHAINS, steps=STEPS, seed=0, top_k=TOP_K, host_copy=False, focc=args.focc,
                            pair_keys=[k for _, _, k in run])
    if args.shape:   # a fixed launch shape instead of the autotuner's (for profiler captures)
        v, wc, lay = (int(x) for x in args.shape.split(","))
        params = dataclasses.replace(params, search_variant=v, warps_per_cta=wc, map_layout=lay)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(mid=None):
        # the maps in both layouts: the autotuner picks the one the search reads
        gs = ctx.build_grids(dev_rec, my_boxes, types).pack()
        if mid is not None:
            mid.record(stream)
        if world == 1:
            r = ctx.dock(gs, ligs, list(range(len(my_boxes))), params)
        else:
            r = ctx.dock_pairs(gs, ligs, pair_lig, pair_pocket, params)
        return gs, r

    def exchange(r):
        """The job's one exchange step: every rank's ranked kept poses, with global pocket ids,
        gathered and merged per ligand on rank 0 (host records; no data-path collective)."""
        recs = shard.records_from_result(r, my_ligs)
        recs = {l: [(sc, my_pockets[p], c) for sc, p, c in v] for l, v in recs.items()}
        return shard.gather_merge(recs) if world > 1 else shard.merge_records([recs])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    times, grid_t, map_kernel_s, search_s, evals, launches = [], [], 0.0, 0.0, 0, 0
    e0, em, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    merged = None
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()                                  # L2 flushed between timed steps
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            e0.record(stream)
            gs, r = step(em)
            if world > 1:
                merged = exchange(r)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
            grid_t.append(e0.elapsed_time(em) * 1e-3)
            map_kernel_s += gs.build_seconds()
            ev, _, st = r.stats()
            assert (st == 0).all(), st
            s_s, n_l, _ = r.timing()
            shape = r.launch_shape()
            layout = r.map_layout()
            search_s += s_s
            launches += n_l
            evals += ev
    if world == 1:
        merged = exchange(r)
    # search quality of the last timed step: per pocket, the best SF over its chains
    _, chain_best = r.chain_records()
    best_sf = chain_best.min(axis=1)
    step_t = np.array(times)
    if world > 1:
        t = torch.tensor(step_t, device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_t = t.cpu().numpy()
    n_pairs = len(run)
    total_t = float(step_t.sum())
    job_pairs = len(job_ligs) * len(boxes)
    value = job_pairs * args.steps / total_t
    clocks = clk.summary()

    out = None
    if rank == 0:
        flops, gbytes = lig.cost()
        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
        max_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        peak_tflops = n_sm * 128 * 2 * max_mhz * 1e6 / 1e12
        achieved = evals * flops / search_s / 1e12
        prof = stored_profile()
        launch_traffic = prof.get("traffic")
        evals_per_launch = evals / max(launches, 1)
        n_rounds = launches // max(args.steps, 1)
        # the gather alone over the pockets' map set, in both layouts; the search's gathers are
        # compared with the higher of the two ceilings
        gather = {lay: ctx.measure_gather(gs, -1, n_points=1 << 24, reps=10, layout=lay)[2] for lay in (0, 1)}
        gather_gbs = max(gather.values())
        search_gather_gbs = evals * gbytes / search_s / 1e9
        # the map build (Grid_cache): (node, receptor atom within 8 A, type) term evaluations
        terms = grid_term_count(torch, rec.xyz, my_boxes, len(types))
        map_s = map_kernel_s / args.steps
        out = {
            "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_t / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "pairs_per_step": job_pairs, "pairs_per_step_per_gpu": n_pairs,
                       "chains": CHAINS, "mc_steps": STEPS, "top_k": TOP_K, "ligand_atoms": lig.n_atoms,
                       "ligand_torsions": lig.n_rot, "intra_pairs": lig.n_pairs,
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "inputs": "receptor, ligand and boxes resident in HBM; grids rebuilt every step",
                       "parallelism": ("1 GPU" if world == 1 else
                                       f"{world} GPUs: {world} ligands x 10 pockets split into equal pocket-major "
                                       "runs of pairs (job-wide pair keys), ranked poses gathered and merged on "
                                       "rank 0 inside the timed step"),
                       "search_launch": {"variant": shape[0], "warps_per_cta": shape[1], "chains_per_warp": 2 if shape[0] >= 4 else 1,
                                         "map_layout": "cell-packed" if layout == 1 else "plain"},
                       "focc": args.focc},
            "best_sf_per_pocket": {"mean": round(float(best_sf.mean()), 4), "min": round(float(best_sf.min()), 4)},
            "top_pose": {str(l): list(v[0]) for l, v in sorted(merged.items())} if merged else None,
            "evals_per_s": round(evals / total_t * world, 1),
            "breakdown": {"grid_maps_ms": round(float(np.mean(grid_t)) * 1e3, 3),
                          "map_kernel_ms": round(map_s * 1e3, 3),
                          "dock_ms": round((total_t / args.steps - float(np.mean(grid_t))) * 1e3, 3),
                          "dock_only_pairs_per_s": round(n_pairs * world / (total_t / args.steps - float(np.mean(grid_t))), 4)},
            "evals_per_step_per_gpu": evals // max(args.steps, 1),
            "roofline": {"kernel": "search_round_kernel", "bound": "alu", "achieved": round(achieved, 3),
                         "peak": round(peak_tflops, 2), "unit": "TFLOP/s", "frac": round(achieved / peak_tflops, 4),
                         "traffic": (round(launch_traffic) if launch_traffic else None),
                         "peak_source": f"FP32 FMA peak = {n_sm} SMs x 128 lanes x 2 x {max_mhz:.0f} MHz",
                         "flops_per_eval": flops, "evals_per_launch": round(evals_per_launch),
                         "launch_ms": round(search_s / max(launches, 1) * 1e3, 3),
                         "l2_gather_gbs": round(search_gather_gbs, 1),
                         "gather_ceiling_gbs": round(gather_gbs, 1),
                         "gather_ceiling_by_layout_gbs": {"plain": round(gather[0], 1), "cell_packed": round(gather[1], 1)},
                         "gather_frac": round(search_gather_gbs / gather_gbs, 4),
                         "issue": ({"warp_inst_per_eval": prof["inst"],
                                    "achieved_ginst_s": round(evals / search_s * prof["inst"] / 1e9, 1),
                                    "peak_ginst_s": round(n_sm * 4 * max_mhz * 1e6 / 1e9, 1),
                                    "frac": round(evals / search_s * prof["inst"] / (n_sm * 4 * max_mhz * 1e6), 4),
                                    "note": "warp instructions issued per second vs 4 per SM per clock"}
                                   if "inst" in prof else None)},
            "grid_roofline": {"kernel": "grid_kernel", "bound": "alu",
                              "term_evals_per_launch": terms, "flops_per_term": GRID_FLOPS_PER_TERM,
                              "achieved": round(terms * GRID_FLOPS_PER_TERM / map_s / 1e12, 3),
                              "peak": round(peak_tflops, 2), "unit": "TFLOP/s",
                              "frac": round(terms * GRID_FLOPS_PER_TERM / map_s / 1e12 / peak_tflops, 4),
                              "term_evals_per_s": round(terms / map_s, 1), "launch_ms": round(map_s * 1e3, 3),
                              "traffic": (round(stored_grid_profile()) if stored_grid_profile() else None)},
            # per step: typing, 4 binning launches and the map build; one cell-packing launch per
            # pocket; the start stamp, the search rounds, top-k and merge
            "gpu_launches": args.steps * (6 + len(my_boxes) + 1 + n_rounds + 2),
            "clocks": clocks,
        }
        if not args.no_plain:
            out["plain"] = run_plain(ctx, api, gs, lig, list(range(len(my_boxes))), (shape[0], shape[1], layout))
            out["batched_vs_plain"] = round(value / world / out["plain"]["thread_per_chain"]["value"], 2)
            out["batched_vs_plain_warp"] = round(value / world / out["plain"]["warp_per_chain"]["value"], 2)
        if not args.no_micro:
            out["score_microbench"] = run_score_microbench(ctx, api, torch)
        out["rescoring"] = run_rescore_check(ctx, gs, lig, list(range(len(my_boxes))), params)
        if world == 1:
            out["e2e"] = run_e2e(ctx, api, torch, rec, boxes, lig_src, types, list(range(len(boxes))), args.steps, 0,
                                 focc=args.focc)
        if world == 1 and not args.no_cpu:
            out["cpu_baseline"] = run_cpu_baseline(rec, boxes, lig_src, budget_s=args.cpu_budget)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


def run_plain(ctx, api, gs, lig, pockets, shape):
    """The paper's organisation, one launch per pair and a host loop, on one pocket of the
    workload at its full length (1,000 chains x 2,000 MC steps, not extrapolated), in two forms:
    thread per chain (as in the paper's engine) and warp per chain (the batched path's own chain
    kernel and launch shape, one launch per pair with all steps in one block, no queue across pairs,
    no graph), so that the second ratio isolates what batching itself adds."""
    out = {"sample": f"1 pocket x {CHAINS} chains x {STEPS} MC steps, one launch per pair, timed in full"}
    for name, kw in (("thread_per_chain", dict(mode="plain")),
                     ("warp_per_chain", dict(mode="plain_warp", search_variant=shape[0], warps_per_cta=shape[1],
                                             map_layout=shape[2]))):
        r = ctx.dock(gs, [lig], [pockets[0]], chains=CHAINS, steps=STEPS, seed=0, host_copy=False, **kw)
        ev, _, st = r.stats()
        assert (st == 0).all(), st
        s_s, _, total = r.timing()
        out[name] = {"value": round(1.0 / total, 5), "unit": UNIT, "seconds_per_pair": round(total, 4),
                     "evals_per_s": round(ev / s_s, 1)}
    return out


def grid_term_count(torch, rec_xyz, boxes, n_types, chunk=4096):
    """Algorithmic work of the map build: (grid node, receptor atom within 8 A, ligand type)
    triples over all boxes, counted on the GPU (torch arithmetic, measurement only)."""
    import math as _m
    atoms = torch.as_tensor(np.asarray(rec_xyz, np.float32), device="cuda")
    total = 0
    for b in boxes:
        sp = float(np.float32(b.spacing))
        size = np.asarray(b.size, np.float64)
        dims = [int(_m.ceil(float(np.float32(size[k])) / sp - 1e-9)) + 1 for k in range(3)]
        origin = np.asarray(np.float32(np.asarray(b.center, np.float32) - np.float32(size / 2)), np.float64)
        ax = [torch.tensor(origin[k] + sp * np.arange(dims[k]), dtype=torch.float32, device="cuda") for k in range(3)]
        near = atoms[((atoms - torch.tensor(origin + 0.5 * sp * (np.array(dims) - 1), dtype=torch.float32,
                                            device="cuda")).abs() <= torch.tensor(0.5 * sp * (np.array(dims) - 1) + 8.0,
                                                                                  dtype=torch.float32, device="cuda")).all(1)]
        zz, yy, xx = torch.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        nodes = torch.stack([xx.reshape(-1), yy.reshape(-1), zz.reshape(-1)], 1)
        for i in range(0, nodes.shape[0], chunk):
            d2 = ((nodes[i:i + chunk, None, :] - near[None, :, :]) ** 2).sum(-1)
            total += int((d2 < 64.0).sum())
    return total * n_types


def run_rescore_check(ctx, gs, lig, pockets, params):
    """One untimed dock of the workload with rescoring of the kept poses by direct summation over
    the receptor: the grid's interpolation error on the final poses (e_inter grid vs direct)."""
    import dataclasses
    r = ctx.dock(gs, [lig], pockets, dataclasses.replace(params, rescore=True, host_copy=True))
    err = []
    for q in range(r.n_pairs):
        n = int(r.n_kept[q])
        err.extend(np.abs(r.poses[q]["e_inter"][:n] - r.poses[q]["e_inter_grid"][:n]).tolist())
    err = np.array(err)
    return {"kept_poses": int(len(err)), "mean_abs_e_inter_grid_error": round(float(err.mean()), 5),
            "max_abs_e_inter_grid_error": round(float(err.max()), 5), "unit": "kcal/mol"}


def run_score_microbench(ctx, api, torch, reps=20):
    """Score + adjoint gradient over 65,536 random poses of a 32-atom / 8-torsion ligand in a 24 A
    box of a 4,000-atom receptor (L2-resident maps: the gather is L2-bound by design)."""
    rec, box, lig_src, poses = S.score_microbench()
    lig = ctx.ligand(lig_src)
    # with the cell-packed copy, which the score calls read when the set holds it
    gs = ctx.build_grids(rec, [box], sorted(set(lig.xs_types.tolist()))).pack()
    p = torch.tensor(poses, dtype=torch.float32, device="cuda")
    for _ in range(3):
        ctx.score(gs, lig, 0, p)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(reps):
        ctx.score(gs, lig, 0, p)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) * 1e-3 / reps
    flops, gbytes = lig.cost()
    n = len(poses)
    # the gather step alone on the same maps, in both layouts: the faster bounds the score kernel's
    # gather
    probes = {name: ctx.measure_gather(gs, 0, n_points=1 << 24, reps=10, layout=lay)
              for name, lay in (("plain", 0), ("cell_packed", 1))}
    _, g_pts, g_gbs = max(probes.values(), key=lambda t: t[2])
    l2 = n * gbytes / dt / 1e9
    return {"evals_per_s": round(n / dt, 1), "ms_per_launch": round(dt * 1e3, 4), "poses": n,
            "map_layout": "cell-packed", "achieved_tflops": round(n * flops / dt / 1e12, 3),
            "l2_gather_gbs": round(l2, 1),
            "gather_probe": {"gbs": round(g_gbs, 1), "interpolations_per_s": round(g_pts, 1),
                             "by_layout_gbs": {k: round(v[2], 1) for k, v in probes.items()},
                             "note": "trilinear value + gradient alone, hashed positions in the box, 32 B per point"},
            "gather_frac": round(l2 / g_gbs, 4)}


def run_e2e(ctx, api, torch, rec, boxes, lig_src, types, pockets, steps, seed, focc=0):
    """The same metric through the public API from pinned host buffers: every step uploads the
    receptor and ligand, builds the grids, docks, and reads the ranked poses back."""
    pin = {k: torch.tensor(np.asarray(getattr(rec, k), dtype=np.float32 if k == "xyz" else np.uint8)).pin_memory()
           for k in ("xyz", "element", "donor", "acceptor")}
    host_rec = S.Receptor(pin["xyz"], pin["element"], pin["donor"], pin["acceptor"])
    h2d = sum(t.numel() * t.element_size() for t in pin.values())
    h2d += sum(np.asarray(a).nbytes for a in (np.asarray(lig_src.xyz, np.float32), lig_src.element, lig_src.donor,
                                              lig_src.acceptor, np.asarray(lig_src.bonds, np.int32), lig_src.rotatable))
    d2h = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        gs = ctx.build_grids(host_rec, boxes, types).pack()
        lig = ctx.ligand(lig_src)
        r = ctx.dock(gs, [lig], pockets, chains=CHAINS, steps=STEPS, seed=seed, top_k=TOP_K, host_copy=True,
                     focc=focc)
        poses, kept, pots, xyz = r.fetch()
        rank = r.ranking(0)
        d2h = (poses.nbytes + kept.nbytes + pots.nbytes + xyz.nbytes + rank.nbytes)
    dt = time.perf_counter() - t0
    return {"value": round(len(pockets) * steps / dt, 4), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h)}


# ----------------------------------------------------------------- oracle (CPU) arm --
def oracle_sample(rec, boxes, lig_src, budget_s=12.0):
    """Times the FP64 oracle on a bounded sample of one pair: the grid maps of one pocket, then
    chains of the full 2,000-step search; returns seconds per docked pair (extrapolated to the
    1,000 chains of the workload) and the sample description."""
    import oracle as O
    cores = len(os.sched_getaffinity(0))
    L = O.OracleLigand(lig_src)
    box = boxes[0]
    t0 = time.perf_counter()
    og = O.OracleGrid(rec, box, L.xs, rec_types=O.xs_type_receptor(rec), threads=cores)
    t_grid = time.perf_counter() - t0
    # calibrate on one chain-batch of one MC step block, then size the sample to the budget
    p = O.SearchParams(seed=0, steps=STEPS)
    n_chains = cores
    t0 = time.perf_counter()
    _, _, ev = O.mc_chains(L, og, box, O.SearchParams(seed=0, steps=50), unit=0, n_chains=n_chains, threads=cores)
    t_cal = time.perf_counter() - t0
    per_chain_full = t_cal / n_chains * (STEPS / 50) * cores     # core-seconds per full chain
    fit = max(1, int((budget_s - t_grid) * cores / max(per_chain_full, 1e-9)))
    n_chains = int(min(CHAINS, max(cores, (fit // cores) * cores)))
    t0 = time.perf_counter()
    _, _, ev = O.mc_chains(L, og, box, p, unit=0, n_chains=n_chains, threads=cores)
    t_dock = time.perf_counter() - t0
    per_pair = t_grid + t_dock * CHAINS / n_chains
    # one core: two chains of 100 MC steps
    t0 = time.perf_counter()
    _, _, ev1 = O.mc_chains(L, og, box, O.SearchParams(seed=1, steps=100), unit=0, n_chains=2, threads=1)
    single_core_evals_s = float(ev1.sum()) / (time.perf_counter() - t0)
    sample = (f"1 pocket: full FP64 grid maps ({len(set(L.xs.tolist()))} types) + {n_chains} of {CHAINS} "
              f"chains x {STEPS} MC steps; time scaled x {CHAINS / n_chains:.1f} to the pair")
    return per_pair, float(ev.sum()) / t_dock, cores, sample, t_grid + t_dock, single_core_evals_s


def run_cpu_baseline(rec, boxes, lig_src, budget_s=12.0):
    per_pair, evals_s, cores, sample, _, single = oracle_sample(rec, boxes, lig_src, budget_s)
    return {"value": round(1.0 / per_pair, 6), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "evals_per_s": round(evals_s, 1), "single_core_evals_per_s": round(single, 1)}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return None
    import oracle as O
    O.build()
    rec, boxes, lig_src = workload(seed=0)
    for _ in range(args.warmup):   # untimed: short samples (page in code and data)
        oracle_sample(rec, boxes, lig_src, budget_s=1.0)
    times, last = [], None
    for _ in range(args.steps):
        last = oracle_sample(rec, boxes, lig_src, budget_s=args.cpu_budget)
        times.append(last[0])
    per_pair = float(np.mean(times))
    value = 1.0 / per_pair
    cores, sample = last[2], last[3]
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_pair * len(boxes) * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "pairs_per_step_per_gpu": len(boxes)},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_batch_workload(args):
    """The uneven-batch and screening shapes (one GPU), each step building every grid map and
    docking every pair in one batched call; its own JSON line (pairs/s, evals/s, the search
    kernel's roofline). uneven: a 6,000-atom receptor with 5 pockets x 512 ligands of 10-60 atoms and
    0-15 torsions, 64 chains x 1,000 MC steps per pair. screening: 256 receptors of 1,500-8,000
    atoms with 3 pockets each (768 pockets of maps resident in HBM), --ligands-per-receptor
    30-atom / 6-torsion ligands docked into their receptor's 3 pockets, 32 chains x 1,000 steps."""
    import torch
    import paper_2506_20043_gb300 as pv
    pv.build()
    from paper_2506_20043_gb300 import api
    ctx = api.Context(0)
    t_gen = time.perf_counter()
    if args.workload == "tiny":
        w = S.tiny()
        recs, boxes = w.receptors, w.boxes
        pair_lig, pair_pocket = [0], [0]
        desc = ("tiny: 2,000-atom receptor, one 8 A pocket in a 20 A box (0.375 A), one ligand of 20 atoms / "
                "4 torsions, 8 chains x 1,000 MC steps")
    elif args.workload == "boxsweep":
        w = S.box_sweep(seed=0)
        recs, boxes = w.receptors, w.boxes
        pair_lig = [0] * len(boxes[0])
        pair_pocket = list(range(len(boxes[0])))
        desc = ("box sweep: 5,000-atom receptor, its 5 top-ranked pockets each in boxes of 15-30 A by 1 A "
                "(80 boxes, 0.375 A), one ligand of 30 atoms / 6 torsions, 256 chains x 1,000 MC steps, top-9")
    elif args.workload == "uneven":
        w = S.uneven(seed=0)
        recs, boxes = w.receptors, w.boxes
        pair_lig = [li for li in range(len(w.ligands)) for _ in range(len(boxes[0]))]
        pair_pocket = [p for _ in range(len(w.ligands)) for p in range(len(boxes[0]))]
        desc = ("uneven batch: 6,000-atom receptor, 5 pockets (24 A boxes), 512 ligands of 10-60 atoms and "
                "0-15 torsions, 64 chains x 1,000 MC steps per pair, top-9")
    else:
        w = S.screening(seed=0, ligands_per_receptor=args.ligands_per_receptor)
        recs, boxes = w.receptors, w.boxes
        pair_lig, pair_pocket = [], []
        for r, ids in enumerate(w.ligands_per_receptor):
            for li in ids:
                for p in range(len(boxes[r])):
                    pair_lig.append(li)
                    pair_pocket.append(3 * r + p)
        desc = (f"screening: 256 receptors of 1,500-8,000 atoms, 3 pockets each (768 x 24 A boxes), "
                f"{args.ligands_per_receptor} ligands of 30 atoms / 6 torsions per receptor into its 3 pockets, "
                f"32 chains x 1,000 MC steps, top-9")
    t_gen = time.perf_counter() - t_gen
    ligs = [ctx.ligand(l) for l in w.ligands]
    types = sorted(set(int(t) for l in ligs for t in l.xs_types.tolist()))
    dev_recs = [S.Receptor(torch.tensor(r.xyz, dtype=torch.float32, device="cuda"), torch.tensor(r.element, device="cuda"),
                           torch.tensor(r.donor, device="cuda"), torch.tensor(r.acceptor, device="cuda")) for r in recs]
    params = api.DockParams(chains=w.chains, steps=w.steps, seed=0, top_k=w.top_k, host_copy=False)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = ctx.stream

    def step():
        # both map layouts (appended receptors are packed too): the autotuner picks the one it reads
        gs = ctx.build_grids(dev_recs[0], boxes[0], types).pack()
        for r in range(1, len(recs)):
            gs.append(dev_recs[r], boxes[r])
        return gs, ctx.dock_pairs(gs, ligs, pair_lig, pair_pocket, params)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times, evals, search_s, map_bytes = [], 0, 0.0, 0
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0.record(stream)
            gs, r = step()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
            ev, _, st = r.stats()
            assert (st == 0).all(), st
            s_s, _, _ = r.timing()
            evals += ev
            search_s += s_s
            shape = r.launch_shape()
            layout = r.map_layout()
            map_bytes = gs.bytes
    total_t = float(np.sum(times))
    n_pairs = len(pair_lig)
    extra = {}
    if args.workload == "boxsweep":
        _, es = r.chain_records()
        best = es.min(axis=1).reshape(-1, 16)            # [pocket, size]
        extra["best_sf_by_box_size"] = {f"{15 + k} A": round(float(best[:, k].mean()), 3) for k in range(16)}
    # roofline of the search kernel: the pair-weighted mean cost of the batch's ligands
    costs = [l.cost() for l in ligs]
    w_flops = float(np.mean([costs[li][0] for li in pair_lig]))
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    clocks = clk.summary()
    max_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = n_sm * 128 * 2 * max_mhz * 1e6 / 1e12
    achieved = evals * w_flops / search_s / 1e12
    return {"metric": METRIC, "value": round(n_pairs * args.steps / total_t, 3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_t / args.steps * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "pairs_per_step": n_pairs, "ligands": len(ligs), "pockets": gs.n_pockets,
                       "map_bytes": int(map_bytes), "chains": w.chains, "mc_steps": w.steps,
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "inputs": "receptors and ligands resident in HBM; grids rebuilt every step",
                       "search_launch": {"variant": shape[0], "warps_per_cta": shape[1],
                                         "map_layout": "cell-packed" if layout == 1 else "plain"},
                       "host_generation_s": round(t_gen, 1)},
            "evals_per_s": round(evals / total_t, 1), "search_s_per_step": round(search_s / args.steps, 3),
            "roofline": {"kernel": "search_round_kernel", "bound": "alu", "achieved": round(achieved, 3),
                         "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                         "flops_per_eval": round(w_flops, 1)},
            "clocks": clocks, **extra,
            "cpu_baseline": (None if args.no_cpu else
                             oracle_pairs_sample(w, pair_lig, pair_pocket, args.workload, budget_s=args.cpu_budget,
                                                 n_pairs=1 if len(pair_lig) == 1 else 3))}


def run_pocket_workload(args):
    """Pocket prediction (Supplementary Algorithm 1, Steps 1, 2, 4, 5; the classifier of Step 3 is
    replaced by a synthetic score given as input): each step takes 16 receptors of 8,000 atoms
    with 10 carved pockets each to SAS points (100 lattice points per atom, 1.6 A probe, Bondi
    radii), their Eq. 1 sums over 7 property columns with the protrusion count, and the ranked
    single-linkage clusters of the points scoring >= 0.5 (surfaces and clusters of the 16 receptors
    in one batched call each). Its own JSON line: receptors/s, with the feature kernel's roofline."""
    import torch
    import paper_2506_20043_gb300 as pv
    pv.build()
    from paper_2506_20043_gb300 import api
    ctx = api.Context(0)
    n_rec, n_atoms, n_pockets = 16, 8000, 10
    prm = api.PocketParams(n_sphere=100)
    sites = [S.pocket_site(seed, n_atoms, n_pockets) for seed in range(n_rec)]
    dev = torch.device("cuda", 0)
    recs = [S.Receptor(torch.tensor(s.receptor.xyz, dtype=torch.float32, device=dev),
                       torch.tensor(s.receptor.element, device=dev), torch.tensor(s.receptor.donor, device=dev),
                       torch.tensor(s.receptor.acceptor, device=dev)) for s in sites]
    host_recs = [S.Receptor(np.asarray(s.receptor.xyz, np.float32), s.receptor.element, s.receptor.donor,
                            s.receptor.acceptor) for s in sites]
    props_h = [S.atom_properties(s.receptor, i) for i, s in enumerate(sites)]
    props = [torch.tensor(p, device=dev) for p in props_h]
    # the stand-in scores of every receptor's points (an input of Step 4, computed once)
    scores_h = []
    for i, r in enumerate(recs):
        surf = ctx.surface(r, params=prm)
        scores_h.append(S.ligandability(surf.points().cpu().numpy(), sites[i], i))
    scores = [torch.tensor(x, device=dev) for x in scores_h]
    stream = ctx.stream
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    feat_ms = []

    def step():
        # the 16 receptors' surfaces in one call, their features, their clusters in one call
        surfs = ctx.surfaces(recs, params=prm)
        feats = [s.features(props[i], params=prm) for i, s in enumerate(surfs)]
        cls = ctx.cluster_many([(s, scores[i]) for i, s in enumerate(surfs)], prm)
        return [(surfs[i], feats[i][0], feats[i][1], cls[i]) for i in range(n_rec)]

    def step_e2e():
        h2d = d2h = 0
        surfs = ctx.surfaces(host_recs, params=prm)
        feats = [s.features(props_h[i], params=prm) for i, s in enumerate(surfs)]
        cls = ctx.cluster_many([(s, scores_h[i]) for i, s in enumerate(surfs)], prm)
        for i in range(n_rec):
            r = host_recs[i]
            res = cls[i].read()
            feat_h = feats[i][0].cpu().numpy()
            h2d += r.xyz.nbytes + r.element.nbytes + props_h[i].nbytes + scores_h[i].nbytes
            d2h += feat_h.nbytes + sum(v.nbytes for v in res.values()) + 8
        return h2d, d2h

    for _ in range(args.warmup):
        out = step()
    torch.cuda.synchronize()
    n_points = sum(o[0].n_points for o in out)
    n_clusters = [o[3].n_clusters for o in out]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
        e2e_t = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h2d, d2h = step_e2e()
            torch.cuda.synchronize()
            e2e_t.append(time.perf_counter() - t0)
    clocks = clk.summary()
    # the feature kernel alone (events around its one launch), and its algorithmic work: the
    # distance test of every (point, atom) pair within r_protrusion, plus the weight and the
    # 2 x 7 property FLOPs of every pair within r_feature (counted with r_protrusion = r_feature)
    # 20 back-to-back launches per receptor through the C ABI (outputs preallocated), so that the
    # events time the kernel rather than the host's call overhead
    import ctypes as C
    cp = prm.to_c()
    reps = 20
    for i in range(n_rec):
        surf = out[i][0]
        feat = torch.empty((surf.n_points, props[i].shape[1]), dtype=torch.float32, device=dev)
        prot = torch.empty(surf.n_points, dtype=torch.int32, device=dev)
        args_c = (ctx.h, surf.h, surf.n_points, None, 1, int(props[i].shape[1]), props[i].data_ptr(), 1, C.byref(cp),
                  feat.data_ptr(), prot.data_ptr())
        ctx.lib.pv_surface_features(*args_c)
        f0.record(stream)
        for _ in range(reps):
            ctx.lib.pv_surface_features(*args_c)
        f1.record(stream)
        f1.synchronize()
        feat_ms.append(f0.elapsed_time(f1) / reps)
    feat_s = float(np.mean(feat_ms)) * 1e-3
    # host-clocked phases of one receptor through the single-receptor calls (each call ends
    # synchronised here)
    phase = {"surface": [], "features": [], "clusters": []}
    for i in range(n_rec):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        surf = ctx.surface(recs[i], params=prm)
        t1 = time.perf_counter()
        surf.features(props[i], params=prm)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        ctx.cluster(surf.points(), scores[i], prm)
        t3 = time.perf_counter()
        phase["surface"].append(t1 - t0)
        phase["features"].append(t2 - t1)
        phase["clusters"].append(t3 - t2)
    breakdown = {k: round(float(np.mean(v)) * 1e3, 4) for k, v in phase.items()}
    pairs10 = pairs6 = 0
    n6 = api.PocketParams(n_sphere=100, r_protrusion=6.0)
    for i in range(n_rec):
        surf = out[i][0]
        pairs10 += int(out[i][2].to(torch.int64).sum())
        pairs6 += int(surf.features(props[i][:, :1], params=n6)[1].to(torch.int64).sum())
    flops = (pairs10 * 8 + pairs6 * (4 + 2 * 7)) / n_rec
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    max_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = n_sm * 128 * 2 * max_mhz * 1e6 / 1e12
    achieved = flops / feat_s / 1e12
    total_t = float(np.sum(times))
    cpu = None
    if not args.no_cpu:
        import oracle as O
        s0 = sites[0]
        rec = s0.receptor
        xyz = np.asarray(rec.xyz, np.float32).astype(np.float64)
        rad = np.asarray(S.vdw_radii(rec), np.float32).astype(np.float64)
        t0 = time.perf_counter()
        keep, pts, _ = O.sas_points(xyz, rad, prm.probe, prm.n_sphere)
        pts = pts[keep == 1]
        O.point_features(xyz, props_h[0].astype(np.float64), pts)
        O.cluster_points(pts, S.ligandability(pts, s0, 0).astype(np.float64), prm.threshold, prm.link)
        dt = time.perf_counter() - t0
        cpu = {"value": round(1.0 / dt, 4), "unit": "receptors/s", "cores": len(os.sched_getaffinity(0)),
               "kind": "oracle", "sample": "one whole 8,000-atom receptor: FP64 SAS points, Eq. 1 sums and "
                                           "protrusion at its points, clusters (brute force over all pairs)"}
    return {"metric": "pocket predictions/sec (SAS points, Eq. 1 features, Eq. 2 clusters) at 1 GB300",
            "value": round(n_rec * args.steps / total_t, 2), "unit": "receptors/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_t / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "pocket prediction: 16 receptors of 8,000 atoms (0.05 per cubic A) with 10 carved "
                                   "pockets each; 100 lattice points per atom, 1.6 A probe, Bondi radii; Eq. 1 over 7 "
                                   "property columns (6 A), protrusion (10 A); clusters of points scoring >= 0.5 "
                                   "(synthetic score), 3 A single linkage; surfaces and clusters of the 16 receptors in one "
                                   "batched call each",
                       "points_per_receptor": round(n_points / n_rec, 1),
                       "clusters_per_receptor": round(float(np.mean(n_clusters)), 1),
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "inputs": "receptors, property columns and scores resident in HBM"},
            "points_per_s": round(n_points * args.steps / total_t, 1),
            "single_calls_ms_per_receptor": breakdown,
            "roofline": {"kernel": "feature_kernel", "bound": "alu", "achieved": round(achieved, 4),
                         "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 5),
                         "traffic": None, "launch_ms": round(feat_s * 1e3, 4),
                         "flops_per_launch": round(flops, 1)},
            "e2e": {"value": round(n_rec * args.steps / float(np.sum(e2e_t)), 2), "unit": "receptors/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "clocks": clocks, "cpu_baseline": cpu}


def oracle_pairs_sample(w, pair_lig, pair_pocket, name, budget_s=12.0, n_pairs=3, seed=7):
    """The FP64 oracle on a seeded sample of the workload's pairs: for each sampled pair, the
    pocket's full grid maps (their cost shared by the pairs docked into that pocket) and as many
    full-length chains as fit the budget, extrapolated to the pair's chain count."""
    import oracle as O
    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(seed)
    picks = rng.choice(len(pair_lig), size=min(n_pairs, len(pair_lig)), replace=False)
    rec_of = []
    for r, bx in enumerate(w.boxes):
        rec_of += [r] * len(bx)
    flat_boxes = [b for bx in w.boxes for b in bx]
    pairs_per_pocket = np.bincount(np.asarray(pair_pocket), minlength=len(flat_boxes))
    per_pair, evals, secs, chains_run = [], 0, 0.0, []
    for q in picks:
        L = O.OracleLigand(w.ligands[pair_lig[q]])
        k = pair_pocket[q]
        rec, box = w.receptors[rec_of[k]], flat_boxes[k]
        t0 = time.perf_counter()
        og = O.OracleGrid(rec, box, L.xs, rec_types=O.xs_type_receptor(rec), threads=cores)
        t_grid = time.perf_counter() - t0
        t0 = time.perf_counter()
        _, _, ev = O.mc_chains(L, og, box, O.SearchParams(seed=0, steps=min(w.steps, 50)), unit=int(q),
                               n_chains=cores, threads=cores)
        per_chain = (time.perf_counter() - t0) / cores * (w.steps / min(w.steps, 50)) * cores
        n_ch = int(min(w.chains, max(cores, (budget_s / n_pairs) * cores / max(per_chain, 1e-9) // cores * cores)))
        t0 = time.perf_counter()
        _, _, ev = O.mc_chains(L, og, box, O.SearchParams(seed=0, steps=w.steps), unit=int(q), n_chains=n_ch,
                               threads=cores)
        t_dock = time.perf_counter() - t0
        per_pair.append(t_grid / pairs_per_pocket[k] + t_dock * w.chains / n_ch)
        evals += int(ev.sum())
        secs += t_dock
        chains_run.append(n_ch)
    value = 1.0 / float(np.mean(per_pair))
    return {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"{len(picks)} seeded pairs of the {name} workload: each pocket's full FP64 grid maps "
                       f"(shared by its {int(np.median(pairs_per_pocket[pairs_per_pocket > 0]))} pairs) + "
                       f"{'/'.join(map(str, chains_run))} of {w.chains} chains x {w.steps} MC steps, scaled to the pair"),
            "evals_per_s": round(evals / secs, 1)}


def run_small_case(args):
    """One short untimed pass for profiler captures: the multi-pocket workload (10 pockets x 1,000
    chains) for --small-steps MC steps in one search launch with a fixed launch shape (--variant,
    --warps; no autotuning), plus one score launch over the 65,536 microbenchmark poses."""
    import torch
    import paper_2506_20043_gb300 as pv
    pv.build()
    from paper_2506_20043_gb300 import api
    ctx = api.Context(0)
    rec, boxes, lig_src = workload(seed=0)
    lig = ctx.ligand(lig_src)
    gs = ctx.build_grids(rec, boxes, sorted(set(lig.xs_types.tolist())))
    if args.layout == 1:
        gs.pack()
    r = ctx.dock(gs, [lig], list(range(len(boxes))), chains=CHAINS, steps=args.small_steps, seed=0, host_copy=False,
                 search_variant=args.variant, warps_per_cta=args.warps, steps_per_round=args.small_steps,
                 map_layout=args.layout)
    ev, sec, st = r.stats()
    mrec, mbox, mlig_src, mposes = S.score_microbench()
    mlig = ctx.ligand(mlig_src)
    mgs = ctx.build_grids(mrec, [mbox], sorted(set(mlig.xs_types.tolist())))
    ctx.score(mgs, mlig, 0, torch.tensor(mposes, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    s_s, _, _ = r.timing()
    return {"case": "small", "evals": int(ev), "seconds": round(sec, 4), "search_seconds": round(s_s, 5),
            "evals_per_s": round(ev / s_s, 1), "launch": r.launch_shape(), "layout": r.map_layout(),
            "status_ok": bool((st == 0).all())}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work per sample")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-micro", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", choices=["multipocket", "tiny", "uneven", "screening", "boxsweep", "pockets"],
                    default="multipocket",
                    help="multipocket: the headline line; uneven / screening / boxsweep: other shapes, their own line")
    ap.add_argument("--focc", type=int, default=0,
                    help="consistency check (Eq. 4-5) with this many neighbours per chain; 0 = off (headline)")
    ap.add_argument("--ligands-per-receptor", type=int, default=10, help="screening: ligands docked per receptor")
    ap.add_argument("--case", choices=["full", "small"], default="full",
                    help="small: one untimed small pass for profiler captures")
    ap.add_argument("--variant", type=int, default=0, help="search kernel variant of --case small")
    ap.add_argument("--warps", type=int, default=2, help="warps per CTA of --case small")
    ap.add_argument("--small-steps", type=int, default=20, help="MC steps of --case small (one launch)")
    ap.add_argument("--layout", type=int, default=0, choices=[0, 1], help="map layout of --case small (1: cell-packed)")
    ap.add_argument("--shape", default="", help="variant,warps,layout: fix the headline's launch shape (profiler "
                                                "captures, whose trials would be profiled too); default autotuned")
    args = ap.parse_args()
    if args.case == "small":
        out = run_small_case(args)
    elif args.workload == "pockets" and args.impl == "ours":
        out = run_pocket_workload(args)
    elif args.workload != "multipocket" and args.impl == "ours":
        out = run_batch_workload(args)
    else:
        out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
