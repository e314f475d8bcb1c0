"""Benchmark of the GB300 octree build: one JSON line on rank 0.

Workload (one step): N = 2^27 particles, float64 coordinates from 1,000 Gaussian clumps
(sigma log-uniform in 1e-4..1e-2 of the box) plus 20% uniform background, float32 log-normal
masses, 63-bit Hilbert keys, Ncrit = 64. A step runs the whole path on the device: bounding cube,
keys, radix sort with permutation, cornerstone leaf loop, linked octree, node-count upsweep and
the FP32 compensated monopole/quadrupole upsweep. Inputs (3.5 GB) are larger than the 129 MB L2,
so no explicit flush is needed between steps.

``--impl reference`` times the plain CPU oracle instead (on every host core, bounded sample of
the same workload); under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_FULL = 1 << 27
NCRIT = 64
SEED = 20230626 + 2
METRIC = "particles/s full octree build (keys->sort->leaves->tree) @1 GB300, % HBM roofline"
WORKLOAD = "2^27 Gaussian clumps + 20% uniform, Hilbert keys, Ncrit=64, with count + multipole upsweep"
CPU_SAMPLE = 1 << 25  # about 8 s of the oracle on 16 Arm cores, plus 5 s single-threaded on a quarter
REF_SAMPLE = 1 << 22  # per step of the reference arm (its --steps K --warmup W run stays within minutes)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N_FULL)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-timesteps", action="store_true")
    p.add_argument("--ts-steps", type=int, default=100)
    p.add_argument("--no-table1", action="store_true")
    p.add_argument("--no-keys30", action="store_true")
    p.add_argument("--no-focus", action="store_true")
    p.add_argument("--no-configs", action="store_true")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(n: int, rank: int = 0):
    from paper_2307_06345_gb300 import workloads as w
    x, y, z = w.clumps(n, SEED + 7919 * rank)
    m = w.lognormal_masses(n, SEED + 1 + 7919 * rank)
    return x, y, z, m


def max_over_ranks(value: float, dist, device=None) -> float:
    """Largest value over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM bytes per particle of the bounding cube, the key pass with multipole records, the sort
# (per-pass tile counts and scans, 8 passes) and the multipole upsweep (leaf sums and levels),
# measured with ncu (dram__bytes_read.sum + dram__bytes_write.sum over the phase's launches) on
# 2^24 particles of the same workload and scaled by the particle count (these phases stream or
# gather per particle, so traffic grows with n).
MEASURED_DRAM_BYTES_PER_PARTICLE = {"bbox": 24.2, "keys": 64.7, "sort": 233.5, "multipoles": 139.8}


def algorithmic_bytes(n: int, n_leaves: int, iter_leaves: int, n_nodes: int):
    """Compulsory DRAM traffic of one step (bytes), by phase."""
    return {
        "bbox": 24 * n,
        "keys": 68 * n,                         # read x, y, z, m; write the key and the 32-byte record
        "sort": (20 + 24 * 7) * n,              # 8 passes (the first has no value read)
        "leaves": 24 * iter_leaves + 8 * n,     # K + pos read/written per pass; P read by searches once
        "link": 40 * n_nodes,
        "counts": 8 * n_nodes,
        "multipoles": 36 * n + 48 * n_nodes,    # record gather + perm; per-node outputs + scratch
    }


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    import paper_2307_06345_gb300 as cs

    cs.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    n = args.n
    x, y, z, m = workload(n, rank)
    X, Y, Z, M = (torch.from_numpy(a).to(dev) for a in (x, y, z, m))
    stream = torch.cuda.current_stream()

    # warm-up (also sizes the buffers)
    out = cs.build_octree(X, Y, Z, curve=cs.HILBERT, ncrit=NCRIT, masses=M)
    buffers = out["buffers"]
    for _ in range(max(args.warmup - 1, 0)):
        out = cs.build_octree(X, Y, Z, curve=cs.HILBERT, ncrit=NCRIT, masses=M, buffers=buffers)
    torch.cuda.synchronize()
    n_leaves, iters = out["n_leaves"], out["iters"]
    n_nodes = cs.n_nodes(n_leaves)

    # per-phase events recorded inside the timed steps (same stream as the library launches)
    phases = ["bbox", "keys", "sort", "leaves", "link", "counts", "multipoles"]
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(phases) + 1)] for _ in range(K)]
    b = buffers

    def step(k):
        e = ev[k]
        e[0].record(stream)
        cs.cstone_bbox(X, Y, Z, b.box, b.ws)
        e[1].record(stream)
        cs.cstone_keys_records(X, Y, Z, M, b.box, cs.HILBERT, b.keys, b.records, b.rws)
        e[2].record(stream)
        cs.cstone_sort(b.keys, b.sorted_keys, b.perm, b.ws)
        e[3].record(stream)
        nl, _ = cs.cstone_build_leaves(b.sorted_keys, NCRIT, b.leaves, b.counts, b.offsets, 0, 64, b.ws)
        e[4].record(stream)
        t = b.tree_buffers(nl)
        cs.cstone_link_tree(b.leaves, nl, t["NK"], t["CO"], t["LO"], t["leaf_to_node"], t["parent"], b.ws)
        e[5].record(stream)
        cs.cstone_upsweep_counts(b.counts, nl, t["leaf_to_node"], t["CO"], t["LO"], t["counts"], b.ws)
        e[6].record(stream)
        cs.cstone_upsweep_multipoles_records(b.records, b.perm, n, b.offsets, nl, t["leaf_to_node"], t["CO"],
                                             t["LO"], b.box, t["mass"], t["com"], t["quad"], b.ws)
        e[7].record(stream)
        return nl

    step(0)  # one more warm-up through the exact timed sequence
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        launches0 = cs.cstone_kernel_launches()
        start.record(stream)
        for k in range(K):
            step(k)
        stop.record(stream)
        launches = cs.cstone_kernel_launches() - launches0  # the library's own count of its launches
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    elapsed_ms = max_over_ranks(start.elapsed_time(stop), dist, dev)
    phase_ms = {p: float(np.mean([ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(K)]))
                for i, p in enumerate(phases)}
    ms_per_step = elapsed_ms / K
    value = world * n / (ms_per_step * 1e-3)

    # roofline of the dominant kernel group: the radix sort (8 digit passes)
    hbm, peak_kind = peaks()
    algo = algorithmic_bytes(n, n_leaves, int(n_leaves * 1.3), n_nodes)
    dom = max(phase_ms, key=phase_ms.get)
    achieved = algo[dom] / (phase_ms[dom] * 1e-3) / 1e9
    step_bytes = sum(algo.values())

    # end to end through the C entry points that take host buffers (cstone_host_stage,
    # cstone_host_build, driven by StreamedBuilder): every step copies its inputs in from pinned host
    # memory and its tree out to pinned host memory; the copy-in of the next step, the build and
    # the copy-out of the previous step overlap on three streams
    e2e = None
    if not args.no_e2e:
        hx, hy, hz, hm = (torch.from_numpy(a).pin_memory() for a in (x, y, z, m))
        sb = cs.StreamedBuilder(n, dev, curve=cs.HILBERT, ncrit=NCRIT)
        sb.run([(hx, hy, hz, hm)] * 2)  # warm-up: sizes both slots' buffers and host outputs
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        # the host link alone (three copies each way of the x coordinates: the best and the worst
        # rate), to read the figure against
        link = {}
        dx = torch.empty(hx.shape, dtype=hx.dtype, device=dev)
        for name, dst, src in (("h2d_gbs", dx, hx), ("d2h_gbs", hx, dx)):
            copy_ms = []
            for _ in range(3):
                l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                l0.record()
                dst.copy_(src, non_blocking=True)
                l1.record()
                torch.cuda.synchronize()
                copy_ms.append(l0.elapsed_time(l1))
            link[name] = hx.numel() * hx.element_size() / (min(copy_ms) * 1e-3) / 1e9
            link[name + "_worst"] = hx.numel() * hx.element_size() / (max(copy_ms) * 1e-3) / 1e9
        del dx
        # three runs of ke streamed steps each; the figure is the run of median time per step (the
        # host link is shared with the machine's other GPUs and can be loaded for seconds at a time),
        # every run's time is listed
        ke = max(2, min(K, 20))
        runs = []
        for _ in range(3):
            s2, t2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            starts = []
            h2d, d2h = sb.run([(hx, hy, hz, hm)] * ke, events=(s2, t2), build_starts=starts)
            torch.cuda.synchronize()
            # steady state: the interval between consecutive builds' starts (the pipeline's period,
            # without its fill by the first copy-in and its drain by the last build and copy-out)
            runs.append((max_over_ranks(s2.elapsed_time(t2) / ke, dist, dev),
                         starts[0].elapsed_time(starts[-1]) / (len(starts) - 1)))
        e2e_ms, period_ms = sorted(runs)[1]
        copy_in_ms = h2d / ke / (link["h2d_gbs"] * 1e9) * 1e3
        e2e = {"value": world * n / (e2e_ms * 1e-3), "unit": "particles/s", "h2d_bytes_per_step": h2d // ke,
               "d2h_bytes_per_step": d2h // ke, "ms_per_step": e2e_ms, "steps": ke,
               "runs_ms_per_step": [r[0] for r in runs],
               "method": "C ABI cstone_host_stage + cstone_host_build (StreamedBuilder): per step H2D of x, y, "
                         "z, m from pinned host memory, full build with multipoles, D2H of leaves, counts, NK, CO, "
                         "LO, node counts, mass, com, quad to pinned host memory; copies overlapped with the "
                         f"neighbouring steps' builds; the median of three runs of {ke} steps",
               "host_link": link, "steady_ms_per_step": period_ms,
               "copy_in_floor_ms": copy_in_ms,
               "note": "the host link carries about 210 GB/s host to device whether one copy, several "
                       "streams or a kernel reading pinned memory moves the data, so a step's copy-in is "
                       "the floor of the streamed period"}
        del sb

    extra = {}
    if rank == 0 and not args.no_focus:
        extra["focused_tree"] = measure_focus(b, n_leaves)
    if rank == 0 and not args.no_keys30:
        extra["keys30_same_workload"] = measure_keys30(X, Y, Z, M, K=max(3, min(K, 10)))
    if rank == 0 and not args.no_configs:
        extra["other_configs"] = measure_configs(dev, X, Y, Z, M, K=max(3, min(K, 10)))
    if rank == 0 and not args.no_batched:
        extra["batched_512_sets"] = measure_batched(dev)
    if rank == 0 and (not args.no_timesteps and args.ts_steps > 0 or not args.no_table1):
        del X, Y, Z, M, buffers, b, out
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_timesteps and args.ts_steps > 0:
        extra["timesteps_8x2p26"] = measure_timesteps(dev, args.ts_steps)
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_table1:
        extra["table1_gaussian"] = measure_table1(dev)
    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(CPU_SAMPLE)
        line = {
            "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_particles": n, "ncrit": NCRIT, "curve": "hilbert",
                       "l2_flush": "inputs (3.5 GB) larger than L2", "parallelism": "replicas" if world > 1 else "1gpu",
                       "n_leaves": n_leaves, "n_nodes": n_nodes, "leaf_iterations": iters,
                       "arith": "f64 grid mapping, u64 keys/sort/tree, f32 compensated multipoles"},
            "phase_ms": phase_ms,
            "step_algorithmic_bytes": step_bytes,
            "step_hbm_frac": step_bytes / (ms_per_step * 1e-3) / 1e9 / hbm,
            "build_hbm_frac_without_multipoles": (step_bytes - algo["multipoles"]) /
                                                 ((ms_per_step - phase_ms["multipoles"]) * 1e-3) / 1e9 / hbm,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "peak_source": peak_kind,
                         "traffic": (MEASURED_DRAM_BYTES_PER_PARTICLE[dom] * n
                                     if dom in MEASURED_DRAM_BYTES_PER_PARTICLE else None),
                         "algorithmic_bytes_per_launch": algo[dom]},
            "roofline_phases": {p: {"achieved_gbs": algo[p] / (phase_ms[p] * 1e-3) / 1e9,
                                    "frac": algo[p] / (phase_ms[p] * 1e-3) / 1e9 / hbm,
                                    "traffic": (MEASURED_DRAM_BYTES_PER_PARTICLE[p] * n
                                                if p in MEASURED_DRAM_BYTES_PER_PARTICLE else None)}
                                for p in phases},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks.summary(),
            "gpu_launches": launches,
            "extra": extra,
        }
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return line


def run_global(args, rank, world, local):
    """N > 1 processes, one per GPU (Sec. 6): every rank holds 2^27 clump particles of its own; a step
    builds the global octree of all ranks' particles (global bounding cube from bounds reduced over
    the ranks, local keys and sort, then f on the rank's own keys, one allreduce(SUM) of the leaf
    counts over NCCL and the same g on every rank, per pass), cuts it into one SFC domain per rank,
    sends every particle (and its mass) to the rank owning its key (all_to_all), and builds the
    rank's full local octree with node counts and multipoles in the global frame. Weak scaling:
    value = all ranks' particles / the slowest rank's step time."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2307_06345_gb300 as cs
    from paper_2307_06345_gb300 import distributed as D

    os.environ.setdefault("NCCL_DEBUG", "INFO")  # NCCL's communicator lines name the ranks and devices
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    cs.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist.init_process_group("nccl", device_id=dev)
    n = args.n
    x, y, z, m = workload(n, rank)
    X, Y, Z, M = (torch.from_numpy(a).to(dev) for a in (x, y, z, m))
    ops = D.DeviceOps(dev)
    stream = torch.cuda.current_stream()
    state = {}

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        t = D.build_global_tree(X, Y, Z, curve=cs.HILBERT, ncrit=NCRIT, ops=ops)
        cuts = D.decompose(ops, t["N_global"], world)
        if ev:
            ev[1].record(stream)
        rx, ry, rz, rm = D.exchange(ops, X, Y, Z, t["P"], t["perm"], t["K"], cuts, extra=(M,))
        if ev:
            ev[2].record(stream)
        out = cs.build_octree(rx, ry, rz, curve=cs.HILBERT, ncrit=NCRIT, box=t["box"], masses=rm,
                              buffers=state.get("buffers") if state.get("n") == rx.numel() else None)
        state["buffers"], state["n"] = out["buffers"], rx.numel()
        if ev:
            ev[3].record(stream)
        return t, out

    for _ in range(max(args.warmup, 1)):
        t, out = step()
    torch.cuda.synchronize()
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    dist.barrier()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        launches0 = cs.cstone_kernel_launches()
        start.record(stream)
        for k in range(K):
            t, out = step(evs[k])
        stop.record(stream)
        launches = cs.cstone_kernel_launches() - launches0
        torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    ms_per_step = max_over_ranks(start.elapsed_time(stop), dist, dev) / K
    phase = {name: float(np.mean([e[i].elapsed_time(e[i + 1]) for e in evs]))
             for i, name in enumerate(("global_tree", "exchange", "local_build"))}
    n_local = out["perm"].numel()
    # end to end: the same step with this rank's inputs copied in from pinned host memory and its
    # local tree's leaves and node counts copied out, every step
    hx, hy, hz, hm = (torch.from_numpy(a).pin_memory() for a in (x, y, z, m))
    ke = max(2, min(K, 5))
    dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h2d = d2h = 0
    e0.record(stream)
    for _ in range(ke):
        for dst, src in zip((X, Y, Z, M), (hx, hy, hz, hm)):
            dst.copy_(src, non_blocking=True)
            h2d += src.numel() * src.element_size()
        t, out = step()
        for key in ("leaves", "node_counts"):
            host = out[key].cpu()
            d2h += host.numel() * host.element_size()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / ke, dist, dev)
    hbm, peak_kind = peaks()
    nl_local = out["n_leaves"]
    local_bytes = sum(v for k2, v in algorithmic_bytes(n_local, nl_local, int(nl_local * 1.3),
                                                        cs.n_nodes(nl_local)).items() if k2 != "bbox")
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": world * n / (ms_per_step * 1e-3), "unit": "particles/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD + f", {n} particles per rank", "n_particles_per_rank": n,
                       "ncrit": NCRIT, "curve": "hilbert", "l2_flush": "inputs (3.5 GB per rank) larger than L2",
                       "parallelism": f"global octree over {world} ranks (Sec. 6): allreduce(SUM) of the leaf counts "
                                      "per f/g pass over NCCL, SFC decomposition, all_to_all exchange, local build",
                       "global_leaves": int(t["n_leaves"]), "global_passes": int(t["passes"]),
                       "rank0_local_particles": n_local, "rank0_local_leaves": out["n_leaves"]},
            "phase_ms": phase,
            "roofline": {"bound": "hbm", "kernel": "local_build", "achieved": local_bytes / (phase["local_build"] * 1e-3)
                         / 1e9, "peak": hbm, "unit": "GB/s", "peak_source": peak_kind,
                         "frac": local_bytes / (phase["local_build"] * 1e-3) / 1e9 / hbm, "traffic": None},
            "cpu_baseline": None,
            "e2e": {"value": world * n / (e2e_ms * 1e-3), "unit": "particles/s", "h2d_bytes_per_step": h2d // ke,
                    "d2h_bytes_per_step": d2h // ke, "ms_per_step": e2e_ms, "steps": ke},
            "clocks": clocks.summary(),
            "gpu_launches": launches,
        }
    dist.barrier()
    dist.destroy_process_group()
    return line


def measure_focus(b, n_leaves: int, reps: int = 5):
    """The locally essential tree of Sec. 7 on the benchmark workload: focus on the key range of the
    5th of 8 equal-count domains (the domain an 8-rank decomposition gives rank 4), minimum-distance
    MAC with theta 0.5, warm-started from the balanced tree of all particles; f and g^LE per pass."""
    import torch

    import paper_2307_06345_gb300 as cs
    from paper_2307_06345_gb300 import distributed as D

    Kg = b.leaves[: n_leaves + 1].clone()
    N = torch.empty(n_leaves, dtype=torch.int32, device=Kg.device)
    cs.cstone_leaf_counts(b.sorted_keys, Kg, n_leaves, N)
    cuts = D.decompose(D.DeviceOps(Kg.device), N, 8)
    f = [int(v) for v in Kg[cuts[4:6]].cpu().tolist()]
    f = [v + (1 << 64) if v < 0 else v for v in f]
    ws = cs.Workspace(Kg.device)
    out = cs.build_focus_leaves(b.sorted_keys, NCRIT, f[0], f[1], 0.5, cs.HILBERT, warm_leaves=Kg, ws=ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        e0.record()
        out = cs.build_focus_leaves(b.sorted_keys, NCRIT, f[0], f[1], 0.5, cs.HILBERT, warm_leaves=Kg, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    K, Nf, passes = out
    c4, c5 = (int(v) for v in cuts[4:6].cpu().tolist())
    inside = int(N[c4: c5].sum().item())
    return {"focus_keys": f, "theta": 0.5, "ncrit": NCRIT, "ms": sorted(ts)[len(ts) // 2], "passes": passes,
            "n_leaves_focused": K.numel() - 1, "n_leaves_global": n_leaves, "particles_in_focus": inside,
            "start": "balanced tree of all particles"}


def measure_keys30(X, Y, Z, M, K: int = 10):
    """The same workload and step with 30-bit keys (L = 10, Sec. 3's other key length): bbox, keys,
    a 4-pass sort of 32-bit words, leaves, link, counts and multipoles; CUDA events per phase."""
    import numpy as np
    import torch

    import paper_2307_06345_gb300 as cs

    stream = torch.cuda.current_stream()
    out = cs.build_octree(X, Y, Z, curve=cs.HILBERT, ncrit=NCRIT, masses=M, levels=10)
    b = out["buffers"]
    torch.cuda.synchronize()
    phases = ["bbox", "keys", "sort", "leaves", "link", "counts", "multipoles"]
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(phases) + 1)] for _ in range(K)]
    nl = 0
    for k in range(K + 2):
        e = ev[k - 2] if k >= 2 else ev[0]  # two untimed warm-up steps
        e[0].record(stream)
        cs.cstone_bbox(X, Y, Z, b.box, b.ws)
        e[1].record(stream)
        cs.cstone_keys_records(X, Y, Z, M, b.box, cs.HILBERT, b.keys, b.records, b.rws, levels=10)
        e[2].record(stream)
        cs.cstone_sort(b.keys, b.sorted_keys, b.perm, b.ws, levels=10)
        e[3].record(stream)
        nl, it = cs.cstone_build_leaves(b.sorted_keys, NCRIT, b.leaves, b.counts, b.offsets, 0, 64, b.ws, levels=10)
        e[4].record(stream)
        t = b.tree_buffers(nl)
        cs.cstone_link_tree(b.leaves, nl, t["NK"], t["CO"], t["LO"], t["leaf_to_node"], t["parent"], b.ws,
                            levels=10)
        e[5].record(stream)
        cs.cstone_upsweep_counts(b.counts, nl, t["leaf_to_node"], t["CO"], t["LO"], t["counts"], b.ws, levels=10)
        e[6].record(stream)
        nn = cs.n_nodes(nl)
        cs.cstone_upsweep_multipoles_records(b.records, b.perm, X.numel(), b.offsets, nl, t["leaf_to_node"], t["CO"],
                                             t["LO"], b.box, t["mass"][:nn], t["com"][: 3 * nn], t["quad"][: 6 * nn],
                                             b.ws, levels=10)
        e[7].record(stream)
    torch.cuda.synchronize()
    phase_ms = {p: float(np.mean([ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(K)]))
                for i, p in enumerate(phases)}
    step_ms = sum(phase_ms.values())
    n = X.numel()
    counts = t["counts"][:nn]
    return {"levels": 10, "key_bits": 30, "n_particles": n, "ncrit": NCRIT, "curve": "hilbert",
            "ms_per_step": step_ms, "particles_per_s": n / (step_ms * 1e-3), "phase_ms": phase_ms,
            "n_leaves": nl, "leaf_iterations": it,
            "max_leaf_count": int(b.counts[:nl].max().item()), "root_count": int(counts[0].item()),
            "sort_algorithmic_bytes_per_key": 12 + 3 * 16}


def _timed_builds(X, Y, Z, M, curve, ncrit, box, K, masses=True):
    """ms per full build (CUDA events over K builds after two warm-ups) and the built tree."""
    import torch

    import paper_2307_06345_gb300 as cs

    kw = dict(curve=curve, ncrit=ncrit, box=box, masses=M if masses else None)
    out = cs.build_octree(X, Y, Z, **kw)
    b = out["buffers"]
    out = cs.build_octree(X, Y, Z, buffers=b, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        out = cs.build_octree(X, Y, Z, buffers=b, **kw)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / K, out


def measure_configs(dev, X, Y, Z, M, K: int = 10):
    """Throughput of the other single-set workloads: 65,536 uniform particles (unit cube, Morton,
    Ncrit 64), 2^25 Plummer particles (bounding cube, Hilbert, Ncrit 64), and the benchmark workload
    at Ncrit 16; full builds with the count upsweep (and multipoles for the clump workload), CUDA
    events around K back-to-back builds (each build synchronises once for its leaf count)."""
    import numpy as np
    import torch

    import paper_2307_06345_gb300 as cs
    from paper_2307_06345_gb300 import workloads as w

    res = {}
    n1 = 65_536
    x, y, z = w.uniform(n1, w.BASE_SEED)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    unit = torch.tensor([0.0, 0.0, 0.0, 1.0], dtype=torch.float64, device=dev)
    ms, out = _timed_builds(to(x), to(y), to(z), None, cs.MORTON, 64, unit, max(K, 20), masses=False)
    res["uniform_65536_morton_ncrit64"] = {"ms": ms, "particles_per_s": n1 / (ms * 1e-3), "n_leaves": out["n_leaves"]}
    n2 = 1 << 25
    x, y, z = w.plummer(n2, w.BASE_SEED + 1)
    ms, out = _timed_builds(to(x), to(y), to(z), None, cs.HILBERT, 64, None, K, masses=False)
    res["plummer_2p25_hilbert_ncrit64"] = {"ms": ms, "particles_per_s": n2 / (ms * 1e-3), "n_leaves": out["n_leaves"],
                                           "iters": out["iters"]}
    del x, y, z, out
    ms, out = _timed_builds(X, Y, Z, M, cs.HILBERT, 16, None, K)
    res["clumps_2p27_hilbert_ncrit16_multipoles"] = {"ms": ms, "particles_per_s": X.numel() / (ms * 1e-3),
                                                     "n_leaves": out["n_leaves"], "iters": out["iters"]}
    del out
    torch.cuda.empty_cache()
    res["note"] = ("full builds through build_octree (bounding cube unless given, keys, sort, leaves, link, node "
                   "counts; multipoles where named); the uniform set is latency bound (n_l = 4096)")
    return res


def measure_batched(dev, reps: int = 5):
    """512 independent sets (sizes log-uniform in [2^10, 2^20), uniform in the unit cube or Plummer in
    its bounding cube), Morton keys, Ncrit 32: one batched build (one launch per phase for all sets)
    against 512 plain single-set builds on the same GPU."""
    import numpy as np
    import torch

    import paper_2307_06345_gb300 as cs
    from paper_2307_06345_gb300 import workloads as w

    sets = w.batched_sets(512, w.BASE_SEED + 3)
    sizes = np.array([len(st[0]) for st in sets], np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    X, Y, Z = (torch.from_numpy(np.concatenate([st[k] for st in sets])).to(dev) for k in range(3))
    OFF = torch.from_numpy(off).to(dev)
    boxes = torch.empty((512, 4), dtype=torch.float64, device=dev)
    cs.cstone_bbox_batched(X, Y, Z, OFF, boxes)
    unit = torch.tensor([0.0, 0.0, 0.0, 1.0], dtype=torch.float64, device=dev)
    for i, st in enumerate(sets):
        if st[3] == "uniform":
            boxes[i] = unit
    ws = cs.Workspace(dev)
    stream = torch.cuda.current_stream()
    out = cs.build_octrees_batched(X, Y, Z, OFF, curve=cs.MORTON, ncrit=32, boxes=boxes, ws=ws)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(reps):
        out = cs.build_octrees_batched(X, Y, Z, OFF, curve=cs.MORTON, ncrit=32, boxes=boxes, ws=ws)
    s1.record(stream)
    torch.cuda.synchronize()
    batched_ms = s0.elapsed_time(s1) / reps
    # plain builds, one set after the other, buffers allocated beforehand
    views = [(X[off[i]:off[i + 1]], Y[off[i]:off[i + 1]], Z[off[i]:off[i + 1]], boxes[i].contiguous())
             for i in range(512)]
    bufs = [cs.build_octree(*v[:3], curve=cs.MORTON, ncrit=32, box=v[3])["buffers"] for v in views]
    torch.cuda.synchronize()
    s0.record(stream)
    for v, b in zip(views, bufs):
        cs.build_octree(*v[:3], curve=cs.MORTON, ncrit=32, box=v[3], buffers=b)
    s1.record(stream)
    torch.cuda.synchronize()
    seq_ms = s0.elapsed_time(s1)
    n = int(off[-1])
    return {"sets": 512, "particles": n, "ncrit": 32, "curve": "morton", "batched_ms": batched_ms,
            "batched_particles_per_s": n / (batched_ms * 1e-3), "plain_sequential_ms": seq_ms,
            "speedup_vs_plain": seq_ms / batched_ms, "leaf_iterations": out["iters"]}


def measure_timesteps(dev, steps: int, runs: int = 8, n: int = 1 << 26):
    """8 runs of 2^26 Plummer particles, `steps` steps, Gaussian displacements of 1e-3 of the box
    per step (drawn on the device), Hilbert keys, Ncrit 64: every step rebuilds all runs in one
    batched build warm-started from the previous step's leaves, in the step-0 bounding cube padded
    by 10% of its side on every side. The rebuild is one CUDA graph replayed per step; the same
    steps launched one phase at a time are timed for comparison."""
    import torch

    import paper_2307_06345_gb300 as cs
    from paper_2307_06345_gb300 import workloads as w

    xs, ys, zs = [], [], []
    for r in range(runs):
        x, y, z = w.plummer_device(n, w.BASE_SEED + 5 + r, dev)
        xs.append(x), ys.append(y), zs.append(z)
    X, Y, Z = torch.cat(xs), torch.cat(ys), torch.cat(zs)
    del xs, ys, zs
    OFF = torch.arange(runs + 1, dtype=torch.int64, device=dev) * n
    st = cs.GraphTimeStepper(X, Y, Z, OFF, curve=cs.HILBERT, ncrit=64)
    sigma = 1e-3 * float(st.boxes[0, 3]) / 1.2
    g = torch.Generator(device=dev)
    g.manual_seed(w.BASE_SEED + 6)
    stream = torch.cuda.current_stream()

    def move():
        for c in (X, Y, Z):
            c.add_(torch.randn(c.shape, dtype=torch.float64, device=dev, generator=g), alpha=sigma)

    out = st.rebuild(warm=False)
    move()
    out = st.rebuild(warm=True)  # captures the step's graph (not timed)
    torch.cuda.synchronize()
    total_ms, iters = 0.0, []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for step in range(steps):
        move()
        e0.record(stream)
        out = st.rebuild(warm=True)  # one graph replay + one read-back of the leaf loop's outcome
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        iters.append(out["iters"])
    # the same steps without the graph (launch by launch, host reads between phases), for comparison
    eager = cs.TimeStepper(X, Y, Z, OFF, curve=cs.HILBERT, ncrit=64)
    eager.boxes = st.boxes
    eager.rebuild(warm=False)
    eager_ms, eager_steps = 0.0, min(steps, 10)
    for _ in range(eager_steps):
        move()
        e0.record(stream)
        eager.rebuild(warm=True)
        e1.record(stream)
        torch.cuda.synchronize()
        eager_ms += e0.elapsed_time(e1)
    out = st.rebuild(warm=True)
    cold = cs.build_octrees_batched(X, Y, Z, OFF, curve=cs.HILBERT, ncrit=64, boxes=st.boxes)
    same = bool(torch.equal(cold["elements"], out["elements"]) and torch.equal(cold["NK"], out["NK"]))
    lo, side = st.boxes[:, :3], st.boxes[:, 3:4]
    clamped = 0
    for r in range(runs):
        sl = slice(r * n, (r + 1) * n)
        pts = torch.stack([X[sl], Y[sl], Z[sl]], 1)
        clamped += int(((pts < lo[r]) | (pts >= lo[r] + side[r])).any(1).sum())
    return {"runs": runs, "particles_per_run": n, "steps": steps, "graph": True, "ms_per_step": total_ms / steps,
            "eager_ms_per_step": eager_ms / eager_steps,
            "particles_per_s": runs * n * steps / (total_ms * 1e-3), "leaf_iterations_max": max(iters),
            "leaf_iterations_mean": sum(iters) / len(iters), "last_step_warm_equals_cold": same,
            "clamped_particles": clamped}


# Table 1 of the paper, NVIDIA A100 rows (ms), for context: another GPU, its own Gaussian width.
TABLE1_A100_MS = {
    "1M": {"keys_morton": 0.018, "keys_hilbert": 0.084, "sort": 0.483, "leaf_update": 0.11, "internal_nodes": 0.19},
    "32M": {"keys_morton": 0.31, "keys_hilbert": 1.9, "sort": 5.0, "leaf_update": 0.51, "internal_nodes": 0.65},
    "512M": {"keys_morton": 7.9, "keys_hilbert": 30.0, "sort": 73.0, "leaf_update": 2.5, "internal_nodes": 5.4},
}


def measure_table1(dev):
    """Replay of the paper's Table 1 workload: one 3D Gaussian (sigma 0.1 of the unit box, drawn on
    the device) of 2^20, 2^25 and 2^29 particles, Ncrit 64, each step of the build timed on its own
    (median of several runs, CUDA events): Morton keys, Hilbert keys, the sort of the Hilbert keys,
    the leaf update (one rebalance pass from the converged leaves, and the full convergence from
    the root), and the internal nodes (linked octree from the leaves)."""
    import torch

    import paper_2307_06345_gb300 as cs
    from paper_2307_06345_gb300 import workloads as w

    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sorted(ts)[len(ts) // 2]

    res = {}
    for label, n, reps in (("1M", 1 << 20, 20), ("32M", 1 << 25, 10), ("512M", 1 << 29, 5)):
        X, Y, Z = w.gaussian_device(n, w.BASE_SEED + 7, dev)
        ws = cs.Workspace(dev)
        box = torch.empty(4, dtype=torch.float64, device=dev)
        cs.cstone_bbox(X, Y, Z, box, ws)
        keys = torch.empty(n, dtype=torch.int64, device=dev)
        r = {"particles": n}
        r["keys_morton"] = timed(lambda: cs.cstone_keys(X, Y, Z, box, cs.MORTON, keys), reps)
        r["keys_hilbert"] = timed(lambda: cs.cstone_keys(X, Y, Z, box, cs.HILBERT, keys), reps)
        del X, Y, Z
        sk = torch.empty_like(keys)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        r["sort"] = timed(lambda: cs.cstone_sort(keys, sk, perm, ws), reps)
        del keys
        cap = cs.leaf_capacity(n, 64)
        leaves = torch.empty(cap + 1, dtype=torch.int64, device=dev)
        counts = torch.empty(cap, dtype=torch.int32, device=dev)
        state = {}

        def cold():
            state["nl"], state["it"] = cs.cstone_build_leaves(sk, 64, leaves, counts, None, 0, 64, ws)

        r["leaf_build_from_root"] = timed(cold, reps)
        nl = state["nl"]
        r["leaf_build_iterations"] = state["it"]
        converged = leaves[: nl + 1].clone()

        def warm():
            leaves[: nl + 1].copy_(converged)
            state["nl"], state["it"] = cs.cstone_build_leaves(sk, 64, leaves, counts, None, nl, 64, ws)

        copy_ms = timed(lambda: leaves[: nl + 1].copy_(converged), reps)
        r["leaf_update"] = max(timed(warm, reps) - copy_ms, 0.0)
        r["leaf_update_iterations"] = state["it"]
        nn = cs.n_nodes(nl)
        NK = torch.empty(nn, dtype=torch.int64, device=dev)
        CO = torch.empty(nn, dtype=torch.int32, device=dev)
        LO = torch.empty(23, dtype=torch.int32, device=dev)
        l2n = torch.empty(nl, dtype=torch.int32, device=dev)
        r["internal_nodes"] = timed(lambda: cs.cstone_link_tree(leaves, nl, NK, CO, LO, l2n, None, ws), reps)
        r["n_leaves"] = nl
        res[label] = r
        del sk, perm, leaves, counts, converged, NK, CO, LO, l2n, ws
        torch.cuda.empty_cache()
    res["paper_a100_ms"] = TABLE1_A100_MS
    res["note"] = ("ms per step, median; leaf_update = one rebalance pass from the converged leaves; the paper's "
                   "rows are an A100 with its own (unstated) Gaussian width, context only")
    return res


def cpu_model() -> str:
    """The host CPU's model name (from /proc/cpuinfo or lscpu)."""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_step(oracle, x, y, z, m):
    t0 = time.perf_counter()
    ref = oracle.full_build(x, y, z, oracle.HILBERT, NCRIT)
    oracle.multipoles(x, y, z, m, ref["P"], ref["perm"], ref["NK"])
    return time.perf_counter() - t0


def multipole_errors_on_sample(oracle, x, y, z, m):
    """The library's multipoles of the sample's full build against the oracle's FP64 moments of the
    oracle's own tree (equal to the library's, which the tests check), over every non-empty node:
    mass |dM| / M, centre max-norm |d com| / node side, quadrupole max_ab |dQ_ab| / max_ab |Q_ab|."""
    import numpy as np
    import torch

    import paper_2307_06345_gb300 as cs

    ref = oracle.full_build(x, y, z, oracle.HILBERT, NCRIT)
    M_ref, c_ref, q_ref = oracle.multipoles(x, y, z, m, ref["P"], ref["perm"], ref["NK"])
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = cs.build_octree(to(x), to(y), to(z), curve=cs.HILBERT, ncrit=NCRIT, masses=to(m))
    torch.cuda.synchronize()
    if out["NK"].numel() != ref["NK"].size or not np.array_equal(out["NK"].cpu().numpy().view(np.uint64), ref["NK"]):
        return {"error": "trees differ"}
    M = out["mass"].cpu().numpy().astype(np.float64)
    com = out["com"].cpu().numpy().T
    q = out["quad"].cpu().numpy().T.astype(np.float64)
    lev = np.zeros(ref["NK"].size, np.int64)
    for lv in range(1, 22):
        lev += ref["NK"] >= np.uint64(1 << (3 * lv))
    side = ref["box"][3] * 2.0 ** (-lev.astype(np.float64))
    nz = M_ref > 0
    qn = np.maximum(np.max(np.abs(q_ref), axis=1), 1e-12 * M_ref * side ** 2)
    return {"mass": float(np.max(np.abs(M[nz] - M_ref[nz]) / M_ref[nz])),
            "com": float(np.max(np.max(np.abs(com[nz] - c_ref[nz]), axis=1) / side[nz])),
            "quad": float(np.max(np.max(np.abs(q[nz] - q_ref[nz]), axis=1) / qn[nz])),
            "nodes": int(nz.sum()), "tolerance": 1e-6}


def cpu_baseline(sample: int, rank_seed: int = 0):
    """The oracle as it stands on a bounded sample of the same workload: on every host core (its
    parallel loops over particles, leaves and nodes), and single-threaded on a quarter of the sample.
    Also the multipole errors of the library's build of that sample against the oracle."""
    import oracle

    oracle.build()
    x, y, z, m = workload(sample, rank_seed)
    cores = oracle.set_threads(0)
    dt = _oracle_step(oracle, x, y, z, m)
    errors = multipole_errors_on_sample(oracle, x, y, z, m)
    s1 = sample // 4
    oracle.set_threads(1)
    dt1 = _oracle_step(oracle, x[:s1], y[:s1], z[:s1], m[:s1])
    oracle.set_threads(0)
    return {"value": sample / dt, "unit": "particles/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{sample} particles of the same clump distribution, full path incl. multipoles, "
                      f"{dt:.1f} s on {cores} threads",
            "single_thread": {"value": s1 / dt1, "unit": "particles/s", "cores": 1,
                              "sample": f"the first {s1} of those particles, {dt1:.1f} s"},
            "multipole_max_errors_on_sample": errors}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle

    oracle.build()
    sample = REF_SAMPLE
    x, y, z, m = workload(sample)
    cores = oracle.set_threads(0)
    for _ in range(args.warmup):
        pass  # the oracle has no warm state; warm-up steps would only repeat the timed work
    times = [_oracle_step(oracle, x, y, z, m) for _ in range(args.steps)]
    dt = sum(times) / len(times)
    value = sample / dt
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64/u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_particles": sample, "ncrit": NCRIT, "curve": "hilbert"},
            "cpu_baseline": {"value": value, "unit": "particles/s", "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"{sample} particles per step of the same clump distribution, "
                                       f"{cores} threads"},
            "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    elif world > 1:
        line = run_global(args, rank, world, local)
    else:
        line = run_ours(args, rank, world, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
