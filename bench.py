#!/usr/bin/env python
"""Benchmark: Potts site-updates/s of the hybrid Monte Carlo hot path on GB300.

Workload (default): the 3D 1024^3 periodic simple cubic lattice, 26-neighbour
8-colour sweep, 10^6 Voronoi grains of FCC nickel with SO(3)-uniform
orientations, driven by the per-material-point field of the Monte Carlo crystal
plasticity (Table 1 constants, Taylor increment 1e-4), kT = 0.7, refreshed every
50 MCS by two increments (the plain-solver arm of the 1024^3 surrogate-vs-plain
configuration).  One step = one refresh period on the device-resident state:
the plasticity update of every material point (two increments, new field)
followed by 50 MCS of the sweep.  The line also carries the time to texture
(500 MCS) of the plain and the surrogate-driven hybrids at the same size.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload ...]

Prints ONE JSON line (rank 0).  With N > 1 (torchrun, one rank per GPU) every
rank runs its own independent lattice (its own seed): weak scaling, no
collective on the data path; the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mproc
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1007_3509_gb300 import synth  # noqa: E402

W4 = synth.W3D_SURROGATE          # 1024^3, 10^6 grains, kT 0.7, refresh every 50 MCS
W = synth.W2D_MOORE               # 4096^2 Moore: secondary line (L2-assisted)
BYTES_3D_POINT = 24               # q, b, mp read and written once per site-update
BYTES_2D_GRAIN = 8                # q read and written; the per-grain field from L1/L2
L2_BYTES = 129 * 1024 * 1024


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-secondary", action="store_true")
    p.add_argument("--no-texture", action="store_true", help="skip the time-to-texture runs of both arms")
    p.add_argument("--mcs", type=int, default=None, help="MCS per step (default: the workload's)")
    p.add_argument("--variant", type=int, default=None, help="fused-sweep tile variant (default: autotuned)")
    p.add_argument("--edge", type=int, default=None,
                   help="3D workloads: lattice edge (default 1024, or 512 for 3d-cp); grains scale with the volume")
    p.add_argument("--workload", choices=["3d", "2d", "3d-cp", "ensemble", "surrogate", "sweep3d", "texture2d",
                                          "texture3d", "texture-seeds", "3d-eq", "aniso", "mcp-vs-det", "surrogate-train", "small2d"],
                   default="3d",
                   help="3d: 1024^3 plasticity-driven hybrid (default line); 2d: 4096^2 Moore; 3d-cp: 512^3 "
                        "plasticity-driven whole job; ensemble: 256 replicas; surrogate: 1024^3 plain vs surrogate "
                        "time-to-texture; texture-seeds: both arms over 8 seeds each")
    p.add_argument("--seeds", type=int, default=8, help="texture-seeds: seeds per arm")
    p.add_argument("--train-steps", type=int, default=60000, help="surrogate-train: Adam steps")
    p.add_argument("--no-autotune", action="store_true")
    a = p.parse_args()
    if a.mcs is None:
        a.mcs = {"3d": 50, "2d": W.n_mcs, "3d-cp": 500, "ensemble": 200, "surrogate": 500, "sweep3d": 20,
                 "texture2d": 1000, "texture3d": 400, "texture-seeds": 500, "3d-eq": 500, "aniso": 200,
                 "mcp-vs-det": 0, "surrogate-train": 0, "small2d": 100}[a.workload]
    return a


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            return None
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def aggregate(local_ms, local_units, world, device):
    """Whole-job throughput over ranks: every rank processed `local_units`; the
    job time is the slowest rank's.  Returns (max_ms, units per second)."""
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.barrier()
    max_ms = float(t.item())
    return max_ms, local_units * world / (max_ms / 1e3)


# ---------------------------------------------------------------------------
# our arm: the 3D plasticity-driven hybrid
# ---------------------------------------------------------------------------
def shape3d(edge):
    """Lattice, grain count (10^6 at 1024^3, same mean grain volume at other edges)."""
    e = int(edge or W4.L[0])
    N = e ** 3
    return (e, e, e), N, max(1, round(W4.G * N / W4.N))


class Hybrid3D:
    """Device-resident state of the plasticity-driven 3D hybrid (one lattice)."""

    def __init__(self, torch, hm, hybrid, edge, seed):
        self.torch, self.hm = torch, hm
        ex = W4.extra
        self.L, self.N, self.G = shape3d(edge)
        self.seed = seed
        self.every, self.incr_per = ex["refresh_every"], ex["incr_per_refresh"]
        self.prm = hybrid.cp_params_table1(ex["e_incr"], ex["energy_scale"])
        N, dev = self.N, "cuda"
        self.lat = hm.Lattice(3, self.L, 26, 256, seed, self.G, hm.FIELD_POINT)
        self.q = torch.empty(N, dtype=torch.int32, device=dev)
        self.mp = torch.empty(N, dtype=torch.int32, device=dev)
        self.lat.hp_bind(self.q, self.mp)
        self.quat = torch.empty(self.G, 4, dtype=torch.float32, device=dev)
        self.eps = torch.empty(6 * N, dtype=torch.float32, device=dev)
        self.gam = torch.empty(N, dtype=torch.float32, device=dev)
        self.g = torch.empty(N, dtype=torch.float32, device=dev)
        self.b = torch.empty(N, dtype=torch.int32, device=dev)
        thr, D = hm.hp_build_threshold_table(W4.kT)
        self.lat.hp_set_threshold_table(thr, D)
        self.lat.hp_set_field(self.b)
        self.tuned = None
        self.reset()

    def reset(self):
        """Voronoi polycrystal, material point p in the grain of site p, no plastic strain."""
        self.lat.hp_init_voronoi(self.hm.ORIENT_SO3, self.quat)
        self.grain = self.q.clone()
        self.hm.hp_cp_reset(self.prm, self.N, self.eps, self.gam, self.g)
        self.lat.hp_set_sweep_counter(0)
        self.incr = 0

    def autotune(self):
        """Pick the fastest sweep tile on the current lattice (lattice and counter restored)."""
        self.refresh()
        chosen, ms = self.lat.hp_sweep_autotune(2)
        self.tuned = {"variant": int(chosen), "ms_per_2_mcs": [round(float(x), 3) for x in ms]}
        self.reset()

    def refresh(self):
        self.hm.hp_cp_step(self.prm, self.seed, self.grain, self.quat, self.incr, self.incr_per, self.eps, self.gam,
                           self.g, b=self.b)
        self.incr += self.incr_per

    def step(self, ev=None):
        """One refresh period: plasticity update (new field), then `every` MCS."""
        if ev:
            ev[0].record()
        self.refresh()
        if ev:
            ev[1].record()
        self.lat.hp_sweep(self.every)
        if ev:
            ev[2].record()

    def close(self):
        self.lat.close()


# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the 3D sweep
# kernel (one plane parity, the point-field lean window), from an ncu capture of
# that exact kernel on the bench lattice (profiles/k_lean26_3d1024_point_field.md);
# keyed by (edge, tile variant).  None for any other kernel or lattice.
MEASURED_TRAFFIC_3D = {(1024, 11): 13.069e9 + 4.277e9}


def sweep_kernel_name(nbr, variant):
    """Kernel family of a fused-sweep tile variant (numbering of hp_sweep_variants)."""
    v = int(variant or 0)
    if nbr == 26:
        kind = "k_plane" if v < 4 else ("k_tile" if v < 8 else "k_lean26")
    else:
        kind = "k_plane" if v < 3 else "k_tile"
    return f"{kind}<{nbr}> (fused MCS, variant {v})"


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1007_3509_gb300 import build, hmcpotts as hm, hybrid
    torch.cuda.set_device(local_rank)
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    hm.lib()
    job = Hybrid3D(torch, hm, hybrid, args.edge, W4.seed + rank)
    job.every = args.mcs
    if args.variant is not None:
        job.lat.hp_set_sweep_variant(args.variant)
        job.tuned = {"variant": int(args.variant), "ms_per_2_mcs": None}
    elif not args.no_autotune:
        job.autotune()
    for _ in range(args.warmup):
        job.step()
    torch.cuda.synchronize()

    clocks = Clocks(local_rank)
    launches0 = hm.hp_kernel_launches()
    step_ms, cp_ms, sweep_ms = [], [], []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(args.steps):
        e0, e1 = _events(torch)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
              torch.cuda.Event(enable_timing=True))
        e0.record()
        job.step(ev)
        e1.record()
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        cp_ms.append(ev[0].elapsed_time(ev[1]))
        sweep_ms.append(ev[1].elapsed_time(ev[2]))
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = hm.hp_kernel_launches() - launches0
    total_ms = sum(step_ms)
    max_ms, value = aggregate(total_ms, job.N * job.every * args.steps, world, "cuda")

    # dominant kernel: the sweep, two launches per MCS (even then odd planes),
    # each over N/2 site-updates of 24 algorithmic bytes
    launch_s = statistics.mean(sweep_ms) / 1e3 / (2 * job.every)
    achieved = BYTES_3D_POINT * (job.N / 2) / launch_s / 1e9
    peak, peak_kind = peaks()
    variant = job.tuned.get("variant") if job.tuned else None
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": MEASURED_TRAFFIC_3D.get((job.L[0], variant)),
            "peak_source": peak_kind, "kernel": sweep_kernel_name(26, variant),
            "bytes_per_site_update": BYTES_3D_POINT, "site_updates_per_launch": job.N // 2,
            "launch_ms": round(launch_s * 1e3, 4),
            "sweep_site_updates_per_s": round(job.N / (2 * launch_s), 1),
            "share_of_step": round(sum(sweep_ms) / total_ms, 4)}
    plast = {"point_increments_per_s": round(job.N * job.incr_per / (statistics.mean(cp_ms) / 1e3), 1),
             "ms_per_refresh": round(statistics.mean(cp_ms), 3), "share_of_step": round(sum(cp_ms) / total_ms, 4)}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(torch, hm, job, args)
    tuned = job.tuned
    job.close()
    del job
    torch.cuda.empty_cache()
    ttt = None
    if not args.no_texture and rank == 0 and world == 1:
        ttt = time_to_texture(torch, hm, hybrid, args)
    secondary = None
    if not args.no_secondary and rank == 0:
        secondary = {"2d_4096_moore_L2_assisted": run_2d_secondary(torch, hm)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(args)
    if rank != 0:
        return
    L, N, G = shape3d(args.edge)
    line = {
        "metric": "Potts site-updates/s",
        "value": round(value, 1),
        "unit": "site-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(max_ms / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32 sweep; fp32 plasticity with fp64 return map",
        "data": "synthetic (seeded Voronoi polycrystal, SO(3)-uniform FCC Ni orientations)",
        "config": {"workload": f"3d-{L[0]}-moore26-g{G}-plain-mcp-hybrid", "lattice": list(L), "nbr": 26,
                   "colours": 8, "grains": G, "kT": W4.kT, "mcs_per_step": args.mcs,
                   "field": "per material point: MCP (Table 1 Ni), 2 Taylor increments of 1e-4 per step",
                   "step": "MCP refresh of every material point + 50 MCS", "l2": "inputs larger than L2 (4 GB per array)",
                   "parallelism": f"replicas x{world}", "tile": tuned},
        "roofline": roof,
        "plasticity": plast,
        "time_to_texture": ttt,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "secondary": secondary,
    }
    print(json.dumps(line))


def run_e2e(torch, hm, job, args):
    """The same step through the public C ABI with host buffers: the lattice state
    (q, mp) goes in from pinned host memory (hp_set_spins), the plasticity refresh
    and the 50 MCS run, and the state (hp_get_spins) and the grain statistics and
    texture (hp_measure) come back to the host, every step.  The copies run on a
    second stream: the upload of a step's state overlaps that step's plasticity
    refresh (which reads only the material-point state), and its read-back
    overlaps the grain statistics; the sweep waits for the upload, and the timed
    region ends when the read-back has landed."""
    N = job.N
    h_q = torch.empty(N, dtype=torch.int32).pin_memory()
    h_mp = torch.empty(N, dtype=torch.int32).pin_memory()
    job.lat.hp_get_spins(h_q, h_mp)
    torch.cuda.synchronize()
    # The host link itself, outside the timed region: one plain pinned copy of
    # the q array each way (h_q holds the device lattice's values, so the upload
    # leaves the state unchanged).  The copies of a step move twice this.
    link = {}
    for name, dst, src in (("h2d", job.q, h_q), ("d2h", h_q, job.q)):
        e0, e1 = _events(torch)
        e0.record()
        dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        link[name] = round(4 * N / (e0.elapsed_time(e1) * 1e6), 1)
    main = torch.cuda.current_stream()
    copy = torch.cuda.Stream()

    def one():
        copy.wait_stream(main)
        job.lat.hp_set_spins(h_q, h_mp, stream=copy)
        up = torch.cuda.Event()
        up.record(copy)
        job.refresh()
        main.wait_event(up)
        job.lat.hp_sweep(job.every)
        copy.wait_stream(main)
        job.lat.hp_get_spins(h_q, h_mp, stream=copy)
        st, hist = job.lat.hp_measure(hm.ORIENT_SO3, job.quat)  # synchronises the main stream
        main.wait_stream(copy)
        return st

    one()
    torch.cuda.synchronize()
    ms = []
    steps = max(2, min(args.steps, 3))
    for _ in range(steps):
        e0, e1 = _events(torch)
        e0.record()
        one()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    per = statistics.mean(ms) / 1e3
    return {"value": round(N * job.every / per, 1), "unit": "site-updates/s", "h2d_bytes_per_step": 8 * N,
            "d2h_bytes_per_step": 8 * N + 24 * 8, "ms_per_step": round(per * 1e3, 3),
            "host_link_gbs": link,
            "path": "hp_set_spins (host, copy stream) overlapping hp_cp_step, then hp_sweep; hp_get_spins (host, "
                    "copy stream) overlapping hp_measure"}


def time_to_texture(torch, hm, hybrid, args):
    """Wall time to 500 MCS of both arms at the bench size from a fresh polycrystal:
    the plain hybrid (plasticity at every material point each refresh) and the
    surrogate-driven one (its training data generated and the network trained in
    the timed region, then one network evaluation per grain each refresh)."""
    L, N, G = shape3d(args.edge)
    cfg = hybrid.HybridConfig(L=L, G=G, seed=W4.seed, kT=W4.kT, n_mcs=500)
    prm = hybrid.cp_params_table1(cfg.e_incr, cfg.energy_scale)
    plain = hybrid.run_plain(torch, cfg, time_it=False)
    torch.cuda.empty_cache()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    params, load, loss, _ = hybrid.train_surrogate(torch, prm)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    sur = hybrid.run_surrogate(torch, cfg, params, load, time_it=False)
    torch.cuda.empty_cache()
    return {"mcs": 500, "plain_s": round(plain["wall_s"], 3), "surrogate_s": round(train_s + sur["wall_s"], 3),
            "surrogate_train_s": round(train_s, 3), "surrogate_run_s": round(sur["wall_s"], 3),
            "speedup": round(plain["wall_s"] / (train_s + sur["wall_s"]), 3),
            "families_plain": [round(x, 5) for x in plain["families"]],
            "families_surrogate": [round(x, 5) for x in sur["families"]],
            "mean_mmax_plain": round(plain["mean_mmax"], 5), "mean_mmax_surrogate": round(sur["mean_mmax"], 5),
            "seeds_per_arm": 1, "final_train_loss": loss}


def run_2d_secondary(torch, hm):
    """The 2D 4096^2 Moore sweep with the closed-form per-grain field (1000 MCS of
    the lean tile kernel): partly L2-resident, not an HBM figure."""
    try:
        L, G = W.L, W.G
        N = int(np.prod(L))
        lat = hm.Lattice(2, L, W.nbr, int(256 * W.J), W.seed, G, hm.FIELD_GRAIN)
        q = torch.empty(N, dtype=torch.int32, device="cuda")
        lat.hp_bind(q)
        quat = torch.empty(G, 4, dtype=torch.float32, device="cuda")
        bg = torch.empty(G, dtype=torch.int32, device="cuda")
        lat.hp_init_voronoi(hm.ORIENT_SO3, quat)
        hm.hp_grain_field(quat, *[synth.NI_BJ[k] for k in ("C11", "C12", "C44")], W.sigma, W.k_disl,
                          W.energy_scale, bg)
        lat.hp_set_field(bg)
        lat.hp_set_threshold_table(*hm.hp_build_threshold_table(W.kT))
        chosen, _ = lat.hp_sweep_autotune(8)
        lat.hp_sweep(20)
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        lat.hp_sweep(W.n_mcs)
        e1.record()
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) / 1e3
        peak, _ = peaks()
        rate = N * W.n_mcs / s
        lat.close()
        return {"workload": W.name, "site_updates_per_s": round(rate, 1), "mcs": W.n_mcs,
                "kernel": sweep_kernel_name(W.nbr, chosen), "bytes_per_site_update": BYTES_2D_GRAIN,
                "achieved_gbs": round(rate * BYTES_2D_GRAIN / 1e9, 1),
                "frac_of_measured_hbm": round(rate * BYTES_2D_GRAIN / 1e9 / peak, 4),
                "note": "two 64 MB lattices, partly L2-resident"}
    except Exception as e:  # secondary numbers must not break the main line
        return {"error": str(e)[:200]}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and the reference arm)
# ---------------------------------------------------------------------------
SAMPLE_EDGE = 56   # 3D sample of the bench workload family: same mean grain volume (about 1074 sites)


def oracle_job3d(edge, mcs, seed, n_refresh=1):
    """The oracle running the bench's job on an edge^3 lattice of the same grain
    density: Voronoi, then n_refresh periods of (2 plasticity increments at every
    material point, the Eq. (4) field, `mcs` Monte Carlo steps), then grain counts.
    Returns (site-updates, seconds)."""
    import oracle
    t0 = time.perf_counter()
    L = (edge, edge, edge)
    N = edge ** 3
    G = max(1, round(W4.G * N / W4.N))
    ex = W4.extra
    q, _ = oracle.voronoi(3, L, G, seed)
    quat = oracle.orientations(G, seed, 1)
    c = synth.TABLE1
    P = oracle.cp_params(c["C11"], c["C12"], c["C44"], c["tau0"], c["taus"], c["h0"], c["beta"], ex["e_incr"])
    grain = q.copy()
    mp = np.arange(N, dtype=np.int32)
    ep = np.zeros((N, 6))
    gm = np.zeros(N)
    thr, D = oracle.threshold_table(W4.kT)
    sweep0 = 0
    for r in range(n_refresh):
        ep, gm, sg, _, _ = oracle.mcp_run(P, seed, grain, quat, r * ex["incr_per_refresh"], ex["incr_per_refresh"], ep,
                                          gm)
        w, er = oracle.mcp_energies(P, sg, gm)
        bmp = oracle.quantise(ex["energy_scale"] * (w + er))
        q, _, mp, _ = oracle.sweep(3, L, 26, 256, seed, sweep0, mcs, thr, D, q, bmp[mp], mp)
        sweep0 += mcs
    oracle.grain_counts(q, G)
    return N * mcs * n_refresh, time.perf_counter() - t0


def _oracle_worker(a):
    edge, mcs, seed = a
    return oracle_job3d(edge, mcs, seed)


def cpu_baseline_sample(args, target_s=15.0):
    """The oracle as it stands on the host cores: one process per core, each on
    its own seed (independent replicas, as the GPU ranks), then one process alone."""
    mcs = int(args.mcs)
    n1, dt1 = oracle_job3d(SAMPLE_EDGE, mcs, W4.seed)
    cores = os.cpu_count() or 1
    ctx = mproc.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(SAMPLE_EDGE, mcs, W4.seed + 1 + i) for i in range(cores)])
    dt = time.perf_counter() - t0
    n = sum(r[0] for r in res)
    return {"value": round(n / dt, 1), "unit": "site-updates/s", "cores": cores, "kind": "oracle",
            "single_thread_value": round(n1 / dt1, 1),
            "sample": f"{SAMPLE_EDGE}^3 lattice of the same grain density ({max(1, round(W4.G * SAMPLE_EDGE**3 / W4.N))} "
                      f"grains), one refresh period (2 plasticity increments at every material point, Eq. (4) field, "
                      f"{mcs} MCS), Voronoi and counts included; {cores} independent processes (one per host core) "
                      f"for `value`, one process alone for `single_thread_value`",
            "seconds": round(dt, 2), "single_thread_seconds": round(dt1, 2)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    mcs = int(args.mcs)
    for _ in range(args.warmup):
        oracle_job3d(16, 2, W4.seed)
    tot_n, tot_s = 0, 0.0
    for k in range(args.steps):
        n, dt = oracle_job3d(SAMPLE_EDGE, mcs, W4.seed + k)
        tot_n += n
        tot_s += dt
    v = tot_n / tot_s
    L, N, G = shape3d(args.edge)
    line = {
        "metric": "Potts site-updates/s", "value": round(v, 1), "unit": "site-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot_s / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32 sweep; fp64 plasticity", "data": "synthetic", "impl": "reference",
        "config": {"workload": f"3d-{L[0]}-moore26-g{G}-plain-mcp-hybrid", "lattice": list(L), "nbr": 26,
                   "grains": G, "kT": W4.kT, "mcs_per_step": mcs, "parallelism": "cpu oracle, one process"},
        "cpu_baseline": {"value": round(v, 1), "unit": "site-updates/s", "kind": "oracle", "cores": 1,
                         "sample": f"each step: {SAMPLE_EDGE}^3 lattice of the same grain density, one refresh "
                                   f"period (2 plasticity increments, Eq. (4) field, {mcs} MCS), own seed"},
        "e2e": {"value": round(v, 1), "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# other workloads (one JSON line each; not part of the default run)
# ---------------------------------------------------------------------------
def run_3d_cp(args):
    """512^3, 26 neighbours, 2e5 grains, MCP refresh every 50 MCS (2 increments of 1e-4), kT 0.7."""
    import torch
    from paper_1007_3509_gb300 import build, hmcpotts as hm, hybrid
    build.build()
    torch.cuda.set_device(0)
    Wc = synth.W3D_CP
    L, G, N = Wc.L, Wc.G, Wc.N
    name = Wc.name
    if args.edge and args.edge != L[0]:
        e = int(args.edge)
        L, N = (e, e, e), e ** 3
        G = max(1, round(Wc.G * N / Wc.N))
        name = f"3d-{e}-moore26-g{G}-cp"
    ex = Wc.extra
    lat = hm.Lattice(3, L, 26, 256, Wc.seed, G, hm.FIELD_POINT)
    q = torch.empty(N, dtype=torch.int32, device="cuda")
    mp = torch.empty(N, dtype=torch.int32, device="cuda")
    lat.hp_bind(q, mp)
    quat = torch.empty(G, 4, dtype=torch.float32, device="cuda")
    prm = hybrid.cp_params_table1(ex["e_incr"], 7.0)
    eps = torch.empty(6 * N, device="cuda"); gam = torch.empty(N, device="cuda"); g = torch.empty(N, device="cuda")
    b = torch.empty(N, dtype=torch.int32, device="cuda")
    thr, D = hm.hp_build_threshold_table(Wc.kT)
    lat.hp_set_threshold_table(thr, D)
    lat.hp_set_field(b)
    lat.hp_init_voronoi(hm.ORIENT_SO3, quat)
    grain = q.clone()
    hm.hp_cp_reset(prm, N, eps, gam, g)
    hm.hp_cp_step(prm, Wc.seed, grain, quat, 0, 2, eps, gam, g, b=b)
    chosen, ms = lat.hp_sweep_autotune(2)
    res = []
    for rep in range(args.warmup + args.steps):
        timed = rep >= args.warmup
        e0, e1 = _events(torch)
        cp_ms = sw_ms = 0.0
        e0.record()
        lat.hp_set_sweep_counter(0)
        lat.hp_init_voronoi(hm.ORIENT_SO3, quat)
        grain.copy_(q)
        hm.hp_cp_reset(prm, N, eps, gam, g)
        incr = 0
        for k in range(args.mcs // ex["refresh_every"]):
            c0, c1 = _events(torch)
            c0.record()
            hm.hp_cp_step(prm, Wc.seed, grain, quat, incr, ex["incr_per_refresh"], eps, gam, g, b=b)
            c1.record()
            incr += ex["incr_per_refresh"]
            s0, s1 = _events(torch)
            s0.record()
            lat.hp_sweep(ex["refresh_every"])
            s1.record()
            torch.cuda.synchronize()
            cp_ms += c0.elapsed_time(c1)
            sw_ms += s0.elapsed_time(s1)
        counts = torch.empty(G, dtype=torch.int64, device="cuda")
        alive = torch.empty(1, dtype=torch.int32, device="cuda")
        lat.hp_grain_counts(counts, alive)
        e1.record()
        torch.cuda.synchronize()
        if timed:
            res.append((e0.elapsed_time(e1), cp_ms, sw_ms))
    tot = sum(r[0] for r in res) / len(res) / 1e3
    cp = sum(r[1] for r in res) / len(res) / 1e3
    sw = sum(r[2] for r in res) / len(res) / 1e3
    peak, _ = peaks()
    rate_sw = N * args.mcs / sw
    print(json.dumps({
        "metric": "Potts site-updates/s", "value": round(N * args.mcs / tot, 1), "unit": "site-updates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot * 1e3, 2),
        "higher_is_better": True, "dtype": "int32 sweep / fp32+fp64 plasticity", "data": "synthetic",
        "config": {"workload": name, "lattice": list(L), "grains": G, "kT": Wc.kT, "mcs": args.mcs,
                   "refresh": "MCP every 50 MCS, 2 increments of 1e-4", "tile": {"variant": int(chosen),
                   "ms_per_2_mcs": [round(float(x), 3) for x in ms]}},
        "sweep": {"site_updates_per_s": round(rate_sw, 1), "bytes_per_site_update": BYTES_3D_POINT,
                  "achieved_gbs": round(rate_sw * BYTES_3D_POINT / 1e9, 1),
                  "frac_of_measured_hbm": round(rate_sw * BYTES_3D_POINT / 1e9 / peak, 4),
                  "seconds": round(sw, 3)},
        "plasticity": {"point_increments_per_s": round(N * incr / cp, 1), "seconds": round(cp, 3),
                       "increments": incr, "points": N},
        "alive_grains": int(alive.item())}))


def run_ensemble(args):
    """256 replicas, edges {64..256}, kT U[0.5,0.9], load U[50,200] MPa, 500-20000 grains, 200 MCS."""
    import torch
    from paper_1007_3509_gb300 import build, hmcpotts as hm
    build.build()
    torch.cuda.set_device(0)
    members, bufs = [], []
    C = [synth.NI_BJ[k] for k in ("C11", "C12", "C44")]
    t0 = time.perf_counter()
    for m in synth.ensemble_members():
        L = (m["edge"],) * 3
        N = m["edge"] ** 3
        lat = hm.Lattice(3, L, 26, 256, m["seed"], m["G"], hm.FIELD_GRAIN)
        q = torch.empty(N, dtype=torch.int32, device="cuda")
        lat.hp_bind(q)
        quat = torch.empty(m["G"], 4, device="cuda")
        lat.hp_init_voronoi(hm.ORIENT_SO3, quat)
        bg = torch.empty(m["G"], dtype=torch.int32, device="cuda")
        hm.hp_grain_field(quat, *C, m["sigma"], 0.05, 1.0, bg)
        lat.hp_set_field(bg)
        thr, D = hm.hp_build_threshold_table(m["kT"])
        lat.hp_set_threshold_table(thr, D)
        members.append(lat)
        bufs.append((q, quat, bg))
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    sites = sum(l.N for l in members)
    ens = hm.Ensemble(members)
    chosen, ms = ens.hp_ensemble_autotune(1)
    times = []
    for rep in range(args.warmup + args.steps):
        e0, e1 = _events(torch)
        e0.record()
        ens.hp_ensemble_sweep(args.mcs)
        e1.record()
        torch.cuda.synchronize()
        if rep >= args.warmup:
            times.append(e0.elapsed_time(e1) / 1e3)
    t = sum(times) / len(times)
    rate = sites * args.mcs / t
    peak, _ = peaks()
    print(json.dumps({
        "metric": "Potts site-updates/s", "value": round(rate, 1), "unit": "site-updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 2), "higher_is_better": True,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": "ensemble-256-replicas-3d-moore26", "replicas": len(members), "sites": sites,
                   "mcs": args.mcs, "launch": "one CUDA graph replay per step (2 batched kernels per MCS)",
                   "tile": {"variant": int(chosen), "ms_per_mcs": [round(float(x), 3) for x in ms]},
                   "init_seconds": round(init_s, 2)},
        "roofline": {"bound": "hbm", "bytes_per_site_update": 8, "achieved": round(rate * 8 / 1e9, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(rate * 8 / 1e9 / peak, 4)}}))


def run_surrogate(args):
    """1024^3, 10^6 grains: plain MCP-driven hybrid vs surrogate-driven hybrid, wall time to 500 MCS
    (surrogate time includes generating its data and training it) and texture fractions."""
    import torch
    from paper_1007_3509_gb300 import build, hmcpotts as hm, hybrid
    build.build()
    torch.cuda.set_device(0)
    Wc = synth.W3D_SURROGATE
    cfg = hybrid.HybridConfig(L=Wc.L, G=Wc.G, seed=Wc.seed, kT=Wc.kT, n_mcs=args.mcs)
    t0 = time.perf_counter()
    prm = hybrid.cp_params_table1(cfg.e_incr, cfg.energy_scale)
    params, load, loss, _ = hybrid.train_surrogate(torch, prm)
    train_s = time.perf_counter() - t0
    sur = hybrid.run_surrogate(torch, cfg, params, load)
    torch.cuda.empty_cache()
    plain = hybrid.run_plain(torch, cfg)
    print(json.dumps({
        "metric": "time-to-texture (s)", "value": round(train_s + sur["wall_s"], 2), "unit": "s",
        "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
        "config": {"workload": Wc.name, "lattice": list(Wc.L), "grains": Wc.G, "mcs": args.mcs,
                   "refresh": "every 50 MCS"},
        "surrogate": {"train_seconds": round(train_s, 2), "run_seconds": round(sur["wall_s"], 2),
                      "final_loss": loss, "families": [round(x, 5) for x in sur["families"]],
                      "field_seconds": round(sur["field_s"], 3)},
        "plain": {"run_seconds": round(plain["wall_s"], 2), "families": [round(x, 5) for x in plain["families"]],
                  "field_seconds": round(plain["field_s"], 3)},
        "speedup": round(plain["wall_s"] / (train_s + sur["wall_s"]), 3)}))


def run_sweep3d(args):
    """The 3D 26-neighbour sweep alone on an edge^3 lattice (default 512^3, 2e5 grains
    at that size, the same mean grain volume at others) with a per-point field and
    the material-point index carried."""
    import torch
    from paper_1007_3509_gb300 import build, hmcpotts as hm
    build.build()
    torch.cuda.set_device(0)
    e = int(args.edge or 512)
    L, N = (e, e, e), e ** 3
    G = max(1, round(200_000 * N / 512 ** 3))
    lat = hm.Lattice(3, L, 26, 256, 1002, G, hm.FIELD_POINT)
    q = torch.empty(N, dtype=torch.int32, device="cuda")
    mp = torch.empty(N, dtype=torch.int32, device="cuda")
    lat.hp_bind(q, mp)
    lat.hp_init_voronoi(hm.ORIENT_SO3, None)
    bmp = torch.randint(0, 30, (N,), dtype=torch.int32, device="cuda", generator=torch.Generator("cuda").manual_seed(7))
    lat.hp_set_field(bmp)
    thr, D = hm.hp_build_threshold_table(0.7)
    lat.hp_set_threshold_table(thr, D)
    if args.variant is None:
        chosen, _ = lat.hp_sweep_autotune(2)
    else:
        chosen = args.variant
        lat.hp_set_sweep_variant(chosen)
    for _ in range(args.warmup):
        lat.hp_sweep(1)
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    lat.hp_sweep(args.mcs)
    e1.record()
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1e3
    rate = N * args.mcs / s
    peak, _ = peaks()
    print(json.dumps({"metric": "Potts site-updates/s", "value": round(rate, 1), "unit": "site-updates/s",
                      "config": {"workload": f"3d-{e}-moore26-g{G}-point-field", "variant": int(chosen),
                                 "kernel": sweep_kernel_name(26, chosen), "mcs": args.mcs},
                      "roofline": {"bound": "hbm", "bytes_per_site_update": BYTES_3D_POINT,
                                   "achieved": round(rate * BYTES_3D_POINT / 1e9, 1),
                                   "peak": peak, "frac": round(rate * BYTES_3D_POINT / 1e9 / peak, 4)}}))


def run_texture(args):
    """Sec. 5 texture experiments: the 2D Gaussian bulk energy of Eq. (9) over a 100-replica
    ensemble of 500^2 lattices, or the 3D plastic case with the g(t) fit of Eq. (10)."""
    import torch
    from paper_1007_3509_gb300 import build, texture
    build.build()
    torch.cuda.set_device(0)
    # one untimed run of the same configuration first: the first run in a process
    # also pays one-time start-up (module loading, first graph instantiation)
    if args.workload == "texture2d":
        sl = (0, args.mcs // 10, args.mcs // 3, args.mcs)
        texture.run_gaussian_2d(torch, slices=(0, 10))
        r = texture.run_gaussian_2d(torch, slices=sl)
        low = list(range(0, 10)) + list(range(80, 90))
        print(json.dumps({"workload": "texture2d-gaussian-eq9-100x500^2", "slices": list(sl),
                          "mean_b_J": [round(x, 5) for x in r["mean_b"]],
                          "low_energy_fraction": [round(float(h[low].sum() / h.sum()), 4) for h in r["hist"]],
                          "seconds": round(r["seconds"], 3), "warmup": "one untimed run of 10 MCS",
                          "timed": "sweeps + per-slice measurement of all 100 members",
                          "site_updates_per_s": round(100 * 500 * 500 * args.mcs / r["seconds"], 1)}))
    else:
        n_incr = max(1, args.mcs // 2)
        kw = dict(L=(256, 256, 256), G=32000, kT=1.0, mcs_per_incr=2, e_incr=1e-4, energy_scale=200.0)
        texture.run_plastic_3d(torch, n_incr=2, every=1, **kw)
        r = texture.run_plastic_3d(torch, n_incr=n_incr, every=max(1, n_incr // 10), **kw)
        print(json.dumps({"workload": "texture3d-plastic-zrot-256^3", "grains": 32000, "kT": 1.0,
                          "e_incr": 1e-4, "energy_scale": 200.0, "mcs": 2 * n_incr, "t": r["t"],
                          "g_deg": [round(x, 3) for x in r["g"]], "seconds": round(r["seconds"], 3),
                          "warmup": "one untimed run of 2 increments"}))


def run_2d(args):
    """The 4096^2 Moore line on its own (partly L2-resident; not the HBM figure)."""
    import torch
    from paper_1007_3509_gb300 import build, hmcpotts as hm
    build.build()
    torch.cuda.set_device(0)
    print(json.dumps({"metric": "Potts site-updates/s", **run_2d_secondary(torch, hm)}))


def run_texture_seeds(args):
    """Both 1024^3 hybrids over `--seeds` seeds each: the texture family fractions
    and the mean max Schmid factor of the two arms compared within two standard
    errors, and each arm's wall time to 500 MCS (the surrogate trained once)."""
    import torch
    from paper_1007_3509_gb300 import build, hmcpotts as hm, hybrid
    build.build()
    torch.cuda.set_device(0)
    L, N, G = shape3d(args.edge)
    prm = hybrid.cp_params_table1(1e-4, 7.0)
    t0 = time.perf_counter()
    params, load, loss, _ = hybrid.train_surrogate(torch, prm)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    plain, sur = [], []
    for k in range(args.seeds):
        cfg = hybrid.HybridConfig(L=L, G=G, seed=W4.seed + 100 * k, kT=W4.kT, n_mcs=args.mcs)
        plain.append(hybrid.run_plain(torch, cfg, time_it=False))
        torch.cuda.empty_cache()
        sur.append(hybrid.run_surrogate(torch, cfg, params, load, time_it=False))
        torch.cuda.empty_cache()
    fp = np.array([r["families"] for r in plain])
    fs = np.array([r["families"] for r in sur])
    mp_ = np.array([r["mean_mmax"] for r in plain])
    ms = np.array([r["mean_mmax"] for r in sur])
    rows = []
    for name, a, b in [("none", fp[:, 0], fs[:, 0]), ("100", fp[:, 1], fs[:, 1]), ("110", fp[:, 2], fs[:, 2]),
                       ("111", fp[:, 3], fs[:, 3]), ("mean_mmax", mp_, ms)]:
        se = float(np.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b)))
        d = float(a.mean() - b.mean())
        rows.append({"quantity": name, "plain_mean": round(float(a.mean()), 6), "surrogate_mean": round(float(b.mean()), 6),
                     "difference": round(d, 6), "two_se": round(2 * se, 6), "within_2se": bool(abs(d) <= 2 * se + 1e-9)})
    print(json.dumps({"workload": f"texture-seeds-3d-{L[0]}-g{G}", "seeds_per_arm": args.seeds, "mcs": args.mcs,
                      "agreement": rows, "all_within_2se": all(r["within_2se"] for r in rows),
                      "plain_s_mean": round(float(np.mean([r["wall_s"] for r in plain])), 3),
                      "surrogate_run_s_mean": round(float(np.mean([r["wall_s"] for r in sur])), 3),
                      "surrogate_train_s": round(train_s, 3),
                      "time_to_texture_s": {"plain": round(float(np.mean([r["wall_s"] for r in plain])), 3),
                                            "surrogate": round(train_s + float(np.mean([r["wall_s"] for r in sur])), 3)},
                      "final_train_loss": loss}))


def run_3d_eq(args):
    """The plasticity-driven hybrid with each increment iterated to periodic elastic
    equilibrium (Sec. 5) against the Taylor coupling of Eq. (3), same lattice
    (default 256^3, 32000 grains), 500 MCS, refresh every 50 MCS (2 increments)."""
    import torch
    from paper_1007_3509_gb300 import build, hybrid
    build.build()
    torch.cuda.set_device(0)
    e = int(args.edge or 256)
    L = (e, e, e)
    G = max(1, round(W4.G * e ** 3 / W4.N))
    cfg = hybrid.HybridConfig(L=L, G=G, seed=1002, kT=W4.kT, n_mcs=args.mcs)
    hybrid.run_plain(torch, hybrid.HybridConfig(L=L, G=G, seed=1002, kT=W4.kT, n_mcs=50), coupling="equilibrium")
    out = {}
    for coupling in ("taylor", "equilibrium"):
        r = hybrid.run_plain(torch, cfg, coupling=coupling)
        out[coupling] = {"wall_s": round(r["wall_s"], 3), "field_s": round(r["field_s"], 3),
                         "families": [round(x, 5) for x in r["families"]], "mean_mmax": round(r["mean_mmax"], 5),
                         "alive": r["alive"]}
        if coupling == "equilibrium":
            it = r["elastic_iterations"]
            out[coupling]["elastic_solves"] = len(it)
            out[coupling]["elastic_iterations_mean"] = round(float(np.mean(it)), 2)
        torch.cuda.empty_cache()
    print(json.dumps({"workload": f"3d-{e}-moore26-g{G}-equilibrium-vs-taylor", "mcs": args.mcs,
                      "refresh": "every 50 MCS, 2 increments of 1e-4", "elastic_tolerance": 1e-5, **out}))


def run_aniso(args):
    """Misorientation-dependent pair energy (Read-Shockley, theta_m = 15 degrees) and
    mobility on the 2D Moore lattice of grains rotated about z (1024^2, 625 grains:
    the 4096^2 workload's grain density), kT 0.6: site-updates/s of the per-colour
    kernel with the tables against the same kernel and the fused kernel without."""
    import torch
    from paper_1007_3509_gb300 import build, hmcpotts as hm
    build.build()
    torch.cuda.set_device(0)
    L, G, N = (1024, 1024), 625, 1024 * 1024
    out = {}
    for name in ("pair_energy_and_mobility", "constant_J_per_colour", "constant_J_fused"):
        lat = hm.Lattice(2, L, 8, 256, 1001, G, hm.FIELD_NONE)
        q = torch.empty(N, dtype=torch.int32, device="cuda")
        lat.hp_bind(q)
        ang = torch.empty(G, device="cuda")
        lat.hp_init_voronoi(hm.ORIENT_ANGLE, ang)
        lat.hp_set_threshold_table(*hm.hp_build_threshold_table(0.6))
        if name == "pair_energy_and_mobility":
            units = torch.empty(G, dtype=torch.int32, device="cuda")
            hm.hp_angle_units(G, hm.ORIENT_ANGLE, ang, 1000, 90000, units)
            J, m = hm.hp_build_read_shockley(1.0, 15.0, 250, 181, 1000, mobility=True)
            lat.hp_set_anisotropy(units, 90000, 250, J, m)
        if name == "constant_J_per_colour":
            lat.hp_set_sweep_kernel(hm.SWEEP_PHASE)
        lat.hp_sweep(5)
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        lat.hp_sweep(args.mcs)
        e1.record()
        torch.cuda.synchronize()
        st, _ = lat.hp_measure()
        out[name] = {"site_updates_per_s": round(N * args.mcs / (e0.elapsed_time(e1) / 1e3), 1),
                     "alive_after": int(st.alive)}
        lat.close()
    print(json.dumps({"workload": "aniso-2d-1024-moore8-g625-read-shockley", "mcs": args.mcs, "kT": 0.6, **out}))


def run_small2d(args):
    """The small 2D workload: 128^2, 4 neighbours (red/black), 64 Voronoi grains
    with one angle each, per-grain stored energy U[0, 0.1] J in fixed point, J = 1,
    kT 0.5, 100 MCS per step.  A 64 KB lattice, so launch- and latency-bound:
    site-updates/s with the sweep's kernel launches issued per call (hp_sweep)
    against one CUDA-graph replay per step (a one-lattice hp_ensemble); both
    lattices must agree site for site.  The oracle's time for the same job is the
    CPU baseline."""
    import torch
    from paper_1007_3509_gb300 import build, hmcpotts as hm
    build.build()
    torch.cuda.set_device(0)
    Wk = synth.W2D_SMALL
    N = Wk.N
    b_grain = np.rint(256.0 * synth.uniform_energies(Wk.G, 0.1, Wk.seed + 1)).astype(np.int32)
    thr, D = hm.hp_build_threshold_table(Wk.kT)

    def make():
        lat = hm.Lattice(2, Wk.L, 4, 256, Wk.seed, Wk.G, hm.FIELD_GRAIN)
        q = torch.empty(N, dtype=torch.int32, device="cuda")
        lat.hp_bind(q)
        ang = torch.empty(Wk.G, device="cuda")
        lat.hp_init_voronoi(hm.ORIENT_ANGLE, ang)
        b = torch.from_numpy(b_grain).cuda()
        lat.hp_set_field(b)
        lat.hp_set_threshold_table(thr, D)
        return lat, q, b

    lat, q, b = make()
    q0 = q.cpu().numpy()
    glat, gq, gb = make()
    ens = hm.Ensemble([glat])
    # each path runs the tile variant its own autotuner picks (state restored)
    v_launch, _ = lat.hp_sweep_autotune(2)
    v_graph, _ = ens.hp_ensemble_autotune(2)
    out = {"variant_launches": int(v_launch), "variant_graph": int(v_graph)}
    for name, run in (("launches", lambda: lat.hp_sweep(args.mcs)), ("graph", lambda: ens.hp_ensemble_sweep(args.mcs))):
        times = []
        for rep in range(args.warmup + args.steps):
            e0, e1 = _events(torch)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            if rep >= args.warmup:
                times.append(e0.elapsed_time(e1) / 1e3)
        t = statistics.median(times)
        out[name] = {"site_updates_per_s": round(N * args.mcs / t, 1), "us_per_mcs": round(t / args.mcs * 1e6, 2)}
    same = bool(torch.equal(q, gq))
    import oracle
    othr, oD = oracle.threshold_table(Wk.kT)
    t0 = time.perf_counter()
    ref, _, _, _ = oracle.sweep(2, Wk.L, 4, 256, Wk.seed, 0, args.mcs, othr, oD, q0, b_grain[q0])
    cpu_s = time.perf_counter() - t0
    # the GPU lattice after its first step equals the oracle's after the same MCS
    lat2, q2, b2 = make()
    lat2.hp_sweep(args.mcs)
    torch.cuda.synchronize()
    exact = bool(np.array_equal(q2.cpu().numpy(), ref))
    print(json.dumps({"workload": Wk.name, "lattice": list(Wk.L), "nbr": 4, "grains": Wk.G, "kT": Wk.kT,
                      "mcs_per_step": args.mcs, "steps": args.steps, "warmup": args.warmup, **out,
                      "graph_over_launches": round(out["graph"]["site_updates_per_s"] /
                                                   out["launches"]["site_updates_per_s"], 3),
                      "graph_and_launches_agree": same, "bit_exact_vs_oracle_first_step": exact,
                      "cpu_baseline": {"value": round(N * args.mcs / cpu_s, 1), "unit": "site-updates/s",
                                       "kind": "oracle", "cores": 1, "sample": f"the same {args.mcs} MCS"}}))
    for l in (lat, glat, lat2):
        l.close()


def run_surrogate_train(args):
    """The surrogate's training on its own: 65536 orientations x 20 load steps of
    plasticity samples (128 histories each), Adam on 972-orientation minibatches
    (one wave of 128-row tiles) for --train-steps steps; time per step, and the
    field error on 256 held-out orientations against 4096-history averages."""
    import torch
    from paper_1007_3509_gb300 import build, hmcpotts as hm, hybrid
    build.build()
    torch.cuda.set_device(0)
    prm = hybrid.cp_params_table1(1e-4, 7.0)
    hybrid.train_surrogate(torch, prm, steps=100)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    params, load, loss, _ = hybrid.train_surrogate(torch, prm, steps=args.train_steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    n_orient, K, n_incr = 256, 4096, 20
    quat = torch.empty(n_orient, 4, device="cuda")
    hm.hp_orientations(n_orient, 999, hm.ORIENT_SO3, quat)
    X = torch.empty(n_orient * n_incr, 11, device="cuda")
    Y = torch.empty(n_orient * n_incr, 2, device="cuda")
    hm.hp_sur_generate(prm, 4242, quat, n_orient, K, n_incr, X, Y)
    P = torch.empty_like(Y)
    hm.hp_mlp_forward(params, X, P)
    torch.cuda.synchronize()
    y, pr = Y.cpu().numpy().astype(np.float64), P.cpu().numpy().astype(np.float64)
    sw, se = hm.SUR_SCALES.w, hm.SUR_SCALES.erho
    e_ref = y[:, 0] * sw + y[:, 1] * se
    e_sur = pr[:, 0] * sw + pr[:, 1] * se
    err = float(np.linalg.norm(e_sur - e_ref) / np.linalg.norm(e_ref))
    print(json.dumps({"workload": "surrogate-train-65536x20-batch19440", "steps": args.train_steps,
                      "train_s": round(dt, 3), "us_per_step": round(dt / args.train_steps * 1e6, 2),
                      "final_loss": loss, "field_rel_error": round(err, 5), "bound": 1e-2}))


def run_mcp_vs_det(args):
    """Sec. 2, Fig. 1 at scale: the Monte Carlo plasticity against the deterministic
    multi-slip model (FP64, pseudo-inverse of the active constraints).  (1) Speed:
    10^6 material points of random orientation, 20 Taylor increments of 1e-4 from
    rest (the hybrid's refresh load), point-increments/s of each kernel.  (2)
    Agreement: 4096 orientations, 2000 increments of 1e-6 (the paper's test),
    sample-frame sigma_xx of both models every increment."""
    import torch
    from paper_1007_3509_gb300 import build, hmcpotts as hm, synth
    build.build()
    torch.cuda.set_device(0)
    T = synth.TABLE1
    out = {}
    rng = np.random.default_rng(1007)
    for P, e, n, tag in ((1_000_000, 1e-4, 20, "speed"), (4096, 1e-6, 2000, "agreement")):
        q = rng.normal(size=(P, 4)).astype(np.float32)
        q /= np.linalg.norm(q, axis=1, keepdims=True)
        quat = torch.from_numpy(q).cuda()
        grain = torch.arange(P, dtype=torch.int32, device="cuda")
        prm = hm.cp_params(T["C11"], T["C12"], T["C44"], T["tau0"], T["taus"], T["h0"], T["beta"], e)
        mep, mgm, mg = (torch.empty(6 * P, device="cuda"), torch.empty(P, device="cuda"),
                        torch.empty(P, device="cuda"))
        dep, dgm = torch.empty(6 * P, dtype=torch.float64, device="cuda"), torch.empty(P, dtype=torch.float64,
                                                                                       device="cuda")
        ms = torch.empty(6 * P, device="cuda")
        ds = torch.empty(6 * P, dtype=torch.float64, device="cuda")
        na = torch.empty(P, dtype=torch.int32, device="cuda")
        if tag == "speed":
            times = {}
            for rep in range(3):
                for model in ("mcp", "det"):
                    hm.hp_cp_reset(prm, P, mep, mgm, mg)
                    hm.hp_det_reset(P, dep, dgm)
                    torch.cuda.synchronize()
                    e0, e1 = _events(torch)
                    e0.record()
                    if model == "mcp":
                        hm.hp_cp_step(prm, 7, grain, quat, 0, n, mep, mgm, mg, sigma=ms)
                    else:
                        hm.hp_det_step(prm, grain, quat, 0, n, dep, dgm, sigma=ds, n_active=na)
                    e1.record()
                    torch.cuda.synchronize()
                    if rep:
                        times.setdefault(model, []).append(e0.elapsed_time(e1))
            act = na.cpu().numpy()
            out[tag] = {"points": P, "increments": n, "e": e,
                        "mcp_point_increments_per_s": round(P * n / (np.median(times["mcp"]) / 1e3), 1),
                        "det_point_increments_per_s": round(P * n / (np.median(times["det"]) / 1e3), 1),
                        "mcp_ms": round(float(np.median(times["mcp"])), 3),
                        "det_ms": round(float(np.median(times["det"])), 3),
                        "det_active_systems_hist": np.bincount(act[act >= 0], minlength=9)[:9].tolist(),
                        "det_unsettled": int((act < 0).sum())}
            out[tag]["det_over_mcp_time"] = round(out[tag]["det_ms"] / out[tag]["mcp_ms"], 2)
        else:
            hm.hp_cp_reset(prm, P, mep, mgm, mg)
            hm.hp_det_reset(P, dep, dgm)
            R = torch.from_numpy(np.stack([_rot_np(v) for v in q])).cuda()
            r0 = R[:, 0, :]

            def sxx(v):
                v = v.view(6, P).double()
                return (r0[:, 0] ** 2 * v[0] + r0[:, 1] ** 2 * v[1] + r0[:, 2] ** 2 * v[2] +
                        2 * (r0[:, 1] * r0[:, 2] * v[3] + r0[:, 0] * r0[:, 2] * v[4] + r0[:, 0] * r0[:, 1] * v[5]))

            Dc, Mc, Ac = [], [], []
            for t in range(n):
                hm.hp_det_step(prm, grain, quat, t, 1, dep, dgm, sigma=ds, n_active=na)
                hm.hp_cp_step(prm, 13, grain, quat, t, 1, mep, mgm, mg, sigma=ms)
                Dc.append(sxx(ds))
                Mc.append(sxx(ms))
                Ac.append(na.clone())
            torch.cuda.synchronize()
            D = torch.stack(Dc).cpu().numpy()
            M = torch.stack(Mc).cpu().numpy()
            A = torch.stack(Ac).cpu().numpy()
            rel = (M - D) / D
            multi = A >= 2
            means = np.array([rel[multi[:, i], i].mean() for i in range(P) if multi[:, i].sum() > 200])
            out[tag] = {"orientations": P, "increments": n, "e": e,
                        "multi_slip_mean_rel_dev": round(float(means.mean()), 5),
                        "multi_slip_mean_rel_dev_q05_q95": [round(float(np.quantile(means, 0.05)), 5),
                                                            round(float(np.quantile(means, 0.95)), 5)],
                        "orientations_with_multi_slip": int(means.size),
                        "max_active_systems": int(A.max()), "det_unsettled": int((A < 0).sum()),
                        "curve_orientation0_MPa_every_200": {
                            "strain": [round((t + 1) * e, 6) for t in range(0, n, 200)],
                            "det": [round(float(D[t, 0]), 4) for t in range(0, n, 200)],
                            "mcp": [round(float(M[t, 0]), 4) for t in range(0, n, 200)]}}
        del mep, mgm, mg, dep, dgm, ms, ds, na
        torch.cuda.empty_cache()
    print(json.dumps({"workload": "mcp-vs-det-ni-single-crystals", "material": "Table 1 nickel", **out}))


def _rot_np(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def main():
    args = parse()
    if args.impl == "ours" and args.workload not in ("3d",):
        {"2d": run_2d, "3d-cp": run_3d_cp, "ensemble": run_ensemble, "surrogate": run_surrogate,
         "sweep3d": run_sweep3d, "texture2d": run_texture, "texture3d": run_texture,
         "texture-seeds": run_texture_seeds, "3d-eq": run_3d_eq, "aniso": run_aniso,
         "mcp-vs-det": run_mcp_vs_det, "surrogate-train": run_surrogate_train,
         "small2d": run_small2d}[args.workload](args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
