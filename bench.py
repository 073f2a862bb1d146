#!/usr/bin/env python
"""Benchmark: Potts site-updates/s of the hybrid Monte Carlo hot path on GB300.

Workload (default): 2D 4096x4096 periodic lattice, Moore 8-neighbour 4-colour
sweep, 10^4 Voronoi grains with SO(3)-uniform cubic-Ni orientations, per-grain
field = elastic energy under uniaxial 100 MPa + dislocation energy weighted by
the max Schmid factor, kT = 0.6, 1000 MCS.  One step = the whole job on
synthetic input already in HBM: Voronoi initialisation, closed-form field,
1000 MCS, grain counts and texture histogram.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  With N > 1 (torchrun, one rank per GPU) every
rank runs its own independent lattice (its own seed): weak scaling, no
collective on the data path; the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1007_3509_gb300 import synth  # noqa: E402

W = synth.W2D_MOORE
BYTES_PER_SITE_UPDATE = 8  # q read + q write per site per MCS; field looked up per grain (L1/L2)
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
    p.add_argument("--mcs", type=int, default=None, help="MCS per step (default: the workload's)")
    p.add_argument("--variant", type=int, default=None, help="fused-sweep tile variant (default: autotuned)")
    p.add_argument("--workload", choices=["2d", "3d-cp", "ensemble", "surrogate", "sweep3d", "texture2d",
                                          "texture3d"], default="2d",
                   help="2d: 4096^2 Moore (default line); 3d-cp: 512^3 plasticity-driven hybrid; ensemble: 256 "
                        "replicas; surrogate: 1024^3 plain vs surrogate time-to-texture")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--edge", type=int, default=None,
                   help="3d-cp: lattice edge (default 512); grains scale with the volume")
    a = p.parse_args()
    if a.mcs is None:
        a.mcs = {"2d": W.n_mcs, "3d-cp": 500, "ensemble": 200, "surrogate": 500, "sweep3d": 20, "texture2d": 1000,
                 "texture3d": 400}[a.workload]
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


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
class Job:
    """Device-resident buffers of one lattice of the workload."""

    def __init__(self, torch, hm, seed, mcs):
        self.torch, self.hm, self.mcs = torch, hm, mcs
        L, G = W.L, W.G
        self.N = int(np.prod(L))
        dev = "cuda"
        self.lat = hm.Lattice(2, L, W.nbr, int(256 * W.J), seed, G, hm.FIELD_GRAIN)
        self.q = torch.empty(self.N, dtype=torch.int32, device=dev)
        self.lat.hp_bind(self.q)
        self.quat = torch.empty(G, 4, dtype=torch.float32, device=dev)
        self.bgrain = torch.empty(G, dtype=torch.int32, device=dev)
        self.counts = torch.empty(G, dtype=torch.int64, device=dev)
        self.alive = torch.empty(1, dtype=torch.int32, device=dev)
        self.bins = torch.empty(2 * G, dtype=torch.int32, device=dev)
        self.hist = torch.empty(24, dtype=torch.int64, device=dev)
        thr, D = hm.hp_build_threshold_table(W.kT)
        self.lat.hp_set_threshold_table(thr, D)
        self.lat.hp_set_field(self.bgrain)
        self.C = [synth.NI_BJ[k] for k in ("C11", "C12", "C44")]
        self.tuned = None

    def autotune(self):
        """Pick the fastest tile shape on the initialised lattice (state restored)."""
        self.lat.hp_init_voronoi(self.hm.ORIENT_SO3, self.quat)
        self.field()
        chosen, ms = self.lat.hp_sweep_autotune(8)
        self.tuned = {"variant": int(chosen), "ms_per_8_mcs": [round(float(x), 3) for x in ms]}

    def field(self):
        self.hm.hp_grain_field(self.quat, *self.C, W.sigma, W.k_disl, W.energy_scale, self.bgrain)

    def measure(self):
        self.lat.hp_grain_counts(self.counts, self.alive)
        self.hm.hp_texture(W.G, self.hm.ORIENT_SO3, self.quat, self.counts, self.bins, self.hist)

    def step(self, ev_sweep=None):
        """Whole job: init, field, sweep, measure."""
        self.lat.hp_init_voronoi(self.hm.ORIENT_SO3, self.quat)
        self.field()
        self.lat.hp_set_sweep_counter(0)
        if ev_sweep:
            ev_sweep[0].record()
        self.lat.hp_sweep(self.mcs)
        if ev_sweep:
            ev_sweep[1].record()
        self.measure()


# algorithmic bytes per site-update of the 3D per-material-point-field sweep:
# the per-site state (grain id q, stored energy b, material point mp) read and
# written once per MCS
BYTES_3D_POINT = 24

# dram__bytes_read.sum + dram__bytes_write.sum per launch, ncu capture of the
# 4096^2 Moore workload, keyed by (neighbours, tile variant)
MEASURED_TRAFFIC = {(8, 10): 67.998208e6 + 19.811072e6}


def sweep_kernel_name(nbr, variant):
    """Kernel family of a fused-sweep tile variant (variant numbering of hp_sweep_variants)."""
    v = int(variant or 0)
    plane_n = 6 if nbr == 26 else 5
    strip_end = 9
    if v < plane_n:
        kind = "k_plane_tma" if (v >= plane_n - 2) else "k_plane"
    elif v < strip_end:
        kind = "k_strip"
    else:
        kind = "k_tile"
    return f"{kind}<{nbr}> (fused MCS, variant {v})"


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1007_3509_gb300 import build, hmcpotts as hm
    torch.cuda.set_device(local_rank)
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    hm.lib()
    job = Job(torch, hm, W.seed + rank, args.mcs)
    if args.variant is not None:
        job.lat.hp_set_sweep_variant(args.variant)
        job.tuned = {"variant": int(args.variant), "ms_per_8_mcs": None}
    elif not args.no_autotune:
        job.autotune()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        job.step()
    torch.cuda.synchronize()

    clocks = Clocks(local_rank)
    launches0 = hm.hp_kernel_launches()
    step_ms, sweep_ms = [], []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        job.step((s0, s1))
        e1.record()
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        sweep_ms.append(s0.elapsed_time(s1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = hm.hp_kernel_launches() - launches0
    total_ms = sum(step_ms)
    max_ms, value = aggregate(total_ms, job.N * args.mcs * args.steps, world, "cuda")

    # dominant kernel: one fused-plane launch per MCS over N sites
    per_launch_s = statistics.mean(sweep_ms) / 1e3 / args.mcs
    achieved = BYTES_PER_SITE_UPDATE * job.N / per_launch_s / 1e9
    peak, peak_kind = peaks()
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None, "peak_source": peak_kind,
            "kernel": sweep_kernel_name(W.nbr, job.tuned.get("variant") if job.tuned else 0),
            "bytes_per_site_update": BYTES_PER_SITE_UPDATE,
            "sweep_site_updates_per_s": round(job.N / per_launch_s, 1)}
    # DRAM bytes of one launch of the kernel, from an ncu capture of that exact
    # variant (profiles/k_tile8_2d4096_moore.md); null for any other kernel
    traffic = MEASURED_TRAFFIC.get((W.nbr, job.tuned.get("variant") if job.tuned else None))
    if traffic is not None:
        roof["traffic"] = traffic

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(torch, hm, job, args)
    secondary = None
    if not args.no_secondary and rank == 0:
        secondary = run_secondary(torch, hm)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(target_s=12.0)
    if rank != 0:
        return
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
        "dtype": "int32",
        "data": "synthetic (seeded Voronoi polycrystal, SO(3)-uniform orientations)",
        "config": {"workload": W.name, "lattice": list(W.L), "nbr": W.nbr, "colours": 4, "grains": W.G,
                   "kT": W.kT, "mcs_per_step": args.mcs, "field": "per-grain closed form (100 MPa, Ni)",
                   "step": "voronoi init + field + sweep + counts/texture", "l2": "flushed between steps",
                   "parallelism": f"replicas x{world}", "tile": job.tuned},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "secondary": secondary,
    }
    print(json.dumps(line))


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


def run_e2e(torch, hm, job, args):
    """Same metric through the public API with host buffers: pinned H2D of the
    initial lattice and orientations, field + sweep + measure, D2H of the final
    lattice, counts and histogram, every step."""
    G, N = W.G, job.N
    job.lat.hp_init_voronoi(hm.ORIENT_SO3, job.quat)
    h_q = job.q.cpu().pin_memory()
    h_quat = job.quat.cpu().pin_memory()
    o_q = torch.empty(N, dtype=torch.int32).pin_memory()
    o_counts = torch.empty(G, dtype=torch.int64).pin_memory()
    o_hist = torch.empty(24, dtype=torch.int64).pin_memory()

    def one():
        job.q.copy_(h_q, non_blocking=True)
        job.quat.copy_(h_quat, non_blocking=True)
        job.field()
        job.lat.hp_set_sweep_counter(0)
        job.lat.hp_sweep(args.mcs)
        job.measure()
        o_q.copy_(job.q, non_blocking=True)
        o_counts.copy_(job.counts, non_blocking=True)
        o_hist.copy_(job.hist, non_blocking=True)

    one()
    torch.cuda.synchronize()
    ms = []
    steps = max(2, min(args.steps, 3))
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        one()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    per = statistics.mean(ms) / 1e3
    h2d = h_q.numel() * 4 + h_quat.numel() * 4
    d2h = o_q.numel() * 4 + o_counts.numel() * 8 + o_hist.numel() * 8
    return {"value": round(N * args.mcs / per, 1), "unit": "site-updates/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": round(per * 1e3, 3)}


def run_secondary(torch, hm):
    """The 3D 512^3 26-neighbour 8-colour sweep with a per-material-point field
    (two fused launches per MCS), for the HBM roofline of the 3D path."""
    try:
        L = (512, 512, 512)
        N = 512 ** 3
        lat = hm.Lattice(3, L, 26, 256, 1002, 200_000, hm.FIELD_POINT)
        q = torch.empty(N, dtype=torch.int32, device="cuda")
        mp = torch.empty(N, dtype=torch.int32, device="cuda")
        lat.hp_bind(q, mp)
        lat.hp_init_voronoi(hm.ORIENT_SO3, None)
        bmp = torch.randint(0, 30, (N,), dtype=torch.int32, device="cuda")
        lat.hp_set_field(bmp)
        thr, D = hm.hp_build_threshold_table(0.7)
        lat.hp_set_threshold_table(thr, D)
        chosen, ms = lat.hp_sweep_autotune(4)
        lat.hp_sweep(4)
        torch.cuda.synchronize()
        n = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        lat.hp_sweep(n)
        e1.record()
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) / 1e3
        rate = N * n / s
        bytes_per = BYTES_3D_POINT
        peak, _ = peaks()
        lat.close()
        del q, mp, bmp
        torch.cuda.empty_cache()
        return {"workload": "3d-512-moore26-point-field", "site_updates_per_s": round(rate, 1),
                "bytes_per_site_update": bytes_per, "achieved_gbs": round(rate * bytes_per / 1e9, 1),
                "frac_of_measured_hbm": round(rate * bytes_per / 1e9 / peak, 4), "mcs_timed": n,
                "tile": {"variant": int(chosen), "ms_per_4_mcs": [round(float(x), 3) for x in ms]}}
    except Exception as e:  # secondary numbers must not break the main line
        return {"error": str(e)[:200]}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_job(L, G, mcs, seed):
    """The oracle running the same job on a smaller lattice of the same grain
    density: Voronoi, closed-form field, mcs Monte Carlo steps, counts."""
    import oracle
    t0 = time.perf_counter()
    q, _ = oracle.voronoi(2, L, G, seed)
    quat = oracle.orientations(G, seed, 1)
    Cc = np.array([synth.NI_BJ[k] for k in ("C11", "C12", "C44")])
    _, _, _, b = oracle.grain_field(quat, Cc, W.sigma, W.k_disl, W.energy_scale)
    thr, D = oracle.threshold_table(W.kT)
    q2, _, _, _ = oracle.sweep(2, L, W.nbr, int(256 * W.J), seed, 0, mcs, thr, D, q, b[q], None)
    counts, alive = oracle.grain_counts(q2, G)
    bins, _ = oracle.grain_bins(quat, 1)
    oracle.histogram(counts, bins, 1)
    dt = time.perf_counter() - t0
    return int(np.prod(L)) * mcs, dt


SAMPLE_L = (1024, 1024)
SAMPLE_G = 625  # same sites per grain as 4096^2 / 10^4


def cpu_baseline_sample(target_s=12.0):
    mcs = 60
    n, dt = oracle_job(SAMPLE_L, SAMPLE_G, mcs, W.seed)
    return {"value": round(n / dt, 1), "unit": "site-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{SAMPLE_L[0]}x{SAMPLE_L[1]} lattice, {SAMPLE_G} grains (same density), {mcs} MCS, "
                      f"whole job (voronoi, field, sweep, counts/texture), single thread", "seconds": round(dt, 2)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    mcs = 40
    for _ in range(args.warmup):
        oracle_job((256, 256), 39, 4, W.seed)
    tot_n, tot_s = 0, 0.0
    for _ in range(args.steps):
        n, dt = oracle_job(SAMPLE_L, SAMPLE_G, mcs, W.seed)
        tot_n += n
        tot_s += dt
    v = tot_n / tot_s
    line = {
        "metric": "Potts site-updates/s", "value": round(v, 1), "unit": "site-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot_s / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": W.name, "lattice": list(W.L), "nbr": W.nbr, "grains": W.G, "kT": W.kT,
                   "mcs_per_step": W.n_mcs, "parallelism": "cpu oracle"},
        "cpu_baseline": {"value": round(v, 1), "unit": "site-updates/s", "kind": "oracle", "cores": 1,
                         "sample": f"each step: {SAMPLE_L[0]}x{SAMPLE_L[1]}, {SAMPLE_G} grains, {mcs} MCS whole job"},
        "e2e": {"value": round(v, 1), "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# other workloads (one JSON line each; not part of the default run)
# ---------------------------------------------------------------------------
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


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
    """The 3D 512^3 26-neighbour sweep alone (per-point field, material-point index carried)."""
    import torch
    from paper_1007_3509_gb300 import build, hmcpotts as hm
    build.build()
    torch.cuda.set_device(0)
    L, N = (512, 512, 512), 512 ** 3
    lat = hm.Lattice(3, L, 26, 256, 1002, 200_000, hm.FIELD_POINT)
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
                      "config": {"workload": "3d-512-moore26-point-field", "variant": int(chosen), "mcs": args.mcs},
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


def main():
    args = parse()
    if args.workload in ("texture2d", "texture3d") and args.impl == "ours":
        run_texture(args)
        return
    if args.workload != "2d" and args.impl == "ours":
        {"3d-cp": run_3d_cp, "ensemble": run_ensemble, "surrogate": run_surrogate,
         "sweep3d": run_sweep3d}[args.workload](args)
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
