"""Texture experiments of Sec. 5 as sequences of C-ABI calls (no arithmetic here).

* 2D texture under the orientation-dependent Gaussian bulk energy of Eq. (9)
  (Fig. 3): an ensemble of independent replicas swept together; the
  orientation distribution is read at several time slices.
* 3D texture under plastic loading (Figs. 5 and 7): grains distinguished by
  one rotation angle about z (0-90 degrees), the Monte Carlo plasticity of
  Sec. 2 at every material point with the elastic driving force suppressed as
  in Sec. 5, one load increment per refresh, and the Gaussian width g(t) of
  Eq. (10) fitted to the angle histogram.
"""
from __future__ import annotations

import time

import numpy as np

from . import hmcpotts as hm
from .hybrid import cp_params_table1


def run_gaussian_2d(torch, R=100, L=(500, 500), G=5000, kT=1.0, slices=(0, 100, 300, 1000), seed=7000, nbr=8):
    """Returns {"slices": [...], "hist": [R-summed 90-bin angle histograms], "mean_b": [...], "seconds": s}."""
    members, keep = [], []
    for r in range(R):
        lat = hm.Lattice(2, L, nbr, 256, seed + r, G, hm.FIELD_GRAIN)
        q = torch.empty(int(np.prod(L)), dtype=torch.int32, device="cuda")
        lat.hp_bind(q)
        ang = torch.empty(G, dtype=torch.float32, device="cuda")
        lat.hp_init_voronoi(hm.ORIENT_ANGLE, ang)
        b = torch.empty(G, dtype=torch.int32, device="cuda")
        hm.hp_gaussian_field(G, ang, 1.0, b)
        lat.hp_set_field(b)
        thr, D = hm.hp_build_threshold_table(kT)
        lat.hp_set_threshold_table(thr, D)
        members.append(lat)
        keep.append((q, ang, b))
    ens = hm.Ensemble(members)
    out = {"slices": list(slices), "hist": [], "mean_b": []}
    t0 = time.perf_counter()
    done = 0
    for t in slices:
        if t > done:
            ens.hp_ensemble_sweep(t - done)
            done = t
        acc = None
        for lat, (q, ang, b) in zip(members, keep):  # one hp_stats gathers the whole ensemble
            acc = lat.hp_measure(hm.ORIENT_ANGLE, ang, acc=acc)
        out["hist"].append(acc[1].copy())
        out["mean_b"].append(acc[0].mean_field)
    torch.cuda.synchronize()
    out["seconds"] = time.perf_counter() - t0
    ens.close()
    for lat in members:
        lat.close()
    return out


def run_plastic_3d(torch, L=(128, 128, 128), G=4000, seed=11, kT=2.6, n_incr=100, mcs_per_incr=1, e_incr=2e-5,
                   energy_scale=50.0, w_weight=0.0, every=10):
    """Returns {"t": [MCS], "g": [fitted g in degrees], "hist": [...], "seconds": s}."""
    N = int(np.prod(L))
    lat = hm.Lattice(3, L, 26, 256, seed, G, hm.FIELD_POINT)
    q = torch.empty(N, dtype=torch.int32, device="cuda")
    mp = torch.empty(N, dtype=torch.int32, device="cuda")
    lat.hp_bind(q, mp)
    quat = torch.empty(G, 4, dtype=torch.float32, device="cuda")
    lat.hp_init_voronoi(hm.ORIENT_ZROT, quat)
    grain = q.clone()
    prm = cp_params_table1(e_incr, energy_scale, w_weight)
    eps = torch.empty(6 * N, device="cuda")
    gam = torch.empty(N, device="cuda")
    g = torch.empty(N, device="cuda")
    b = torch.empty(N, dtype=torch.int32, device="cuda")
    hm.hp_cp_reset(prm, N, eps, gam, g)
    thr, D = hm.hp_build_threshold_table(kT)
    lat.hp_set_threshold_table(thr, D)
    lat.hp_set_field(b)
    out = {"t": [], "g": [], "hist": []}

    def measure(t):
        _, h = lat.hp_measure(hm.ORIENT_ZROT, quat)
        out["t"].append(t)
        out["g"].append(hm.hp_texture_fit(h)[0])
        out["hist"].append(h)

    t0 = time.perf_counter()
    measure(0)
    for k in range(n_incr):
        hm.hp_cp_step(prm, seed, grain, quat, k, 1, eps, gam, g, b=b)
        lat.hp_sweep(mcs_per_incr)
        if (k + 1) % every == 0:
            measure((k + 1) * mcs_per_incr)
    torch.cuda.synchronize()
    out["seconds"] = time.perf_counter() - t0
    lat.close()
    return out
