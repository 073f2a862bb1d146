"""Hybrid Monte Carlo drivers: sequences of C-ABI calls, no arithmetic here.

The paper's loop (Sec. 5): apply a load increment, let the Monte Carlo crystal
plasticity split it into elastic and plastic parts at every material point
(Sec. 2), convert the resulting energies into the bulk energy of the Potts
model (Sec. 3), and evolve the microstructure by Monte Carlo steps (Sec. 4).
Here the load is the Taylor increment of Eq. (3) and the field is refreshed
every `refresh_every` MCS by `incr_per_refresh` increments.

* plain:     per-material-point MCP (``hp_cp_step``) -> per-point field
             (``HP_FIELD_POINT``, material-point index carried by the sweep)
* surrogate: the trained network evaluated once per grain (``hp_sur_field``)
             -> per-grain field (``HP_FIELD_GRAIN``)
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import hmcpotts as hm
from . import synth


@dataclass
class HybridConfig:
    L: tuple = (64, 64, 64)
    G: int = 300
    seed: int = 1002
    kT: float = 0.7
    n_mcs: int = 500
    refresh_every: int = 50
    incr_per_refresh: int = 2
    e_incr: float = 1e-4
    energy_scale: float = 7.0  # J per MJ/m^3: population maximum of b near 0.1 J


def cp_params_table1(e_incr, energy_scale, w_weight=1.0):
    c = synth.TABLE1
    return hm.cp_params(c["C11"], c["C12"], c["C44"], c["tau0"], c["taus"], c["h0"], c["beta"], e_incr,
                        energy_scale=energy_scale, w_weight=w_weight)


def _texture(lat, quat):
    """hp_measure of the final lattice: SO(3) texture families, mean max Schmid
    factor, the 24-bin histogram (counts) and grains alive."""
    st, hist = lat.hp_measure(hm.ORIENT_SO3, quat)
    return {"families": list(st.families), "mean_mmax": st.mean_mmax, "hist": hist, "alive": int(st.alive)}


def run_plain(torch, cfg: HybridConfig, time_it=True, coupling="taylor", el_tol=1e-5):
    """Plain hybrid: MCP at every material point at each refresh.  coupling
    "taylor": every point takes the prescribed strain of Eq. (3); "equilibrium":
    each increment first solves periodic elastic equilibrium with the current
    plastic strain (hp_elastic_solve) and every point takes its own strain
    (hp_cp_step_strain)."""
    N = int(np.prod(cfg.L))
    lat = hm.Lattice(3, cfg.L, 26, 256, cfg.seed, cfg.G, hm.FIELD_POINT)
    q = torch.empty(N, dtype=torch.int32, device="cuda")
    mp = torch.empty(N, dtype=torch.int32, device="cuda")
    lat.hp_bind(q, mp)
    quat = torch.empty(cfg.G, 4, dtype=torch.float32, device="cuda")
    lat.hp_init_voronoi(hm.ORIENT_SO3, quat)
    grain = q.clone()  # material point p belongs to the grain of site p at the start
    prm = cp_params_table1(cfg.e_incr, cfg.energy_scale)
    eps = torch.empty(6 * N, dtype=torch.float32, device="cuda")
    gam = torch.empty(N, dtype=torch.float32, device="cuda")
    g = torch.empty(N, dtype=torch.float32, device="cuda")
    b = torch.empty(N, dtype=torch.int32, device="cuda")
    hm.hp_cp_reset(prm, N, eps, gam, g)
    thr, D = hm.hp_build_threshold_table(cfg.kT)
    lat.hp_set_threshold_table(thr, D)
    lat.hp_set_field(b)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t_field = 0.0
    incr = 0
    eq = coupling == "equilibrium"
    eps_tot = torch.empty(6 * N, dtype=torch.float32, device="cuda") if eq else None
    el_iters = []
    for k in range(cfg.n_mcs // cfg.refresh_every):
        if time_it:
            torch.cuda.synchronize()
        f0 = time.perf_counter()
        if eq:
            for j in range(cfg.incr_per_refresh):
                t = incr + j + 1
                E = (t * cfg.e_incr, -0.5 * t * cfg.e_incr, -0.5 * t * cfg.e_incr, 0.0, 0.0, 0.0)
                it, _ = hm.hp_elastic_solve(prm, cfg.L, grain, quat, E, eps_tot, eps_p=eps, tol=el_tol,
                                            start_from_mean=(t == 1))
                el_iters.append(it)
                hm.hp_cp_step_strain(prm, cfg.seed, grain, quat, t, eps_tot, eps, gam, g, b=b)
        else:
            hm.hp_cp_step(prm, cfg.seed, grain, quat, incr, cfg.incr_per_refresh, eps, gam, g, b=b)
        if time_it:
            torch.cuda.synchronize()
        t_field += time.perf_counter() - f0
        incr += cfg.incr_per_refresh
        lat.hp_sweep(cfg.refresh_every)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    tex = _texture(lat, quat)
    lat.close()
    out = {"wall_s": wall, "field_s": t_field, **tex}
    if eq:
        out["elastic_iterations"] = el_iters
    return out


def train_surrogate(torch, prm, n_orient=65536, K=128, n_incr=20, steps=60000, lr=3e-3, seed=3000, log_every=0,
                    batch=19440):
    """Generate samples with the MCP kernel and fit the network with the library's training
    loop (hp_sur_train: Adam on contiguous minibatches of `batch` rows taken in turn, cosine
    learning-rate decay to 2 % of lr; rows are orientation-major, so each minibatch holds whole
    orientations at every increment; batch=None uses all rows).
    Returns (params tensor, load table [n_incr, 7] (numpy), final minibatch loss, history)."""
    quat = torch.empty(n_orient, 4, dtype=torch.float32, device="cuda")
    hm.hp_orientations(n_orient, seed, hm.ORIENT_SO3, quat)
    M = n_orient * n_incr
    X = torch.empty(M, 11, dtype=torch.float32, device="cuda")
    Y = torch.empty(M, 2, dtype=torch.float32, device="cuda")
    load = torch.empty(n_incr, 7, dtype=torch.float32, device="cuda")
    hm.hp_sur_generate(prm, seed, quat, n_orient, K, n_incr, X, Y, load)
    init = np.concatenate([p.ravel() for p in synth.mlp_init(seed + 1)]).astype(np.float32)
    params = torch.from_numpy(init).cuda()
    n = params.numel()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    loss = torch.zeros(1, device="cuda")
    log = hm.hp_sur_train(params, m, v, X, Y, steps, batch=batch or 0, group=n_incr, lr=lr, lr_floor=0.02,
                          loss=loss, log_every=log_every)
    torch.cuda.synchronize()
    hist = [((i + 1) * log_every, float(x)) for i, x in enumerate(log)]
    return params, load.cpu().numpy(), float(loss.item()), hist


def run_surrogate(torch, cfg: HybridConfig, params, load_table, time_it=True):
    """Surrogate hybrid: the trained network evaluated once per grain at each refresh."""
    N = int(np.prod(cfg.L))
    lat = hm.Lattice(3, cfg.L, 26, 256, cfg.seed, cfg.G, hm.FIELD_GRAIN)
    q = torch.empty(N, dtype=torch.int32, device="cuda")
    lat.hp_bind(q)
    quat = torch.empty(cfg.G, 4, dtype=torch.float32, device="cuda")
    lat.hp_init_voronoi(hm.ORIENT_SO3, quat)
    b = torch.empty(cfg.G, dtype=torch.int32, device="cuda")
    thr, D = hm.hp_build_threshold_table(cfg.kT)
    lat.hp_set_threshold_table(thr, D)
    lat.hp_set_field(b)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t_field = 0.0
    incr = 0
    for k in range(cfg.n_mcs // cfg.refresh_every):
        incr += cfg.incr_per_refresh
        if time_it:
            torch.cuda.synchronize()
        f0 = time.perf_counter()
        hm.hp_sur_field(params, quat, cfg.G, load_table[min(incr, len(load_table)) - 1], cfg.energy_scale, b)
        if time_it:
            torch.cuda.synchronize()
        t_field += time.perf_counter() - f0
        lat.hp_sweep(cfg.refresh_every)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    tex = _texture(lat, quat)
    lat.close()
    return {"wall_s": wall, "field_s": t_field, **tex}
