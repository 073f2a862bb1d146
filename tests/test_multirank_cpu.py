"""Multi-rank paths on CPU ranks (gloo, world size 2).

* The paper's parallelisation (Sec. 4): the lattice is divided among
  processors that exchange boundary layers at every half step.  Two ranks each
  own a slab of the slowest axis, exchange one ghost layer with their periodic
  neighbours before every colour phase, and update their own sites with the
  oracle's per-phase slab update.  Because the draws are keyed by the global
  site index, the gathered lattice must equal the undecomposed oracle run.
* A rank that dies between steps is noticed by its peer through a short
  process-group timeout, not by hanging.
* bench.py's whole-job aggregation takes the slowest rank's time.
"""
import datetime
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port, timeout_s=60):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=timeout_s))
    return dist


def _slab_worker(rank, world, port, case, out_dir):
    sys.path.insert(0, ROOT)
    import torch
    import oracle
    dist = _init(rank, world, port)
    dim, L, nbr, n_mcs = case
    q0 = np.load(os.path.join(out_dir, "q0.npy"))
    b0 = np.load(os.path.join(out_dir, "b0.npy"))
    Ls = L[-1]
    layer = int(np.prod(L[:-1]))
    ns = Ls // world
    s0 = rank * ns
    # slab with one ghost layer below and above
    idx = [(s0 - 1 + t) % Ls for t in range(ns + 2)]
    q = np.concatenate([q0[i * layer:(i + 1) * layer] for i in idx]).astype(np.int32)
    b = np.concatenate([b0[i * layer:(i + 1) * layer] for i in idx]).astype(np.int32)
    mp = np.concatenate([np.arange(i * layer, (i + 1) * layer) for i in idx]).astype(np.int32)
    thr, D = oracle.threshold_table(0.8)
    up, down = (rank + 1) % world, (rank - 1) % world
    C = {4: 2, 6: 2, 8: 4, 26: 8}[nbr]

    def exchange():
        for arr in (q, b, mp):
            first = torch.from_numpy(arr[layer:2 * layer].copy())
            last = torch.from_numpy(arr[ns * layer:(ns + 1) * layer].copy())
            g_lo = torch.empty(layer, dtype=torch.int32)
            g_hi = torch.empty(layer, dtype=torch.int32)
            reqs = [dist.isend(last, up), dist.isend(first, down), dist.irecv(g_lo, down), dist.irecv(g_hi, up)]
            for r in reqs:
                r.wait()
            arr[:layer] = g_lo.numpy()
            arr[(ns + 1) * layer:] = g_hi.numpy()

    for t in range(n_mcs):
        for c in range(C):
            exchange()
            oracle.sweep_phase_slab(dim, L, nbr, 256, 99, t, c, thr, D, s0, ns, q, b, mp)
    own = slice(layer, (ns + 1) * layer)
    parts = [torch.from_numpy(a[own].copy()) for a in (q, b, mp)]
    gathered = [[torch.empty_like(p) for _ in range(world)] for p in parts]
    for p, g in zip(parts, gathered):
        dist.all_gather(g, p)
    if rank == 0:
        for name, g in zip(("q", "b", "mp"), gathered):
            np.save(os.path.join(out_dir, f"{name}.npy"), torch.cat(g).numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("case", [(2, (24, 16), 8, 3), (2, (18, 12), 4, 3), (3, (10, 8, 8), 26, 2),
                                  (3, (8, 6, 6), 6, 2)])
def test_slab_decomposition_matches_single_domain(oracle, tmp_path, case):
    from paper_1007_3509_gb300 import synth
    dim, L, nbr, n_mcs = case
    q0 = synth.blocky_lattice(L, 6, 3, block=2)
    b0 = synth.random_field(q0.size, -30, 30, 4)
    np.save(tmp_path / "q0.npy", q0)
    np.save(tmp_path / "b0.npy", b0)
    tmp.spawn(_slab_worker, args=(2, _port(), case, str(tmp_path)), nprocs=2, join=True)
    thr, D = oracle.threshold_table(0.8)
    rq, rb, rmp, _ = oracle.sweep(dim, L, nbr, 256, 99, 0, n_mcs, thr, D, q0, b0, np.arange(q0.size))
    np.testing.assert_array_equal(np.load(tmp_path / "q.npy"), rq)
    np.testing.assert_array_equal(np.load(tmp_path / "b.npy"), rb)
    np.testing.assert_array_equal(np.load(tmp_path / "mp.npy"), rmp)


def _fault_worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch
    dist = _init(rank, world, port, timeout_s=3)
    x = torch.ones(4)
    dist.all_reduce(x)  # one healthy step
    if rank == 1:
        os._exit(0)     # the rank leaves between steps, with nothing in flight
    try:
        dist.all_reduce(x)
        status = "no error"
    except Exception as e:  # noqa: BLE001
        status = "detected: " + type(e).__name__
    with open(os.path.join(out_dir, "status.txt"), "w") as f:
        f.write(status)
    os._exit(0)


def test_dead_rank_detected_by_timeout(tmp_path):
    ctx = tmp.start_processes(_fault_worker, args=(2, _port(), str(tmp_path)), nprocs=2, join=False,
                              start_method="spawn")
    for p in ctx.processes:
        p.join(60)
    status = (tmp_path / "status.txt").read_text()
    assert status.startswith("detected"), status


def _agg_worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    _init(rank, world, port)
    import bench
    ms = 100.0 if rank == 0 else 250.0
    max_ms, value = bench.aggregate(ms, 1000, world, "cpu")
    if rank == 0:
        with open(os.path.join(out_dir, "agg.txt"), "w") as f:
            f.write(f"{max_ms} {value}")
    import torch.distributed as dist
    dist.destroy_process_group()


def test_bench_aggregation_takes_slowest_rank(tmp_path):
    tmp.spawn(_agg_worker, args=(2, _port(), str(tmp_path)), nprocs=2, join=True)
    max_ms, value = map(float, (tmp_path / "agg.txt").read_text().split())
    assert max_ms == 250.0 and abs(value - 2000 / 0.25) < 1e-6
