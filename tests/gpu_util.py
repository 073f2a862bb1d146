"""Helpers for the GPU tests: drive the C ABI through the binding on torch
CUDA tensors and hand the same seeded inputs to the oracle."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_3509_gb300 import build, hmcpotts
    build.build()
    return torch, hmcpotts


def run_gpu_sweep(torch, hm, dim, L, nbr, J_fix, seed, n_mcs, kT, q0, field_mode, table=None, mp0=None,
                  kernel=0, zero_rule=0, sweep0=0, chunks=None, variant=None):
    """Sweep n_mcs on the GPU; returns (q, mp) as numpy arrays."""
    G = int(max(q0.max() + 1, (table.size if (table is not None and field_mode == hm.FIELD_GRAIN) else 1)))
    lat = hm.Lattice(dim, L, nbr, J_fix, seed, G, field_mode)
    q = torch.from_numpy(np.ascontiguousarray(q0, dtype=np.int32)).cuda()
    mp = None if mp0 is None else torch.from_numpy(np.ascontiguousarray(mp0, dtype=np.int32)).cuda()
    lat.hp_bind(q, mp)
    if field_mode != hm.FIELD_NONE:
        t = torch.from_numpy(np.ascontiguousarray(table, dtype=np.int32)).cuda()
        lat.hp_set_field(t)
    thr, D = hm.hp_build_threshold_table(kT, zero_rule)
    lat.hp_set_threshold_table(thr, D)
    lat.hp_set_sweep_kernel(kernel)
    if variant is not None:
        lat.hp_set_sweep_variant(variant)
    lat.hp_set_sweep_counter(sweep0)
    for n in (chunks or [n_mcs]):
        lat.hp_sweep(n)
    torch.cuda.synchronize()
    assert lat.hp_get_sweep_counter() == sweep0 + n_mcs
    out_q = q.cpu().numpy()
    out_mp = None if mp is None else mp.cpu().numpy()
    lat.close()
    return out_q, out_mp
