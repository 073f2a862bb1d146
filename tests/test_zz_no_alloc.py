"""The no-allocation Voronoi entry point against the allocating one.

hp_init_voronoi_static serves callers that cannot allocate device memory while
they run (all device memory pre-reserved by another allocator, or a loop that
must never enter the allocator).  Its scratch is a fixed 16 MiB device array
shared by every call, so this test makes two calls in a row on different
lattices (the second call must not see the first call's leftovers) and checks
both, through the C ABI, against hp_init_voronoi: the tessellation is integer
work, so the tolerance is bit-exactness.  This file is collected last so a
run that stops at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

CASES = [
    # dim, L, nbr, G, seed, orient kind
    (3, (96, 80, 64), 26, 20_000, 2000, 1),
    (2, (1024, 768), 8, 5_000, 2001, 0),
]


def _tessellate(torch, hm, dim, L, nbr, G, seed, kind, static):
    N = int(np.prod(L))
    lat = hm.Lattice(dim, L, nbr, 256, seed, G)
    q = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    mp = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    pos = torch.full((G,), -7, dtype=torch.int64, device="cuda")
    orient = torch.zeros(G * (1 if kind == 0 else 4), dtype=torch.float32, device="cuda")
    lat.hp_bind(q, mp)
    if static:
        lat.hp_init_voronoi_static(kind, orient, pos)
    else:
        lat.hp_init_voronoi(kind, orient, pos)
    torch.cuda.synchronize()
    out = [t.cpu().numpy() for t in (q, mp, pos, orient)]
    lat.close()
    return out


def test_static_voronoi_matches_allocating_twice():
    torch, hm = need_gpu()
    for dim, L, nbr, G, seed, kind in CASES:  # two calls in a row, different sizes
        ref = _tessellate(torch, hm, dim, L, nbr, G, seed, kind, static=False)
        got = _tessellate(torch, hm, dim, L, nbr, G, seed, kind, static=True)
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b)
        assert np.all(ref[0] >= 0) and np.all(ref[0] < G)


def test_static_voronoi_rejects_too_many_grains():
    torch, hm = need_gpu()
    G = 300_000  # above HP_VORONOI_STATIC_MAX_GRAINS
    lat = hm.Lattice(2, (1024, 1024), 8, 256, 1, G)
    q = torch.empty(1024 * 1024, dtype=torch.int32, device="cuda")
    lat.hp_bind(q)
    with pytest.raises(hm.HPError) as e:
        lat.hp_init_voronoi_static(0, None, None)
    assert e.value.code == hm.HP_ERR_ARG


def _bare(torch, hm, dim, L, nbr, G, seed, static):
    """q and mp after a tessellation with neither orientations nor seed sites
    requested, so the static call also carves its seed-site scratch."""
    N = int(np.prod(L))
    lat = hm.Lattice(dim, L, nbr, 256, seed, G)
    q = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    mp = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    lat.hp_bind(q, mp)
    if static:
        lat.hp_init_voronoi_static(0, None, None)
    else:
        lat.hp_init_voronoi(0, None, None)
    torch.cuda.synchronize()
    out = [q.cpu().numpy(), mp.cpu().numpy()]
    lat.close()
    return out


def test_static_voronoi_without_outputs_twice():
    torch, hm = need_gpu()
    for dim, L, nbr, G, seed in [(3, (64, 48, 40), 26, 9_000, 2010), (2, (512, 384), 8, 700, 2011)]:
        ref = _bare(torch, hm, dim, L, nbr, G, seed, static=False)
        got = _bare(torch, hm, dim, L, nbr, G, seed, static=True)
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b)


def _device_memory(cudart, dev):
    free, total = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert cudart.cudaMemGetInfo(ctypes.byref(free), ctypes.byref(total)) == 0
    pool = ctypes.c_void_p(0)
    assert cudart.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), ctypes.c_int(dev)) == 0
    vals = []
    for attr in (5, 7):  # cudaMemPoolAttrReservedMemCurrent, cudaMemPoolAttrUsedMemCurrent
        v = ctypes.c_uint64(0)
        assert cudart.cudaMemPoolGetAttribute(pool, ctypes.c_int(attr), ctypes.byref(v)) == 0
        vals.append(v.value)
    return free.value, vals[0], vals[1]


def test_static_voronoi_leaves_device_memory_unchanged():
    """Neither the device's free memory nor the default stream-ordered pool
    (which torch's allocator statistics do not see) changes across the call."""
    torch, hm = need_gpu()
    hm.lib()
    cudart = ctypes.CDLL("libcudart.so.13")
    dev = torch.cuda.current_device()
    L, G = (96, 64, 48), 12_000
    N = int(np.prod(L))
    lat = hm.Lattice(3, L, 26, 256, 2020, G)
    q = torch.empty(N, dtype=torch.int32, device="cuda")
    lat.hp_bind(q)
    lat.hp_init_voronoi_static(0, None, None)  # loads the kernels' module on first use
    torch.cuda.synchronize()
    before = _device_memory(cudart, dev)
    lat.hp_init_voronoi_static(0, None, None)
    torch.cuda.synchronize()
    after = _device_memory(cudart, dev)
    lat.close()
    assert after == before, (before, after)
