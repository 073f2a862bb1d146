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
