"""GPU parity of the checkerboard Potts sweep against the oracle: lattices
must be bit-identical (spins and carried material-point indices)."""
import numpy as np
import pytest

from paper_1007_3509_gb300 import synth
from tests.gpu_util import need_gpu, run_gpu_sweep

pytestmark = pytest.mark.gpu

GEOMS = [
    # dim, L, nbr
    (2, (136, 72), 4), (2, (4, 4), 4), (2, (2, 6), 4), (2, (128, 128), 4),
    (2, (200, 130), 8), (2, (4, 4), 8), (2, (66, 2), 8),
    (3, (20, 18, 14), 6), (3, (4, 4, 4), 6), (3, (2, 2, 2), 6),
    (3, (70, 40, 12), 26), (3, (4, 4, 4), 26), (3, (66, 34, 6), 26), (3, (2, 4, 2), 26),
]


def _kernels(nbr):
    return [1] if nbr == 6 else [1, 2]


def _inputs(L, Q, seed):
    q0 = synth.blocky_lattice(L, Q, seed, block=3)
    N = q0.size
    rng = np.random.default_rng(seed + 1)
    bgrain = rng.integers(-60, 60, size=Q).astype(np.int32)
    bmp = rng.integers(-60, 60, size=N).astype(np.int32)
    mp0 = rng.integers(0, N, size=N).astype(np.int32)
    return q0, bgrain, bmp, mp0


@pytest.mark.parametrize("dim,L,nbr", GEOMS)
@pytest.mark.parametrize("mode", ["none", "grain", "point"])
def test_sweep_bit_exact(oracle, dim, L, nbr, mode):
    torch, hm = need_gpu()
    Q = 7
    q0, bgrain, bmp, mp0 = _inputs(L, Q, 100 + nbr)
    seed, kT, J, n = 0xC0FFEE + nbr, 0.7, 256, 3
    thr, D = oracle.threshold_table(kT)
    if mode == "none":
        ref_q, _, ref_mp, _ = oracle.sweep(dim, L, nbr, J, seed, 5, n, thr, D, q0, None, mp0)
    elif mode == "grain":
        ref_q, ref_b, ref_mp, _ = oracle.sweep(dim, L, nbr, J, seed, 5, n, thr, D, q0, bgrain[q0], mp0)
        np.testing.assert_array_equal(ref_b, bgrain[ref_q])
    else:
        ref_q, ref_b, ref_mp, _ = oracle.sweep(dim, L, nbr, J, seed, 5, n, thr, D, q0, bmp[mp0], mp0)
        np.testing.assert_array_equal(ref_b, bmp[ref_mp])
    fm = {"none": hm.FIELD_NONE, "grain": hm.FIELD_GRAIN, "point": hm.FIELD_POINT}[mode]
    table = {"none": None, "grain": bgrain, "point": bmp}[mode]
    for kern in _kernels(nbr):
        q, mp = run_gpu_sweep(torch, hm, dim, L, nbr, J, seed, n, kT, q0, fm, table, mp0, kernel=kern, sweep0=5)
        assert np.array_equal(q, ref_q), f"kernel {kern}: {np.count_nonzero(q != ref_q)} sites differ"
        assert np.array_equal(mp, ref_mp), f"kernel {kern}: mp differs"


@pytest.mark.parametrize("dim,L,nbr", [(2, (96, 64), 8), (3, (34, 66, 8), 26), (2, (64, 70), 4)])
def test_sweep_grain_mode_without_mp_and_chunked(oracle, dim, L, nbr):
    """No material-point buffer; the MCS count split over several calls gives the same lattice."""
    torch, hm = need_gpu()
    q0, bgrain, _, _ = _inputs(L, 12, 7)
    seed, kT, J = 77, 0.6, 256
    thr, D = oracle.threshold_table(kT)
    ref_q, _, _, _ = oracle.sweep(dim, L, nbr, J, seed, 0, 6, thr, D, q0, bgrain[q0], None)
    for kern in _kernels(nbr):
        q, _ = run_gpu_sweep(torch, hm, dim, L, nbr, J, seed, 6, kT, q0, hm.FIELD_GRAIN, bgrain, None,
                             kernel=kern, chunks=[1, 2, 3])
        np.testing.assert_array_equal(q, ref_q)


@pytest.mark.parametrize("kT,zero_rule,J", [(0.0, 1, 256), (0.0, 0, 256), (2.0, 0, 256), (0.7, 1, 0), (0.7, 0, 0)])
def test_sweep_temperatures_and_rules(oracle, kT, zero_rule, J):
    """kT = 0 (frozen table), both dE = 0 rules, and J = 0."""
    torch, hm = need_gpu()
    L = (72, 70)
    q0, bgrain, _, _ = _inputs(L, 5, 3)
    if J == 0:
        bgrain[:] = 0
    thr, D = oracle.threshold_table(kT, zero_rule)
    ref_q, _, _, flips = oracle.sweep(2, L, 8, J, 9, 0, 4, thr, D, q0, bgrain[q0], None)
    for kern in (1, 2):
        q, _ = run_gpu_sweep(torch, hm, 2, L, 8, J, 9, 4, kT, q0, hm.FIELD_GRAIN, bgrain, None, kernel=kern,
                             zero_rule=zero_rule)
        np.testing.assert_array_equal(q, ref_q)
    if J == 0 and zero_rule == 1:
        assert flips == 0 and np.array_equal(ref_q, q0)


def test_sweep_zero_mcs_is_noop():
    torch, hm = need_gpu()
    q0 = synth.random_lattice((16, 16), 4, 1)
    q, _ = run_gpu_sweep(torch, hm, 2, (16, 16), 8, 256, 1, 0, 0.5, q0, hm.FIELD_NONE)
    np.testing.assert_array_equal(q, q0)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
def test_sweep_full_size_2d_moore_two_mcs(oracle, variant):
    """4096^2 Moore lattice, 10^4 grains, grain field: 2 MCS bit-exact (plane and lean tile variants)."""
    torch, hm = need_gpu()
    L, G = (4096, 4096), 10_000
    q0 = synth.blocky_lattice(L, G, 5, block=40)
    bgrain = np.random.default_rng(6).integers(0, 26, size=G).astype(np.int32)
    thr, D = oracle.threshold_table(0.6)
    ref_q, _, _, _ = oracle.sweep(2, L, 8, 256, 1001, 0, 2, thr, D, q0, bgrain[q0], None)
    q, _ = run_gpu_sweep(torch, hm, 2, L, 8, 256, 1001, 2, 0.6, q0, hm.FIELD_GRAIN, bgrain, None, kernel=0,
                         variant=variant)
    np.testing.assert_array_equal(q, ref_q)
    assert hm.hp_sweep_status() == 0


@pytest.mark.parametrize("variant", [2, 4, 5, 6, 7, 8, 9])
def test_sweep_full_size_3d_point_field_one_mcs(oracle, variant):
    """512^3 26-neighbour lattice with a per-material-point field: one MCS bit-exact."""
    torch, hm = need_gpu()
    L = (512, 512, 512)
    N = 512 ** 3
    q0 = synth.blocky_lattice(L, 200_000, 8, block=9)
    bmp = np.random.default_rng(9).integers(0, 30, size=N).astype(np.int32)
    mp0 = np.arange(N, dtype=np.int32)
    thr, D = oracle.threshold_table(0.7)
    ref_q, _, ref_mp, _ = oracle.sweep(3, L, 26, 256, 1002, 0, 1, thr, D, q0, bmp, mp0)
    q, mp = run_gpu_sweep(torch, hm, 3, L, 26, 256, 1002, 1, 0.7, q0, hm.FIELD_POINT, bmp, mp0, kernel=0,
                          variant=variant)
    np.testing.assert_array_equal(q, ref_q)
    np.testing.assert_array_equal(mp, ref_mp)


@pytest.mark.parametrize("kind", ["monotone", "perturbed"])
@pytest.mark.parametrize("variant", [0, 4])
def test_sweep_arbitrary_threshold_table(oracle, kind, variant):
    """The threshold table is input data: a table that is not of the exp form (any
    monotone table, or an exp table with one entry moved) gives the oracle's
    lattice too, on the plane and the tile kernels."""
    torch, hm = need_gpu()
    L, nbr, Q = (200, 130), 8, 9
    q0, bgrain, _, _ = _inputs(L, Q, 41)
    thr, D = oracle.threshold_table(0.8)
    thr = thr.copy()
    if kind == "monotone":
        rng = np.random.default_rng(5)
        thr[1:] = np.sort(rng.integers(1, 2**32 - 2, size=D, dtype=np.uint64))[::-1].astype(np.uint32)
    else:
        thr[256] = np.uint32(int(thr[256]) // 2)   # d = 256: one unlike bond and no field change
    seed, n = 1234, 3
    ref_q, _, _, _ = oracle.sweep(2, L, nbr, 256, seed, 0, n, thr, D, q0, bgrain[q0], None)
    lat = hm.Lattice(2, L, nbr, 256, seed, Q, hm.FIELD_GRAIN)
    q = torch.from_numpy(q0.copy()).cuda()
    lat.hp_bind(q, None)
    tab = torch.from_numpy(bgrain).cuda()
    lat.hp_set_field(tab)
    lat.hp_set_threshold_table(thr, D)
    lat.hp_set_sweep_kernel(0)
    lat.hp_set_sweep_variant(variant)
    lat.hp_sweep(n)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(q.cpu().numpy(), ref_q)
    lat.close()


@pytest.mark.parametrize("mode", ["none", "grain", "point"])
@pytest.mark.parametrize("variant", [8, 9, 10, 11])
def test_lean_3d_interior_and_edge_windows(oracle, mode, variant):
    """The lean 3D kernel fills windows inside the lattice by tiled TMA boxes and
    windows that cross the periodic edge by 16-byte asynchronous copies; a
    lattice with several of each gives the oracle's lattice and material points."""
    torch, hm = need_gpu()
    L, Q = (176, 124, 10), 11
    q0, bgrain, bmp, mp0 = _inputs(L, Q, 77)
    seed, kT, n = 0x5EED, 0.7, 3
    thr, D = oracle.threshold_table(kT)
    if mode == "none":
        ref_q, _, ref_mp, _ = oracle.sweep(3, L, 26, 256, seed, 2, n, thr, D, q0, None, mp0)
    elif mode == "grain":
        ref_q, _, ref_mp, _ = oracle.sweep(3, L, 26, 256, seed, 2, n, thr, D, q0, bgrain[q0], mp0)
    else:
        ref_q, _, ref_mp, _ = oracle.sweep(3, L, 26, 256, seed, 2, n, thr, D, q0, bmp[mp0], mp0)
    fm = {"none": hm.FIELD_NONE, "grain": hm.FIELD_GRAIN, "point": hm.FIELD_POINT}[mode]
    table = {"none": None, "grain": bgrain, "point": bmp}[mode]
    q, mp = run_gpu_sweep(torch, hm, 3, L, 26, 256, seed, n, kT, q0, fm, table, mp0, kernel=2, sweep0=2,
                          variant=variant)
    np.testing.assert_array_equal(q, ref_q)
    np.testing.assert_array_equal(mp, ref_mp)
    assert hm.hp_sweep_status() == 0
