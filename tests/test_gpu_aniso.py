"""GPU parity of the misorientation-dependent sweep (pair energy J_{q_i,q_n} of
Eq. (7) and boundary mobility) against the oracle: integer arithmetic, so the
lattices and carried material points must be bit-identical."""
import numpy as np
import pytest

from paper_1007_3509_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

PERIOD = 90000


@pytest.mark.parametrize("dim,L,nbr", [(2, (96, 70), 4), (2, (130, 66), 8), (3, (20, 18, 14), 6), (3, (34, 22, 12), 26)])
@pytest.mark.parametrize("mode", ["none", "grain", "point"])
def test_aniso_sweep_bit_exact(oracle, dim, L, nbr, mode):
    torch, hm = need_gpu()
    Q = 9
    q0 = synth.blocky_lattice(L, Q, 31, block=3)
    N = q0.size
    rng = np.random.default_rng(32)
    ang = rng.integers(0, PERIOD, size=Q).astype(np.int32)
    Jtab, mtab = hm.hp_build_read_shockley(1.0, 15.0, 500, 91, 1000, mobility=True)
    bgrain = rng.integers(-40, 40, size=Q).astype(np.int32)
    bmp = rng.integers(-40, 40, size=N).astype(np.int32)
    mp0 = rng.integers(0, N, size=N).astype(np.int32)
    thr, D = oracle.threshold_table(0.9)
    seed, n = 0xA11, 3
    b = {"none": None, "grain": bgrain[q0], "point": bmp[mp0]}[mode]
    ref_q, _, ref_mp, _ = oracle.sweep_aniso(dim, L, nbr, seed, 4, n, thr, D, q0, ang, PERIOD, 500, Jtab, mtab, b, mp0)
    fm = {"none": hm.FIELD_NONE, "grain": hm.FIELD_GRAIN, "point": hm.FIELD_POINT}[mode]
    lat = hm.Lattice(dim, L, nbr, 256, seed, Q, fm)
    q = torch.from_numpy(q0.copy()).cuda()
    mp = torch.from_numpy(mp0.copy()).cuda()
    lat.hp_bind(q, mp)
    table = {"grain": bgrain, "point": bmp}.get(mode)
    if table is not None:
        tt = torch.from_numpy(table).cuda()
        lat.hp_set_field(tt)
    lat.hp_set_threshold_table(*hm.hp_build_threshold_table(0.9))
    ta = torch.from_numpy(ang).cuda()
    lat.hp_set_anisotropy(ta, PERIOD, 500, Jtab, mtab)
    lat.hp_set_sweep_counter(4)
    lat.hp_sweep(n)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(q.cpu().numpy(), ref_q)
    np.testing.assert_array_equal(mp.cpu().numpy(), ref_mp)
    # clearing the tables returns to the constant-J sweep
    lat.hp_set_anisotropy(None, 0, 0, None)
    q.copy_(torch.from_numpy(q0))
    mp.copy_(torch.from_numpy(mp0))
    lat.hp_set_sweep_counter(4)
    lat.hp_sweep(n)
    torch.cuda.synchronize()
    iso_q, _, _, _ = oracle.sweep(dim, L, nbr, 256, seed, 4, n, thr, D, q0, b, mp0)
    np.testing.assert_array_equal(q.cpu().numpy(), iso_q)
    lat.close()


def test_aniso_angles_from_orientations_and_frozen_boundary(oracle):
    """Angles converted by the library from HP_ORIENT_ANGLE orientations; a
    zero-mobility bin freezes exactly the boundaries whose misorientation falls
    in it, as in the oracle."""
    torch, hm = need_gpu()
    L, G = (256, 200), 60
    lat = hm.Lattice(2, L, 8, 256, 7, G, hm.FIELD_NONE)
    q = torch.empty(L[0] * L[1], dtype=torch.int32, device="cuda")
    lat.hp_bind(q)
    ang_f = torch.empty(G, device="cuda")
    lat.hp_init_voronoi(hm.ORIENT_ANGLE, ang_f)
    units = torch.empty(G, dtype=torch.int32, device="cuda")
    hm.hp_angle_units(G, hm.ORIENT_ANGLE, ang_f, 1000, PERIOD, units)
    torch.cuda.synchronize()
    a = units.cpu().numpy()
    af = ang_f.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(a - np.floor(af * 180 / np.pi * 1000)) <= 1)   # float rounding of the degree product
    Jtab, mtab = hm.hp_build_read_shockley(1.0, 15.0, 1000, 46, 1000, mobility=True)
    mtab[10:20] = 0
    q0 = q.cpu().numpy()
    thr, D = oracle.threshold_table(0.8)
    ref_q, _, _, _ = oracle.sweep_aniso(2, L, 8, 7, 0, 10, thr, D, q0, a, PERIOD, 1000, Jtab, mtab)
    lat.hp_set_threshold_table(*hm.hp_build_threshold_table(0.8))
    lat.hp_set_anisotropy(units, PERIOD, 1000, Jtab, mtab)
    lat.hp_sweep(10)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(q.cpu().numpy(), ref_q)
    lat.close()


def test_aniso_at_the_bench_size_bit_exact(oracle):
    """The anisotropic workload's lattice (1024^2 Moore, 625 grains rotated about
    z, Read-Shockley energy and mobility, kT 0.6) for 6 MCS against the oracle,
    site for site."""
    torch, hm = need_gpu()
    L, G, N = (1024, 1024), 625, 1024 * 1024
    lat = hm.Lattice(2, L, 8, 256, 1001, G, hm.FIELD_NONE)
    q = torch.empty(N, dtype=torch.int32, device="cuda")
    lat.hp_bind(q)
    ang = torch.empty(G, device="cuda")
    lat.hp_init_voronoi(hm.ORIENT_ANGLE, ang)
    units = torch.empty(G, dtype=torch.int32, device="cuda")
    hm.hp_angle_units(G, hm.ORIENT_ANGLE, ang, 1000, PERIOD, units)
    J, m = hm.hp_build_read_shockley(1.0, 15.0, 250, 181, 1000, mobility=True)
    torch.cuda.synchronize()
    q0 = q.cpu().numpy()
    a = units.cpu().numpy()
    thr, D = oracle.threshold_table(0.6)
    lat.hp_set_threshold_table(*hm.hp_build_threshold_table(0.6))
    lat.hp_set_anisotropy(units, PERIOD, 250, J, m)
    lat.hp_sweep(6)
    torch.cuda.synchronize()
    ref_q, _, _, _ = oracle.sweep_aniso(2, L, 8, 1001, 0, 6, thr, D, q0, a, PERIOD, 250, J, m)
    np.testing.assert_array_equal(q.cpu().numpy(), ref_q)
    assert np.count_nonzero(ref_q != q0) > 1000
    lat.close()
