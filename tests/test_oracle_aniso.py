"""Pins of the misorientation-dependent sweep of the oracle (pair energy
J_{q_i,q_n} of Eq. (7), boundary mobility), CPU only.

* A constant table J = J_fix without mobility is the isotropic sweep, whose own
  pins (exact transition probabilities, voter model, invariants) stand.
* One MCS is re-run here through the global Hamiltonian: the energy of the
  whole lattice summed bond by bond (each unordered pair once) before and after
  each trial flip, the draws taken from the oracle's Philox, and the mobility
  applied to the threshold: the same lattice must come out.
* Only misorientations matter: a common rotation or a reflection of every
  grain's angle leaves the trajectory unchanged.
* A boundary of zero mobility never moves.
* The Read-Shockley table takes its closed-form values.
"""
import math

import numpy as np
import pytest

from paper_1007_3509_gb300 import synth

PERIOD = 90000  # millidegrees: a cubic crystal rotated about z


def _angles(G, seed):
    return np.random.default_rng(seed).integers(0, PERIOD, size=G).astype(np.int32)


def _table(nb, seed, lo=30, hi=400):
    return np.random.default_rng(seed).integers(lo, hi, size=nb).astype(np.int32)


@pytest.mark.parametrize("dim,L,nbr", [(2, (12, 10), 4), (2, (14, 8), 8), (3, (6, 6, 4), 6), (3, (6, 4, 4), 26)])
def test_constant_table_is_the_isotropic_sweep(oracle, dim, L, nbr):
    Q = 5
    q0 = synth.random_lattice(L, Q, 3)
    N = q0.size
    b0 = np.random.default_rng(4).integers(-40, 40, size=N).astype(np.int32)
    mp0 = np.arange(N, dtype=np.int32)
    thr, D = oracle.threshold_table(0.8)
    ref = oracle.sweep(dim, L, nbr, 256, 77, 3, 4, thr, D, q0, b0, mp0)
    got = oracle.sweep_aniso(dim, L, nbr, 77, 3, 4, thr, D, q0, _angles(Q, 5), PERIOD, 500,
                             np.full(91, 256, np.int32), None, b0, mp0)
    for a, b in zip(ref[:3], got[:3]):
        np.testing.assert_array_equal(a, b)
    assert ref[3] == got[3]


def _global_energy(q, nbr_index, J):
    e = 0
    for i in range(q.size):
        for n in nbr_index[i]:
            if n > i and q[n] != q[i]:
                e += J(q[i], q[n])
    return e


def _neighbours(L, nbr):
    Lx, Ly = L
    offs = {4: [(1, 0), (-1, 0), (0, 1), (0, -1)],
            8: [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if dx or dy]}[nbr]
    # row-major (dy, dx) order for 8 neighbours, (+x, -x, +y, -y) for 4
    if nbr == 8:
        offs = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if dx or dy]
    idx = []
    for y in range(Ly):
        for x in range(Lx):
            idx.append([(x + dx) % Lx + Lx * ((y + dy) % Ly) for dx, dy in offs])
    return idx


@pytest.mark.parametrize("nbr,mobility", [(8, False), (8, True), (4, True)])
def test_one_mcs_through_the_global_hamiltonian(oracle, nbr, mobility):
    L = (8, 6)
    Lx, Ly = L
    N = Lx * Ly
    Q = 6
    q0 = synth.random_lattice(L, Q, 11)
    b0 = np.random.default_rng(12).integers(-300, 300, size=N).astype(np.int32)
    ang = _angles(Q, 13)
    bin_w, nbins = 1500, 31
    Jtab = _table(nbins, 14)
    mtab = np.random.default_rng(15).integers(0, 2**32, size=nbins, dtype=np.uint64).astype(np.uint32) if mobility else None
    thr, D = oracle.threshold_table(1.3)
    seed, sweep = 99, 7

    def mis(a, b):
        d = abs(int(ang[a]) - int(ang[b])) % PERIOD
        return min(min(d, PERIOD - d) // bin_w, nbins - 1)

    def J(a, b):
        return int(Jtab[mis(a, b)])

    nb = _neighbours(L, nbr)
    q = q0.copy()
    bfield = b0.copy()
    C = 2 if nbr == 4 else 4
    for c in range(C):
        for y in range(Ly):
            for x in range(Lx):
                colour = (x + y) & 1 if nbr == 4 else (x & 1) + 2 * (y & 1)
                if colour != c:
                    continue
                i = x + Lx * y
                u = oracle.philox(seed, oracle.counters([i], sweep, 0, c))[0]
                j = nb[i][(int(u[0]) * nbr) >> 32]
                if q[j] == q[i]:
                    continue
                e0 = _global_energy(q, nb, J) + int(bfield.sum())
                trial, tb = q.copy(), bfield.copy()
                trial[i], tb[i] = q[j], bfield[j]
                d = _global_energy(trial, nb, J) + int(tb.sum()) - e0
                if d > D:
                    continue
                t = 0xFFFFFFFF if d < 0 else int(thr[d])
                m = 0xFFFFFFFF if mtab is None else int(mtab[mis(q[i], q[j])])
                eff = t if m == 0xFFFFFFFF else (m if t == 0xFFFFFFFF else (t * m) >> 32)
                if eff == 0xFFFFFFFF or int(u[1]) < eff:
                    q, bfield = trial, tb
    got_q, got_b, _, _ = oracle.sweep_aniso(2, L, nbr, seed, sweep, 1, thr, D, q0, ang, PERIOD, bin_w, Jtab, mtab, b0)
    np.testing.assert_array_equal(got_q, q)
    np.testing.assert_array_equal(got_b, bfield)
    assert np.count_nonzero(q != q0) > 0


def test_only_misorientations_matter(oracle):
    L, Q = (16, 12), 7
    q0 = synth.random_lattice(L, Q, 21)
    thr, D = oracle.threshold_table(0.9)
    ang = _angles(Q, 22)
    Jtab = _table(91, 23)
    mtab = np.random.default_rng(24).integers(2**31, 2**32, size=91, dtype=np.uint64).astype(np.uint32)
    ref = oracle.sweep_aniso(2, L, 8, 5, 0, 6, thr, D, q0, ang, PERIOD, 500, Jtab, mtab)[0]
    rotated = ((ang.astype(np.int64) + 31337) % PERIOD).astype(np.int32)
    reflected = ((PERIOD - ang.astype(np.int64)) % PERIOD).astype(np.int32)
    for a in (rotated, reflected):
        np.testing.assert_array_equal(oracle.sweep_aniso(2, L, 8, 5, 0, 6, thr, D, q0, a, PERIOD, 500, Jtab, mtab)[0], ref)
    # a different set of misorientations does change the trajectory
    other = _angles(Q, 25)
    assert np.count_nonzero(oracle.sweep_aniso(2, L, 8, 5, 0, 6, thr, D, q0, other, PERIOD, 500, Jtab, mtab)[0]
                            != ref) > 0


def test_zero_mobility_boundary_is_frozen(oracle):
    """Two grains 5 degrees apart share a boundary of zero mobility: at any
    temperature and with a bulk driving force towards either, it never moves."""
    L = (24, 16)
    q0 = synth.half_plane_lattice(L)
    ang = np.array([0, 5000], dtype=np.int32)
    Jtab = np.full(46, 256, np.int32)
    mtab = np.full(46, 0xFFFFFFFF, np.uint32)
    mtab[5] = 0                                    # 5-6 degrees
    thr, D = oracle.threshold_table(2.0)
    b = np.where(q0 == 0, 200, -200).astype(np.int32)
    got = oracle.sweep_aniso(2, L, 8, 3, 0, 20, thr, D, q0, ang, PERIOD, 1000, Jtab, mtab, b)[0]
    np.testing.assert_array_equal(got, q0)
    mtab[5] = 0xFFFFFFFF
    moved = oracle.sweep_aniso(2, L, 8, 3, 0, 20, thr, D, q0, ang, PERIOD, 1000, Jtab, mtab, b)[0]
    assert np.count_nonzero(moved != q0) > 0


def test_read_shockley_closed_form(oracle):
    """Bin centres (k + 1/2) * 0.25 degrees, theta_m = 15 degrees: J = J_max x (1 - ln x)
    for x = theta/theta_m < 1, J_max beyond; mobility 1 - exp(-5 x^4)."""
    J, m = oracle.read_shockley(2.0, 15.0, 250, 181, 1000, mobility=True)
    for k in (0, 7, 20, 59, 60, 100, 180):
        th = (k + 0.5) * 0.25
        x = th / 15.0
        e = 2.0 * x * (1 - math.log(x)) if x < 1 else 2.0
        assert J[k] == round(256 * e), (k, J[k], 256 * e)
        mm = 1 - math.exp(-5 * x ** 4)
        assert abs(int(m[k]) / 2**32 - mm) < 2**-31
    # maximum of x (1 - ln x) at x = 1: the energy rises monotonically to J_max
    assert np.all(np.diff(J[:60]) >= 0) and J[60] == 512
