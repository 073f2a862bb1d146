"""CPU check of the warp-strip kernel's skewed row schedule against the oracle.

The strip kernel (csrc/strip.cu) walks one strip of a plane two rows per step
with the colour phases skewed across rows (Sec. 4 colourings), streaming rows
through a small ring in shared memory that is refilled two row pairs ahead.
This test restates that schedule in Python -- strip geometry, ring slots
holding random stale values until written, the issue order, the per-row
phase order, the narrowing column ranges and the masked core store -- and
checks the lattice against the oracle bit for bit.  It shares nothing with the
CUDA path; the GPU parity tests check the kernel itself.
"""
import numpy as np
import pytest

from paper_1007_3509_gb300 import synth


def _offset(nbr, k):
    if nbr == 4:
        return [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)][k]
    if nbr == 8:
        kk = k + (k >= 4)
        return kk % 3 - 1, kk // 3 - 1, 0
    kk = k + (k >= 13)
    return kk % 3 - 1, (kk // 3) % 3 - 1, kk // 9 - 1


def _geometry(Lx, Ly, cpl, ty_max):
    maxcore = 32 * cpl - 8
    nsx = -(-Lx // maxcore)
    core = (-(-Lx // nsx) + 3) & ~3
    nsx = -(-Lx // core)
    nsy = -(-Ly // ty_max)
    ty = (-(-Ly // nsy) + 1) & ~1
    return core, nsx, ty, -(-Ly // ty)


def _strip_launch(oracle, L3, nbr, J, seed, sweep, thr, D, src, nb, out, table, field, zpar, cpl, ty_max, rng,
                  order="paper"):
    (q_in, mp_in), (q_nb, mp_nb), (q_out, mp_out) = src, nb, out
    Lx, Ly, Lz = L3
    Z = nbr == 26
    hasmp = mp_in is not None
    arrays = ["q"] + (["mp"] if hasmp else []) + (["lo", "hi"] if Z else [])
    RING = 8 if nbr == 4 else 6
    RS = 32 * cpl + 8                      # row stride: four padding values on each side
    core, nsx, ty, nsy = _geometry(Lx, Ly, cpl, ty_max)
    W = core + 8
    n_tab = table.size

    def tab(i):
        u = int(i) & 0xFFFFFFFF
        return int(table[u if u < n_tab else n_tab - 1])

    for zi in range(Lz // 2 if Z else 1):
        z = 2 * zi + zpar if Z else 0
        zlo, zhi = (z - 1) % Lz, (z + 1) % Lz
        for sy in range(nsy):
            for sx in range(nsx):
                x0, y0 = sx * core, sy * ty
                ring = {a: rng.integers(-9, 9, size=(RING, RS)).astype(np.int64) for a in arrays}

                def R(r, a):
                    return ring[a][(r + 2 * RING) % RING]

                def source(a):
                    return {"q": q_in[z], "mp": mp_in[z] if hasmp else None, "lo": q_nb[zlo] if Z else None,
                            "hi": q_nb[zhi] if Z else None}[a]

                def issue(r0):  # rows r0, r0 + 1 of every array, W columns each
                    for h in (0, 1):
                        gy = (y0 + r0 + h) % Ly
                        for a in arrays:
                            row = source(a)[gy]
                            R(r0 + h, a)[4:4 + W] = row[(x0 - 4 + np.arange(W)) % Lx]

                def update(r, col, colour):
                    gx, gy = (x0 - 4 + col) % Lx, (y0 + r) % Ly
                    ctr = np.array([[(gx + Lx * gy + Lx * Ly * z) & 0xFFFFFFFF, 0, sweep, colour]], dtype=np.uint32)
                    u = oracle.philox(seed, ctr)[0]
                    dx, dy, dz = _offset(nbr, (int(u[0]) * nbr) >> 32)
                    own = R(r, "q")
                    qi = own[4 + col]
                    qj = R(r + dy, "q" if dz == 0 else ("lo" if dz < 0 else "hi"))[4 + col + dx]
                    if qj == qi:
                        return
                    mpj = 0
                    if hasmp:
                        mpj = (R(r + dy, "mp")[4 + col + dx] if dz == 0 else
                               (mp_nb[zlo] if dz < 0 else mp_nb[zhi])[(gy + dy) % Ly][(gx + dx) % Lx])
                    if field == "grain":
                        bi, bj = tab(qi), tab(qj)
                    else:
                        bi, bj = tab(R(r, "mp")[4 + col]), tab(mpj)
                    if nbr == 4:
                        nbrs = [own[3 + col], own[5 + col], R(r - 1, "q")[4 + col], R(r + 1, "q")[4 + col]]
                    else:
                        nbrs = []
                        for ddy in (-1, 0, 1):
                            for ddx in (-1, 0, 1):
                                if ddx or ddy:
                                    nbrs.append(R(r + ddy, "q")[4 + col + ddx])
                                if Z:
                                    nbrs += [R(r + ddy, "lo")[4 + col + ddx], R(r + ddy, "hi")[4 + col + ddx]]
                    d = J * (sum(v == qi for v in nbrs) - sum(v == qj for v in nbrs)) + (bj - bi)
                    if d < 0 or (d <= D and (thr[d] == 0xFFFFFFFF or int(u[1]) < int(thr[d]))):
                        own[4 + col] = qj
                        if hasmp:
                            R(r, "mp")[4 + col] = mpj

                def phase_row(px, r, p, colour):
                    # sites of column parity px in [p + 1, W - p - 1); interior ones are no-ops
                    for col in range(p + 1 + ((p + 1 + px) & 1), W - p - 1, 2):
                        update(r, col, colour)

                def store(r):
                    if y0 + r >= Ly:
                        return
                    for c in range(4, W - 4):
                        if x0 - 4 + c >= Lx:
                            break
                        q_out[z][y0 + r][x0 - 4 + c] = R(r, "q")[4 + c]
                        if hasmp:
                            mp_out[z][y0 + r][x0 - 4 + c] = R(r, "mp")[4 + c]

                OFF, K = -2, ty // 2
                issue(OFF)
                issue(2 + OFF)
                cz = 4 * zpar if Z else 0
                for k in range(K + 1):
                    if k + 2 <= K + 1:
                        issue(2 * (k + 2) + OFF)
                    if nbr == 4:
                        phase_row(1, 2 * k - 1, 0, 0)
                        phase_row(0, 2 * k, 0, 0)
                        if k > 0:
                            phase_row(1, 2 * k - 2, 1, 1)
                            phase_row(0, 2 * k - 1, 1, 1)
                    elif order == "paper":
                        phase_row(0, 2 * k, 0, cz + 0)
                        phase_row(1, 2 * k, 1, cz + 1)
                        if k > 0:
                            phase_row(0, 2 * k - 1, 2, cz + 2)
                            phase_row(1, 2 * k - 1, 3, cz + 3)
                    else:  # a wrong skew: the odd row's phases before the even row's
                        if k > 0:
                            phase_row(0, 2 * k - 1, 2, cz + 2)
                            phase_row(1, 2 * k - 1, 3, cz + 3)
                        phase_row(0, 2 * k, 0, cz + 0)
                        phase_row(1, 2 * k, 1, cz + 1)
                    if k > 0:
                        store(2 * k - 2)
                        store(2 * k - 1)


def _schedule_sweep(oracle, L, nbr, seed, n, thr, D, q0, mp0, table, field, cpl, ty_max, order="paper"):
    L3 = tuple(L) + (1,) * (3 - len(L))
    Lx, Ly, Lz = L3
    q = q0.reshape(Lz, Ly, Lx).astype(np.int64)
    mp = None if mp0 is None else mp0.reshape(Lz, Ly, Lx).astype(np.int64)
    rng = np.random.default_rng(0)
    for t in range(n):
        qa = np.full_like(q, -999)
        ma = None if mp is None else np.full_like(mp, -999)
        args = (oracle, L3, nbr, 256, seed, 5 + t, thr, D)
        if nbr == 26:
            _strip_launch(*args, (q, mp), (q, mp), (qa, ma), table, field, 0, cpl, ty_max, rng, order)
            _strip_launch(*args, (q, mp), (qa, ma), (qa, ma), table, field, 1, cpl, ty_max, rng, order)
        else:
            _strip_launch(*args, (q, mp), (None, None), (qa, ma), table, field, 0, cpl, ty_max, rng, order)
        q, mp = qa, ma
    return q.reshape(-1), (None if mp is None else mp.reshape(-1))


def _case(oracle, L, nbr, field):
    q0 = synth.blocky_lattice(L, 7, 100 + nbr, block=3)
    rng = np.random.default_rng(101 + nbr)
    bgrain = rng.integers(-60, 60, size=7).astype(np.int32)
    bmp = rng.integers(-60, 60, size=q0.size).astype(np.int32)
    mp0 = rng.integers(0, q0.size, size=q0.size).astype(np.int32)
    thr, D = oracle.threshold_table(0.7)
    seed = 0xC0FFEE + nbr
    if field == "grain":
        ref_q, _, ref_mp, _ = oracle.sweep(len(L), L, nbr, 256, seed, 5, 2, thr, D, q0, bgrain[q0], None)
        return (q0, None, bgrain, thr, D, seed), (ref_q, ref_mp)
    ref_q, _, ref_mp, _ = oracle.sweep(len(L), L, nbr, 256, seed, 5, 2, thr, D, q0, bmp[mp0], mp0)
    return (q0, mp0, bmp, thr, D, seed), (ref_q, ref_mp)


# (lattice, neighbours, field, columns per lane, most core rows per strip): the
# shapes of the strip variants (2D: 8 or 4 columns per lane, 16 or 32 rows; 3D:
# 2 or 4 columns, 32 or 64 rows) on lattices with several strips, ragged
# strips, and a lattice narrower than any window
CASES = [
    ((136, 72), 4, "grain", 8, 16), ((136, 72), 4, "point", 4, 32),
    ((200, 130), 8, "point", 8, 32), ((200, 130), 8, "grain", 4, 16),
    ((4, 4), 8, "point", 8, 16), ((66, 2), 8, "grain", 4, 32),
    ((70, 20, 4), 26, "point", 2, 64), ((136, 20, 4), 26, "grain", 4, 64), ((70, 20, 4), 26, "grain", 2, 32),
]


@pytest.mark.parametrize("L,nbr,field,cpl,ty_max", CASES)
def test_strip_schedule_matches_oracle(oracle, L, nbr, field, cpl, ty_max):
    (q0, mp0, table, thr, D, seed), (ref_q, ref_mp) = _case(oracle, L, nbr, field)
    q, mp = _schedule_sweep(oracle, L, nbr, seed, 2, thr, D, q0, mp0, table, field, cpl, ty_max)
    np.testing.assert_array_equal(q, ref_q)
    if mp0 is not None:
        np.testing.assert_array_equal(mp, ref_mp)


def test_strip_schedule_detects_a_wrong_skew(oracle):
    """The check has teeth: running the odd row's phases before the even row's differs."""
    L, nbr = (200, 130), 8
    (q0, mp0, table, thr, D, seed), (ref_q, _) = _case(oracle, L, nbr, "grain")
    q, _ = _schedule_sweep(oracle, L, nbr, seed, 2, thr, D, q0, mp0, table, "grain", 4, 16, order="wrong")
    assert np.count_nonzero(q != ref_q) > 0
