"""CPU check of the fused tile kernel's window schedule against the oracle.

The tile kernel (csrc/tile.cu) runs all colour phases of a plane inside a
shared-memory window and writes back only the window's core.  Its halo (four
columns, two rows) rests on which earlier colour phases each phase reads
(Sec. 4 colourings: red/black, and the four colours (x&1) + 2(y&1) of a Moore
plane).  This test restates that schedule in numpy -- window gather with
periodic wrap, phase p updating columns [p+1, WX-p-1) and rows
[y_p, WY-y_p), y_p = p+1 (red/black) or 1 + p/2 (four colours), then the
core store with ragged-edge skip -- and checks the result against the oracle
bit for bit.  Sites a phase leaves outside its range are poisoned afterwards,
so any later read of one would show.  It shares nothing with the CUDA path;
the GPU parity tests check the kernel itself.
"""
import numpy as np
import pytest

from paper_1007_3509_gb300 import synth

HX, HY = 4, 2


def _offsets(nbr):
    if nbr == 4:
        return [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)]
    if nbr == 8:
        return [(k % 3 - 1, k // 3 - 1, 0) for k in range(9) if k != 4]
    return [(k % 3 - 1, (k // 3) % 3 - 1, k // 9 - 1) for k in range(27) if k != 13]


def _ylo(nbr, p):
    return p + 1 if nbr == 4 else 1 + (p >> 1)


def _colour_mask(nbr, p, r, c):
    if nbr == 4:
        return ((r + c) & 1) == p
    return ((c & 1) == (p & 1)) & ((r & 1) == (p >> 1))


def _launch(oracle, L3, nbr, J, seed, sweep, thr, D, src, nb, out, table, field, zpar, WX, TY, poison, ylo=_ylo):
    (q_in, mp_in), (q_nb, mp_nb), (q_out, mp_out) = src, nb, out
    Lx, Ly, Lz = L3
    Z = nbr == 26
    hasmp = mp_in is not None
    WY, TX = TY + 2 * HY, WX - 2 * HX
    O = _offsets(nbr)
    ox = np.array([o[0] for o in O]); oy = np.array([o[1] for o in O]); oz = np.array([o[2] for o in O])
    n_tab = table.size

    def tab(i):
        u = i & 0xFFFFFFFF
        return table[np.where(u < n_tab, u, n_tab - 1)].astype(np.int64)

    for zi in range(Lz // 2 if Z else 1):
        z = 2 * zi + zpar if Z else 0
        zlo, zhi = (z - 1) % Lz, (z + 1) % Lz
        for y0 in range(0, Ly, TY):
            for x0 in range(0, Lx, TX):
                gys = (y0 - HY + np.arange(WY)) % Ly
                gxs = (x0 - HX + np.arange(WX)) % Lx
                win = np.ix_(gys, gxs)
                S = q_in[z][win].astype(np.int64)
                SMP = mp_in[z][win].astype(np.int64) if hasmp else None
                planes = {0: S}
                if Z:
                    planes[-1] = q_nb[zlo][win].astype(np.int64)
                    planes[1] = q_nb[zhi][win].astype(np.int64)
                for p in range(2 if nbr == 4 else 4):
                    lo, hi = p + 1, WX - p - 1
                    yl = ylo(nbr, p)
                    r, c = np.meshgrid(np.arange(yl, WY - yl), np.arange(lo, hi), indexing="ij")
                    sel = _colour_mask(nbr, p, r, c)
                    r, c = r[sel], c[sel]
                    colour = p if nbr == 4 else 4 * zpar * Z + p
                    u = oracle.philox(seed, oracle.counters(gxs[c] + Lx * gys[r] + Lx * Ly * z, sweep, 0, colour))
                    k = ((u[:, 0].astype(np.uint64) * np.uint64(len(O))) >> np.uint64(32)).astype(np.int64)
                    dx, dy, dz = ox[k], oy[k], oz[k]
                    qi = S[r, c]
                    qj = np.select([dz < 0, dz > 0], [planes[-1][r + dy, c + dx] if Z else qi,
                                                      planes[1][r + dy, c + dx] if Z else qi], S[r + dy, c + dx])
                    mpj = np.zeros_like(qi)
                    if hasmp:
                        mpj = SMP[r + dy, c + dx]
                        if Z:
                            gxn, gyn = (gxs[c] + dx) % Lx, (gys[r] + dy) % Ly
                            mpj = np.select([dz < 0, dz > 0], [mp_nb[zlo][gyn, gxn], mp_nb[zhi][gyn, gxn]], mpj)
                    bi, bj = (tab(qi), tab(qj)) if field == "grain" else (tab(SMP[r, c]), tab(mpj))
                    so = np.zeros_like(qi); sn = np.zeros_like(qi)
                    for a, b, e in O:
                        v = planes[e][r + b, c + a]
                        so += v == qi
                        sn += v == qj
                    d = J * (so - sn) + (bj - bi)
                    t = thr[np.clip(d, 0, D)].astype(np.int64)
                    acc = (qj != qi) & ((d < 0) | ((d <= D) & ((t == 0xFFFFFFFF) | (u[:, 1].astype(np.int64) < t))))
                    S[r[acc], c[acc]] = qj[acc]
                    if hasmp:
                        SMP[r[acc], c[acc]] = mpj[acc]
                    if poison:
                        ar, ac = np.meshgrid(np.arange(WY), np.arange(WX), indexing="ij")
                        inside = (ar >= yl) & (ar < WY - yl) & (ac >= lo) & (ac < hi)
                        bad = _colour_mask(nbr, p, ar, ac) & ~inside
                        S[bad] = -7 - p
                        if hasmp:
                            SMP[bad] = -7 - p
                ny, nx = min(TY, Ly - y0), min(TX, Lx - x0)
                q_out[z][y0:y0 + ny, x0:x0 + nx] = S[HY:HY + ny, HX:HX + nx]
                if hasmp:
                    mp_out[z][y0:y0 + ny, x0:x0 + nx] = SMP[HY:HY + ny, HX:HX + nx]


def _schedule_sweep(oracle, L, nbr, J, seed, sweep0, n, thr, D, q0, mp0, table, field, WX, TY, **kw):
    L3 = tuple(L) + (1,) * (3 - len(L))
    Lx, Ly, Lz = L3
    q = q0.reshape(Lz, Ly, Lx).astype(np.int64)
    mp = None if mp0 is None else mp0.reshape(Lz, Ly, Lx).astype(np.int64)
    # poisoning is exact only when the window holds no second copy of a site
    poison = Lx >= WX and Ly >= TY + 2 * HY
    for t in range(n):
        qa = np.full_like(q, -999)
        ma = None if mp is None else np.full_like(mp, -999)
        args = (oracle, L3, nbr, J, seed, sweep0 + t, thr, D)
        if nbr == 26:  # even planes against the old odd ones, then odd planes against the new even ones
            _launch(*args, (q, mp), (q, mp), (qa, ma), table, field, 0, WX, TY, poison, **kw)
            _launch(*args, (q, mp), (qa, ma), (qa, ma), table, field, 1, WX, TY, poison, **kw)
        else:
            _launch(*args, (q, mp), (None, None), (qa, ma), table, field, 0, WX, TY, poison, **kw)
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


# (lattice, neighbours, tile shape (WX, core rows TY)) -- the shapes of the tile
# variants, on lattices with several tiles, ragged tails, and wrapped windows
CASES = [
    ((136, 72), 4, (128, 60)), ((132, 130), 4, (64, 60)), ((4, 4), 4, (128, 28)),
    ((200, 130), 8, (128, 60)), ((250, 62), 8, (128, 28)), ((128, 128), 8, (64, 60)), ((66, 2), 8, (128, 60)),
    ((70, 40, 4), 26, (64, 36)), ((136, 40, 4), 26, (128, 28)), ((64, 74, 4), 26, (64, 28)), ((12, 10, 4), 26, (64, 60)),
    # the lean 3D kernel's windows (64 x 44, core 56 x 40; 64 x 40, core 56 x 36) follow the same schedule
    ((120, 86, 4), 26, (64, 40)), ((64, 44, 4), 26, (64, 40)), ((118, 74, 4), 26, (64, 36)),
]


@pytest.mark.parametrize("L,nbr,shape", CASES)
@pytest.mark.parametrize("field", ["grain", "point"])
def test_tile_schedule_matches_oracle(oracle, L, nbr, shape, field):
    (q0, mp0, table, thr, D, seed), (ref_q, ref_mp) = _case(oracle, L, nbr, field)
    q, mp = _schedule_sweep(oracle, L, nbr, 256, seed, 5, 2, thr, D, q0, mp0, table, field, *shape)
    np.testing.assert_array_equal(q, ref_q)
    if mp0 is not None:
        np.testing.assert_array_equal(mp, ref_mp)


def test_tile_schedule_detects_a_short_phase_range(oracle):
    """The check has teeth: phase 3 of a Moore plane one row short differs from the oracle."""
    L, nbr = (200, 130), 8
    (q0, mp0, table, thr, D, seed), (ref_q, _) = _case(oracle, L, nbr, "grain")
    short = lambda nb, p: 1 + (p >> 1) + (p == 3)  # noqa: E731
    q, _ = _schedule_sweep(oracle, L, nbr, 256, seed, 5, 2, thr, D, q0, mp0, table, "grain", 128, 60, ylo=short)
    assert np.count_nonzero(q != ref_q) > 0
