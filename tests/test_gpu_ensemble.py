"""GPU parity of the fused-kernel tile variants, the autotuner and batched
ensembles of independent replicas against the oracle (bit-exact)."""
import numpy as np
import pytest

from paper_1007_3509_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _member(torch, hm, dim, L, nbr, seed, kT, mode, G=40, rs=0):
    N = int(np.prod(L))
    q0 = synth.blocky_lattice(L, G, rs + 3, block=3)
    rng = np.random.default_rng(rs)
    bgrain = rng.integers(-40, 40, size=G).astype(np.int32)
    bmp = rng.integers(-40, 40, size=N).astype(np.int32)
    mp0 = rng.permutation(N).astype(np.int32)
    fm = hm.FIELD_GRAIN if mode == "grain" else hm.FIELD_POINT
    lat = hm.Lattice(dim, L, nbr, 256, seed, G, fm)
    q = torch.from_numpy(q0.copy()).cuda()
    mp = torch.from_numpy(mp0.copy()).cuda() if mode == "point" else None
    lat.hp_bind(q, mp)
    tab = torch.from_numpy(bgrain if mode == "grain" else bmp).cuda()
    lat.hp_set_field(tab)
    thr, D = hm.hp_build_threshold_table(kT)
    lat.hp_set_threshold_table(thr, D)
    lat._bufs = (q, mp, tab)
    ref = dict(q0=q0, b0=(bgrain[q0] if mode == "grain" else bmp[mp0]), mp0=mp0 if mode == "point" else None,
               seed=seed, kT=kT, L=L, dim=dim, nbr=nbr)
    return lat, ref


def _oracle_run(oracle, ref, n, sweep0=0):
    thr, D = oracle.threshold_table(ref["kT"])
    q, b, mp, _ = oracle.sweep(ref["dim"], ref["L"], ref["nbr"], 256, ref["seed"], sweep0, n, thr, D, ref["q0"],
                               ref["b0"], ref["mp0"])
    return q, mp


# includes shapes whose tiles are all wrapped (manual loads) and shapes with
# interior tiles (TMA copies in the TMA-fed variants)
VARIANT_GEOMS = [(2, (250, 140), 8), (2, (64, 70), 8), (2, (132, 96), 4), (2, (512, 200), 8), (2, (516, 132), 4),
                 (3, (136, 40, 8), 26), (3, (64, 34, 6), 26), (3, (12, 10, 4), 26), (3, (256, 96, 8), 26),
                 (3, (200, 72, 6), 26),
                 # whole numbers of tile cores (120 x 60 and 56 x 36): no ragged tile
                 (2, (240, 120), 8), (3, (112, 72, 4), 26),
                 # lattices smaller than any window: every window row and column wraps
                 (2, (4, 4), 8), (2, (4, 4), 4), (2, (2, 6), 4), (2, (66, 2), 8)]


@pytest.mark.parametrize("dim,L,nbr", VARIANT_GEOMS)
@pytest.mark.parametrize("mode", ["grain", "point"])
def test_every_tile_variant_bit_exact(oracle, dim, L, nbr, mode):
    torch, hm = need_gpu()
    ref_q = ref_mp = None
    for v in range(hm.hp_sweep_variants(nbr)):
        lat, ref = _member(torch, hm, dim, L, nbr, 4321, 0.8, mode, rs=7)
        if ref_q is None:
            ref_q, ref_mp = _oracle_run(oracle, ref, 3)
        lat.hp_set_sweep_variant(v)
        lat.hp_sweep(3)
        torch.cuda.synchronize()
        assert hm.hp_sweep_status() == 0
        q, mp, _ = lat._bufs
        np.testing.assert_array_equal(q.cpu().numpy(), ref_q, err_msg=f"variant {v}")
        if mode == "point":
            np.testing.assert_array_equal(mp.cpu().numpy(), ref_mp, err_msg=f"variant {v}")
        lat.close()


def test_autotune_restores_state(oracle):
    torch, hm = need_gpu()
    lat, ref = _member(torch, hm, 3, (136, 72, 10), 26, 99, 0.7, "point", rs=2)
    chosen, ms = lat.hp_sweep_autotune(2)
    assert 0 <= chosen < len(ms) and ms[chosen] > 0
    assert lat.hp_get_sweep_counter() == 0
    lat.hp_sweep(3)
    torch.cuda.synchronize()
    ref_q, ref_mp = _oracle_run(oracle, ref, 3)
    q, mp, _ = lat._bufs
    np.testing.assert_array_equal(q.cpu().numpy(), ref_q)
    np.testing.assert_array_equal(mp.cpu().numpy(), ref_mp)


ENS = {
    "3d": [((64, 64, 64), 0.5), ((34, 66, 8), 0.9), ((130, 40, 12), 0.7), ((8, 8, 8), 0.6), ((96, 96, 16), 0.8)],
    "2d": [((256, 130), 0.6), ((64, 64), 0.5), ((130, 258), 0.9), ((4, 6), 0.7)],
}


@pytest.mark.parametrize("kind", ["3d", "2d"])
@pytest.mark.parametrize("mode", ["grain", "point"])
def test_ensemble_bit_exact(oracle, kind, mode):
    torch, hm = need_gpu()
    dim, nbr = (3, 26) if kind == "3d" else (2, 8)
    members, refs = [], []
    for r, (L, kT) in enumerate(ENS[kind]):
        lat, ref = _member(torch, hm, dim, L, nbr, 2000 + r, kT, mode, G=30 + 7 * r, rs=r)
        members.append(lat)
        refs.append(ref)
    ens = hm.Ensemble(members)
    chosen, _ = ens.hp_ensemble_autotune(1)
    ens.hp_ensemble_sweep(3)   # odd count: state copied back from the second buffers
    ens.hp_ensemble_sweep(2)
    ens.hp_ensemble_sweep(2)   # replays the captured graph
    torch.cuda.synchronize()
    for lat, ref in zip(members, refs):
        assert lat.hp_get_sweep_counter() == 7
        rq, rmp = _oracle_run(oracle, ref, 7)
        q, mp, _ = lat._bufs
        np.testing.assert_array_equal(q.cpu().numpy(), rq, err_msg=f"{ref['L']} variant {chosen}")
        if mode == "point":
            np.testing.assert_array_equal(mp.cpu().numpy(), rmp)
    ens.close()
    for lat in members:
        lat.close()


def test_ensemble_rejects_mixed_members():
    torch, hm = need_gpu()
    a, _ = _member(torch, hm, 3, (8, 8, 8), 26, 1, 0.7, "grain")
    b, _ = _member(torch, hm, 2, (8, 8), 8, 1, 0.7, "grain")
    with pytest.raises(hm.HPError):
        hm.Ensemble([a, b])


@pytest.mark.parametrize("kind", ["3d", "2d"])
@pytest.mark.parametrize("mode", ["grain", "point"])
def test_ensemble_every_batch_variant_bit_exact(oracle, kind, mode):
    """Every tile variant that ensembles accept (plane and lean tiles), replayed twice."""
    torch, hm = need_gpu()
    dim, nbr = (3, 26) if kind == "3d" else (2, 8)
    geoms = ENS[kind][:3]
    tried = 0
    for v in range(hm.hp_sweep_variants(nbr)):
        members, refs = [], []
        for r, (L, kT) in enumerate(geoms):
            lat, ref = _member(torch, hm, dim, L, nbr, 3000 + r, kT, mode, G=25 + 5 * r, rs=10 + r)
            members.append(lat)
            refs.append(ref)
        ens = hm.Ensemble(members)
        try:
            ens.hp_ensemble_set_variant(v)
        except hm.HPError:
            ens.close()
            for lat in members:
                lat.close()
            continue
        tried += 1
        ens.hp_ensemble_sweep(2)
        ens.hp_ensemble_sweep(2)
        torch.cuda.synchronize()
        for lat, ref in zip(members, refs):
            rq, rmp = _oracle_run(oracle, ref, 4)
            q, mp, _ = lat._bufs
            np.testing.assert_array_equal(q.cpu().numpy(), rq, err_msg=f"{ref['L']} variant {v}")
            if mode == "point":
                np.testing.assert_array_equal(mp.cpu().numpy(), rmp, err_msg=f"{ref['L']} variant {v}")
        ens.close()
        for lat in members:
            lat.close()
    assert tried >= 4
