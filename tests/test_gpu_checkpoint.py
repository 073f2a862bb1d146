"""Checkpoint / resume: a run split by save and load is bit-identical to the
uninterrupted run and to the oracle; corrupted, truncated, foreign or mismatched
files are refused."""
import numpy as np
import pytest

from paper_1007_3509_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _lattice(torch, hm, L, q0, mp0, table):
    lat = hm.Lattice(3, L, 26, 256, 77, int(q0.max()) + 1, hm.FIELD_POINT)
    q = torch.from_numpy(q0.copy()).cuda()
    mp = torch.from_numpy(mp0.copy()).cuda()
    lat.hp_bind(q, mp)
    t = torch.from_numpy(table).cuda()
    lat.hp_set_field(t)
    thr, D = hm.hp_build_threshold_table(0.8)
    lat.hp_set_threshold_table(thr, D)
    lat._bufs = (q, mp, t)
    return lat


def test_checkpoint_resume_bit_exact(oracle, tmp_path):
    torch, hm = need_gpu()
    L = (136, 40, 10)
    N = int(np.prod(L))
    q0 = synth.blocky_lattice(L, 20, 1, block=3)
    mp0 = np.arange(N, dtype=np.int32)
    table = synth.random_field(N, -30, 30, 2)
    a = _lattice(torch, hm, L, q0, mp0, table)
    a.hp_sweep(5)
    path = tmp_path / "ck.bin"
    a.hp_checkpoint_save(path)
    a.hp_sweep(4)
    torch.cuda.synchronize()
    qa, mpa = (x.cpu().numpy() for x in a._bufs[:2])
    b = _lattice(torch, hm, L, synth.random_lattice(L, 20, 9), mp0, table)
    b.hp_checkpoint_load(path)
    assert b.hp_get_sweep_counter() == 5
    b.hp_sweep(4)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(b._bufs[0].cpu().numpy(), qa)
    np.testing.assert_array_equal(b._bufs[1].cpu().numpy(), mpa)
    thr, D = oracle.threshold_table(0.8)
    rq, _, rmp, _ = oracle.sweep(3, L, 26, 256, 77, 0, 9, thr, D, q0, table, mp0)
    np.testing.assert_array_equal(qa, rq)
    np.testing.assert_array_equal(mpa, rmp)
    # a flipped byte is caught by the checksum
    raw = bytearray(path.read_bytes())
    raw[len(raw) // 2] ^= 0x40
    bad = tmp_path / "bad.bin"
    bad.write_bytes(bytes(raw))
    with pytest.raises(hm.HPError) as e:
        b.hp_checkpoint_load(bad)
    assert e.value.code == hm.HP_ERR_CHECKSUM
    # a truncated file and a file that is not a checkpoint are refused the same
    # way, and a refused load leaves the handle as it was
    for raw2 in (path.read_bytes()[:-7], b"not a checkpoint" * 8):
        bad.write_bytes(raw2)
        with pytest.raises(hm.HPError) as e:
            b.hp_checkpoint_load(bad)
        assert e.value.code == hm.HP_ERR_CHECKSUM
    assert b.hp_get_sweep_counter() == 9
    np.testing.assert_array_equal(b._bufs[0].cpu().numpy(), qa)
    # a checkpoint of another lattice is refused
    c = hm.Lattice(3, (8, 8, 8), 26, 256, 77, 5, hm.FIELD_POINT)
    qc = torch.zeros(512, dtype=torch.int32, device="cuda")
    c.hp_bind(qc, torch.zeros(512, dtype=torch.int32, device="cuda"))
    with pytest.raises(hm.HPError) as e:
        c.hp_checkpoint_load(path)
    assert e.value.code == hm.HP_ERR_ARG
