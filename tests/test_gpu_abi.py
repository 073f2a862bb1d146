"""GPU checks of the boundary calls that move state in and out and measure it:
hp_set_spins / hp_get_spins with host and device buffers, the synchronous
hp_measure (counts, alive, texture, family fractions, volume-weighted field)
against the oracle, and the library's training loop hp_sur_train against the
same Adam steps issued one by one."""
import math

import numpy as np
import pytest

from paper_1007_3509_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_host_buffers_in_sweep_out_bit_exact(oracle):
    """Host arrays in (hp_set_spins), 3 MCS, host arrays out (hp_get_spins): the
    oracle's lattice and carried material points, for host and device sources."""
    torch, hm = need_gpu()
    L, Q, seed, kT = (70, 40, 12), 9, 0xABC, 0.7
    N = int(np.prod(L))
    q0 = synth.blocky_lattice(L, Q, 5, block=3)
    rng = np.random.default_rng(6)
    mp0 = rng.permutation(N).astype(np.int32)
    bmp = rng.integers(-40, 40, size=N).astype(np.int32)
    thr, D = oracle.threshold_table(kT)
    ref_q, _, ref_mp, _ = oracle.sweep(3, L, 26, 256, seed, 0, 3, thr, D, q0, bmp[mp0], mp0)
    for source in ("host", "device"):
        lat = hm.Lattice(3, L, 26, 256, seed, Q, hm.FIELD_POINT)
        q = torch.empty(N, dtype=torch.int32, device="cuda")
        mp = torch.empty(N, dtype=torch.int32, device="cuda")
        lat.hp_bind(q, mp)
        table = torch.from_numpy(bmp).cuda()
        lat.hp_set_field(table)
        t, d = hm.hp_build_threshold_table(kT)
        lat.hp_set_threshold_table(t, d)
        if source == "host":
            lat.hp_set_spins(q0.copy(), mp0.copy())
        else:
            lat.hp_set_spins(torch.from_numpy(q0).cuda(), torch.from_numpy(mp0).cuda())
        lat.hp_sweep(3)
        oq = np.full(N, -1, dtype=np.int32)
        om = torch.full((N,), -1, dtype=torch.int32).pin_memory()
        lat.hp_get_spins(oq, om)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(oq, ref_q)
        np.testing.assert_array_equal(om.numpy(), ref_mp)
        lat.close()


def test_measure_matches_oracle(oracle):
    torch, hm = need_gpu()
    L, G = (600, 500), 1500
    N = L[0] * L[1]
    q0 = synth.blocky_lattice(L, G, 8, block=6)
    rng = np.random.default_rng(3)
    bg = rng.integers(-30, 200, size=G).astype(np.int32)
    ref_c, ref_alive = oracle.grain_counts(q0, G)
    for kind in (0, 1, 2):
        orient = oracle.orientations(G, 77, kind)
        lat = hm.Lattice(2, L, 8, 256, 1, G, hm.FIELD_GRAIN)
        q = torch.from_numpy(q0).cuda()
        lat.hp_bind(q)
        table = torch.from_numpy(bg).cuda()
        lat.hp_set_field(table)
        to = torch.from_numpy(np.ascontiguousarray(orient)).cuda()
        st, hist = lat.hp_measure(kind, to)
        rb, near = oracle.grain_bins(orient, kind)
        assert np.all(near > 1e-9)  # no orientation on a bin edge in this draw
        ref_h = oracle.histogram(ref_c, rb, kind)
        np.testing.assert_array_equal(hist[:ref_h.size], ref_h)
        assert st.sites == N and st.alive == ref_alive
        assert st.mean_area == N / ref_alive
        assert st.field_sum == int(np.sum(bg[q0].astype(np.int64)))
        assert abs(st.mean_field - st.field_sum / 256.0 / N) < 1e-15
        if kind == 1:
            tot = ref_h[:20].sum()
            assert st.hist_total == tot == N
            np.testing.assert_allclose(list(st.families), ref_h[20:] / tot, rtol=0, atol=1e-15)
            ref_m = float(ref_h[:20] @ ((np.arange(20) + 0.5) / 40)) / tot
            assert abs(st.mean_mmax - ref_m) < 1e-12
        # a second lattice accumulated into the same stats doubles every sum
        f1 = st.field_sum
        st2, hist2 = lat.hp_measure(kind, to, acc=(st, hist.copy()))
        assert st2.sites == 2 * N and st2.alive == 2 * ref_alive and st2.field_sum == 2 * f1
        np.testing.assert_array_equal(hist2[:ref_h.size], 2 * ref_h)
        lat.close()


def test_measure_point_field_and_bad_ids(oracle):
    torch, hm = need_gpu()
    L = (40, 36, 20)
    N = int(np.prod(L))
    G = 50
    q0 = synth.blocky_lattice(L, G, 9, block=4)
    rng = np.random.default_rng(12)
    mp0 = rng.integers(0, N, size=N).astype(np.int32)
    bmp = rng.integers(-1000, 1000, size=N).astype(np.int32)
    lat = hm.Lattice(3, L, 26, 256, 1, G, hm.FIELD_POINT)
    q = torch.from_numpy(q0).cuda()
    mp = torch.from_numpy(mp0).cuda()
    lat.hp_bind(q, mp)
    table = torch.from_numpy(bmp).cuda()
    lat.hp_set_field(table)
    st, _ = lat.hp_measure()
    assert st.field_sum == int(np.sum(bmp[mp0].astype(np.int64)))
    assert st.alive == oracle.grain_counts(q0, G)[1]
    q.fill_(G + 3)
    with pytest.raises(hm.HPError) as e:
        lat.hp_measure()
    assert e.value.code == hm.HP_ERR_STATE
    lat.close()


def test_sur_train_equals_stepwise_adam(oracle):
    """The library's loop against the same minibatches, learning rates and Adam
    steps issued one call at a time (gradients are summed with atomics, so the
    two runs agree to rounding, not bit for bit)."""
    torch, hm = need_gpu()
    from paper_1007_3509_gb300 import hybrid
    prm = hybrid.cp_params_table1(1e-4, 7.0)
    n_orient, K, n_incr = 512, 8, 4
    quat = torch.empty(n_orient, 4, device="cuda")
    hm.hp_orientations(n_orient, 31, hm.ORIENT_SO3, quat)
    M = n_orient * n_incr
    X = torch.empty(M, 11, device="cuda")
    Y = torch.empty(M, 2, device="cuda")
    hm.hp_sur_generate(prm, 31, quat, n_orient, K, n_incr, X, Y)
    init = np.concatenate([p.ravel() for p in synth.mlp_init(32)]).astype(np.float32)
    steps, batch, lr, floor = 240, 1000, 2e-3, 0.02
    B = batch // n_incr * n_incr
    nb = M // B
    runs = []
    for mode in ("library", "stepwise"):
        params = torch.from_numpy(init).cuda()
        m = torch.zeros_like(params)
        v = torch.zeros_like(params)
        loss = torch.zeros(1, device="cuda")
        if mode == "library":
            log = hm.hp_sur_train(params, m, v, X, Y, steps, batch=batch, group=n_incr, lr=lr, lr_floor=floor,
                                  loss=loss, log_every=40)
            assert log.size == steps // 40 and log[-1] < log[0]
        else:
            grads = torch.empty_like(params)
            lr32 = float(np.float32(lr))
            fl32 = float(np.float32(floor))
            for step in range(1, steps + 1):
                c = 0.5 * (1.0 + math.cos(math.pi * step / steps))
                r0 = ((step - 1) % nb) * B
                hm.hp_mlp_gradients(params, X[r0:r0 + B], Y[r0:r0 + B], grads, loss)
                hm.hp_mlp_adam(params, grads, m, v, step, lr32 * (fl32 + (1.0 - fl32) * c))
        torch.cuda.synchronize()
        runs.append((params.cpu().numpy(), float(loss.item())))
    (pa, la), (pb, lb) = runs
    assert np.linalg.norm(pa - pb) <= 1e-3 * np.linalg.norm(pb)
    assert abs(la - lb) <= 1e-2 * abs(lb)
