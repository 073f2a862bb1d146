"""The learned surrogate end to end on the GPU: training samples produced by
the crystal-plasticity kernel (against the oracle), the per-grain field from
the network (against the FP64 network oracle), the trained accuracy, and what
the surrogate gains over the plain hybrid (same texture within ensemble error,
cheaper field refresh)."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from oracle import surrogate as osur
from paper_1007_3509_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu
SC = (100.0, 1e-3, 0.01, 0.002)


def _prm(hm, e=1e-4, scale=7.0):
    c = synth.TABLE1
    return hm.cp_params(c["C11"], c["C12"], c["C44"], c["tau0"], c["taus"], c["h0"], c["beta"], e, energy_scale=scale)


def test_generate_matches_oracle():
    torch, hm = need_gpu()
    n_orient, K, n_incr, seed = 48, 4, 6, 77
    quat = oracle.orientations(n_orient, 5, 1)
    X = torch.empty(n_orient * n_incr, 11, device="cuda")
    Y = torch.empty(n_orient * n_incr, 2, device="cuda")
    load = torch.empty(n_incr, 7, device="cuda")
    hm.hp_sur_generate(_prm(hm), seed, torch.from_numpy(quat).cuda(), n_orient, K, n_incr, X, Y, load)
    torch.cuda.synchronize()
    c = synth.TABLE1
    P = oracle.cp_params(c["C11"], c["C12"], c["C44"], c["tau0"], c["taus"], c["h0"], c["beta"], 1e-4)
    Xr, Yr, Lr, near = osur.samples(P, seed, quat, K, n_incr, SC)
    assert near.mean() < 0.1
    ok = np.repeat(~near, n_incr)
    np.testing.assert_allclose(Y.cpu().numpy()[ok], Yr[ok], rtol=2e-4, atol=1e-6)
    tol = 1e-4 if not near.any() else 5e-3
    np.testing.assert_allclose(load.cpu().numpy(), Lr, rtol=tol, atol=1e-4)
    np.testing.assert_allclose(X.cpu().numpy()[:, :4], Xr[:, :4], atol=2e-6)
    np.testing.assert_allclose(X.cpu().numpy()[:, 4:], Xr[:, 4:], rtol=tol, atol=1e-5)


def test_field_matches_network_oracle():
    torch, hm = need_gpu()
    import torch as T_
    G = 5000
    params = synth.mlp_init(11)
    flat = np.concatenate([p.ravel() for p in params]).astype(np.float32)
    quat = synth.random_quaternions(G, 12)
    load = np.array([60.0, -25.0, -30.0, 3.0, -2.0, 1.0, 2.5e-3], dtype=np.float32)
    b = torch.empty(G, dtype=torch.int32, device="cuda")
    e = torch.empty(G, dtype=torch.float32, device="cuda")
    hm.hp_sur_field(torch.from_numpy(flat).cuda(), torch.from_numpy(quat).cuda(), G, load, 7.0, b, e)
    x = np.concatenate([osur.orientation_features(quat), np.tile(load[:6] / SC[0], (G, 1)),
                        np.full((G, 1), load[6] / SC[1])], axis=1)

    def bf(a):
        return T_.from_numpy(np.asarray(a, dtype=np.float32)).to(T_.bfloat16).to(T_.float64).numpy()

    pb = [bf(p) if i % 2 == 0 else p for i, p in enumerate(params)]
    y, _ = omlp.forward(pb, bf(x))
    e_ref = 7.0 * (y[:, 0] * SC[2] + y[:, 1] * SC[3])
    eg = e.cpu().numpy()
    assert np.linalg.norm(eg - e_ref) <= 2e-2 * np.linalg.norm(e_ref)
    assert np.all(np.abs(b.cpu().numpy() - np.rint(256 * eg)) <= 0)
    assert np.mean(np.abs(b.cpu().numpy() - oracle.quantise(e_ref)) <= 1) > 0.999


@pytest.fixture(scope="module")
def trained():
    torch, hm = need_gpu()
    from paper_1007_3509_gb300 import hybrid
    prm = hybrid.cp_params_table1(1e-4, 7.0)
    params, load, L, hist = hybrid.train_surrogate(torch, prm, log_every=5000)
    return params, load, L, hist, prm


def test_surrogate_accuracy_against_many_histories(trained):
    """Held-out orientations, targets averaged over 4096 histories (their own
    noise is about 0.27 %): the network's driving field w + E_rho is within 1e-2
    relative (L2 over samples) of the plain solver's expectation; about 0.9 % is
    measured."""
    torch, hm = need_gpu()
    params, load, L, hist, prm = trained
    assert hist[-1][1] < hist[0][1]
    n_orient, K, n_incr = 256, 4096, 20
    quat = torch.empty(n_orient, 4, device="cuda")
    hm.hp_orientations(n_orient, 999, hm.ORIENT_SO3, quat)
    X = torch.empty(n_orient * n_incr, 11, device="cuda")
    Y = torch.empty(n_orient * n_incr, 2, device="cuda")
    hm.hp_sur_generate(prm, 4242, quat, n_orient, K, n_incr, X, Y)
    P = torch.empty_like(Y)
    hm.hp_mlp_forward(params, X, P)
    torch.cuda.synchronize()
    y, p = Y.cpu().numpy(), P.cpu().numpy()
    e_ref = y[:, 0] * SC[2] + y[:, 1] * SC[3]
    e_sur = p[:, 0] * SC[2] + p[:, 1] * SC[3]
    err = np.linalg.norm(e_sur - e_ref) / np.linalg.norm(e_ref)
    print(f"surrogate relative field error {err:.4f}; final training loss {L:.3e}")
    assert err <= 1e-2


def test_surrogate_hybrid_matches_plain_texture(trained):
    """8 seeds of each hybrid on a 64^3 lattice: texture fractions agree within two
    standard errors."""
    torch, hm = need_gpu()
    from paper_1007_3509_gb300 import hybrid
    params, load, L, hist, prm = trained
    plain, sur = [], []
    for s in range(8):
        cfg = hybrid.HybridConfig(L=(64, 64, 64), G=300, seed=5000 + s, kT=0.7, n_mcs=500)
        plain.append(hybrid.run_plain(torch, cfg))
        sur.append(hybrid.run_surrogate(torch, cfg, params, load))
    fp = np.array([r["families"] for r in plain])
    fs = np.array([r["families"] for r in sur])
    mp_ = np.array([r["mean_mmax"] for r in plain])
    ms = np.array([r["mean_mmax"] for r in sur])
    # the library's mean max Schmid factor is the volume-weighted bin centre of its histogram
    for r in plain[:2] + sur[:2]:
        h = r["hist"][:20].astype(np.float64)
        assert abs(r["mean_mmax"] - h @ ((np.arange(20) + 0.5) / 40) / h.sum()) < 1e-12
    for a, b in [(fp[:, k], fs[:, k]) for k in range(4)] + [(mp_, ms)]:
        se = np.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
        assert abs(a.mean() - b.mean()) <= 2 * se + 1e-6, (a, b)
    t_plain = np.mean([r["field_s"] for r in plain[1:]])
    t_sur = np.mean([r["field_s"] for r in sur[1:]])
    print(f"field refresh per run: plain {t_plain*1e3:.2f} ms, surrogate {t_sur*1e3:.2f} ms")


def test_surrogate_refresh_cheaper_at_scale(trained):
    """What the network saves: a plasticity refresh costs per material point, the
    surrogate's per grain.  On a 160^3 lattice of 4700 grains one refresh (two
    increments) of each, timed with the GPU work included, best of three."""
    import time
    torch, hm = need_gpu()
    params, load, L, hist, prm = trained
    P, G = 160 ** 3, 4700
    quat = torch.empty(G, 4, device="cuda")
    hm.hp_orientations(G, 77, hm.ORIENT_SO3, quat)
    grain = torch.randint(0, G, (P,), dtype=torch.int32, device="cuda")
    eps = torch.empty(6 * P, device="cuda"); gam = torch.empty(P, device="cuda"); g = torch.empty(P, device="cuda")
    b = torch.empty(P, dtype=torch.int32, device="cuda")
    bg = torch.empty(G, dtype=torch.int32, device="cuda")
    hm.hp_cp_reset(prm, P, eps, gam, g)
    t_plain, t_sur = [], []
    for rep in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hm.hp_cp_step(prm, 5, grain, quat, 2 * rep, 2, eps, gam, g, b=b)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        hm.hp_sur_field(params, quat, G, load[min(2 * rep + 2, len(load)) - 1], 7.0, bg)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if rep:
            t_plain.append(t1 - t0)
            t_sur.append(t2 - t1)
    print(f"one refresh at 160^3: plain {min(t_plain)*1e3:.2f} ms, surrogate {min(t_sur)*1e3:.2f} ms")
    assert min(t_sur) < min(t_plain)
