"""GPU parity of the deterministic multi-slip comparator (FP64) against the
oracle, and the Fig. 1 comparison of Sec. 2 (Monte Carlo plasticity against the
deterministic model under the prescribed strain increment, e = 1e-6) run on the
GPU over a population of orientations."""
import numpy as np
import pytest

from paper_1007_3509_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

T1 = synth.TABLE1


def _prm(hm, e, **kw):
    p = dict(T1)
    p.update(kw)
    return hm.cp_params(p["C11"], p["C12"], p["C44"], p["tau0"], p["taus"], p["h0"], p["beta"], e)


def _quats(n, seed):
    q = np.random.default_rng(seed).normal(size=(n, 4)).astype(np.float32)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _R(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _t(v):
    return np.array([[v[0], v[5], v[4]], [v[5], v[1], v[3]], [v[4], v[3], v[2]]])


def _state(torch, P):
    return (torch.zeros(6 * P, dtype=torch.float64, device="cuda"), torch.zeros(P, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("P,split", [(64 * 3 + 37, False), (200, True)])
def test_det_matches_oracle_along_a_loading_path(P, split):
    """Every point its own orientation, 40 increments of 5e-5 (well into multiple
    slip), in one launch or one launch per increment; stress, plastic strain and
    slip of every 7th point against the oracle to 1e-9 (relative)."""
    torch, hm = need_gpu()
    from oracle import svdcp
    e, n = 5e-5, 40
    quat = _quats(P, P)
    grain = torch.arange(P, dtype=torch.int32, device="cuda")
    tq = torch.from_numpy(quat).cuda()
    ep, gm = _state(torch, P)
    sig = torch.empty(6 * P, dtype=torch.float64, device="cuda")
    na = torch.empty(P, dtype=torch.int32, device="cuda")
    prm = _prm(hm, e)
    p = dict(T1)
    C = svdcp.stiffness(p["C11"], p["C12"], p["C44"])
    sample = list(range(0, P, 7))
    ref = {i: (np.zeros((3, 3)), 0.0) for i in sample}
    t_done = 0
    for t_end in (range(1, n + 1) if split else [n]):
        hm.hp_det_step(prm, grain, tq, t_done, t_end - t_done, ep, gm, sigma=sig, n_active=na)
        torch.cuda.synchronize()
        s = sig.view(6, P).cpu().numpy().T
        g = gm.cpu().numpy()
        act = na.cpu().numpy()
        e_p = ep.view(6, P).cpu().numpy().T
        mism = 0
        for i in sample:
            R = _R(quat[i])
            U = R.T @ np.diag([1.0, -0.5, -0.5]) @ R
            epo, go = ref[i]
            for t in range(t_done + 1, t_end + 1):
                epo, go, so, idx, _ = svdcp.step(p, C, t * e * U, epo, go)
            ref[i] = (epo, go)
            assert np.abs(_t(s[i]) - so).max() <= 1e-9 * np.abs(so).max(), (i, t_end)
            assert np.abs(_t(e_p[i]) - epo).max() <= 1e-9 * max(np.abs(epo).max(), 1e-12)
            assert abs(g[i] - go) <= 1e-9 * max(go, 1e-12)
            mism += int(act[i] != idx.size)
        assert mism <= 1
        t_done = t_end
    assert (act >= 2).mean() > 0.5


def test_det_perfect_plasticity_along_100():
    """No hardening, <100> loading: 8 systems active and the stress held at
    C : U e_y past the yield strain e_y = tau0 / |P : C : U| (closed form)."""
    torch, hm = need_gpu()
    from oracle import svdcp
    p = dict(T1)
    P = 5
    C = svdcp.stiffness(p["C11"], p["C12"], p["C44"])
    Pm = svdcp.schmid()
    U = np.diag([1.0, -0.5, -0.5])
    CU = np.einsum("ijkl,kl->ij", C, U)
    e_y = p["tau0"] / np.abs(np.einsum("aij,ij->a", Pm, CU)).max()
    e = e_y / 4
    prm = _prm(hm, e, taus=p["tau0"])
    quat = torch.tensor([[1.0, 0.0, 0.0, 0.0]] * P, device="cuda")
    grain = torch.arange(P, dtype=torch.int32, device="cuda")
    ep, gm = _state(torch, P)
    sig = torch.empty(6 * P, dtype=torch.float64, device="cuda")
    na = torch.empty(P, dtype=torch.int32, device="cuda")
    hm.hp_det_step(prm, grain, quat, 0, 28, ep, gm, sigma=sig, n_active=na)
    torch.cuda.synchronize()
    s = sig.view(6, P).cpu().numpy().T
    for i in range(P):
        np.testing.assert_allclose(_t(s[i]), CU * e_y, atol=1e-9 * np.abs(CU * e_y).max())
    assert np.all(na.cpu().numpy() == 8)
    np.testing.assert_allclose(gm.cpu().numpy(), 6.0 * e_y * np.sqrt(6.0), rtol=1e-9)


def test_det_strain_driven_matches_oracle():
    """Each point's own sample-frame total strain (one increment from rest and one
    more from the committed state)."""
    torch, hm = need_gpu()
    from oracle import svdcp
    P = 150
    rng = np.random.default_rng(5)
    quat = _quats(P, 6)
    E = rng.normal(size=(P, 6)) * 1.2e-3
    E2 = E * 1.3
    grain = torch.arange(P, dtype=torch.int32, device="cuda")
    tq = torch.from_numpy(quat).cuda()
    ep, gm = _state(torch, P)
    sig = torch.empty(6 * P, dtype=torch.float64, device="cuda")
    prm = _prm(hm, 1e-6)
    p = dict(T1)
    C = svdcp.stiffness(p["C11"], p["C12"], p["C44"])
    for Es in (E, E2):
        et = torch.from_numpy(np.ascontiguousarray(Es.T.astype(np.float32))).cuda()
        hm.hp_det_step_strain(prm, grain, tq, et, ep, gm, sigma=sig)
    torch.cuda.synchronize()
    s = sig.view(6, P).cpu().numpy().T
    for i in range(P):
        R = _R(quat[i])
        epo, go = np.zeros((3, 3)), 0.0
        for Es in (E, E2):
            Ec = R.T @ _t(Es[i].astype(np.float32).astype(np.float64)) @ R
            epo, go, so, _, _ = svdcp.step(p, C, Ec, epo, go)
        assert np.abs(_t(s[i]) - so).max() <= 1e-9 * np.abs(so).max()
    assert (gm.cpu().numpy() > 0).mean() > 0.8


def test_fig1_monte_carlo_follows_the_deterministic_model_over_orientations(oracle):
    """Fig. 1 on the GPU: 2048 orientations, 2000 increments of 1e-6.  The
    deterministic curve of two orientations is checked against the oracle; over
    the population, the MCP (FP32, one slip system per increment) curve sits
    within 2.5 % of the deterministic one on average once several systems are
    active (95 % of orientations within 3 %; 100-increment averages within 3.5 %
    for 95 % of them, 5 % for all), and while a single system is active the two
    agree to FP32 rounding on at least 90 % of the increments."""
    torch, hm = need_gpu()
    from oracle import svdcp
    P, e, n = 2048, 1e-6, 2000
    quat = _quats(P, 41)
    grain = torch.arange(P, dtype=torch.int32, device="cuda")
    tq = torch.from_numpy(quat).cuda()
    prm = _prm(hm, e)
    ep, gm = _state(torch, P)
    sd = torch.empty(6 * P, dtype=torch.float64, device="cuda")
    na = torch.empty(P, dtype=torch.int32, device="cuda")
    mep = torch.empty(6 * P, device="cuda")
    mgm = torch.empty(P, device="cuda")
    mg = torch.empty(P, device="cuda")
    hm.hp_cp_reset(prm, P, mep, mgm, mg)
    sm = torch.empty(6 * P, device="cuda")
    Rs = torch.from_numpy(np.stack([_R(q) for q in quat])).cuda()
    r0 = Rs[:, 0, :]  # first row: sigma_xx = r0 . sigma_c . r0

    def sxx(v):  # v: [6, P] crystal-frame Voigt
        v = v.double()
        return (r0[:, 0] ** 2 * v[0] + r0[:, 1] ** 2 * v[1] + r0[:, 2] ** 2 * v[2] +
                2 * (r0[:, 1] * r0[:, 2] * v[3] + r0[:, 0] * r0[:, 2] * v[4] + r0[:, 0] * r0[:, 1] * v[5]))

    det_c, mcp_c, act = [], [], []
    for t in range(n):
        hm.hp_det_step(prm, grain, tq, t, 1, ep, gm, sigma=sd, n_active=na)
        hm.hp_cp_step(prm, 13, grain, tq, t, 1, mep, mgm, mg, sigma=sm)
        det_c.append(sxx(sd.view(6, P)))
        mcp_c.append(sxx(sm.view(6, P)))
        act.append(na.clone())
    torch.cuda.synchronize()
    D = torch.stack(det_c).cpu().numpy()   # [n, P]
    M = torch.stack(mcp_c).cpu().numpy()
    A = torch.stack(act).cpu().numpy()
    assert A.min() >= 0
    # the deterministic curve of two orientations against the oracle
    p = dict(T1)
    for i in (0, 1):
        ref, nact = svdcp.uniaxial(p, _R(quat[i]), e, n)
        np.testing.assert_allclose(D[:, i], ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
        np.testing.assert_array_equal(A[:, i], nact)
    rel = (M - D) / D
    # single slip before any multiple slip: where the MCP's candidate set is that
    # one system too the two return maps coincide (to the MCP kernel's FP32);
    # near the onset of multiple slip a second candidate can already pass the
    # trial test and be picked, which the deterministic model drops again
    single = (A == 1) & (np.maximum.accumulate(A, axis=0) < 2)
    assert single.sum() > 0
    agree = np.abs(rel[single]) <= 2e-5
    assert agree.mean() >= 0.9, agree.mean()
    multi = A >= 2
    means = np.array([rel[multi[:, i], i].mean() for i in range(P) if multi[:, i].sum() > 200])
    assert means.size > 0.9 * P
    assert 0 <= means.mean() <= 0.025, means.mean()
    assert np.quantile(means, 0.95) <= 0.03
    # 100-increment windows once several systems are active
    worst = []
    for i in range(0, P, 16):
        first = int(np.argmax(multi[:, i]))
        if multi[:, i].sum() < 300:
            continue
        worst.append(np.abs(np.convolve(rel[first:, i], np.ones(100) / 100, mode="valid")).max())
    assert np.quantile(worst, 0.95) <= 0.035 and max(worst) <= 0.05, (np.quantile(worst, 0.95), max(worst))


def test_det_at_the_bench_size_sampled():
    """The speed configuration of the comparison workload: 10^6 points of random
    orientation, 20 increments of 1e-4 in one launch; 48 sampled points against
    the oracle to 1e-9 and every point's active set settled."""
    torch, hm = need_gpu()
    from oracle import svdcp
    P, e, n = 1_000_000, 1e-4, 20
    quat = _quats(P, 2024)
    grain = torch.arange(P, dtype=torch.int32, device="cuda")
    tq = torch.from_numpy(quat).cuda()
    ep, gm = _state(torch, P)
    sig = torch.empty(6 * P, dtype=torch.float64, device="cuda")
    na = torch.empty(P, dtype=torch.int32, device="cuda")
    hm.hp_det_step(_prm(hm, e), grain, tq, 0, n, ep, gm, sigma=sig, n_active=na)
    torch.cuda.synchronize()
    act = na.cpu().numpy()
    assert act.min() >= 0 and (act >= 2).mean() > 0.5
    p = dict(T1)
    C = svdcp.stiffness(p["C11"], p["C12"], p["C44"])
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(P, size=48, replace=False))
    s = sig.view(6, P)[:, torch.from_numpy(idx).cuda()].cpu().numpy().T
    g = gm[torch.from_numpy(idx).cuda()].cpu().numpy()
    for k, i in enumerate(idx):
        R = _R(quat[i])
        U = R.T @ np.diag([1.0, -0.5, -0.5]) @ R
        epo, go = np.zeros((3, 3)), 0.0
        for t in range(1, n + 1):
            epo, go, so, _, _ = svdcp.step(p, C, t * e * U, epo, go)
        assert np.abs(_t(s[k]) - so).max() <= 1e-9 * np.abs(so).max(), i
        assert abs(g[k] - go) <= 1e-9 * max(go, 1e-12)
