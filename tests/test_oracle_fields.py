"""Pins of the oracle's initial polycrystal, statistics, closed-form energies,
crystal plasticity and surrogate network (CPU only)."""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

from oracle import mlp
from paper_1007_3509_gb300 import synth


# --------------------------------------------------------------------------
# Voronoi polycrystal
# --------------------------------------------------------------------------
def _site_xyz(idx, L):
    idx = np.asarray(idx, dtype=np.int64)
    if len(L) == 2:
        return np.stack([idx % L[0], idx // L[0]], axis=1)
    return np.stack([idx % L[0], (idx // L[0]) % L[1], idx // (L[0] * L[1])], axis=1)


@pytest.mark.parametrize("L,G", [((64, 48), 40), ((20, 16, 12), 60)])
def test_voronoi_matches_periodic_kdtree(oracle, L, G):
    """Nearest seed under periodic distance equals scipy's periodic cKDTree; ties go to the lowest index."""
    dim = len(L)
    q, pos = oracle.voronoi(dim, L, G, 4242)
    assert len(np.unique(pos)) == G
    tree = cKDTree(_site_xyz(pos, L).astype(float), boxsize=np.array(L, dtype=float))
    xyz = _site_xyz(np.arange(q.size), L).astype(float)
    dist, _ = tree.query(xyz, k=8)
    # the oracle's seed is at the minimum distance
    chosen = _site_xyz(pos[q], L).astype(float)
    d = np.abs(xyz - chosen)
    d = np.minimum(d, np.array(L) - d)
    dq = np.sqrt((d * d).sum(1))
    np.testing.assert_allclose(dq, dist[:, 0], rtol=0, atol=1e-9)
    # ties: every seed at the minimum distance has an index >= the chosen one
    _, idx = tree.query(xyz, k=8)
    for s in range(q.size):
        tied = idx[s][np.abs(dist[s] - dist[s, 0]) < 1e-9]
        assert q[s] == tied.min()


def test_voronoi_seed_rounds_fill_every_site(oracle):
    """With as many seeds as sites, the collision rounds must end with every site owned once."""
    pos = oracle.voronoi_seeds(2, (8, 8), 64, 5)
    assert sorted(pos.tolist()) == list(range(64))


def test_voronoi_seed_positions_uniform(oracle):
    pos = oracle.voronoi_seeds(2, (64, 64), 3000, 9)
    xy = _site_xyz(pos, (64, 64))
    for c in range(2):
        h = np.bincount(xy[:, c] // 4, minlength=16)
        assert stats.chisquare(h).pvalue > 1e-4


def test_quaternion_rotation_matches_scipy(oracle):
    """R(q) maps crystal to sample axes; the loading axis in the crystal frame is R^T e_x."""
    qs = synth.random_quaternions(50, 3)
    for q in qs:
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(oracle.loading_axis(q), R.T @ np.array([1.0, 0, 0]), atol=1e-6)


def test_zrot_quaternion_is_angle_about_z(oracle):
    """Kind 2 is the rotation by the kind-0 angle about z (scipy rotation vector (0, 0, t))."""
    a = oracle.orientations(200, 17, 0).astype(np.float64)
    q = oracle.orientations(200, 17, 2)
    ref = Rotation.from_rotvec(np.stack([np.zeros_like(a), np.zeros_like(a), a], 1)).as_quat()  # x,y,z,w
    np.testing.assert_allclose(q, np.stack([ref[:, 3], ref[:, 0], ref[:, 1], ref[:, 2]], 1), atol=1e-7)
    bins, near = oracle.grain_bins(q, 2)
    b0, _ = oracle.grain_bins(a.astype(np.float32), 0)
    ok = near > 1e-6
    np.testing.assert_array_equal(bins[ok], b0[ok])


def test_orientations_uniform_on_so3(oracle):
    """Shoemake quaternions: rotation angle has CDF (t - sin t)/pi; the loading axis is uniform on the sphere."""
    q = oracle.orientations(20000, 31, 1).astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=2e-7)
    theta = 2.0 * np.arccos(np.clip(np.abs(q[:, 0]), 0, 1))
    assert stats.kstest(theta, lambda t: (t - np.sin(t)) / np.pi).pvalue > 1e-3
    d = np.array([oracle.loading_axis(x.astype(np.float32)) for x in q[:4000]])
    assert stats.kstest(d[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-3
    a = oracle.orientations(20000, 32, 0)
    assert a.min() >= 0 and a.max() < np.pi / 2
    assert stats.kstest(a, "uniform", args=(0, np.pi / 2)).pvalue > 1e-3


# --------------------------------------------------------------------------
# Grain statistics and texture bins
# --------------------------------------------------------------------------
def test_grain_counts_match_bincount(oracle):
    q = synth.random_lattice((100, 70), 300, 8)
    counts, alive = oracle.grain_counts(q, 310)
    np.testing.assert_array_equal(counts, np.bincount(q, minlength=310))
    assert alive == np.count_nonzero(np.bincount(q, minlength=310))


def test_angle_bins_match_numpy_histogram(oracle):
    a = oracle.orientations(5000, 3, 0)
    bins, near = oracle.grain_bins(a, 0)
    ok = near > 1e-9
    ref = np.digitize(np.degrees(a.astype(np.float64)), np.arange(1, 90))
    np.testing.assert_array_equal(bins[ok], ref[ok])


def test_so3_bins_known_directions(oracle):
    """Family bins of exact <100>, <110>, <111> loading axes and a direction away from all three."""
    def q_from_R(R):
        x, y, z, w = Rotation.from_matrix(R).as_quat()
        return np.array([w, x, y, z], dtype=np.float32)

    def axis_to_quat(d):
        d = np.asarray(d, float) / np.linalg.norm(d)
        # rotation whose first row (R^T e_x) is d
        a = np.cross(d, [0.0, 0.0, 1.0]) if abs(d[2]) < 0.9 else np.cross(d, [0.0, 1.0, 0.0])
        a /= np.linalg.norm(a)
        c = np.cross(d, a)
        return q_from_R(np.stack([d, a, c]))

    cases = {(1, 0, 0): 21, (1, 1, 0): 22, (1, 1, 1): 23, (0.35, 0.8, 0.05): 20}
    for d, fam in cases.items():
        b, _ = oracle.grain_bins(axis_to_quat(d)[None, :], 1)
        assert b[0, 1] == fam, (d, b)


# --------------------------------------------------------------------------
# Closed-form energies (Sec. 5)
# --------------------------------------------------------------------------
def _E_textbook(C11, C12, C44, d):
    """Cubic directional modulus: 1/E = S11 - 2 (S11 - S12 - S44/2)(l^2 m^2 + m^2 n^2 + n^2 l^2)."""
    den = (C11 - C12) * (C11 + 2 * C12)
    S11, S12, S44 = (C11 + C12) / den, -C12 / den, 1.0 / C44
    l, m, n = np.asarray(d, float) / np.linalg.norm(d)
    return 1.0 / (S11 - 2 * (S11 - S12 - 0.5 * S44) * (l * l * m * m + m * m * n * n + n * n * l * l))


def test_directional_modulus_textbook(oracle):
    rng = np.random.default_rng(1)
    for consts in (synth.TABLE1, synth.NI_BJ):
        Cc = np.array([consts["C11"], consts["C12"], consts["C44"]])
        for d in rng.normal(size=(30, 3)):
            np.testing.assert_allclose(oracle.directional_modulus(Cc, d), _E_textbook(*Cc, d), rtol=1e-12)


def test_modulus_order_about_z_rotation(oracle):
    """Sec. 5: grains at 23-45 deg about z have a larger Young's modulus along x than 0-22 deg."""
    Cc = np.array([synth.TABLE1[k] for k in ("C11", "C12", "C44")])
    E = [oracle.directional_modulus(Cc, [math.cos(math.radians(t)), -math.sin(math.radians(t)), 0.0])
         for t in (0.0, 22.5, 45.0)]
    assert E[0] < E[1] < E[2]
    # <100> and <110> closed forms
    den = Cc[0] + Cc[1]
    E100 = (Cc[0] - Cc[1]) * (Cc[0] + 2 * Cc[1]) / den
    assert abs(E[0] - E100) < 1e-6 * E100


def test_schmid_factor_closed_forms(oracle):
    """FCC {111}<110>: m_max(<100>) = m_max(<110>) = 1/sqrt6, m_max(<111>) = 2/(3 sqrt6);
    about z the maxima sit near 22.5 and 67.5 deg, and 0 deg equals 45 deg (Sec. 5, Fig. 4)."""
    assert abs(oracle.max_schmid([1, 0, 0]) - 1 / math.sqrt(6)) < 1e-12
    assert abs(oracle.max_schmid([1, 1, 0]) - 1 / math.sqrt(6)) < 1e-12
    assert abs(oracle.max_schmid([1, 1, 1]) - 2 / (3 * math.sqrt(6))) < 1e-12
    th = np.radians(np.arange(0, 90.01, 0.25))
    m = np.array([oracle.max_schmid([math.cos(t), math.sin(t), 0.0]) for t in th])
    deg = np.degrees(th)
    a1 = deg[np.argmax(np.where(deg <= 45, m, -1))]
    a2 = deg[np.argmax(np.where(deg >= 45, m, -1))]
    assert abs(a1 - 22.5) <= 2.0 and abs(a2 - 67.5) <= 2.0
    np.testing.assert_allclose(m, m[::-1], atol=1e-12)
    n, mm = oracle.slip_systems()
    assert np.allclose((n * mm).sum(1), 0) and np.allclose(np.linalg.norm(n, axis=1), 1)
    # the 12 systems are distinct up to sign
    keys = {tuple(np.round(np.sign(n[a][0] or 1) * np.concatenate([n[a], mm[a] * np.sign(mm[a][np.nonzero(mm[a])[0][0]])]), 6)) for a in range(12)}
    assert len(keys) == 12


def test_grain_field_uniaxial_energy(oracle):
    """w = sigma^2 / (2 E(d)); identity orientation loads along <100>."""
    Cc = np.array([synth.NI_BJ[k] for k in ("C11", "C12", "C44")])
    q = np.array([[1, 0, 0, 0]], dtype=np.float32)
    w, mm, e, b = oracle.grain_field(q, Cc, 100.0, 0.05, 1.0)
    E100 = (Cc[0] - Cc[1]) * (Cc[0] + 2 * Cc[1]) / (Cc[0] + Cc[1])
    assert abs(w[0] - 100.0 ** 2 / (2 * E100)) < 1e-12
    assert abs(w[0] - 0.03668) < 5e-5
    assert abs(mm[0] - 1 / math.sqrt(6)) < 1e-7
    assert b[0] == int(np.rint(256 * (w[0] + 0.05 * mm[0])))


def test_gaussian_bulk_energy_eq9(oracle):
    """Eq. (9): symmetric about n = 46 with peak (32 pi)^(-1/2); orientation n = floor(degrees) + 1."""
    deg = np.arange(90) + 0.5
    e, b = oracle.gaussian_field(np.radians(deg).astype(np.float32))
    assert abs(e[45] - 1 / math.sqrt(32 * math.pi)) < 1e-15 and np.argmax(e) == 45
    for k in range(1, 45):   # e(46 - k) == e(46 + k)
        assert abs(e[45 - k] - e[45 + k]) < 1e-15
    assert abs(e[0] - math.exp(-45 ** 2 / (2 * 46 ** 2)) / math.sqrt(32 * math.pi)) < 1e-15
    np.testing.assert_array_equal(b, np.rint(256 * e).astype(np.int32))


def test_quantise_round_half_even(oracle):
    e = np.array([0.5, 1.5, 2.5, -0.5, -1.5, 1e9, -1e9]) / 256.0
    np.testing.assert_array_equal(oracle.quantise(e), [0, 2, 2, 0, -2, 1 << 20, -(1 << 20)])


# --------------------------------------------------------------------------
# Monte Carlo crystal plasticity (Sec. 2)
# --------------------------------------------------------------------------
def _P(**kw):
    import oracle as o
    c = dict(synth.TABLE1)
    c.update(kw)
    return o.cp_params(c["C11"], c["C12"], c["C44"], c["tau0"], c["taus"], c["h0"], c["beta"],
                       kw.get("e_incr", 1e-4))


IDENT = np.array([1, 0, 0, 0], dtype=np.float32)


def test_mcp_elastic_range_closed_form(oracle):
    """Below yield the response is elastic: sigma = C : eps with eps = t e diag(1, -1/2, -1/2)."""
    P = _P(e_incr=1e-5)
    ep, g, s, _, _, ch, nc = oracle.mcp_increment(P, 1, 0, 3, IDENT, np.zeros(6), 0.0)
    e = 3e-5
    C11, C12 = synth.TABLE1["C11"], synth.TABLE1["C12"]
    assert nc == 0 and ch == -1
    np.testing.assert_allclose(s, [(C11 - C12) * e, -(C11 - C12) * e / 2, -(C11 - C12) * e / 2, 0, 0, 0],
                               rtol=1e-12, atol=1e-12)


def test_mcp_first_yield_closed_form(oracle):
    """<100> loading: max |tau| = (C11 - C12) e sqrt(6)/4 on 8 systems; yield where it reaches tau_0."""
    C11, C12 = synth.TABLE1["C11"], synth.TABLE1["C12"]
    ey = synth.TABLE1["tau0"] / ((C11 - C12) * math.sqrt(6) / 4)
    below = _P(e_incr=ey * (1 - 1e-6))
    above = _P(e_incr=ey * (1 + 1e-6))
    assert oracle.mcp_increment(below, 1, 0, 1, IDENT, np.zeros(6), 0.0)[6] == 0
    assert oracle.mcp_increment(above, 1, 0, 1, IDENT, np.zeros(6), 0.0)[6] == 8


def test_mcp_single_slip_without_hardening(oracle):
    """tau_s = tau_0: dgamma = (|tau_tr| - tau_0)/(P:C:P) for a lone candidate, then |tau| = tau_0."""
    import oracle as o
    P = _P(taus=synth.TABLE1["tau0"], e_incr=1e-4)
    q = synth.random_quaternions(400, 12)
    n, m = o.slip_systems()
    Cc = [synth.TABLE1[k] for k in ("C11", "C12", "C44")]

    def Cmul(e):
        C11, C12, C44 = Cc
        s = np.zeros((3, 3))
        tr = np.trace(e)
        for i in range(3):
            s[i, i] = (C11 - C12) * e[i, i] + C12 * tr
        for i, j in ((0, 1), (0, 2), (1, 2)):
            s[i, j] = s[j, i] = 2 * C44 * e[i, j]
        return s

    found = 0
    for qq in q:
        # scale the strain so the largest |tau| just exceeds tau_0 (single candidate)
        R = Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix()
        es = np.diag([1.0, -0.5, -0.5])
        ec = R.T @ es @ R
        s1 = Cmul(ec)
        taus = np.array([np.sum(s1 * 0.5 * (np.outer(m[a], n[a]) + np.outer(n[a], m[a]))) for a in range(12)])
        order = np.argsort(-np.abs(taus))
        if abs(taus[order[1]]) > 0.999 * abs(taus[order[0]]):
            continue
        e_need = synth.TABLE1["tau0"] / abs(taus[order[0]])
        e = e_need * 1.0005
        P = _P(taus=synth.TABLE1["tau0"], e_incr=e)
        ep, g, s, _, _, ch, nc = o.mcp_increment(P, 3, 0, 1, qq, np.zeros(6), 0.0)
        assert nc == 1 and ch == order[0]
        a = order[0]
        Pa = 0.5 * (np.outer(m[a], n[a]) + np.outer(n[a], m[a]))
        k = np.sum(Pa * Cmul(Pa))
        dg_ref = (abs(taus[a]) * e - synth.TABLE1["tau0"]) / k
        assert abs(g - dg_ref) < 1e-12 * max(dg_ref, 1e-30) + 1e-18
        S = np.array([[s[0], s[5], s[4]], [s[5], s[1], s[3]], [s[4], s[3], s[2]]])
        assert abs(abs(np.sum(S * Pa)) - synth.TABLE1["tau0"]) < 1e-9
        found += 1
    assert found > 50


def test_mcp_consistency_after_step(oracle):
    """After each plastic increment the chosen system sits on the Voce yield surface |tau| = g(gamma)."""
    import oracle as o
    P = _P(e_incr=2e-4)
    n, m = o.slip_systems()
    qs = synth.random_quaternions(60, 5)
    t0, tau0, taus, h0 = 0, synth.TABLE1["tau0"], synth.TABLE1["taus"], synth.TABLE1["h0"]
    checked = 0
    for p, qq in enumerate(qs):
        ep, gam = np.zeros(6), 0.0
        for t in range(1, 8):
            ep, gam, s, _, _, ch, nc = o.mcp_increment(P, 9, p, t, qq, ep, gam)
            if ch < 0:
                continue
            Pa = 0.5 * (np.outer(m[ch], n[ch]) + np.outer(n[ch], m[ch]))
            S = np.array([[s[0], s[5], s[4]], [s[5], s[1], s[3]], [s[4], s[3], s[2]]])
            g = taus - (taus - tau0) * math.exp(-h0 * gam / (taus - tau0))
            assert abs(abs(np.sum(S * Pa)) - g) < 1e-9 * g
            checked += 1
    assert checked > 100


def test_mcp_selection_frequencies(oracle):
    """Eq. (2): the chosen system follows p_alpha of Eq. (1); sum p = 1."""
    import oracle as o
    P = _P(e_incr=3e-4, beta=2.0e3)
    qq = synth.random_quaternions(1, 77)[0]
    cand, prob = o.mcp_probabilities(P, 1, qq, np.zeros(6), 0.0)
    assert len(cand) >= 2 and abs(prob.sum() - 1) < 1e-12
    S = 20000
    picks = np.array([o.mcp_increment(P, 1, p, 1, qq, np.zeros(6), 0.0)[5] for p in range(S)])
    obs = np.array([(picks == a).sum() for a in cand])
    assert obs.sum() == S
    exp_ = prob * S
    keep = exp_ >= 5
    chi = ((obs[keep] - exp_[keep]) ** 2 / exp_[keep]).sum()
    assert stats.chi2.sf(chi, max(keep.sum() - 1, 1)) > 1e-4


def test_mcp_energies_closed_form(oracle):
    """Eq. (4): E_rho = 2 sigma_f^2 / G with sigma_f = g(gamma); w = sigma^2/(2 E100) for sigma along <100>."""
    import oracle as o
    P = _P()
    C11, C12 = synth.TABLE1["C11"], synth.TABLE1["C12"]
    sig = np.array([[50.0, 0, 0, 0, 0, 0], [0.0, 0, 0, 0, 0, 30.0]])
    gam = np.array([0.0, 0.01])
    w, er = o.mcp_energies(P, sig, gam)
    E100 = (C11 - C12) * (C11 + 2 * C12) / (C11 + C12)
    assert abs(w[0] - 50.0 ** 2 / (2 * E100)) < 1e-12
    assert abs(w[1] - 30.0 ** 2 / (2 * synth.TABLE1["C44"])) < 1e-12
    G = (C11 - C12 + 3 * synth.TABLE1["C44"]) / 5
    tau0, taus, h0 = synth.TABLE1["tau0"], synth.TABLE1["taus"], synth.TABLE1["h0"]
    g1 = taus - (taus - tau0) * math.exp(-h0 * 0.01 / (taus - tau0))
    np.testing.assert_allclose(er, [2 * tau0 ** 2 / G, 2 * g1 ** 2 / G], rtol=1e-14)


# --------------------------------------------------------------------------
# Surrogate MLP (FP64)
# --------------------------------------------------------------------------
def test_mlp_gradients_finite_differences():
    params = synth.mlp_init(3)
    rng = np.random.default_rng(4)
    for p in params[1::2]:
        p += rng.normal(0, 0.1, size=p.shape)
    X = rng.normal(size=(7, 11))
    T = rng.normal(size=(7, 2))
    L0, grads = mlp.loss_and_grads(params, X, T)
    h = 1e-6
    for k, p in enumerate(params):
        flat = p.ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            Lp, _ = mlp.loss_and_grads(params, X, T)
            flat[idx] = old - h
            Lm, _ = mlp.loss_and_grads(params, X, T)
            flat[idx] = old
            fd = (Lp - Lm) / (2 * h)
            g = grads[k].ravel()[idx]
            assert abs(fd - g) <= 1e-6 * max(abs(g), 1e-3), (k, idx, fd, g)


def test_mlp_matches_torch_autograd_fp64():
    import torch
    params = synth.mlp_init(8)
    rng = np.random.default_rng(9)
    X = rng.normal(size=(33, 11))
    T = rng.normal(size=(33, 2))
    L0, grads = mlp.loss_and_grads(params, X, T)
    tp = [torch.tensor(p, dtype=torch.float64, requires_grad=True) for p in params]
    a = torch.tensor(X)
    for l in range(4):
        a = a @ tp[2 * l].T + tp[2 * l + 1]
        if l < 3:
            a = torch.nn.functional.gelu(a)
    Lt = ((a - torch.tensor(T)) ** 2).sum() / (2 * X.shape[0])
    Lt.backward()
    assert abs(Lt.item() - L0) < 1e-12 * abs(L0)
    for p, g in zip(tp, grads):
        np.testing.assert_allclose(p.grad.numpy(), g, rtol=1e-10, atol=1e-14)


def test_adam_matches_torch():
    import torch
    params = synth.mlp_init(1)
    rng = np.random.default_rng(2)
    grads = [rng.normal(size=p.shape) for p in params]
    m = [np.zeros_like(p) for p in params]
    v = [np.zeros_like(p) for p in params]
    tp = [torch.tensor(p, dtype=torch.float64, requires_grad=True) for p in params]
    opt = torch.optim.Adam(tp, lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    p_np = params
    for t in range(1, 4):
        for x, g in zip(tp, grads):
            x.grad = torch.tensor(g)
        opt.step()
        p_np, m, v = mlp.adam_step(p_np, grads, m, v, t, 1e-3)
    for x, p in zip(tp, p_np):
        np.testing.assert_allclose(x.detach().numpy(), p, rtol=1e-12, atol=1e-15)
