"""Pins of the deterministic multi-slip comparator (``oracle/svdcp.py``), CPU,
and its agreement with the Monte Carlo plasticity on the single-crystal test of
Sec. 2 (Fig. 1: strain steps of 1e-6, the two stress-strain curves agree)."""
import numpy as np
import pytest

from paper_1007_3509_gb300 import synth

T1 = synth.TABLE1


def _p(**kw):
    p = dict(T1)
    p.update(kw)
    return p


def _rot(seed):
    q = np.random.default_rng(seed).normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]]), q


def test_elastic_range_is_hooke():
    from oracle import svdcp
    p = _p()
    C = svdcp.stiffness(p["C11"], p["C12"], p["C44"])
    R, _ = _rot(1)
    eps = 2e-6 * R.T @ np.diag([1, -0.5, -0.5]) @ R
    ep, g, s, idx, x = svdcp.step(p, C, eps, np.zeros((3, 3)), 0.0)
    assert idx.size == 0 and np.all(ep == 0)
    np.testing.assert_allclose(s, np.einsum("ijkl,kl->ij", C, eps), rtol=1e-14)


def test_single_slip_without_hardening_closed_form():
    """Just past first yield of a general orientation only one system is active;
    without hardening its slip is (|tau_tr| - tau0) / (P : C : P)."""
    from oracle import svdcp
    p = _p(taus=T1["tau0"])
    C = svdcp.stiffness(p["C11"], p["C12"], p["C44"])
    P = svdcp.schmid()
    R, _ = _rot(7)
    U = R.T @ np.diag([1, -0.5, -0.5]) @ R
    tau_unit = np.abs(np.einsum("aij,ijkl,kl->a", P, C, U))
    a = int(np.argmax(tau_unit))
    e_yield = p["tau0"] / tau_unit[a]
    eps = 1.02 * e_yield * U
    ep, g, s, idx, x = svdcp.step(p, C, eps, np.zeros((3, 3)), 0.0)
    assert list(idx) == [a]
    k = np.einsum("ij,ijkl,kl->", P[a], C, P[a])
    assert abs(x[0] - (tau_unit[a] * 1.02 * e_yield - p["tau0"]) / k) < 1e-12 * x[0]


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_consistency_along_a_loading_path(seed):
    from oracle import svdcp
    p = _p()
    C = svdcp.stiffness(p["C11"], p["C12"], p["C44"])
    P = svdcp.schmid()
    R, _ = _rot(seed)
    U = R.T @ np.diag([1, -0.5, -0.5]) @ R
    ep, gam = np.zeros((3, 3)), 0.0
    multi = 0
    for t in range(1, 61):
        ep, gam, s, idx, x = svdcp.step(p, C, t * 5e-5 * U, ep, gam)
        g = svdcp.voce(p, gam)
        tau = np.abs(np.einsum("aij,ij->a", P, s))
        assert np.all(tau <= g * (1 + 1e-9))
        if idx.size:
            assert np.all(np.abs(tau[idx] - g) <= 1e-9 * g)
            assert np.all(x >= -1e-15)
        multi = max(multi, idx.size)
    assert multi >= 2  # multiple slip develops


def test_symmetric_100_loading_slips_equally():
    """Loading along <100> stresses 8 systems equally (Schmid factor 1/sqrt 6): all
    8 activate together with equal slip."""
    from oracle import svdcp
    p = _p()
    C = svdcp.stiffness(p["C11"], p["C12"], p["C44"])
    U = np.diag([1.0, -0.5, -0.5])
    ep, gam = np.zeros((3, 3)), 0.0
    for t in range(1, 40):
        ep, gam, s, idx, x = svdcp.step(p, C, t * 2e-5 * U, ep, gam)
    assert idx.size == 8
    assert np.ptp(x) <= 1e-12 * x.max()


def test_perfect_plasticity_along_100_holds_the_yield_stress():
    """Without hardening under <100> loading the 8 active systems' combined slip
    is parallel to the applied strain, so past the yield strain
    e_y = tau0 / |P_a : C : U| all further strain is plastic and the stress stays
    C : U e_y: a closed form, reached through the pseudo-inverse of the rank
    deficient 8 x 8 constraint matrix."""
    from oracle import svdcp
    p = _p(taus=T1["tau0"])
    C = svdcp.stiffness(p["C11"], p["C12"], p["C44"])
    P = svdcp.schmid()
    U = np.diag([1.0, -0.5, -0.5])
    CU = np.einsum("ijkl,kl->ij", C, U)
    e_y = p["tau0"] / np.abs(np.einsum("aij,ij->a", P, CU)).max()
    ep, gam = np.zeros((3, 3)), 0.0
    for t in (0.5, 1.5, 3.0, 7.0):
        ep, gam, s, idx, x = svdcp.step(p, C, t * e_y * U, ep, gam)
        want = CU * min(t, 1.0) * e_y
        np.testing.assert_allclose(s, want, atol=1e-9 * abs(want).max())
        assert idx.size == (8 if t > 1 else 0)
    K = np.einsum("aij,ijkl,bkl->ab", P, C, P)[np.ix_(idx, idx)]
    assert np.linalg.matrix_rank(K, tol=1e-9 * abs(K).max()) < 8
    # every active system has |P_xx| = 1/sqrt 6, so the plastic strain (7 - 1) e_y
    # along x takes total slip 6 e_y sqrt 6, shared equally
    np.testing.assert_allclose(gam, 6.0 * e_y * np.sqrt(6.0), rtol=1e-9)
    np.testing.assert_allclose(ep, 6.0 * e_y * U, atol=1e-9 * e_y)


def test_wrong_sign_products_break_consistency(monkeypatch):
    """Planted mistake: the constraint matrix without the sign products s_a s_b."""
    from oracle import svdcp
    right = svdcp._solve

    def wrong(active, sgn, tau_tr, K, p, gamma, tol):
        return right(active, np.ones_like(sgn), tau_tr, K, p, gamma, tol)

    monkeypatch.setattr(svdcp, "_solve", wrong)
    p = _p()
    C = svdcp.stiffness(p["C11"], p["C12"], p["C44"])
    P = svdcp.schmid()
    R, _ = _rot(4)
    U = R.T @ np.diag([1, -0.5, -0.5]) @ R
    ep, gam = np.zeros((3, 3)), 0.0
    bad = 0.0
    for t in range(1, 61):
        try:
            ep, gam, s, idx, x = svdcp.step(p, C, t * 5e-5 * U, ep, gam)
        except RuntimeError:
            bad = 1.0
            break
        g = svdcp.voce(p, gam)
        tau = np.abs(np.einsum("aij,ij->a", P, s))
        bad = max(bad, (tau.max() - g) / g)
    assert bad > 1e-3


@pytest.mark.parametrize("seed", [8, 3])
def test_monte_carlo_plasticity_follows_the_deterministic_curve(oracle, seed):
    """Fig. 1 of Sec. 2: a nickel single crystal, strain steps of 1e-6 to 2e-3.
    While one system is active the Monte Carlo return map is the deterministic
    one (agreement to FP64 rounding of the two formulations); once several are
    active the MCP relaxes one system per step, so its stress rides a little
    above the deterministic curve with per-step scatter: mean within 2.5 %,
    every 100-step average within 3 %, every step within
    12 %."""
    from oracle import svdcp
    p = _p()
    R, q = _rot(seed)
    e, n = 1e-6, 2000
    s_svd, nact = svdcp.uniaxial(p, R, e, n)
    P = oracle.cp_params(T1["C11"], T1["C12"], T1["C44"], T1["tau0"], T1["taus"], T1["h0"], T1["beta"], e)
    quat = np.array([q], dtype=np.float32)
    Rf = svdcp_rot(quat[0])
    ep, gm = np.zeros((1, 6)), np.zeros(1)
    s_mcp = []
    for t in range(1, n + 1):
        ep, gm, sg, _, _ = oracle.mcp_run(P, 13, np.zeros(1, np.int32), quat, t - 1, 1, ep, gm)
        S = np.array([[sg[0, 0], sg[0, 5], sg[0, 4]], [sg[0, 5], sg[0, 1], sg[0, 3]], [sg[0, 4], sg[0, 3], sg[0, 2]]])
        s_mcp.append((Rf @ S @ Rf.T)[0, 0])
    rel = (np.array(s_mcp) - s_svd) / s_svd
    assert (nact > 0).mean() > 0.5 and nact.max() >= 3
    assert np.abs(rel[np.maximum.accumulate(nact) <= 1]).max() <= 1e-6  # before any multiple slip
    multi = nact >= 2
    assert 0 <= rel[multi].mean() <= 0.025, rel[multi].mean()
    first = int(np.argmax(multi))
    ma = np.convolve(rel[first:], np.ones(100) / 100, mode="valid")
    assert np.abs(ma).max() <= 0.03
    assert np.abs(rel[multi]).max() <= 0.12


def svdcp_rot(q):
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_large_increments_settle_consistently():
    """One-shot strains far beyond yield (about 20 yield strains, random
    directions): the active set settles, every active system sits on the yield
    surface with non-negative slip, no system lies outside it, and the plastic
    strain is the slips along the final resolved-shear signs."""
    from oracle import svdcp
    p = _p()
    C = svdcp.stiffness(p["C11"], p["C12"], p["C44"])
    P = svdcp.schmid()
    rng = np.random.default_rng(5)
    for i in range(60):
        R, _ = _rot(100 + i)
        e = rng.normal(size=6) * 1.2e-3
        E = np.array([[e[0], e[5], e[4]], [e[5], e[1], e[3]], [e[4], e[3], e[2]]])
        Ec = R.T @ E @ R
        ep, gam, s, idx, x = svdcp.step(p, C, Ec, np.zeros((3, 3)), 0.0)
        g = svdcp.voce(p, gam)
        tau = np.einsum("aij,ij->a", P, s)
        assert np.all(np.abs(tau) <= g * (1 + 1e-9))
        assert np.all(np.abs(np.abs(tau[idx]) - g) <= 1e-9 * g)
        assert np.all(x >= -1e-15) and idx.size >= 1
        # the committed plastic strain is the slips along the final signs
        np.testing.assert_allclose(ep, np.einsum("a,aij->ij", x * np.sign(tau[idx]), P[idx]), atol=1e-15)
