"""Pins of the periodic elastic-equilibrium oracle (``oracle/elastic.py``), CPU.

What fixes the solution independently of the solver:
* a single crystal (homogeneous stiffness and eigenstrain) takes the mean strain
  E everywhere, with the stress of the rotated cubic stiffness applied to
  E - eps_p (closed form);
* a laminate of crystals in layers normal to x has, exactly, a strain that is
  uniform in each layer, E + sym(a_l (x) n) with zero mean jump, and a traction
  sigma . n equal in every layer: a small linear system (solved here from the
  rotated stiffness tensors, not with the solver's Green operator);
* any polycrystal reaches equilibrium (xi . sigma^hat = 0) with <eps> = E.
A planted mistake in the Green operator (the wrong sign of its volumetric term)
must fail the laminate.
"""
import numpy as np
import pytest

from paper_1007_3509_gb300 import synth

C3 = (synth.TABLE1["C11"], synth.TABLE1["C12"], synth.TABLE1["C44"])


def _stiffness(q):
    """Cubic stiffness rotated into the sample frame, C'_ijkl = R_ia R_jb R_kc R_ld C_abcd,
    with R the active rotation of q (w, x, y, z) built from quaternion products."""
    q = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    w, v = q[0], q[1:]
    R = np.empty((3, 3))
    for a, e in enumerate(np.eye(3)):   # image of the crystal axis e under q e q*
        t = 2.0 * np.cross(v, e)
        R[:, a] = e + w * t + np.cross(v, t)
    C = np.zeros((3, 3, 3, 3))
    C11, C12, C44 = C3
    for i in range(3):
        for j in range(3):
            if i == j:
                C[i, i, i, i] = C11
            else:
                C[i, i, j, j] = C12
                C[i, j, i, j] = C[i, j, j, i] = C44
    return np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, C), R


def _sym(v):
    v = np.asarray(v, dtype=np.float64)
    return np.array([[v[0], v[5], v[4]], [v[5], v[1], v[3]], [v[4], v[3], v[2]]])


def _voigt(t):
    return np.array([t[0, 0], t[1, 1], t[2, 2], t[1, 2], t[0, 2], t[0, 1]])


def _quats(n, seed):
    q = np.random.default_rng(seed).normal(size=(n, 4)).astype(np.float32)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


E0 = np.array([1e-3, -4e-4, -6e-4, 2e-4, -1e-4, 3e-4])


def test_single_crystal_takes_the_mean_strain():
    from oracle import elastic
    shape = (6, 4, 5)
    N = 120
    quat = _quats(1, 3)
    epc = np.array([2e-4, -1e-4, -1e-4, 5e-5, 0.0, -3e-5])  # crystal-frame eigenstrain
    eps, sig, it, ch = elastic.solve(shape, np.zeros(N, int), quat, C3, E0, eps_p=np.tile(epc, (N, 1)))
    assert np.abs(eps - E0).max() < 1e-14
    Cs, R = _stiffness(quat[0].astype(np.float64))
    ref = _voigt(np.einsum("ijkl,kl->ij", Cs, _sym(E0) - R @ _sym(epc) @ R.T))
    assert np.abs(sig - ref).max() < 1e-9 * np.abs(ref).max()
    assert it <= 2


def _laminate(quat, frac, epc_layers, E):
    """Exact laminate (layers normal to x): returns per-layer strain (sample frame)."""
    n = np.array([1.0, 0.0, 0.0])
    L = len(frac)
    Cs = [_stiffness(q.astype(np.float64)) for q in quat]
    A = np.zeros((3 * L + 3, 3 * L + 3))
    b = np.zeros(3 * L + 3)
    Et = _sym(E)
    for l in range(L):
        C, R = Cs[l]
        epl = R @ _sym(epc_layers[l]) @ R.T
        acoustic = np.einsum("ijkh,j,h->ik", C, n, n)
        A[3 * l:3 * l + 3, 3 * l:3 * l + 3] = acoustic
        A[3 * l:3 * l + 3, 3 * L:3 * L + 3] = -np.eye(3)
        b[3 * l:3 * l + 3] = -np.einsum("ijkh,kh,j->i", C, Et - epl, n)
        A[3 * L:3 * L + 3, 3 * l:3 * l + 3] = frac[l] * np.eye(3)
    x = np.linalg.solve(A, b)
    return [Et + 0.5 * (np.outer(x[3 * l:3 * l + 3], n) + np.outer(n, x[3 * l:3 * l + 3])) for l in range(L)]


def _laminate_case(elastic):
    # odd length across the layers: no Nyquist plane there
    shape = (9, 3, 2)
    N = 54
    x = np.arange(N) % 9
    grain = (x >= 3).astype(int)
    quat = _quats(2, 11)
    epc = np.array([[1e-4, 0, -1e-4, 2e-5, 0, 0], [-5e-5, 5e-5, 0, 0, 3e-5, -1e-5]])
    eps, sig, it, ch = elastic.solve(shape, grain, quat, C3, E0, eps_p=epc[grain], tol=1e-12)
    ref = _laminate(quat, [3 / 9, 6 / 9], epc, E0)
    want = np.stack([_voigt(ref[g]) for g in grain])
    return np.abs(eps - want).max() / np.abs(E0).max(), it


def test_laminate_matches_the_exact_solution():
    from oracle import elastic
    err, it = _laminate_case(elastic)
    assert err < 1e-9, err


def test_laminate_fails_with_a_wrong_green_operator(monkeypatch):
    from oracle import elastic
    right = elastic.green_apply

    def wrong(tau_hat, xi, lam0, mu0):
        # the volumetric term with the wrong sign
        nrm = np.linalg.norm(xi, axis=1)
        n = np.where(nrm[:, None] > 0, xi / np.where(nrm > 0, nrm, 1.0)[:, None], 0.0)
        c = np.einsum("pi,pij,pj->p", n, tau_hat, n)
        kappa = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0))
        return right(tau_hat, xi, lam0, mu0) - 2.0 * kappa * c[:, None, None] * np.einsum("pi,pj->pij", n, n)

    monkeypatch.setattr(elastic, "green_apply", wrong)
    err, _ = _laminate_case(elastic)
    assert err > 1e-3, err


@pytest.mark.parametrize("shape", [(8, 8, 8), (12, 6, 4), (9, 7, 5)])
def test_polycrystal_reaches_equilibrium(shape):
    from oracle import elastic
    N = int(np.prod(shape))
    rng = np.random.default_rng(5)
    grain = rng.integers(0, 6, size=N)
    quat = _quats(6, 7)
    eps, sig, it, ch = elastic.solve(shape, grain, quat, C3, E0, tol=1e-11)
    assert ch < 1e-11 and it < 200
    assert np.abs(eps.mean(axis=0) - E0).max() < 1e-15
    assert elastic.equilibrium_residual(shape, sig) < 1e-9
    # heterogeneous: the strain is not uniform, and it differs from the Taylor strain
    assert np.abs(eps - E0).max() > 1e-2 * np.abs(E0).max()
