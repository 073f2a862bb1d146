"""Deterministic rate-independent multi-slip crystal plasticity (FP64 numpy):
the comparator the paper checks its Monte Carlo plasticity against (Sec. 2,
Fig. 1: a single nickel crystal under the prescribed strain increment
e diag(1, -1/2, -1/2), e = 1e-6, stress-strain curves of both methods agree).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Small strain, crystal frame, the 12 FCC {111}<110> systems with Schmid tensors
P_a = sym(m_a (x) n_a), cubic stiffness C, isotropic Voce hardening shared by
all systems, g(gamma) = taus - (taus - tau0) exp(-h0 gamma / (taus - tau0)),
gamma the accumulated slip.  One step from (eps_p, gamma) to the total strain
eps (the increment is the same for every system, as in the Taylor load):

  trial stress s_tr = C : (eps - eps_p), resolved shear tau_a = P_a : s_tr,
  signs s_a = sign(tau_a), active set A = {a : |tau_a| - g(gamma) > 0};
  on A solve  s_a tau_a - sum_b A_ab x_b - g(gamma + sum_b x_b) = 0,
  A_ab = s_a s_b P_a : C : P_b, by Newton steps x <- x - J^+ r with
  J = -(A + g'(gamma + sum x) 1 1^T) and J^+ its pseudo-inverse (numpy pinv:
  the SVD, singular values below 1e-10 of the largest dropped) -- the FCC
  constraints are linearly dependent, hence ill-conditioned;
  while a slip comes out below -1e-6 tol, drop the system of the most negative
  slip and solve again; then, while an inactive system's resolved shear exceeds
  g by more than 10 tol, add the most over-stressed one, with s_a the sign of
  its current resolved shear (a large increment can reverse it from the
  trial's), and solve again; at most 50 passes; commit
  eps_p += sum_a x_a s_a P_a, gamma += sum_a x_a.  Ties go to the lowest
  system index (the order of FCC_N / FCC_M below).

The paper gives neither the active-set strategy nor the SVD cut-off; the two
choices above are a reading.  One change at a time matters: dropping every
negative slip and adding every over-stressed system at once cycles between two
sets on increments far beyond the yield strain.
"""
from __future__ import annotations

import numpy as np

SN = 1.0 / np.sqrt(3.0)
SM = 1.0 / np.sqrt(2.0)
FCC_N = np.array([[1, 1, 1], [1, 1, 1], [1, 1, 1], [-1, 1, 1], [-1, 1, 1], [-1, 1, 1],
                  [1, -1, 1], [1, -1, 1], [1, -1, 1], [1, 1, -1], [1, 1, -1], [1, 1, -1]], float) * SN
FCC_M = np.array([[0, 1, -1], [-1, 0, 1], [1, -1, 0], [0, 1, -1], [1, 0, 1], [1, 1, 0],
                  [0, 1, 1], [1, 0, -1], [1, 1, 0], [0, 1, 1], [1, 0, 1], [1, -1, 0]], float) * SM


def schmid():
    return np.stack([0.5 * (np.outer(m, n) + np.outer(n, m)) for m, n in zip(FCC_M, FCC_N)])


def stiffness(C11, C12, C44):
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            C[i, i, j, j] = C12
            C[i, j, i, j] += C44
            C[i, j, j, i] += C44
        C[i, i, i, i] = C11
    return C


def voce(p, gamma):
    ds = p["taus"] - p["tau0"]
    if ds <= 0 or p["h0"] <= 0:
        return p["tau0"] + 0.0 * gamma  # no hardening
    return p["taus"] - ds * np.exp(-p["h0"] * gamma / ds)


def voce_slope(p, gamma):
    ds = p["taus"] - p["tau0"]
    if ds <= 0 or p["h0"] <= 0:
        return 0.0 * gamma
    return p["h0"] * np.exp(-p["h0"] * gamma / ds)


def _solve(active, sgn, tau_tr, K, p, gamma, tol):
    idx = np.flatnonzero(active)
    x = np.zeros(idx.size)
    A = sgn[idx, None] * sgn[None, idx] * K[np.ix_(idx, idx)]
    for _ in range(100):
        gam = gamma + x.sum()
        r = sgn[idx] * tau_tr[idx] - A @ x - voce(p, gam)
        if np.abs(r).max() < tol:
            break
        J = -(A + voce_slope(p, gam) * np.ones((idx.size, idx.size)))
        x = x - np.linalg.pinv(J, rcond=1e-10) @ r
    return idx, x


def step(p, C, eps, eps_p, gamma, tol=None):
    """One deterministic step to total strain eps (crystal frame 3x3); returns
    (eps_p, gamma, stress, active systems, slips)."""
    P = schmid()
    K = np.einsum("aij,ijkl,bkl->ab", P, C, P)
    tol = 1e-12 * p["tau0"] if tol is None else tol
    s_tr = np.einsum("ijkl,kl->ij", C, eps - eps_p)
    tau = np.einsum("aij,ij->a", P, s_tr)
    sgn = np.where(tau >= 0, 1.0, -1.0)
    g0 = voce(p, gamma)
    active = np.abs(tau) - g0 > tol
    if not active.any():
        return eps_p, gamma, s_tr, np.zeros(0, int), np.zeros(0)
    for _ in range(50):
        idx, x = _solve(active, sgn, tau, K, p, gamma, tol)
        if (x < -tol * 1e-6).any():
            active[idx[np.argmin(x)]] = False
            if not active.any():
                return eps_p, gamma, s_tr, np.zeros(0, int), np.zeros(0)
            continue
        dep = np.einsum("a,aij->ij", x * sgn[idx], P[idx])
        s = np.einsum("ijkl,kl->ij", C, eps - eps_p - dep)
        t = np.einsum("aij,ij->a", P, s)
        g = voce(p, gamma + x.sum())
        over = np.where(active, -np.inf, np.abs(t) - g)
        if over.max() > tol * 10:
            a = int(np.argmax(over))
            sgn[a] = 1.0 if t[a] >= 0 else -1.0  # slips along its current resolved shear
            active[a] = True
            continue
        return eps_p + dep, gamma + x.sum(), s, idx, x
    raise RuntimeError("active set did not settle")


def uniaxial(p, R, e, n_steps):
    """Single crystal of orientation R (crystal -> sample) under total sample
    strain t e diag(1, -1/2, -1/2), t = 1..n_steps; returns the sample-frame
    sigma_xx history and the number of active systems per step."""
    C = stiffness(p["C11"], p["C12"], p["C44"])
    eps_p = np.zeros((3, 3))
    gamma = 0.0
    sxx, nact = [], []
    U = R.T @ np.diag([1.0, -0.5, -0.5]) @ R
    for t in range(1, n_steps + 1):
        eps_p, gamma, s, idx, _ = step(p, C, t * e * U, eps_p, gamma)
        sxx.append((R @ s @ R.T)[0, 0])
        nact.append(idx.size)
    return np.array(sxx), np.array(nact)
