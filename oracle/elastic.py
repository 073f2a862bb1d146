"""Periodic elastic equilibrium of a cubic polycrystal on the lattice grid (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 5 couples the Monte Carlo crystal plasticity to a deformation solver
(the material point method of the authors' earlier work) and iterates every
load increment to quasi-static equilibrium, so that each material point sees
its own strain increment instead of the uniform Taylor strain of Eq. (3).  The
solver here is the periodic Lippmann-Schwinger fixed point of Moulinec and
Suquet (Comput. Methods Appl. Mech. Engrg. 157 (1998) 69-94) on the voxel grid
of the Potts lattice, one material point per voxel:

    sigma(x) = C(x) : (eps(x) - eps_p(x)),   C(x) the cubic stiffness rotated
               into the sample frame by the orientation of the voxel's grain,
    tau = sigma - C0 : eps,                  C0 isotropic (lambda0, mu0),
    eps^hat(xi) = -Gamma0(xi) : tau^hat(xi) (xi != 0),   eps^hat(0) = E,

with the Green operator of the isotropic reference medium applied as
    Gamma0 : tau = (n (x) a + a (x) n) / (2 mu0) - kappa (n . a) n (x) n,
    n = xi / |xi|, a = tau n, kappa = (lambda0 + mu0) / (mu0 (lambda0 + 2 mu0)).
On even grid lengths the strain fluctuation is set to zero on the Nyquist
planes (any wave-vector component equal to -n/2): there the sign of the
frequency is ambiguous and the operator would break the Hermitian symmetry of
a real field (the usual convention of FFT homogenisation codes).  Iterations
stop when the largest change of any strain component is below tol * max|E|.
Stresses are evaluated in the crystal frame (eps_c = R^T eps R,
sigma = R (C : (eps_c - eps_p,c)) R^T), the plastic strain being stored in the
crystal frame as in ``oracle_mcp_*``.  numpy's FFT is the library primitive.

Voigt order everywhere: xx yy zz yz xz xy (tensor components, not engineering).
"""
from __future__ import annotations

import numpy as np

VI = (0, 1, 2, 1, 0, 0)
VJ = (0, 1, 2, 2, 2, 1)


def rotations(quat):
    """R (crystal -> sample) of unit quaternions (w, x, y, z), [n, 3, 3]."""
    q = np.asarray(quat, dtype=np.float64).reshape(-1, 4)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z); R[:, 0, 1] = 2 * (x * y - w * z); R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z); R[:, 1, 1] = 1 - 2 * (x * x + z * z); R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y); R[:, 2, 1] = 2 * (y * z + w * x); R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def tensor(v):
    """Symmetric [n, 3, 3] from Voigt [n, 6]."""
    v = np.asarray(v, dtype=np.float64).reshape(-1, 6)
    t = np.empty((v.shape[0], 3, 3))
    for c in range(6):
        t[:, VI[c], VJ[c]] = v[:, c]
        t[:, VJ[c], VI[c]] = v[:, c]
    return t


def voigt(t):
    return np.stack([t[:, VI[c], VJ[c]] for c in range(6)], axis=1)


def cubic_stress(Cc, e):
    """C : e for the cubic stiffness in its own frame, e [n, 3, 3]."""
    C11, C12, C44 = Cc
    tr = np.trace(e, axis1=1, axis2=2)
    s = 2.0 * C44 * e
    for i in range(3):
        s[:, i, i] = (C11 - C12) * e[:, i, i] + C12 * tr
    return s


def reference_medium(Cc):
    """Isotropic reference (lambda0, mu0): the mean of the two shear moduli of the
    cubic crystal, C44 and (C11 - C12)/2, and its bulk modulus (C11 + 2 C12)/3."""
    C11, C12, C44 = Cc
    mu0 = 0.5 * (C44 + 0.5 * (C11 - C12))
    K = (C11 + 2.0 * C12) / 3.0
    return K - 2.0 * mu0 / 3.0, mu0


def green_apply(tau_hat, xi, lam0, mu0):
    """eps^hat = -Gamma0(xi) : tau^hat for xi != 0 (rows with xi = 0 give 0)."""
    nrm = np.linalg.norm(xi, axis=1)
    n = np.where(nrm[:, None] > 0, xi / np.where(nrm > 0, nrm, 1.0)[:, None], 0.0)
    a = np.einsum("pij,pj->pi", tau_hat, n)
    c = np.einsum("pi,pi->p", n, a)
    kappa = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0))
    g = (np.einsum("pi,pj->pij", n, a) + np.einsum("pi,pj->pij", a, n)) / (2.0 * mu0) \
        - kappa * c[:, None, None] * np.einsum("pi,pj->pij", n, n)
    return -g


def wave_vectors(shape):
    """Integer wave vectors (x, y, z components) of a grid [nz, ny, nx], flattened
    in the grid's linear order x + nx (y + ny z)."""
    nx, ny, nz = shape
    kx = np.fft.fftfreq(nx) * nx
    ky = np.fft.fftfreq(ny) * ny
    kz = np.fft.fftfreq(nz) * nz
    Z, Y, X = np.meshgrid(kz, ky, kx, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def nyquist(shape):
    """Modes (grid linear order) with a Nyquist component on an even axis."""
    nx, ny, nz = shape
    xi = wave_vectors(shape)
    m = np.zeros(xi.shape[0], dtype=bool)
    for c, n in enumerate((nx, ny, nz)):
        if n % 2 == 0:
            m |= xi[:, c] == -(n // 2)
    return m


def solve(shape, grain, quat, Cc, E, eps_p=None, lam0=None, mu0=None, tol=1e-10, max_iter=500):
    """Strain and stress fields (sample frame, Voigt [N, 6]) of the periodic grid
    shape = (nx, ny, nz) under mean strain E (Voigt 6) with plastic strain eps_p
    (crystal frame, Voigt [N, 6], or None); returns (eps, sigma, iterations,
    last relative change)."""
    nx, ny, nz = shape
    N = nx * ny * nz
    grain = np.asarray(grain, dtype=np.int64).ravel()
    R = rotations(quat)[grain]
    Ep = tensor(np.asarray(E, dtype=np.float64)[None, :])[0]
    epc = np.zeros((N, 3, 3)) if eps_p is None else tensor(eps_p)
    if lam0 is None or mu0 is None:
        lam0, mu0 = reference_medium(Cc)
    xi = wave_vectors(shape)
    nyq = nyquist(shape)
    eps = np.broadcast_to(Ep, (N, 3, 3)).copy()
    scale = max(np.abs(Ep).max(), 1e-300)
    it, change = 0, np.inf
    sig = None
    for it in range(1, max_iter + 1):
        ec = np.einsum("pki,pkl,plj->pij", R, eps, R)               # R^T eps R
        sc = cubic_stress(Cc, ec - epc)
        sig = np.einsum("pik,pkl,pjl->pij", R, sc, R)               # R sigma_c R^T
        tr = np.trace(eps, axis1=1, axis2=2)
        tau = sig - 2.0 * mu0 * eps
        for i in range(3):
            tau[:, i, i] -= lam0 * tr
        th = np.fft.fftn(tau.reshape(nz, ny, nx, 3, 3), axes=(0, 1, 2)).reshape(N, 3, 3)
        eh = green_apply(th, xi, lam0, mu0)
        eh[nyq] = 0.0
        eh[0] = Ep * N
        new = np.fft.ifftn(eh.reshape(nz, ny, nx, 3, 3), axes=(0, 1, 2)).real.reshape(N, 3, 3)
        change = np.abs(new - eps).max() / scale
        eps = new
        if change < tol:
            break
    ec = np.einsum("pki,pkl,plj->pij", R, eps, R)
    sig = np.einsum("pik,pkl,pjl->pij", R, cubic_stress(Cc, ec - epc), R)
    return voigt(eps), voigt(sig), it, change


def equilibrium_residual(shape, sigma):
    """max over xi != 0 off the Nyquist planes of |xi . sigma^hat(xi)| / (|xi|
    max|<sigma>| N): zero at equilibrium."""
    nx, ny, nz = shape
    N = nx * ny * nz
    s = tensor(sigma)
    sh = np.fft.fftn(s.reshape(nz, ny, nx, 3, 3), axes=(0, 1, 2)).reshape(N, 3, 3)
    xi = wave_vectors(shape)
    nrm = np.linalg.norm(xi, axis=1)
    d = np.einsum("pij,pj->pi", sh, xi)
    ok = (nrm > 0) & ~nyquist(shape)
    r = np.abs(d[ok]).max(axis=1) / nrm[ok]
    return float(r.max() / (np.abs(s.mean(axis=0)).max() * N))
