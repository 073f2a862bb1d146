"""Reference training samples of the field surrogate (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Each sample follows Sec. 2: an orientation is driven through Taylor load
increments (Eq. (3)) by the Monte Carlo crystal plasticity of the C oracle in
K stochastic histories; after increment t the sample holds the orientation,
the population-average sample-frame stress R sigma R^T and slip, and the
K-history averages of the elastic energy density and of E_rho (Eq. (4)).
Rotations come from scipy (quaternion (w,x,y,z) -> matrix).  The orientation
enters the samples through four cubic invariants of the loading axis
d = R^T e_x (|d| sorted decreasingly, and d1^2 d2^2 + d2^2 d3^2 + d3^2 d1^2):
under the axisymmetric Taylor strain of Eq. (3) only d, modulo the cubic
symmetry of the crystal, affects the response.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation

import oracle


def orientation_features(quat):
    """Four cubic invariants of the loading axis d = R(q)^T e_x, one row per
    quaternion (w, x, y, z): |d| sorted decreasingly and
    d1^2 d2^2 + d2^2 d3^2 + d3^2 d1^2.  Row 0 of R is R^T e_x."""
    q = np.asarray(quat, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    R = Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], axis=1)).as_matrix()
    a = -np.sort(-np.abs(R[:, 0, :]), axis=1)
    inv4 = (a[:, 0] * a[:, 1]) ** 2 + (a[:, 1] * a[:, 2]) ** 2 + (a[:, 2] * a[:, 0]) ** 2
    return np.concatenate([a, inv4[:, None]], axis=1)


def sample_frame_stress(R, sigma_crystal):
    """Crystal-frame stresses (Voigt order xx yy zz yz xz xy, [n, 6]) rotated
    into the sample frame, R sigma R^T ([n, 3, 3]); R [n, 3, 3] maps crystal
    vectors to sample vectors (the rotation of the orientation quaternion)."""
    sg = np.asarray(sigma_crystal, dtype=np.float64)
    S = np.zeros((sg.shape[0], 3, 3))
    S[:, 0, 0], S[:, 1, 1], S[:, 2, 2] = sg[:, 0], sg[:, 1], sg[:, 2]
    S[:, 1, 2] = S[:, 2, 1] = sg[:, 3]
    S[:, 0, 2] = S[:, 2, 0] = sg[:, 4]
    S[:, 0, 1] = S[:, 1, 0] = sg[:, 5]
    return np.einsum("pik,pkl,pjl->pij", R, S, R)


def samples(P, seed, quat, K, n_incr, scales):
    """Returns X [n_orient*n_incr, 11], Y [n_orient*n_incr, 2] (row o*n_incr + t-1),
    load [n_incr, 7], and a per-orientation near-tie flag (any history within
    1e-5 of a decision)."""
    quat = np.ascontiguousarray(quat, dtype=np.float32)
    n_orient = quat.shape[0]
    grain = np.repeat(np.arange(n_orient, dtype=np.int32), K)
    npts = grain.size
    ep = np.zeros((npts, 6))
    gm = np.zeros(npts)
    q64 = quat.astype(np.float64)
    q64 /= np.linalg.norm(q64, axis=1, keepdims=True)
    R = Rotation.from_quat(np.stack([q64[:, 1], q64[:, 2], q64[:, 3], q64[:, 0]], axis=1)).as_matrix()[grain]
    X, Y, load = [], [], []
    near = np.zeros(n_orient, dtype=bool)
    for t in range(1, n_incr + 1):
        ep, gm, sg, nR, nT = oracle.mcp_run(P, seed, grain, quat, t - 1, 1, ep, gm)
        near |= ((nR < 1e-5) | (nT < 1e-5)).reshape(n_orient, K).any(axis=1)
        w, er = oracle.mcp_energies(P, sg, gm)
        Ss = sample_frame_stress(R, sg)
        sh = np.array([Ss[:, 0, 0].mean(), Ss[:, 1, 1].mean(), Ss[:, 2, 2].mean(), Ss[:, 1, 2].mean(),
                       Ss[:, 0, 2].mean(), Ss[:, 0, 1].mean()])
        gh = gm.mean()
        load.append(np.concatenate([sh, [gh]]))
        x = np.concatenate([orientation_features(quat), np.tile(sh / scales[0], (n_orient, 1)),
                            np.full((n_orient, 1), gh / scales[1])], axis=1)
        y = np.stack([w.reshape(n_orient, K).mean(1) / scales[2], er.reshape(n_orient, K).mean(1) / scales[3]], axis=1)
        X.append(x)
        Y.append(y)
    X = np.stack(X, axis=1).reshape(n_orient * n_incr, 11)
    Y = np.stack(Y, axis=1).reshape(n_orient * n_incr, 2)
    return X, Y, np.array(load), near
