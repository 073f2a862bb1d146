"""Pins of the surrogate's reference data (``oracle/surrogate.py``), CPU only.

Two functions feed every surrogate parity claim: the orientation encoding
(four cubic invariants of the loading axis d = R^T e_x) and the sample-frame
stress R sigma R^T averaged over the population.  Both are fixed by the
mathematics, independently of the code:

* the loading axis seen from the crystal does not change when the crystal is
  replaced by a symmetry-equivalent one (R -> R S, S one of the 24 proper
  rotations of the cube), and takes known values on <100>, <110>, <111>;
* in the elastic range (Sec. 2: no slip below the critical resolved shear
  stress) the crystal stress is C : (R^T eps R) and so the sample-frame stress
  is the cubic stiffness rotated into the sample frame, C'_ijkl =
  R_ia R_jb R_kc R_ld C_abcd, applied to the Taylor strain e diag(1, -1/2, -1/2)
  of Eq. (3).

Rotations here come from quaternion products (q v q*), not from scipy or the
C oracle, and a planted mistake (the column R e_x instead of the row R^T e_x,
or R^T sigma R instead of R sigma R^T) must fail each pin.
"""
import itertools

import numpy as np
import pytest

from paper_1007_3509_gb300 import synth


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _rotate(q, v):
    """Active rotation of vector v by unit quaternion q = (w, x, y, z): q v q*."""
    q = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    qc = q * np.array([1.0, -1.0, -1.0, -1.0])
    return _qmul(_qmul(q, np.concatenate([[0.0], v])), qc)[1:]


def _matrix(q):
    """R with columns = images of the crystal axes (crystal -> sample)."""
    return np.stack([_rotate(q, e) for e in np.eye(3)], axis=1)


def _quat_taking(d, target=(1.0, 0.0, 0.0)):
    """Unit quaternion of the rotation that takes unit vector d onto target
    (axis d x target, angle between them)."""
    d = np.asarray(d, dtype=np.float64) / np.linalg.norm(d)
    t = np.asarray(target, dtype=np.float64)
    ax = np.cross(d, t)
    s = np.linalg.norm(ax)
    if s < 1e-15:
        return np.array([1.0, 0.0, 0.0, 0.0])
    ang = np.arctan2(s, float(d @ t))
    return np.concatenate([[np.cos(ang / 2)], np.sin(ang / 2) * ax / s])


def _cube_rotations():
    """The 24 proper rotations of the cube: signed permutation matrices of det +1."""
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1.0, -1.0), repeat=3):
            S = np.zeros((3, 3))
            for i, j in enumerate(perm):
                S[i, j] = signs[i]
            if np.linalg.det(S) > 0:
                out.append(S)
    assert len(out) == 24
    return out


def _quat_of(R):
    """Quaternion (w, x, y, z) of a proper rotation matrix (Shepperd's branch choice)."""
    tr = np.trace(R)
    cands = [1 + tr, 1 + 2 * R[0, 0] - tr, 1 + 2 * R[1, 1] - tr, 1 + 2 * R[2, 2] - tr]
    k = int(np.argmax(cands))
    if k == 0:
        w = np.sqrt(cands[0]) / 2
        q = [w, (R[2, 1] - R[1, 2]) / (4 * w), (R[0, 2] - R[2, 0]) / (4 * w), (R[1, 0] - R[0, 1]) / (4 * w)]
    elif k == 1:
        x = np.sqrt(cands[1]) / 2
        q = [(R[2, 1] - R[1, 2]) / (4 * x), x, (R[0, 1] + R[1, 0]) / (4 * x), (R[0, 2] + R[2, 0]) / (4 * x)]
    elif k == 2:
        y = np.sqrt(cands[2]) / 2
        q = [(R[0, 2] - R[2, 0]) / (4 * y), (R[0, 1] + R[1, 0]) / (4 * y), y, (R[1, 2] + R[2, 1]) / (4 * y)]
    else:
        z = np.sqrt(cands[3]) / 2
        q = [(R[1, 0] - R[0, 1]) / (4 * z), (R[0, 2] + R[2, 0]) / (4 * z), (R[1, 2] + R[2, 1]) / (4 * z), z]
    return np.array(q)


def _column_features(quat):
    """Planted mistake: the same invariants of the column R e_x (the sample
    image of the crystal x axis) instead of the row R^T e_x."""
    from scipy.spatial.transform import Rotation
    q = np.asarray(quat, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    R = Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], axis=1)).as_matrix()
    a = -np.sort(-np.abs(R[:, :, 0]), axis=1)
    inv4 = (a[:, 0] * a[:, 1]) ** 2 + (a[:, 1] * a[:, 2]) ** 2 + (a[:, 2] * a[:, 0]) ** 2
    return np.concatenate([a, inv4[:, None]], axis=1)


def _max_symmetry_spread(features):
    """Largest change of the features over the 24 symmetry-equivalent copies
    R S of 40 random orientations."""
    rng = np.random.default_rng(11)
    q0 = rng.normal(size=(40, 4))
    q0 /= np.linalg.norm(q0, axis=1, keepdims=True)
    worst = 0.0
    for q in q0:
        R = _matrix(q)
        eq = np.stack([_quat_of(R @ S) for S in _cube_rotations()])
        f = features(eq)
        worst = max(worst, float(np.abs(f - f[0]).max()))
    return worst


def test_features_invariant_under_cube_symmetry():
    from oracle import surrogate as osur
    assert _max_symmetry_spread(osur.orientation_features) < 1e-12
    # the column of R is not a property of the crystal's symmetry class
    assert _max_symmetry_spread(_column_features) > 1e-2


@pytest.mark.parametrize("d,expect", [
    ((1, 0, 0), (1.0, 0.0, 0.0, 0.0)),
    ((0, 0, -1), (1.0, 0.0, 0.0, 0.0)),
    ((1, 1, 0), (2 ** -0.5, 2 ** -0.5, 0.0, 0.25)),
    ((0, -1, 1), (2 ** -0.5, 2 ** -0.5, 0.0, 0.25)),
    ((1, 1, 1), (3 ** -0.5, 3 ** -0.5, 3 ** -0.5, 1.0 / 3.0)),
    ((-1, 1, 1), (3 ** -0.5, 3 ** -0.5, 3 ** -0.5, 1.0 / 3.0)),
    ((1, 2, 3), (3 / 14 ** 0.5, 2 / 14 ** 0.5, 1 / 14 ** 0.5, 0.25)),
])
def test_features_exact_on_known_axes(d, expect):
    """An orientation whose rotation takes crystal direction d onto the sample
    loading axis x has loading axis d in the crystal frame."""
    from oracle import surrogate as osur
    q = _quat_taking(d)
    # a spin about x after the alignment leaves the loading axis unchanged
    spin = np.array([np.cos(0.35), np.sin(0.35), 0.0, 0.0])
    for qq in (q, _qmul(spin, q)):
        f = osur.orientation_features(qq[None, :])[0]
        assert np.allclose(f, expect, atol=1e-12), (d, f)


def _cubic_tensor(C11, C12, C44):
    """Cubic stiffness in the crystal frame from its three independent
    components: C_iiii = C11, C_iijj = C12 (i != j), C_ijij = C_ijji = C44 (i != j)."""
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            if i == j:
                C[i, i, i, i] = C11
            else:
                C[i, i, j, j] = C12
                C[i, j, i, j] = C44
                C[i, j, j, i] = C44
    return C


def _elastic_sample_stress(quats, e):
    c = synth.TABLE1
    C = _cubic_tensor(c["C11"], c["C12"], c["C44"])
    eps = np.diag([e, -0.5 * e, -0.5 * e])
    out = []
    for q in quats:
        R = _matrix(q)
        Cs = np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, C)
        out.append(np.einsum("ijkl,kl->ij", Cs, eps))
    return np.mean(out, axis=0)


def _load_of_samples(oracle, quat, e):
    from oracle import surrogate as osur
    c = synth.TABLE1
    P = oracle.cp_params(c["C11"], c["C12"], c["C44"], c["tau0"], c["taus"], c["h0"], c["beta"], e)
    _, _, load, _ = osur.samples(P, 5, quat, 3, 1, (1.0, 1.0, 1.0, 1.0))
    return load[0]


def test_sample_frame_stress_elastic_closed_form(oracle):
    """Taylor strain 1e-5 keeps every grain elastic (resolved shear below tau0 =
    8 MPa), so the population-average stress equals the rotated stiffness applied
    to e diag(1, -1/2, -1/2); components in the order xx yy zz yz xz xy."""
    rng = np.random.default_rng(4)
    quat = rng.normal(size=(12, 4)).astype(np.float32)
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    e = 1e-5
    ref = _elastic_sample_stress(quat.astype(np.float64), e)
    ref6 = np.array([ref[0, 0], ref[1, 1], ref[2, 2], ref[1, 2], ref[0, 2], ref[0, 1]])
    got = _load_of_samples(oracle, quat, e)
    scale = np.abs(ref6).max()
    assert np.abs(got[:6] - ref6).max() < 1e-9 * scale, (got[:6], ref6)
    assert got[6] == 0.0  # no slip in the elastic range
    # single orientations, one by one: shear components are nonzero for a general grain
    for q in quat[:3]:
        r = _elastic_sample_stress(q[None, :].astype(np.float64), e)
        g = _load_of_samples(oracle, q[None, :], e)
        r6 = np.array([r[0, 0], r[1, 1], r[2, 2], r[1, 2], r[0, 2], r[0, 1]])
        assert np.abs(g[:6] - r6).max() < 1e-9 * np.abs(r6).max()
        assert np.abs(r6[3:]).max() > 1e-3 * np.abs(r6).max()


def test_sample_frame_stress_transposed_rotation_fails(oracle, monkeypatch):
    """Planted mistake: R^T sigma R in place of R sigma R^T must break the pin."""
    from oracle import surrogate as osur
    right = osur.sample_frame_stress

    def transposed(R, sigma_crystal):
        return right(np.transpose(R, (0, 2, 1)), sigma_crystal)

    rng = np.random.default_rng(9)
    quat = rng.normal(size=(4, 4)).astype(np.float32)
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    e = 1e-5
    ref = _elastic_sample_stress(quat.astype(np.float64), e)
    ref6 = np.array([ref[0, 0], ref[1, 1], ref[2, 2], ref[1, 2], ref[0, 2], ref[0, 1]])
    monkeypatch.setattr(osur, "sample_frame_stress", transposed)
    got = _load_of_samples(oracle, quat, e)
    assert np.abs(got[:6] - ref6).max() > 1e-3 * np.abs(ref6).max()
