"""Texture experiments of Sec. 5 on the GPU (statistical direction checks; the
kernels they use are bit-exact against the oracle in the other GPU tests)."""
import numpy as np
import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_gaussian_field_matches_oracle(oracle):
    torch, hm = need_gpu()
    ang = oracle.orientations(20000, 5, 0)
    b = torch.empty(20000, dtype=torch.int32, device="cuda")
    hm.hp_gaussian_field(20000, torch.from_numpy(ang).cuda(), 1.0, b)
    e, rb = oracle.gaussian_field(ang)
    _, near = oracle.grain_bins(ang, 0)
    ok = near > 1e-9
    np.testing.assert_array_equal(b.cpu().numpy()[ok], rb[ok])


def test_gaussian_bulk_energy_texture_2d():
    """Eq. (9), Fig. 3: lower bulk energy is favoured -- the volume-weighted bulk energy
    falls and the lowest-energy orientations gain volume."""
    torch, hm = need_gpu()
    from paper_1007_3509_gb300 import texture
    r = texture.run_gaussian_2d(torch, R=8, L=(256, 256), G=600, kT=1.0, slices=(0, 100, 400))
    assert r["mean_b"][2] < r["mean_b"][0]
    h0, h2 = r["hist"][0], r["hist"][-1]
    low = list(range(0, 10)) + list(range(80, 90))
    assert h2[low].sum() / h2.sum() > h0[low].sum() / h0.sum()
    assert all(abs(h.sum() - 8 * 256 * 256) == 0 for h in r["hist"])


def test_plastic_texture_sharpens_3d():
    """Figs. 5 and 7: under plastic loading (elastic driving suppressed) the angle
    distribution concentrates and the fitted Gaussian width g(t) of Eq. (10) falls."""
    torch, hm = need_gpu()
    from paper_1007_3509_gb300 import texture
    r = texture.run_plastic_3d(torch, L=(96, 96, 96), G=2000, kT=1.0, n_incr=100, mcs_per_incr=2, e_incr=1e-4,
                               energy_scale=200.0, every=25)
    g = np.array(r["g"])
    assert g[-1] < 0.9 * g[0], g
    assert all(abs(h.sum() - 96 ** 3) == 0 for h in r["hist"])
