"""GPU parity of the periodic elastic-equilibrium solve (FP32 FFT fixed point)
against the FP64 oracle, and of the plasticity increment driven by the solved
per-point strain (Sec. 5: the plasticity coupled to a deformation solver)."""
import numpy as np
import pytest

from paper_1007_3509_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

C = synth.TABLE1
E0 = np.array([1e-3, -5e-4, -5e-4, 0.0, 0.0, 0.0])   # Taylor-type load of Eq. (3)
E1 = np.array([8e-4, -3e-4, -6e-4, 2e-4, -1e-4, 3e-4])


def _prm(hm, e=1e-4):
    return hm.cp_params(C["C11"], C["C12"], C["C44"], C["tau0"], C["taus"], C["h0"], C["beta"], e)


def _case(shape, G, seed):
    N = int(np.prod(shape))
    rng = np.random.default_rng(seed)
    grain = rng.integers(0, G, size=N).astype(np.int32)
    q = rng.normal(size=(G, 4)).astype(np.float32)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    epc = (rng.normal(size=(N, 6)) * 2e-4).astype(np.float32)
    return grain, q, epc


@pytest.mark.parametrize("shape,G,E", [((32, 16, 8), 9, E0), ((16, 16, 16), 13, E1), ((8, 4, 64), 5, E1)])
def test_elastic_solve_matches_oracle(shape, G, E):
    torch, hm = need_gpu()
    from oracle import elastic
    grain, quat, epc = _case(shape, G, sum(shape))
    N = int(np.prod(shape))
    ref_e, ref_s, ref_it, _ = elastic.solve(shape, grain, quat, (C["C11"], C["C12"], C["C44"]), E,
                                            eps_p=epc.astype(np.float64), tol=1e-11)
    eps = torch.empty(6 * N, device="cuda")
    sig = torch.empty(6 * N, device="cuda")
    it, ch = hm.hp_elastic_solve(_prm(hm), shape, torch.from_numpy(grain).cuda(), torch.from_numpy(quat).cuda(), E,
                                 eps, eps_p=torch.from_numpy(np.ascontiguousarray(epc.T)).cuda(), sigma=sig,
                                 tol=1e-6)
    torch.cuda.synchronize()
    assert ch < 1e-6 and it < 100
    ge = eps.view(6, N).cpu().numpy().T
    gs = sig.view(6, N).cpu().numpy().T
    emax = np.abs(E).max()
    assert np.abs(ge - ref_e).max() <= 2e-5 * emax, np.abs(ge - ref_e).max() / emax
    assert np.abs(ge.mean(axis=0) - E).max() <= 1e-6 * emax
    smax = np.abs(ref_s).max()
    assert np.abs(gs - ref_s).max() <= 5e-5 * smax


def test_single_crystal_is_uniform():
    torch, hm = need_gpu()
    shape, N = (16, 8, 4), 512
    quat = torch.tensor([[0.9, 0.1, -0.3, 0.2]], device="cuda")
    grain = torch.zeros(N, dtype=torch.int32, device="cuda")
    eps = torch.empty(6 * N, device="cuda")
    it, ch = hm.hp_elastic_solve(_prm(hm), shape, grain, quat, E1, eps, tol=1e-6)
    torch.cuda.synchronize()
    assert it <= 2
    e = eps.view(6, N).cpu().numpy().T
    assert np.abs(e - E1).max() <= 1e-6 * np.abs(E1).max()


def test_plasticity_driven_by_the_solved_strain(oracle):
    """One solve then one strain-driven increment at a load past first yield; the
    oracle runs the same increment from the GPU's strain field.  Stress within
    1e-5 relative away from decision ties (as for the Taylor increment)."""
    torch, hm = need_gpu()
    shape, G = (32, 16, 16), 20
    N = int(np.prod(shape))
    grain, quat, _ = _case(shape, G, 3)
    prm = _prm(hm)
    t = 12                                            # 1.2e-3 strain: most grains yield
    E = np.array([t * 1e-4, -0.5 * t * 1e-4, -0.5 * t * 1e-4, 0, 0, 0])
    tg, tq = torch.from_numpy(grain).cuda(), torch.from_numpy(quat).cuda()
    eps = torch.empty(6 * N, device="cuda")
    hm.hp_elastic_solve(prm, shape, tg, tq, E, eps, tol=1e-6)
    ep = torch.zeros(6 * N, device="cuda")
    gam = torch.zeros(N, device="cuda")
    g = torch.empty(N, device="cuda")
    hm.hp_cp_reset(prm, N, ep, gam, g)
    sig = torch.empty(6 * N, device="cuda")
    hm.hp_cp_step_strain(prm, 77, tg, tq, t, eps, ep, gam, g, sigma=sig)
    torch.cuda.synchronize()
    et = eps.view(6, N).cpu().numpy().T.astype(np.float64)
    Por = oracle.cp_params(C["C11"], C["C12"], C["C44"], C["tau0"], C["taus"], C["h0"], C["beta"], 1e-4)
    ref_ep, ref_gm, ref_s, nR, nT = oracle.mcp_run_strain(Por, 77, grain, quat, t, et, np.zeros((N, 6)), np.zeros(N))
    near = (nR < 1e-5) | (nT < 1e-5)
    assert near.mean() < 0.02
    ok = ~near
    s = sig.view(6, N).cpu().numpy().T
    rel = np.linalg.norm(s - ref_s, axis=1) / np.maximum(np.linalg.norm(ref_s, axis=1), 1e-30)
    assert rel[ok].max() <= 1e-5, rel[ok].max()
    gm = gam.cpu().numpy()
    np.testing.assert_allclose(gm[ok], ref_gm[ok], rtol=1e-5, atol=1e-9)
    assert (ref_gm > 0).mean() > 0.5                 # the load reached the plastic range
    # the strain field is heterogeneous: points of one orientation see different strains
    assert np.abs(et - E).max() > 0.05 * np.abs(E).max()


def test_elastic_at_the_bench_size_properties():
    """The equilibrium workload's grid (256^3 voxels, 15625 Voronoi grains, Taylor
    mean strain 1e-3): the solution keeps the prescribed mean strain, satisfies
    div sigma = 0 (the stress's Fourier transform orthogonal to every wave
    vector off the Nyquist planes, relative to the mean stress), and varies from
    grain to grain."""
    torch, hm = need_gpu()
    e = 256
    shape, N, G = (e, e, e), e ** 3, 15625
    lat = hm.Lattice(3, shape, 26, 256, 1002, G, hm.FIELD_NONE)
    q = torch.empty(N, dtype=torch.int32, device="cuda")
    lat.hp_bind(q)
    quat = torch.empty(G, 4, device="cuda")
    lat.hp_init_voronoi(hm.ORIENT_SO3, quat)
    E = np.array([1e-3, -5e-4, -5e-4, 0.0, 0.0, 0.0])
    eps = torch.empty(6 * N, device="cuda")
    sig = torch.empty(6 * N, device="cuda")
    it, ch = hm.hp_elastic_solve(_prm(hm), shape, q, quat, E, eps, sigma=sig, tol=1e-5)
    torch.cuda.synchronize()
    assert it < 100 and ch < 1e-5
    ev = eps.view(6, N).double()
    assert (ev.mean(dim=1).cpu().numpy() - E).__abs__().max() <= 1e-6 * np.abs(E).max()
    sv = sig.view(6, e, e, e)  # [component][z][y][x]
    fi = torch.fft.fftfreq(e, device="cuda") * e
    kz, ky, kx = torch.meshgrid(fi, fi, fi, indexing="ij")
    full = [[0, 5, 4], [5, 1, 3], [4, 3, 2]]
    sh = [torch.fft.fftn(sv[c].to(torch.float64)) for c in range(6)]
    k = (kx, ky, kz)
    res = torch.zeros((e, e, e), dtype=torch.float64, device="cuda")
    for i in range(3):
        d = sum(sh[full[i][j]] * k[j] for j in range(3))
        res = torch.maximum(res, d.abs())
    nrm = torch.sqrt(kx * kx + ky * ky + kz * kz)
    nyq = (kx == -e // 2) | (ky == -e // 2) | (kz == -e // 2)
    ok = (nrm > 0) & ~nyq
    mean_s = sv.double().mean(dim=(1, 2, 3)).abs().max()
    r = float((res[ok] / nrm[ok]).max() / (mean_s * N))
    print(f"256^3 equilibrium residual {r:.2e} after {it} iterations")
    assert r <= 1e-5  # a converged solve leaves FP32 rounding (about 5e-8 measured)
    # stress heterogeneity: the sample-frame sigma_xx spreads well beyond rounding
    sxx = sv[0].flatten()
    assert float(sxx.std() / sxx.mean().abs()) > 0.05
    lat.close()
