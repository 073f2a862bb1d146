"""GPU parity of the tensor-core surrogate kernels against the FP64 oracle.

The oracle runs on the same BF16-rounded weights and inputs; the kernels also
round hidden activations to BF16, so outputs and gradients agree to BF16
precision: <= 2e-2 relative (norm-wise) per tensor and cosine >= 0.999."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1007_3509_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def bf16(a):
    import torch
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _params(seed):
    p = synth.mlp_init(seed)
    rng = np.random.default_rng(seed + 1)
    for b in p[1::2]:
        b += rng.normal(0, 0.2, size=b.shape)
    return p


def _flat(p):
    return np.concatenate([x.ravel() for x in p]).astype(np.float32)


def _unflat(v, like):
    out, o = [], 0
    for x in like:
        out.append(v[o:o + x.size].reshape(x.shape).astype(np.float64))
        o += x.size
    return out


def _close(a, b, rel=2e-2, cos=0.999):
    a = np.ravel(a).astype(np.float64)
    b = np.ravel(b).astype(np.float64)
    r = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
    c = a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
    assert r <= rel and c >= cos, (r, c)


@pytest.mark.parametrize("M", [1, 127, 1000, 40_000])
def test_forward_matches_oracle(M):
    torch, hm = need_gpu()
    assert hm.hp_mlp_param_count() == sum(x.size for x in _params(0))
    p = _params(3)
    X = np.random.default_rng(4).normal(size=(M, 11)).astype(np.float32)
    tp = torch.from_numpy(_flat(p)).cuda()
    tx = torch.from_numpy(X).cuda()
    ty = torch.empty(M, 2, dtype=torch.float32, device="cuda")
    hm.hp_mlp_forward(tp, tx, ty)
    torch.cuda.synchronize()
    assert hm.hp_mlp_status() == 0
    pb = [bf16(x) if i % 2 == 0 else x for i, x in enumerate(p)]
    ref, _ = omlp.forward(pb, bf16(X))
    _close(ty.cpu().numpy(), ref)


@pytest.mark.parametrize("M", [128, 777, 40_000])
def test_gradients_match_oracle(M):
    torch, hm = need_gpu()
    p = _params(5)
    rng = np.random.default_rng(6)
    X = rng.normal(size=(M, 11)).astype(np.float32)
    T = rng.normal(size=(M, 2)).astype(np.float32)
    tp = torch.from_numpy(_flat(p)).cuda()
    g = torch.empty_like(tp)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hm.hp_mlp_gradients(tp, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), g, loss)
    torch.cuda.synchronize()
    assert hm.hp_mlp_status() == 0
    pb = [bf16(x) if i % 2 == 0 else x for i, x in enumerate(p)]
    L_ref, g_ref = omlp.loss_and_grads(pb, bf16(X), T.astype(np.float64))
    assert abs(loss.item() - L_ref) <= 2e-2 * abs(L_ref)
    for k, (a, b) in enumerate(zip(_unflat(g.cpu().numpy(), p), g_ref)):
        _close(a, b), k


def test_adam_matches_oracle():
    torch, hm = need_gpu()
    p = _params(7)
    rng = np.random.default_rng(8)
    grads = [rng.normal(size=x.shape) for x in p]
    n = hm.hp_mlp_param_count()
    tp = torch.from_numpy(_flat(p)).cuda()
    tg = torch.from_numpy(_flat(grads)).cuda()
    m = torch.zeros(n, dtype=torch.float32, device="cuda")
    v = torch.zeros(n, dtype=torch.float32, device="cuda")
    pm, mm, vv = p, [np.zeros_like(x) for x in p], [np.zeros_like(x) for x in p]
    for t in range(1, 4):
        hm.hp_mlp_adam(tp, tg, m, v, t, 1e-3)
        pm, mm, vv = omlp.adam_step(pm, grads, mm, vv, t, 1e-3)
    torch.cuda.synchronize()
    np.testing.assert_allclose(tp.cpu().numpy(), _flat(pm), rtol=1e-5, atol=1e-6)


def test_training_reduces_loss():
    """Adam on the tensor-core gradients fits a smooth teacher function."""
    torch, hm = need_gpu()
    rng = np.random.default_rng(9)
    M = 16384
    X = rng.uniform(-1, 1, size=(M, 11)).astype(np.float32)
    T = np.stack([np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2], np.cos(X[:, 3]) * X[:, 4] - 0.5 * X[:, 5] ** 2],
                 axis=1).astype(np.float32)
    tp = torch.from_numpy(_flat(synth.mlp_init(10))).cuda()
    n = tp.numel()
    g = torch.empty_like(tp)
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    loss = torch.zeros(1, device="cuda")
    tx, tt = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    hist = []
    for step in range(1, 301):
        hm.hp_mlp_gradients(tp, tx, tt, g, loss)
        hm.hp_mlp_adam(tp, g, m, v, step, 3e-3)
        if step in (1, 300):
            torch.cuda.synchronize()
            hist.append(loss.item())
    assert hm.hp_mlp_status() == 0
    assert hist[1] < hist[0] / 10, hist


def test_activation_within_the_erf_approximation_bound():
    """The kernels' GELU and its derivative (erf by Abramowitz and Stegun 7.1.26,
    |error| <= 1.5e-7, with fast exp and reciprocal) against FP64 erf: within
    5e-7 (1 + |z|) for GELU and 5e-7 for the derivative over [-30, 30]."""
    import math
    torch, hm = need_gpu()
    z = np.concatenate([np.linspace(-10, 10, 200001), [-30.0, -12.0, -1e-30, 0.0, 1e-30, 12.0, 30.0]]).astype(np.float32)
    tz = torch.from_numpy(z).cuda()
    g = torch.empty_like(tz)
    dg = torch.empty_like(tz)
    hm.hp_debug_gelu(tz, g, dg)
    torch.cuda.synchronize()
    zd = z.astype(np.float64)
    cdf = np.array([0.5 * (1.0 + math.erf(v / math.sqrt(2.0))) for v in zd])
    pdf = np.exp(-0.5 * zd * zd) / math.sqrt(2.0 * math.pi)
    eg = np.abs(g.cpu().numpy() - zd * cdf)
    ed = np.abs(dg.cpu().numpy() - (cdf + zd * pdf))
    assert np.all(eg <= 5e-7 * (1.0 + np.abs(zd))), eg.max()
    assert np.all(ed <= 5e-7), ed.max()
