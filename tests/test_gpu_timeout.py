"""The bounded device waits give up cleanly: a probe block whose mbarrier wait
has nothing to complete (no copy, no tensor-core operation in flight) runs out
after a short limit, the host reads HP_ERR_TIMEOUT through hp_sweep_status /
hp_mlp_status, the flag is cleared by that read, and the same context still
sweeps bit-exactly and evaluates the network afterwards.  No GPU fault or hang
is involved: the wait ends by its own clock limit."""
import ctypes as C

import numpy as np
import pytest

from paper_1007_3509_gb300 import synth
from tests.gpu_util import need_gpu, run_gpu_sweep

pytestmark = pytest.mark.gpu

LIMIT = 2_000_000  # SM clock cycles, about a millisecond


def _status(hm, fn):
    v = C.c_int32(-1)
    rc = fn(C.byref(v))
    return rc, v.value


def test_sweep_wait_timeout_is_reported_and_context_survives(oracle):
    torch, hm = need_gpu()
    rc, v = _status(hm, hm.lib().hp_sweep_status)
    assert rc == hm.HP_OK and v == 0
    hm.hp_debug_wait_timeout(0, LIMIT, late=True)
    torch.cuda.synchronize()
    rc, v = _status(hm, hm.lib().hp_sweep_status)
    assert rc == hm.HP_ERR_TIMEOUT and v == 1  # gave up, and the drain saw the late arrival
    rc, v = _status(hm, hm.lib().hp_sweep_status)
    assert rc == hm.HP_OK and v == 0           # the read cleared the flag
    hm.hp_debug_wait_timeout(0, LIMIT, late=False)
    torch.cuda.synchronize()
    assert _status(hm, hm.lib().hp_sweep_status) == (hm.HP_ERR_TIMEOUT, 2)  # the drain ran out too
    # the context still runs the TMA-fed sweeps bit-exactly
    L, Q = (70, 40, 12), 7
    q0 = synth.blocky_lattice(L, Q, 4, block=3)
    bg = np.random.default_rng(2).integers(-50, 50, size=Q).astype(np.int32)
    thr, D = oracle.threshold_table(0.7)
    ref_q, _, _, _ = oracle.sweep(3, L, 26, 256, 99, 0, 2, thr, D, q0, bg[q0], None)
    for variant in (7, 8):  # a lean tile and a lean 3D window
        q, _ = run_gpu_sweep(torch, hm, 3, L, 26, 256, 99, 2, 0.7, q0, hm.FIELD_GRAIN, bg, None, kernel=2,
                             variant=variant)
        np.testing.assert_array_equal(q, ref_q)
    assert _status(hm, hm.lib().hp_sweep_status) == (hm.HP_OK, 0)


def test_surrogate_wait_timeout_is_reported_and_context_survives():
    torch, hm = need_gpu()
    assert _status(hm, hm.lib().hp_mlp_status) == (hm.HP_OK, 0)
    P = hm.hp_mlp_param_count()
    params = torch.from_numpy(np.concatenate([p.ravel() for p in synth.mlp_init(5)]).astype(np.float32)).cuda()
    assert params.numel() == P
    X = torch.randn(300, 11, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    Y0 = torch.empty(300, 2, device="cuda")
    hm.hp_mlp_forward(params, X, Y0)
    hm.hp_debug_wait_timeout(1, LIMIT, late=True)
    torch.cuda.synchronize()
    assert _status(hm, hm.lib().hp_mlp_status) == (hm.HP_ERR_TIMEOUT, 1)
    assert _status(hm, hm.lib().hp_mlp_status) == (hm.HP_OK, 0)
    hm.hp_debug_wait_timeout(1, LIMIT, late=False)
    torch.cuda.synchronize()
    assert _status(hm, hm.lib().hp_mlp_status) == (hm.HP_ERR_TIMEOUT, 2)
    Y1 = torch.empty(300, 2, device="cuda")
    hm.hp_mlp_forward(params, X, Y1)
    torch.cuda.synchronize()
    assert torch.equal(Y0, Y1)
    assert _status(hm, hm.lib().hp_mlp_status) == (hm.HP_OK, 0)


def test_wait_probe_rejects_bad_limits():
    torch, hm = need_gpu()
    for unit, limit in ((0, 0), (1, -5), (0, 1 << 40), (2, 1000)):
        with pytest.raises(hm.HPError) as e:
            hm.hp_debug_wait_timeout(unit, limit)
        assert e.value.code == hm.HP_ERR_ARG
