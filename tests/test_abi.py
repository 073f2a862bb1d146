"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/hmcpotts.h declares, and its host-side threshold table builder agrees
bit for bit with the oracle's (both are FP64 libm on the same host)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "hmcpotts.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hp_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def hm():
    from paper_1007_3509_gb300 import build, hmcpotts
    build.build()
    return hmcpotts


def test_library_exports_every_declared_symbol(hm):
    L = hm.lib()
    decl = _declared()
    assert len(decl) >= 20
    missing = [s for s in decl if not hasattr(L, s)]
    assert not missing, missing
    # the binding covers the whole header
    assert set(decl) <= set(hm.exported_symbols()), set(decl) - set(hm.exported_symbols())
    assert "sm_103a" in hm.version()


@pytest.mark.parametrize("kT,zero_rule", [(0.0, 0), (0.5, 0), (0.6, 1), (0.7, 0), (0.9, 0), (2.6, 1)])
def test_threshold_table_matches_oracle(hm, oracle, kT, zero_rule):
    t_lib, D_lib = hm.hp_build_threshold_table(kT, zero_rule)
    t_or, D_or = oracle.threshold_table(kT, zero_rule)
    assert D_lib == D_or
    np.testing.assert_array_equal(t_lib, t_or)


def test_bad_arguments_are_rejected(hm):
    with pytest.raises(hm.HPError) as e:
        hm.Lattice(2, (7, 8), 8, 256, 1, 4)
    assert e.value.code == hm.HP_ERR_ARG
    with pytest.raises(hm.HPError):
        hm.Lattice(2, (8, 8), 6, 256, 1, 4)
    with pytest.raises(hm.HPError):
        hm.hp_build_threshold_table(0.9, 0, cap=16)
    lat = hm.Lattice(2, (8, 8), 8, 256, 1, 4)
    with pytest.raises(hm.HPError) as e:
        lat.hp_sweep(1, stream=0)
    assert e.value.code == hm.HP_ERR_STATE


def test_last_error_copies_the_message(hm):
    with pytest.raises(hm.HPError):
        hm.Lattice(2, (7, 8), 8, 256, 1, 4)
    msg = hm.hp_last_error()
    assert "even" in msg
    import ctypes as C
    buf = C.create_string_buffer(6)
    assert hm.lib().hp_last_error(None, buf, 6) == hm.HP_OK
    assert buf.value.decode() == msg[:5]
    assert hm.lib().hp_last_error(None, None, 8) == hm.HP_ERR_ARG


def test_state_and_argument_errors_of_io_and_measure(hm):
    """Calls on a handle with nothing bound fail before touching the device."""
    lat = hm.Lattice(2, (8, 8), 8, 256, 1, 4)
    q = np.zeros(64, dtype=np.int32)
    with pytest.raises(hm.HPError) as e:
        lat.hp_set_spins(q, stream=0)
    assert e.value.code == hm.HP_ERR_STATE
    with pytest.raises(hm.HPError) as e:
        lat.hp_get_spins(q, stream=0)
    assert e.value.code == hm.HP_ERR_STATE
    with pytest.raises(hm.HPError) as e:
        lat.hp_measure(stream=0)
    assert e.value.code == hm.HP_ERR_STATE
    # the binding refuses short or mistyped host buffers
    with pytest.raises(hm.HPError) as e:
        lat.hp_set_spins(np.zeros(63, dtype=np.int32), stream=0)
    assert e.value.code == hm.HP_ERR_ARG
    with pytest.raises(hm.HPError):
        lat.hp_set_spins(np.zeros(64, dtype=np.int64), stream=0)
    assert hm.lib().hp_measure(None, 0, None, 0, None, None, 0, None) == hm.HP_ERR_ARG


def test_sur_train_argument_errors(hm):
    """hp_sur_train validates its schedule before any device work."""
    import ctypes as C
    tp = hm.hp_sur_train_params(10, 0, 0, 1e-3, 0.02, 0.9, 0.999, 1e-8, 0)  # group 0
    dummy = C.c_void_p(16)
    rc = hm.lib().hp_sur_train(dummy, dummy, dummy, dummy, dummy, 100, C.byref(tp), 0, None, None, None)
    assert rc == hm.HP_ERR_ARG
    tp = hm.hp_sur_train_params(10, 0, 1, 1e-3, 1.5, 0.9, 0.999, 1e-8, 0)  # floor above 1
    assert hm.lib().hp_sur_train(dummy, dummy, dummy, dummy, dummy, 100, C.byref(tp), 0, None, None, None) == \
        hm.HP_ERR_ARG
    tp = hm.hp_sur_train_params(10, 0, 1, 1e-3, 0.02, 0.9, 0.999, 1e-8, 5)  # a log without a host array
    assert hm.lib().hp_sur_train(dummy, dummy, dummy, dummy, dummy, 100, C.byref(tp), 0, None, None, None) == \
        hm.HP_ERR_ARG


def test_read_shockley_table_matches_oracle(hm, oracle):
    for args in [(1.0, 15.0, 250, 181, 1000), (2.5, 10.0, 1000, 46, 1000), (0.7, 20.0, 100, 451, 1000)]:
        J, m = hm.hp_build_read_shockley(*args, mobility=True)
        rJ, rm = oracle.read_shockley(*args, mobility=True)
        np.testing.assert_array_equal(J, rJ)
        np.testing.assert_array_equal(m, rm)


def test_si_links_invert_eq8(hm):
    """The three links of Eq. (8) hold with the returned E0, t0 and b conversion;
    choosing the physical mobility that makes one MCS last 10 minutes (Sec. 5)
    gives back 600 s."""
    gamma_s, m_s, l0, gamma_mc, m_mc, Delta, J, tau = 0.9, 3e-14, 2e-7, 0.7, 0.45, 1.0, 1.0, 1.0
    r = hm.hp_si_links(gamma_s, m_s, l0, gamma_mc, m_mc, Delta, J, tau)
    E0, t0 = r["E0"], r["t0"]
    assert abs(gamma_mc * E0 / (Delta ** 2 * J * l0 ** 2) - gamma_s) <= 1e-12 * gamma_s
    assert abs(Delta ** 4 * m_mc * l0 ** 4 / (J * tau * E0 * t0) - m_s) <= 1e-12 * m_s
    b_s = 5e5  # J/m^3
    b = r["b_per_bs"] * b_s
    assert abs(2 * b * E0 / (Delta ** 3 * l0 ** 3) - b_s) <= 1e-12 * b_s
    m10 = Delta ** 4 * m_mc * l0 ** 4 / (J * tau * E0 * 600.0)
    assert abs(hm.hp_si_links(gamma_s, m10, l0, gamma_mc, m_mc, Delta, J, tau)["seconds_per_mcs"] - 600.0) < 1e-9
    with pytest.raises(hm.HPError):
        hm.hp_si_links(0.0, m_s, l0, gamma_mc, m_mc)


def test_det_argument_errors(hm):
    """The deterministic comparator validates its arguments before any device work."""
    import ctypes as C
    T = dict(C11=250.8e3, C12=150.0e3, C44=123.5e3, tau0=8.0, taus=122.0, h0=440.0, beta=1000.0)
    prm = hm.cp_params(T["C11"], T["C12"], T["C44"], T["tau0"], T["taus"], T["h0"], T["beta"], 1e-6)
    dummy = C.c_void_p(16)
    st = hm.hp_det_state(0, dummy, dummy)  # no points
    assert hm.lib().hp_det_step(C.byref(prm), dummy, dummy, 0, 1, C.byref(st), None, None, None) == hm.HP_ERR_ARG
    st = hm.hp_det_state(4, None, dummy)  # no plastic-strain buffer
    assert hm.lib().hp_det_step(C.byref(prm), dummy, dummy, 0, 1, C.byref(st), None, None, None) == hm.HP_ERR_ARG
    assert hm.lib().hp_det_reset(C.byref(st), None) == hm.HP_ERR_ARG
    st = hm.hp_det_state(4, dummy, dummy)
    assert hm.lib().hp_det_step(C.byref(prm), dummy, dummy, 0, -1, C.byref(st), None, None, None) == hm.HP_ERR_ARG
    bad = hm.cp_params(T["C12"], T["C11"], T["C44"], T["tau0"], T["taus"], T["h0"], T["beta"], 1e-6)  # C11 < C12
    assert hm.lib().hp_det_step(C.byref(bad), dummy, dummy, 0, 1, C.byref(st), None, None, None) == hm.HP_ERR_ARG
    assert hm.lib().hp_det_step_strain(C.byref(prm), dummy, dummy, None, C.byref(st), None, None, None) == \
        hm.HP_ERR_ARG
