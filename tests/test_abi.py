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
