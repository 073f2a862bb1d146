"""Printed values of the paper, as cited fixtures under tests/golden/ (CPU only).

Each fixture file carries its citation in its header.  These tests check the
constants the oracle and the library are driven with against those printed
values, so a mistyped digit or a unit slip (GPa against MPa) fails here."""
import os

import pytest

from paper_1007_3509_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TO_MPA = {"GPa": 1e3, "MPa": 1.0, "1": 1.0}


def _table(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                key, value, unit = line
                out[key] = float(value) * TO_MPA[unit]
    return out


def test_table1_constants_drive_the_plasticity():
    t1 = _table("table1_nickel.txt")
    assert set(t1) == {"C11", "C12", "C44", "tau0", "taus", "h0", "beta"}
    for k, v in t1.items():
        assert synth.TABLE1[k] == pytest.approx(v, rel=1e-12), k


def test_table1_reaches_the_library_parameters():
    from paper_1007_3509_gb300 import hybrid
    t1 = _table("table1_nickel.txt")
    prm = hybrid.cp_params_table1(1e-4, 7.0)
    for k, v in t1.items():
        assert getattr(prm, k) == pytest.approx(v, rel=1e-12), k
    # shear modulus of Eq. (4): the Voigt average of the printed cubic constants
    assert prm.G == pytest.approx((t1["C11"] - t1["C12"] + 3 * t1["C44"]) / 5, rel=1e-12)
