"""Fixtures the paper prints (tests/golden/paper_numbers.json, each entry cited)."""
import json
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))

G_CGS = 6.67430e-8
MSUN = 1.98841e33
RSUN = 6.957e10


def test_table1_code_units_imply_G_is_one_over_4pi():
    """Table 1's code units (M0 = 1 Msun, L0 = 2 Rsun, t0 = 1270.9 s) make
    G = 1/(4 pi) in code units, and v0 = L0/t0, rho0 = M0/L0^3."""
    u = GOLD["code_units"]
    M0, L0, t0 = u["M0_Msun"] * MSUN, u["L0_Rsun"] * RSUN, u["t0_s"]
    assert G_CGS * M0 * t0 ** 2 / L0 ** 3 == pytest.approx(1 / (4 * np.pi), rel=1e-3)
    assert L0 / t0 == pytest.approx(u["v0_cm_s"], rel=1e-3)
    assert M0 / L0 ** 3 == pytest.approx(u["rho0_g_cm3"], rel=1e-3)


def test_entropy_wave_mach_number_matches_paper_setup():
    """Sec. 6.3: V_adv = 1e8 at Mach 7.75e7 means c_s = 1.29 = sqrt(5/3) for
    rho = P = 1 (the setup the oracle pin uses)."""
    d = GOLD["dual_energy"]
    assert d["entropy_wave_vadv"] / np.sqrt(5.0 / 3.0) == pytest.approx(d["entropy_wave_mach"], rel=1e-3)


def test_oracle_beats_paper_dual_energy_bound(oracle):
    """Our dual-energy pressure error is at or below the paper's 4.0e-12 scale and
    conservation at the paper's 6.0e-16 scale (same test, Sec. 6.3)."""
    from test_oracle_hydro import entropy_wave_run
    dP, dE, _ = entropy_wave_run(oracle, 1)
    d = GOLD["dual_energy"]
    assert dP < 25 * d["dP_inf_with"]
    assert dE < 10 * d["energy_conservation"]
    dP_off, _, _ = entropy_wave_run(oracle, 0)
    assert dP_off > 0.05 * d["dP_inf_without"]
