"""Pins of the oracle's Saha H/He equation of state and its table (Sec. 4.2).

Every expected value here comes from a closed form written in this file with
textbook constants, not from the oracle's own formulas.
"""
import numpy as np
import pytest

# textbook constants, typed independently of the oracle (eV-based)
K_EV = 8.617333262e-5        # Boltzmann constant, eV/K
SAHA_COEF = 2.4147e15        # (2 pi m_e k / h^2)^{3/2}, cm^-3 K^-3/2
AMU = 1.66053906660e-24
KB = 1.380649e-16
ARAD = 4 * 5.670374419e-5 / 2.99792458e10   # 4 sigma_SB / c (CODATA 2018)
CHI = (13.598434, 24.587389, 54.417765)
X, Y = 0.7, 0.3
AH, AHE = 1.00794, 4.002602


def saha_S(G, chi, T):
    return G * SAHA_COEF * T ** 1.5 * np.exp(-chi / (K_EV * T))


@pytest.mark.parametrize("rho,T", [(1e-8, 1.0e4), (1e-6, 1.2e4), (1e-10, 8e3), (1e-3, 2e4)])
def test_pure_hydrogen_saha_quadratic(oracle, rho, T):
    """Pure H: x^2 / (1 - x) = S / n_H, solved here as a quadratic."""
    nH = rho / (AH * AMU)
    S = saha_S(1.0, CHI[0], T)
    r = S / nH
    x = 0.5 * (-r + np.sqrt(r * r + 4 * r))
    assert 0.01 < x < 0.99  # a partially ionised point
    assert oracle.lib().tref_saha_pure_h_xe(rho, T) == pytest.approx(x, rel=2e-4)
    assert oracle.saha_state(rho, T, 1.0, 0.0)["xH"] == pytest.approx(x, rel=2e-4)


@pytest.mark.parametrize("rho,T", [(1e-8, 1.5e4), (1e-8, 3e4), (1e-6, 5e4)])
def test_pure_helium_two_stage_saha(oracle, rho, T):
    """Pure He: n_e (n_e^2 + S1 n_e + S1 S2) = n_He (S1 n_e + 2 S1 S2), a cubic."""
    nHe = rho / (AHE * AMU)
    S1 = saha_S(4.0, CHI[1], T)
    S2 = saha_S(1.0, CHI[2], T)
    roots = np.roots([1.0, S1, S1 * S2 - nHe * S1, -2 * nHe * S1 * S2])
    ne = max(r.real for r in roots if abs(r.imag) < 1e-6 * abs(r.real) and r.real > 0)
    D = ne * ne + S1 * ne + S1 * S2
    y1, y2 = S1 * ne / D, S1 * S2 / D
    s = oracle.saha_state(rho, T, 0.0, 1.0)
    assert s["yHe1"] == pytest.approx(y1, rel=3e-4, abs=1e-12)
    assert s["yHe2"] == pytest.approx(y2, rel=3e-4, abs=1e-12)
    assert s["ne"] == pytest.approx(ne, rel=3e-4)


def test_neutral_limit(oracle):
    """Cold gas: P_gas = rho k T / (mu m_u), mu = 1 / (X/A_H + Y/A_He); e = 3/2 P_gas/rho + a T^4/rho."""
    rho, T = 1e-6, 400.0
    s = oracle.saha_state(rho, T)
    mu = 1.0 / (X / AH + Y / AHE)
    Pg = rho * KB * T / (mu * AMU)
    assert s["Pgas"] == pytest.approx(Pg, rel=1e-12)
    assert s["mu"] == pytest.approx(mu, rel=1e-12)
    assert s["P"] == pytest.approx(Pg + ARAD * T ** 4 / 3, rel=1e-9)
    assert s["e"] == pytest.approx(1.5 * Pg / rho + ARAD * T ** 4 / rho, rel=1e-9)


def test_ionised_limit(oracle):
    """Hot dilute gas: mu = 1 / (2X/A_H + 3Y/A_He) and the full ionisation energy."""
    rho, T = 1e-10, 1e8
    s = oracle.saha_state(rho, T)
    assert s["xH"] == pytest.approx(1.0, abs=1e-12)
    assert s["yHe2"] == pytest.approx(1.0, abs=1e-9)
    mu = 1.0 / (2 * X / AH + 3 * Y / AHE)
    Pg = rho * KB * T / (mu * AMU)
    assert s["Pgas"] == pytest.approx(Pg, rel=1e-9)
    eion = (X / (AH * AMU) * CHI[0] + Y / (AHE * AMU) * (CHI[1] + CHI[2])) * 1.602176634e-12
    e = 1.5 * Pg / rho + eion + ARAD * T ** 4 / rho
    assert s["e"] == pytest.approx(e, rel=1e-9)


def gamma1_mixture(beta):
    """Gamma_1 of an ideal gas (gamma = 5/3) plus radiation with gas pressure fraction beta."""
    g = 5.0 / 3.0
    return beta + (4 - 3 * beta) ** 2 * (g - 1) / (beta + 12 * (g - 1) * (1 - beta))


@pytest.mark.parametrize("lr,lT", [(-14.0, 3.2), (-6.0, 2.5), (-12.0, 7.8), (-13.0, 7.0), (-4.0, 2.0)])
def test_gamma1_gas_radiation_closed_form(oracle, lr, lT):
    """Where the composition is frozen (neutral or fully ionised), Gamma_1 of the
    table equals Chandrasekhar's gas+radiation formula; it tends to 5/3 for gas
    and 4/3 for radiation domination."""
    n_rho, n_T = 2, 2
    le, lp, lc, g1 = (np.zeros((2, 2)) for _ in range(4))
    oracle.lib().tref_eos_build(n_rho, n_T, lr, lr + 1.0, lT, lT + 0.5, X, Y, oracle.P(le),
                                oracle.P(lp), oracle.P(lc), oracle.P(g1))
    s = oracle.saha_state(10 ** lr, 10 ** lT)
    assert min(s["xH"], 1 - s["xH"]) < 1e-10 and min(s["yHe2"], 1 - s["yHe2"] - s["yHe1"]) < 1e-8
    beta = s["Pgas"] / s["P"]
    assert g1[0, 0] == pytest.approx(gamma1_mixture(beta), rel=1e-6)
    assert lc[0, 0] == pytest.approx(np.log10(g1[0, 0] * s["P"] / 10 ** lr), rel=1e-12)


def test_gamma1_limits_in_table(saha_table):
    g1 = saha_table.gamma1
    assert g1[-1, 0] == pytest.approx(5 / 3, abs=1e-6)    # dense, cold, neutral: gas dominated
    assert g1[0, -1] == pytest.approx(4 / 3, abs=1e-4)    # dilute, hot: radiation dominated
    assert g1.min() > 0.5 and g1.max() < 5 / 3 + 1e-6


def test_columns_strictly_increasing(saha_table):
    assert (np.diff(saha_table.log10_e, axis=1) > 0).all()
    assert (np.diff(saha_table.log10_P, axis=1) > 0).all()


def test_node_round_trip(saha_table):
    """invert(rho_i, e_ij) returns T_j, P_ij at every interior node."""
    rng = np.random.default_rng(1)
    lr = np.linspace(-14, 2, 256)
    lt = np.linspace(2, 8, 256)
    for _ in range(400):
        i, j = rng.integers(0, 255), rng.integers(1, 254)
        e = 10 ** saha_table.log10_e[i, j]
        T, Pr, c2, cl = saha_table.invert(10 ** lr[i], e)
        assert not cl
        assert np.log10(T) == pytest.approx(lt[j], abs=1e-11)
        assert np.log10(Pr) == pytest.approx(saha_table.log10_P[i, j], abs=1e-11)
        assert np.log10(c2) == pytest.approx(saha_table.log10_cs2[i, j], abs=1e-11)


def test_bilinear_interpolation_closed_form(saha_table):
    """At the centre of a table cell the interpolant is the mean of the 4 corner logs."""
    t = saha_table
    lr = np.linspace(-14, 2, 256)
    lt = np.linspace(2, 8, 256)
    i, j = 100, 137
    rho = 10 ** (0.5 * (lr[i] + lr[i + 1]))
    T = 10 ** (0.5 * (lt[j] + lt[j + 1]))
    Pr, e, c2 = t.eval_rhoT(rho, T)
    for f, val in ((t.log10_P, Pr), (t.log10_e, e), (t.log10_cs2, c2)):
        mean = 0.25 * (f[i, j] + f[i, j + 1] + f[i + 1, j] + f[i + 1, j + 1])
        assert np.log10(val) == pytest.approx(mean, abs=1e-11)
    # and the inversion at that point returns the same T
    T2, P2, _, cl = t.invert(rho, e)
    assert not cl and T2 == pytest.approx(T, rel=1e-11) and P2 == pytest.approx(Pr, rel=1e-11)


def test_inversion_random_consistency(saha_table):
    """invert(rho, e(rho, T)) == T for random in-range points (any cell)."""
    rng = np.random.default_rng(7)
    for _ in range(500):
        lr = rng.uniform(-14, 2)
        lT = rng.uniform(2.01, 7.99)
        Pr, e, c2 = saha_table.eval_rhoT(10 ** lr, 10 ** lT)
        T, P2, c22, cl = saha_table.invert(10 ** lr, e)
        assert not cl
        assert np.log10(T) == pytest.approx(lT, abs=1e-10)
        assert P2 == pytest.approx(Pr, rel=1e-10)
        assert c22 == pytest.approx(c2, rel=1e-10)


def test_inversion_clamps(saha_table):
    e_cold = 10 ** saha_table.log10_e[50, 0] * 0.5
    T, Pr, c2, cl = saha_table.invert(10 ** (-14 + 16 * 50 / 255), e_cold)
    assert cl and T == pytest.approx(100.0, rel=1e-12)
    T, Pr, c2, cl = saha_table.invert(1e-8, -1.0)
    assert cl and T == pytest.approx(100.0, rel=1e-12)
    e_hot = 10 ** saha_table.log10_e[50, -1] * 2
    T, Pr, c2, cl = saha_table.invert(10 ** (-14 + 16 * 50 / 255), e_hot)
    assert cl and T == pytest.approx(1e8, rel=1e-12)


def test_T_from_P(saha_table):
    rho = 1e-8
    Pr, e, c2 = saha_table.eval_rhoT(rho, 1e3)
    assert saha_table.T_from_P(rho, Pr) == pytest.approx(1e3, rel=1e-12)


def test_invert_from_guess_equals_bisection(saha_table):
    """Any guess gives the bisection result bit for bit; a guess in the right
    temperature cell is accepted (the one Newton step is exact there)."""
    t = saha_table
    rng = np.random.default_rng(3)
    d = 6.0 / 255
    n_acc = 0
    for k in range(3000):
        lr = rng.uniform(-14, 2)
        lT = rng.uniform(2.0, 8.0)
        Pr, e, c2 = t.eval_rhoT(10 ** lr, 10 ** lT)
        want = t.invert(10 ** lr, e)
        guess = {0: lT, 1: lT + rng.normal(0, 0.5), 2: rng.uniform(-1, 11)}[k % 3]
        T, P2, c22, acc = t.invert_guess(10 ** lr, e, guess)
        assert (T, P2, c22) == want[:3]
        if k % 3 == 0:
            # exact guess: accepted unless it sits on the upper edge of a cell
            xj = (lT - 2.0) / d
            if 1e-9 < xj - np.floor(xj) < 1 - 1e-9:
                assert acc
        n_acc += acc
    assert n_acc > 1000
    # out of range input: never accepted, clamped like the plain inversion
    T, P2, c22, acc = t.invert_guess(1e-20, 1e10, 3.0)
    assert not acc and (T, P2, c22) == t.invert(1e-20, 1e10)[:3]


def test_guess_acceptance_rule_brute_force(saha_table):
    """Acceptance is decided by where the one Newton step lands: a guess k cells
    off is accepted exactly when the cell of j + (y - g_j) / (g_{j+1} - g_j),
    recomputed here from the table arrays, brackets y (or j itself does)."""
    t = saha_table
    rng = np.random.default_rng(31)
    nT = t.n_T
    d = 6.0 / (nT - 1)
    le = t.log10_e
    seen = {True: 0, False: 0}
    for k in range(2000):
        lr = rng.uniform(-13.9, 1.9)
        lT = rng.uniform(2.05, 7.95)
        e = t.eval_rhoT(10 ** lr, 10 ** lT)[1]
        x = (np.log10(10 ** lr) + 14.0) * (nT - 1) / 16.0
        i = min(int(np.floor(x)), t.n_rho - 2)
        w = x - i
        g = (1 - w) * le[i] + w * le[i + 1]       # the column at this density
        y = np.log10(e)
        jt = int(np.searchsorted(g, y, side="right") - 1)   # the bracketing cell
        off = int(rng.integers(-4, 5))
        jg = min(max(jt + off, 0), nT - 2)
        guess = 2.0 + (jg + 0.5) * d
        xn = jg + (y - g[jg]) / (g[jg + 1] - g[jg])
        predict = jg == jt or (0 <= xn < nT - 1 and int(np.floor(xn)) == jt)
        _, _, _, acc = t.invert_guess(10 ** lr, e, guess)
        if abs(xn - round(xn)) > 1e-9:       # skip landings within rounding of a node
            assert acc == predict, (k, off, jg, jt, xn)
            seen[acc] += 1
    assert seen[True] > 500 and seen[False] > 100


def test_c3_band_edges_are_the_ionisation_thresholds(oracle):
    """The EOS-inversion workload's band (data written from the oracle's Saha
    solver): at its lower edge hydrogen is 1 % ionised and at its upper edge helium
    99 % doubly ionised (or the table's top where that is not reached), the band
    rises with density, and the generator's samples stay inside it."""
    import os
    torch = pytest.importorskip("torch")
    from paper_2609_37859_gb300 import workloads as wl
    d = np.load(wl.C3_BAND_FILE)
    assert os.path.basename(wl.C3_BAND_FILE) == "c3_recombination_band.npz"
    for k in range(0, len(d["lrho"]), 32):
        rho = 10.0 ** d["lrho"][k]
        lo, hi = d["lT_lo"][k], d["lT_hi"][k]
        assert oracle.saha_state(rho, 10.0 ** lo)["xH"] == pytest.approx(0.01, rel=1e-6)
        if hi < 8.0:
            assert oracle.saha_state(rho, 10.0 ** hi)["yHe2"] == pytest.approx(0.99, rel=1e-6)
        else:
            assert oracle.saha_state(rho, 1e8)["yHe2"] < 0.99
    assert np.all(np.diff(d["lT_lo"]) > 0) and np.all(d["lT_hi"] > d["lT_lo"])
    g = torch.Generator()
    g.manual_seed(3)
    r, T = wl.c3_inputs(20000, g, "cpu")
    lr, lT = np.log10(r.numpy()), np.log10(T.numpy())
    assert lr.min() >= -14 and lr.max() <= 2
    assert np.all(lT >= np.interp(lr, d["lrho"], d["lT_lo"]) - 1e-12)
    assert np.all(lT <= np.interp(lr, d["lrho"], d["lT_hi"]) + 1e-12)
