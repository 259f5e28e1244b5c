"""Pins of the oracle's dual-energy compression source (Sec. 6.2,
Eqs. dual-compression-continuous, dual-divv, dual-tabulated-compression).

The source acts only where the face velocities diverge, so every test here runs
with div v != 0:

* one stage on a linear velocity field, whose discrete divergence is known in
  closed form: the auxiliary energy after the stage against the analytic
  exponential (ideal gas) and the tabulated pressure work with the stage's
  updated density (Eq. dual-tabulated-compression), for Delta t_l = dt (stage 1)
  and dt/2 (stage 2), expanding and compressing;
* a linear sound wave whose pressure comes from U_aux alone (eta_1 = eta_2 = 1:
  the closure never takes the conservative subtraction and the resync never
  overwrites U_aux), with an ideal gas and with the Saha table where the gas is
  neutral and gas-dominated (Gamma_1 = 5/3): second-order convergence to the
  closed-form linear solution.  A wrong sign, a wrong stage weight or a dropped
  direction changes the wave's speed, and the error stops converging.
"""
import numpy as np
import pytest

from paper_2609_37859_gb300 import workloads as wl

G53 = 5.0 / 3.0
SLOPES = (1.0, -0.5, 2.0)     # dv_x/dx, dv_y/dy, dv_z/dz of the linear field (sum 2.5)


def linear_flow(lay, rho, P, scale):
    """Uniform rho and P, v_d = scale * SLOPES[d] * (x_d - 1/2)."""
    x, y, z = lay.cell_centres()
    v = [scale * s * (c - 0.5) for s, c in zip(SLOPES, (x, y, z))]
    one = np.ones_like(x)
    return wl.prim_state(lay, rho * one, v[0], v[1], v[2], P * one)


def inner(G, lo=2):
    """Cells whose PLM stencils lie inside the linear data (outflow ghosts copy
    the edge cell, so the two cells at each boundary see a kinked profile)."""
    return G[..., lo:-lo, lo:-lo, lo:-lo]


def one_stage(oracle, params, table, stage, rho, P, scale, dt):
    """Run the stage on the linear flow; returns (U0, Uin, Uout) interiors.
    Stage 2 (index 1) takes U0 = the uniform gas at rest and Uin = the linear flow."""
    lay = wl.uniform_layout((16, 16, 16), (8, 8, 8), bc=(0, 0, 0), ng=2)
    m = oracle.Mesh(lay, params, table)
    Uin = m.prim_to_cons(linear_flow(lay, rho, P, scale))
    U0 = Uin.copy() if stage == 0 else m.prim_to_cons(linear_flow(lay, 1.25 * rho, 1.5 * P, 0.0))
    m.ghost_fill(Uin)
    Uout = m.new_state()
    nb = lay.nb
    m.stage(stage, U0, Uin, Uout, np.full(nb, dt), np.zeros(nb))
    return inner(m.interior(U0)), inner(m.interior(Uin)), inner(m.interior(Uout))


def advected(U0, Uin, stage, Ddt):
    """Closed form of the conservative part: a uniform density / energy density
    q on the linear field has flux q v_face, so the stage's update is
    q (1 - dt D) with D = sum of the slopes; stage 2 averages with U0."""
    q = lambda X: X * (1.0 - Ddt)
    rho = q(Uin[0]) if stage == 0 else 0.5 * (U0[0] + q(Uin[0]))
    A = q(Uin[5]) if stage == 0 else 0.5 * (U0[5] + q(Uin[5]))
    return rho, A


@pytest.mark.parametrize("stage", [0, 1])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_ideal_gas_compression_single_stage(oracle, stage, sign):
    """U_aux = U* exp(-(gamma - 1) div v Delta t_l), Delta t_l = dt, dt/2
    (Eq. dual-compression-continuous integrated at fixed div v)."""
    dt = 0.02
    p = oracle.make_params(dual=1, eta1=1e-3, eta2=1e-4)
    U0, Uin, Uout = one_stage(oracle, p, None, stage, 1.0, 1.0, sign, dt)
    D = sign * sum(SLOPES)
    rho, Astar = advected(U0, Uin, stage, D * dt)
    dtl = dt if stage == 0 else 0.5 * dt
    want = Astar * np.exp(-(G53 - 1.0) * D * dtl)
    assert np.allclose(Uout[0], rho, rtol=1e-13, atol=0)
    assert np.allclose(Uout[5], want, rtol=1e-12, atol=0), np.max(np.abs(Uout[5] / want - 1))
    # the alternatives a plausible mistake would give are far outside that bound
    for wrong in (Astar * np.exp(+(G53 - 1.0) * D * dtl),                    # sign
                  Astar * np.exp(-(G53 - 1.0) * D * (dt + 0.5 * dt - dtl)),  # stage weight
                  Astar * np.exp(-(G53 - 1.0) * (D - SLOPES[2] * sign) * dtl)):   # a direction
        assert np.min(np.abs(Uout[5] / wrong - 1)) > 1e-4


@pytest.mark.parametrize("stage", [0, 1])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_tabulated_compression_single_stage(oracle, saha_table, stage, sign):
    """U_aux = U* - P(rho^(l), U*/rho^(l)) div v Delta t_l with the stage's
    updated density (Eq. dual-tabulated-compression, reading 5), at rho = 1e-8
    g/cm^3, T = 1e4 K, where hydrogen is partly ionised and P(rho, U/rho) at
    fixed U moves by about 6 % for a 10 % change of rho: the pre-update density
    fails the check by far more than its tolerance."""
    t = saha_table
    rho0, T0 = 1e-8, 1e4
    P0, e0, _ = t.eval_rhoT(rho0, T0)
    p = oracle.make_params(eos=1, dual=1, eta1=1e-3, eta2=1e-4, rho_floor=1e-30, p_floor=1e-30,
                           u_floor=1e-30)
    scale = sign * 2e4          # |v| <= 2e4 cm/s, well below c_s ~ 1e6 cm/s
    dt = 0.04 / 2e4             # dt D = +-0.1
    U0, Uin, Uout = one_stage(oracle, p, t, stage, rho0, P0, scale, dt)
    D = scale * sum(SLOPES)
    rho, Astar = advected(U0, Uin, stage, D * dt)
    dtl = dt if stage == 0 else 0.5 * dt
    assert np.allclose(Uout[0], rho, rtol=1e-13, atol=0)
    # the expression is evaluated at one cell (uniform up to rounding): the
    # table's inversion is pinned separately (tests/test_oracle_eos.py)
    r, a = rho.ravel()[0], Astar.ravel()[0]
    Pw = t.invert(r, a / r)[1]
    want = a - Pw * D * dtl
    assert np.allclose(Uout[5], want, rtol=1e-12, atol=0), np.max(np.abs(Uout[5] / want - 1))
    r_pre = Uin[0].ravel()[0] if stage == 0 else 0.5 * (U0[0] + Uin[0]).ravel()[0]
    wrong = [a - t.invert(r_pre, a / r_pre)[1] * D * dtl,     # pre-update density
             a + Pw * D * dtl,                                 # sign
             a - Pw * D * (1.5 * dt - dtl)]                    # stage weight
    for w in wrong:
        assert abs(w / want - 1) > 1e-5, w / want - 1


def sound_wave_pressure_errors(oracle, table, Ns, amp=1e-6):
    """L1 error of the pressure recovered from U_aux after one period, over the
    amplitude, on 1-D periodic grids of N cells; the closure reads U_aux only."""
    errs = []
    for N in Ns:
        lay = wl.uniform_layout((N, 1, 1), (min(N, 32), 1, 1), bc=(1, 1, 1), ng=2)
        if table is None:
            rho0, P0, g1 = 1.0, 1.0 / G53, G53
            p = oracle.make_params(dual=1, eta1=1.0, eta2=1.0)
        else:
            rho0, T0 = 1e-4, 1e3
            P0, _, cs2 = table.eval_rhoT(rho0, T0)
            g1 = rho0 * cs2 / P0
            p = oracle.make_params(eos=1, dual=1, eta1=1.0, eta2=1.0, rho_floor=1e-30,
                                   p_floor=1e-30, u_floor=1e-30)
        cs = np.sqrt(g1 * P0 / rho0)
        m = oracle.Mesh(lay, p, table)
        U = m.prim_to_cons(wl.sound_wave(lay, amp=amp, rho0=rho0, P0=P0, gamma=g1))
        c = oracle.Counts()
        t, S = 0.0, m.new_state()
        while t < (1.0 / cs) * (1 - 1e-14):
            dt = min(m.cfl_dt(U, 0.3).min(), 1.0 / cs - t)
            m.step(U, dt, t, S, c)
            t += dt
        G = m.interior(U)[:, 0, 0]
        if table is None:
            Pn = (G53 - 1.0) * G[5]
        else:
            Pn = np.array([table.invert(r, a / r)[1] for r, a in zip(G[0], G[5])])
        x = lay.cell_centres()[0][0, 0]
        exact = P0 * (1 + g1 * amp * np.sin(2 * np.pi * x))
        errs.append(np.mean(np.abs(Pn - exact)) / (P0 * g1 * amp))
        # every conversion took U_aux, and the resync never replaced it
        assert c.dual_aux_used > 0 and c.synced == 0
    return np.array(errs)


def test_sound_wave_from_aux_energy_ideal_gas(oracle):
    """Pressure from U_aux alone converges to the linear sound wave at order >= 1.8."""
    e = sound_wave_pressure_errors(oracle, None, (32, 64, 128))
    order = np.log2(e[:-1] / e[1:])
    assert np.all(order >= 1.8), (e, order)
    assert e[-1] < 4e-3, e


def test_sound_wave_from_aux_energy_saha_table(oracle, saha_table):
    """The same through the table's pressure work: rho = 1e-4 g/cm^3, T = 1e3 K
    (neutral, radiation pressure 4e-7 of the gas's, Gamma_1 = 5/3 to 1e-9)."""
    P0, _, cs2 = saha_table.eval_rhoT(1e-4, 1e3)
    assert abs(1e-4 * cs2 / P0 - G53) < 1e-8
    e = sound_wave_pressure_errors(oracle, saha_table, (32, 64, 128))
    order = np.log2(e[:-1] / e[1:])
    assert np.all(order >= 1.8), (e, order)
    assert e[-1] < 4e-3, e
