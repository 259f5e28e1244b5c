"""Pins of the oracle's conserved-variable remap (Sec. 5.2): identity on the
same grid, exact reproduction of linear fields, and the thermal- vs
total-energy forms (the total form heats by exactly the kinetic energy the
target grid cannot represent; the paper's Orszag-Tang comparison, here with
the hydrodynamic Orszag-Tang velocity field)."""
import numpy as np
import pytest

from paper_2609_37859_gb300 import workloads as wl

G53 = 5.0 / 3.0


def mesh(oracle, N, block, domain, bc=(0, 0, 0), dual=0):
    lay = wl.uniform_layout(N, block, domain=domain, bc=bc, ng=2)
    return lay, oracle.Mesh(lay, oracle.make_params(dual=dual))


@pytest.mark.parametrize("dual", [0, 1])
def test_identity_on_the_same_grid(oracle, dual):
    lay, m = mesh(oracle, (16, 12, 8), (8, 4, 8), ((0, 1), (0, 1), (0, 0.5)), dual=dual)
    U = m.prim_to_cons(wl.random_smooth(lay, seed=2))
    V = oracle.remap(m, m, U)
    assert np.array_equal(lay.to_global(V), lay.to_global(U))


def test_linear_fields_reproduced(oracle):
    """Trilinear interpolation and midpoint quadrature are exact for linear
    fields: a coarser, shifted target grid sees rho, m and U exactly (away from
    the source boundary, where the outflow edge copy is not linear)."""
    src_lay, src = mesh(oracle, (32, 32, 16), (16, 16, 8), ((0, 2), (0, 2), (0, 1)))
    dst_lay, dst = mesh(oracle, (12, 12, 6), (6, 6, 6), ((0.3, 1.5), (0.3, 1.5), (0.2, 0.8)))
    x, y, z = src_lay.cell_centres()
    lin = lambda x, y, z, a: a[0] + a[1] * x + a[2] * y + a[3] * z
    rho = lin(x, y, z, (1.0, 0.1, 0.05, -0.02))
    mx, my, mz = lin(x, y, z, (0.2, 0.01, 0.0, 0.03)), lin(x, y, z, (-0.1, 0.02, 0.04, 0.0)), 0 * x + 0.05
    Uth = lin(x, y, z, (2.0, -0.1, 0.2, 0.1))
    E = Uth + 0.5 * (mx ** 2 + my ** 2 + mz ** 2) / rho
    U = src_lay.from_global(np.stack([rho, mx, my, mz, E]))
    V = dst_lay.to_global(oracle.remap(dst, src, U))
    X, Y, Z = dst_lay.cell_centres()
    assert np.allclose(V[0], lin(X, Y, Z, (1.0, 0.1, 0.05, -0.02)), rtol=1e-13)
    assert np.allclose(V[1], lin(X, Y, Z, (0.2, 0.01, 0.0, 0.03)), rtol=1e-12, atol=1e-14)
    ke = 0.5 * (V[1] ** 2 + V[2] ** 2 + V[3] ** 2) / V[0]
    assert np.allclose(V[4] - ke, lin(X, Y, Z, (2.0, -0.1, 0.2, 0.1)), rtol=1e-12)


def test_thermal_vs_total_energy_forms(oracle):
    """Hydrodynamic Orszag-Tang state (v = (-sin 2 pi y, sin 2 pi x, sin 2 pi z / 2),
    uniform rho and P), remapped onto a grid twice as coarse: carrying thermal
    energy keeps the internal energy (uniform here: exactly), carrying total
    energy raises it by exactly the kinetic energy lost, cell by cell."""
    src_lay, src = mesh(oracle, (32, 32, 32), (16, 16, 16), ((0, 1),) * 3, bc=(1, 1, 1))
    dst_lay, dst = mesh(oracle, (16, 16, 16), (8, 8, 8), ((0, 1),) * 3, bc=(1, 1, 1))
    x, y, z = src_lay.cell_centres()
    rho = 25.0 / (36.0 * np.pi) + 0 * x
    W = src_lay.from_global(np.stack([rho, -np.sin(2 * np.pi * y), np.sin(2 * np.pi * x),
                                      0.5 * np.sin(2 * np.pi * z), 5.0 / (12.0 * np.pi) + 0 * x]))
    U = src.prim_to_cons(W)
    Vth = dst_lay.to_global(oracle.remap(dst, src, U, oracle.REMAP_THERMAL))
    Vto = dst_lay.to_global(oracle.remap(dst, src, U, oracle.REMAP_TOTAL))
    assert np.array_equal(Vth[:4], Vto[:4])
    ke = 0.5 * (Vth[1] ** 2 + Vth[2] ** 2 + Vth[3] ** 2) / Vth[0]
    ein_th, ein_to = Vth[4] - ke, Vto[4] - ke
    G = src_lay.to_global(U)
    ein0 = (G[4] - 0.5 * (G[1] ** 2 + G[2] ** 2 + G[3] ** 2) / G[0]).sum() / 8
    ke_src = (0.5 * (G[1] ** 2 + G[2] ** 2 + G[3] ** 2) / G[0]).sum() / 8
    rel_th = ein_th.sum() / ein0 - 1.0
    rel_to = ein_to.sum() / ein0 - 1.0
    print("internal energy change: thermal form %.2e, total form %.3f %%" % (rel_th, 100 * rel_to))
    assert abs(rel_th) < 1e-13
    assert 1e-3 < rel_to < 0.05
    # the total form's extra heat is the kinetic energy the coarse grid cannot hold
    assert (ein_to - ein_th).sum() == pytest.approx(ke_src - ke.sum(), rel=1e-9)
