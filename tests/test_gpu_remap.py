"""GPU parity of the domain remap (Sec. 5.2) against the oracle, through the C
ABI: identity on the same grid (bit for bit), coarsening of a periodic
Orszag-Tang velocity field in both energy forms, refinement and shifts onto
mixed and ragged MeshBlocks, targets reaching past a non-periodic source (floor
samples), a two-dimensional target, and dual / non-dual crossings."""
import numpy as np
import pytest

from parity import assert_parity
from paper_2609_37859_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_hydro import tde, ctx  # noqa: E402,F401

TOL = 1e-13
FLOORS = dict(rho_floor=1e-6, u_floor=1e-7)


class Side:
    """One mesh on both sides: oracle mesh and GPU mesh over the same layout."""

    def __init__(self, oracle, tde, ctx, layout, dual):
        self.layout = layout
        self.om = oracle.Mesh(layout, oracle.make_params(dual=dual, **FLOORS))
        self.gm = tde.Mesh(ctx, layout, tde.make_params(dual=dual, **FLOORS))


def remap_both(oracle, tde, S, D, U, mode):
    S.gm.U.copy_(torch.from_numpy(U))
    want = D.layout.to_global(oracle.remap(D.om, S.om, U, mode, FLOORS["rho_floor"], FLOORS["u_floor"]))
    D.gm.U.zero_()
    D.gm.remap_from(S.gm, S.gm.U, mode)
    torch.cuda.synchronize()
    got = D.layout.to_global(D.gm.U.cpu().numpy())
    return got, want


@pytest.mark.parametrize("dual", [0, 1])
def test_identity_is_bitwise(oracle, tde, ctx, dual):
    lay = wl.uniform_layout((24, 20, 16), (8, 8, 8), bc=(0, 1, 0), ng=2)
    S = Side(oracle, tde, ctx, lay, dual)
    D = Side(oracle, tde, ctx, lay, dual)
    U = S.om.prim_to_cons(wl.random_smooth(lay, seed=5))
    got, want = remap_both(oracle, tde, S, D, U, tde.REMAP_THERMAL)
    assert np.array_equal(got, lay.to_global(U))
    assert np.array_equal(want, lay.to_global(U))


def orszag_tang(lay):
    x, y, z = lay.cell_centres()
    rho = 25.0 / (36.0 * np.pi) * (1.0 + 0.2 * np.sin(2 * np.pi * (x + z)))
    return wl.prim_state(lay, rho, -np.sin(2 * np.pi * y), np.sin(2 * np.pi * x), 0.5 * np.sin(2 * np.pi * z),
                         5.0 / (12.0 * np.pi) * (1.0 + 0.1 * np.cos(2 * np.pi * y)))


def test_coarsening_both_energy_forms(oracle, tde, ctx):
    """Periodic Orszag-Tang velocity field (with density and pressure ripples)
    remapped to a grid twice as coarse: parity in both forms, and on the GPU the
    total form's extra internal energy equals the kinetic energy the coarse grid
    lost, cell by cell."""
    S = Side(oracle, tde, ctx, wl.uniform_layout((64, 64, 32), (16, 16, 16), ((0, 1), (0, 1), (0, 0.5)),
                                                 bc=(1, 1, 1)), 1)
    D = Side(oracle, tde, ctx, wl.uniform_layout((32, 32, 16), (8, 16, 8), ((0, 1), (0, 1), (0, 0.5)),
                                                 bc=(1, 1, 1)), 1)
    U = S.om.prim_to_cons(orszag_tang(S.layout))
    gth, oth = remap_both(oracle, tde, S, D, U, tde.REMAP_THERMAL)
    gto, oto = remap_both(oracle, tde, S, D, U, tde.REMAP_TOTAL)
    assert_parity(gth, oth, TOL, "thermal form")
    assert_parity(gto, oto, TOL, "total form")
    ke = 0.5 * (gth[1] ** 2 + gth[2] ** 2 + gth[3] ** 2) / gth[0]
    Gs = S.layout.to_global(U)
    ke_src = (0.5 * (Gs[1] ** 2 + Gs[2] ** 2 + Gs[3] ** 2) / Gs[0]).sum() / 8
    heat = (gto[4] - gth[4]).sum()
    assert heat == pytest.approx(ke_src - ke.sum(), rel=1e-9)
    assert np.allclose(gth[5], gth[4] - ke, rtol=1e-13, atol=0)


@pytest.mark.parametrize("dual_src,dual_dst", [(0, 1), (1, 0), (1, 1)])
def test_refine_and_shift_onto_mixed_blocks(oracle, tde, ctx, dual_src, dual_dst):
    """Outflow source; the target is finer, shifted, reaches past the source on
    two faces (floor samples) and is made of mixed 8^3 / 4^3 MeshBlocks."""
    src_lay = wl.uniform_layout((20, 18, 12), (8, 8, 8), ((-1, 1), (-0.9, 0.9), (-0.6, 0.6)), bc=(0, 0, 0))
    S = Side(oracle, tde, ctx, src_lay, dual_src)
    dst_lay = wl.mixed_layout((32, 32, 16), 8, {(0, 0, 0), (3, 2, 1)},
                              ((-0.7, 1.3), (-1.1, 0.9), (-0.5, 0.5)), (0, 0, 0), 2)
    D = Side(oracle, tde, ctx, dst_lay, dual_dst)
    U = S.om.prim_to_cons(wl.random_smooth(src_lay, seed=11, P0=3.0))
    for mode in (tde.REMAP_THERMAL, tde.REMAP_TOTAL):
        got, want = remap_both(oracle, tde, S, D, U, mode)
        assert_parity(got, want, TOL, "mode %d" % mode)
        # samples past the source's +x and -y faces: floor cells exist
        assert np.any(np.isclose(got[0], FLOORS["rho_floor"], rtol=1e-14, atol=0))


def test_ragged_coarsening_and_two_dimensional_target(oracle, tde, ctx):
    src_lay = wl.uniform_layout((30, 26, 22), (8, 8, 8), ((0, 1.5), (0, 1.3), (0, 1.1)), bc=(1, 0, 1))
    S = Side(oracle, tde, ctx, src_lay, 1)
    U = S.om.prim_to_cons(wl.random_smooth(src_lay, seed=13, P0=2.0))
    # 3:1-ish non-integer coarsening with ragged blocks
    D = Side(oracle, tde, ctx, wl.uniform_layout((11, 10, 7), (4, 4, 4), ((0, 1.5), (0.1, 1.2), (0, 1.1)),
                                                 bc=(1, 0, 1)), 1)
    got, want = remap_both(oracle, tde, S, D, U, tde.REMAP_THERMAL)
    assert_parity(got, want, TOL, "ragged coarsening")
    # a single-cell-thick z slab: samples in x and y only (N_qd = 4)
    D2 = Side(oracle, tde, ctx, wl.uniform_layout((40, 36, 1), (16, 16, 1), ((0, 1.5), (0, 1.3), (0.4, 0.45)),
                                                  bc=(1, 0, 0)), 1)
    got, want = remap_both(oracle, tde, S, D2, U, tde.REMAP_THERMAL)
    assert_parity(got, want, TOL, "two-dimensional target")


def test_invalid_arguments(tde, ctx):
    lay = wl.uniform_layout((8, 8, 8), (8, 8, 8))
    a = tde.Mesh(ctx, lay, tde.make_params())
    b = tde.Mesh(ctx, lay, tde.make_params())
    with pytest.raises(RuntimeError):
        b.remap_from(a, a.U, mode=7)
    with pytest.raises(RuntimeError):
        a.remap_from(a, a.U, out=a.U)
