"""Sweep tile shapes and their autotuner (the batching part of a9): every shape
computes the same operations on the same data, so a step gives identical bits
whichever shape each direction uses; the autotuner leaves the state alone."""
import numpy as np
import pytest

from paper_2609_37859_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_hydro import Pair, c2_pair, tde, ctx, tables  # noqa: E402,F401

SHAPES = ((0, 0, 0), (1, 1, 1), (2, 2, 2), (2, 0, 1))


def run_steps(P, tiles, n, bh=None):
    P.gm.set_tiles(tiles)
    P.gm.U.copy_(torch.from_numpy(P.U))
    P.gm.set_time(0.0)
    for _ in range(n):
        P.gm.step(cfl=0.3, bh=bh)
    return P.gpu("U").copy()


def test_tile_shapes_identical_c2(oracle, tde, ctx, tables):
    """32^3 blocks, PLM, Saha table, dual energy: 3 steps under each shape."""
    P, _ = c2_pair(oracle, tde, ctx, tables, 64, 32, seed=3)
    ref = run_steps(P, SHAPES[0], 3)
    for t in SHAPES[1:]:
        assert np.array_equal(run_steps(P, t, 3), ref), t


def test_tile_shapes_identical_mixed_ppm_bh(oracle, tde, ctx, tables):
    """Mixed 8^3 / 4^3 blocks (ragged lane tiles), PPM, point mass with excision."""
    rho0, v0 = 0.7382, 1.0948e8
    lay = wl.mixed_layout((16, 16, 8), 8, {(0, 0, 0), (1, 1, 0)},
                          ((-2.0, 2.0), (-2.0, 2.0), (-1.0, 1.0)), (0, 0, 0), 3)
    x, y, z = lay.cell_centres()
    r = np.sqrt(x ** 2 + y ** 2 + z ** 2)
    rho = 1e-6 + 1e-3 * np.exp(-((r - 1.0) / 0.3) ** 2)
    Pc = rho * rho0 * 1.380649e-16 * 1e4 / (0.6 * 1.6605e-24) / (rho0 * v0 * v0)
    W = wl.prim_state(lay, rho, -y * 0.3, x * 0.3, 0 * rho, Pc)
    bh = dict(on=1, excise=1, GM=1000 / (4 * np.pi), r_soft=0.005, r_exc=0.35, x0=(0.05, -0.02, 0.0),
              v0=(0.1, 0.0, 0.0))
    P = Pair(oracle, tde, ctx, lay, W, tables, bh=bh, eos=1, recon=1, dual=1, eta1=1e-3, eta2=1e-4,
             rho_floor=1e-10, p_floor=1e-16, u_floor=1.5e-16, unit_rho=rho0, unit_e=v0 * v0)
    ref = run_steps(P, SHAPES[0], 2, P.bh)
    for t in SHAPES[1:]:
        assert np.array_equal(run_steps(P, t, 2, P.bh), ref), t
    # and through a LAT window with mixed factors (flux registers, refluxing)
    f = np.where(np.arange(lay.nb) % 3 == 0, 2, 1).astype(np.int32)
    outs = []
    for t in (SHAPES[0], SHAPES[2]):
        P.gm.set_tiles(t)
        P.gm.U.copy_(torch.from_numpy(P.U))
        P.gm.set_time(0.0)
        P.gm.lat_set_factors(f, 1e-4)
        P.gm.lat_window(bh=P.bh, use_graph=True)
        outs.append(P.gpu("U").copy())
    assert np.array_equal(outs[0], outs[1])


def test_autotune_leaves_state_untouched(oracle, tde, ctx, tables):
    P, _ = c2_pair(oracle, tde, ctx, tables, 64, 32, seed=5)
    P.gm.set_time(0.25)
    P.gm.step(cfl=0.3)
    U0 = P.gpu("U").copy()
    c0 = P.gm.counts()
    t0 = P.gm.get_time()
    tiles, ms = P.gm.autotune(reps=2)
    assert np.array_equal(P.gpu("U"), U0)
    assert P.gm.counts() == c0 and P.gm.get_time() == t0
    assert P.gm.get_tiles() == tiles
    for d in range(3):
        assert 0 <= tiles[d] < 3
        assert ms[d][tiles[d]] == min(v for v in ms[d] if v >= 0)
    # the next step is the step it would have been
    P.gm.step(cfl=0.3)
    A = P.gpu("U").copy()
    P.gm.set_tiles((0, 0, 0))
    P.gm.U.copy_(torch.from_numpy(U0))
    P.gm.set_time(t0)
    P.gm.step(cfl=0.3)
    assert np.array_equal(P.gpu("U"), A)


def test_set_tiles_rejects_bad_shapes(tde, ctx):
    lay = wl.uniform_layout((8, 8, 8), (8, 8, 8), bc=(1, 1, 1), ng=2)
    m = tde.Mesh(ctx, lay, tde.make_params())
    for bad in ((3, 0, 0), (0, -1, 0)):
        with pytest.raises(tde.TDEError):
            m.set_tiles(bad)
    assert m.get_tiles() == [0, 0, 0]
