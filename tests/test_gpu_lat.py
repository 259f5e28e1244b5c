"""GPU parity of localized adaptive time stepping (Sec. 7) against the oracle,
through the C ABI: factor assignment, windows with mixed factors (ghost modes,
flux registers, refluxing with gravity), the all-ones reduction to the
synchronised step, and CUDA-graph replay of a window."""
import numpy as np
import pytest

from parity import assert_parity
from paper_2609_37859_gb300 import workloads as wl
from test_gpu_hydro import Pair, TABLE_FILE  # noqa: F401  (fixtures below)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_hydro import tde, ctx, tables  # noqa: E402,F401


def band_factors(lay, levels):
    f = np.ones(lay.nb, dtype=np.int32)
    for b, blk in enumerate(lay.blocks):
        f[b] = levels[(blk[0] // blk[3]) % len(levels)]
    return f


def smooth_pair(oracle, tde, ctx, bh=None, recon=0, dual=1):
    lay = wl.uniform_layout((32, 16, 16), (8, 8, 8), bc=(1, 1, 1), ng=2 + recon)
    W = wl.random_smooth(lay, seed=31, P0=2.0)
    return Pair(oracle, tde, ctx, lay, W, bh=bh, recon=recon, dual=dual, eta1=1e-3, eta2=1e-4)


def test_lat_factor_assignment_parity(oracle, tde, ctx):
    lay = wl.uniform_layout((64, 16, 16), (8, 8, 8), domain=((0, 4), (0, 1), (0, 1)), bc=(1, 1, 1), ng=2)
    bh = dict(on=1, GM=20.0, r_soft=0.02, x0=(0.3, 0.5, 0.5))
    P = Pair(oracle, tde, ctx, lay, wl.random_smooth(lay, seed=31, P0=2.0), bh=bh, dual=1)
    for n_lat, merge in ((3, 0.0), (5, 0.05)):
        dt = P.om.cfl_dt(P.U, 0.3, np.zeros(P.nb))
        fo, dt0o, fmo = P.om.lat_factors(dt, n_lat, merge)
        fg, dt0g, fmg = P.gm.lat_assign(n_lat, 0.3, merge, bh=P.bh)
        assert np.array_equal(fg, fo) and fmg == fmo
        assert dt0g == pytest.approx(dt0o, rel=1e-14)
    assert fo.max() > 1


def test_lat_all_ones_is_the_synchronised_step(oracle, tde, ctx):
    bh = dict(on=1, excise=1, GM=0.05, r_soft=0.05, r_exc=0.06, x0=(0.4, 0.5, 0.5), v0=(0.5, 0, 0))
    P = smooth_pair(oracle, tde, ctx, bh=bh, recon=1)
    dt = 0.5 * P.om.cfl_dt(P.U, 0.3).min()
    P.gm.set_time(0.05)
    P.gm.step(dt=dt, bh=P.bh)
    A = P.gpu("U").copy()
    P.gm.U.copy_(torch.from_numpy(P.U))
    P.gm.set_time(0.05)
    P.gm.lat_set_factors(np.ones(P.nb, dtype=np.int32), dt)
    assert P.gm.lat_window(bh=P.bh) == P.nb
    B = P.gpu("U")
    # interiors equal bit for bit (LAT also refreshes U's ghost layer, the
    # synchronised path only the primitives' one)
    assert np.array_equal(P.layout.to_global(A), P.layout.to_global(B))
    assert P.gm.get_time() == pytest.approx(0.05 + dt, rel=1e-15)


@pytest.mark.parametrize("levels,with_bh", [((1, 2), False), ((1, 2, 4, 2), True)])
def test_lat_mixed_factor_windows_parity(oracle, tde, ctx, levels, with_bh):
    bh = dict(on=1, GM=0.02, r_soft=0.1, x0=(0.5, 0.25, 0.25), v0=(0.2, 0.1, 0.0)) if with_bh else None
    P = smooth_pair(oracle, tde, ctx, bh=bh)
    f = band_factors(P.layout, levels)
    dt0 = 0.4 * P.om.cfl_dt(P.U, 0.3).min() / f.max()
    U = P.U.copy()
    P.gm.set_time(0.0)
    P.gm.lat_set_factors(f, dt0)
    G0 = P.layout.to_global(U)
    t = 0.0
    for w in range(3):
        fmax, upd_o = P.om.lat_window(U, f, dt0, t)
        upd_g = P.gm.lat_window(bh=P.bh)
        assert upd_g == upd_o == int(sum(fmax // f))
        t += fmax * dt0
        G = P.layout.to_global(P.gpu("U"))
        assert_parity(G, P.layout.to_global(U), 1e-11 * (w + 1), "window %d" % w)
    assert P.gm.get_time() == pytest.approx(t, rel=1e-14)
    if not with_bh:
        for v in range(5):
            assert abs(G[v].sum() - G0[v].sum()) <= 1e-14 * np.abs(G[v]).sum()


def test_lat_graph_replay_equals_eager(oracle, tde, ctx):
    P = smooth_pair(oracle, tde, ctx, bh=dict(on=1, GM=0.02, r_soft=0.1, x0=(0.5, 0.25, 0.25)))
    f = band_factors(P.layout, (1, 2, 4, 2))
    dt0 = 0.4 * P.om.cfl_dt(P.U, 0.3).min() / f.max()
    outs = []
    for use_graph in (False, True):
        P.gm.U.copy_(torch.from_numpy(P.U))
        P.gm.set_time(0.0)
        P.gm.lat_set_factors(f, dt0)
        for _ in range(3):
            P.gm.lat_window(bh=P.bh, use_graph=use_graph)
        outs.append(P.gpu("U").copy())
    assert np.array_equal(outs[0], outs[1])


def test_lat_mixed_block_sizes_table_eos_bh_excision(oracle, tde, ctx, tables):
    """C4-like physics: mixed 8^3 / 4^3 blocks, PPM, Saha table in code units, dual
    energy, moving point mass with excision, factors from the CFL assignment."""
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
    U = P.U.copy()
    t = 0.0
    P.gm.set_time(0.0)
    for w in range(2):
        dt = P.om.cfl_dt(U, 0.3, np.full(P.nb, t))
        fo, dt0, fmax = P.om.lat_factors(dt, 4, 0.0)
        fg, dt0g, fmaxg = P.gm.lat_assign(4, 0.3, 0.0, bh=P.bh)
        assert np.array_equal(fg, fo)
        P.om.lat_window(U, fo, dt0, t)
        P.gm.lat_window(bh=P.bh)
        t += fmax * dt0
    assert fmax > 1
    assert_parity(lay.to_global(P.gpu("U")), lay.to_global(U), 1e-10, "C4-like LAT")
    assert P.gm.counts()["nonfinite"] == 0


def test_lat_graph_survives_reassignment_with_same_levels(oracle, tde, ctx):
    """A re-assignment that keeps the levels and their sizes (here: the factors
    moved between blocks) keeps the captured window, which then reads the new
    block lists; the result equals eager windows with the same factors."""
    P = smooth_pair(oracle, tde, ctx, bh=dict(on=1, GM=0.02, r_soft=0.1, x0=(0.5, 0.25, 0.25)))
    f1 = band_factors(P.layout, (1, 2, 4, 2))
    f2 = np.roll(f1, 3)
    assert sorted(f1) == sorted(f2) and not np.array_equal(f1, f2)
    dt0 = 0.4 * P.om.cfl_dt(P.U, 0.3).min() / f1.max()
    outs = []
    for use_graph in (False, True):
        P.gm.U.copy_(torch.from_numpy(P.U))
        P.gm.set_time(0.0)
        for f in (f1, f2, f1):
            P.gm.lat_set_factors(f, dt0)
            P.gm.lat_window(bh=P.bh, use_graph=use_graph)
        outs.append(P.gpu("U").copy())
    assert np.array_equal(outs[0], outs[1])
