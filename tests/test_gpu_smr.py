"""GPU parity on statically refined meshes (LAT across coarse-fine interfaces,
Sec. 7.1) against the oracle, through the C ABI: ghost cells by copy,
restriction and prolongation; synchronised steps (one window with every factor
1, the coarse-fine flux correction at its end); factor assignment with
f_fine <= f_coarse <= 2 f_fine; mixed-factor windows with the point mass and
dual energy; conservation; graph replay; a two-dimensional refined mesh; and the
layouts the library must refuse."""
import numpy as np
import pytest

from parity import assert_parity
from paper_2609_37859_gb300 import workloads as wl
from test_gpu_hydro import Pair  # noqa: F401

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_hydro import tde, ctx  # noqa: E402,F401


def sphere(centre, r):
    def refine(lo, hi, L):
        d2 = sum(max(lo[a] - centre[a], 0.0, centre[a] - hi[a]) ** 2 for a in range(3))
        return d2 < r * r
    return refine


def smr(bc=(1, 1, 1), ng=2, max_level=2, N=(16, 16, 16), block=(4, 4, 4), centre=(0.3, 0.4, 0.55), r=0.08):
    return wl.smr_layout(N, block, ((0, 1),) * 3, bc, ng, sphere(centre, r), max_level)


def smooth_W(lay, seed=3, amp=1.0):
    rng = np.random.default_rng(seed)
    x, y, z, _ = lay.interior_centres()
    k = rng.integers(1, 3, (5, 3))
    ph = rng.uniform(0, 2 * np.pi, 5)
    f = [np.sin(2 * np.pi * (k[q, 0] * x + k[q, 1] * y + k[q, 2] * z) + ph[q]) for q in range(5)]
    return wl.prim_cells(lay, 1.0 + 0.3 * amp * f[0], 0.4 * amp * f[1], 0.3 * amp * f[2], 0.2 * amp * f[3],
                         1.0 + 0.25 * amp * f[4])


def interior(lay, U):
    return np.asarray(U)[:, lay.interior_flat()]


def totals(lay, U):
    _, _, _, vol = lay.interior_centres()
    F = interior(lay, U)
    return (F[:5] * vol).sum(axis=1), (np.abs(F[:5]) * vol).sum(axis=1)


@pytest.mark.parametrize("bc,recon", [((1, 1, 1), 0), ((0, 0, 0), 1)])
def test_ghost_fill_parity(oracle, tde, ctx, bc, recon):
    lay = smr(bc=bc, ng=2 + recon, r=0.12)
    assert lay.levels.max() == 2
    P = Pair(oracle, tde, ctx, lay, smooth_W(lay), recon=recon, dual=1)
    U = P.U.copy()
    P.om.ghost_fill(U)
    P.gm.ghost_fill(P.gm.U)
    G = P.gpu("U")
    # every padded cell (interiors untouched, ghosts by copy / restriction / prolongation)
    assert_parity(G, U, 1e-14, "ghost fill")


def test_synchronised_steps_parity(oracle, tde, ctx):
    lay = smr(r=0.1)
    P = Pair(oracle, tde, ctx, lay, smooth_W(lay), dual=1, eta1=1e-3, eta2=1e-4)
    U = P.U.copy()
    P.gm.set_time(0.0)
    t = 0.0
    for s in range(3):
        dt = P.om.cfl_dt(U, 0.3, np.full(lay.nb, t)).min()
        P.om.step(U, dt, t)
        P.gm.step(dt=dt)
        t += dt
        assert_parity(interior(lay, P.gpu("U")), interior(lay, U), 1e-12 * (s + 1), "step %d" % s)
    assert P.gm.get_time() == pytest.approx(t, rel=1e-14)
    # the CFL path: the same dt chosen on both sides
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    P.gm.step(cfl=0.3, dt_out=dt_dev)
    dto = P.om.cfl_dt(U, 0.3, np.full(lay.nb, t)).min()
    assert float(dt_dev) == pytest.approx(dto, rel=1e-13)


def test_factor_assignment_parity(oracle, tde, ctx):
    lay = smr(r=0.1)
    bh = dict(on=1, GM=5.0, r_soft=0.03, x0=(0.3, 0.4, 0.55))
    P = Pair(oracle, tde, ctx, lay, smooth_W(lay), bh=bh, dual=1)
    for n_lat in (2, 4):
        dt = P.om.cfl_dt(P.U, 0.3, np.zeros(lay.nb))
        fo, dt0o, fmo = P.om.lat_factors(dt, n_lat, 0.0)
        fg, dt0g, fmg = P.gm.lat_assign(n_lat, 0.3, 0.0, bh=P.bh)
        assert np.array_equal(fg, fo) and fmg == fmo
        assert dt0g == pytest.approx(dt0o, rel=1e-13)
    assert fo.max() > 1 and len(set(fo)) > 1


@pytest.mark.parametrize("with_bh", [False, True])
def test_mixed_factor_windows_parity(oracle, tde, ctx, with_bh):
    lay = smr(r=0.1)
    bh = dict(on=1, GM=0.02, r_soft=0.05, x0=(0.3, 0.4, 0.55), v0=(0.2, 0.1, 0.0)) if with_bh else None
    P = Pair(oracle, tde, ctx, lay, smooth_W(lay), bh=bh, dual=1, eta1=1e-3, eta2=1e-4)
    U = P.U.copy()
    T0, scale = totals(lay, U)
    t = 0.0
    P.gm.set_time(0.0)
    for w in range(2):
        dt = P.om.cfl_dt(U, 0.3, np.full(lay.nb, t))
        f, dt0, fmax = P.om.lat_factors(dt, 3, 0.0)
        assert fmax > 1
        P.gm.lat_set_factors(f, dt0)
        fo, upd_o = P.om.lat_window(U, f, dt0, t)
        upd_g = P.gm.lat_window(bh=P.bh)
        assert upd_g == upd_o
        t += fmax * dt0
        assert_parity(interior(lay, P.gpu("U")), interior(lay, U), 1e-11 * (w + 1), "window %d" % w)
    assert P.gm.get_time() == pytest.approx(t, rel=1e-14)
    if not with_bh:
        T1, _ = totals(lay, P.gpu("U"))
        assert np.all(np.abs(T1 - T0) <= 1e-13 * scale)


def test_graph_replay_equals_eager(oracle, tde, ctx):
    lay = smr(r=0.1)
    P = Pair(oracle, tde, ctx, lay, smooth_W(lay), dual=1)
    dt = P.om.cfl_dt(P.U, 0.3, np.zeros(lay.nb))
    f, dt0, fmax = P.om.lat_factors(dt, 3, 0.0)
    outs = []
    for use_graph in (False, True):
        P.gm.U.copy_(torch.from_numpy(P.U))
        P.gm.set_time(0.0)
        P.gm.lat_set_factors(f, dt0)
        for _ in range(2):
            P.gm.lat_window(use_graph=use_graph)
        outs.append(P.gpu("U").copy())
    assert np.array_equal(outs[0], outs[1])


def test_two_dimensional_refined_mesh(oracle, tde, ctx):
    def disc(lo, hi, L):
        c = (0.5, 0.5)
        d2 = sum(max(lo[a] - c[a], 0.0, c[a] - hi[a]) ** 2 for a in range(2))
        return d2 < 0.15 ** 2
    lay = wl.smr_layout((32, 32, 1), (8, 8, 1), ((0, 1), (0, 1), (0, 0.05)), (1, 1, 0), 2, disc, 2)
    assert lay.levels.max() == 2
    x, y, z, _ = lay.interior_centres()
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2
    W = wl.prim_cells(lay, 1.0, 0.0, 0.0, 0.0, 1.0 + 10.0 * np.exp(-r2 / 0.005))   # a blast
    P = Pair(oracle, tde, ctx, lay, W, dual=1)
    U = P.U.copy()
    P.gm.set_time(0.0)
    t = 0.0
    for w in range(2):
        dt = P.om.cfl_dt(U, 0.3, np.full(lay.nb, t))
        f, dt0, fmax = P.om.lat_factors(dt, 3, 0.0)
        P.gm.lat_set_factors(f, dt0)
        P.om.lat_window(U, f, dt0, t)
        P.gm.lat_window()
        t += fmax * dt0
    assert_parity(interior(lay, P.gpu("U")), interior(lay, U), 1e-11, "2D blast")


def test_refused_layouts(tde, ctx):
    # level 2 next to level 0
    blocks = [(0, 0, 0, 4, 4, 4)] + [(16 + 8 * di, 8 * dj, 8 * dk, 8, 8, 8)
                                     for dk in (0, 1) for dj in (0, 1) for di in (0, 1)]
    bad = wl.MeshLayout(np.array(blocks, dtype=np.int32), (8, 4, 4), (0, 0, 0), (1 / 8, 1 / 4, 1 / 4),
                        (0, 0, 0), 2, np.array([0] + [2] * 8))
    with pytest.raises(tde.TDEError):
        tde.Mesh(ctx, bad, tde.make_params())
    # a refined block not aligned to 4 cells
    blocks = [(0, 0, 0, 4, 4, 4), (8, 0, 0, 2, 8, 8), (10, 0, 0, 6, 8, 8)]
    bad = wl.MeshLayout(np.array(blocks, dtype=np.int32), (8, 4, 4), (0, 0, 0), (1 / 8, 1 / 4, 1 / 4),
                        (0, 0, 0), 2, np.array([0, 1, 1]))
    with pytest.raises(tde.TDEError):
        tde.Mesh(ctx, bad, tde.make_params())
    # a single stage on a refined mesh
    lay = smr(r=0.1)
    m = tde.Mesh(ctx, lay, tde.make_params())
    with pytest.raises(tde.TDEError):
        m.hydro_stage(0, torch.ones(lay.nb, dtype=torch.float64, device="cuda"))


def test_frame_reduction_and_excision_on_a_refined_mesh(oracle, tde, ctx):
    """The frame acceleration (Eq. frame-acceleration) weighs each cell by its
    volume; LAT windows with the point mass's excision sphere inside the finest
    level; both against the oracle."""
    lay = smr(bc=(0, 0, 0), r=0.12, centre=(0.5, 0.45, 0.5))
    bh = dict(on=1, excise=1, GM=0.01, r_soft=0.04, r_exc=0.05, x0=(0.52, 0.45, 0.5), v0=(0.1, 0.0, 0.0))
    P = Pair(oracle, tde, ctx, lay, smooth_W(lay, seed=9), bh=bh, dual=1, eta1=1e-3, eta2=1e-4,
             rho_floor=1e-6, p_floor=1e-8, u_floor=1.5e-8)
    P.gm.set_time(0.0)
    Ao, mo = P.om.frame_acceleration(P.U, 0.0, 0.5)
    Ag, mg = P.gm.frame_acceleration(P.bh, 0.5)
    assert mg == pytest.approx(mo, rel=1e-13)
    assert np.allclose(Ag, Ao, rtol=1e-12, atol=1e-14 * np.abs(Ao).max())
    U = P.U.copy()
    t = 0.0
    for w in range(2):
        dt = P.om.cfl_dt(U, 0.3, np.full(lay.nb, t))
        f, dt0, fmax = P.om.lat_factors(dt, 3, 0.0)
        P.gm.lat_set_factors(f, dt0)
        P.om.lat_window(U, f, dt0, t)
        P.gm.lat_window(bh=P.bh)
        t += fmax * dt0
    assert_parity(interior(lay, P.gpu("U")), interior(lay, U), 2e-11, "refined windows with excision")
    assert P.gm.counts()["excised"] > 0
