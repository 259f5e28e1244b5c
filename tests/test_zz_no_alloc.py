"""tde_compute_dt_noalloc: the CFL step for callers that may not allocate device
memory (their device memory belongs to another allocator, or allocation is
forbidden after start-up).  It must give what tde_compute_dt gives, bit for
bit, call after call, although its scratch is one fixed device array shared by
all calls.

This file is collected last so that a failure here leaves every other test run.
"""
import os

import numpy as np
import pytest

from paper_2609_37859_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLE = os.path.join(ROOT, "paper_2609_37859_gb300", "data", "eos_saha_hhe_256.npz")


@pytest.fixture(scope="module")
def tde():
    from paper_2609_37859_gb300 import build, tde as T
    build.build()
    return T


def test_noalloc_dt_equals_compute_dt_on_two_calls(tde):
    ctx = tde.Context(0)
    d = np.load(TABLE)
    eos = tde.EOS.from_file(ctx, TABLE)
    dev = torch.device("cuda", 0)
    view = (int(d["n_rho"]), int(d["n_T"]), tuple(d["lrho"]), tuple(d["lT"]),
            torch.from_numpy(d["log10_e"].copy()).to(dev), torch.from_numpy(d["log10_P"].copy()).to(dev),
            torch.from_numpy(d["log10_cs2"].copy()).to(dev))
    # tabulated, dual-energy entropy wave on 4 x 4 x 2 blocks of 16^3 (the bench physics)
    lay = wl.uniform_layout((64, 64, 32), (16, 16, 16), bc=(1, 1, 1), ng=2)
    P0 = 639.748076615761   # pressure at rho = 1e-8, T = 1e3 of the stored table (any level works)
    W, _ = wl.entropy_wave(lay, 1e-8, P0, 3e12, amp=1e-3, seed=5)
    params = tde.make_params(eos=tde.EOS_TABLE, dual=1, eta1=1e-3, eta2=1e-4, rho_floor=1e-20,
                             p_floor=1e-20, u_floor=1e-20)
    mesh = tde.Mesh(ctx, lay, params, eos)
    mesh.prim_to_cons(torch.from_numpy(np.ascontiguousarray(W)).to(dev))
    nb = lay.nb
    for call in range(2):
        want = torch.zeros(nb, dtype=torch.float64, device=dev)
        want_min = torch.zeros(1, dtype=torch.float64, device=dev)
        mesh.compute_dt(0.3, want, want_min)
        got = torch.full((nb,), -1.0, dtype=torch.float64, device=dev)
        got_min = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
        tde.compute_dt_noalloc(ctx, lay, params, mesh.U, 0.3, got, got_min, table=view)
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy(), want.cpu().numpy()), call
        assert float(got_min) == float(want_min)
        mesh.step(cfl=0.3)    # a new state for the second call


def test_noalloc_dt_with_point_mass_and_excision_then_size_limit(tde):
    ctx = tde.Context(0)
    dev = torch.device("cuda", 0)
    lay = wl.uniform_layout((24, 16, 16), (8, 8, 8), bc=(1, 0, 1), ng=2)
    params = tde.make_params(dual=1)
    mesh = tde.Mesh(ctx, lay, params)
    mesh.prim_to_cons(torch.from_numpy(np.ascontiguousarray(wl.random_smooth(lay, seed=6))).to(dev))
    bh = tde.make_bh(on=1, excise=1, GM=0.2, r_soft=0.05, r_exc=0.15, x0=(0.5, 0.5, 0.5),
                     v0=(0.3, 0.0, 0.0))
    tb = torch.linspace(0.0, 0.2, lay.nb, dtype=torch.float64, device=dev)
    for _ in range(2):
        want = torch.zeros(lay.nb, dtype=torch.float64, device=dev)
        mesh.compute_dt(0.4, want, t_block=tb, bh=bh)
        got = torch.zeros(lay.nb, dtype=torch.float64, device=dev)
        tde.compute_dt_noalloc(ctx, lay, params, mesh.U, 0.4, got, t_block=tb, bh=bh)
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy(), want.cpu().numpy())
        tb += 0.05
    big = wl.uniform_layout((8, 8, 4097), (8, 8, 1), bc=(1, 1, 1), ng=2)
    with pytest.raises(tde.TDEError) as ei:
        tde.compute_dt_noalloc(ctx, big, params, mesh.U, 0.4, got)
    assert ei.value.code == tde.TDE_EINVAL and "4096" in str(ei.value)


def test_noalloc_dt_on_a_refined_mesh(tde):
    """Blocks on three refinement levels (cells dx / 2^level): the same per-block
    CFL step as tde_compute_dt."""
    ctx = tde.Context(0)
    dev = torch.device("cuda", 0)

    def ball(lo, hi, L):
        c = (0.4, 0.5, 0.5)
        return sum(max(lo[a] - c[a], 0.0, c[a] - hi[a]) ** 2 for a in range(3)) < 0.1 ** 2
    lay = wl.smr_layout((16, 16, 16), (4, 4, 4), ((0, 1),) * 3, (1, 1, 1), 2, ball, 2)
    assert lay.levels.max() == 2
    params = tde.make_params(dual=1)
    mesh = tde.Mesh(ctx, lay, params)
    x, y, z, _ = lay.interior_centres()
    W = wl.prim_cells(lay, 1.0 + 0.2 * np.sin(2 * np.pi * x), 0.3 * np.cos(2 * np.pi * y), 0.0, 0.1, 1.0)
    mesh.prim_to_cons(torch.from_numpy(np.ascontiguousarray(W)).to(dev))
    bh = tde.make_bh(on=1, excise=1, GM=0.05, r_soft=0.05, r_exc=0.08, x0=(0.4, 0.5, 0.5))
    want = torch.zeros(lay.nb, dtype=torch.float64, device=dev)
    mesh.compute_dt(0.3, want, bh=bh)
    got = torch.zeros(lay.nb, dtype=torch.float64, device=dev)
    tde.compute_dt_noalloc(ctx, lay, params, mesh.U, 0.3, got, bh=bh)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), want.cpu().numpy())


def test_noalloc_rejects_bad_table_views_and_blocks(tde):
    """The checks of tde_mesh_create, and the table view's shape, before any GPU work."""
    from types import SimpleNamespace
    ctx = tde.Context(0)
    dev = torch.device("cuda", 0)
    lay = wl.uniform_layout((32, 32, 32), (16, 16, 16), bc=(1, 1, 1), ng=2)
    params = tde.make_params(dual=1)
    U = torch.zeros((6, lay.ntot), dtype=torch.float64, device=dev)
    out = torch.zeros(lay.nb, dtype=torch.float64, device=dev)

    def fails(layout, prm=params, table=None, what=""):
        with pytest.raises(tde.TDEError) as ei:
            tde.compute_dt_noalloc(ctx, layout, prm, U, 0.3, out, table=table)
        assert ei.value.code == tde.TDE_EINVAL and what in str(ei.value), str(ei.value)

    def with_blocks(blocks, N=lay.N):
        blocks = np.asarray(blocks, dtype=np.int32)
        return SimpleNamespace(nb=len(blocks), blocks=blocks, N=N, xmin=lay.xmin, dx=lay.dx, bc=lay.bc,
                               ng=lay.ng, level=lambda q: 0)
    edge = "edge above 32 cells"
    fails(with_blocks([(0, 0, 0, 33, 16, 16)], N=(64, 32, 32)), what=edge)        # edge > 32
    fails(with_blocks([(24, 0, 0, 16, 16, 16)]), what=edge)                       # past the grid
    fails(with_blocks([(-1, 0, 0, 16, 16, 16)]), what=edge)                       # negative origin
    fails(with_blocks([(0, 0, 0, 16, 16, 2)], N=(32, 32, 1)), what=edge)          # inactive axis, 2 cells
    tp = tde.make_params(eos=tde.EOS_TABLE, dual=1)
    col = torch.zeros((4, 4), dtype=torch.float64, device=dev)
    fails(lay, tp, table=(4, 4, (-14.0, 2.0), (2.0, 8.0), col, None, col), what="table view")
    fails(lay, tp, table=(4, 1, (-14.0, 2.0), (2.0, 8.0), col, col, col), what="table view")
    fails(lay, tp, table=(4, 4, (2.0, -14.0), (2.0, 8.0), col, col, col), what="table view")
    fails(lay, tp, table=(4, 4, (-14.0, 2.0), (8.0, 8.0), col, col, col), what="table view")
