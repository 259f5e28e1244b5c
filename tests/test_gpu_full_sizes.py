"""Parity at the benchmark's full sizes, in its launch configurations, on sampled
outputs the oracle computes one by one, and properties that hold at any size:

* C3: 2^24 table inversions in the three modes (identical results), sampled
  cells against the oracle's inversion;
* C4: the 13.1 M-cell stream (512 mixed 32^3 / 16^3 MeshBlocks, PPM, Saha table,
  dual energy, point mass with excision): the factor assignment of every block
  against the oracle's, one stage of sampled blocks recomputed by the oracle from
  the same input, and a full LAT window (graph) that stays finite;
* C5: the 67 M-cell production shape (2048 x 32^3, learned-guess closure): the
  same checks.

The oracle builds its own state from the same seeded primitives (its own EOS
evaluation and prim -> cons); nothing the GPU computes enters it."""
import numpy as np
import pytest

from parity import assert_parity_stencil, stencil_scale
from paper_2609_37859_gb300 import workloads as wl
from test_gpu_hydro import Pair, STAGE_TOL, TABLE_FILE  # noqa: F401

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_hydro import tde, ctx, tables  # noqa: E402,F401


def test_c3_full_size_inversion_sampled(oracle, tde, ctx, tables):
    ot, eos = tables
    n = 1 << 24
    g = torch.Generator(device="cuda")
    g.manual_seed(2609)
    rho_d, T_d = wl.c3_inputs(n, g, "cuda")   # the benchmark's inputs
    rho_h, T_h = rho_d.cpu().numpy(), T_d.cpu().numpy()
    del rho_d, T_d
    # the energies from the oracle's table (nothing from the GPU enters the oracle)
    _, e_h, _ = ot.eval_rhoT_n(rho_h, T_h)
    rho, e = torch.from_numpy(rho_h).cuda(), torch.from_numpy(e_h).cuda()
    outs = []
    for mode in (tde.INVERT_BISECT, tde.INVERT_BISECT_PLAIN):
        T, P, c2 = (torch.empty_like(rho) for _ in range(3))
        eos.invert(rho, e, T=T, P=P, cs2=c2, mode=mode)
        outs.append((T, P, c2))
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    rng = np.random.default_rng(5)
    idx = rng.integers(0, n, 2000)
    Tg, Pg = outs[0][0][idx].cpu().numpy(), outs[0][1][idx].cpu().numpy()
    for q in range(len(idx)):
        want = ot.invert(rho_h[idx[q]], e_h[idx[q]])
        assert Tg[q] == pytest.approx(want[0], rel=1e-12)
        assert Pg[q] == pytest.approx(want[1], rel=1e-12)


def sampled_stage(P, sample, dtb):
    """One stage of the sampled blocks on both sides from the same input."""
    om, gm = P.om, P.gm
    U0 = P.U.copy()
    om.ghost_fill(U0, ids=sample)
    O1 = om.new_state()
    om.stage(0, U0, U0, O1, dtb, np.zeros(P.nb), ids=sample)
    ids = torch.tensor(sample, dtype=torch.int32, device="cuda")
    gm.U.copy_(torch.from_numpy(P.U))
    gm.hydro_stage(0, torch.from_numpy(dtb).cuda(), torch.zeros(P.nb, dtype=torch.float64, device="cuda"), ids=ids,
                   bh=P.bh)
    G1 = P.gpu("U1")
    lay = P.layout
    for b in sample:
        flat, _ = lay.interior_index(b)
        px, py, pz = lay.pd[b]
        block = U0[:, lay.off[b]:lay.off[b + 1]].reshape(-1, pz, py, px)
        g = [lay.gofs(a) for a in range(3)]
        i0, j0, k0, nx, ny, nz = lay.blocks[b]
        scale = stencil_scale(block, lay.active, lay.ng)[:, g[2]:g[2] + nz, g[1]:g[1] + ny, g[0]:g[0] + nx]
        assert_parity_stencil(G1[:, flat], O1[:, flat], scale, STAGE_TOL, "block %d" % b)


def full_checks(P, n_lat, merge, sample, graph_window=True):
    dt = P.om.cfl_dt(P.U, 0.3, np.zeros(P.nb))
    fo, dt0, fmax = P.om.lat_factors(dt, n_lat, merge)
    fg, dt0g, fmaxg = P.gm.lat_assign(n_lat, 0.3, merge, bh=P.bh)
    assert np.array_equal(fg, fo) and fmaxg == fmax
    assert dt0g == pytest.approx(dt0, rel=1e-12)
    assert len(np.unique(fo)) >= 3
    sampled_stage(P, sample, fo * dt0)
    # a whole window in the benchmark's configuration (graph replay)
    P.gm.U.copy_(torch.from_numpy(P.U))
    P.gm.set_time(0.0)
    P.gm.counts(reset=True)
    P.gm.lat_set_factors(fo, dt0)
    P.gm.lat_window(bh=P.bh, use_graph=graph_window)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(P.gm.U).all())
    assert P.gm.counts()["nonfinite"] == 0
    assert P.gm.get_time() == pytest.approx(fmax * dt0, rel=1e-13)


def test_c4_full_size(oracle, tde, ctx, tables):
    ot, _ = tables
    lay, f, bhp = wl.stream_c4()
    assert lay.ncells == 13107200 and lay.nb == 512
    Pc, _, _ = ot.eval_rhoT_n(f["rho"] * wl.RHO0_CGS, f["T"])
    P_code = (Pc / (wl.RHO0_CGS * wl.V0_CGS ** 2)).reshape(f["rho"].shape)
    W = wl.prim_state(lay, f["rho"], f["vx"], f["vy"], f["vz"], P_code)
    del f, Pc, P_code
    bh = dict(on=1, excise=1, GM=bhp["GM"], r_soft=bhp["r_soft"], r_exc=bhp["r_exc"], x0=bhp["x0"])
    P = Pair(oracle, tde, ctx, lay, W, tables, bh=bh, eos=1, recon=1, dual=1, eta1=1e-3, eta2=1e-4,
             rho_floor=1e-17, p_floor=1e-30, u_floor=1.5e-30, unit_rho=wl.RHO0_CGS, unit_e=wl.V0_CGS ** 2)
    del W
    # sampled: a 16^3 block near pericentre, three 32^3 blocks across the grid
    small = [b for b in range(lay.nb) if lay.blocks[b][3] == 16]
    sample = [small[0], small[-1], 7, 300]
    full_checks(P, 5, 0.01, sample)


def test_c5_full_size(oracle, tde, ctx, tables):
    ot, eos = tables
    eos.reset_weights_for_training()
    eos.train(seed=2609, n_samples=1 << 20, epochs=30, batch=4096, lr=3e-3)
    floors = (1e-8, 1e-10)
    lay, f, bhp = wl.star_c5(seed=2609, rho_floor=floors[0], p_floor=floors[1])
    assert lay.ncells == 67108864 and lay.nb == 2048
    W = wl.prim_state(lay, f["rho"], f["vx"], f["vy"], f["vz"], f["P"])
    del f
    bh = dict(on=1, excise=1, GM=bhp["GM"], r_soft=bhp["r_soft"], r_exc=bhp["r_exc"], x0=bhp["x0"],
              v0=bhp["v0"])
    scheme = dict(eos=1, recon=1, dual=1, eta1=1e-3, eta2=1e-4, rho_floor=floors[0], p_floor=floors[1],
                  u_floor=1.5 * floors[1], unit_rho=wl.RHO0_CGS, unit_e=wl.V0_CGS ** 2)
    P = Pair(oracle, tde, ctx, lay, W, tables, bh=bh, **scheme)
    del W
    from test_gpu_hydro import SCHEME_KEYS
    P.gm.set_params(tde.make_params(eos_mode=tde.INVERT_SURROGATE,
                                    **{k: v for k, v in scheme.items() if k in SCHEME_KEYS}))
    # sampled: the block holding the star's centre, the point mass's block, two others
    def block_at(x):
        g = [int((x[a] - lay.xmin[a]) / lay.dx[a]) for a in range(3)]
        for b, (i0, j0, k0, nx, ny, nz) in enumerate(lay.blocks):
            if i0 <= g[0] < i0 + nx and j0 <= g[1] < j0 + ny and k0 <= g[2] < k0 + nz:
                return b
    sample = sorted({block_at((0.0, 0.0, 0.0)), block_at(bhp["x0"]), 5, 1500})
    full_checks(P, 6, 0.01, sample)
