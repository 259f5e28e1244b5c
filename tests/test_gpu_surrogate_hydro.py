"""The learned-guess closure inside the hydro stage: with the table inverted by
the network's guess + one FP64 Newton step (+ bisection of the cells it does
not settle) the stage gives the same bits as with table bisection, FP32-guided
or plain -- for synchronised steps and for LAT windows (whose slow blocks
convert their padded cells)."""
import numpy as np
import pytest

from parity import assert_parity
from paper_2609_37859_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_hydro import Pair, SCHEME_KEYS, c2_pair, tde, ctx, tables  # noqa: E402,F401

MODES = ("INVERT_BISECT", "INVERT_BISECT_PLAIN", "INVERT_SURROGATE")


@pytest.fixture(scope="module")
def trained_tables(tde, tables):
    tables[1].reset_weights_for_training()
    tables[1].train(seed=77, n_samples=1 << 20, epochs=30, batch=4096, lr=3e-3)
    return tables


def with_mode(tde, P, scheme, mode):
    kw = {k: v for k, v in scheme.items() if k in SCHEME_KEYS}
    P.gm.set_params(tde.make_params(eos_mode=getattr(tde, mode), **kw))


def test_closure_modes_identical_c2(oracle, tde, ctx, trained_tables):
    P, _ = c2_pair(oracle, tde, ctx, trained_tables, 64, 32, seed=11)
    scheme = dict(eos=1, dual=1, eta1=1e-3, eta2=1e-4, rho_floor=1e-20, p_floor=1e-20, u_floor=1e-20)
    outs, counts = {}, {}
    for mode in MODES:
        with_mode(tde, P, scheme, mode)
        P.gm.U.copy_(torch.from_numpy(P.U))
        P.gm.set_time(0.0)
        P.gm.counts(reset=True)
        dts = []
        for _ in range(3):
            dt = torch.zeros(1, dtype=torch.float64, device="cuda")
            P.gm.step(cfl=0.3, dt_out=dt)
            dts.append(float(dt))
        outs[mode] = (P.gpu("U").copy(), dts)
        counts[mode] = P.gm.counts()
    for mode in MODES[1:]:
        assert np.array_equal(outs[mode][0], outs["INVERT_BISECT"][0]), mode
        assert outs[mode][1] == outs["INVERT_BISECT"][1], mode
    acc = counts["INVERT_SURROGATE"].pop("surrogate_accepted")
    ncell = 64 ** 3 * 2 * 3
    print("surrogate acceptance in the hydro closure", acc / ncell)
    assert acc > 0.5 * ncell
    counts["INVERT_BISECT"].pop("surrogate_accepted")
    assert counts["INVERT_SURROGATE"] == counts["INVERT_BISECT"]


def test_closure_modes_identical_lat_window(oracle, tde, ctx, trained_tables):
    """Mixed 8^3 / 4^3 blocks, PPM, point mass with excision, factors (1, 2, 4): the
    slow blocks convert all padded cells (time-interpolated ghosts)."""
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
    scheme = dict(eos=1, recon=1, dual=1, eta1=1e-3, eta2=1e-4, rho_floor=1e-10, p_floor=1e-16,
                  u_floor=1.5e-16, unit_rho=rho0, unit_e=v0 * v0)
    P = Pair(oracle, tde, ctx, lay, W, trained_tables, bh=bh, **scheme)
    f = np.array([(1, 2, 4)[b % 3] for b in range(lay.nb)], dtype=np.int32)
    outs = {}
    for mode in MODES:
        with_mode(tde, P, scheme, mode)
        P.gm.U.copy_(torch.from_numpy(P.U))
        P.gm.set_time(0.0)
        P.gm.lat_set_factors(f, 2e-4)
        for use_graph in (False, True):
            P.gm.lat_window(bh=P.bh, use_graph=use_graph)
        outs[mode] = P.gpu("U").copy()
    for mode in MODES[1:]:
        assert np.array_equal(outs[mode], outs["INVERT_BISECT"]), mode


def test_surrogate_closure_needs_a_network(tde, ctx):
    from test_gpu_hydro import TABLE_FILE
    lay = wl.uniform_layout((8, 8, 8), (8, 8, 8), bc=(1, 1, 1), ng=2)
    fresh = tde.EOS.from_file(ctx, TABLE_FILE)   # no network
    m = tde.Mesh(ctx, lay, tde.make_params(eos=1, eos_mode=tde.INVERT_SURROGATE, rho_floor=1e-20,
                                           p_floor=1e-20), fresh)
    for call in (lambda: m.step(dt=1e-3), lambda: m.lat_assign(3, 0.3)):
        with pytest.raises(tde.TDEError) as ei:
            call()
        assert ei.value.code == tde.TDE_EINVAL


def test_c5_like_star_lat_surrogate_parity(oracle, tde, ctx, trained_tables):
    """Reduced production-shaped run: a stretched n = 1.5 polytrope passing a
    moving point mass with excision, PPM, Saha table in code units, dual energy,
    the learned-guess closure, factors on 6 levels from the CFL assignment;
    two LAT windows against the oracle (which inverts the table by its own
    bisection)."""
    # a resolved star (transverse radius ~3.4 cells) and floors 10^-4 / 10^-6: at
    # this size the paper's floors leave a 10^11 density jump across a cell or two
    lay, f, bhp = wl.star_c5(n_blocks=(4, 4, 2), block=8, half_rsun=(4.0, 4.0, 2.0),
                             bh_at_rsun=(3.0, 2.5, 0.0), stretch=2.0, r_star_rsun=1.2, inflow_rsun=1.5,
                             rho_floor=1e-4, p_floor=1e-6, seed=5)
    W = wl.prim_state(lay, f["rho"], f["vx"], f["vy"], f["vz"], f["P"])
    bh = dict(on=1, excise=1, GM=bhp["GM"], r_soft=bhp["r_soft"], r_exc=bhp["r_exc"], x0=bhp["x0"],
              v0=bhp["v0"])
    scheme = dict(eos=1, recon=1, dual=1, eta1=1e-3, eta2=1e-4, rho_floor=1e-4, p_floor=1e-6,
                  u_floor=1.5e-6, unit_rho=wl.RHO0_CGS, unit_e=wl.V0_CGS ** 2)
    P = Pair(oracle, tde, ctx, lay, W, trained_tables, bh=bh, **scheme)
    with_mode(tde, P, scheme, "INVERT_SURROGATE")
    U = P.U.copy()
    t = 0.0
    P.gm.set_time(0.0)
    P.gm.counts(reset=True)
    for w in range(2):
        dt = P.om.cfl_dt(U, 0.3, np.full(P.nb, t))
        fo, dt0, fmax = P.om.lat_factors(dt, 6, 0.0)
        fg, dt0g, fmaxg = P.gm.lat_assign(6, 0.3, 0.0, bh=P.bh)
        assert np.array_equal(fg, fo) and fmaxg == fmax
        P.om.lat_window(U, fo, dt0, t)
        P.gm.lat_window(bh=P.bh, use_graph=(w == 1))
        t += fmax * dt0
    assert len(np.unique(fo)) >= 3
    assert_parity(lay.to_global(P.gpu("U")), lay.to_global(U), 1e-10, "C5-like LAT, learned closure")
    c = P.gm.counts()
    assert c["nonfinite"] == 0 and c["surrogate_accepted"] > 0
