"""The learned-guess closure inside the hydro stage: with the table inverted by
the network's guess + one FP64 Newton step (+ bisection of the cells it does
not settle) the stage gives the same bits as with table bisection, FP32-guided
or plain -- for synchronised steps and for LAT windows (whose slow blocks
convert their padded cells)."""
import numpy as np
import pytest

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


def test_surrogate_closure_needs_a_network(tde, ctx, tables):
    lay = wl.uniform_layout((8, 8, 8), (8, 8, 8), bc=(1, 1, 1), ng=2)
    tables[1].reset_weights_for_training()   # no network
    m = tde.Mesh(ctx, lay, tde.make_params(eos=1, eos_mode=tde.INVERT_SURROGATE, rho_floor=1e-20,
                                           p_floor=1e-20), tables[1])
    with pytest.raises(tde.TDEError):
        m.step(dt=1e-3)
