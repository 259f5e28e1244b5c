"""The persistent form of a LAT level sub-step (Sec. 7.1): every phase of a level
sub-step inside one cooperative launch with grid barriers.  Its results must
be those of the launch sequence bit for bit (which the LAT parity tests pin to
the oracle), with either sweep staging path, eagerly and replayed as a graph;
a barrier whose wait runs out must end the launch and be reported, not hang."""
import numpy as np
import pytest

from parity import assert_parity
from paper_2609_37859_gb300 import workloads as wl
from test_gpu_hydro import Pair  # noqa: F401

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_hydro import tde, ctx, tables  # noqa: E402,F401
from test_gpu_lat import band_factors  # noqa: E402


def windows(P, f, dt0, mode, n=3, use_graph=False):
    """n windows from P's start in the given mode; the state and the counters."""
    assert P.gm.set_lat_mode(mode) == (mode == P.tde.LAT_PERSISTENT)
    P.gm.U.copy_(torch.from_numpy(P.U))
    P.gm.set_time(0.0)
    P.gm.counts(reset=True)
    P.gm.lat_set_factors(f, dt0)
    for _ in range(n):
        P.gm.lat_window(bh=P.bh, use_graph=use_graph)
    U = P.gpu("U")
    P.gm.check()
    return U, P.gm.counts(reset=True)


def smooth(oracle, tde, ctx, block, n=(32, 16, 16), ng=2, recon=0):
    lay = wl.uniform_layout(n, block, bc=(1, 1, 1), ng=ng)
    bh = dict(on=1, GM=0.02, r_soft=0.1, x0=(0.5, 0.25, 0.25), v0=(0.2, 0.1, 0.0))
    return Pair(oracle, tde, ctx, lay, wl.random_smooth(lay, seed=31, P0=2.0), bh=bh, recon=recon, dual=1,
                eta1=1e-3, eta2=1e-4)


@pytest.mark.parametrize("block,ng,recon", [((8, 8, 8), 2, 0),    # TMA staging (padded x width 12)
                                            ((8, 8, 8), 3, 1),    # PPM, odd ghost width (TMA, shifted rows)
                                            ((7, 8, 8), 2, 0)])   # copy loop (padded x width 11)
def test_persistent_level_equals_launch_sequence(oracle, tde, ctx, block, ng, recon):
    n = (4 * block[0], 16, 16)
    P = smooth(oracle, tde, ctx, block, n, ng, recon)
    f = band_factors(P.layout, (1, 2, 4, 2))
    dt0 = 0.4 * P.om.cfl_dt(P.U, 0.3).min() / f.max()
    A, ca = windows(P, f, dt0, tde.LAT_SEQUENCE)
    B, cb = windows(P, f, dt0, tde.LAT_PERSISTENT)
    C, cc = windows(P, f, dt0, tde.LAT_PERSISTENT, use_graph=True)
    assert np.array_equal(A, B) and np.array_equal(A, C)
    assert ca == cb == cc
    # and the oracle's three windows
    U = P.U.copy()
    t = 0.0
    for _ in range(3):
        fmax, _ = P.om.lat_window(U, f, dt0, t)
        t += fmax * dt0
    assert_parity(P.layout.to_global(B), P.layout.to_global(U), 3e-11, "persistent LAT windows")


def test_persistent_level_table_eos_bh_excision_mixed_blocks(oracle, tde, ctx, tables):
    """Mixed 8^3 / 4^3 blocks, PPM, Saha table, dual energy, moving point mass
    with excision, factors from the CFL assignment: plain and FP32-guided
    bisection, the same bits and the same counted events as the sequence."""
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
    P = Pair(oracle, tde, ctx, lay, W, tables, bh=bh, **scheme)
    fg, dt0, fmax = P.gm.lat_assign(4, 0.3, 0.0, bh=P.bh)
    assert fmax > 1
    for mode in (tde.INVERT_BISECT, tde.INVERT_BISECT_PLAIN):
        P.gm.set_params(tde.make_params(eos_mode=mode, **scheme))
        A, ca = windows(P, fg, dt0, tde.LAT_SEQUENCE, n=2)
        B, cb = windows(P, fg, dt0, tde.LAT_PERSISTENT, n=2, use_graph=True)
        assert np.array_equal(A, B), mode
        assert ca == cb and ca["excised"] > 0 and ca["nonfinite"] == 0
    # the learned-guess closure keeps the launch sequence
    P.gm.set_params(tde.make_params(eos_mode=tde.INVERT_SURROGATE, **scheme))
    assert P.gm.set_lat_mode(tde.LAT_PERSISTENT) is False


def test_persistent_level_launch_count(oracle, tde, ctx):
    """One launch per level sub-step (and its barrier reset, a memset); what
    remains outside is the completion work (refluxing, and the dual-energy
    resync with its ghost fill of the auxiliary energy at each of the f_max
    completing sub-steps)."""
    P = smooth(oracle, tde, ctx, (8, 8, 8))
    f = band_factors(P.layout, (1, 2, 4, 2))
    dt0 = 0.4 * P.om.cfl_dt(P.U, 0.3).min() / f.max()
    P.gm.set_lat_mode(tde.LAT_PERSISTENT)
    P.gm.lat_set_factors(f, dt0)
    P.ctx.profile(True)
    P.gm.lat_window(bh=P.bh)
    k = P.ctx.profile_read()
    P.ctx.profile(False)
    sub_steps = sum(4 // lv for lv in (1, 2, 4))   # f_max = 4: levels 1, 2, 4
    assert k["lat_level"][0] == sub_steps
    assert k["sweep_x"][0] == k["sweep_y"][0] == k["sweep_z"][0] == k["c2p"][0] == 0
    assert k["ghost"][0] == k["sync"][0] == 4


def test_persistent_mode_applies_only_where_admitted(oracle, tde, ctx):
    """2-D meshes and refined meshes keep the launch sequence (a window there
    gives the sequence's bits in either mode); an unknown mode is refused."""
    from test_gpu_smr import smr, smooth_W
    lay2 = wl.uniform_layout((32, 32, 1), (16, 16, 1), bc=(1, 1, 1), ng=2)
    Q = Pair(oracle, tde, ctx, lay2, wl.random_smooth(lay2, seed=3, P0=2.0), dual=1)
    assert Q.gm.set_lat_mode(tde.LAT_PERSISTENT) is False
    lay3 = smr(r=0.1)
    R = Pair(oracle, tde, ctx, lay3, smooth_W(lay3), dual=1, eta1=1e-3, eta2=1e-4)
    f, dt0, fmax = R.gm.lat_assign(3, 0.3, 0.0)
    assert fmax > 1
    outs = []
    for mode in (tde.LAT_SEQUENCE, tde.LAT_PERSISTENT):
        assert R.gm.set_lat_mode(mode) is False
        R.gm.U.copy_(torch.from_numpy(R.U))
        R.gm.set_time(0.0)
        R.gm.lat_set_factors(f, dt0)
        R.gm.lat_window()
        outs.append(R.gpu("U"))
    assert np.array_equal(outs[0], outs[1])
    P = smooth(oracle, tde, ctx, (8, 8, 8))
    assert P.gm.set_lat_mode(tde.LAT_PERSISTENT) is True
    assert P.gm.set_lat_mode(tde.LAT_SEQUENCE) is False
    with pytest.raises(tde.TDEError):
        P.gm.set_lat_mode(7)


def test_persistent_level_barrier_expiry_is_reported_not_hung(oracle, tde, ctx):
    """The test hook keeps CTA 0 from arriving at the first grid barrier: every
    CTA's wait there runs out after one second, the launch ends, and
    TDE_ETIMEOUT is reported once; the context stays usable and the next window
    equals the launch sequence's."""
    P = smooth(oracle, tde, ctx, (8, 8, 8))
    ones = np.ones(P.nb, dtype=np.int32)
    dt0 = 0.4 * P.om.cfl_dt(P.U, 0.3).min()
    A, _ = windows(P, ones, dt0, tde.LAT_SEQUENCE, n=1)
    P.gm.set_lat_mode(tde.LAT_PERSISTENT)
    P.gm.U.copy_(torch.from_numpy(P.U))
    P.gm.set_time(0.0)
    P.gm.lat_set_factors(ones, dt0)
    P.gm.inject_barrier_drop(True)
    P.gm.lat_window(bh=P.bh)        # one level sub-step: one launch, one expiry
    torch.cuda.synchronize()
    with pytest.raises(tde.TDEError) as ei:
        P.gm.check()
    assert ei.value.code == tde.TDE_ETIMEOUT
    P.gm.check()                    # reported once
    P.gm.inject_barrier_drop(False)
    B, _ = windows(P, ones, dt0, tde.LAT_PERSISTENT, n=1)
    assert np.array_equal(A, B)
