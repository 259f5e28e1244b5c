"""Self-gravity (Sec. 3.2) on the GPU through the C ABI: the multigrid against
the oracle's (same V-cycles) and against the FFT solution of the discrete
periodic problem, and the hydro stage with the frozen potential (steps and a
LAT window with refluxing) against the oracle."""
import numpy as np
import pytest

from parity import assert_parity
from paper_2609_37859_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_hydro import Pair, STEPS_TOL, tde, ctx  # noqa: E402,F401

G = 1.0 / (4.0 * np.pi)


def periodic_pair(oracle, tde, ctx, N=(32, 32, 16), block=(16, 16, 8), **scheme):
    lay = wl.uniform_layout(N, block, domain=((0, 1), (0, 1), (0, 0.5)), bc=(1, 1, 1), ng=2)
    W = wl.random_smooth(lay, seed=17, drho=0.4, P0=1.0)
    return Pair(oracle, tde, ctx, lay, W, **scheme)


def oracle_phi(oracle, P, U, cycles, rho_min=0.0):
    rho = P.layout.to_global(U)[0]
    S = np.where(rho > rho_min, -4.0 * np.pi * G * rho, 0.0)
    phi, _, d = oracle.mg_solve(S, list(P.layout.dx), max_cycles=cycles, tol=0.0)
    return phi, d


def padded(oracle, P, phi):
    A = P.layout.from_global(phi[None])
    P.om.ghost_fill(A, nvar=1)
    return A[0]


def test_multigrid_matches_oracle_cycle_for_cycle(oracle, tde, ctx):
    P = periodic_pair(oracle, tde, ctx)
    for cycles in (1, 4):
        n, d = P.gm.gravity_solve(G, 0.0, tol=0.0, max_cycles=cycles, warm=False)
        phi_o, d_o = oracle_phi(oracle, P, P.U, cycles)
        phi_g = P.gm.gravity_phi().cpu().numpy()
        assert n == cycles
        assert np.allclose(phi_g, phi_o, rtol=0, atol=1e-12 * np.abs(phi_o).max())
        assert d == pytest.approx(d_o, rel=1e-8)


def test_multigrid_converges_to_fft_solution(oracle, tde, ctx):
    P = periodic_pair(oracle, tde, ctx)
    n, d = P.gm.gravity_solve(G, 0.0, tol=1e-11, max_cycles=30, warm=False)
    assert d < 1e-11 and n < 30
    rho = P.layout.to_global(P.U)[0]
    S = -4.0 * np.pi * G * rho
    S -= S.mean()
    dx = P.layout.dx
    nz, ny, nx = S.shape
    kk = [2 * np.pi * np.fft.fftfreq(m, d=h) for m, h in zip((nx, ny, nz), dx)]
    kz, ky, kx = np.meshgrid(kk[2], kk[1], kk[0], indexing="ij")
    lam = sum((2 - 2 * np.cos(k * h)) / h ** 2 for k, h in zip((kx, ky, kz), dx))
    lam[0, 0, 0] = 1.0
    Sh = np.fft.fftn(S)
    Sh[0, 0, 0] = 0.0
    exact = np.real(np.fft.ifftn(Sh / lam))
    phi = P.gm.gravity_phi().cpu().numpy()
    assert np.allclose(phi - phi.mean(), exact, rtol=0, atol=1e-8 * np.abs(exact).max())
    # warm start: already converged, no cycle needed
    n2, _ = P.gm.gravity_solve(G, 0.0, tol=1e-11, max_cycles=30, warm=True)
    assert n2 == 0


def test_steps_with_frozen_self_gravity(oracle, tde, ctx):
    P = periodic_pair(oracle, tde, ctx, dual=1, eta1=1e-3, eta2=1e-4)
    rho_min = 0.9
    P.gm.gravity_solve(G, rho_min, tol=0.0, max_cycles=6, warm=False)
    P.gm.gravity_enable(True)
    phi_o, _ = oracle_phi(oracle, P, P.U, 6, rho_min)
    P.om.set_phi_sg(padded(oracle, P, phi_o))
    U = P.U.copy()
    for _ in range(4):
        d = P.om.cfl_dt(U, 0.3).min()
        P.om.step(U, d, 0.0)
        P.gm.step(cfl=0.3)
    assert_parity(P.layout.to_global(P.gpu("U")), P.layout.to_global(U), STEPS_TOL, "self-gravity steps")
    # the potential matters: without it the result differs
    P.gm.gravity_enable(False)
    P.gm.U.copy_(torch.from_numpy(P.U))
    for _ in range(4):
        P.gm.step(cfl=0.3)
    assert np.abs(P.gpu("U") - P.layout.from_global(P.layout.to_global(U))).max() > 1e-6


def test_lat_window_with_frozen_self_gravity(oracle, tde, ctx):
    P = periodic_pair(oracle, tde, ctx, N=(32, 16, 16), block=(8, 8, 8), dual=1, eta1=1e-3, eta2=1e-4)
    P.gm.gravity_solve(G, 0.0, tol=0.0, max_cycles=6, warm=False)
    P.gm.gravity_enable(True)
    phi_o, _ = oracle_phi(oracle, P, P.U, 6)
    P.om.set_phi_sg(padded(oracle, P, phi_o))
    f = np.array([(1, 2, 4, 2)[(blk[0] // blk[3]) % 4] for blk in P.layout.blocks], dtype=np.int32)
    dt0 = 0.4 * P.om.cfl_dt(P.U, 0.3).min() / f.max()
    U = P.U.copy()
    P.gm.set_time(0.0)
    P.gm.lat_set_factors(f, dt0)
    P.om.lat_window(U, f, dt0, 0.0)
    P.gm.lat_window()
    G0 = P.layout.to_global(P.U)
    G1 = P.layout.to_global(P.gpu("U"))
    assert_parity(G1, P.layout.to_global(U), 1e-11, "self-gravity LAT window")
    # mass and momentum-free refluxing keep the totals (no point mass: momentum
    # changes only through the self-gravity force, mass exactly conserved)
    assert abs(G1[0].sum() - G0[0].sum()) <= 1e-14 * G0[0].sum()


def test_gravity_needs_periodic_power_of_two(tde, ctx):
    lay = wl.uniform_layout((16, 16, 16), (8, 8, 8), bc=(0, 0, 0), ng=2)
    m = tde.Mesh(ctx, lay, tde.make_params())
    with pytest.raises(tde.TDEError) as ei:
        m.gravity_solve(G, 0.0)
    assert ei.value.code == tde.TDE_EINVAL
    with pytest.raises(tde.TDEError):
        m.gravity_enable(True)


# ------------------------------------------- isolated boundaries and FMG ----

def isolated_pair(oracle, tde, ctx, n=32, **scheme):
    lay = wl.uniform_layout((n, n, n), (16, 16, 16), domain=((-1, 1),) * 3, bc=(0, 0, 0), ng=2)
    x, y, z = lay.cell_centres()
    rho = (1e-3 + np.exp(-((x - 0.2) ** 2 + (y + 0.1) ** 2 + (z - 0.05) ** 2) / (2 * 0.15 ** 2)) +
           0.6 * np.exp(-((x + 0.25) ** 2 + (y - 0.2) ** 2 + (z + 0.1) ** 2) / (2 * 0.1 ** 2)))
    W = wl.prim_state(lay, rho, 0.0, 0.0, 0.0, 0.1 * rho)
    return Pair(oracle, tde, ctx, lay, W, **scheme)


def oracle_phi_iso(oracle, P, cycles, fmg, lmax=4, rho_min=0.0):
    rho = P.layout.to_global(P.U)[0]
    S = np.where(rho > rho_min, -4.0 * np.pi * G * rho, 0.0)
    return oracle.mg_solve_bc(S, list(P.layout.dx), xmin=P.layout.xmin, isolated=True, lmax=lmax, fmg=fmg,
                              max_cycles=cycles, tol=0.0)


@pytest.mark.parametrize("fmg", [False, True])
def test_isolated_multigrid_matches_oracle_cycle_for_cycle(oracle, tde, ctx, fmg):
    P = isolated_pair(oracle, tde, ctx)
    for cycles in (0, 1, 3) if fmg else (1, 3):
        n, d = P.gm.gravity_solve(G, 0.0, tol=0.0, max_cycles=cycles, warm=False, isolated=True, lmax=4, fmg=fmg)
        phi_o, _, d_o, _, _ = oracle_phi_iso(oracle, P, cycles, fmg)
        phi_g = P.gm.gravity_phi().cpu().numpy()
        assert n == cycles
        assert np.allclose(phi_g, phi_o, rtol=0, atol=1e-12 * np.abs(phi_o).max()), cycles
        assert d == pytest.approx(d_o, rel=1e-7)


def test_isolated_full_multigrid_convergence(oracle, tde, ctx):
    """From the full-multigrid start a handful of V-cycles reach 1e-12 of the
    source's scale (the paper: five V-cycles to 1e-12, contraction about 0.1)."""
    P = isolated_pair(oracle, tde, ctx, n=64)
    n0, d0 = P.gm.gravity_solve(G, 0.0, tol=0.0, max_cycles=0, warm=False, isolated=True, fmg=True)
    n, d = P.gm.gravity_solve(G, 0.0, tol=1e-12, max_cycles=30, warm=False, isolated=True, fmg=True)
    print("isolated 64^3: defect after FMG %.2e, %d V-cycles to %.2e" % (d0, n, d))
    assert d < 1e-12 and n <= 9


def test_steps_with_isolated_self_gravity(oracle, tde, ctx):
    """The hydro stage with the isolated potential, ghosts beyond the outflow
    boundary taking the expansion at their centres, against the oracle."""
    P = isolated_pair(oracle, tde, ctx, dual=1, eta1=1e-3, eta2=1e-4)
    P.gm.gravity_solve(G, 0.0, tol=0.0, max_cycles=8, warm=False, isolated=True, fmg=True)
    P.gm.gravity_enable(True)
    lay = P.layout
    # the oracle's padded potential: interior and in-domain ghosts from the solve,
    # ghosts beyond the boundary from the expansion
    ghosts = []
    for b in range(lay.nb):
        i0, j0, k0, nx, ny, nz = lay.blocks[b]
        px, py, pz = lay.pd[b]
        k, j, i = np.meshgrid(np.arange(pz), np.arange(py), np.arange(px), indexing="ij")
        gi, gj, gk = i0 + i - 2, j0 + j - 2, k0 + k - 2
        out = (gi < 0) | (gj < 0) | (gk < 0) | (gi >= lay.N[0]) | (gj >= lay.N[1]) | (gk >= lay.N[2])
        flat = lay.off[b] + (k * py + j) * px + i
        xs = np.stack([lay.xmin[0] + (gi + 0.5) * lay.dx[0], lay.xmin[1] + (gj + 0.5) * lay.dx[1],
                       lay.xmin[2] + (gk + 0.5) * lay.dx[2]], axis=-1)
        ghosts.append((flat[out], xs[out]))
    gq = np.concatenate([g[1] for g in ghosts])
    rho = lay.to_global(P.U)[0]
    phi_o, _, _, _, phiq = oracle.mg_solve_bc(-4.0 * np.pi * G * rho, list(lay.dx), xmin=lay.xmin, isolated=True,
                                              lmax=4, fmg=True, max_cycles=8, tol=0.0, query=gq)
    A = padded(oracle, P, phi_o)
    A[np.concatenate([g[0] for g in ghosts])] = phiq
    P.om.set_phi_sg(A)
    U = P.U.copy()
    for _ in range(3):
        d = P.om.cfl_dt(U, 0.3).min()
        P.om.step(U, d, 0.0)
        P.gm.step(cfl=0.3)
    assert_parity(lay.to_global(P.gpu("U")), lay.to_global(U), STEPS_TOL, "isolated self-gravity steps")


def test_isolated_argument_checks(tde, ctx):
    lay = wl.uniform_layout((16, 16, 16), (8, 8, 8), bc=(0, 0, 0), ng=2)
    m = tde.Mesh(ctx, lay, tde.make_params())
    with pytest.raises(tde.TDEError):
        m.gravity_solve(G, 0.0, isolated=True, lmax=5)
    m.gravity_solve(G, 0.0, isolated=True, lmax=2, max_cycles=2)   # outflow mesh, isolated: fine
    lay = wl.uniform_layout((24, 16, 16), (8, 8, 8), bc=(0, 0, 0), ng=2)
    m = tde.Mesh(ctx, lay, tde.make_params())
    with pytest.raises(tde.TDEError):
        m.gravity_solve(G, 0.0, isolated=True)   # 24 is not a power of two


def test_isolated_two_dimensional_grid(oracle, tde, ctx):
    """A one-cell-thick grid (z inactive: no faces, no weight along z) against the oracle."""
    lay = wl.uniform_layout((32, 32, 1), (16, 16, 1), domain=((-1, 1), (-1, 1), (0, 0.0625)), bc=(0, 0, 0), ng=2)
    x, y, z = lay.cell_centres()
    rho = 1e-3 + np.exp(-((x - 0.2) ** 2 + (y + 0.1) ** 2) / (2 * 0.2 ** 2))
    P = Pair(oracle, tde, ctx, lay, wl.prim_state(lay, rho, 0.0, 0.0, 0.0, 0.1 * rho))
    for fmg, cycles in ((True, 0), (True, 2), (False, 3)):
        n, d = P.gm.gravity_solve(G, 0.0, tol=0.0, max_cycles=cycles, warm=False, isolated=True, lmax=3, fmg=fmg)
        phi_o, _, d_o, _, _ = oracle_phi_iso(oracle, P, cycles, fmg, lmax=3)
        phi_g = P.gm.gravity_phi().cpu().numpy()
        assert np.allclose(phi_g, phi_o, rtol=0, atol=1e-12 * np.abs(phi_o).max())
        assert d == pytest.approx(d_o, rel=1e-7)
