"""Pins of the oracle's localized adaptive time stepping (Sec. 7).

- Eq. lat-factor, bin merging and neighbour limiting against brute force;
- LAT with every factor 1 is the synchronised update, bit for bit (Sec. 7.1,
  last paragraph: "reduces to the standard update when all factors are unity");
- with mixed factors the refluxing keeps mass, momentum and energy conserved to
  roundoff at the window end, and with a static point mass it keeps
  sum(E + rho Phi) conserved (Eq. lat-grav-reflux);
- LAT stays close to the synchronised run on a smooth flow (the density-norm
  metrics of Eq. lat-density-error-norms).
"""
import itertools

import numpy as np
import pytest

from paper_2609_37859_gb300 import workloads as wl


def block_grid_neighbours(nbx, periodic):
    """Face/edge/corner adjacency of a lexicographic block grid (x fastest)."""
    idx = lambda i, j, k: (k * nbx[1] + j) * nbx[0] + i
    nb = nbx[0] * nbx[1] * nbx[2]
    adj = [set() for _ in range(nb)]
    for k, j, i in itertools.product(range(nbx[2]), range(nbx[1]), range(nbx[0])):
        for dk, dj, di in itertools.product((-1, 0, 1), repeat=3):
            c = [i + di, j + dj, k + dk]
            ok = True
            for a in range(3):
                if c[a] < 0 or c[a] >= nbx[a]:
                    if periodic[a]:
                        c[a] %= nbx[a]
                    else:
                        ok = False
            if ok and idx(*c) != idx(i, j, k):
                adj[idx(i, j, k)].add(idx(*c))
    return adj


def brute_factors(dt, n_lat, merge_frac, adj):
    dt0 = dt.min()
    f = np.zeros(len(dt), dtype=np.int64)
    for b, d in enumerate(dt):
        k = 0
        while k < n_lat and 2.0 ** (k + 1) <= d / dt0:
            k += 1
        f[b] = 2 ** k
    while f.max() > 1 and (f == f.max()).sum() < merge_frac * len(f):
        f[f == f.max()] //= 2
    changed = True
    while changed:
        changed = False
        for b in range(len(f)):
            lim = 2 * min(f[n] for n in adj[b])
            if f[b] > lim:
                f[b] = lim
                changed = True
    return f, dt0


@pytest.mark.parametrize("seed", range(6))
def test_factors_brute_force(oracle, seed):
    nbx = (4, 3, 2)
    periodic = (seed % 2 == 0, True, seed % 3 == 0)
    lay = wl.uniform_layout((16, 12, 8), (4, 4, 4), bc=tuple(int(x) for x in periodic), ng=2)
    m = oracle.Mesh(lay, oracle.make_params())
    rng = np.random.default_rng(seed)
    dt = 10 ** rng.uniform(-3, -1, lay.nb)
    dt[rng.integers(0, lay.nb)] = 1e-3 * 0.999
    n_lat = 2 + seed % 4
    f, dt0, fmax = m.lat_factors(dt, n_lat, 0.1)
    fb, dt0b = brute_factors(dt, n_lat, 0.1, block_grid_neighbours(nbx, periodic))
    assert dt0 == dt0b
    assert np.array_equal(f, fb), (f, fb)
    assert fmax == fb.max()
    assert f.max() <= 2 ** n_lat


def test_factor_exact_powers_of_two(oracle):
    """dt_b / dt0 exactly 2^k gives f = 2^k (floor(log2) is exact at the boundary)."""
    lay = wl.uniform_layout((8, 8, 8), (4, 8, 8), bc=(0, 0, 0), ng=2)
    m = oracle.Mesh(lay, oracle.make_params())
    f, dt0, fmax = m.lat_factors(np.array([1.0, 2.0]), 5, 0.0)
    assert list(f) == [1, 2]
    f, dt0, fmax = m.lat_factors(np.array([1.0, np.nextafter(2.0, 0)]), 5, 0.0)
    assert list(f) == [1, 1]


def smooth_mesh(oracle, bh=False, dual=1, recon=0):
    lay = wl.uniform_layout((16, 16, 8), (4, 4, 4), bc=(1, 1, 1), ng=2 + recon)
    kw = dict(dual=dual, recon=recon, eta1=1e-3, eta2=1e-4)
    if bh:
        kw.update(bh_on=1, GM=0.02, r_soft=0.1, bh_x0=(0.5, 0.5, 0.25))
    m = oracle.Mesh(lay, oracle.make_params(**kw))
    U = m.prim_to_cons(wl.random_smooth(lay, seed=21, P0=2.0))
    return lay, m, U


def test_all_factors_one_is_the_synchronised_step(oracle):
    lay, m, U = smooth_mesh(oracle, bh=True, recon=1)
    p = m.params
    p.excision_on = 1
    p.r_exc = 0.08
    m.set_params(p)
    dt = 0.5 * m.cfl_dt(U, 0.3).min()
    A = U.copy()
    B = U.copy()
    m.step(A, dt, 0.1)
    fmax, upd = m.lat_window(B, np.ones(lay.nb, dtype=np.int32), dt, 0.1)
    assert fmax == 1 and upd == lay.nb
    assert np.array_equal(A, B)


def band_factors(lay, levels):
    """Factors by block z-layer and x column, neighbours differing by at most 2."""
    f = np.ones(lay.nb, dtype=np.int32)
    for b, blk in enumerate(lay.blocks):
        ix = blk[0] // blk[3]
        f[b] = levels[ix % len(levels)]
    return f


@pytest.mark.parametrize("levels", [(1, 2), (1, 2, 4, 2), (4, 2, 2, 1)])
def test_mixed_factors_conserve_mass_momentum_energy(oracle, levels):
    lay, m, U = smooth_mesh(oracle)
    f = band_factors(lay, levels)
    dt0 = 0.5 * m.cfl_dt(U, 0.3).min() / f.max()
    G0 = m.interior(U).reshape(m.nvar, -1)
    fmax, upd = m.lat_window(U, f, dt0, 0.0)
    assert fmax == max(levels)
    assert upd == int(sum(fmax // f))
    G1 = m.interior(U).reshape(m.nvar, -1)
    for v in range(5):
        scale = np.abs(G1[v]).sum()
        assert abs(G1[v].sum() - G0[v].sum()) <= 4e-15 * scale, (v, (G1[v].sum() - G0[v].sum()) / scale)


def test_mixed_factors_without_reflux_would_not_conserve(oracle):
    """Control: the same window with the slow side's correction removed changes the
    total mass at first order (so the conservation pin above is not vacuous)."""
    lay, m, U = smooth_mesh(oracle)
    f = band_factors(lay, (1, 2))
    dt0 = 0.5 * m.cfl_dt(U, 0.3).min() / 2
    # two synchronised-in-time but factor-mixed sub-steps built from stages only:
    # advance factor-2 blocks by 2 dt0 with frozen neighbours and factor-1 blocks by
    # two dt0 steps, no refluxing
    U2 = U.copy()
    nb = lay.nb
    slow = [b for b in range(nb) if f[b] == 2]
    fast = [b for b in range(nb) if f[b] == 1]
    S = m.new_state()
    m.ghost_fill(U2)
    dts = np.full(nb, 2 * dt0)
    m.stage(0, U2, U2, S, dts, np.zeros(nb), ids=slow)
    m.ghost_fill(S, ids=slow)
    m.stage(1, U2, S, U2, dts, np.zeros(nb), ids=slow)
    G0 = m.interior(U).reshape(m.nvar, -1)[0].sum()
    Gs = m.interior(U2).reshape(m.nvar, -1)[0].sum()
    assert abs(Gs - G0) > 1e-10 * abs(G0)


def test_mixed_factors_keep_E_plus_rho_phi_with_static_point_mass(oracle):
    lay, m, U = smooth_mesh(oracle, bh=True, dual=0)
    f = band_factors(lay, (1, 2, 4, 2))
    dt0 = 0.3 * m.cfl_dt(U, 0.3).min() / f.max()
    x, y, z = lay.cell_centres()
    phi = -0.02 / np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.25) ** 2 + 0.1 ** 2)
    G0 = m.interior(U)
    m.lat_window(U, f, dt0, 0.0)
    G1 = m.interior(U)
    W0 = (G0[4] + G0[0] * phi).sum()
    W1 = (G1[4] + G1[0] * phi).sum()
    scale = np.abs(G0[4]).sum() + np.abs(G0[0] * phi).sum()
    assert abs(W1 - W0) < 5e-15 * scale
    assert abs(G1[0].sum() - G0[0].sum()) < 4e-15 * G0[0].sum()


def lat_metrics(rho_lat, rho_sync, floor):
    """Eq. lat-density-error-norms, C_logrho and J_dense (Sec. 7.4)."""
    d = (rho_lat - rho_sync) / rho_sync
    L1, L2, Linf = np.mean(np.abs(d)), np.sqrt(np.mean(d * d)), np.max(np.abs(d))
    q1, q2 = np.log10(rho_lat), np.log10(rho_sync)
    C = np.sum((q1 - q1.mean()) * (q2 - q2.mean())) / np.sqrt(np.sum((q1 - q1.mean()) ** 2) *
                                                               np.sum((q2 - q2.mean()) ** 2))
    D1, D2 = rho_lat > 1e2 * floor, rho_sync > 1e2 * floor
    J = (D1 & D2).sum() / max((D1 | D2).sum(), 1)
    return L1, L2, Linf, C, J


def test_lat_close_to_synchronised_run(oracle):
    lay, m, U = smooth_mesh(oracle, dual=0)
    f = band_factors(lay, (1, 2))
    dt0 = 0.5 * m.cfl_dt(U, 0.3).min() / 2
    A = U.copy()
    B = U.copy()
    for w in range(4):
        m.lat_window(A, f, dt0, w * 2 * dt0)
        m.step(B, dt0, w * 2 * dt0)
        m.step(B, dt0, (w * 2 + 1) * dt0)
    L1, L2, Linf, C, J = lat_metrics(m.interior(A)[0], m.interior(B)[0], 1e-10)
    assert L1 < 1e-4 and Linf < 1e-3 and C > 0.9999 and J == 1.0
