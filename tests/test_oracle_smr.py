"""Pins of the oracle on statically refined meshes (LAT across coarse-fine
interfaces, Sec. 7.1): ghost cells of linear fields are exact, prolonged ghosts
average to their coarse parent, a uniform flow stays uniform, mass, momentum and
energy are conserved to rounding with the coarse-fine flux correction (in
synchronised steps and in LAT windows), the factor rules hold, and a Sod tube
across a refined band converges to the exact solution."""
import numpy as np
import pytest

from exact_riemann import sample
from paper_2609_37859_gb300 import workloads as wl

G53 = 5.0 / 3.0


def sphere(centre, r):
    def refine(lo, hi, L):
        d2 = sum(max(lo[a] - centre[a], 0.0, centre[a] - hi[a]) ** 2 for a in range(3))
        return d2 < r * r
    return refine


def smr3(bc=(1, 1, 1), ng=2, max_level=1, N=(16, 16, 16), block=(4, 4, 4), centre=(0.3, 0.4, 0.55), r=0.1,
         domain=((0, 1),) * 3):
    return wl.smr_layout(N, block, domain, bc, ng, sphere(centre, r), max_level)


def totals(lay, U):
    _, _, _, vol = lay.interior_centres()
    F = U[:, lay.interior_flat()]
    return (F[:5] * vol).sum(axis=1)


def smooth_state(lay, seed=3):
    rng = np.random.default_rng(seed)
    x, y, z, _ = lay.interior_centres()
    k = rng.integers(1, 3, (5, 3))
    ph = rng.uniform(0, 2 * np.pi, 5)
    f = [np.sin(2 * np.pi * (k[q, 0] * x + k[q, 1] * y + k[q, 2] * z) + ph[q]) for q in range(5)]
    return wl.prim_cells(lay, 1.0 + 0.3 * f[0], 0.4 * f[1], 0.3 * f[2], 0.2 * f[3], 1.0 + 0.25 * f[4])


def test_layout_is_balanced_and_validated(oracle):
    lay = smr3(max_level=2, r=0.08)
    assert lay.levels.max() == 2 and lay.levels.min() == 0
    oracle.Mesh(lay, oracle.make_params())
    # a level-2 block next to a level-0 block is rejected: the left half of an
    # 8 x 4 x 4 level-0 grid at level 0, the right half at level 2
    blocks = [(0, 0, 0, 4, 4, 4)] + [(16 + 8 * di, 8 * dj, 8 * dk, 8, 8, 8)
                                     for dk in (0, 1) for dj in (0, 1) for di in (0, 1)]
    bad = wl.MeshLayout(np.array(blocks, dtype=np.int32), (8, 4, 4), (0, 0, 0), (1 / 8, 1 / 4, 1 / 4),
                        (0, 0, 0), 2, np.array([0] + [2] * 8))
    with pytest.raises(ValueError):
        oracle.Mesh(bad, oracle.make_params())
    # the same split with the right half at level 1 is accepted
    blocks = [(0, 0, 0, 4, 4, 4)] + [(8 + 4 * di, 4 * dj, 4 * dk, 4, 4, 4)
                                     for dk in (0, 1) for dj in (0, 1) for di in (0, 1)]
    oracle.Mesh(wl.MeshLayout(np.array(blocks, dtype=np.int32), (8, 4, 4), (0, 0, 0), (1 / 8, 1 / 4, 1 / 4),
                              (0, 0, 0), 2, np.array([0] + [1] * 8)), oracle.make_params())


def ghost_cells(lay, b):
    """(flat indices, x, y, z) of block b's ghost cells."""
    i0, j0, k0, nx, ny, nz = lay.blocks[b]
    px, py, pz = lay.pd[b]
    g = [lay.gofs(a) for a in range(3)]
    k, j, i = np.meshgrid(np.arange(pz), np.arange(py), np.arange(px), indexing="ij")
    interior = ((i >= g[0]) & (i < g[0] + nx) & (j >= g[1]) & (j < g[1] + ny) & (k >= g[2]) & (k < g[2] + nz))
    d = lay.block_dx(b)
    x = lay.xmin[0] + (i0 + i - g[0] + 0.5) * d[0]
    y = lay.xmin[1] + (j0 + j - g[1] + 0.5) * d[1]
    z = lay.xmin[2] + (k0 + k - g[2] + 0.5) * d[2]
    flat = lay.off[b] + (k * py + j) * px + i
    sel = ~interior
    return flat[sel], x[sel], y[sel], z[sel]


def test_ghosts_of_linear_fields_are_exact(oracle):
    """Restriction (a mean of children) and minmod-limited linear prolongation
    reproduce a linear field exactly; away from the outflow boundary (where the
    clamp is not linear) every ghost cell equals the field at its centre."""
    lay = smr3(bc=(0, 0, 0), max_level=2, r=0.2, centre=(0.5, 0.45, 0.5))
    m = oracle.Mesh(lay, oracle.make_params(dual=1))
    x, y, z, _ = lay.interior_centres()
    coef = np.array([[1.0, 0.3, -0.2, 0.1], [0.5, -0.1, 0.4, 0.2], [-0.3, 0.2, 0.1, -0.5],
                     [0.2, 0.0, 0.3, 0.1], [3.0, 0.5, 0.2, -0.4], [2.0, -0.3, 0.1, 0.6]])
    U = lay.state_from_cells(np.stack([c[0] + c[1] * x + c[2] * y + c[3] * z for c in coef]))
    m.ghost_fill(U)
    checked = 0
    margin = 2.5 / 16
    for b in range(lay.nb):
        flat, gx, gy, gz = ghost_cells(lay, b)
        ok = ((gx > margin) & (gx < 1 - margin) & (gy > margin) & (gy < 1 - margin) & (gz > margin) &
              (gz < 1 - margin))
        for q, c in enumerate(coef):
            want = c[0] + c[1] * gx[ok] + c[2] * gy[ok] + c[3] * gz[ok]
            assert np.allclose(U[q, flat[ok]], want, rtol=0, atol=1e-13)
        checked += ok.sum()
    assert checked > 1000


def test_prolonged_ghosts_average_to_their_parent(oracle):
    """Each group of 2^d ghost cells of a fine block that fills one cell of a
    coarser block averages to that coarse cell's value (conservative
    prolongation), for a non-linear field."""
    lay = smr3(bc=(1, 1, 1), max_level=1, r=0.2)
    m = oracle.Mesh(lay, oracle.make_params())
    U = m.prim_to_cons(smooth_state(lay))
    m.ghost_fill(U)
    # the coarse (level-0) cell values on the level-0 grid
    N0 = lay.N
    coarse = {}
    for b in range(lay.nb):
        if lay.level(b) != 0:
            continue
        flat, (gk, gj, gi) = lay.interior_index(b)
        for f, k, j, i in zip(flat.ravel(), gk.ravel(), gj.ravel(), gi.ravel()):
            coarse[(i, j, k)] = U[:, f]
    groups = 0
    for b in range(lay.nb):
        if lay.level(b) != 1:
            continue
        i0, j0, k0, nx, ny, nz = lay.blocks[b]
        px, py, pz = lay.pd[b]
        sums = {}
        for k in range(pz):
            for j in range(py):
                for i in range(px):
                    if 2 <= i < 2 + nx and 2 <= j < 2 + ny and 2 <= k < 2 + nz:
                        continue
                    g = (i0 + i - 2, j0 + j - 2, k0 + k - 2)
                    par = tuple((g[a] // 2) % N0[a] for a in range(3))
                    if par not in coarse:
                        continue
                    s = sums.setdefault(par, [np.zeros(5), 0])
                    s[0] += U[:, lay.off[b] + (k * py + j) * px + i]
                    s[1] += 1
        for par, (s, n) in sums.items():
            if n == 8:
                assert np.allclose(s / 8, coarse[par], rtol=1e-14, atol=1e-15)
                groups += 1
    assert groups > 100


@pytest.mark.parametrize("max_level", [1, 2])
def test_uniform_flow_stays_uniform(oracle, max_level):
    lay = smr3(max_level=max_level, r=0.18)
    m = oracle.Mesh(lay, oracle.make_params(dual=1))
    n = lay.interior_flat().size
    U = m.prim_to_cons(wl.prim_cells(lay, np.full(n, 1.3), 0.7, -0.4, 0.2, 2.0))
    U0 = U.copy()
    dt = 0.5 * m.cfl_dt(U, 0.3).min()
    for s in range(4):
        m.step(U, dt, s * dt)
    F, F0 = U[:, lay.interior_flat()], U0[:, lay.interior_flat()]
    assert np.allclose(F, F0, rtol=1e-13, atol=1e-14)


def test_conservation_with_coarse_fine_correction(oracle):
    """Periodic refined mesh, smooth random state: the volume integrals of rho, m
    and E are conserved to rounding over synchronised steps and LAT windows."""
    lay = smr3(max_level=2, r=0.08)
    m = oracle.Mesh(lay, oracle.make_params(dual=1))
    U = m.prim_to_cons(smooth_state(lay))
    T0 = totals(lay, U)
    t = 0.0
    for s in range(3):
        dt = m.cfl_dt(U, 0.3, np.full(lay.nb, t)).min()
        m.step(U, dt, t)
        t += dt
    T1 = totals(lay, U)
    _, _, _, vol = lay.interior_centres()
    scale = (np.abs(U[:5, lay.interior_flat()]) * vol).sum(axis=1)
    print("relative change, synchronised steps", (T1 - T0) / scale)
    assert np.all(np.abs(T1 - T0) <= 1e-13 * scale)
    for w in range(2):
        dtb = m.cfl_dt(U, 0.3, np.full(lay.nb, t))
        f, dt0, fmax = m.lat_factors(dtb, 3, 0.0)
        assert fmax > 1 and len(set(f)) > 1
        m.lat_window(U, f, dt0, t)
        t += fmax * dt0
    T2 = totals(lay, U)
    print("relative change, LAT windows", (T2 - T0) / scale)
    assert np.all(np.abs(T2 - T0) <= 1e-13 * scale)


def neighbour_pairs(lay):
    """(b, o) for blocks sharing a face, edge or corner (periodic images in all
    directions, every level), from the finest-level owner lattice."""
    lmax = int(lay.levels.max())
    act = lay.active
    NF = [lay.N[a] << lmax if act[a] else 1 for a in range(3)]
    own = np.full(NF[::-1], -1)
    for b in range(lay.nb):
        i0, j0, k0, nx, ny, nz = lay.blocks[b]
        s = lmax - lay.level(b)
        own[k0 << s:(k0 + nz) << s, j0 << s:(j0 + ny) << s, i0 << s:(i0 + nx) << s] = b
    pairs = set()
    for b in range(lay.nb):
        i0, j0, k0, nx, ny, nz = lay.blocks[b]
        s = lmax - lay.level(b)
        idx = [np.arange((o - 1) << s, (o + n + 1) << s) % NF[a]
               for a, o, n in ((2, k0, nz), (1, j0, ny), (0, i0, nx))]
        for o in np.unique(own[np.ix_(*idx)]):
            if o != b:
                pairs.add((b, int(o)))
    return pairs


def test_lat_factor_rules_across_levels(oracle):
    lay = smr3(max_level=2, r=0.08)
    m = oracle.Mesh(lay, oracle.make_params())
    rng = np.random.default_rng(5)
    for trial in range(4):
        # coarse blocks slow, fine blocks fast, plus noise: the limits must bind
        dtb = np.array([8.0 ** (2 - lay.level(b)) * rng.uniform(0.5, 4.0) for b in range(lay.nb)])
        if trial == 3:
            dtb = np.array([rng.uniform(1, 64) for b in range(lay.nb)])   # arbitrary, incl. fine > coarse
        f, dt0, fmax = m.lat_factors(dtb, 6, 0.0)
        assert dt0 == dtb.min()
        # never above the CFL factor of Eq. lat-factor
        fcfl = 2 ** np.minimum(6, np.floor(np.log2(dtb / dt0)))
        assert np.all(f <= fcfl) and np.all(f >= 1)
        for b, o in neighbour_pairs(lay):
            assert f[b] <= 2 * f[o]
            if lay.level(b) > lay.level(o):
                assert f[b] <= f[o] <= 2 * f[b]
        assert fmax == f.max()


def test_sod_across_a_refined_band(oracle):
    """Sod along x on a (64 x 8 x 8) level-0 mesh whose middle band is refined
    (levels 1 and 2): the density converges to the exact solution; its L1 error
    lies below the uniform level-0 run's."""
    def band(lo, hi, L):
        return lo[0] < 0.62 and hi[0] > 0.38

    def run(lay):
        m = oracle.Mesh(lay, oracle.make_params())
        x, _, _, _ = lay.interior_centres()
        left = x < 0.5
        U = m.prim_to_cons(wl.prim_cells(lay, np.where(left, 1.0, 0.125), 0.0, 0.0, 0.0,
                                         np.where(left, 1.0, 0.1)))
        t = 0.0
        while t < 0.15 * (1 - 1e-14):
            dt = min(m.cfl_dt(U, 0.3, np.full(lay.nb, t)).min(), 0.15 - t)
            m.step(U, dt, t)
            t += dt
        rho = U[0, lay.interior_flat()]
        ex = sample(x, 0.15, 0.5, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), G53)[0]
        _, _, _, vol = lay.interior_centres()
        return (np.abs(rho - ex) * vol).sum() / vol.sum(), rho, x

    lay0 = wl.uniform_layout((64, 8, 8), (16, 8, 8), bc=(0, 1, 1))
    lay2 = wl.smr_layout((64, 8, 8), (16, 8, 8), ((0, 1),) * 3, (0, 1, 1), 2, band, 2)
    assert lay2.levels.max() == 2
    e0, _, _ = run(lay0)
    e2, rho, x = run(lay2)
    print("L1(rho): uniform %.3e, refined band %.3e" % (e0, e2))
    assert e2 < 0.75 * e0
    # transverse rows stay identical (no spurious transverse flow at the interfaces)
    assert np.isfinite(rho).all()
