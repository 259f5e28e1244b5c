"""Pins of the oracle's self-gravity multigrid (Sec. 3.2): the discrete
operator's Fourier modes (closed form), the FFT solution of the discrete
periodic problem for a random source (a library routine on the same discrete
equation), the anisotropic stencil, and the V-cycle convergence rate."""
import numpy as np
import pytest


def grid(n, L):
    x = [(np.arange(n[a]) + 0.5) * L[a] / n[a] for a in range(3)]
    z, y, xx = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    return xx, y, z


@pytest.mark.parametrize("n,L", [((32, 16, 8), (1.0, 1.0, 1.0)), ((16, 16, 16), (1.0, 1.0, 0.5))])
def test_fourier_mode_closed_form(oracle, n, L):
    """A_h cos(k.x) = lambda_k cos(k.x) with lambda_k = sum_a (2 - 2 cos(k_a h_a)) / h_a^2,
    so phi = S / lambda_k exactly (anisotropic cells included)."""
    dx = [L[a] / n[a] for a in range(3)]
    x, y, z = grid(n, L)
    k = [2 * np.pi * 2 / L[0], 2 * np.pi * 1 / L[1], 2 * np.pi * 1 / L[2]]
    S = np.cos(k[0] * x) * np.cos(k[1] * y) * np.cos(k[2] * z)
    lam = sum((2 - 2 * np.cos(k[a] * dx[a])) / dx[a] ** 2 for a in range(3))
    phi, cyc, d = oracle.mg_solve(S, dx, max_cycles=30, tol=1e-12)
    assert d < 1e-12 and cyc < 30
    assert np.allclose(phi - phi.mean(), S / lam, rtol=0, atol=1e-11 * np.abs(S / lam).max())


def test_random_source_matches_fft_solution(oracle):
    """The discrete periodic Poisson problem solved by FFT with the operator's
    eigenvalues (mean zero) against the multigrid solution."""
    rng = np.random.default_rng(7)
    n, L = (32, 32, 16), (1.0, 1.0, 0.5)
    dx = [L[a] / n[a] for a in range(3)]
    S = rng.normal(size=(n[2], n[1], n[0]))
    S -= S.mean()
    kk = [2 * np.pi * np.fft.fftfreq(n[a], d=dx[a]) for a in range(3)]
    kz, ky, kx = np.meshgrid(kk[2], kk[1], kk[0], indexing="ij")
    lam = ((2 - 2 * np.cos(kx * dx[0])) / dx[0] ** 2 + (2 - 2 * np.cos(ky * dx[1])) / dx[1] ** 2 +
           (2 - 2 * np.cos(kz * dx[2])) / dx[2] ** 2)
    lam[0, 0, 0] = 1.0
    Sh = np.fft.fftn(S)
    Sh[0, 0, 0] = 0.0
    exact = np.real(np.fft.ifftn(Sh / lam))
    phi, cyc, d = oracle.mg_solve(S, dx, max_cycles=40, tol=1e-11)
    assert d < 1e-11
    assert np.allclose(phi - phi.mean(), exact, rtol=0, atol=1e-9 * np.abs(exact).max())


def test_vcycle_convergence_factor(oracle):
    """Red-black Gauss-Seidel (omega 1.15, two pre- and two post-sweeps) with a
    full-approximation coarse correction reduces the defect by an order of
    magnitude or more per V-cycle on a smooth + rough source."""
    n = (64, 64, 64)
    dx = [1.0 / 64] * 3
    x, y, z = grid(n, (1.0, 1.0, 1.0))
    rng = np.random.default_rng(3)
    S = np.sin(2 * np.pi * x) * np.cos(4 * np.pi * y) + 0.1 * rng.normal(size=x.shape)
    S -= S.mean()
    ds = []
    phi = None
    for c in range(5):
        phi, _, d = oracle.mg_solve(S, dx, phi=phi, max_cycles=1, tol=0.0)
        ds.append(d)
    d0 = oracle.mg_defect(S, np.zeros_like(S), dx)
    rates = np.array(ds[1:]) / np.array(ds[:-1])
    assert ds[0] < 0.1 * d0
    assert rates.max() < 0.12, rates


def test_tricubic_prolongation_exact_on_cubics(oracle):
    """The V-cycle's prolongation is tricubic (Sec. 3.2): it reproduces any
    product of cubic polynomials at the fine cell centres wherever its 4^3
    stencil lies inside the coarse grid, in every combination of halved and
    kept directions; beyond an isolated face it mirrors the field about zero,
    which reproduces fields odd about that face."""
    rng = np.random.default_rng(11)

    def cubic():
        c = rng.normal(size=4)
        return lambda t: ((c[3] * t + c[2]) * t + c[1]) * t + c[0]
    P, Q, R = cubic(), cubic(), cubic()
    for nf, nc in (((16, 16, 16), (8, 8, 8)), ((16, 8, 1), (8, 8, 1)), ((8, 16, 16), (8, 8, 8))):
        cen = [np.arange(n) + 0.5 for n in nc]          # coarse centres, coarse cell width 1
        e = P(cen[0])[None, None, :] * Q(cen[1])[None, :, None] * R(cen[2])[:, None, None]
        out = oracle.mg_prolong(e, nf)
        fine = [(np.arange(m) + 0.5) * (n / m) for m, n in zip(nf, nc)]
        want = P(fine[0])[None, None, :] * Q(fine[1])[None, :, None] * R(fine[2])[:, None, None]
        ok = []
        for a in range(3):
            f = np.arange(nf[a])
            if nf[a] == nc[a]:
                ok.append(np.ones(nf[a], dtype=bool))
            else:
                p = f // 2
                lo = np.where(f % 2 == 1, p - 1, p - 2)
                ok.append((lo >= 0) & (lo + 3 < nc[a]))
        m = ok[2][:, None, None] & ok[1][None, :, None] & ok[0][None, None, :]
        assert m.sum() > 0
        assert np.abs(out - want)[m].max() <= 1e-12 * np.abs(want).max(), nf
        # a trilinear prolongation misses the cubic part by far more than that
        assert np.abs(want).max() > 0
    # isolated: x^3 - 2x is odd about the low x face (x = 0), so its mirror image
    # beyond that face is the field itself and the cells next to the face are exact
    nc, nf = (8, 8, 8), (16, 16, 16)
    cen = [np.arange(n) + 0.5 for n in nc]
    odd = lambda t: t ** 3 - 2.0 * t   # noqa: E731
    e = odd(cen[0])[None, None, :] * Q(cen[1])[None, :, None] * R(cen[2])[:, None, None]
    out = oracle.mg_prolong(e, nf, isolated=True)
    fine = [(np.arange(m) + 0.5) / 2 for m in nf]
    want = odd(fine[0])[None, None, :] * Q(fine[1])[None, :, None] * R(fine[2])[:, None, None]
    inner = slice(4, 12)
    assert np.abs(out - want)[inner, inner, :8].max() <= 1e-12 * np.abs(want).max()
    # the even part's mirror is not the field: the face cells then differ
    e2 = Q(cen[0])[None, None, :] * Q(cen[1])[None, :, None] * R(cen[2])[:, None, None]
    want2 = Q(fine[0])[None, None, :] * Q(fine[1])[None, :, None] * R(fine[2])[:, None, None]
    out2 = oracle.mg_prolong(e2, nf, isolated=True)
    assert np.abs(out2 - want2)[inner, inner, 0].max() > 1e-3 * np.abs(want2).max()


# ------------------------------------------------ isolated boundaries, FMG ----

def centred_grid(n, half):
    dx = [2.0 * half / n] * 3
    x = (np.arange(n) + 0.5) * dx[0] - half
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    return xx, y, z, dx


def blobs(x, y, z):
    """Two off-centre Gaussian clumps (S = -4 pi G rho < 0)."""
    return (-np.exp(-((x - 0.2) ** 2 + (y + 0.1) ** 2 + (z - 0.05) ** 2) / (2 * 0.08 ** 2)) -
            0.6 * np.exp(-((x + 0.15) ** 2 + (y - 0.2) ** 2 + (z + 0.1) ** 2) / (2 * 0.06 ** 2)))


def test_multipole_expansion_matches_the_direct_sum(oracle):
    """The boundary expansion against brute force, phi(x) = (1/4 pi) sum S dV / |x - x'|,
    at points outside the source: the error falls with the order, as (r'/r)^(l+1)."""
    x, y, z, dx = centred_grid(32, 1.0)
    S = blobs(x, y, z)
    rng = np.random.default_rng(4)
    u = rng.normal(size=(200, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    dV = dx[0] ** 3
    src = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    for R, bound8 in ((1.3, 2e-5), (4.0, 1e-8)):
        q = R * u
        direct = np.array([(S.ravel() * dV / np.linalg.norm(src - p, axis=1)).sum() for p in q]) / (4 * np.pi)
        errs = []
        for lmax in (0, 2, 4, 8):
            _, _, _, _, val = oracle.mg_solve_bc(S, dx, xmin=(-1.0, -1.0, -1.0), lmax=lmax, fmg=False,
                                                 max_cycles=0, query=q)
            errs.append(np.abs(val - direct).max() / np.abs(direct).max())
        print("r = %.1f, multipole errors (l_max 0, 2, 4, 8):" % R, errs)
        assert errs[0] > 100 * errs[3] and errs[3] < bound8
        assert errs[0] > errs[1] > errs[2] > errs[3]


@pytest.mark.parametrize("n", [32, 64])
def test_isolated_uniform_sphere(oracle, n):
    """rho = 1 inside r < 0.4 with 4 pi G = 1 on [-1, 1]^3: the isolated solution
    is -M / (4 pi r) outside and -(R^2 - r^2 / 3) / 2 inside (M the discrete
    mass), to the discretisation error, which falls with resolution."""
    x, y, z, dx = centred_grid(n, 1.0)
    r = np.sqrt(x * x + y * y + z * z)
    rho = (r < 0.4).astype(float)
    S = -rho
    phi, cyc, d, d0, _ = oracle.mg_solve_bc(S, dx, xmin=(-1.0, -1.0, -1.0), lmax=4, max_cycles=30, tol=1e-12)
    assert d < 1e-12
    M = rho.sum() * dx[0] ** 3
    Reff = (3 * M / (4 * np.pi)) ** (1.0 / 3.0)   # the radius of the discrete mass
    inside = r < 0.2
    outside = r > 0.6
    ein = np.abs(phi[inside] + 0.5 * (Reff ** 2 - r[inside] ** 2 / 3)).max() / (0.5 * Reff ** 2)
    eout = np.abs(phi[outside] + M / (4 * np.pi * r[outside])).max() / (M / (4 * np.pi * 0.6))
    print("n=%d: inside %.2e, outside %.2e, V-cycles %d" % (n, ein, eout, cyc))
    assert ein < 1.5e-2 and eout < 1e-2


def test_full_multigrid_start_and_contraction(oracle):
    """Full multigrid leaves a defect an order of magnitude or more below the zero
    start's; the V-cycles then contract the defect by about 0.1 each (Sec. 3.2:
    five V-cycles to 1e-12 from the full-multigrid guess), isolated and periodic."""
    x, y, z, dx = centred_grid(64, 1.0)
    S = blobs(x, y, z)
    for iso in (True, False):
        Sm = S if iso else S - S.mean()
        d_zero = oracle.mg_defect(Sm, np.zeros_like(S), dx) if not iso else None
        _, _, _, d0z, _ = oracle.mg_solve_bc(S, dx, xmin=(-1.0, -1.0, -1.0), isolated=iso, fmg=False,
                                              max_cycles=0)
        ds = []
        phi, _, _, d0, _ = oracle.mg_solve_bc(S, dx, xmin=(-1.0, -1.0, -1.0), isolated=iso, fmg=True,
                                              max_cycles=0)
        for c in range(5):
            phi, _, d, _, _ = oracle.mg_solve_bc(S, dx, xmin=(-1.0, -1.0, -1.0), isolated=iso, fmg=False,
                                                 phi=phi, max_cycles=1)
            ds.append(d)
        rates = np.array(ds) / np.array([d0] + ds[:-1])
        print("iso=%s: zero-start defect %.2e, FMG %.2e, rates %s" % (iso, d0z, d0, rates))
        assert d0 < 0.1 * d0z
        assert rates.max() < 0.15
        assert ds[-1] < 1e-5 * d0z
        if d_zero is not None:
            assert d0z == pytest.approx(d_zero, rel=1e-12)


def test_jeans_wave_oscillates_at_the_linear_frequency(oracle):
    """A stable Jeans wave (Eqs. jeans-initial, jeans-analytic, with the adiabatic
    sound speed c_s^2 = gamma P / rho): lambda / lambda_J = 0.8, so
    omega^2 = c_s^2 k^2 - 4 pi G rho = 0.36 c_s^2 k^2; the density's Fourier
    amplitude follows a cos(omega t) over one period, the potential solved by the
    multigrid before every step and frozen over it."""
    from paper_2609_37859_gb300 import workloads as wl
    n = 64
    lay = wl.uniform_layout((n, 4, 4), (32, 4, 4), domain=((0, 1), (0, 4.0 / n), (0, 4.0 / n)), bc=(1, 1, 1))
    gam = 5.0 / 3.0
    k = 2 * np.pi
    fourpiG = 0.64 * k * k           # k_J = 0.8 k with rho = 1, c_s = 1
    a = 1e-3
    x, y, z = lay.cell_centres()
    W = wl.prim_state(lay, 1.0 + a * np.cos(k * x), 0.0, 0.0, 0.0, (1.0 + gam * a * np.cos(k * x)) / gam)
    m = oracle.Mesh(lay, oracle.make_params(gamma=gam))
    U = m.prim_to_cons(W)
    omega = np.sqrt(k * k - fourpiG)
    T = 2 * np.pi / omega
    t, worst = 0.0, 0.0
    phi = None
    S_scr = m.new_state()
    checks = [T / 4, T / 2, 3 * T / 4, T]
    while checks:
        rho = lay.to_global(U)[0]
        phi, _, _ = oracle.mg_solve(-fourpiG * rho, lay.dx, phi=phi, max_cycles=20, tol=1e-13)
        A = lay.from_global(phi[None])
        m.ghost_fill(A, nvar=1)
        m.set_phi_sg(A[0])
        dt = min(0.3 * lay.dx[0] / np.sqrt(gam), checks[0] - t)
        m.step(U, dt, t, S_scr)
        t += dt
        if t >= checks[0] * (1 - 1e-12):
            rho = lay.to_global(U)[0][0, 0]
            amp = 2.0 / n * (rho * np.cos(k * (np.arange(n) + 0.5) / n)).sum()
            worst = max(worst, abs(amp - a * np.cos(omega * t)) / a)
            checks.pop(0)
    m.set_phi_sg(None)
    print("Jeans wave: max normalised amplitude error over one period %.2e" % worst)
    # (the PLM limiter clips the extrema: 4.0e-2 at 64 cells per wavelength, 1.9e-2
    # at 128; without gravity, or with its sign reversed, the phase at T / 4
    # alone would be off by O(1))
    assert worst < 5e-2
