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
