"""The sweeps' Riemann solvers (a5: HLLC and HLLE with the dual-energy flux and
face velocity) on random face-state pairs through the C ABI, against the
oracle's independent implementation: every direction, the tabulated-EOS form
(per-state Gamma_e, Gamma_1) and the ideal gas, with and without dual energy,
over general subsonic pairs, supersonic pairs both ways, stationary contacts,
identical states and pairs with density and pressure ratios of 10^6."""
import numpy as np
import pytest

from test_oracle_hydro import _face_states

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_hydro import tde, ctx  # noqa: E402,F401


def pairs(rng, n, table, d):
    wl, wr = _face_states(rng, n, table), _face_states(rng, n, table)
    k = n // 6
    c = np.sqrt(np.maximum(wl[:, 6] * wl[:, 4] / wl[:, 0], wr[:, 6] * wr[:, 4] / wr[:, 0]))
    # supersonic to the right, to the left
    for sl, sgn in ((slice(k, 2 * k), 1.0), (slice(2 * k, 3 * k), -1.0)):
        wl[sl, 1 + d] = sgn * (2 * c[sl] + np.abs(wl[sl, 1 + d]))
        wr[sl, 1 + d] = sgn * (2 * c[sl] + np.abs(wr[sl, 1 + d]))
    # stationary contacts
    sl = slice(3 * k, 4 * k)
    wr[sl] = wl[sl]
    wl[sl, 1:4] = 0.0
    wr[sl, 1:4] = 0.0
    wr[sl, 0] *= 10 ** rng.uniform(-2, 2, k)
    # identical states
    sl = slice(4 * k, 5 * k)
    wr[sl] = wl[sl]
    # strong jumps
    sl = slice(5 * k, n)
    wl[sl, 0] *= 1e3
    wr[sl, 0] *= 1e-3
    wl[sl, 4] *= 1e3
    wr[sl, 4] *= 1e-3
    return wl, wr


def scales(wl, wr, d):
    """Per pair and component, the size of the terms the flux is made of: both
    physical fluxes and the fastest signal speed times both conserved states;
    for the face velocity, the mass-flux scale over the densities."""
    sc = np.zeros((len(wl), 6))
    msc = np.zeros(len(wl))
    for w in (wl, wr):
        rho, P = w[:, 0], w[:, 4]
        c = np.sqrt(w[:, 6] * P / rho)
        E = P / (w[:, 5] - 1.0) + 0.5 * rho * (w[:, 1:4] ** 2).sum(axis=1)
        s = np.abs(w[:, 1 + d]) + c
        m = rho * s   # bounds |rho u| and the signal speed times rho
        msc += 2 * m
        for q in range(3):
            sc[:, 1 + q] += 2 * m * np.abs(w[:, 1 + q]) + (P if q == d else 0.0)
        sc[:, 4] += (E + P) * np.abs(w[:, 1 + d]) + E * s
    sc[:, 0] = msc
    sc[:, 5] = msc * (wl[:, 7] / wl[:, 0] + wr[:, 7] / wr[:, 0])
    vsc = msc * (1 / wl[:, 0] + 1 / wr[:, 0])
    return sc, vsc


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("table,dual", [(1, 1), (1, 0), (0, 1), (0, 0)])
def test_riemann_face_pairs_against_oracle(oracle, tde, ctx, solver, table, dual):
    rng = np.random.default_rng(100 + 10 * solver + 2 * table + dual)
    n = 60000
    worst = 0.0
    for d in range(3):
        wl, wr = pairs(rng, n, table, d)
        Fo, vfo = oracle.riemann(solver, d, dual, wl, wr)
        dl, dr = torch.from_numpy(wl).cuda(), torch.from_numpy(wr).cuda()
        F = torch.empty((n, 6), dtype=torch.float64, device="cuda")
        vf = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.riemann_probe(solver, d, dl, dr, F, vf, eos_table=table, dual=dual)
        torch.cuda.synchronize()
        Fg, vfg = F.cpu().numpy(), vf.cpu().numpy()
        sc, vsc = scales(wl, wr, d)
        err = np.abs(Fg - Fo) / np.maximum(sc, 1e-300)   # a zero scale demands equality
        worst = max(worst, float(err.max()))
        assert err.max() <= 1e-13, (d, np.unravel_index(err.argmax(), err.shape), err.max())
        assert np.all(np.abs(vfg - vfo) <= 1e-13 * vsc)
        if not dual:
            assert np.all(Fg[:, 5] == 0.0) and np.all(vfg == 0.0)
    print("worst scaled flux difference", worst)


def test_riemann_probe_rejects_bad_arguments(tde, ctx):
    x = torch.zeros((4, 8), dtype=torch.float64, device="cuda")
    F = torch.zeros((4, 6), dtype=torch.float64, device="cuda")
    vf = torch.zeros(4, dtype=torch.float64, device="cuda")
    for solver, d, gamma in ((2, 0, 5 / 3), (0, 3, 5 / 3), (0, 0, 1.0)):
        with pytest.raises(tde.TDEError):
            ctx.riemann_probe(solver, d, x, x, F, vf, gamma=gamma)
