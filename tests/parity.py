"""Per-cell comparison of a GPU state with the oracle's.

Error measure (per interior cell, per conserved variable), chosen so that every
variable is compared with a quantity of its own physical scale:
    rho, E, U_aux:  |a - b| / |b|
    m_d:            |a - b| / sqrt(2 rho E)      (sqrt(2 rho E) >= |m|; equal
                                                  when kinetic energy dominates)
The tolerances (1e-12 after one stage, 1e-10 after many steps) are the ones
the hydro stage is specified to: FP64 with a different but equally rounded
operation order (FMA contraction, reciprocal multiplies) on the GPU.
"""
import numpy as np


def cell_errors(G, O):
    """G, O: [nvar, ...] interior arrays (GPU, oracle).  Returns max error per variable."""
    G = np.asarray(G, dtype=np.float64)
    O = np.asarray(O, dtype=np.float64)
    rho, E = O[0], O[4]
    scale_m = np.sqrt(2.0 * np.abs(rho) * np.abs(E))
    errs = []
    for v in range(O.shape[0]):
        if v in (1, 2, 3):
            den = scale_m
        else:
            den = np.abs(O[v])
        d = np.abs(G[v] - O[v])
        with np.errstate(divide="ignore", invalid="ignore"):
            e = np.where(d == 0, 0.0, d / den)
        errs.append(float(np.max(e)) if e.size else 0.0)
    return np.array(errs)


def assert_parity(G, O, tol, what=""):
    e = cell_errors(G, O)
    assert np.all(np.isfinite(G)), "non-finite GPU values " + what
    assert e.max() <= tol, "%s: per-variable max error %s > %g" % (what, e, tol)
    return e
