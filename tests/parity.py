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


def stencil_scale(Uin_block, active, radius):
    """Per interior cell and variable: the largest input magnitude within `radius`
    cells (the reconstruction stencil) of a padded, ghost-filled block
    [nvar, pz, py, px], for the momentum the largest sqrt(2 rho E).  A stage's
    output is a combination of these inputs with coefficients of order one (the
    time step obeys the CFL condition), so its rounding is a few ulps of this
    scale: where inflow multiplies a cell's density by 1e4 in one stage, its own
    value is the wrong yardstick."""
    from scipy.ndimage import maximum_filter
    U = np.abs(np.asarray(Uin_block, dtype=np.float64))
    size = tuple((2 * radius + 1) if active[a] else 1 for a in (2, 1, 0))
    sm = np.sqrt(2.0 * U[0] * U[4])
    out = []
    for v in range(U.shape[0]):
        out.append(maximum_filter(sm if v in (1, 2, 3) else U[v], size=size, mode="nearest"))
    return np.stack(out)


def assert_parity_stencil(G, O, scale, tol, what=""):
    """assert_parity with the denominators raised to `scale` (stencil_scale of the
    stage's input, interior cells, same shape as G and O)."""
    G = np.asarray(G, dtype=np.float64)
    O = np.asarray(O, dtype=np.float64)
    assert np.all(np.isfinite(G)), "non-finite GPU values " + what
    rho, E = O[0], O[4]
    own = np.sqrt(2.0 * np.abs(rho) * np.abs(E))
    errs = []
    for v in range(O.shape[0]):
        den = np.maximum(own if v in (1, 2, 3) else np.abs(O[v]), scale[v])
        d = np.abs(G[v] - O[v])
        with np.errstate(divide="ignore", invalid="ignore"):
            e = np.where(d == 0, 0.0, d / den)
        errs.append(float(np.max(e)) if e.size else 0.0)
    errs = np.array(errs)
    assert errs.max() <= tol, "%s: per-variable max error %s > %g" % (what, errs, tol)
    return errs


def error_report(G, O, scale=None, thresh=1e-12, mask=None):
    """Both readings of a comparison, per conserved variable: the plain per-cell
    error of cell_errors (max, and the number of cells above `thresh`), and, with
    `scale` (stencil_scale of the input, same shape), the error against the larger
    of the cell's own scale and its stencil's; plus the number of cells where
    the two readings disagree about `thresh`.  `mask` (boolean, the grid's
    shape) restricts the comparison to those cells."""
    G = np.asarray(G, dtype=np.float64)
    O = np.asarray(O, dtype=np.float64)
    if mask is not None:
        G, O = G[:, mask], O[:, mask]
        scale = None if scale is None else scale[:, mask]
    rho, E = O[0], O[4]
    own_m = np.sqrt(2.0 * np.abs(rho) * np.abs(E))
    out = {"plain_max": [], "plain_cells_above": [], "stencil_max": [], "disagree_cells": []}
    for v in range(O.shape[0]):
        own = own_m if v in (1, 2, 3) else np.abs(O[v])
        d = np.abs(G[v] - O[v])
        with np.errstate(divide="ignore", invalid="ignore"):
            e = np.where(d == 0, 0.0, d / own)
        out["plain_max"].append(float(e.max()) if e.size else 0.0)
        out["plain_cells_above"].append(int((e > thresh).sum()))
        if scale is not None:
            with np.errstate(divide="ignore", invalid="ignore"):
                es = np.where(d == 0, 0.0, d / np.maximum(own, scale[v]))
            out["stencil_max"].append(float(es.max()) if es.size else 0.0)
            out["disagree_cells"].append(int(((e > thresh) != (es > thresh)).sum()))
    return out
