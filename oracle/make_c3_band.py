"""Write the recombination band of the EOS-inversion workload (2^24 cells).

Calls only the oracle (the Saha H/He solver of oracle/tref_eos.c, X = 0.7,
Y = 0.3): for 257 densities evenly spaced in log10 rho over [-14, 2] g/cm^3, the
temperature at which the ionised hydrogen fraction reaches 0.01 (T_lo) and the
one at which the He2+ fraction reaches 0.99 (T_hi), by bisection in log10 T over
the table's range [2, 8] (a fraction that is not reached inside the range gives
the range's edge).  The workload draws log10 rho uniformly and log10 T uniformly
between the two edges, interpolated linearly in log10 rho.
Output: paper_2609_37859_gb300/data/c3_recombination_band.npz

    python oracle/make_c3_band.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
from oracle import tref  # noqa: E402

OUT = os.path.join(os.path.dirname(HERE), "paper_2609_37859_gb300", "data", "c3_recombination_band.npz")
N_RHO, LRHO, LT, X, Y = 257, (-14.0, 2.0), (2.0, 8.0), 0.7, 0.3


def crossing(rho, key, target):
    """log10 T in LT at which the ionisation fraction `key` reaches target (the
    fractions grow with T at fixed density)."""
    frac = lambda lT: tref.saha_state(rho, 10.0 ** lT, X, Y)[key]   # noqa: E731
    lo, hi = LT
    if frac(lo) >= target:
        return lo
    if frac(hi) < target:
        return hi
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if frac(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def make():
    lrho = np.linspace(LRHO[0], LRHO[1], N_RHO)
    lo = np.array([crossing(10.0 ** r, "xH", 0.01) for r in lrho])
    hi = np.array([crossing(10.0 ** r, "yHe2", 0.99) for r in lrho])
    return dict(lrho=lrho, lT_lo=lo, lT_hi=hi, X=X, Y=Y)


if __name__ == "__main__":
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    np.savez_compressed(OUT, **make())
    print("wrote", OUT)
