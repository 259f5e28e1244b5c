"""Write the Saha H/He EOS table used as input data by the benchmark and tests.

Calls only the oracle (oracle/tref_eos.c): 256 x 256 points on
log10 rho in [-14, 2] g/cm^3 and log10 T in [2, 8] K, X = 0.7, Y = 0.3, with
radiation (the table the hydro stage's tabulated-EOS workload runs on).
Output: paper_2609_37859_gb300/data/eos_saha_hhe_256.npz

    python oracle/make_saha_table.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
from oracle import tref  # noqa: E402

OUT = os.path.join(os.path.dirname(HERE), "paper_2609_37859_gb300", "data", "eos_saha_hhe_256.npz")
SPEC = dict(n_rho=256, n_T=256, lrho=(-14.0, 2.0), lT=(2.0, 8.0), X=0.7, Y=0.3)


def make():
    t = tref.EOSTable.saha(SPEC["n_rho"], SPEC["n_T"], SPEC["lrho"], SPEC["lT"], SPEC["X"], SPEC["Y"])
    return dict(n_rho=SPEC["n_rho"], n_T=SPEC["n_T"], lrho=np.array(SPEC["lrho"]),
                lT=np.array(SPEC["lT"]), X=SPEC["X"], Y=SPEC["Y"], log10_e=t.log10_e,
                log10_P=t.log10_P, log10_cs2=t.log10_cs2, gamma1=t.gamma1)


if __name__ == "__main__":
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    np.savez_compressed(OUT, **make())
    print("wrote", OUT)
