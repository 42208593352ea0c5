"""Writes lake_hump_exact_rhs.npz: the exact right-hand side of the
lake-plus-hump configuration (N=3, 8x8 curved periodic quads, entropy-stable
interface flux; the smoothness indicator leaves every element inviscid on
these states) at t = 0 and after 50 LSRK4(5) steps of the FP64 oracle at
CFL 0.5 with the limiter on.

The exact right-hand side is the multi-precision brute-force evaluation
(oracle/bruteforce.py, 40 digits) of the stored float64 state, rounded to
float64 once. The states, coordinates and bathymetry are stored with it, so
a reader on another host (whose libm may round the generator's sines
differently) compares against the same input bits. Calls only oracle/ and the seeded
input generator.

  python tests/golden/make_lake_hump_exact.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from oracle.bruteforce import BruteForce  # noqa: E402
from paper_1804_02221_gb300 import inputs as I  # noqa: E402


def main():
    p = I.lake_hump(N=3, K1=8)
    kw = dict(flux=1, av=True, eps0=0.01, limiter=True, rk=0, cfl=0.5)
    o = O.Oracle(p, **kw)
    W0 = np.ascontiguousarray(p.W)
    o.rhs(W0)
    assert o.epsilon().max() == 0.0
    W50, rc, _ = o.step(W0, 0.0, 50)
    assert rc == 0
    o.rhs(W50)
    assert o.epsilon().max() == 0.0
    bf = BruteForce(p.N, p.x, p.y, p.b, p.g)
    R0 = bf.rhs(W0, flux=1)
    R50 = bf.rhs(W50, flux=1)
    np.savez_compressed(os.path.join(HERE, "lake_hump_exact_rhs.npz"), x=p.x, y=p.y, b=p.b,
                        W0=W0, R0=R0, W50=W50, R50=R50)


if __name__ == "__main__":
    main()
