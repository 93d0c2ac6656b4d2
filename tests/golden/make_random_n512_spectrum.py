"""Writes tests/golden/random_n512_d4_spectrum.txt: the 8 smallest-|lambda| nonzero eigenvalues of the
random Lindbladian n = 512, d = 4, seed 0 (H = (A + A^dag)/(2 sqrt n), Var L_ij = 1/n), computed by the
oracle's Alg. 5 (oracle/krylov.py, shift-invert Arnoldi with recycled inner solves, FP64, mu = 0,
eta = 1) and checked by its
eigen-residual ||L v - lambda v||_max / ||v||_max.  Uses only oracle/ and lindblad_inputs/.

    python tests/golden/make_random_n512_spectrum.py        (tens of minutes on 8 cores)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import lindblad_inputs as gi  # noqa: E402
from oracle import krylov as K  # noqa: E402


def main():
    H, Ls = gi.random_lindbladian(512, d=4, seed=0)
    s = K.System(H, Ls)
    t0 = time.time()
    lam, vecs, info = K.low_spectrum_shift_invert(s, k=8, mu=0.0, eta=1.0, tol=1e-10, m=24, restarts=30,
                                                  inner_tol=1e-12, k_recycle=8, inner_m=40)
    res = [float(np.abs(s.L(v) - l * v).max() / np.abs(v).max()) for l, v in zip(lam, vecs)]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "random_n512_d4_spectrum.txt")
    with open(out, "w") as f:
        f.write("# The 8 smallest-|lambda| nonzero eigenvalues of L for the random Lindbladian n = 512, d = 4,\n")
        f.write("# seed 0 (the configured random workload), sorted by |lambda|, then Re descending.\n")
        f.write("# Source: the oracle's Alg. 5 (shift-invert Arnoldi with recycled inner solves, Sec. 4.2), written by\n")
        f.write("# tests/golden/make_random_n512_spectrum.py; eigen-residuals ||L v - lambda v||_max / ||v||_max:\n")
        f.write("# " + " ".join(f"{r:.2e}" for r in res) + f"  ({time.time() - t0:.0f} s)\n")
        f.write("re = " + " ".join(repr(float(x)) for x in lam.real) + "\n")
        f.write("im = " + " ".join(repr(float(x)) for x in lam.imag) + "\n")
    print(out, lam, res, info)


if __name__ == "__main__":
    main()
