"""Writes the stored expected values under tests/golden/ from the oracle only.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2411_07920_gb300 import inputs as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    with open(os.path.join(HERE, "pool_sizes.txt"), "w") as f:
        f.write("# Size of the generalized singles and doubles pool (Sec. II.C) per spin-orbital count,\n")
        f.write("# S_z-conserving singles p<q and doubles over disjoint pairs, as enumerated by the oracle.\n")
        f.write("# Closed form 2C(m,2) + 6C(m,4) + (m(m-1))^2/2 with m = n_so/2 (checked in the test).\n")
        for n_so in (8, 12, 16, 28, 52):
            f.write(f"{n_so} {O.pool_ops(n_so).shape[0]}\n")
    w = I.workload("so12_e4")
    k, a = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 0)
    e, n2 = O.energy(w.n_so, w.h, w.g, k, a)
    g = O.pool_gradients(w.n_so, w.h, w.g, k, a)
    _, d = O.energy_grad(w.n_so, w.n_e, w.h, w.g, w.ops, w.theta, 0)
    with open(os.path.join(HERE, "so12_e4_oracle.txt"), "w") as f:
        f.write("# 12 spin-orbitals / 4 electrons, seed 1, 10 gates (Eq. 1), no truncation.\n")
        f.write("# Written by tests/golden/make_golden.py from the oracle only.\n")
        f.write(f"n_det {len(k)}\nenergy {e!r}\nnorm2 {n2!r}\n")
        f.write("dtheta " + " ".join(repr(float(x)) for x in d) + "\n")
        top = np.argsort(-np.abs(g))[:10]
        f.write("pool_top " + " ".join(f"{int(i)}:{float(g[i])!r}" for i in top) + "\n")


if __name__ == "__main__":
    main()
