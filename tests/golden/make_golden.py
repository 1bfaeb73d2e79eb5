"""Writes tests/golden/*.txt from the oracle alone (no library code).

Fixtures:
  sweep2d_tiny.txt   one 3x2-cell, 8-direction, 2-group sweep with moments
                     (regression record of the pinned oracle; any later change
                     to the oracle's arithmetic must regenerate it and say why)
Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402


def tiny_case():
    nx, ny, G = 3, 2, 2
    edges = np.array([0.05, 0.5, 5.0])
    T = np.array([[0.2, 0.4, 0.3, 0.5], [0.6, 0.5, 0.4, 0.7], [0.1, 0.2, 0.3, 0.2],
                  [0.9, 0.8, 0.7, 1.0], [0.3, 0.3, 0.3, 0.3], [0.5, 0.1, 0.2, 0.4]])
    scale = np.array([1.0, 2.0, 0.5, 4.0, 1.5, 0.8])
    ox, oy, w = O.quadrature(2, 1, 2)
    sig = O.opacity(1, 10.0, edges, T, scale)
    q = O.emission(edges, 1.0, 1.0, T, sig)
    infl = O.inflow(edges, 1.0, 1.0, [1.0, 0.0, 0.5, 0.0])
    Ip = np.zeros((len(w), G, nx * ny, 4))
    I = O.sweep(2, nx, ny, (0.0, 1.0, 0.0, 1.0), ox, oy, sig, 100.0, q, Ip, infl)
    mom = O.moments(2, ox, oy, w, sig, I)
    return I, mom


def main():
    I, mom = tiny_case()
    path = os.path.join(HERE, "sweep2d_tiny.txt")
    with open(path, "w") as f:
        f.write("# oracle regression fixture: 3x2 cells, 8 directions, 2 groups; see make_golden.py tiny_case()\n")
        f.write("# I[d][g][cell][node] flattened, then mom[cell][node][9] flattened\n")
        for v in I.ravel():
            f.write(f"{v:.17e}\n")
        for v in mom.ravel():
            f.write(f"{v:.17e}\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
