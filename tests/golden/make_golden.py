"""Writes the oracle-derived golden fixtures of this folder.

Calls only ``oracle/``.  Run from the repository root:
    python tests/golden/make_golden.py
Outputs (float64 values as hex, exact):
  d2q37_constants.txt  - r, w_l, and the wall ratios q_l for a few wall
                         temperatures (bottom and top walls).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import lattice, model  # noqa: E402

WALL_TEMPERATURES = (0.5, 1.0, 1.5, 0.9)


def main():
    k = lattice.constants()
    lines = ["# D2Q37 constants from the oracle's 60-digit solve, rounded once to float64.",
             "# Regenerate with: python tests/golden/make_golden.py",
             f"r {k['r'].hex()}"]
    for l in range(37):
        lines.append(f"w_{l} {k['w'][l].hex()}")
    for T in WALL_TEMPERATURES:
        for wall in ("bottom", "top"):
            q = model.wall_q(T, wall)
            for l in range(37):
                if q[l] != 0.0:
                    lines.append(f"q_{wall}_{T!r}_{l} {q[l].hex()}")
    with open(os.path.join(HERE, "d2q37_constants.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
