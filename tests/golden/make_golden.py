"""Writes the stored expected values under tests/golden/ from the oracle only.

    python tests/golden/make_golden.py

mc_table.txt: the face-consistent marching-cubes table derived by the oracle
(Sec. 2.4, Eq. 28 reading), one line per corner configuration (bit k = corner
k inside), listing triangles as flat triples of cube edge ids.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import mc  # noqa: E402


def main():
    with open(os.path.join(HERE, "mc_table.txt"), "w") as f:
        f.write("# face-consistent marching-cubes table written by tests/golden/make_golden.py\n")
        f.write("# line c (0..255): triangles of corner configuration c as flat edge-id triples\n")
        for c in range(256):
            f.write(" ".join(str(e) for tri in mc.case_triangles(c) for e in tri) + "\n")


if __name__ == "__main__":
    main()
