"""Parser for the hand-derived worked examples under tests/golden/*.txt.

Each file lists the lattice size, the budget, m_max, the flipped links of the
noise realisation N ("N x|y X Y" means e_x or e_y of site (X, Y)), and the
expected step count, failure flag and correction links.  An optional
"tie_order" line names the tie orders of Eq. degbreak (0 lexicographic,
1 literal key) under which the expectation holds; without it the case holds
under both (no exact key tie arises in it).  The derivations and
the paper passages they follow are in each file's comment header.
"""
import glob
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_case(path):
    L = max_steps = m_max = None
    n_links, c_links = [], []
    steps = flag = None
    ties = [0, 1]
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            key = tok[0]
            if key == "L":
                L = int(tok[1])
            elif key == "max_steps":
                max_steps = int(tok[1])
            elif key == "m_max":
                m_max = int(tok[1])
            elif key == "N":
                n_links.append((tok[1], int(tok[2]), int(tok[3])))
            elif key == "expect_C":
                c_links.append((tok[1], int(tok[2]), int(tok[3])))
            elif key == "expect_steps":
                steps = int(tok[1])
            elif key == "expect_flag":
                flag = int(tok[1])
            elif key == "tie_order":
                ties = [int(t) for t in tok[1:]]
            else:
                raise ValueError(f"{path}: unknown key {key}")
    N = np.zeros((2, L, L), dtype=np.uint8)
    for d, x, y in n_links:
        N[0 if d == "x" else 1, y, x] ^= 1
    C = np.zeros((2, L, L), dtype=np.uint8)
    for d, x, y in c_links:
        C[0 if d == "x" else 1, y, x] ^= 1
    return dict(name=os.path.basename(path)[:-4], L=L, max_steps=max_steps, m_max=m_max, N=N,
                C=C, steps=steps, flag=flag, tie_orders=ties)


def all_cases():
    return [load_case(p) for p in sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))
            if not os.path.basename(p).startswith("splitmix64")]
