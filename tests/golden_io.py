"""Readers for the text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_fig2():
    th = n = None
    delegates, edges = {}, []
    with open(os.path.join(GOLDEN, "fig2_separation.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "th":
                th = int(line[1])
            elif line[0] == "n":
                n = int(line[1])
            elif line[0] == "delegate":
                delegates[int(line[1])] = int(line[2])
            elif line[0] == "edge":
                edges.append((int(line[1]), int(line[2])))
    e = np.asarray(edges, dtype=np.int32)
    return th, n, delegates, e[:, 0].copy(), e[:, 1].copy()
