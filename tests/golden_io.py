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


def read_directions():
    """Graphs and hand-worked direction sequences of directions_worked.txt:
    (graphs {name: (n, src, dst)}, cases [(graph, source, rule, p0, p1, dirs)])."""
    graphs, cases = {}, []
    with open(os.path.join(GOLDEN, "directions_worked.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "graph":
                pairs = [tuple(int(x) for x in t.split("-")) for t in line[3:]]
                e = np.asarray(pairs, dtype=np.int32)
                graphs[line[1]] = (int(line[2]), e[:, 0].copy(), e[:, 1].copy())
            elif line[0] == "case":
                k = line.index(":")
                cases.append((line[1], int(line[2]), line[3], float(line[4]), float(line[5]),
                              [int(x) for x in line[k + 1:]]))
    return graphs, cases


def read_subgraph_directions():
    """Graphs and hand-worked per-subgraph direction sequences of
    subgraph_directions_worked.txt: (graphs {name: (n, th, src, dst)},
    cases [(graph, source, factor0[3], factor1[3], dirs)])."""
    graphs, cases = {}, []
    with open(os.path.join(GOLDEN, "subgraph_directions_worked.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "graph":
                pairs = [tuple(int(x) for x in t.split("-")) for t in line[4:]]
                e = np.asarray(pairs, dtype=np.int32)
                graphs[line[1]] = (int(line[2]), int(line[3]), e[:, 0].copy(), e[:, 1].copy())
            elif line[0] == "case":
                k = line.index(":")
                f = [float(x) for x in line[3:9]]
                cases.append((line[1], int(line[2]), f[:3], f[3:], [int(x) for x in line[k + 1:]]))
    return graphs, cases
