"""Writes tests/golden/fj_small.json: exact Friedkin-Johnsen equilibria and
Table 1 measures of small graphs.

The paper prints no worked example, so these values come from the
definitions alone, independently of the oracle: z = (I + L)^{-1} s solved by
Gauss-Jordan elimination in rational arithmetic (fractions.Fraction), with
L = D - A and D the weighted out-degrees (Section 3.2; row u of A lists the
nodes u listens to), then the Table 1 sums C = sum z^2, P = sum (z - mean)^2,
I = sum (z - s)^2, D = sum over arcs of a_uv (z_u - z_v)^2 (an undirected
edge counted once).  Weights and opinions are dyadic rationals, so the float
inputs are exact.  Run: python tests/golden/make_golden.py
"""
import json
import os
from fractions import Fraction as F

GRAPHS = [
    # name, n, directed, arcs (u, v, weight): u listens to v, opinions
    ("path5_undirected", 5, False,
     [(0, 1, 1), (1, 2, 1), (2, 3, 1), (3, 4, 1)],
     [F(0), F(1, 4), F(1, 2), F(3, 4), F(1)]),
    ("star4_directed_in", 5, True,
     [(1, 0, 1), (2, 0, 1), (3, 0, 1), (4, 0, 1)],  # leaves listen to the centre
     [F(1), F(0), F(1, 2), F(1, 4), F(3, 4)]),
    ("weighted_digraph_unheard_node3", 4, True,
     [(0, 1, F(1, 2)), (0, 2, F(3, 2)), (1, 2, 1), (2, 0, F(1, 4)), (3, 2, 2)],
     [F(1, 8), F(5, 8), F(1), F(0)]),
    ("complete4_undirected", 4, False,
     [(u, v, 1) for u in range(4) for v in range(u + 1, 4)],
     [F(1), F(0), F(1, 2), F(1, 2)]),
]


def arcs_of(n, directed, edges):
    arcs = []
    for u, v, wt in edges:
        arcs.append((u, v, F(wt)))
        if not directed:
            arcs.append((v, u, F(wt)))
    return arcs


def solve_exact(n, arcs, s):
    m = [[F(0)] * n + [s[i]] for i in range(n)]
    for u, v, wt in arcs:
        m[u][u] += wt
        m[u][v] -= wt
    for i in range(n):
        m[i][i] += 1
    for c in range(n):
        p = next(r for r in range(c, n) if m[r][c] != 0)
        m[c], m[p] = m[p], m[c]
        piv = m[c][c]
        m[c] = [x / piv for x in m[c]]
        for r in range(n):
            if r != c and m[r][c] != 0:
                f = m[r][c]
                m[r] = [a - f * b for a, b in zip(m[r], m[c])]
    return [m[i][n] for i in range(n)]


def table1(n, directed, edges, s, z):
    mean = sum(z) / n
    d = sum(F(wt) * (z[u] - z[v]) ** 2 for u, v, wt in edges)  # each edge once
    return {"mean_z": mean, "C": sum(x * x for x in z), "P": sum((x - mean) ** 2 for x in z),
            "I": sum((x - y) ** 2 for x, y in zip(z, s)), "D": d}


def main():
    out = []
    for name, n, directed, edges, s in GRAPHS:
        arcs = arcs_of(n, directed, edges)
        z = solve_exact(n, arcs, s)
        met = table1(n, directed, edges, s, z)
        out.append({
            "name": name, "n": n, "directed": directed,
            "arcs": [[u, v, float(wt)] for u, v, wt in arcs],
            "s": [float(x) for x in s],
            "z": [float(x) for x in z], "z_exact": [str(x) for x in z],
            "metrics": {k: float(v) for k, v in met.items()},
            "metrics_exact": {k: str(v) for k, v in met.items()},
        })
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fj_small.json")
    with open(path, "w") as f:
        json.dump({"source": "exact rational solution of (I + L) z = s and Table 1 from their definitions",
                   "graphs": out}, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
