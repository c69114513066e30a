"""Helpers shared by the GPU parity tests: graph construction on both sides and
the comparison rules (tolerances stated where they are used)."""
import numpy as np

import oracle
from fjsynth import workloads as W

FP64_TOL = 1e-6   # ||z - z*||_inf / ||z*||_inf for the FP64 path
FP32_TOL = 1e-5   # the same for the FP32 paths
METRIC_TOL = 1e-5  # relative error of P, D, I, C against the oracle's values on z*


def csr_of(g):
    """Oracle-side CSR of a workload dict (undirected edge lists become both arcs)."""
    if g["directed"]:
        return oracle.csr_from_arcs(g["n"], g["src"], g["dst"], g["w"])
    a, b, c = W.symmetrize_arcs(g["src"], g["dst"], g["w"])
    return oracle.csr_from_arcs(g["n"], a, b, c)


def rel_inf(z, z_star):
    return float(np.max(np.abs(z - z_star)) / np.max(np.abs(z_star)))


def to_dev(*arrays):
    import torch
    out = []
    for a in arrays:
        out.append(None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda())
    return out


def certificate_holds(n, rp, col, w, s, z, c_eff, epsp, slack=1.0):
    """Recompute the FP64 residual of the GPU result on the CPU (Lemma 5's premise)."""
    r = oracle.residual(n, rp, col, w, s + c_eff, z + c_eff)
    return bool(np.all(np.abs(r) <= slack * epsp * (s + c_eff) * (1 + 1e-9) + 1e-300)), r
