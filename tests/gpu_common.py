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


U64 = 2.0 ** -53  # unit roundoff of FP64


def certificate_holds(n, rp, col, w, s, z, c_eff, epsp, slack=1.0):
    """Recompute the certificate of the GPU result on the CPU (Lemma 5's premise).

    The shifted system's residual s' - (I + L)(z + c_eff) equals s - (I + L) z
    (rows of L sum to zero), so it is evaluated on the returned z, with
    compensated sums (exact to a few ulp).  Allowed per node: the solver's test
    max(eps' s'_v, 2^-51 (1 + d_v) |z'_v|) (the second term is the FP64
    resolution of row v: one ulp of z'_v moves r_v by (1 + d_v) ulp), plus
    what rounding z' - c_eff and s + c_eff once per entry can change:
    u ((1 + d_v)|z_v| + sum_c a_vc |z_c| + |s'_v|).
    """
    r = oracle.residual_accurate(n, rp, col, w, s, z)
    d = oracle.out_degree(n, rp, w)
    sp = s + c_eff
    zp = z + c_eff
    wa = np.ones(col.shape[0]) if w is None else np.asarray(w, np.float64)
    rows = np.repeat(np.arange(n), np.diff(rp))
    nb = np.bincount(rows, weights=wa * np.abs(z[col]), minlength=n)
    thr = np.maximum(epsp * sp, 2.0 ** -51 * (1.0 + d) * np.abs(zp))
    rnd = U64 * ((1.0 + d) * np.abs(z) + nb + np.abs(sp))
    ok = bool(np.all(np.abs(r) <= slack * thr * (1 + 1e-9) + 2.0 * rnd + 1e-300))
    return ok, r
