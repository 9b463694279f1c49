"""Error metrics used by the tests (no method arithmetic).

Spectra of distant bins cross zero, so errors are normalised by the auto
spectra: e_ij(l) = |C_ij - C_ij,ref| / sqrt(C_ii^AA C_jj^BB), the error in
correlation-coefficient units, with the pair order gg (i <= j), gs (all i, j),
ss (i <= j).
"""
import numpy as np


def pair_list(ng, ns):
    """[(type, i, j)] in output order; type 0 = gg, 1 = gs, 2 = ss."""
    out = [(0, i, j) for i in range(ng) for j in range(i, ng)]
    out += [(1, i, j) for i in range(ng) for j in range(ns)]
    out += [(2, i, j) for i in range(ns) for j in range(i, ns)]
    return out


def auto_index(ng, ns):
    """Row of each auto spectrum: gg(i,i) and ss(i,i)."""
    pl = pair_list(ng, ns)
    g = {i: pl.index((0, i, i)) for i in range(ng)}
    s = {i: pl.index((2, i, i)) for i in range(ns)}
    return g, s


def eij(C, ref, ng, ns):
    """e_ij(l) for every pair and ell, as an array shaped like C."""
    C = np.asarray(C, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    pl = pair_list(ng, ns)
    g, s = auto_index(ng, ns)
    out = np.empty_like(ref)
    for p, (t, i, j) in enumerate(pl):
        a = ref[g[i]] if t < 2 else ref[s[i]]
        b = ref[g[j]] if t == 0 else ref[s[j]]
        out[p] = np.abs(C[p] - ref[p]) / np.sqrt(np.abs(a * b))
    return out
