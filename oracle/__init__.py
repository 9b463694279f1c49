"""Plain FP64 CPU oracle for the Blast beyond-Limber C_l path (arXiv:2410.03632).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product library never calls it and shares no code with it; the C source
``oracle.c`` defines every step (see its header for the paper passages).

This module compiles ``oracle.c`` with the host compiler into
``oracle/_build/liboracle.so`` and wraps each C function with numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_LIB = None
_LOCK = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP, -O2, no fast-math)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            L = ctypes.CDLL(_SO)
            i, d = ctypes.c_int, ctypes.c_double
            L.orc_chi_grid.argtypes = [i, d, d, _dp, _dp]
            L.orc_R_grid.argtypes = [i, d, d, _dp, _dp]
            L.orc_R_grid_sym.argtypes = [i, _dp, _dp]
            L.orc_cc_grid.argtypes = [i, d, d, _dp, _dp, _dp, i]
            L.orc_cheb_knodes.argtypes = [i, d, d, i, _dp, _dp]
            L.orc_jl.argtypes = [i, d, _dp]
            L.orc_basis.argtypes = [i, _dp, i, _dp, _dp, i, d, d, i, i, i, _dp]
            L.orc_jnu.argtypes = [d, d, _dp]
            L.orc_cheb_dct.argtypes = [i, _dp, _dp]
            L.orc_spline_natural.argtypes = [i, _dp, _dp, i, _dp, _dp]
            L.orc_fit.argtypes = [i, d, d, i, i, _dp, _dp, _dp]
            L.orc_prefactor.argtypes = [i, d]
            L.orc_prefactor.restype = d
            L.orc_npairs.argtypes = [i, i]
            L.orc_cl.argtypes = [i, _dp, i, i, _dp, _dp, _dp, _dp, i, _dp, _dp, i, i,
                                 _dp, _dp, _dp, _dp, _dp, i, i]
            L.orc_limber.argtypes = [i, _dp, i, _dp, _dp, i, i, _dp, _dp, _dp, i, _dp]
            L.orc_cl_nonsep.argtypes = [i, _dp, i, i, _dp, _dp, _dp, i, _dp, _dp, i, i, _dp, _dp, _dp]
            L.orc_limber_plin.argtypes = [i, _dp, i, _dp, _dp, i, _dp, _dp, _dp]
            _LIB = L
    return _LIB


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


# --------------------------------------------------------------------------- grids
def chi_grid(X, lo, hi):
    chi, w = np.empty(X), np.empty(X)
    _check(lib().orc_chi_grid(X, lo, hi, _d(chi)[1], _d(w)[1]), "chi_grid")
    return chi, w


def R_grid(Rn, lo, hi):
    R, w = np.empty(Rn), np.empty(Rn)
    _check(lib().orc_R_grid(Rn, lo, hi, _d(R)[1], _d(w)[1]), "R_grid")
    return R, w


def R_grid_sym(Rn):
    """R nodes and weights on (0, 1] of the symmetrised form (App. A)."""
    R, w = np.empty(Rn), np.empty(Rn)
    _check(lib().orc_R_grid_sym(Rn, _d(R)[1], _d(w)[1]), "R_grid_sym")
    return R, w


def cc_grid(Nk, kmin, kmax, nthreads=0):
    k, x, w = np.empty(Nk), np.empty(Nk), np.empty(Nk)
    _check(lib().orc_cc_grid(Nk, kmin, kmax, _d(k)[1], _d(x)[1], _d(w)[1], nthreads), "cc_grid")
    return k, x, w


def cheb_knodes(N, kmin, kmax, kmap=0):
    t, k = np.empty(N), np.empty(N)
    _check(lib().orc_cheb_knodes(N, kmin, kmax, kmap, _d(t)[1], _d(k)[1]), "cheb_knodes")
    return t, k


# --------------------------------------------------------------------------- Bessel
def jl(lmax, x):
    out = np.empty(lmax + 1)
    _check(lib().orc_jl(int(lmax), float(x), _d(out)[1]), "jl")
    return out


def jnu(nu, x):
    """Spherical Bessel j_nu(x) of real order nu >= 0."""
    out = np.empty(1)
    _check(lib().orc_jnu(float(nu), float(x), _d(out)[1]), "jnu")
    return float(out[0])


# --------------------------------------------------------------------------- basis
def basis(ells, chi1, chi2, N, kmin, kmax, Nk, kmap=0, nthreads=0):
    """T~[t][e][n][q] for point pairs (chi1[q], chi2[q]); t = gg, gs, ss."""
    ells, pe = _d(ells)
    chi1, p1 = _d(chi1)
    chi2, p2 = _d(chi2)
    nq = chi1.size
    T = np.empty((3, ells.size, N, nq))
    _check(lib().orc_basis(ells.size, pe, nq, p1, p2, N, kmin, kmax, kmap, Nk, nthreads, _d(T)[1]), "basis")
    return T


# --------------------------------------------------------------------------- fit
def cheb_dct(vals):
    vals, pv = _d(vals)
    a = np.empty(vals.size)
    _check(lib().orc_cheb_dct(vals.size, pv, _d(a)[1]), "cheb_dct")
    return a


def spline_natural(u, v, uq):
    u, pu = _d(u)
    v, pv = _d(v)
    uq, pq = _d(uq)
    out = np.empty(uq.size)
    _check(lib().orc_spline_natural(u.size, pu, pv, uq.size, pq, _d(out)[1]), "spline_natural")
    return out


def fit(N, kmin, kmax, ktab, ptab, kmap=0):
    ktab, pk = _d(ktab)
    ptab, pp = _d(ptab)
    a = np.empty(N)
    _check(lib().orc_fit(N, kmin, kmax, kmap, ktab.size, pk, pp, _d(a)[1]), "fit")
    return a


def prefactor(t, ell):
    return lib().orc_prefactor(int(t), float(ell))


def npairs(ng, ns):
    return lib().orc_npairs(int(ng), int(ns))


# --------------------------------------------------------------------------- C_l
def cl(ells, chi, wchi, R, wR, T, a, ng, ns, kchi, kRchi, Dchi, DRchi, nthreads=0, sym=False):
    """C[p][e] from T~[3][n_ell][N][X*Rn] and the fitted a_n (steps 5-6);
    nthreads 0 = every OpenMP thread (independent (type, ell) items); sym: the
    symmetrised form of App. A (R in (0, 1], both kernel orders)."""
    ells, pe = _d(ells)
    chi, pc = _d(chi)
    wchi, pwc = _d(wchi)
    R, pR = _d(R)
    wR, pwR = _d(wR)
    T, pT = _d(T)
    a, pa = _d(a)
    kchi, pkc = _d(kchi)
    kRchi, pkR = _d(kRchi)
    Dchi, pDc = _d(Dchi)
    DRchi, pDR = _d(DRchi)
    N = a.size
    X, Rn = chi.size, R.size
    assert T.shape == (3, ells.size, N, X * Rn), T.shape
    C = np.empty((npairs(ng, ns), ells.size))
    _check(lib().orc_cl(ells.size, pe, X, Rn, pc, pwc, pR, pwR, N, pT, pa, ng, ns,
                        pkc, pkR, pDc, pDR, _d(C)[1], int(nthreads), int(bool(sym))), "cl")
    return C


# --------------------------------------------------------------------------- Limber
def limber(ells, chi, wchi, ng, ns, kchi, Dchi, P, extended=False):
    """Limber (or extended Limber) C[p][e] on the chi rule, P[e][a] = P(nu/chi_a, chi_a)."""
    ells, pe = _d(ells)
    chi, pc = _d(chi)
    wchi, pw = _d(wchi)
    kchi, pk = _d(kchi)
    Dchi, pD = _d(Dchi)
    P, pP = _d(P)
    assert P.shape == (ells.size, chi.size), P.shape
    C = np.empty((npairs(ng, ns), ells.size))
    _check(lib().orc_limber(ells.size, pe, chi.size, pc, pw, ng, ns, pk, pD, pP, int(bool(extended)),
                            _d(C)[1]), "limber")
    return C


def limber_plin(ells, chi, Dchi, ktab, ptab):
    """D(chi_a)^2 P(nu/chi_a) from a P table (natural spline in (ln k, ln P)), [e][a]."""
    ells, pe = _d(ells)
    chi, pc = _d(chi)
    Dchi, pD = _d(Dchi)
    ktab, pk = _d(ktab)
    ptab, pp = _d(ptab)
    P = np.empty((ells.size, chi.size))
    _check(lib().orc_limber_plin(ells.size, pe, chi.size, pc, pD, ktab.size, pk, pp, _d(P)[1]), "limber_plin")
    return P


def cl_nonsep(ells, chi, wchi, wR, T, Pq, ng, ns, kchi, kRchi):
    """C[p][e] for a non-separable P sampled at the Chebyshev k-nodes of every
    chi-R node, Pq[q][j] (q = a n_R + r)."""
    ells, pe = _d(ells)
    chi, pc = _d(chi)
    wchi, pw = _d(wchi)
    wR, pwR = _d(wR)
    T, pT = _d(T)
    Pq, pP = _d(Pq)
    kchi, pk = _d(kchi)
    kRchi, pkR = _d(kRchi)
    X, Rn, N = chi.size, wR.size, Pq.shape[1]
    assert T.shape == (3, ells.size, N, X * Rn) and Pq.shape == (X * Rn, N)
    C = np.empty((npairs(ng, ns), ells.size))
    _check(lib().orc_cl_nonsep(ells.size, pe, X, Rn, pc, pw, pwR, N, pT, pP, ng, ns, pk, pkR, _d(C)[1]),
           "cl_nonsep")
    return C


# --------------------------------------------------------------------------- plan-level helpers
class Grid:
    """The oracle's own grids for one plan description (all FP64)."""

    def __init__(self, ells, X, chi_min, chi_max, Rn, R_min, R_max, N, k_min, k_max, Nk, k_map=0, r_form=0):
        """r_form 0: R in [R_min, R_max] (two panels meeting at R = 1); 1: the
        symmetrised form on (0, 1] (App. A; R_min, R_max unused)."""
        self.ells = np.asarray(ells, dtype=np.float64)
        self.X, self.Rn, self.N, self.Nk, self.k_map = X, Rn, N, Nk, k_map
        self.k_min, self.k_max = k_min, k_max
        self.r_form = int(r_form)
        self.chi, self.wchi = chi_grid(X, chi_min, chi_max)
        self.R, self.wR = R_grid_sym(Rn) if self.r_form else R_grid(Rn, R_min, R_max)
        self.chi1 = np.repeat(self.chi, Rn)                 # q = a*Rn + r
        self.chi2 = (self.chi[:, None] * self.R[None, :]).ravel()

    def basis(self, ell_subset=None, nthreads=0):
        ells = self.ells if ell_subset is None else np.asarray(ell_subset, dtype=np.float64)
        return basis(ells, self.chi1, self.chi2, self.N, self.k_min, self.k_max, self.Nk,
                     self.k_map, nthreads)

    def fit(self, ktab, ptab):
        return fit(self.N, self.k_min, self.k_max, ktab, ptab, self.k_map)

    def cl_nonsep(self, T, Pq, ng, ns, kchi, kRchi, ell_subset=None):
        if self.r_form:
            raise NotImplementedError("the non-separable oracle uses the R in [R_min, R_max] form")
        ells = self.ells if ell_subset is None else np.asarray(ell_subset, dtype=np.float64)
        return cl_nonsep(ells, self.chi, self.wchi, self.wR, T, Pq, ng, ns, kchi, kRchi)

    def limber(self, ng, ns, kchi, Dchi, P, extended=False, ell_subset=None):
        ells = self.ells if ell_subset is None else np.asarray(ell_subset, dtype=np.float64)
        return limber(ells, self.chi, self.wchi, ng, ns, kchi, Dchi, P, extended)

    def limber_plin(self, Dchi, ktab, ptab, ell_subset=None):
        ells = self.ells if ell_subset is None else np.asarray(ell_subset, dtype=np.float64)
        return limber_plin(ells, self.chi, Dchi, ktab, ptab)

    def cl(self, T, a, ng, ns, kchi, kRchi, Dchi, DRchi, ell_subset=None, nthreads=0):
        ells = self.ells if ell_subset is None else np.asarray(ell_subset, dtype=np.float64)
        return cl(ells, self.chi, self.wchi, self.R, self.wR, T, a, ng, ns, kchi, kRchi, Dchi, DRchi,
                  nthreads, sym=self.r_form == 1)
