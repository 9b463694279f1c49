"""Seeded synthetic inputs shaped like the paper's 3x2pt workload.

This module produces only what a caller of the library supplies: the multipole
list, tracer kernels sampled at given comoving distances, the linear growth
factor at those distances and a tabulated linear P(k).  It holds none of the
method's arithmetic (no Chebyshev fit, no Bessel integral, no C_l quadrature),
so both the CUDA path and the CPU oracle can be fed from it.

Physics of the stand-in inputs (flat LCDM, distances in Mpc/h, k in h/Mpc):
  * E(z) = sqrt(Om (1+z)^3 + 1 - Om), chi(z) = (c/H0) int_0^z dz'/E(z'),
    c/H0 = 2997.92458 Mpc/h;
  * growth D(a) proportional to E(a) int_0^a da' / (a' E(a'))^3, D(z=0) = 1;
  * tomographic n_i(z): Gaussians truncated at z >= 0, unit normalised;
  * clustering kernel W^g_i(chi) = H(z) n_i(z) b with b = 1 (Sec. 3.1 of the
    paper), i.e. n_i(z) dz/dchi;
  * lensing kernel W^s_i(chi) = (3 H0^2 Om / 2a) chi int_z^inf dz' n_i(z')
    (chi(z') - chi) / chi(z'), passed to the library divided by chi^2 as the
    paper's calligraphic K (Eq. final_cls);
  * P(k) = A (k/kp) / (1 + (k/kp)^(1-n2)) (1 + a_w sin(k r_w + phi) exp(-(k/0.3)^2))
    on 256 log-spaced points in [1e-4, 10], kp = 0.02, r_w = 105, A = 5e4 (s8/0.8)^2.
"""
from __future__ import annotations

import dataclasses

import numpy as np

C_OVER_H0 = 2997.92458  # Mpc/h


# ----------------------------------------------------------------------------- multipoles
def ell_list(n: int, lo: int, hi: int) -> np.ndarray:
    """n distinct integer multipoles, log-spaced over [lo, hi]: round each point
    of geomspace(lo, hi, n) and move a collision to the next unused integer."""
    out = []
    for v in np.geomspace(lo, hi, n):
        l = int(round(v))
        if out and l <= out[-1]:
            l = out[-1] + 1
        out.append(l)
    return np.asarray(out, dtype=np.int32)


# ----------------------------------------------------------------------------- cosmology
class Cosmology:
    """Flat LCDM background: chi(z), z(chi), E(z), D(z) from fine tables."""

    def __init__(self, Om: float = 0.3, zmax: float = 60.0, nz: int = 60001):
        self.Om = float(Om)
        # dense near z = 0 (where small chi lives), coarser at high z
        u = np.linspace(0.0, np.log1p(zmax), nz)
        z = np.expm1(u)
        E = self.E(z)
        dchi = C_OVER_H0 / E * np.gradient(z, u)  # dchi/du
        chi = np.concatenate([[0.0], np.cumsum(0.5 * (dchi[1:] + dchi[:-1]) * np.diff(u))])
        self._z, self._chi = z, chi
        # growth: D(a) ~ E(a) int_0^a da'/(a'E)^3 (integrand ~ a'^{3/2}/Om^{3/2} near 0)
        a = np.linspace(1e-6, 1.0, 200001)
        za = 1.0 / a - 1.0
        integrand = 1.0 / (a * self.E(za)) ** 3
        I = np.concatenate([[0.0], np.cumsum(0.5 * (integrand[1:] + integrand[:-1]) * np.diff(a))])
        g = self.E(za) * I
        self._a, self._D = a, g / g[-1]

    def E(self, z):
        return np.sqrt(self.Om * (1.0 + z) ** 3 + 1.0 - self.Om)

    def chi(self, z):
        return np.interp(z, self._z, self._chi)

    def z_of_chi(self, chi):
        return np.interp(chi, self._chi, self._z)

    def growth(self, chi):
        z = self.z_of_chi(chi)
        return np.interp(1.0 / (1.0 + z), self._a, self._D)


def nz_gaussian(z, mu, sigma):
    """Gaussian n(z) truncated at z >= 0 and normalised to unit integral."""
    from math import erf, sqrt
    norm = 0.5 * (1.0 - erf(-mu / (sqrt(2.0) * sigma)))
    return np.where(z >= 0.0, np.exp(-0.5 * ((z - mu) / sigma) ** 2)
                    / (sigma * np.sqrt(2.0 * np.pi) * norm), 0.0)


def clustering_kernel(cosmo: Cosmology, mu, sigma, chi):
    """W^g(chi) = n(z(chi)) H(z)/c with unit bias."""
    chi = np.asarray(chi, dtype=np.float64)
    z = cosmo.z_of_chi(chi)
    return nz_gaussian(z, mu, sigma) * cosmo.E(z) / C_OVER_H0


def lensing_kernel_over_chi2(cosmo: Cosmology, mu, sigma, chi, nzg: int = 20001):
    """W^s(chi) / chi^2 for a source distribution n(z) = Gaussian(mu, sigma)."""
    chi = np.asarray(chi, dtype=np.float64)
    zhi = mu + 12.0 * sigma
    zg = np.linspace(0.0, zhi, nzg)
    zg[0] = 1e-7
    n = nz_gaussian(zg, mu, sigma)
    chig = cosmo.chi(zg)
    # tail integrals int_z^zhi n dz' and int_z^zhi n / chi(z') dz' (trapezoid from the top)
    def tail(f):
        seg = 0.5 * (f[1:] + f[:-1]) * np.diff(zg)
        return np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
    N1 = tail(n)
    N2 = tail(n / chig)
    z = cosmo.z_of_chi(chi)
    t1 = np.interp(z, zg, N1, right=0.0)
    t2 = np.interp(z, zg, N2, right=0.0)
    pref = 1.5 * cosmo.Om / C_OVER_H0 ** 2 * (1.0 + z)
    W = pref * chi * np.maximum(t1 - chi * t2, 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(chi > 0.0, W / chi ** 2, 0.0)


def pk_eval(k, n2=-2.0, a_w=0.05, phi=0.0, s8=0.8):
    """Smooth broken power law with damped BAO-like wiggles, at any k (h/Mpc)."""
    k = np.asarray(k, dtype=np.float64)
    kp, rw = 0.02, 105.0
    A = 5e4 * (s8 / 0.8) ** 2
    x = k / kp
    return A * x / (1.0 + x ** (1.0 - n2)) * (1.0 + a_w * np.sin(k * rw + phi) * np.exp(-(k / 0.3) ** 2))


def pk_table(n2=-2.0, a_w=0.05, phi=0.0, s8=0.8, n=256, kmin=1e-4, kmax=10.0):
    """pk_eval tabulated on n log-spaced points."""
    k = np.geomspace(kmin, kmax, n)
    return k, pk_eval(k, n2, a_w, phi, s8)


# ----------------------------------------------------------------------------- workloads
@dataclasses.dataclass
class PlanSpec:
    """Grid description shared by the library plan and the oracle grid."""
    ells: np.ndarray
    n_chi: int
    chi_min: float
    chi_max: float
    n_R: int
    R_min: float
    R_max: float
    n_cheb: int
    k_min: float
    k_max: float
    k_map: int
    n_kquad: int
    max_clust: int
    max_lens: int
    r_form: int = 0  # 0: R in [R_min, R_max]; 1: the symmetrised form on (0, 1]


def kquad_points(k_min, k_max, chi_max, R_max):
    """Clenshaw-Curtis size 2^m + 1 with 2^m >= (k_max - k_min)/2 (1 + R_max) chi_max:
    the highest frequency of j_l(k chi1) j_l(k chi2) in the Chebyshev variable."""
    need = 0.5 * (k_max - k_min) * (1.0 + R_max) * chi_max
    m = max(4, int(np.ceil(np.log2(need))))
    return 2 ** m + 1


@dataclasses.dataclass
class Request:
    """One cosmology's inputs at the plan nodes (all float64, C order)."""
    n_clust: int
    n_lens: int
    kern_chi: np.ndarray    # [n_clust + n_lens][n_chi]
    kern_Rchi: np.ndarray   # [n_clust + n_lens][n_chi * n_R]
    growth_chi: np.ndarray  # [n_chi]
    growth_Rchi: np.ndarray # [n_chi * n_R]
    k_tab: np.ndarray
    p_tab: np.ndarray
    ell_mask: int = 0       # bitmask over plan ells (0 = all)


def bins(n, lo=0.2, hi=1.5, slo=0.05, shi=0.15):
    if n == 1:
        return np.array([0.5]), np.array([0.1])
    return np.linspace(lo, hi, n), np.linspace(slo, shi, n)


def make_request(chi, R, n_clust, n_lens, Om=0.3, n2=-2.0, a_w=0.05, phi=0.0, s8=0.8,
                 mus_g=None, sig_g=None, mus_s=None, sig_s=None, ell_mask=0) -> Request:
    """Kernels and growth at the nodes chi[a] and R[r] chi[a] for one cosmology."""
    chi = np.asarray(chi, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    chiR = (chi[:, None] * R[None, :]).ravel()
    cosmo = Cosmology(Om)
    if mus_g is None:
        mus_g, sig_g = bins(n_clust)
    if mus_s is None:
        mus_s, sig_s = bins(n_lens)
    kc, kR = [], []
    for i in range(n_clust):
        kc.append(clustering_kernel(cosmo, mus_g[i], sig_g[i], chi))
        kR.append(clustering_kernel(cosmo, mus_g[i], sig_g[i], chiR))
    for i in range(n_lens):
        kc.append(lensing_kernel_over_chi2(cosmo, mus_s[i], sig_s[i], chi))
        kR.append(lensing_kernel_over_chi2(cosmo, mus_s[i], sig_s[i], chiR))
    ktab, ptab = pk_table(n2, a_w, phi, s8)
    return Request(n_clust, n_lens,
                   np.ascontiguousarray(np.array(kc).reshape(n_clust + n_lens, chi.size)),
                   np.ascontiguousarray(np.array(kR).reshape(n_clust + n_lens, chiR.size)),
                   cosmo.growth(chi), cosmo.growth(chiR), ktab, ptab, ell_mask)


# Grid shapes of the benchmark workloads (the config numbering follows the
# workload list this project benchmarks against): 0 small FP64, 1 the 3x2pt
# 5+5 bin workload, 2 the 10+10 bin precision workload.
def plan_spec(name: str) -> PlanSpec:
    if name == "c0":
        e, X, cmax, Rn, N, ng, ns = ell_list(16, 2, 200), 64, 2600.0, 64, 32, 1, 1
    elif name == "c1":
        e, X, cmax, Rn, N, ng, ns = ell_list(64, 2, 1000), 128, 4100.0, 128, 64, 5, 5
    elif name == "c2":
        e, X, cmax, Rn, N, ng, ns = ell_list(100, 2, 2000), 256, 4100.0, 192, 96, 10, 10
    elif name == "tiny":
        # several ragged tiles in every dimension, k range cut so the oracle is fast
        return PlanSpec(np.array([2, 3, 7, 15, 40], np.int32), 13, 60.0, 900.0, 10, 0.3, 1.7,
                        20, 1e-3, 1.0, 1, kquad_points(1e-3, 1.0, 900.0, 1.7), 2, 2)
    elif name == "small":
        return PlanSpec(ell_list(11, 2, 120), 41, 40.0, 2400.0, 26, 0.2, 1.8, 35, 1e-4, 1.0, 1,
                        kquad_points(1e-4, 1.0, 2400.0, 1.8), 3, 2)
    elif name == "c2s":
        # the 10+10-bin grid's shapes (n_R = 192, order 96, 20 tracers, chi to 4100) on
        # few ells and chi nodes with k_max = 1, so the oracle's basis takes seconds
        return PlanSpec(np.array([2, 30, 120, 300], np.int32), 24, 26.0, 4100.0, 192, 0.2, 1.8, 96, 1e-4, 1.0, 1,
                        kquad_points(1e-4, 1.0, 4100.0, 1.8), 10, 10)
    elif name == "c1hi":
        # the 3x2pt grid's k range (to 10 h/Mpc), order 64, bins and chi range on
        # nine chi nodes, n_R = 64 and four ells to 1000: high-l lensing spectra of
        # the z = 0.2 bin, where the Chebyshev sum cancels hardest, at a size the
        # oracle's basis finishes in about a minute
        return PlanSpec(np.array([2, 300, 600, 1000], np.int32), 9, 26.0, 4100.0, 64, 0.2, 1.8, 64,
                        1e-4, 10.0, 1, kquad_points(1e-4, 10.0, 4100.0, 1.8), 5, 5)
    elif name == "tcg":
        # tensor-core shapes with two groups of tracer weights (7 + 6 tracers), order 40
        return PlanSpec(ell_list(6, 2, 250), 13, 40.0, 2400.0, 64, 0.2, 1.8, 40, 1e-4, 1.0, 1,
                        kquad_points(1e-4, 1.0, 2400.0, 1.8), 7, 6)
    elif name == "tck":
        # tensor-core shapes with the order past 64 (two K chunks, four TMEM levels), order 80
        return PlanSpec(ell_list(6, 2, 250), 13, 40.0, 2400.0, 64, 0.2, 1.8, 80, 1e-4, 1.0, 1,
                        kquad_points(1e-4, 1.0, 2400.0, 1.8), 3, 2)
    elif name == "tc":
        # tensor-core path shapes: n_R a multiple of 32, n_cheb <= 64, <= 5 tracers per kind
        return PlanSpec(ell_list(9, 2, 300), 21, 40.0, 2400.0, 64, 0.2, 1.8, 40, 1e-4, 1.0, 1,
                        kquad_points(1e-4, 1.0, 2400.0, 1.8), 3, 2)
    else:
        raise KeyError(name)
    return PlanSpec(e, X, 26.0, cmax, Rn, 0.2, 1.8, N, 1e-4, 10.0, 1,
                    kquad_points(1e-4, 10.0, cmax, 1.8), ng, ns)


def ragged_request(chi, R, idx: int, n_ell: int):
    """Request idx of the ragged batch on the 10+10-bin grid: its own tracer
    counts drawn from 2..10 of each kind, its own ell set (a random subset of
    16..n_ell of the plan's ells) and cosmology (seed 1003 + 7919 idx).
    Returns (Request, sorted list of selected plan-ell indices)."""
    rng = np.random.default_rng(1003 + 7919 * idx)
    ng, ns = int(rng.integers(2, 11)), int(rng.integers(2, 11))
    k = int(rng.integers(16, n_ell + 1))
    sel = sorted(int(x) for x in rng.choice(n_ell, size=k, replace=False))
    n2, a_w = rng.uniform(-2.5, -1.5), rng.uniform(0.03, 0.08)
    phi, Om, s8 = rng.uniform(0.0, 2 * np.pi), rng.uniform(0.25, 0.35), rng.uniform(0.7, 0.9)
    return make_request(chi, R, ng, ns, Om=Om, n2=n2, a_w=a_w, phi=phi, s8=s8), sel


def config_request(name: str, chi, R, idx: int = 0) -> Request:
    """The seeded request of a workload: seed 1000 + config + 7919 idx."""
    spec = plan_spec(name)
    cfg = {"c0": 0, "c1": 1, "c2": 2, "tiny": 10, "small": 11, "tc": 12, "c2s": 13, "c1hi": 1, "tcg": 14,
           "tck": 15}[name]
    rng = np.random.default_rng(1000 + cfg + 7919 * idx)
    ng, ns = spec.max_clust, spec.max_lens
    zb = {}
    if name == "tiny":   # grid reaches z ~ 0.33
        zb = dict(mus_g=np.array([0.1, 0.2]), sig_g=np.array([0.02, 0.04]),
                  mus_s=np.array([0.22, 0.3]), sig_s=np.array([0.03, 0.05]))
    elif name in ("small", "tc", "tcg", "tck"):  # grid reaches z ~ 1.1
        zb = dict(mus_g=np.linspace(0.2, 0.7, ng), sig_g=np.linspace(0.05, 0.1, ng),
                  mus_s=np.linspace(0.5, 0.8, ns), sig_s=np.linspace(0.08, 0.12, ns))
    if name == "c0" and idx == 0:
        return make_request(chi, R, ng, ns, Om=0.3, n2=-2.0, a_w=0.05, phi=0.0)
    n2 = rng.uniform(-2.5, -1.5)
    a_w = rng.uniform(0.03, 0.08)
    phi = 0.0 if idx == 0 else rng.uniform(0.0, 2 * np.pi)
    Om = 0.3 if idx == 0 else rng.uniform(0.25, 0.35)
    s8 = 0.8 if idx == 0 else rng.uniform(0.7, 0.9)
    return make_request(chi, R, ng, ns, Om=Om, n2=n2, a_w=a_w, phi=phi, s8=s8, **zb)
