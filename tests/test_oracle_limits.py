"""Pins of the oracle's whole C_l against two limits that share none of its code.

O4, Limber limit: at high l, C^AB_ij tends to the Limber integral
    gg: int dchi W_i W_j P(nu/chi) / chi^2
    gs: sqrt((l+2)(l+1)l(l-1)) / nu^2 int dchi W_i K_j P(nu/chi)
    ss: (l+2)(l+1)l(l-1) / nu^4 int dchi K_i K_j chi^2 P(nu/chi)
with nu = l + 1/2, P(k) D^2 the same Chebyshev interpolant (zero outside
[k_min, k_max]) and K = W / chi^2 the lensing kernel (Sec. 2, Limber limit of
Eqs. gg, gs, ss).  The relative gap shrinks as l grows.

O5, brute force: the triple integral of Eqs. gg, gs, ss over the same
chi1-in-[chi_min, chi_max], chi2/chi1-in-[R_min, R_max] domain by Gauss-Legendre
in chi1, R and k, with the exact P(k) and scipy's spherical Bessel functions
(no Chebyshev fit, no basis table).  The gap is the oracle's discretisation:
Chebyshev order, chi and R rules and the k quadrature.
"""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as cheb

import oracle as orc
from paper_2410_03632_gb300 import synth


def _gl(n, lo, hi):
    u, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (hi - lo) * (u + 1.0) + lo, 0.5 * (hi - lo) * w


def _f4(l):
    return (l + 2.0) * (l + 1.0) * l * (l - 1.0)


def test_limber_limit_at_high_ell():
    ells = np.array([25, 50, 100], np.int32)
    cmin, cmax, kmin, kmax, N = 200.0, 3000.0, 1e-3, 1.0, 32
    g = orc.Grid(ells, 64, cmin, cmax, 64, 0.2, 1.8, N, kmin, kmax, synth.kquad_points(kmin, kmax, cmax, 1.8), 1)
    T = g.basis()
    mg, sg, ms, ss = 0.45, 0.08, 0.9, 0.1
    rq = synth.make_request(g.chi, g.R, 1, 1, mus_g=np.array([mg]), sig_g=np.array([sg]),
                            mus_s=np.array([ms]), sig_s=np.array([ss]))
    a = g.fit(rq.k_tab, rq.p_tab)
    C = g.cl(T, a, 1, 1, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi)

    cos = synth.Cosmology(0.3)
    xs = np.linspace(cmin, cmax, 100001)
    Wg = synth.clustering_kernel(cos, mg, sg, xs)
    Ks = synth.lensing_kernel_over_chi2(cos, ms, ss, xs)
    D2 = cos.growth(xs) ** 2
    gap = np.empty((3, ells.size))
    for e, l in enumerate(ells):
        nu = l + 0.5
        k = nu / xs
        x = 2.0 * (np.log(k) - np.log(kmin)) / (np.log(kmax) - np.log(kmin)) - 1.0
        P = np.where((k >= kmin) & (k <= kmax), cheb.chebval(np.clip(x, -1.0, 1.0), a), 0.0) * D2
        gg = np.trapezoid(Wg * Wg * P / xs ** 2, xs)
        gs = np.sqrt(_f4(l)) / nu ** 2 * np.trapezoid(Wg * Ks * P, xs)
        sss = _f4(l) / nu ** 4 * np.trapezoid(Ks * Ks * P * xs ** 2, xs)
        gap[:, e] = C[:, e] / np.array([gg, gs, sss]) - 1.0
    # close to Limber (a dropped prefactor, growth or 1/chi^2 would be O(1) off) ...
    assert np.all(np.abs(gap[0]) < 2e-2)
    assert np.all(np.abs(gap[1]) < 5e-3)
    assert np.all(np.abs(gap[2]) < 1e-3)
    # ... and closer as l grows
    assert abs(gap[0, -1]) < 0.5 * abs(gap[0, 0])
    assert abs(gap[1, -1]) < 0.5 * abs(gap[1, 0])


@pytest.mark.slow
def test_brute_force_triple_integral_at_low_ell():
    from scipy.special import spherical_jn
    spec = synth.plan_spec("tiny")
    ells = np.array([2, 5, 10], np.int32)
    g = orc.Grid(ells, 49, spec.chi_min, spec.chi_max, 48, spec.R_min, spec.R_max, spec.n_cheb, spec.k_min,
                 spec.k_max, spec.n_kquad, spec.k_map)
    T = g.basis()
    mg, sg, ms, ss = 0.15, 0.06, 0.25, 0.05
    rq = synth.make_request(g.chi, g.R, 1, 1, mus_g=np.array([mg]), sig_g=np.array([sg]),
                            mus_s=np.array([ms]), sig_s=np.array([ss]))
    a = g.fit(rq.k_tab, rq.p_tab)
    Co = g.cl(T, a, 1, 1, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi)

    cos = synth.Cosmology(0.3)

    def kern(x):  # [clustering, lensing] kernels times growth
        return np.stack([synth.clustering_kernel(cos, mg, sg, x),
                         synth.lensing_kernel_over_chi2(cos, ms, ss, x)]) * cos.growth(x)

    kb = 0.05  # k rule: Gauss-Legendre in ln k below kb, in k above (oscillations)
    la, wa = _gl(384, np.log(spec.k_min), np.log(kb))
    kh, wh = _gl(2048, kb, spec.k_max)
    kk = np.concatenate([np.exp(la), kh])
    wk = np.concatenate([wa * np.exp(la), wh])
    P = synth.pk_eval(kk)  # exact P, not the table
    c1, w1 = _gl(100, spec.chi_min, spec.chi_max)
    Rg, wR = _gl(100, spec.R_min, spec.R_max)
    K1 = kern(c1)
    c2 = c1[:, None] * Rg[None, :]
    K2 = kern(c2.ravel()).reshape(2, c1.size, Rg.size)
    f_k = {0: kk ** 2, 1: np.ones_like(kk), 2: kk ** -2.0}
    pairs = [(0, 0, 0), (1, 0, 1), (2, 1, 1)]  # (type, A tracer, B tracer): gg, gs, ss
    for e, l in enumerate(ells):
        acc = np.zeros(3)
        for i0 in range(0, kk.size, 256):
            ks = slice(i0, i0 + 256)
            j1 = spherical_jn(l, kk[ks, None] * c1[None, :])
            j2 = spherical_jn(l, kk[ks, None, None] * c2[None, :, :])
            for p, (t, A, B) in enumerate(pairs):
                inner = np.einsum("kar,r,ar->ka", j2, wR, K2[B])       # dchi2 = chi1 dR
                F = np.einsum("ka,a->k", j1 * inner, w1 * c1 * K1[A])
                acc[p] += np.sum(wk[ks] * f_k[t][ks] * P[ks] * F)
        N_AB = np.array([2 / np.pi, 2 / np.pi * np.sqrt(_f4(l)), 2 / np.pi * _f4(l)])
        bf = N_AB * acc
        assert np.all(np.abs(Co[:, e] / bf - 1.0) < 1e-2), (l, Co[:, e] / bf - 1.0)
