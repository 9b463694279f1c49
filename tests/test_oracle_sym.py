"""Pins of the oracle's symmetrised form (App. A: Eq. app1 and the change of
variables after it, R = chi2/chi1 in (0, 1] with both kernel orders) against
mathematics that shares none of its code.

S1  the R rule on (0, 1] (positive half of an odd first-kind Chebyshev rule
    with its Fejer-1 weights): even powers R^2k integrate exactly, odd powers
    converge, nodes lie in (0, 1) in increasing order;
S2  brute force: C_ij of gg, gs and ss at l = 2, 5, 10 against the double
    integral over (chi1, chi2) of K_i(chi1) K_j(chi2) w(chi1, chi2), with
    w from Gauss-Legendre in k with the exact P(k) and scipy's spherical Bessel
    functions, over the domain the symmetrised form covers
    (max(chi1, chi2) in [chi_min, chi_max]) -- no change of variables, no
    symmetrisation, no Chebyshev fit;
S3  for kernels whose support lies inside R in [R_min, R_max] of the split
    form, the symmetrised and the split forms give the same C_l.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2410_03632_gb300 import synth


def _gl(n, lo, hi):
    u, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (hi - lo) * (u + 1.0) + lo, 0.5 * (hi - lo) * w


def _f4(l):
    return (l + 2.0) * (l + 1.0) * l * (l - 1.0)


def _fejer1_mid(M):
    """Fejer-1 weight of the middle node (x = 0) of the M-point rule, from
    the rule's definition as the interpolatory quadrature on the nodes."""
    k = np.arange(M)
    x = np.cos((2 * k + 1) * np.pi / (2 * M))
    V = np.polynomial.chebyshev.chebvander(x, M - 1).T  # V[j][k] = T_j(x_k)
    m = np.array([2.0 / (1.0 - j * j) if j % 2 == 0 else 0.0 for j in range(M)])  # int T_j over [-1, 1]
    w = np.linalg.solve(V, m)
    return w[M // 2]


def test_s1_r_rule():
    for Rn in (8, 24, 48, 64):
        R, w = orc.R_grid_sym(Rn)
        assert np.all(np.diff(R) > 0) and R[0] > 0 and R[-1] < 1
        M = 2 * Rn + 1
        # even powers below the rule's degree that vanish at R = 0 (the dropped
        # middle node), and the constant with that node's half weight restored
        for k in range(2, M, 2):
            assert abs(np.sum(w * R ** k) - 1.0 / (k + 1)) < 1e-13, (Rn, k)
        assert abs(np.sum(w) - 0.5 * (2.0 - _fejer1_mid(M))) < 1e-13
    errs = []
    for Rn in (8, 16, 32, 64):
        R, w = orc.R_grid_sym(Rn)
        errs.append(abs(np.sum(w * R ** 3) - 0.25))
    assert errs[-1] < 1e-6 and errs[-1] < errs[0] / 50


def _sym_grid(ells, X=49, Rn=48):
    spec = synth.plan_spec("tiny")
    return orc.Grid(ells, X, spec.chi_min, spec.chi_max, Rn, spec.R_min, spec.R_max, spec.n_cheb, spec.k_min,
                    spec.k_max, spec.n_kquad, spec.k_map, r_form=1), spec


def test_s2_brute_force_over_the_plane():
    from scipy.special import spherical_jn
    ells = np.array([2, 5, 10], np.int32)
    g, spec = _sym_grid(ells)
    T = g.basis()
    mus_g, sig_g = np.array([0.12, 0.2]), np.array([0.04, 0.05])
    mus_s, sig_s = np.array([0.22]), np.array([0.04])
    rq = synth.make_request(g.chi, g.R, 2, 1, mus_g=mus_g, sig_g=sig_g, mus_s=mus_s, sig_s=sig_s)
    a = g.fit(rq.k_tab, rq.p_tab)
    Co = g.cl(T, a, 2, 1, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi)

    cos = synth.Cosmology(0.3)

    def kern(x):  # clustering 0, 1 and lensing 0 kernels times growth
        return np.stack([synth.clustering_kernel(cos, mus_g[0], sig_g[0], x),
                         synth.clustering_kernel(cos, mus_g[1], sig_g[1], x),
                         synth.lensing_kernel_over_chi2(cos, mus_s[0], sig_s[0], x)]) * cos.growth(x)

    kb = 0.05  # k rule: Gauss-Legendre in ln k below kb, in k above (oscillations)
    la, wa = _gl(384, np.log(spec.k_min), np.log(kb))
    kh, wh = _gl(2048, kb, spec.k_max)
    kk = np.concatenate([np.exp(la), kh])
    wk = np.concatenate([wa * np.exp(la), wh])
    P = synth.pk_eval(kk)
    # chi nodes on [0, chi_min] and [chi_min, chi_max]: the domain is every pair but
    # the ones with both chi below chi_min
    ca, wca = _gl(48, 0.0, spec.chi_min)
    cb, wcb = _gl(160, spec.chi_min, spec.chi_max)
    c = np.concatenate([ca, cb])
    wc = np.concatenate([wca, wcb])
    low = c < spec.chi_min
    mask = ~(low[:, None] & low[None, :])
    K = kern(c)
    f_k = {0: kk ** 2, 1: np.ones_like(kk), 2: kk ** -2.0}
    # pairs in the oracle's order: gg (0,0), (0,1), (1,1); gs (0,s), (1,s); ss (s,s)
    pairs = [(0, 0, 0), (0, 0, 1), (0, 1, 1), (1, 0, 2), (1, 1, 2), (2, 2, 2)]
    for e, l in enumerate(ells):
        J = spherical_jn(l, kk[:, None] * c[None, :])  # [k][node]
        N_AB = [2 / np.pi, 2 / np.pi * np.sqrt(_f4(l)), 2 / np.pi * _f4(l)]
        Wt = {}
        for t in range(3):
            Wt[t] = (J * (wk * f_k[t] * P)[:, None]).T @ J  # w(chi_a, chi_b) without N_AB
        for p, (t, A, B) in enumerate(pairs):
            bf = N_AB[t] * np.sum(mask * Wt[t] * np.outer(wc * K[A], wc * K[B]))
            assert abs(Co[p, e] / bf - 1.0) < 1e-2, (l, p, Co[p, e] / bf - 1.0)


def test_s3_split_and_symmetrised_forms_agree_inside_the_split_domain():
    ells = np.array([2, 10, 40], np.int32)
    spec = synth.plan_spec("tiny")
    # two narrow clustering bins around z ~ 0.2: their support (chi ~ 440..700)
    # lies inside both domains, chi2 / chi1 within [0.2, 1.8] and chi above 300
    kw = dict(mus_g=np.array([0.2, 0.21]), sig_g=np.array([0.012, 0.012]))
    out = []
    # with 96 R nodes the two rules differ by 4e-3 at l = 40, with 192 by 1.5e-5:
    # the forms converge to the same integral
    for r_form, Rn in ((0, 192), (1, 192)):
        g = orc.Grid(ells, 97, 300.0, spec.chi_max, Rn, 0.2, 1.8, spec.n_cheb, spec.k_min, spec.k_max,
                     synth.kquad_points(spec.k_min, spec.k_max, spec.chi_max, 1.8), spec.k_map, r_form=r_form)
        T = g.basis()
        rq = synth.make_request(g.chi, g.R, 2, 0, **kw)
        a = g.fit(rq.k_tab, rq.p_tab)
        out.append(g.cl(T, a, 2, 0, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi))
    assert np.max(np.abs(out[1] / out[0] - 1.0)) < 1e-4, out[1] / out[0] - 1.0
