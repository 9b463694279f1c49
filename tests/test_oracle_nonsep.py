"""Pins of the oracle's non-separable C_l (general c_n(chi1, chi2), Eqs.
cheb_pk and pmd) against the pinned growth-separable oracle.

N1  a separable spectrum D(chi1) D(chi2) P(k) sampled at the Chebyshev
    k-nodes of every chi-R node gives the separable oracle's C_l;
N2  a rank-two spectrum D1 D2 P_A(k) + G1 G2 P_B(k) (two growth laws, so no
    single c_n(chi1) c_n(chi2) factorisation) gives the sum of the two
    separable results (the per-node fit and contraction are linear).
"""
import numpy as np
from numpy.polynomial import chebyshev as cheb

import oracle as orc
from paper_2410_03632_gb300 import synth


def _case():
    spec = synth.plan_spec("tiny")
    g = orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min, spec.R_max,
                 spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map)
    T = g.basis()
    rq = synth.config_request("tiny", g.chi, g.R, 1)
    t, _ = orc.cheb_knodes(spec.n_cheb, spec.k_min, spec.k_max, spec.k_map)
    return spec, g, T, rq, t


def test_n1_separable_spectrum_reduces_to_the_separable_oracle():
    spec, g, T, rq, t = _case()
    a = g.fit(rq.k_tab, rq.p_tab)
    Pn = cheb.chebval(t, a)                              # P at the nodes: the interpolant through them
    D1 = np.repeat(rq.growth_chi, spec.n_R)
    Pq = (D1 * rq.growth_Rchi)[:, None] * Pn[None, :]
    C = g.cl_nonsep(T, Pq, rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi)
    Cs = g.cl(T, a, rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi)
    assert np.allclose(C, Cs, rtol=1e-12, atol=1e-14 * np.max(np.abs(Cs)))


def test_n2_rank_two_spectrum_is_the_sum_of_two_separable_ones():
    spec, g, T, rq, t = _case()
    kA, pA = synth.pk_table(-2.0, 0.05, 0.0, 0.8)
    kB, pB = synth.pk_table(-1.6, 0.02, 1.0, 0.5)
    aA, aB = g.fit(kA, pA), g.fit(kB, pB)
    GA_chi, GA_R = rq.growth_chi, rq.growth_Rchi
    GB_chi = 1.0 / (1.0 + g.chi / 3000.0)
    GB_R = 1.0 / (1.0 + g.chi2 / 3000.0)
    Pq = ((np.repeat(GA_chi, spec.n_R) * GA_R)[:, None] * cheb.chebval(t, aA)[None, :]
          + (np.repeat(GB_chi, spec.n_R) * GB_R)[:, None] * cheb.chebval(t, aB)[None, :])
    C = g.cl_nonsep(T, Pq, rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi)
    Cs = (g.cl(T, aA, rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, GA_chi, GA_R)
          + g.cl(T, aB, rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, GB_chi, GB_R))
    assert np.allclose(C, Cs, rtol=1e-11, atol=1e-13 * np.max(np.abs(Cs)))
