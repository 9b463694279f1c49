"""Pins of the oracle's non-integer multipoles (App. A evaluates the basis at
l = 211.63, not an integer) against mathematics that shares none of its code.

E1  j_nu(x) for real nu against mpmath's J_{nu+1/2} at 40 digits times
    sqrt(pi/2x), over small, transitional and large arguments (scipy's own
    J is off by 1e-11 of the envelope at x ~ 1e4 and nu ~ 200, the oracle by
    under 1e-12); at integer nu it equals the integer ladder;
E2  the basis of every type at real ells against composite Gauss-Legendre in k
    with scipy's Bessel functions (no Clenshaw-Curtis rule, no recurrence);
E3  the prefactors at real l against Gamma(l + 3) / Gamma(l - 1).
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import oracle as orc
from paper_2410_03632_gb300 import synth


def _jnu_ref(nu, x):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    return float(mp.sqrt(mp.pi / (2 * mp.mpf(x))) * mp.besselj(mp.mpf(nu) + mp.mpf(1) / 2, mp.mpf(x)))


@pytest.mark.parametrize("nu", [2.3, 7.5, 17.25, 211.63, 999.9])
def test_e1_jnu_against_mpmath(nu):
    xs = np.concatenate([np.geomspace(1e-2, 0.9 * nu, 25), np.linspace(0.9 * nu, 1.1 * nu, 21),
                         np.geomspace(1.1 * nu, 8e3, 20)])
    for x in xs:
        got = orc.jnu(nu, x)
        if abs(math.sqrt(math.pi / (2.0 * x)) * sp.jv(nu + 0.5, x)) < 1e-280:  # deep in the tail: both vanish
            assert abs(got) < 1e-270
            continue
        ref = _jnu_ref(nu, x)
        # relative to the envelope of j_nu near x (zeros of the oscillation)
        env = max(abs(ref), 1.0 / max(x, nu + 0.5) if x > nu else abs(ref))
        assert abs(got - ref) <= 2e-12 * env, (nu, x, got, ref)


def test_e1_integer_orders_match_the_ladder():
    for x in (0.3, 5.0, 40.0, 700.0):
        lad = orc.jl(60, x)
        for l in (2, 7, 33, 60):
            assert abs(orc.jnu(float(l), x) - lad[l]) <= 1e-13 * max(abs(lad[l]), 1e-300) + 1e-300


@pytest.mark.parametrize("kmap", [0, 1])
def test_e2_basis_at_real_ells_against_direct_quadrature(kmap):
    kmin, kmax, N = 1e-3, 2.0, 5
    ells = [2.5, 11.3, 40.77]
    pts = [(300.0, 240.0), (350.0, 350.0)]
    Nk = synth.kquad_points(kmin, kmax, 350.0, 1.0)
    u, w = np.polynomial.legendre.leggauss(24)
    edges = np.geomspace(kmin, kmax, 2001) if kmap else np.linspace(kmin, kmax, 2001)
    lo, hi = edges[:-1, None], edges[1:, None]
    kk = (0.5 * (hi - lo) * (u[None, :] + 1.0) + lo).ravel()
    wk = (0.5 * (hi - lo) * w[None, :]).ravel()
    if kmap:
        x = 2.0 * (np.log(kk) - np.log(kmin)) / (np.log(kmax) - np.log(kmin)) - 1.0
    else:
        x = 2.0 * (kk - kmin) / (kmax - kmin) - 1.0
    Tn = np.polynomial.chebyshev.chebvander(x, N - 1)
    f = [kk ** 2, np.ones_like(kk), kk ** -2.0]
    c1 = np.array([p[0] for p in pts])
    c2 = np.array([p[1] for p in pts])
    T = orc.basis(np.array(ells), c1, c2, N, kmin, kmax, Nk, kmap=kmap)
    for q, (a, b) in enumerate(pts):
        for e, l in enumerate(ells):
            jj = np.sqrt(np.pi / (2 * kk * a)) * sp.jv(l + 0.5, kk * a) * np.sqrt(np.pi / (2 * kk * b)) * \
                sp.jv(l + 0.5, kk * b)
            for t in range(3):
                ref = (wk * f[t] * jj) @ Tn
                assert np.max(np.abs(T[t, e, :, q] - ref)) <= 5e-12 * np.max(np.abs(ref)), (kmap, l, q, t)


def test_e3_prefactors_at_real_ell():
    for l in (2.5, 211.63, 999.9):
        r = math.exp(math.lgamma(l + 3.0) - math.lgamma(l - 1.0))
        assert abs(orc.prefactor(0, l) - 2 / math.pi) < 1e-15
        assert abs(orc.prefactor(1, l) / (2 / math.pi * math.sqrt(r)) - 1) < 1e-12
        assert abs(orc.prefactor(2, l) / (2 / math.pi * r) - 1) < 1e-12
