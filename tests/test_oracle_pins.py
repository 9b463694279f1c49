"""Pins of the FP64 oracle against what mathematics and the paper fix.

Each test checks one oracle step against something other than the oracle
itself: a library routine (scipy, numpy), a closed form, an exactness property
of a quadrature rule, or an invariant of the definitions.  A dropped term, a
wrong sign or a transposed index in ``oracle/oracle.c`` fails one of these.
"""
import math

import numpy as np
import pytest
import scipy.special as sp
from scipy.interpolate import CubicSpline

import oracle as orc
from paper_2410_03632_gb300 import synth
from tests.metrics import eij


# ---------------------------------------------------------------- Bessel j_l
@pytest.mark.parametrize("lmax", [2, 40, 300, 2000])
def test_jl_matches_scipy(lmax):
    """Oracle j_l against scipy.special.spherical_jn over x < l, x ~ l, x > l."""
    xs = np.concatenate([[5e-4, 1e-2, 0.7, 3.0], np.geomspace(0.05, 3 * lmax + 10, 60),
                         [lmax - 0.5, lmax + 0.5, 7.3e4]])
    ls = np.unique(np.linspace(0, lmax, 12).astype(int))
    for x in xs:
        j = orc.jl(lmax, x)
        ref = sp.spherical_jn(ls, x)
        for l, r in zip(ls, ref):
            if abs(r) < 1e-280:
                assert abs(j[l]) < 1e-270
                continue
            # relative away from zeros; near a zero of an oscillating j_l the
            # absolute error is measured against the envelope 1/x
            env = 1.0 / max(x, 1.0) if x > 0.5 * l else 0.0
            assert abs(j[l] - r) <= 2e-12 * abs(r) + 1e-14 * env, (l, x, j[l], r)


def test_jl_high_precision_points():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for l, x in [(2, 1e-3), (10, 9.7), (200, 180.0), (200, 211.63), (1000, 1000.5), (3, 7.3e4)]:
        ref = mp.sqrt(mp.pi / (2 * x)) * mp.besselj(l + mp.mpf(1) / 2, x)
        got = orc.jl(l, x)[l]
        assert abs(got - float(ref)) <= 5e-14 * abs(float(ref)), (l, x)


def test_jl_zero_argument():
    j = orc.jl(5, 0.0)
    assert j[0] == 1.0 and np.all(j[1:] == 0.0)


# ---------------------------------------------------------------- grids
@pytest.mark.parametrize("X", [5, 6, 41, 64, 128])
def test_chi_grid_simpson_exact_for_cubics(X):
    lo, hi = 26.0, 4100.0
    chi, w = orc.chi_grid(X, lo, hi)
    assert np.allclose(np.diff(chi), (hi - lo) / (X - 1), rtol=1e-12)
    s = (chi - lo) / (hi - lo)
    for p in range(4):
        exact = (hi - lo) / (p + 1)
        assert abs(np.dot(w, s ** p) - exact) <= 1e-12 * exact, p


@pytest.mark.parametrize("Rn", [2, 10, 64, 192])
def test_R_grid_fejer_exact_per_panel(Rn):
    lo, hi = 0.2, 1.8
    R, w = orc.R_grid(Rn, lo, hi)
    n = Rn // 2
    assert np.all(np.diff(R) > 0)
    # nodes of each panel are the roots of T_n mapped to the panel (Eq. chebpoints)
    x1 = (2 * R[:n] - (lo + 1)) / (1 - lo)
    x2 = (2 * R[n:] - (1 + hi)) / (hi - 1)
    for x in (x1, x2):
        assert np.max(np.abs(np.cos(n * np.arccos(np.clip(x, -1, 1))))) < 1e-12
    # every polynomial of degree < n is integrated exactly on each panel
    for p in range(n):
        for (a, b, sl) in ((lo, 1.0, slice(0, n)), (1.0, hi, slice(n, Rn))):
            u = (R[sl] - a) / (b - a)
            exact = (b - a) / (p + 1)
            assert abs(np.dot(w[sl], u ** p) - exact) <= 1e-12 * (b - a), (Rn, p)


@pytest.mark.parametrize("Nk", [3, 5, 129, 4097])
def test_cc_grid_polynomial_exactness(Nk):
    kmin, kmax = 1e-4, 10.0
    k, x, w = orc.cc_grid(Nk, kmin, kmax)
    assert abs(w.sum() - (kmax - kmin)) < 1e-13 * (kmax - kmin)
    assert np.allclose(k, 0.5 * (kmin + kmax) + 0.5 * (kmax - kmin) * x, rtol=1e-15, atol=0)
    n = Nk - 1
    for p in range(0, n + 1):
        exact = (1 - (-1) ** (p + 1)) / (p + 1)  # int_{-1}^{1} x^p
        got = np.dot(w, x ** p) / (0.5 * (kmax - kmin))
        assert abs(got - exact) < 2e-13, (Nk, p)


def test_cc_grid_oscillatory_integral():
    """int cos(w k) dk over [kmin, kmax] for w below the rule's resolution."""
    kmin, kmax = 1e-4, 10.0
    k, x, wt = orc.cc_grid(16385, kmin, kmax)
    for om in (1.0, 300.0, 2000.0):
        exact = (math.sin(om * kmax) - math.sin(om * kmin)) / om
        assert abs(np.dot(wt, np.cos(om * k)) - exact) < 1e-12


# ---------------------------------------------------------------- Chebyshev fit
@pytest.mark.parametrize("N", [1, 2, 7, 32, 96])
def test_cheb_dct_matches_numpy_interpolant(N):
    """c_n of the interpolant at first-kind points: numpy's chebinterpolate."""
    f = lambda t: np.exp(0.7 * t) * np.cos(3 * t) + 1.0 / (2.5 - t)
    t = np.cos(np.pi * (2 * np.arange(N) + 1) / (2 * N))
    a = orc.cheb_dct(f(t))
    ref = np.polynomial.chebyshev.chebinterpolate(f, N - 1)
    assert np.allclose(a, ref, rtol=0, atol=1e-13)


def test_cheb_dct_aliasing_signs():
    """On N first-kind points T_{2N-m} equals -T_m and T_N vanishes (the
    aliasing relation of Eq. cheb2 for first-kind points)."""
    N = 16
    t = np.cos(np.pi * (2 * np.arange(N) + 1) / (2 * N))
    for m in range(1, N):
        a = orc.cheb_dct(np.cos((2 * N - m) * np.arccos(t)))
        e = np.zeros(N); e[m] = -1.0
        assert np.allclose(a, e, atol=1e-13), m
    a = orc.cheb_dct(np.cos(N * np.arccos(t)))
    assert np.allclose(a, 0.0, atol=1e-13)
    a = orc.cheb_dct(np.cos((N + 3) * np.arccos(t)))  # T_{N+3} ~ -T_{N-3}
    e = np.zeros(N); e[N - 3] = -1.0
    assert np.allclose(a, e, atol=1e-13)


def test_spline_natural_matches_scipy():
    rng = np.random.default_rng(3)
    u = np.sort(rng.uniform(-9, 2.3, 40))
    v = np.sin(u) + 0.1 * u ** 2
    uq = rng.uniform(u[0], u[-1], 500)
    got = orc.spline_natural(u, v, uq)
    ref = CubicSpline(u, v, bc_type="natural")(uq)
    assert np.allclose(got, ref, rtol=0, atol=1e-12)
    with pytest.raises(ValueError):
        orc.spline_natural(u, v, [u[-1] + 1.0])


@pytest.mark.parametrize("kmap", [0, 1])
def test_fit_power_law_is_interpolated_exactly(kmap):
    """ln P linear in ln k is reproduced by the natural spline, so the fit is
    exactly the Chebyshev interpolant of the power law (library: numpy)."""
    kmin, kmax, N = 1e-4, 10.0, 48
    k = np.geomspace(1e-4, 10.0, 256)
    P = 3e4 * k ** -1.7
    a = orc.fit(N, kmin, kmax, k, P, kmap)
    if kmap == 0:
        kf = lambda t: 0.5 * (kmin + kmax) + 0.5 * (kmax - kmin) * t
    else:
        kf = lambda t: np.exp(np.log(kmin) + 0.5 * np.log(kmax / kmin) * (t + 1))
    ref = np.polynomial.chebyshev.chebinterpolate(lambda t: 3e4 * kf(t) ** -1.7, N - 1)
    assert np.allclose(a, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_fit_linear_in_P_and_constant():
    k, P = synth.pk_table()
    a1 = orc.fit(40, 1e-4, 10.0, k, P, 1)
    a2 = orc.fit(40, 1e-4, 10.0, k, 3.5 * P, 1)
    assert np.allclose(a2, 3.5 * a1, rtol=0, atol=1e-13 * np.abs(a2).max())
    c = orc.fit(40, 1e-4, 10.0, k, np.full_like(k, 7.0), 1)
    assert abs(c[0] - 7.0) < 1e-13 and np.all(np.abs(c[1:]) < 1e-13)


def test_fit_rejects_table_that_misses_nodes():
    k = np.geomspace(1e-3, 10.0, 64)
    with pytest.raises(ValueError):
        orc.fit(16, 1e-4, 10.0, k, k ** -1.0, 1)


# ---------------------------------------------------------------- basis T~ vs the closed form
def _closed(s, l, c1, c2):
    """int_0^inf k^s j_l(k c1) j_l(k c2) dk, DLMF 10.22.56 with mu = nu = l + 1/2."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    a, b = max(c1, c2), min(c1, c2)
    nu = l + mp.mpf(1) / 2
    pre = (mp.pi / 2 / mp.sqrt(a * b) * b ** nu * mp.gamma((2 * l + 1 + s) / mp.mpf(2))
           / (2 ** (1 - s) * a ** (nu + s) * mp.gamma(1 - mp.mpf(s) / 2) * mp.gamma(l + mp.mpf(3) / 2)))
    return float(pre * mp.hyp2f1((2 * l + 1 + s) / mp.mpf(2), mp.mpf(s) / 2, l + mp.mpf(3) / 2,
                                 (b / a) ** 2))


def _low_tail(s, l, c1, c2, kmin):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    jl = lambda z: mp.sqrt(mp.pi / (2 * z)) * mp.besselj(l + mp.mpf(1) / 2, z)
    return float(mp.quad(lambda k: k ** s * jl(k * c1) * jl(k * c2), [0, kmin]))


@pytest.mark.parametrize("l,c1,c2", [(2, 300.0, 240.0), (5, 300.0, 240.0), (11, 410.0, 350.0)])
def test_basis_matches_closed_form(l, c1, c2):
    """T~ for n = 0, 1, 2 with the linear k map is a combination of
    int k^s j_l j_l dk with s = -2, -1, 0 (types ss and gs); the integral
    outside [kmin, kmax] is bounded analytically and enters the tolerance."""
    kmin, kmax, N = 1e-4, 50.0, 3
    Nk = synth.kquad_points(kmin, kmax, max(c1, c2), 1.0) * 2 - 1
    T = orc.basis([l], [c1], [c2], N, kmin, kmax, Nk, kmap=0)
    al, be = 2.0 / (kmax - kmin), -(kmax + kmin) / (kmax - kmin)  # x = al k + be
    # the closed form is over (0, inf): remove the part below kmin, where
    # k chi << 1 and the integrand is smooth (plain quadrature)
    I = {s: _closed(s, l, c1, c2) - _low_tail(s, l, c1, c2, kmin) for s in (-2, -1, 0)}
    # T_0 = 1, T_1 = al k + be, T_2 = 2 (al k + be)^2 - 1, times 1/k^2 (ss)
    ss = [I[-2], al * I[-1] + be * I[-2], 2 * al * al * I[0] + 4 * al * be * I[-1] + (2 * be * be - 1) * I[-2]]
    # tail above kmax: |j_l(z)| <= 1/z, so |int_K^inf k^s j j| <= K^(s-1) / ((1-s) c1 c2);
    # the oscillating integrand makes the true tail far smaller: bound by 1/(K Delta)
    dlt = abs(c1 - c2)
    tail = {s: kmax ** (s - 2) / (c1 * c2 * dlt) * 4 for s in (-2, -1, 0)}
    tol_ss = [tail[-2], al * tail[-1] + abs(be) * tail[-2],
              2 * al * al * tail[0] + 4 * al * abs(be) * tail[-1] + (2 * be * be + 1) * tail[-2]]
    for n in range(3):
        assert abs(T[2, 0, n, 0] - ss[n]) <= tol_ss[n] + 1e-10 * abs(ss[n]), (n, T[2, 0, n, 0], ss[n])
    # gs, n = 0: int j j dk = pi b^l / (2 (2l+1) a^(l+1))
    assert abs(T[1, 0, 0, 0] - I[0]) <= tail[0] + 1e-10 * abs(I[0])
    full0 = _closed(0, l, c1, c2)
    assert abs(full0 - math.pi * min(c1, c2) ** l / (2 * (2 * l + 1) * max(c1, c2) ** (l + 1))) < 1e-14 * full0


def test_basis_diagonal_matches_closed_form():
    """chi1 = chi2: ss type, n = 0, where the tail above kmax is ~ 1/(6 K^3 chi^2)."""
    l, c = 4, 320.0
    kmin, kmax = 1e-4, 20.0
    Nk = synth.kquad_points(kmin, kmax, c, 1.0)
    T = orc.basis([l], [c], [c], 1, kmin, kmax, Nk, kmap=0)
    ref = _closed(-2, l, c, c) - _low_tail(-2, l, c, c, kmin)
    assert abs(T[2, 0, 0, 0] - ref) <= 1.0 / (6 * kmax ** 3 * c * c) + 1e-10 * ref


@pytest.mark.parametrize("kmap", [0, 1])
def test_basis_all_types_and_both_maps_against_direct_quadrature(kmap):
    """T~ of every type (gg f = k^2, gs f = 1, ss f = 1/k^2) and both k maps,
    orders n < 6, against composite Gauss-Legendre in k with scipy's spherical
    Bessel functions and numpy's Chebyshev polynomials: no Clenshaw-Curtis
    rule, no recurrence, no map code of the oracle.  The panels are short
    against the Bessel period; measured agreement is 1e-12 of the row or
    better (the gg rows, weighted to high k, are the loosest)."""
    kmin, kmax, N = 1e-3, 5.0, 6
    pts = [(2, 300.0, 240.0), (9, 300.0, 300.0), (30, 410.0, 350.0)]
    Nk = synth.kquad_points(kmin, kmax, 410.0, 1.0)
    u, w = np.polynomial.legendre.leggauss(24)
    edges = np.geomspace(kmin, kmax, 4001) if kmap else np.linspace(kmin, kmax, 4001)
    lo, hi = edges[:-1, None], edges[1:, None]
    kk = (0.5 * (hi - lo) * (u[None, :] + 1.0) + lo).ravel()
    wk = (0.5 * (hi - lo) * w[None, :]).ravel()
    if kmap:
        x = 2.0 * (np.log(kk) - np.log(kmin)) / (np.log(kmax) - np.log(kmin)) - 1.0
    else:
        x = 2.0 * (kk - kmin) / (kmax - kmin) - 1.0
    Tn = np.polynomial.chebyshev.chebvander(x, N - 1)  # [k][n]
    f = [kk ** 2, np.ones_like(kk), kk ** -2.0]
    for l, c1, c2 in pts:
        T = orc.basis([l], [c1], [c2], N, kmin, kmax, Nk, kmap=kmap)
        jj = sp.spherical_jn(l, kk * c1) * sp.spherical_jn(l, kk * c2)
        for t in range(3):
            ref = (wk * f[t] * jj) @ Tn
            scale = np.max(np.abs(ref))
            assert np.max(np.abs(T[t, 0, :, 0] - ref)) <= 5e-12 * scale, (kmap, l, t, T[t, 0, :, 0], ref)


def test_basis_quadrature_converged_under_doubling():
    """The Clenshaw-Curtis size rule gives a converged T~ (App. C analog)."""
    spec = synth.plan_spec("tiny")
    g = orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min,
                 spec.R_max, spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map)
    T1 = g.basis()
    g.Nk = 2 * spec.n_kquad - 1
    T2 = g.basis()
    scale = np.abs(T2).max(axis=-1, keepdims=True)
    assert np.max(np.abs(T1 - T2) / scale) < 1e-9


def test_basis_symmetric_in_arguments():
    chi1 = np.array([100.0, 250.0, 512.0])
    chi2 = np.array([180.0, 75.0, 512.0])
    T12 = orc.basis([2, 9], chi1, chi2, 5, 1e-3, 1.0, 2049, kmap=1)
    T21 = orc.basis([2, 9], chi2, chi1, 5, 1e-3, 1.0, 2049, kmap=1)
    assert np.array_equal(T12, T21)


# ---------------------------------------------------------------- prefactors and C_l invariants
def test_prefactors():
    for l in (2, 3, 17, 2000):
        r = math.factorial(l + 2) / math.factorial(l - 2)
        assert orc.prefactor(0, l) == pytest.approx(2 / math.pi, rel=1e-15)
        assert orc.prefactor(1, l) == pytest.approx(2 / math.pi * math.sqrt(r), rel=1e-14)
        assert orc.prefactor(2, l) == pytest.approx(2 / math.pi * r, rel=1e-14)
    assert orc.npairs(5, 5) == 55 and orc.npairs(10, 10) == 210 and orc.npairs(1, 1) == 3


@pytest.fixture(scope="module")
def tiny():
    spec = synth.plan_spec("tiny")
    g = orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min,
                 spec.R_max, spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map)
    return spec, g, g.basis()


def test_cl_single_node_kernel_indexing(tiny):
    """A kernel nonzero at one node picks one entry of w: checks q = a*Rn + r,
    the pair order gg, gs, ss, the prefactor and the weights (Eq. final_cls)."""
    spec, g, T = tiny
    ng, ns = 2, 2
    X, Rn = g.X, g.Rn
    Q = X * Rn
    rng = np.random.default_rng(0)
    Dc, DR = rng.uniform(0.5, 1, X), rng.uniform(0.5, 1, Q)
    a_n = np.zeros(g.N); a_n[0] = 2.5
    for (t, i, j, a, r) in [(0, 0, 1, 3, 7), (1, 1, 0, 9, 2), (2, 1, 1, 12, 9), (2, 0, 1, 0, 0)]:
        kc = np.zeros((ng + ns, X)); kR = np.zeros((ng + ns, Q))
        A = i if t < 2 else ng + i
        B = j if t == 0 else ng + j
        kc[A, a] = 1.3
        kR[B, a * Rn + r] = 0.7
        C = g.cl(T, a_n, ng, ns, kc, kR, Dc, DR)
        if t == 0:
            p = [(0, 0), (0, 1), (1, 1)].index((i, j))
        elif t == 1:
            p = 3 + i * ns + j
        else:
            p = 7 + [(0, 0), (0, 1), (1, 1)].index((i, j))
        for e, l in enumerate(g.ells):
            want = (orc.prefactor(t, l) * g.wchi[a] * g.wR[r] * g.chi[a] * 1.3 * 0.7
                    * Dc[a] * DR[a * Rn + r] * 2.5 * T[t, e, 0, a * Rn + r])
            assert C[p, e] == pytest.approx(want, rel=1e-13, abs=1e-300)
        others = np.delete(C, p, axis=0)
        assert np.all(others == 0.0)


def test_cl_linear_in_P_and_bins_permute(tiny):
    spec, g, T = tiny
    rq = synth.config_request("tiny", g.chi, g.R)
    a1 = g.fit(rq.k_tab, rq.p_tab)
    a2 = g.fit(rq.k_tab, 2.0 * rq.p_tab)
    args = (rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi)
    C1 = g.cl(T, a1, *args)
    C2 = g.cl(T, a2, *args)
    assert np.max(eij(C2, 2 * C1, rq.n_clust, rq.n_lens)) < 1e-11
    # swapping the two clustering bins swaps gg(0,0) <-> gg(1,1) and the gs rows
    perm = [1, 0, 2, 3]
    C3 = g.cl(T, a1, rq.n_clust, rq.n_lens, rq.kern_chi[perm], rq.kern_Rchi[perm],
              rq.growth_chi, rq.growth_Rchi)
    assert np.array_equal(C3[0], C1[2]) and np.array_equal(C3[2], C1[0])
    # gg(0,1) becomes gg(1,0), which the unsymmetrised chi-R form does not
    # equate: each ordering drops the part of the chi1-chi2 plane with
    # chi2/chi1 outside [R_min, R_max], a different part for each ordering
    assert np.array_equal(C3[3:5], C1[5:7]) and np.array_equal(C3[5:7], C1[3:5])
    assert np.array_equal(C3[7:], C1[7:])
    # auto spectra are positive
    assert np.all(C1[[0, 2, 7, 9]] > 0)
