/*
 * Plain FP64 CPU oracle for the Blast beyond-Limber angular power spectrum
 * (Chiarenza, Bonici, Percival, White, arXiv:2410.03632).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file's shared library; the product library never
 * does, and this file shares no code, header, table or constant generator with
 * the CUDA path.  Everything is IEEE double, round to nearest, written as the
 * plain definition of each step with no blocking or fusion beyond loop order.
 *
 * Steps, in the paper's order and notation:
 *   grids        Sec. 3.2: Simpson in chi, first-kind Chebyshev points with
 *                Clenshaw-Curtis-type (Fejer 1) weights in R, Clenshaw-Curtis in k
 *                (App. C); Chebyshev points for the fit (Eq. chebpoints).
 *   j_l(x)       spherical Bessel functions of Eq. cls-general.
 *   T~           basis integrals, Eq. t_tilde, f^gg = k^2, f^ss = 1/k^2, f^gs = 1.
 *   c_n          interpolation coefficients at Chebyshev points (Eq. a2), obtained
 *                from the samples by the discrete cosine transform that Eq. dft
 *                stands for.
 *   w_l          projected matter density, Eq. pmd, with c_n(chi1,chi2) =
 *                D(chi1) D(chi2) a_n (growth-separable P, Sec. 4.2.1).
 *   C_l          chi-R quadrature of Eq. final_cls in its unsymmetrised form
 *                (first line of Eq. app1 with chi2 = R chi1), times the probe
 *                prefactor N(l) of Eqs. gg, ss, gs.
 *
 * Status: every function returns 0 on success and a negative value on bad input.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

static int orc_threads(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Grids (Sec. 3.2)                                                          */
/* ------------------------------------------------------------------------- */

/* X evenly spaced chi nodes on [lo, hi] with composite Simpson weights.  For an
 * odd number of intervals the last three intervals take Simpson's 3/8 rule. */
int orc_chi_grid(int X, double lo, double hi, double *chi, double *w)
{
    if (X < 3 || (X % 2 == 0 && X < 4) || !(hi > lo)) return -1;
    double h = (hi - lo) / (double)(X - 1);
    for (int a = 0; a < X; a++) { chi[a] = lo + h * (double)a; w[a] = 0.0; }
    int n13 = (X % 2 == 1) ? X - 1 : X - 4; /* intervals under the 1/3 rule */
    for (int i = 0; i < n13; i += 2) {
        w[i] += h / 3.0; w[i + 1] += 4.0 * h / 3.0; w[i + 2] += h / 3.0;
    }
    if (X % 2 == 0) {
        int s = X - 4;
        w[s] += 3.0 * h / 8.0; w[s + 1] += 9.0 * h / 8.0;
        w[s + 2] += 9.0 * h / 8.0; w[s + 3] += 3.0 * h / 8.0;
    }
    return 0;
}

/* Fejer first rule on [-1,1]: the n first-kind Chebyshev points
 * x_k = cos((2k+1) pi / 2n) of Eq. chebpoints and the weights that integrate
 * every polynomial of degree < n exactly.  Output ordered by increasing x. */
static void orc_fejer1(int n, double *x, double *w)
{
    for (int i = 0; i < n; i++) {
        int k = n - 1 - i; /* increasing x */
        double th = ORC_PI * (2.0 * k + 1.0) / (2.0 * n);
        double s = 0.0;
        for (int j = 1; j <= n / 2; j++)
            s += cos(2.0 * j * th) / (4.0 * (double)j * j - 1.0);
        x[i] = cos(th);
        w[i] = (2.0 / n) * (1.0 - 2.0 * s);
    }
}

/* R nodes: two panels [lo, 1] and [1, hi], each holding Rn/2 first-kind
 * Chebyshev points with Fejer-1 weights, so that nodes crowd towards R = 1 from
 * both sides (the diagonal chi1 = chi2 that dominates the integral, App. A). */
int orc_R_grid(int Rn, double lo, double hi, double *R, double *w)
{
    if (Rn < 2 || Rn % 2 != 0 || !(lo > 0.0) || !(lo < 1.0) || !(hi > 1.0)) return -1;
    int n = Rn / 2;
    double *x = (double *)malloc(sizeof(double) * n), *wx = (double *)malloc(sizeof(double) * n);
    if (!x || !wx) { free(x); free(wx); return -2; }
    orc_fejer1(n, x, wx);
    double c1 = 0.5 * (lo + 1.0), h1 = 0.5 * (1.0 - lo);
    double c2 = 0.5 * (1.0 + hi), h2 = 0.5 * (hi - 1.0);
    for (int i = 0; i < n; i++) {
        R[i] = c1 + h1 * x[i];         w[i] = h1 * wx[i];
        R[n + i] = c2 + h2 * x[i];     w[n + i] = h2 * wx[i];
    }
    free(x); free(wx);
    return 0;
}

/* R nodes of the symmetrised form (App. A, Eq. app1 and the integral after it:
 * R in (0, 1]): the strictly positive points of the M = 2 Rn + 1 first-kind
 * Chebyshev points on [-1, 1] (the middle one is 0), Rn of them, with the
 * Fejer-1 weights of the M-point rule.  For f on [0, 1] extended evenly,
 * int_0^1 f = (1/2) int_{-1}^{1} f(|x|) dx = sum_{x_k > 0} w_k f(x_k)
 * + (1/2) w_mid f(0); f(0) = 0 here (j_l(0) = 0 for l >= 1), so the middle
 * point is dropped.  Output ordered by increasing R. */
int orc_R_grid_sym(int Rn, double *R, double *w)
{
    if (Rn < 1) return -1;
    int M = 2 * Rn + 1;
    double *x = (double *)malloc(sizeof(double) * M), *wx = (double *)malloc(sizeof(double) * M);
    if (!x || !wx) { free(x); free(wx); return -2; }
    orc_fejer1(M, x, wx);
    /* increasing x: indices Rn + 1 .. 2 Rn are the positive points */
    for (int i = 0; i < Rn; i++) { R[i] = x[Rn + 1 + i]; w[i] = wx[Rn + 1 + i]; }
    free(x); free(wx);
    return 0;
}

/* Clenshaw-Curtis rule with Nk = n+1 points (n even) on [kmin, kmax] (Sec. 3.2,
 * App. C): x_m = cos(m pi / n), k_m = (kmin+kmax)/2 + (kmax-kmin)/2 x_m, and
 * w_m = (c_m/n) [1 - sum_{j=1}^{n/2} b_j cos(2 j m pi / n) / (4 j^2 - 1)] times
 * (kmax-kmin)/2, with c_0 = c_n = 1, c_m = 2 otherwise, b_{n/2} = 1, b_j = 2
 * otherwise.  Every cosine argument is reduced exactly in integers, 2 pi (j m
 * mod n) / n, and read from a table of cos(2 pi p / n). */
int orc_cc_grid(int Nk, double kmin, double kmax, double *k, double *x, double *w, int nthreads)
{
    if (Nk < 3 || (Nk - 1) % 2 != 0 || !(kmax > kmin)) return -1;
    int n = Nk - 1;
    double *tab = (double *)malloc(sizeof(double) * n);
    if (!tab) return -2;
    for (int p = 0; p < n; p++) tab[p] = cos(2.0 * ORC_PI * (double)p / (double)n);
    double kc = 0.5 * (kmin + kmax), kh = 0.5 * (kmax - kmin);
    int nt = orc_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int m = 0; m <= n; m++) {
        double s = 0.0;
        for (int j = 1; j <= n / 2; j++) {
            double b = (j == n / 2) ? 1.0 : 2.0;
            int64_t p = ((int64_t)j * (int64_t)m) % (int64_t)n;
            s += b * tab[p] / (4.0 * (double)j * (double)j - 1.0);
        }
        double c = (m == 0 || m == n) ? 1.0 : 2.0;
        /* x_m = cos(m pi / n) = cos(2 pi m / (2n)) */
        double xm = cos(ORC_PI * (double)m / (double)n);
        x[m] = xm;
        k[m] = kc + kh * xm;
        w[m] = kh * (c / (double)n) * (1.0 - s);
    }
    free(tab);
    return 0;
}

/* Map between k in [kmin, kmax] and the Chebyshev variable in [-1, 1]:
 * kmap 0 is linear in k, kmap 1 is linear in ln k. */
static double orc_k_to_x(int kmap, double k, double kmin, double kmax)
{
    double x = (kmap == 0) ? (2.0 * k - kmin - kmax) / (kmax - kmin)
                           : 2.0 * (log(k) - log(kmin)) / (log(kmax) - log(kmin)) - 1.0;
    return x > 1.0 ? 1.0 : (x < -1.0 ? -1.0 : x);
}

static double orc_x_to_k(int kmap, double x, double kmin, double kmax)
{
    if (kmap == 0) return 0.5 * (kmin + kmax) + 0.5 * (kmax - kmin) * x;
    return exp(log(kmin) + 0.5 * (log(kmax) - log(kmin)) * (x + 1.0));
}

/* Eq. chebpoints: t_j = cos((2j+1) pi / 2N), j < N, and the k they map to. */
int orc_cheb_knodes(int N, double kmin, double kmax, int kmap, double *t, double *k)
{
    if (N < 1 || !(kmax > kmin) || kmap < 0 || kmap > 1 || (kmap == 1 && !(kmin > 0.0))) return -1;
    for (int j = 0; j < N; j++) {
        t[j] = cos(ORC_PI * (2.0 * j + 1.0) / (2.0 * N));
        k[j] = orc_x_to_k(kmap, t[j], kmin, kmax);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Spherical Bessel functions j_0 .. j_lmax at one argument x >= 0.           */
/* For x > lmax the forward recurrence j_{l+1} = (2l+1)/x j_l - j_{l-1} from   */
/* j_0 = sin x / x, j_1 = sin x / x^2 - cos x / x is stable.  Otherwise        */
/* Miller's backward recurrence runs from l0 = lmax + 20 + sqrt(40 lmax) with  */
/* arbitrary start values and is normalised by the addition-theorem sum rule   */
/* sum_l (2l+1) j_l(x)^2 = 1, with the sign taken from j_0 (or j_1).          */
/* ------------------------------------------------------------------------- */
int orc_jl(int lmax, double x, double *j)
{
    if (lmax < 0 || !(x >= 0.0) || isinf(x)) return -1;
    if (x == 0.0) {
        j[0] = 1.0;
        for (int l = 1; l <= lmax; l++) j[l] = 0.0;
        return 0;
    }
    double s = sin(x), c = cos(x);
    double j0 = s / x;
    if (lmax == 0) { j[0] = j0; return 0; }
    if (x > (double)lmax) {
        j[0] = j0;
        j[1] = s / (x * x) - c / x;
        for (int l = 1; l < lmax; l++) j[l + 1] = (2.0 * l + 1.0) / x * j[l] - j[l - 1];
        return 0;
    }
    int l0 = lmax + 20 + (int)sqrt(40.0 * (double)lmax);
    double fp1 = 0.0, f = 1.0, sum = 0.0;
    for (int l = l0; l >= 1; l--) {
        if (l <= lmax) j[l] = f;
        sum += (2.0 * l + 1.0) * f * f;
        double fm1 = (2.0 * l + 1.0) / x * f - fp1;
        fp1 = f;
        f = fm1;
        if (fabs(f) > 1e120) {
            f *= 1e-120; fp1 *= 1e-120; sum *= 1e-240;
            for (int m = l; m <= lmax; m++) j[m] *= 1e-120;
        }
    }
    j[0] = f;
    sum += f * f;
    double norm = 1.0 / sqrt(sum);
    /* sign: from whichever of j_0, j_1 is larger in magnitude */
    double j1 = (x < 1e-3) ? x / 3.0 * (1.0 - x * x / 10.0) : (s / (x * x) - c / x);
    double sg;
    if (fabs(j0) >= fabs(j1)) sg = ((j0 >= 0.0) == (j[0] >= 0.0)) ? 1.0 : -1.0;
    else sg = ((j1 >= 0.0) == (j[1] >= 0.0)) ? 1.0 : -1.0;
    for (int l = 0; l <= lmax; l++) j[l] *= sg * norm;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* j_nu(x) for real nu >= 0 (non-integer multipoles, App. A's l = 211.63):    */
/*   j_nu(x) = sqrt(pi / (2x)) J_{nu+1/2}(x).                                */
/* J by Miller's backward recurrence J_{m-1} = (2m/x) J_m - J_{m+1} on the   */
/* orders m = mu0 + k (mu0 = frac(nu + 1/2)), from k = K well above x and    */
/* nu + 1/2, normalised by Neumann's expansion                                */
/*   (x/2)^mu0 = sum_{i>=0} (mu0 + 2i) Gamma(mu0 + i) / i! J_{mu0+2i}(x)      */
/* (the i = 0 term is Gamma(mu0 + 1) J_mu0).                                 */
/* ------------------------------------------------------------------------- */
int orc_jnu(double nu, double x, double *out)
{
    if (!(nu >= 0.0) || !(x >= 0.0) || isinf(x) || isinf(nu)) return -1;
    if (x == 0.0) { *out = (nu == 0.0) ? 1.0 : 0.0; return 0; }
    const double mu = nu + 0.5;
    const int nmu = (int)floor(mu);
    const double mu0 = mu - (double)nmu;
    const double top = (double)nmu > x ? (double)nmu : x;
    const int K = (int)top + 40 + (int)(10.0 * cbrt(top));
    /* Neumann weights c_i = (mu0 + 2i) Gamma(mu0 + i) / i!, upward from
     * Gamma(mu0 + 1) with the exact ratios (mu0 + i) / (i + 1) (one rounding
     * per step), in a per-thread buffer */
    static _Thread_local double *cbuf = NULL;
    static _Thread_local int ccap = 0;
    const int I = K / 2;
    if (I + 1 > ccap) {
        double *nb = (double *)realloc(cbuf, sizeof(double) * (size_t)(I + 1));
        if (!nb) return -2;
        cbuf = nb;
        ccap = I + 1;
    }
    double *c = cbuf;
    double g = tgamma(mu0 + 1.0); /* Gamma(mu0 + i) / i! at i = 1 */
    c[0] = g;                     /* mu0 Gamma(mu0) = Gamma(mu0 + 1) */
    for (int i = 1; i <= I; i++) {
        c[i] = (mu0 + 2.0 * i) * g;
        g *= (mu0 + i) / (i + 1.0);
    }
    double fp = 0.0, f = 1e-280, rec = 0.0, S = 0.0;
    for (int k = K; k >= 0; k--) {
        /* f = J_{mu0+k} (unnormalised), fp = J_{mu0+k+1} */
        if (k == nmu) rec = f;
        if (k % 2 == 0) S += c[k / 2] * f;
        if (k == 0) break;
        double fm = 2.0 * (mu0 + k) / x * f - fp;
        fp = f;
        f = fm;
        if (fabs(f) > 1e250) { f *= 1e-250; fp *= 1e-250; S *= 1e-250; rec *= 1e-250; }
    }
    double J = rec * pow(0.5 * x, mu0) / S;
    *out = sqrt(ORC_PI / (2.0 * x)) * J;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Basis integrals, Eq. t_tilde:                                             */
/*   T~^{AB}_{n;l}(chi1, chi2) = int_{kmin}^{kmax} dk f^{AB}(k) T_n(x(k))      */
/*                                 j_l(k chi1) j_l(k chi2)                    */
/* with x(k) the map of [kmin, kmax] onto [-1, 1] (linear in k or in ln k),  */
/* evaluated with the                                                         */
/* Clenshaw-Curtis rule of Sec. 3.2 and Neumaier-compensated sums.            */
/* Types: 0 = gg (f = k^2), 1 = gs (f = 1), 2 = ss (f = 1/k^2).              */
/* Output T[t][e][n][q] for the ells ell[0..n_ell) and point pairs            */
/* (chi1[q], chi2[q]), q < nq.                                               */
/* ------------------------------------------------------------------------- */
int orc_basis(int n_ell, const double *ell, int nq, const double *chi1, const double *chi2,
              int N, double kmin, double kmax, int kmap, int Nk, int nthreads, double *T)
{
    if (n_ell < 1 || nq < 1 || N < 1 || !(kmin > 0.0) || kmap < 0 || kmap > 1) return -1;
    int lmax = 0, integer = 1;
    for (int e = 0; e < n_ell; e++) {
        if (!(ell[e] >= 0.0)) return -1;
        if (ell[e] != floor(ell[e])) integer = 0;
        if ((int)ceil(ell[e]) > lmax) lmax = (int)ceil(ell[e]);
    }
    double *k = (double *)malloc(sizeof(double) * Nk);
    double *x = (double *)malloc(sizeof(double) * Nk);
    double *w = (double *)malloc(sizeof(double) * Nk);
    double *A = (double *)malloc(sizeof(double) * (size_t)Nk * 3 * N);
    if (!k || !x || !w || !A) { free(k); free(x); free(w); free(A); return -2; }
    int rc = orc_cc_grid(Nk, kmin, kmax, k, x, w, nthreads);
    if (rc) { free(k); free(x); free(w); free(A); return rc; }
    /* A[m][t][n] = w_m f_t(k_m) T_n(x_m), T_n by the three-term recurrence */
    for (int m = 0; m < Nk; m++) {
        double f[3] = {k[m] * k[m], 1.0, 1.0 / (k[m] * k[m])};
        double xc = orc_k_to_x(kmap, k[m], kmin, kmax);
        double tm1 = 1.0, tn = xc;
        for (int n = 0; n < N; n++) {
            double Tn;
            if (n == 0) Tn = 1.0;
            else if (n == 1) Tn = xc;
            else { Tn = 2.0 * xc * tn - tm1; tm1 = tn; tn = Tn; }
            for (int t = 0; t < 3; t++) A[((size_t)m * 3 + t) * N + n] = w[m] * f[t] * Tn;
        }
    }
    const size_t per_q = (size_t)3 * n_ell * N;
    int nt = orc_threads(nthreads);
    int fail = 0;
#pragma omp parallel num_threads(nt)
    {
        double *acc = (double *)calloc(per_q, sizeof(double));
        double *cmp = (double *)calloc(per_q, sizeof(double));
        double *b1 = (double *)malloc(sizeof(double) * (lmax + 1));
        double *b2 = (double *)malloc(sizeof(double) * (lmax + 1));
        double *bm = (double *)malloc(sizeof(double) * n_ell);
        if (!acc || !cmp || !b1 || !b2 || !bm) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int q = 0; q < nq; q++) {
            if (fail) continue;
            memset(acc, 0, per_q * sizeof(double));
            memset(cmp, 0, per_q * sizeof(double));
            for (int m = 0; m < Nk; m++) {
                if (integer) {  /* one ladder of integer orders serves every ell */
                    orc_jl(lmax, k[m] * chi1[q], b1);
                    orc_jl(lmax, k[m] * chi2[q], b2);
                    for (int e = 0; e < n_ell; e++) bm[e] = b1[(int)ell[e]] * b2[(int)ell[e]];
                } else {
                    for (int e = 0; e < n_ell; e++) {
                        double u, v;
                        orc_jnu(ell[e], k[m] * chi1[q], &u);
                        orc_jnu(ell[e], k[m] * chi2[q], &v);
                        bm[e] = u * v;
                    }
                }
                for (int t = 0; t < 3; t++) {
                    const double *Am = A + ((size_t)m * 3 + t) * N;
                    for (int e = 0; e < n_ell; e++) {
                        double v = bm[e];
                        double *s = acc + ((size_t)t * n_ell + e) * N;
                        double *c = cmp + ((size_t)t * n_ell + e) * N;
                        for (int n = 0; n < N; n++) {
                            double term = Am[n] * v;
                            double tsum = s[n] + term;
                            c[n] += (fabs(s[n]) >= fabs(term)) ? ((s[n] - tsum) + term)
                                                              : ((term - tsum) + s[n]);
                            s[n] = tsum;
                        }
                    }
                }
            }
            for (size_t i = 0; i < per_q; i++) T[i * (size_t)nq + q] = acc[i] + cmp[i];
        }
        free(acc); free(cmp); free(b1); free(b2); free(bm);
    }
    free(k); free(x); free(w); free(A);
    return fail ? -2 : 0;
}

/* ------------------------------------------------------------------------- */
/* Chebyshev interpolation coefficients (Eqs. chebpoints, a2, dft)           */
/* ------------------------------------------------------------------------- */

/* Coefficients c_n of the degree-(N-1) interpolant through the samples
 * vals[j] = f(t_j) at the first-kind points t_j = cos((2j+1) pi / 2N):
 *   c_0 = (1/N) sum_j f(t_j),  c_n = (2/N) sum_j f(t_j) cos(n (2j+1) pi / 2N).
 * Cosine arguments are reduced exactly: n (2j+1) mod 4N. */
int orc_cheb_dct(int N, const double *vals, double *a)
{
    if (N < 1) return -1;
    double *tab = (double *)malloc(sizeof(double) * 4 * N);
    if (!tab) return -2;
    for (int p = 0; p < 4 * N; p++) tab[p] = cos(ORC_PI * (double)p / (2.0 * N));
    for (int n = 0; n < N; n++) {
        double s = 0.0;
        for (int j = 0; j < N; j++) s += vals[j] * tab[((long)n * (2 * j + 1)) % (4 * N)];
        a[n] = (n == 0 ? 1.0 : 2.0) * s / (double)N;
    }
    free(tab);
    return 0;
}

/* Natural cubic spline through (u_i, v_i), i < n, u strictly increasing,
 * evaluated at uq[0..m).  Second derivatives from the tridiagonal system by the
 * Thomas algorithm; a query outside [u_0, u_{n-1}] is an error. */
int orc_spline_natural(int n, const double *u, const double *v, int m, const double *uq, double *out)
{
    if (n < 3 || m < 0) return -1;
    for (int i = 1; i < n; i++) if (!(u[i] > u[i - 1])) return -1;
    double *M = (double *)calloc(n, sizeof(double));
    double *cp = (double *)calloc(n, sizeof(double));
    double *dp = (double *)calloc(n, sizeof(double));
    if (!M || !cp || !dp) { free(M); free(cp); free(dp); return -2; }
    /* unknowns M_1..M_{n-2}; row i: h_{i-1} M_{i-1} + 2(h_{i-1}+h_i) M_i + h_i M_{i+1} = r_i */
    for (int i = 1; i <= n - 2; i++) {
        double hl = u[i] - u[i - 1], hr = u[i + 1] - u[i];
        double r = 6.0 * ((v[i + 1] - v[i]) / hr - (v[i] - v[i - 1]) / hl);
        double b = 2.0 * (hl + hr);
        double lo = (i > 1) ? hl : 0.0;
        double den = b - lo * cp[i - 1];
        cp[i] = hr / den;
        dp[i] = (r - lo * dp[i - 1]) / den;
    }
    M[n - 1] = 0.0;
    for (int i = n - 2; i >= 1; i--) M[i] = dp[i] - cp[i] * M[i + 1];
    M[0] = 0.0;
    int rc = 0;
    for (int q = 0; q < m; q++) {
        double x = uq[q];
        if (!(x >= u[0] && x <= u[n - 1])) { rc = -3; break; }
        int lo = 0, hi = n - 1;
        while (hi - lo > 1) { int mid = (lo + hi) / 2; if (u[mid] <= x) lo = mid; else hi = mid; }
        double h = u[hi] - u[lo], t = (x - u[lo]) / h, s = 1.0 - t;
        out[q] = s * v[lo] + t * v[hi] + h * h / 6.0 * ((s * s * s - s) * M[lo] + (t * t * t - t) * M[hi]);
    }
    free(M); free(cp); free(dp);
    return rc;
}

/* Step a0: Chebyshev coefficients a_n, n < N, of P(k) on [kmin, kmax] (Eq.
 * cheb_pk): natural cubic spline of (ln k_i, ln P_i), P at the N Chebyshev
 * k-nodes, then the transform of orc_cheb_dct. */
int orc_fit(int N, double kmin, double kmax, int kmap, int ntab, const double *ktab, const double *ptab, double *a)
{
    if (N < 1 || ntab < 3) return -1;
    double *u = (double *)malloc(sizeof(double) * ntab), *v = (double *)malloc(sizeof(double) * ntab);
    double *t = (double *)malloc(sizeof(double) * N), *kn = (double *)malloc(sizeof(double) * N);
    double *uq = (double *)malloc(sizeof(double) * N), *pv = (double *)malloc(sizeof(double) * N);
    int rc = (!u || !v || !t || !kn || !uq || !pv) ? -2 : 0;
    for (int i = 0; !rc && i < ntab; i++) {
        if (!(ktab[i] > 0.0) || !(ptab[i] > 0.0)) { rc = -1; break; }
        u[i] = log(ktab[i]); v[i] = log(ptab[i]);
    }
    if (!rc) rc = orc_cheb_knodes(N, kmin, kmax, kmap, t, kn);
    for (int j = 0; !rc && j < N; j++) {
        if (!(kn[j] > 0.0)) { rc = -1; break; }
        uq[j] = log(kn[j]);
    }
    if (!rc) rc = orc_spline_natural(ntab, u, v, N, uq, pv);
    if (!rc) {
        for (int j = 0; j < N; j++) pv[j] = exp(pv[j]);
        rc = orc_cheb_dct(N, pv, a);
    }
    free(u); free(v); free(t); free(kn); free(uq); free(pv);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Prefactors N(l) of Eqs. gg, gs, ss: 2/pi, (2/pi) sqrt((l+2)!/(l-2)!),     */
/* (2/pi) (l+2)!/(l-2)!, with (l+2)!/(l-2)! = (l+2)(l+1) l (l-1).            */
/* ------------------------------------------------------------------------- */
double orc_prefactor(int type, double l)
{
    double L = l;
    double r = (L + 2.0) * (L + 1.0) * L * (L - 1.0);
    if (type == 0) return 2.0 / ORC_PI;
    if (type == 1) return 2.0 / ORC_PI * sqrt(r);
    return 2.0 / ORC_PI * r;
}

/* Number of spectra for ng clustering and ns lensing tracers:
 * gg (i <= j), then gs (every i, j), then ss (i <= j). */
int orc_npairs(int ng, int ns)
{
    return ng * (ng + 1) / 2 + ng * ns + ns * (ns + 1) / 2;
}

/* ------------------------------------------------------------------------- */
/* Steps 5 and 6: w and C.                                                   */
/*   w^{AB}_l(a, r) = D(chi_a) D(R_r chi_a) sum_n a_n T~^{AB}_{n;l}(a, r)      */
/*   C^{AB}_{ij}(l) = N_AB(l) sum_a sum_r wchi_a wR_r chi_a                    */
/*                    K_i^A(chi_a) K_j^B(R_r chi_a) w^{AB}_l(a, r)            */
/* Inputs: T[t][e][n][q] (q = a Rn + r), kernels kchi[tr][a] and              */
/* kRchi[tr][q] (tracers 0..ng-1 clustering, ng..ng+ns-1 lensing, the lensing */
/* ones already divided by chi^2), growth Dchi[a], DRchi[q].                 */
/* Output C[p][e] in the pair order of orc_npairs.                          */
/* ------------------------------------------------------------------------- */
/* sym != 0: the symmetrised form (App. A), R in (0, 1]:                   */
/*   C = N_AB sum_a sum_r wchi_a wR_r chi_a                                  */
/*       [K^A_i(chi_a) K^B_j(R_r chi_a) + K^B_j(chi_a) K^A_i(R_r chi_a)] w    */
/* (the kernels at chi_a are the rows of kchi, at R_r chi_a those of kRchi). */
int orc_cl(int n_ell, const double *ell, int X, int Rn, const double *chi, const double *wchi,
           const double *R, const double *wR, int N, const double *T, const double *a,
           int ng, int ns, const double *kchi, const double *kRchi,
           const double *Dchi, const double *DRchi, double *C, int nthreads, int sym)
{
    (void)R;
    if (n_ell < 1 || X < 1 || Rn < 1 || N < 1 || ng < 0 || ns < 0 || ng + ns < 1) return -1;
    const int Q = X * Rn;
    int p0[3] = {0, ng * (ng + 1) / 2, ng * (ng + 1) / 2 + ng * ns};
    int nt = orc_threads(nthreads);
    int fail = 0;
    /* every (type, ell) result is independent: threads take whole (t, e) items
     * and each keeps its own w, so the arithmetic of every item is unchanged */
#pragma omp parallel num_threads(nt)
    {
    double *w = (double *)malloc(sizeof(double) * Q);
    if (!w) {
#pragma omp atomic write
        fail = 1;
    }
#pragma omp for schedule(dynamic, 1) collapse(2)
    for (int t = 0; t < 3; t++) {
        for (int e = 0; e < n_ell; e++) {
            if (!w) continue;
            const double *Te = T + ((size_t)t * n_ell + e) * N * (size_t)Q;
            for (int q = 0; q < Q; q++) {
                double s = 0.0;
                for (int n = 0; n < N; n++) s += a[n] * Te[(size_t)n * Q + q];
                w[q] = Dchi[q / Rn] * DRchi[q] * s;
            }
            double pref = orc_prefactor(t, ell[e]);
            int p = p0[t];
            int nA = (t == 2) ? ns : ng, nB = (t == 0) ? ng : ns;
            int offA = (t == 2) ? ng : 0, offB = (t == 0) ? 0 : ng;
            for (int i = 0; i < nA; i++) {
                for (int j = (t == 1 ? 0 : i); j < nB; j++) {
                    const double *Ki = kchi + (size_t)(offA + i) * X;
                    const double *Kj = kRchi + (size_t)(offB + j) * Q;
                    const double *Kj1 = kchi + (size_t)(offB + j) * X;  /* sym: B at chi */
                    const double *Ki2 = kRchi + (size_t)(offA + i) * Q; /* sym: A at R chi */
                    double s = 0.0;
                    for (int aa = 0; aa < X; aa++) {
                        if (!sym) {
                            double sr = 0.0;
                            for (int r = 0; r < Rn; r++) {
                                int q = aa * Rn + r;
                                sr += wR[r] * Kj[q] * w[q];
                            }
                            s += wchi[aa] * chi[aa] * Ki[aa] * sr;
                        } else {
                            double sr = 0.0;
                            for (int r = 0; r < Rn; r++) {
                                int q = aa * Rn + r;
                                sr += wR[r] * (Ki[aa] * Kj[q] + Kj1[aa] * Ki2[q]) * w[q];
                            }
                            s += wchi[aa] * chi[aa] * sr;
                        }
                    }
                    C[(size_t)p * n_ell + e] = pref * s;
                    p++;
                }
            }
        }
    }
    free(w);
    }
    return fail ? -2 : 0;
}

/* ------------------------------------------------------------------------- */
/* Limber approximation (Sec. 2.2) on the chi rule of the plan.              */
/*   gg: C = sum_a wchi_a / chi_a^2 W_i W_j P_a                               */
/*   gs: C = sqrt((l+2)(l+1)l(l-1)) / nu^2 sum_a wchi_a / chi_a^2 W_i W_j P_a */
/*   ss: C = (l+2)(l+1)l(l-1) / nu^4   sum_a wchi_a / chi_a^2 W_i W_j P_a     */
/* with nu = l + 1/2, W = the tracer's kernel (clustering: kchi as given;    */
/* lensing: kchi chi^2, since the library's lensing kernels are W / chi^2),  */
/* P_a = P(nu / chi_a, chi_a) given for every ell and node, P[e][a]: the     */
/* closure of the Bessel pair (Sec. 2.2) turns N_AB(l) into these factors,   */
/* the 1 / (k chi)^2 of each lensing side into 1 / nu^2.                     */
/* extended != 0 multiplies each term by the first-order correction of the   */
/* extended Limber approximation (Sec. 2.2):                                 */
/*   1 - (1/nu^2) [chi^2/2 (Kt_i''/Kt_i + Kt_j''/Kt_j)                        */
/*                 + chi^3/6 (Kt_i'''/Kt_i + Kt_j'''/Kt_j)];                   */
/* the printed equation has a plus sign, under which the corrected value     */
/* moves away from the full integral; with the minus sign the gap to the     */
/* full integral shrinks and falls faster with l (pinned in the tests), so   */
/* the print is read as a sign slip.                                         */
/* Kt = W D / sqrt(chi) (the growth belongs to the kernel when P is the      */
/* growth-separable D^2 P(k)); written as products so that no kernel is      */
/* divided by: W_i W_j (Kt_i''/Kt_i) = W_j Kt_i'' sqrt(chi) / D.  The        */
/* derivatives are central differences on the uniform chi nodes (second:     */
/* f[a+1] - 2 f[a] + f[a-1] over h^2; third: f[a+2] - 2 f[a+1] + 2 f[a-1]    */
/* - f[a-2] over 2 h^3), those of the nearest node with a full stencil at    */
/* the first and last two nodes.  Output C[p][e] in the order of orc_npairs. */
/* ------------------------------------------------------------------------- */
static void orc_fd_derivs(int X, double h, const double *f, double *d2, double *d3)
{
    for (int a = 0; a < X; a++) {
        int c2 = a < 1 ? 1 : (a > X - 2 ? X - 2 : a);
        int c3 = a < 2 ? 2 : (a > X - 3 ? X - 3 : a);
        d2[a] = (f[c2 + 1] - 2.0 * f[c2] + f[c2 - 1]) / (h * h);
        d3[a] = (f[c3 + 2] - 2.0 * f[c3 + 1] + 2.0 * f[c3 - 1] - f[c3 - 2]) / (2.0 * h * h * h);
    }
}

int orc_limber(int n_ell, const double *ell, int X, const double *chi, const double *wchi, int ng, int ns,
               const double *kchi, const double *Dchi, const double *P, int extended, double *C)
{
    if (n_ell < 1 || X < 5 || ng < 0 || ns < 0 || ng + ns < 1) return -1;
    const int ntr = ng + ns;
    double *W = (double *)malloc(sizeof(double) * ntr * X);
    double *K2 = (double *)malloc(sizeof(double) * ntr * X);
    double *K3 = (double *)malloc(sizeof(double) * ntr * X);
    double *Kt = (double *)malloc(sizeof(double) * X);
    if (!W || !K2 || !K3 || !Kt) { free(W); free(K2); free(K3); free(Kt); return -2; }
    const double h = chi[1] - chi[0];
    for (int r = 0; r < ntr; r++) {
        for (int a = 0; a < X; a++) {
            W[r * X + a] = (r < ng) ? kchi[r * X + a] : kchi[r * X + a] * chi[a] * chi[a];
            Kt[a] = W[r * X + a] * Dchi[a] / sqrt(chi[a]);
        }
        orc_fd_derivs(X, h, Kt, K2 + r * X, K3 + r * X);
    }
    int p0[3] = {0, ng * (ng + 1) / 2, ng * (ng + 1) / 2 + ng * ns};
    for (int t = 0; t < 3; t++) {
        int nA = (t == 2) ? ns : ng, nB = (t == 0) ? ng : ns;
        int offA = (t == 2) ? ng : 0, offB = (t == 0) ? 0 : ng;
        for (int e = 0; e < n_ell; e++) {
            double l = (double)ell[e], nu = l + 0.5, f4 = (l + 2.0) * (l + 1.0) * l * (l - 1.0);
            double pref = (t == 0) ? 1.0 : (t == 1 ? sqrt(f4) / (nu * nu) : f4 / (nu * nu * nu * nu));
            int p = p0[t];
            for (int i = 0; i < nA; i++) {
                for (int j = (t == 1 ? 0 : i); j < nB; j++) {
                    const double *Wi = W + (offA + i) * X, *Wj = W + (offB + j) * X;
                    double s = 0.0;
                    for (int a = 0; a < X; a++) {
                        double term = Wi[a] * Wj[a];
                        if (extended) {
                            double c = chi[a], r = sqrt(c) / Dchi[a];
                            double t2 = Wj[a] * K2[(offA + i) * X + a] + Wi[a] * K2[(offB + j) * X + a];
                            double t3 = Wj[a] * K3[(offA + i) * X + a] + Wi[a] * K3[(offB + j) * X + a];
                            term -= (c * c / 2.0 * t2 + c * c * c / 6.0 * t3) * r / (nu * nu);
                        }
                        s += wchi[a] / (chi[a] * chi[a]) * term * P[(size_t)e * X + a];
                    }
                    C[(size_t)p * n_ell + e] = pref * s;
                    p++;
                }
            }
        }
    }
    free(W); free(K2); free(K3); free(Kt);
    return 0;
}

/* The linear spectrum at the Limber points k = nu / chi_a, P[e][a] =
 * D(chi_a)^2 P(k), P(k) from the request's table by the natural cubic spline
 * of (ln k, ln P) that the fit uses (orc_spline_natural), zero where k lies
 * outside the table. */
int orc_limber_plin(int n_ell, const double *ell, int X, const double *chi, const double *Dchi, int ntab,
                    const double *ktab, const double *ptab, double *P)
{
    if (n_ell < 1 || X < 1 || ntab < 3) return -1;
    double *u = (double *)malloc(sizeof(double) * ntab), *v = (double *)malloc(sizeof(double) * ntab);
    double *uq = (double *)malloc(sizeof(double) * X), *out = (double *)malloc(sizeof(double) * X);
    int rc = (!u || !v || !uq || !out) ? -2 : 0;
    for (int i = 0; !rc && i < ntab; i++) {
        if (!(ktab[i] > 0.0) || !(ptab[i] > 0.0)) { rc = -1; break; }
        u[i] = log(ktab[i]); v[i] = log(ptab[i]);
    }
    for (int e = 0; !rc && e < n_ell; e++) {
        double nu = (double)ell[e] + 0.5;
        int m = 0;
        int *idx = (int *)malloc(sizeof(int) * X);
        if (!idx) { rc = -2; break; }
        for (int a = 0; a < X; a++) {
            double k = nu / chi[a];
            if (k >= ktab[0] && k <= ktab[ntab - 1]) { uq[m] = log(k); idx[m] = a; m++; }
            P[(size_t)e * X + a] = 0.0;
        }
        if (m > 0) rc = orc_spline_natural(ntab, u, v, m, uq, out);
        for (int q = 0; !rc && q < m; q++) P[(size_t)e * X + idx[q]] = Dchi[idx[q]] * Dchi[idx[q]] * exp(out[q]);
        free(idx);
    }
    free(u); free(v); free(uq); free(out);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Non-separable spectrum (Eqs. cheb_pk, pmd with general c_n(chi1, chi2)).  */
/* Pq[q][j] = P(k_j, chi_a, R_r chi_a) at the N Chebyshev k-nodes for every  */
/* chi-R node q = a Rn + r; per node the coefficients follow from the        */
/* transform of orc_cheb_dct, c_n(q), and                                    */
/*   w_l(a, r) = sum_n c_n(q) T~_{n;l}(a, r)                                 */
/* replaces D(chi_a) D(R_r chi_a) sum_n a_n T~; the chi-R quadrature is that */
/* of orc_cl with the kernels K alone.  Output C[p][e].                      */
/* ------------------------------------------------------------------------- */
int orc_cl_nonsep(int n_ell, const double *ell, int X, int Rn, const double *chi, const double *wchi,
                  const double *wR, int N, const double *T, const double *Pq, int ng, int ns,
                  const double *kchi, const double *kRchi, double *C)
{
    if (n_ell < 1 || X < 1 || Rn < 1 || N < 1 || ng < 0 || ns < 0 || ng + ns < 1) return -1;
    const int Q = X * Rn;
    double *c = (double *)malloc(sizeof(double) * (size_t)Q * N);
    double *w = (double *)malloc(sizeof(double) * Q);
    if (!c || !w) { free(c); free(w); return -2; }
    int rc = 0;
    for (int q = 0; !rc && q < Q; q++) rc = orc_cheb_dct(N, Pq + (size_t)q * N, c + (size_t)q * N);
    int p0[3] = {0, ng * (ng + 1) / 2, ng * (ng + 1) / 2 + ng * ns};
    for (int t = 0; !rc && t < 3; t++) {
        for (int e = 0; e < n_ell; e++) {
            const double *Te = T + ((size_t)t * n_ell + e) * N * (size_t)Q;
            for (int q = 0; q < Q; q++) {
                double s = 0.0;
                for (int n = 0; n < N; n++) s += c[(size_t)q * N + n] * Te[(size_t)n * Q + q];
                w[q] = s;
            }
            double pref = orc_prefactor(t, ell[e]);
            int p = p0[t];
            int nA = (t == 2) ? ns : ng, nB = (t == 0) ? ng : ns;
            int offA = (t == 2) ? ng : 0, offB = (t == 0) ? 0 : ng;
            for (int i = 0; i < nA; i++) {
                for (int j = (t == 1 ? 0 : i); j < nB; j++) {
                    const double *Ki = kchi + (size_t)(offA + i) * X;
                    const double *Kj = kRchi + (size_t)(offB + j) * Q;
                    double s = 0.0;
                    for (int aa = 0; aa < X; aa++) {
                        double sr = 0.0;
                        for (int r = 0; r < Rn; r++) sr += wR[r] * Kj[aa * Rn + r] * w[aa * Rn + r];
                        s += wchi[aa] * chi[aa] * Ki[aa] * sr;
                    }
                    C[(size_t)p * n_ell + e] = pref * s;
                    p++;
                }
            }
        }
    }
    free(c); free(w);
    return rc;
}
