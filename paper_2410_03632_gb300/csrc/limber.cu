// Limber terms of Sec. 2.2 and the non-linear correction of Sec. 3.2:
//
//   C^Limber_ij(l) = pref_AB(l) sum_a wchi_a / chi_a^2 W_i(chi_a) W_j(chi_a) P(nu / chi_a, chi_a),
//   nu = l + 1/2, pref = 1 (gg), sqrt((l+2)(l+1)l(l-1)) / nu^2 (gs), (l+2)(l+1)l(l-1) / nu^4 (ss),
//
// W = the clustering kernel as given, the lensing kernel times chi^2 (the
// library takes lensing kernels divided by chi^2), on the plan's chi rule.
// The linear P is D(chi)^2 P(k) with P(k) from the request's table by the
// same natural cubic spline in (ln k, ln P) the Chebyshev fit uses (second
// derivatives kept by the fit), zero outside the table.  The extended
// (first-order) Limber correction multiplies each term by
//   1 - (1/nu^2) [chi^2/2 (Kt_i''/Kt_i + Kt_j''/Kt_j) + chi^3/6 (Kt_i'''/Kt_i + Kt_j'''/Kt_j)],
// Kt = W D / sqrt(chi), with central differences on the uniform chi nodes
// (the sign of the printed equation is read as a slip: with a plus sign the
// corrected value moves away from the full integral).  The non-linear
// correction C_tot = C_lin + C^Limber_delta - C^Limber_lin uses the caller's
// P_delta at the Limber points k = nu / chi_a.
#include <cmath>

#include "blast_internal.h"

namespace {

constexpr int kLimThreads = 128;

__device__ __forceinline__ double lensing_w(const double *kc, int a, double chi) { return kc[a] * chi * chi; }

// Natural cubic spline of (ln k, ln P) at ln k = x: the fit's second
// derivatives M; zero outside the table.
__device__ double spline_P(const ReqDev &rq, double k)
{
    const int n = rq.n_ptab;
    const double *kt = rq.k_tab, *pt = rq.p_tab;
    if (!(k >= kt[0] && k <= kt[n - 1])) return 0.0;
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (kt[mid] <= k) lo = mid; else hi = mid;
    }
    const double ul = log(kt[lo]), uh = log(kt[hi]);
    const double h = uh - ul, t = (log(k) - ul) / h, s1 = 1.0 - t;
    const double val = s1 * log(pt[lo]) + t * log(pt[hi]) +
                       h * h / 6.0 * ((s1 * s1 * s1 - s1) * rq.spM[lo] + (t * t * t - t) * rq.spM[hi]);
    return exp(val);
}

// One block per (selected ell, request): the spectrum at the chi nodes and the
// tracer weights in shared memory, then one thread per tracer pair.
__global__ void __launch_bounds__(kLimThreads)
k_limber(const ReqDev *__restrict__ reqs, const double *__restrict__ chi, const double *__restrict__ wchi, int X,
         const int *__restrict__ esel, const double *__restrict__ ell, int mode, int extended)
{
    extern __shared__ double lsm[];
    const ReqDev &rq = reqs[blockIdx.y];
    const int e = esel[blockIdx.x];
    const int col = rq.e_out[e];
    if (col < 0) return;
    const int ng = rq.n_clust, ns = rq.n_lens, ntr = ng + ns;
    double *Pv = lsm;                 // [X] P (mode 2: P_delta - P_lin)
    double *W = Pv + X;               // [ntr][X]
    double *K2 = W + (size_t)ntr * X; // [ntr][X] Kt'' (extended only)
    double *K3 = K2 + (size_t)ntr * X;
    const double l = ell[e], nu = l + 0.5;
    for (int a = threadIdx.x; a < X; a += blockDim.x) {
        const double c = chi[a], k = nu / c, D2 = rq.growth_chi[a] * rq.growth_chi[a];
        double v;
        if (mode == 0) v = D2 * spline_P(rq, k);
        else if (mode == 1) v = rq.pnl[(size_t)e * X + a];
        else v = rq.pnl[(size_t)e * X + a] - D2 * spline_P(rq, k);
        Pv[a] = v;
        for (int r = 0; r < ntr; r++)
            W[r * X + a] = (r < ng) ? rq.kern_chi[(size_t)r * X + a] : lensing_w(rq.kern_chi + (size_t)r * X, a, c);
    }
    __syncthreads();
    if (extended) {
        const double h = chi[1] - chi[0];
        for (int i = threadIdx.x; i < ntr * X; i += blockDim.x) {
            const int r = i / X, a = i % X;
            const int c2 = a < 1 ? 1 : (a > X - 2 ? X - 2 : a);
            const int c3 = a < 2 ? 2 : (a > X - 3 ? X - 3 : a);
            auto kt = [&](int m) { return W[r * X + m] * rq.growth_chi[m] / sqrt(chi[m]); };
            K2[i] = (kt(c2 + 1) - 2.0 * kt(c2) + kt(c2 - 1)) / (h * h);
            K3[i] = (kt(c3 + 2) - 2.0 * kt(c3 + 1) + 2.0 * kt(c3 - 1) - kt(c3 - 2)) / (2.0 * h * h * h);
        }
        __syncthreads();
    }
    const int ngg = ng * (ng + 1) / 2, ngs = ng * ns, P = ngg + ngs + ns * (ns + 1) / 2;
    const double f4 = (l + 2.0) * (l + 1.0) * l * (l - 1.0);
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        int t, ia, jb;
        if (p < ngg) {
            int i = 0, rem = p;
            while (rem >= ng - i) { rem -= ng - i; i++; }
            t = 0; ia = i; jb = i + rem;
        } else if (p < ngg + ngs) {
            t = 1; ia = (p - ngg) / ns; jb = ng + (p - ngg) % ns;
        } else {
            int i = 0, rem = p - ngg - ngs;
            while (rem >= ns - i) { rem -= ns - i; i++; }
            t = 2; ia = ng + i; jb = ng + i + rem;
        }
        const double pref = (t == 0) ? 1.0 : (t == 1 ? sqrt(f4) / (nu * nu) : f4 / (nu * nu * nu * nu));
        const double *Wi = W + (size_t)ia * X, *Wj = W + (size_t)jb * X;
        double s = 0.0;
        for (int a = 0; a < X; a++) {
            double term = Wi[a] * Wj[a];
            if (extended) {
                const double c = chi[a], r = sqrt(c) / rq.growth_chi[a];
                const double t2 = Wj[a] * K2[(size_t)ia * X + a] + Wi[a] * K2[(size_t)jb * X + a];
                const double t3 = Wj[a] * K3[(size_t)ia * X + a] + Wi[a] * K3[(size_t)jb * X + a];
                term -= (c * c / 2.0 * t2 + c * c * c / 6.0 * t3) * r / (nu * nu);
            }
            s = fma(wchi[a] / (chi[a] * chi[a]) * term, Pv[a], s);
        }
        double *out = rq.cl + (size_t)p * rq.n_sel + col;
        const double v = rq.status ? nan("") : pref * s;
        if (mode == 2) *out += v;
        else *out = v;
    }
}

}  // namespace

int launch_limber(blast_plan *p, ReqDev *dreq, int nreq, const int *d_esel, int n_esel, int mode, int extended,
                  cudaStream_t s)
{
    const int ntr = p->max_clust + p->max_lens;
    const size_t smem = sizeof(double) * ((size_t)p->X + (size_t)(extended ? 3 : 1) * ntr * p->X);
    if (smem > 220 * 1024) return BLAST_EINVAL;
    BL_CUDA(allow_opt_in_smem(k_limber, p->device));
    dim3 grid(n_esel, nreq);
    k_limber<<<grid, kLimThreads, smem, s>>>(dreq, p->d_chi, p->d_wchi, p->X, d_esel, p->d_ell, mode, extended);
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}
