// Step (pre): the cosmology-independent basis integrals of Eq. t_tilde,
//   T~^{AB}_{n;l}(chi_a, R_r chi_a) = int_{kmin}^{kmax} dk f^{AB}(k) T_n(x(k)) j_l(k chi_a) j_l(k R_r chi_a),
// f^gg = k^2, f^gs = 1, f^ss = 1/k^2, by the Clenshaw-Curtis rule of Sec. 3.2:
// a GEMM over the k nodes m,
//   T~[t n][l, q] = sum_m A[m][t n] B_l[m][q],  A = w_m f_t(k_m) T_n(x_m),
//   B_l[m][q]    = j_l(k_m chi_a) j_l(k_m R_r chi_a),
// with B generated on chip from spherical Bessel recurrences in FP64.
#include <cmath>

#include "blast_internal.h"

namespace {

constexpr int kG = 8;     // plan ells per CTA (one group)
constexpr int kRT = 8;    // R nodes per CTA
constexpr int kMC = 28;   // k nodes per chunk: (1 + kRT) * kMC = 252 Bessel chains per chunk
constexpr int kThreads = 256;

// A[m][t*N + n] = w_m f_t(k_m) T_n(x(k_m)); T_n by the three-term recurrence.
__global__ void k_basis_A(const double *__restrict__ kq, const double *__restrict__ wq, int Nk, int N,
                          int kmap, double kmin, double kmax, double *__restrict__ A)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Nk) return;
    double k = kq[m];
    double x = (kmap == 0) ? (2.0 * k - kmin - kmax) / (kmax - kmin)
                           : 2.0 * (log(k) - log(kmin)) / (log(kmax) - log(kmin)) - 1.0;
    x = fmin(1.0, fmax(-1.0, x));
    double f0 = wq[m] * k * k, f1 = wq[m], f2 = wq[m] / (k * k);
    double *row = A + (size_t)m * 3 * N;
    double tprev = 1.0, tcur = x;
    for (int n = 0; n < N; n++) {
        double Tn;
        if (n == 0) Tn = 1.0;
        else if (n == 1) Tn = x;
        else { Tn = 2.0 * x * tcur - tprev; tprev = tcur; tcur = Tn; }
        row[n] = f0 * Tn;
        row[N + n] = f1 * Tn;
        row[2 * N + n] = f2 * Tn;
    }
}

// j_l(x) for the (at most kG) ascending multipoles lg[0..ng) of one group.
// x > lhi: forward recurrence from j_0, j_1 (stable for l < x).
// x <= lhi: Miller's backward recurrence from lhi + 20 + 10 lhi^(1/3), scaled
// by the least-squares match of the recurrence's two lowest orders to the
// closed forms of j_0 and j_1.  Values below 1e-323 (j_l(x) <= (e x / 2l)^l)
// are returned as zero without a recurrence.
__device__ void jl_group(double x, const int *lg, int ng, double *out)
{
#pragma unroll
    for (int g = 0; g < kG; g++) out[g] = 0.0;
    if (ng <= 0 || !(x > 0.0)) return;
    const int llo = lg[0], lhi = lg[ng - 1];
    if ((double)llo * log(2.718281828459045 * x / (2.0 * llo)) < -744.0) return;
    double s, c;
    sincos(x, &s, &c);
    const double inv = 1.0 / x;
    double j0 = s * inv;
    double j1 = (x < 1e-2) ? x * (1.0 / 3.0 - x * x / 30.0 + x * x * x * x / 840.0) : (j0 - c) * inv;
    if (x > (double)lhi) {
        double jm = j0, jc = j1;
        int gi = 0;
        while (gi < ng && lg[gi] <= 1) { out[gi] = (lg[gi] == 0) ? j0 : j1; gi++; }
        double dl = 3.0;  // 2l + 1 at l = 1, exact in double
        for (int l = 1; l < lhi; l++) {
            double jn = (dl * inv) * jc - jm;  // j_{l+1}
            dl += 2.0;
            jm = jc;
            jc = jn;
            if (gi < ng && l + 1 == lg[gi]) { out[gi] = jc; gi++; }
        }
        return;
    }
    const int l0 = lhi + 20 + (int)(10.0 * cbrt((double)lhi));
    double fp = 0.0, f = 1e-200;
    int gi = ng - 1;
    double dl = 2.0 * l0 + 1.0;  // exact in double
    for (int l = l0; l > 0; l--) {
        if (gi >= 0 && l == lg[gi]) { out[gi] = f; gi--; }
        double fm = (dl * inv) * f - fp;  // f_{l-1}
        dl -= 2.0;
        fp = f;
        f = fm;
        if ((l & 3) == 0 && fabs(f) > 1e200) {
            f *= 1e-200;
            fp *= 1e-200;
#pragma unroll
            for (int g = 0; g < kG; g++)
                if (g > gi) out[g] *= 1e-200;
        }
    }
    // f = f_0, fp = f_1 (arbitrary scale): normalise before squaring
    const double mx = fmax(fabs(f), fabs(fp));
    f /= mx;
    fp /= mx;
    double scale = (j0 * f + j1 * fp) / ((f * f + fp * fp) * mx);
#pragma unroll
    for (int g = 0; g < kG; g++) out[g] *= scale;
}

// j_v0(x) and j_v0+1(x) for a fractional order v0 in [0, 1) (non-integer
// multipoles), j_v = sqrt(pi / 2x) J_{v+1/2}:
// x >= 30: Hankel's asymptotic expansion, j_v = (P cos w - Q sin w) / x with
//   w = x - (v + 1) pi / 2 (formed by angle addition from sincos(x), which
//   keeps the phase exact for large x), P and Q the even and odd terms of
//   a_k = (m - 1)(m - 9)...(m - (2k-1)^2) / (k! (8x)^k), m = 4 (v + 1/2)^2;
// 1e-3 <= x < 30: Miller's backward recurrence on J_{mu0 + k}, mu0 =
//   frac(v0 + 1/2), normalised by Neumann's expansion
//   (x/2)^mu0 = sum_i (mu0 + 2i) Gamma(mu0 + i) / i! J_{mu0 + 2i};
// x < 1e-3: the first three terms of the power series.
__device__ void jnu_start(double v0, double x, double &j0, double &j1)
{
    const double mu = v0 + 0.5;
    if (x >= 30.0) {
        double sx, cx;
        sincos(x, &sx, &cx);
        double out[2];
#pragma unroll
        for (int o = 0; o < 2; o++) {
            const double v = v0 + o, m = 4.0 * (v + 0.5) * (v + 0.5);
            double P = 1.0, Qs = 0.0, t = 1.0;
            for (int k = 1; k < 60; k++) {
                const double c = (double)(2 * k - 1);
                const double tn = t * (m - c * c) / ((double)k * 8.0 * x);
                if (fabs(tn) > fabs(t) && k > 2) break;  // the asymptotic terms start to grow
                t = tn;
                const int r = k & 3;  // signs: k = 1 +Q, 2 -P, 3 -Q, 4 +P
                if (r == 1) Qs += t;
                else if (r == 2) P -= t;
                else if (r == 3) Qs -= t;
                else P += t;
                if (fabs(t) < 1e-18) break;
            }
            double sp, cp;  // phase (v + 1) pi / 2
            sincospi(0.5 * (v + 1.0), &sp, &cp);
            const double cw = cx * cp + sx * sp, sw = sx * cp - cx * sp;
            out[o] = (P * cw - Qs * sw) / x;
        }
        j0 = out[0];
        j1 = out[1];
        return;
    }
    const double pre = sqrt(0.5 * 3.14159265358979323846 / x);
    if (x < 1e-3) {
#pragma unroll
        for (int o = 0; o < 2; o++) {
            const double m = mu + o, h = 0.25 * x * x;
            const double J = pow(0.5 * x, m) / tgamma(m + 1.0) * (1.0 - h / (m + 1.0) + h * h / (2.0 * (m + 1.0) * (m + 2.0)));
            (o ? j1 : j0) = pre * J;
        }
        return;
    }
    const int nb = (int)floor(mu);
    const double mu0 = mu - nb;
    const int K = (int)x + 40;  // <= 69
    double c[36];               // Neumann weights for k = 2i <= K
    double g = tgamma(mu0 + 1.0);
    c[0] = g;
    for (int i = 1; i <= K / 2; i++) {
        c[i] = (mu0 + 2.0 * i) * g;
        g *= (mu0 + i) / (i + 1.0);
    }
    double fp = 0.0, f = 1e-250, S = 0.0, r0 = 0.0, r1 = 0.0;
    for (int k = K; k >= 0; k--) {
        if (k == nb) r0 = f;
        if (k == nb + 1) r1 = f;
        if ((k & 1) == 0) S += c[k / 2] * f;
        if (k == 0) break;
        const double fm = 2.0 * (mu0 + k) / x * f - fp;
        fp = f;
        f = fm;
        if (fabs(f) > 1e200) { f *= 1e-200; fp *= 1e-200; S *= 1e-200; r0 *= 1e-200; r1 *= 1e-200; }
    }
    const double nrm = pow(0.5 * x, mu0) / S;
    j0 = pre * r0 * nrm;
    j1 = pre * r1 * nrm;
}

// j_nu(x) for a real multipole nu >= 2: from j_v0 and j_v0+1 (v0 = frac(nu))
// forward to nu when x > nu, else Miller's backward recurrence from
// nu + 20 + 10 nu^(1/3) down to v0 matched to them (least squares, as for
// integer orders).  Values below 1e-323 are zero.
__device__ double jnu_real(double nu, double x)
{
    if (!(x > 0.0)) return 0.0;
    if (nu * log(2.718281828459045 * x / (2.0 * nu)) < -744.0) return 0.0;
    const int n = (int)floor(nu);
    const double v0 = nu - n;
    double j0, j1;
    jnu_start(v0, x, j0, j1);
    if (n == 0) return j0;
    if (x > nu) {
        double jm = j0, jc = j1, v = v0 + 1.0;
        for (int k = 1; k < n; k++) {
            const double jn = (2.0 * v + 1.0) / x * jc - jm;
            jm = jc;
            jc = jn;
            v += 1.0;
        }
        return jc;
    }
    const int top = n + 20 + (int)(10.0 * cbrt((double)n));
    double fp = 0.0, f = 1e-200, rec = 0.0, v = v0 + top;
    for (int k = top; k > 0; k--) {
        if (k == n) rec = f;
        const double fm = (2.0 * v + 1.0) / x * f - fp;  // order v - 1
        fp = f;
        f = fm;
        v -= 1.0;
        if (fabs(f) > 1e200) { f *= 1e-200; fp *= 1e-200; rec *= 1e-200; }
    }
    const double mx = fmax(fabs(f), fabs(fp));
    f /= mx;
    fp /= mx;
    return rec * (j0 * f + j1 * fp) / ((f * f + fp * fp) * mx);
}

template <int ROWS>
__global__ void __launch_bounds__(kThreads)
k_basis_gemm(const double *__restrict__ A, const double *__restrict__ kq, int Nk, int N,
             const double *__restrict__ ell, int real_ell, int L, int e0, const double *__restrict__ chi,
             const double *__restrict__ R, int Rn, int Q, double *__restrict__ T)
{
    extern __shared__ double sm[];
    const int rows3 = 3 * N;
    double *As = sm;                           // [kMC][3N]
    double *Jv = As + kMC * rows3;             // [(1+kRT) kMC][kG]
    double *Bp = Jv + (1 + kRT) * kMC * kG;    // [kMC][kG*kRT]
    __shared__ int lg[kG];
    __shared__ double lgr[kG];

    const int tid = threadIdx.x;
    const int a = blockIdx.y;
    const int r0 = blockIdx.x * kRT;
    const int ng = min(kG, L - e0);
    if (tid < kG) {
        lgr[tid] = (tid < ng) ? ell[e0 + tid] : 0.0;
        lg[tid] = (int)lgr[tid];
    }
    const double chia = chi[a];
    const int rb = tid >> 3, cb = tid & 7;
    double acc[ROWS][kG];
#pragma unroll
    for (int i = 0; i < ROWS; i++)
#pragma unroll
        for (int g = 0; g < kG; g++) acc[i][g] = 0.0;
    __syncthreads();

    for (int m0 = 0; m0 < Nk; m0 += kMC) {
        const int mcnt = min(kMC, Nk - m0);
        const double *Asrc = A + (size_t)m0 * rows3;
        for (int i = tid; i < mcnt * rows3; i += kThreads) As[i] = Asrc[i];
        if (tid < (1 + kRT) * kMC) {
            const int mi = tid % kMC, side = tid / kMC;
            double out[kG];
            const int r = r0 + side - 1;
            bool ok = mi < mcnt && (side == 0 || r < Rn);
            double dist = (side == 0) ? chia : (ok ? R[r] * chia : 0.0);
            if (ok && !real_ell) {
                jl_group(kq[m0 + mi] * dist, lg, ng, out);
            } else if (ok) {  // each non-integer multipole has its own recurrence
#pragma unroll
                for (int g = 0; g < kG; g++) out[g] = (g < ng) ? jnu_real(lgr[g], kq[m0 + mi] * dist) : 0.0;
            } else {
#pragma unroll
                for (int g = 0; g < kG; g++) out[g] = 0.0;
            }
#pragma unroll
            for (int g = 0; g < kG; g++) Jv[tid * kG + g] = out[g];
        }
        __syncthreads();
        for (int i = tid; i < kMC * kG * kRT; i += kThreads) {
            const int mi = i / (kG * kRT), cmb = i % (kG * kRT);
            const int g = cmb / kRT, rr = cmb % kRT;
            Bp[i] = Jv[mi * kG + g] * Jv[((1 + rr) * kMC + mi) * kG + g];
        }
        __syncthreads();
        for (int mi = 0; mi < mcnt; mi++) {
            double b[kG];
#pragma unroll
            for (int g = 0; g < kG; g++) b[g] = Bp[mi * kG * kRT + g * kRT + cb];
#pragma unroll
            for (int i = 0; i < ROWS; i++) {
                const int row = rb + 32 * i;
                const double av = (row < rows3) ? As[mi * rows3 + row] : 0.0;
#pragma unroll
                for (int g = 0; g < kG; g++) acc[i][g] = fma(av, b[g], acc[i][g]);
            }
        }
        __syncthreads();
    }
    const int r = r0 + cb;
    if (r >= Rn) return;
#pragma unroll
    for (int i = 0; i < ROWS; i++) {
        const int row = rb + 32 * i;
        if (row >= rows3) continue;
        const int t = row / N, n = row % N;
#pragma unroll
        for (int g = 0; g < kG; g++) {
            if (g >= ng) continue;
            T[(((size_t)t * L + e0 + g) * N + n) * Q + (size_t)a * Rn + r] = acc[i][g];
        }
    }
}

// FP64 basis -> FP32 copy (same layout) for the CUDA-core FP32 path.
__global__ void k_basis_to_f32(const double *__restrict__ T, float *__restrict__ T32, size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) T32[i] = (float)T[i];
}

template <int ROWS>
int launch_gemm_rows(blast_plan *p, const double *A, const double *kq, const double *ell, const double *R,
                     cudaStream_t s)
{
    size_t smem = sizeof(double) * ((size_t)kMC * 3 * p->N + (size_t)(1 + kRT) * kMC * kG + (size_t)kMC * kG * kRT);
    BL_CUDA(allow_opt_in_smem(k_basis_gemm<ROWS>, p->device));
    dim3 grid((p->Rn + kRT - 1) / kRT, p->X);
    for (int e0 = 0; e0 < p->L; e0 += kG) {
        k_basis_gemm<ROWS><<<grid, kThreads, smem, s>>>(A, kq, p->Nk, p->N, ell, p->real_ell ? 1 : 0, p->L, e0,
                                                        p->d_chi, R,
                                                        p->Rn, p->Q, p->T64);
        BL_CUDA(cudaGetLastError());
    }
    return BLAST_OK;
}

}  // namespace

int launch_basis(blast_plan *p, cudaStream_t s)
{
    const int rows3 = 3 * p->N;
    if (rows3 > 32 * 12) return BLAST_EINVAL;  // n_cheb <= 128 (ROWS <= 12)
    double *kq = nullptr, *wq = nullptr, *A = nullptr, *R = nullptr;
    double *ell = nullptr;
    int rc = BLAST_OK;
    size_t nA = (size_t)p->Nk * rows3;
    if (cudaMalloc(&kq, sizeof(double) * p->Nk) || cudaMalloc(&wq, sizeof(double) * p->Nk) ||
        cudaMalloc(&A, sizeof(double) * nA) || cudaMalloc(&R, sizeof(double) * p->Rn) ||
        cudaMalloc(&ell, sizeof(double) * p->L)) {
        cudaGetLastError();
        rc = BLAST_ENOMEM;
    }
    if (!rc && (cudaMemcpyAsync(kq, p->kq.data(), sizeof(double) * p->Nk, cudaMemcpyHostToDevice, s) ||
                cudaMemcpyAsync(wq, p->wq.data(), sizeof(double) * p->Nk, cudaMemcpyHostToDevice, s) ||
                cudaMemcpyAsync(R, p->R.data(), sizeof(double) * p->Rn, cudaMemcpyHostToDevice, s) ||
                cudaMemcpyAsync(ell, p->ell.data(), sizeof(double) * p->L, cudaMemcpyHostToDevice, s)))
        rc = BLAST_EDEVICE;
    if (!rc) {
        k_basis_A<<<(p->Nk + 255) / 256, 256, 0, s>>>(kq, wq, p->Nk, p->N, p->kmap, p->k_min, p->k_max, A);
        if (cudaGetLastError() != cudaSuccess) rc = BLAST_EDEVICE;
    }
    if (!rc) {
        int rows = (rows3 + 31) / 32;
        if (rows <= 3) rc = launch_gemm_rows<3>(p, A, kq, ell, R, s);
        else if (rows <= 6) rc = launch_gemm_rows<6>(p, A, kq, ell, R, s);
        else if (rows <= 9) rc = launch_gemm_rows<9>(p, A, kq, ell, R, s);
        else rc = launch_gemm_rows<12>(p, A, kq, ell, R, s);
    }
    cudaStreamSynchronize(s);
    cudaFree(kq); cudaFree(wq); cudaFree(A); cudaFree(R); cudaFree(ell);
    if (!rc && cudaGetLastError() != cudaSuccess) rc = BLAST_EDEVICE;
    return rc;
}

int launch_basis_convert(blast_plan *p, unsigned mask, cudaStream_t s)
{
    size_t n = (size_t)3 * p->L * p->N * p->Q;
    if ((mask & BLAST_BASIS_FP32) && p->T32) {
        k_basis_to_f32<<<152 * 8, 256, 0, s>>>(p->T64, p->T32, n);
        BL_CUDA(cudaGetLastError());
        p->have32 = true;
    }
    if ((mask & BLAST_BASIS_BF16S) && p->Tsl) {
        int rc = launch_basis_slices(p, s);
        if (rc) return rc;
        p->havebf = true;
    }
    return BLAST_OK;
}
