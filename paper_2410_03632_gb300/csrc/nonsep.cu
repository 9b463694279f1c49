// Non-separable spectra (Eqs. cheb_pk and pmd with a general c_n(chi1, chi2)):
// the caller samples P(k_j, chi_a, R_r chi_a) at the N Chebyshev k-nodes of
// every chi-R node q = a n_R + r (scale-dependent growth, massive neutrinos),
// and per node
//   c_n(q)    = (c / N) sum_j P(k_j, q) cos(n (2j+1) pi / 2N),  c = 1 (n = 0), 2
//   w_l(t, q) = sum_n c_n(q) T~^t_{n;l}(q)
// replaces D(chi_a) D(R_r chi_a) sum_n a_n T~; the R sum and the chi sum are
// those of the separable FP64 path.  FP64 on CUDA cores: the coefficient table
// is as large as one ell of the basis per cosmology, so the contraction is a
// batched dot product over n bound by reading the basis.
#include "blast_internal.h"

namespace {

// Per-node Chebyshev coefficients, one thread per node q: c[n][q].
__global__ void k_fit_nodes(const double *__restrict__ Pq, int Q, int N, const double *__restrict__ cos_tab,
                            double *__restrict__ c)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
        const double *row = Pq + (size_t)q * N;
        for (int n = 0; n < N; n++) {
            double acc = 0.0;
            int idx = n;
            const int step = 2 * n, mod = 4 * N;
            for (int j = 0; j < N; j++) {
                acc = fma(row[j], cos_tab[idx], acc);
                idx += step;
                if (idx >= mod) idx -= mod;
            }
            c[(size_t)n * Q + q] = (n == 0 ? 1.0 : 2.0) * acc / (double)N;
        }
    }
}

// w = sum_n c[n][q] T[t][e][n][q] and Y[t][es][a][j] = sum_r V_j(a, r) w, one
// CTA per (chi node a, type t and selected ell) of one request; the R sum is
// reduced with warp shuffles (the layout of the separable path's partials).
__global__ void __launch_bounds__(128)
k_contract_ns(const ReqDev *__restrict__ rq, const double *__restrict__ c, const double *__restrict__ T, int L,
              int N, int X, int Rn, const int *__restrict__ esel, int n_esel, int MT, double *__restrict__ Y)
{
    __shared__ double red[4][BLAST_MAX_TRACERS];
    const int a = blockIdx.x;
    const int t = blockIdx.y / n_esel, es = blockIdx.y % n_esel;
    const int e = esel[es];
    const int ng = rq->n_clust, ns = rq->n_lens;
    const int nB = (t == 0) ? ng : ns, offB = (t == 0) ? 0 : ng;
    const int Q = X * Rn;
    const double *Tb = T + ((size_t)t * L + e) * N * Q + (size_t)a * Rn;
    const double *cb = c + (size_t)a * Rn;
    const double *V = rq->V64 + (size_t)offB * Q + (size_t)a * Rn;
    double part[BLAST_MAX_TRACERS / 2];
#pragma unroll
    for (int j = 0; j < BLAST_MAX_TRACERS / 2; j++) part[j] = 0.0;
    for (int r = threadIdx.x; r < Rn; r += blockDim.x) {
        double w = 0.0;
        for (int n = 0; n < N; n++) w = fma(cb[(size_t)n * Q + r], Tb[(size_t)n * Q + r], w);
#pragma unroll
        for (int j = 0; j < BLAST_MAX_TRACERS / 2; j++)
            if (j < nB) part[j] = fma(V[(size_t)j * Q + r], w, part[j]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < BLAST_MAX_TRACERS / 2; j++) {
        if (j >= nB) break;
        double v = part[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < nB) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w][threadIdx.x];
        Y[(((size_t)t * n_esel + es) * X + a) * MT + threadIdx.x] = s;
    }
}

}  // namespace

int launch_fit_nodes(blast_plan *p, const double *Pq, double *c, cudaStream_t s)
{
    const int Q = p->Q;
    k_fit_nodes<<<(Q + 127) / 128, 128, 0, s>>>(Pq, Q, p->N, p->d_cos_tab, c);
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}

int launch_contract_ns(blast_plan *p, const ReqDev *dreq, const double *c, const int *d_esel, int n_esel, double *Y,
                       cudaStream_t s)
{
    dim3 grid(p->X, 3 * n_esel);
    k_contract_ns<<<grid, 128, 0, s>>>(dreq, c, p->T64, p->L, p->N, p->X, p->Rn, d_esel, n_esel, p->max_tr, Y);
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}
