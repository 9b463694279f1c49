// Per-cosmology evaluation (steps a0, a, b of the hot path):
//   (a0) Chebyshev coefficients a_n of P(k): natural cubic spline of
//        (ln k, ln P) solved by parallel cyclic reduction, P at the N
//        Chebyshev k-nodes (Eq. chebpoints), discrete cosine transform (the
//        transform Eq. dft stands for);
//   (a)  w^{AB}_l(a, r) = sum_n a_n T~^{AB}_{n;l}(a, r)                (Eq. pmd)
//   (b)  Y^{AB}_l(a, j)  = sum_r V_j(a, r) w^{AB}_l(a, r),
//        V_j(a, r) = wR_r D(R_r chi_a) K^B_j(R_r chi_a)
//        C^{AB}_ij(l)   = N_AB(l) sum_a U_i(a) Y^{AB}_l(a, j),
//        U_i(a) = wchi_a chi_a D(chi_a) K^A_i(chi_a)              (Eq. final_cls)
// with c_n(chi1, chi2) = D(chi1) D(chi2) a_n folded into U and V.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "blast_internal.h"

namespace {

constexpr int kFitThreads = 256;
constexpr int kMaxPtab = 1024;

__device__ __forceinline__ int npairs_dev(int ng, int ns)
{
    return ng * (ng + 1) / 2 + ng * ns + ns * (ns + 1) / 2;
}

// Pair p of a (ng, ns) tracer set -> type t (0 gg, 1 gs, 2 ss), A-side tracer
// row i and B-side tracer row j (both as rows of the request's kernel arrays).
__device__ __forceinline__ void pair_decode(int p, int ng, int ns, int &t, int &ia, int &jb, int &jloc)
{
    int ngg = ng * (ng + 1) / 2, ngs = ng * ns;
    if (p < ngg) {
        int i = 0, rem = p;
        while (rem >= ng - i) { rem -= ng - i; i++; }
        t = 0; ia = i; jloc = i + rem; jb = jloc;
    } else if (p < ngg + ngs) {
        int q = p - ngg;
        t = 1; ia = q / ns; jloc = q % ns; jb = ng + jloc;
    } else {
        int i = 0, rem = p - ngg - ngs;
        while (rem >= ns - i) { rem -= ns - i; i++; }
        t = 2; ia = ng + i; jloc = i + rem; jb = ng + jloc;
    }
}

// ---------------------------------------------------------------------------
// (a0) Chebyshev fit, one CTA per request.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kFitThreads)
k_fit(ReqDev *reqs, int N, const double *__restrict__ node_u, const double *__restrict__ cos_tab)
{
    ReqDev &rq = reqs[blockIdx.x];
    const int n = rq.n_ptab;
    extern __shared__ double sh[];
    double *u = sh, *v = u + n;
    double *A0 = v + n, *B0 = A0 + n, *C0 = B0 + n, *D0 = C0 + n;
    double *A1 = D0 + n, *B1 = A1 + n, *C1 = B1 + n, *D1 = C1 + n;
    double *Pn = D1 + n;  // [N]
    __shared__ int bad;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
        double k = rq.k_tab[i], P = rq.p_tab[i];
        if (!(k > 0.0) || !(P > 0.0) || isinf(P) || isinf(k)) bad = 1;
        u[i] = log(k);
        v[i] = log(P);
    }
    __syncthreads();
    for (int i = tid + 1; i < n; i += blockDim.x)
        if (!(u[i] > u[i - 1])) bad = 1;
    // tridiagonal system for the spline second derivatives M_i, M_0 = M_{n-1} = 0
    for (int i = tid; i < n; i += blockDim.x) {
        if (i == 0 || i == n - 1) { A0[i] = 0.0; B0[i] = 1.0; C0[i] = 0.0; D0[i] = 0.0; continue; }
        double hl = u[i] - u[i - 1], hr = u[i + 1] - u[i];
        A0[i] = hl; B0[i] = 2.0 * (hl + hr); C0[i] = hr;
        D0[i] = 6.0 * ((v[i + 1] - v[i]) / hr - (v[i] - v[i - 1]) / hl);
    }
    __syncthreads();
    // parallel cyclic reduction: after ceil(log2 n) sweeps every row is decoupled
    double *a = A0, *b = B0, *c = C0, *d = D0, *a2 = A1, *b2 = B1, *c2 = C1, *d2 = D1;
    for (int s = 1; s < n; s <<= 1) {
        for (int i = tid; i < n; i += blockDim.x) {
            int im = i - s, ip = i + s;
            double al = (im >= 0) ? -a[i] / b[im] : 0.0;
            double ga = (ip < n) ? -c[i] / b[ip] : 0.0;
            a2[i] = (im >= 0) ? al * a[im] : 0.0;
            c2[i] = (ip < n) ? ga * c[ip] : 0.0;
            b2[i] = b[i] + ((im >= 0) ? al * c[im] : 0.0) + ((ip < n) ? ga * a[ip] : 0.0);
            d2[i] = d[i] + ((im >= 0) ? al * d[im] : 0.0) + ((ip < n) ? ga * d[ip] : 0.0);
        }
        __syncthreads();
        double *t;
        t = a; a = a2; a2 = t; t = b; b = b2; b2 = t; t = c; c = c2; c2 = t; t = d; d = d2; d2 = t;
    }
    double *M = a2;  // reuse a free buffer
    for (int i = tid; i < n; i += blockDim.x) {
        M[i] = d[i] / b[i];
        if (rq.spM) rq.spM[i] = M[i];  // kept for the Limber terms
    }
    __syncthreads();
    // spline at the Chebyshev nodes, then exp
    for (int j = tid; j < N; j += blockDim.x) {
        double x = node_u[j];
        if (!(x >= u[0] && x <= u[n - 1])) { bad = 1; Pn[j] = 0.0; continue; }
        int lo = 0, hi = n - 1;
        while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (u[mid] <= x) lo = mid; else hi = mid; }
        double h = u[hi] - u[lo], t = (x - u[lo]) / h, s1 = 1.0 - t;
        double val = s1 * v[lo] + t * v[hi] + h * h / 6.0 * ((s1 * s1 * s1 - s1) * M[lo] + (t * t * t - t) * M[hi]);
        Pn[j] = exp(val);
    }
    __syncthreads();
    // a_n = (c_n / N) sum_j P_j cos(n (2j+1) pi / 2N), c_0 = 1, c_n = 2
    for (int nn = tid; nn < N; nn += blockDim.x) {
        double acc = 0.0;
        int idx = nn, step = 2 * nn, mod = 4 * N;
        for (int j = 0; j < N; j++) {
            acc = fma(Pn[j], cos_tab[idx], acc);
            idx += step;
            if (idx >= mod) idx -= mod;
        }
        double an = (nn == 0 ? 1.0 : 2.0) * acc / (double)N;
        if (bad) an = nan("");
        rq.a64[nn] = an;
        rq.a32[nn] = (float)an;
    }
    if (tid == 0 && bad) rq.status = BLAST_EINVAL;
}

// ---------------------------------------------------------------------------
// Quadrature weights with the growth factor folded in:
//   U[tr][a] = wchi_a chi_a D(chi_a) K_tr(chi_a)
//   V[tr][q] = wR_r D(R_r chi_a) K_tr(R_r chi_a),   q = a n_R + r
// ---------------------------------------------------------------------------
__global__ void k_weights(ReqDev *reqs, int X, int Rn, const double *__restrict__ chi,
                          const double *__restrict__ wchi, const double *__restrict__ wR, int want32, int want_v64)
{
    ReqDev &rq = reqs[blockIdx.y];
    const int ntr = rq.n_clust + rq.n_lens, Q = X * Rn;
    // one thread per chi-R node: its growth factor is read once for every tracer,
    // and each group of tracer values is loaded before any is stored (inputs may
    // be host memory read over the host link, where latency dominates)
    constexpr int kG = 8;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
        const double g = wR[q % Rn] * rq.growth_Rchi[q];
        for (int t0 = 0; t0 < ntr; t0 += kG) {
            double k[kG];
#pragma unroll
            for (int u = 0; u < kG; u++) k[u] = (t0 + u < ntr) ? rq.kern_Rchi[(size_t)(t0 + u) * Q + q] : 0.0;
#pragma unroll
            for (int u = 0; u < kG; u++) {
                if (t0 + u >= ntr) break;
                const size_t i = (size_t)(t0 + u) * Q + q;
                const double vv = g * k[u];
                if (want_v64) rq.V64[i] = vv;
                if (want32) rq.V32[i] = (float)vv;
            }
        }
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ntr * X; i += gridDim.x * blockDim.x) {
        int a = i % X;
        double uu = wchi[a] * chi[a] * rq.growth_chi[a] * rq.kern_chi[i];
        rq.U64[i] = uu;
        if (want32) rq.U32[i] = (float)uu;
    }
}

// ---------------------------------------------------------------------------
// (a) + first half of (b) on CUDA cores.  One CTA per (request, chi node a,
// type t and selected ell); each thread owns R nodes r = tid, tid + blockDim...
//   w = sum_n a_n T[t][e][n][a n_R + r],  Y[j] = sum_r V_j(a, r) w
// reduced over r with warp shuffles, written to Y[b][t][es][a][j].
// ---------------------------------------------------------------------------
template <class T> struct Prec;
template <> struct Prec<double> { static __device__ const double *a(const ReqDev &r) { return r.a64; }
                                  static __device__ const double *V(const ReqDev &r) { return r.V64; } };
template <> struct Prec<float> { static __device__ const float *a(const ReqDev &r) { return r.a32; }
                                 static __device__ const float *V(const ReqDev &r) { return r.V32; } };

// SYM (the symmetrised form of App. A): the gs list holds both kinds, so that
// the reduction can add K^B_j(chi) sum_r V^A_i w to K^A_i(chi) sum_r V^B_j w.
template <class T, bool SYM>
__global__ void __launch_bounds__(128)
k_contract(const ReqDev *__restrict__ reqs, const T *__restrict__ basis, int L, int N, int X, int Rn,
           const int *__restrict__ esel, int n_esel, int MT, T *__restrict__ Y)
{
    constexpr int MJ = SYM ? BLAST_MAX_TRACERS : BLAST_MAX_TRACERS / 2;  // tracers of one list
    extern __shared__ unsigned char smraw[];
    T *as = reinterpret_cast<T *>(smraw);  // [N]
    __shared__ T red[4][BLAST_MAX_TRACERS];
    const int b = blockIdx.x, a = blockIdx.y;
    const int t = blockIdx.z / n_esel, es = blockIdx.z % n_esel;
    const int e = esel[es];
    const ReqDev &rq = reqs[b];
    const int ng = rq.n_clust, ns = rq.n_lens;
    const int nB = (t == 0) ? ng : (SYM && t == 1) ? ng + ns : ns, offB = (t == 0 || (SYM && t == 1)) ? 0 : ng;
    const T *acoef = Prec<T>::a(rq);
    for (int n = threadIdx.x; n < N; n += blockDim.x) as[n] = acoef[n];
    __syncthreads();
    const int Q = X * Rn;
    const T *Tb = basis + ((size_t)t * L + e) * N * Q + (size_t)a * Rn;
    const T *V = Prec<T>::V(rq) + (size_t)offB * Q + (size_t)a * Rn;
    T part[MJ];
#pragma unroll
    for (int j = 0; j < MJ; j++) part[j] = 0;
    for (int r = threadIdx.x; r < Rn; r += blockDim.x) {
        T w = 0;
        for (int n = 0; n < N; n++) w = fma(as[n], Tb[(size_t)n * Q + r], w);
#pragma unroll
        for (int j = 0; j < MJ; j++)
            if (j < nB) part[j] = fma(V[(size_t)j * Q + r], w, part[j]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < MJ; j++) {
        if (j >= nB) break;
        T v = part[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < nB) {
        T s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w][threadIdx.x];
        Y[((((size_t)b * 3 + t) * n_esel + es) * X + a) * MT + threadIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// Second half of (b): C_ij(l) = N_AB(l) sum_a U_i(a) Y[t][es][a][j], summed in
// FP64, scattered to the request's output columns.
// ---------------------------------------------------------------------------
// sym: C_ij also gets N_AB(l) sum_a U_j(a) Y[t][es][a][i] (both kernel orders
// of the symmetrised form, App. A); list positions are tracer rows minus the
// list's first row.
template <class T>
__global__ void k_reduce(const ReqDev *__restrict__ reqs, const T *__restrict__ Y, int X, int L,
                         const int *__restrict__ esel, int n_esel, int MT, const double *__restrict__ pref, int sym)
{
    const int b = blockIdx.y;
    const ReqDev &rq = reqs[b];
    const int ng = rq.n_clust, ns = rq.n_lens, P = npairs_dev(ng, ns);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < P * n_esel; idx += gridDim.x * blockDim.x) {
        const int p = idx / n_esel, es = idx % n_esel, e = esel[es];
        const int col = rq.e_out[e];
        if (col < 0) continue;
        int t, ia, jb, jloc;
        pair_decode(p, ng, ns, t, ia, jb, jloc);
        const double *U = rq.U64 + (size_t)ia * X;
        const int first = (t == 0 || (sym && t == 1)) ? 0 : ng;  // first tracer row of the type's list
        const T *Yb = Y + (((size_t)b * 3 + t) * n_esel + es) * (size_t)X * MT;
        const T *Yp = Yb + (jb - first);
        double s = 0.0;
        for (int a = 0; a < X; a++) s = fma(U[a], (double)Yp[(size_t)a * MT], s);
        if (sym) {
            const double *Uj = rq.U64 + (size_t)jb * X;
            const T *Yi = Yb + (ia - first);
            for (int a = 0; a < X; a++) s = fma(Uj[a], (double)Yi[(size_t)a * MT], s);
        }
        double out = pref[t * L + e] * s;
        if (rq.status) out = nan("");
        rq.cl[(size_t)p * rq.n_sel + col] = out;
    }
}

}  // namespace

int preload_fp64_kernels()
{
    cudaFuncAttributes fa;
    BL_CUDA(cudaFuncGetAttributes(&fa, k_fit));
    BL_CUDA(cudaFuncGetAttributes(&fa, k_weights));
    BL_CUDA(cudaFuncGetAttributes(&fa, k_contract<double, false>));
    BL_CUDA(cudaFuncGetAttributes(&fa, k_contract<double, true>));
    BL_CUDA(cudaFuncGetAttributes(&fa, k_reduce<double>));
    return BLAST_OK;
}

int launch_fit(blast_plan *p, ReqDev *dreq, int nreq, cudaStream_t s)
{
    size_t smem = sizeof(double) * (10 * kMaxPtab + p->N);
    BL_CUDA(allow_opt_in_smem(k_fit, p->device));
    k_fit<<<nreq, kFitThreads, smem, s>>>(dreq, p->N, p->d_kcheb_u, p->d_cos_tab);
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}

int launch_weights(blast_plan *p, ReqDev *dreq, int nreq, int want32, cudaStream_t s, int want_v64)
{
    dim3 grid((p->Q + 255) / 256 < 1024 ? (p->Q + 255) / 256 : 1024, nreq);
    k_weights<<<grid, 256, 0, s>>>(dreq, p->X, p->Rn, p->d_chi, p->d_wchi, p->d_wR, want32, want_v64);
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}

int launch_contract(blast_plan *p, ReqDev *dreq, int nreq, int prec, const int *d_esel, int n_esel,
                    void *ypart, cudaStream_t s)
{
    dim3 grid(nreq, p->X, 3 * n_esel);
    const size_t sm64 = sizeof(double) * p->N, sm32 = sizeof(float) * p->N;
    if (prec == BLAST_FP64) {
        if (p->r_form == 1)
            k_contract<double, true><<<grid, 128, sm64, s>>>(dreq, p->T64, p->L, p->N, p->X, p->Rn, d_esel, n_esel,
                                                             p->max_tr, (double *)ypart);
        else
            k_contract<double, false><<<grid, 128, sm64, s>>>(dreq, p->T64, p->L, p->N, p->X, p->Rn, d_esel, n_esel,
                                                              p->max_tr, (double *)ypart);
    } else {
        if (p->r_form == 1)
            k_contract<float, true><<<grid, 128, sm32, s>>>(dreq, p->T32, p->L, p->N, p->X, p->Rn, d_esel, n_esel,
                                                            p->max_tr, (float *)ypart);
        else
            k_contract<float, false><<<grid, 128, sm32, s>>>(dreq, p->T32, p->L, p->N, p->X, p->Rn, d_esel, n_esel,
                                                             p->max_tr, (float *)ypart);
    }
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}

int launch_reduce(blast_plan *p, ReqDev *dreq, int nreq, int prec, const int *d_esel, int n_esel,
                  const void *ypart, cudaStream_t s)
{
    int pmax = blast_npairs(p->max_clust, p->max_lens);
    dim3 grid((pmax * n_esel + 127) / 128, nreq);
    if (prec == BLAST_FP64)
        k_reduce<double><<<grid, 128, 0, s>>>(dreq, (const double *)ypart, p->X, p->L, d_esel, n_esel, p->max_tr,
                                              p->d_pref, p->r_form);
    else
        k_reduce<float><<<grid, 128, 0, s>>>(dreq, (const float *)ypart, p->X, p->L, d_esel, n_esel, p->max_tr,
                                             p->d_pref, p->r_form);
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}

// ===========================================================================
// Host entry points
// ===========================================================================
namespace {

int validate_request(const blast_plan *p, const blast_request *r)
{
    if (!r) return BLAST_EINVAL;
    if (r->n_clust < 0 || r->n_lens < 0 || r->n_clust + r->n_lens < 1) return BLAST_EINVAL;
    if (r->n_clust > p->max_clust || r->n_lens > p->max_lens) return BLAST_EINVAL;
    if (!r->kern_chi || !r->kern_Rchi || !r->growth_chi || !r->growth_Rchi || !r->k_tab || !r->p_tab)
        return BLAST_EINVAL;
    if (r->n_ptab < 3 || r->n_ptab > kMaxPtab) return BLAST_EINVAL;
    if (r->mem_space != 0 && r->mem_space != 1) return BLAST_EINVAL;
    if (p->L < 64 && (r->ell_mask_lo >> p->L)) return BLAST_EINVAL;
    if (p->L <= 64 && r->ell_mask_hi) return BLAST_EINVAL;
    if (p->L > 64 && p->L < 128 && (r->ell_mask_hi >> (p->L - 64))) return BLAST_EINVAL;
    if (r->mem_space == 0) {
        // host inputs: the P table must bracket every Chebyshev node
        const double *k = r->k_tab, *P = r->p_tab;
        for (int i = 0; i < r->n_ptab; i++) {
            if (!(k[i] > 0) || !(P[i] > 0) || std::isinf(P[i])) return BLAST_EINVAL;
            if (i && !(k[i] > k[i - 1])) return BLAST_EINVAL;
        }
        for (int j = 0; j < p->N; j++)
            if (!(p->kcheb[j] >= k[0] && p->kcheb[j] <= k[r->n_ptab - 1])) return BLAST_EINVAL;
    }
    return BLAST_OK;
}

bool ell_selected(const blast_request *r, int e)
{
    if (!r->ell_mask_lo && !r->ell_mask_hi) return true;
    return e < 64 ? ((r->ell_mask_lo >> e) & 1) : ((r->ell_mask_hi >> (e - 64)) & 1);
}

}  // namespace

int request_check(const blast_plan *p, const blast_request *r) { return validate_request(p, r); }

int request_n_sel(const blast_plan *p, const blast_request *r)
{
    int nsel = 0;
    for (int e = 0; e < p->L; e++) nsel += ell_selected(r, e);
    return nsel;
}

size_t request_in_doubles(const blast_plan *p, int ntr, int nptab)
{
    return (size_t)ntr * (p->X + p->Q) + p->X + p->Q + 2 * (size_t)nptab;
}

extern "C" size_t blast_request_footprint(const blast_plan *p, const blast_request *r)
{
    if (!p || !r) return 0;
    int ntr = r->n_clust + r->n_lens;
    int nsel = 0;
    for (int e = 0; e < p->L; e++) nsel += ell_selected(r, e);
    size_t in = request_in_doubles(p, ntr, r->n_ptab) * 8;
    size_t coef = (size_t)p->N * (8 + 4 + 4);
    size_t wts = (size_t)ntr * (p->X + p->Q) * 12;
    size_t y = (size_t)3 * p->L * p->X * p->max_tr * 8;
    size_t out = (size_t)blast_npairs(r->n_clust, r->n_lens) * nsel * 8;
    return in + coef + wts + y + out + sizeof(ReqDev);
}

// Stage requests, build device descriptors, and run fit + weights.  Shared by
// the CUDA-core and tensor-core paths.  On success *d_esel / *n_esel hold the
// union of the requests' ell selections.
// Device address through which kernels may read or write host memory in place,
// or nullptr: pinned mapped memory, or (when the GPU uses the host's page
// tables, pageable != 0) any host address.
static const void *device_view(const void *hp, int pageable)
{
    // a GPU that walks the host page tables reads any host address as it is:
    // no query (one per array costs about half a microsecond of host time)
    if (pageable) return hp;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, hp) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type == cudaMemoryTypeHost && at.devicePointer) return at.devicePointer;
    if (at.type == cudaMemoryTypeUnregistered && pageable) return hp;
    return nullptr;
}

// The fit (a0) and the quadrature weights of a staged batch: the fit
// (latency bound) runs on the plan's side stream beside the weights kernel
// (HBM bound); both read the staged descriptors, nothing else is shared.
int launch_prep(blast_plan *p, ReqDev *dreq, int n, int prec, cudaStream_t s)
{
    int rc;
    BL_CUDA(cudaEventRecord(p->ev_fork, s));
    BL_CUDA(cudaStreamWaitEvent(p->aux, p->ev_fork, 0));
    if ((rc = prof_launch(p, BLAST_K_FIT, p->aux, [&] { return launch_fit(p, dreq, n, p->aux); }))) return rc;
    BL_CUDA(cudaEventRecord(p->ev_join, p->aux));
    if ((rc = prof_launch(p, BLAST_K_WEIGHTS, s, [&] {
             return launch_weights(p, dreq, n, prec != BLAST_FP64, s, prec == BLAST_FP64);
         })))
        return rc;
    BL_CUDA(cudaStreamWaitEvent(s, p->ev_join, 0));
    return BLAST_OK;
}

// Steps (a) and (b) of a staged and prepared batch in the plan's work space.
int launch_cl_kernels(blast_plan *p, ReqDev *dreq, int n, int prec, const int *d_esel, int n_esel, cudaStream_t s)
{
    int rc;
    if (prec == BLAST_BF16S) {
        const size_t ybytes = tc_y_bytes(p, n, n_esel);
        if ((rc = p->ws.ypart.ensure(ybytes))) return rc;
        if ((rc = prof_launch(p, BLAST_K_CONTRACT_TC, s, [&] {
                 return launch_contract_tc(p, dreq, n, d_esel, n_esel, p->ws.ypart.p, s);
             })))
            return rc;
        return prof_launch(p, BLAST_K_REDUCE, s, [&] {
            return launch_reduce_tc(p, dreq, n, d_esel, n_esel, p->ws.ypart.p, s);
        });
    }
    const size_t ybytes = (size_t)n * 3 * n_esel * p->X * p->max_tr * (prec == BLAST_FP64 ? 8 : 4);
    if ((rc = p->ws.ypart.ensure(ybytes))) return rc;
    if ((rc = prof_launch(p, BLAST_K_CONTRACT, s, [&] {
             return launch_contract(p, dreq, n, prec, d_esel, n_esel, p->ws.ypart.p, s);
         })))
        return rc;
    return prof_launch(p, BLAST_K_REDUCE, s, [&] {
        return launch_reduce(p, dreq, n, prec, d_esel, n_esel, p->ws.ypart.p, s);
    });
}

int stage_batch(blast_plan *p, int n, const blast_request *reqs, int prec, double *const *outs,
                int out_mem_space, cudaStream_t s, ReqDev **dreq_out, int **d_esel, int *n_esel,
                std::vector<ReqDev> &hreq, std::vector<char> &direct_out, const double *const *pnl, bool prep)
{
    Workspace &ws = p->ws;
    int pageable = 0;
    cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccessUsesHostPageTables, p->device);
    direct_out.assign(n, 0);
    const int ntr_max = p->max_clust + p->max_lens;
    // ell union
    std::vector<int> esel;
    for (int e = 0; e < p->L; e++) {
        bool any = false;
        for (int i = 0; i < n && !any; i++) any = ell_selected(&reqs[i], e);
        if (any) esel.push_back(e);
    }
    *n_esel = (int)esel.size();
    // sizes
    // every per-request stride is a multiple of 256 bytes so that each
    // request's double / float arrays stay aligned
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t in_per = al(request_in_doubles(p, ntr_max, kMaxPtab) * 8) / 8;
    // coefficients (FP64, FP32) and the spline second derivatives the Limber terms use
    size_t coef_per = al((size_t)p->N * 8) + al((size_t)p->N * 4) + al((size_t)kMaxPtab * 8);
    const size_t nl_per = al((size_t)p->L * p->X * 8);  // staged non-linear tables (host requests)
    size_t u64 = al((size_t)ntr_max * p->X * 8), v64 = al((size_t)ntr_max * p->Q * 8);
    size_t u32 = al((size_t)ntr_max * p->X * 4), v32 = al((size_t)ntr_max * p->Q * 4);
    size_t wts_per = u64 + v64 + u32 + v32;
    int pmax = blast_npairs(p->max_clust, p->max_lens);
    size_t cl_per = al((size_t)pmax * p->L * 8) / 8;
    int any_host_in = 0;
    for (int i = 0; i < n; i++) any_host_in |= (reqs[i].mem_space == 0);
    int rc;
    if (any_host_in && (rc = ws.in.ensure(in_per * 8 * n))) return rc;
    if ((rc = ws.coef.ensure(coef_per * n)) || (rc = ws.wts.ensure(wts_per * n)) ||
        (rc = ws.meta.ensure(sizeof(ReqDev) * n + sizeof(int) * BLAST_MAX_ELL)))
        return rc;
    if (out_mem_space == 0 && (rc = ws.cl.ensure(cl_per * 8 * n))) return rc;
    if (pnl && any_host_in && (rc = ws.nl.ensure(nl_per * n))) return rc;

    hreq.resize(n);
    char *coef = ws.coef.as<char>(), *wts = ws.wts.as<char>();
    for (int i = 0; i < n; i++) {
        const blast_request &r = reqs[i];
        ReqDev &h = hreq[i];
        memset(&h, 0, sizeof h);
        const int ntr = r.n_clust + r.n_lens;
        h.n_clust = r.n_clust; h.n_lens = r.n_lens; h.n_ptab = r.n_ptab; h.status = 0;
        const double *hv[6] = {r.kern_chi, r.kern_Rchi, r.growth_chi, r.growth_Rchi, r.k_tab, r.p_tab};
        const double *dv[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        // in-place reads only when the call waits for the stream before it
        // returns (host outputs), so host inputs are still read only during the call
        bool direct = (r.mem_space == 0 && out_mem_space == 0);
        for (int k = 0; direct && k < 6; k++) direct = (dv[k] = (const double *)device_view(hv[k], pageable)) != nullptr;
        if (r.mem_space == 1) {
            h.kern_chi = r.kern_chi; h.kern_Rchi = r.kern_Rchi; h.growth_chi = r.growth_chi;
            h.growth_Rchi = r.growth_Rchi; h.k_tab = r.k_tab; h.p_tab = r.p_tab;
        } else if (direct) {
            // host arrays the device can read in place (pinned and mapped, or any
            // host memory on a system whose GPU uses the host page tables): the
            // kernels stream them over the host link, no staging copies
            h.kern_chi = dv[0]; h.kern_Rchi = dv[1]; h.growth_chi = dv[2];
            h.growth_Rchi = dv[3]; h.k_tab = dv[4]; h.p_tab = dv[5];
        } else {
            double *base = ws.in.as<double>() + in_per * i;
            double *kc = base, *kR = kc + (size_t)ntr * p->X, *gc = kR + (size_t)ntr * p->Q;
            double *gR = gc + p->X, *kt = gR + p->Q, *pt = kt + r.n_ptab;
            BL_CUDA(cudaMemcpyAsync(kc, r.kern_chi, sizeof(double) * ntr * p->X, cudaMemcpyHostToDevice, s));
            BL_CUDA(cudaMemcpyAsync(kR, r.kern_Rchi, sizeof(double) * ntr * p->Q, cudaMemcpyHostToDevice, s));
            BL_CUDA(cudaMemcpyAsync(gc, r.growth_chi, sizeof(double) * p->X, cudaMemcpyHostToDevice, s));
            BL_CUDA(cudaMemcpyAsync(gR, r.growth_Rchi, sizeof(double) * p->Q, cudaMemcpyHostToDevice, s));
            BL_CUDA(cudaMemcpyAsync(kt, r.k_tab, sizeof(double) * r.n_ptab, cudaMemcpyHostToDevice, s));
            BL_CUDA(cudaMemcpyAsync(pt, r.p_tab, sizeof(double) * r.n_ptab, cudaMemcpyHostToDevice, s));
            h.kern_chi = kc; h.kern_Rchi = kR; h.growth_chi = gc; h.growth_Rchi = gR; h.k_tab = kt; h.p_tab = pt;
        }
        char *c = coef + coef_per * i;
        h.a64 = (double *)c;
        h.a32 = (float *)(c + al((size_t)p->N * 8));
        h.spM = (double *)(c + al((size_t)p->N * 8) + al((size_t)p->N * 4));
        if (pnl && pnl[i]) {
            if (r.mem_space == 1) h.pnl = pnl[i];
            else {
                double *dst = (double *)(ws.nl.as<char>() + nl_per * i);
                BL_CUDA(cudaMemcpyAsync(dst, pnl[i], sizeof(double) * p->L * p->X, cudaMemcpyHostToDevice, s));
                h.pnl = dst;
            }
        }
        char *w = wts + wts_per * i;
        h.U64 = (double *)w;
        h.V64 = (double *)(w + u64);
        h.U32 = (float *)(w + u64 + v64);
        h.V32 = (float *)(w + u64 + v64 + u32);
        int col = 0;
        for (int e = 0; e < BLAST_MAX_ELL; e++) h.e_out[e] = -1;
        for (int e = 0; e < p->L; e++)
            if (ell_selected(&r, e)) h.e_out[e] = col++;
        h.n_sel = col;
        h.cl = (out_mem_space == 1) ? outs[i] : ws.cl.as<double>() + cl_per * i;
        if (out_mem_space == 0) {  // a device-writable host output is written in place
            double *o = (double *)device_view(outs[i], pageable);
            if (o) { h.cl = o; direct_out[i] = 1; }
        }
        const void *ptrs[] = {h.a64, h.a32, h.U64, h.V64, h.U32, h.V32, h.cl, h.kern_chi, h.kern_Rchi,
                              h.growth_chi, h.growth_Rchi, h.k_tab, h.p_tab};
        for (const void *q : ptrs)
            if (reinterpret_cast<uintptr_t>(q) % 8) return BLAST_EINVAL;  // every array is 8-byte aligned
    }
    ReqDev *dreq = ws.meta.as<ReqDev>();
    int *de = reinterpret_cast<int *>(dreq + n);
    BL_CUDA(cudaMemcpyAsync(dreq, hreq.data(), sizeof(ReqDev) * n, cudaMemcpyHostToDevice, s));
    BL_CUDA(cudaMemcpyAsync(de, esel.data(), sizeof(int) * esel.size(), cudaMemcpyHostToDevice, s));
    if (prep && (rc = launch_prep(p, dreq, n, prec, s))) return rc;
    *dreq_out = dreq;
    *d_esel = de;
    return BLAST_OK;
}

int plan_reserve(blast_plan *p, int nmax, size_t *bytes)
{
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const int ntr_max = p->max_clust + p->max_lens;
    const size_t coef_per = al((size_t)p->N * 8) + al((size_t)p->N * 4) + al((size_t)kMaxPtab * 8);
    const size_t wts_per = al((size_t)ntr_max * p->X * 8) + al((size_t)ntr_max * p->Q * 8) +
                           al((size_t)ntr_max * p->X * 4) + al((size_t)ntr_max * p->Q * 4);
    size_t y = (size_t)nmax * 3 * p->L * p->X * p->max_tr * 8;  // CUDA-core partials (FP64)
    if (tc_supported(p)) y = std::max(y, tc_y_bytes(p, nmax, p->L));
    int rc;
    BL_CUDA(cudaSetDevice(p->device));
    if ((rc = p->ws.coef.ensure(coef_per * nmax)) || (rc = p->ws.wts.ensure(wts_per * nmax)) ||
        (rc = p->ws.meta.ensure(sizeof(ReqDev) * nmax + sizeof(int) * BLAST_MAX_ELL)) ||
        (rc = p->ws.ypart.ensure(y)) || (tc_supported(p) && (rc = tc_reserve(p, nmax))))
        return rc;
    if (bytes)
        *bytes = p->ws.coef.bytes + p->ws.wts.bytes + p->ws.meta.bytes + p->ws.ypart.bytes + p->ws.tc.bytes +
                 p->ws.in.bytes + p->ws.cl.bytes;
    return BLAST_OK;
}

int finish_batch(blast_plan *p, int n, const std::vector<ReqDev> &hreq, const std::vector<char> &direct_out,
                 double *const *outs, int out_mem_space, cudaStream_t s)
{
    if (out_mem_space == 1) return BLAST_OK;
    for (int i = 0; i < n; i++) {
        if (direct_out[i]) continue;  // written in place by the kernel
        size_t bytes = sizeof(double) * blast_npairs(hreq[i].n_clust, hreq[i].n_lens) * hreq[i].n_sel;
        BL_CUDA(cudaMemcpyAsync(outs[i], hreq[i].cl, bytes, cudaMemcpyDeviceToHost, s));
    }
    BL_CUDA(cudaStreamSynchronize(s));
    return BLAST_OK;
}

// One pass over a batch.  lmode 0: beyond-Limber C_l (steps a0, a, b);
// lmode 1: the Limber integral only (no basis), with each request's linear P
// or, when pnl[i] is set, its non-linear table; lmode 2: beyond-Limber C_l
// plus the non-linear correction C^Limber(P_delta) - C^Limber(P_lin).
static int cl_impl(blast_plan *p, int n, const blast_request *reqs, int prec, double *const *outs, int out_mem_space,
                   void *stream, const double *const *pnl, int lmode, int extended)
{
    if (!p || n < 1 || !reqs || !outs) return BLAST_EINVAL;
    if (prec < BLAST_FP64 || prec > BLAST_BF16S) return BLAST_EINVAL;
    if (out_mem_space != 0 && out_mem_space != 1) return BLAST_EINVAL;
    for (int i = 0; i < n; i++) {
        int rc = validate_request(p, &reqs[i]);
        if (rc) return rc;
        if (!outs[i]) return BLAST_EINVAL;
        if (pnl && pnl[i] && reinterpret_cast<uintptr_t>(pnl[i]) % 8) return BLAST_EINVAL;
    }
    if (extended && (lmode != 1 || p->X < 5 || (pnl && pnl[0]))) return BLAST_EINVAL;
    const bool use_tc = (prec == BLAST_BF16S) && lmode != 1;
    if (lmode != 1) {
        if (use_tc && !tc_supported(p)) return BLAST_EINVAL;
        if (prec == BLAST_FP64 && !p->have64) return BLAST_ENOBASIS;
        if (prec == BLAST_FP32 && !p->have32) return BLAST_ENOBASIS;
        if (use_tc && !p->havebf) return BLAST_ENOBASIS;
    }
    if (*p->h_err) {  // a bounded device wait of an earlier call gave up
        *p->h_err = 0;
        return BLAST_ETIMEOUT;
    }
    BL_CUDA(cudaSetDevice(p->device));
    cudaStream_t s = (cudaStream_t)stream;
    ReqDev *dreq = nullptr;
    int *d_esel = nullptr, n_esel = 0;
    std::vector<ReqDev> hreq;
    std::vector<char> direct_out;
    int rc = stage_batch(p, n, reqs, lmode == 1 ? BLAST_FP64 : prec, outs, out_mem_space, s, &dreq, &d_esel, &n_esel,
                         hreq, direct_out, pnl, true);
    if (rc) return rc;
    if (lmode == 1) {
        if ((rc = prof_launch(p, BLAST_K_REDUCE, s, [&] {
                 return launch_limber(p, dreq, n, d_esel, n_esel, (pnl && pnl[0]) ? 1 : 0, extended, s);
             })))
            return rc;
    } else if ((rc = launch_cl_kernels(p, dreq, n, prec, d_esel, n_esel, s))) {
        return rc;
    }
    if (lmode == 2 && (rc = prof_launch(p, BLAST_K_REDUCE, s, [&] {
                           return launch_limber(p, dreq, n, d_esel, n_esel, 2, 0, s);
                       })))
        return rc;
    rc = finish_batch(p, n, hreq, direct_out, outs, out_mem_space, s);
    if (!rc && out_mem_space == 0 && *p->h_err) {
        *p->h_err = 0;
        return BLAST_ETIMEOUT;
    }
    return rc;
}

extern "C" int blast_cl_batch(blast_plan *p, int n, const blast_request *reqs, int prec, double *const *outs,
                              int out_mem_space, void *stream)
{
    return cl_impl(p, n, reqs, prec, outs, out_mem_space, stream, nullptr, 0, 0);
}

extern "C" int blast_cl(blast_plan *p, const blast_request *req, int prec, double *cl_out, int out_mem_space,
                        void *stream)
{
    if (!req || !cl_out) return BLAST_EINVAL;
    double *outs[1] = {cl_out};
    return blast_cl_batch(p, 1, req, prec, outs, out_mem_space, stream);
}

extern "C" int blast_cl_nonsep(blast_plan *p, const blast_request *req, const double *p_nodes, double *cl_out,
                               int out_mem_space, void *stream)
{
    if (!p || !req || !p_nodes || !cl_out) return BLAST_EINVAL;
    if (out_mem_space != 0 && out_mem_space != 1) return BLAST_EINVAL;
    if (p->r_form != 0) return BLAST_EINVAL;  // per-node contraction of the split R form only
    int rc = validate_request(p, req);
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(p_nodes) % 8) return BLAST_EINVAL;
    if (!p->have64) return BLAST_ENOBASIS;
    if (*p->h_err) {
        *p->h_err = 0;
        return BLAST_ETIMEOUT;
    }
    BL_CUDA(cudaSetDevice(p->device));
    cudaStream_t s = (cudaStream_t)stream;
    ReqDev *dreq = nullptr;
    int *d_esel = nullptr, n_esel = 0;
    std::vector<ReqDev> hreq;
    std::vector<char> direct_out;
    double *outs[1] = {cl_out};
    if ((rc = stage_batch(p, 1, req, BLAST_FP64, outs, out_mem_space, s, &dreq, &d_esel, &n_esel, hreq, direct_out,
                          nullptr, true)))
        return rc;
    const size_t qn = (size_t)p->Q * p->N;
    if ((rc = p->ws.ns.ensure(2 * qn * sizeof(double)))) return rc;
    double *coef = p->ws.ns.as<double>();
    const double *Pq = p_nodes;
    if (req->mem_space == 0) {  // host samples: staged behind the coefficients
        BL_CUDA(cudaMemcpyAsync(coef + qn, p_nodes, qn * sizeof(double), cudaMemcpyHostToDevice, s));
        Pq = coef + qn;
    }
    if ((rc = prof_launch(p, BLAST_K_FIT, s, [&] { return launch_fit_nodes(p, Pq, coef, s); }))) return rc;
    if ((rc = p->ws.ypart.ensure((size_t)3 * n_esel * p->X * p->max_tr * sizeof(double)))) return rc;
    if ((rc = prof_launch(p, BLAST_K_CONTRACT, s, [&] {
             return launch_contract_ns(p, dreq, coef, d_esel, n_esel, p->ws.ypart.as<double>(), s);
         })))
        return rc;
    if ((rc = prof_launch(p, BLAST_K_REDUCE, s, [&] {
             return launch_reduce(p, dreq, 1, BLAST_FP64, d_esel, n_esel, p->ws.ypart.p, s);
         })))
        return rc;
    return finish_batch(p, 1, hreq, direct_out, outs, out_mem_space, s);
}

extern "C" int blast_test_trip_wait(blast_plan *p, int tile)
{
    if (!p || tile < -1) return BLAST_EINVAL;
    p->test_trip = tile;
    return BLAST_OK;
}

extern "C" int blast_limber_k(const blast_plan *p, double *k)
{
    if (!p || !k) return BLAST_EINVAL;
    for (int e = 0; e < p->L; e++)
        for (int a = 0; a < p->X; a++) k[(size_t)e * p->X + a] = (p->ell[e] + 0.5) / p->chi[a];
    return BLAST_OK;
}

extern "C" int blast_cl_limber(blast_plan *p, const blast_request *req, const double *p_nl, int extended,
                               double *cl_out, int out_mem_space, void *stream)
{
    if (!req || !cl_out || (extended != 0 && extended != 1)) return BLAST_EINVAL;
    double *outs[1] = {cl_out};
    const double *nl[1] = {p_nl};
    return cl_impl(p, 1, req, BLAST_FP64, outs, out_mem_space, stream, nl, 1, extended);
}

extern "C" int blast_cl_nonlinear(blast_plan *p, const blast_request *req, int prec, const double *p_nl,
                                  double *cl_out, int out_mem_space, void *stream)
{
    if (!req || !cl_out || !p_nl) return BLAST_EINVAL;
    double *outs[1] = {cl_out};
    const double *nl[1] = {p_nl};
    return cl_impl(p, 1, req, prec, outs, out_mem_space, stream, nl, 2, 0);
}

extern "C" int blast_profile_enable(blast_plan *p, int enable)
{
    if (!p) return BLAST_EINVAL;
    p->prof_on = enable != 0;
    return BLAST_OK;
}

extern "C" int blast_profile_read(blast_plan *p, int cls, double *total_ms, long long *launches)
{
    if (!p || cls < 0 || cls >= BLAST_K_CLASSES) return BLAST_EINVAL;
    BL_CUDA(cudaSetDevice(p->device));
    for (auto &ev : p->prof_ev[cls]) {
        float ms = 0.f;
        BL_CUDA(cudaEventSynchronize(ev.second));
        BL_CUDA(cudaEventElapsedTime(&ms, ev.first, ev.second));
        p->prof_ms[cls] += ms;
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    p->prof_ev[cls].clear();
    if (total_ms) *total_ms = p->prof_ms[cls];
    if (launches) *launches = p->launches[cls];
    return BLAST_OK;
}

extern "C" int blast_profile_reset(blast_plan *p)
{
    if (!p) return BLAST_EINVAL;
    for (int c = 0; c < BLAST_K_CLASSES; c++) {
        for (auto &ev : p->prof_ev[c]) {
            cudaEventSynchronize(ev.second);
            cudaEventDestroy(ev.first);
            cudaEventDestroy(ev.second);
        }
        p->prof_ev[c].clear();
        p->prof_ms[c] = 0.0;
        p->launches[c] = 0;
    }
    return BLAST_OK;
}
