// Plan construction: host grids of Sec. 3.2 (Simpson in chi, first-kind
// Chebyshev points with Fejer-1 weights in R, Clenshaw-Curtis in k, Chebyshev
// nodes of Eq. chebpoints for the fit), device constant tables, and basis
// storage / persistence.
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <chrono>

#include "blast_internal.h"

static thread_local char g_err[512];

void blast_last_error(const char *file, int line, const char *msg)
{
    snprintf(g_err, sizeof g_err, "%s:%d: %s", file, line, msg);
    if (getenv("BLAST_VERBOSE")) fprintf(stderr, "[blast] %s\n", g_err);
}

double host_now()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int DevBuf::ensure(size_t nbytes)
{
    if (nbytes <= bytes && p) return BLAST_OK;
    release();
    if (nbytes == 0) return BLAST_OK;
    if (cudaMalloc(&p, nbytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        bytes = 0;
        return BLAST_ENOMEM;
    }
    bytes = nbytes;
    return BLAST_OK;
}

void DevBuf::release()
{
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

static const double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------------------
// Clenshaw-Curtis weights on [-1, 1] for the n+1 Chebyshev extrema
// x_m = cos(m pi / n), n a power of two, from the sum
//   w_m = (c_m / n) (1 - S_m),  S_m = sum_{j=1}^{n/2} b_j cos(2 pi j m / n) / (4 j^2 - 1)
// (c_0 = c_n = 1, else 2; b_{n/2} = 1, else 2).  S is the length-n DFT of a
// symmetric real sequence, evaluated with an iterative radix-2 FFT whose
// twiddles are computed directly (not by recurrence).
// ---------------------------------------------------------------------------
static void fft_inplace(std::vector<std::complex<double>> &a)
{
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; i++) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    std::vector<std::complex<double>> tw(n / 2);
    for (size_t k = 0; k < n / 2; k++) {
        double ang = -2.0 * kPi * (double)k / (double)n;
        tw[k] = std::complex<double>(cos(ang), sin(ang));
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        size_t step = n / len;
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; k++) {
                std::complex<double> u = a[i + k], v = a[i + k + len / 2] * tw[k * step];
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

static int cc_weights(int n, std::vector<double> &x, std::vector<double> &w)
{
    if (n < 2 || (n & (n - 1))) return BLAST_EINVAL;
    std::vector<std::complex<double>> v(n, 0.0);
    for (int j = 1; j <= n / 2; j++) {
        double d = (j == n / 2 ? 1.0 : 2.0) / (4.0 * (double)j * (double)j - 1.0);
        if (j == n / 2) v[j] += d;
        else { v[j] += 0.5 * d; v[n - j] += 0.5 * d; }
    }
    fft_inplace(v);
    x.assign(n + 1, 0.0);
    w.assign(n + 1, 0.0);
    for (int m = 0; m <= n; m++) {
        double S = v[m % n].real();
        double c = (m == 0 || m == n) ? 1.0 : 2.0;
        w[m] = c / n * (1.0 - S);
        x[m] = cos(kPi * (double)m / (double)n);
    }
    return BLAST_OK;
}

// Fejer's first rule: n first-kind Chebyshev points on [-1, 1] (increasing)
// and the weights integrating polynomials of degree < n exactly.
static void fejer1(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; i++) {
        double th = kPi * (double)(2 * (n - 1 - i) + 1) / (2.0 * n);
        double acc = 0.0;
        for (int j = n / 2; j >= 1; j--) acc += cos(2.0 * j * th) / ((2.0 * j - 1.0) * (2.0 * j + 1.0));
        x[i] = cos(th);
        w[i] = 2.0 / n * (1.0 - 2.0 * acc);
    }
}

static uint64_t fnv1a(const void *data, size_t n, uint64_t h = 1469598103934665603ull)
{
    const unsigned char *c = (const unsigned char *)data;
    for (size_t i = 0; i < n; i++) { h ^= c[i]; h *= 1099511628211ull; }
    return h;
}

static double map_x_to_k(int kmap, double x, double kmin, double kmax)
{
    if (kmap == 0) return 0.5 * (kmin + kmax) + 0.5 * (kmax - kmin) * x;
    double lo = log(kmin), hi = log(kmax);
    return exp(lo + 0.5 * (hi - lo) * (x + 1.0));
}

extern "C" int blast_npairs(int ng, int ns)
{
    if (ng < 0 || ns < 0) return 0;
    return ng * (ng + 1) / 2 + ng * ns + ns * (ns + 1) / 2;
}

extern "C" const char *blast_status_str(int s)
{
    switch (s) {
    case BLAST_OK: return "ok";
    case BLAST_EINVAL: return "invalid argument";
    case BLAST_ENOMEM: return "out of memory";
    case BLAST_ENOTREADY: return "not ready";
    case BLAST_ETIMEOUT: return "timed out";
    case BLAST_EDEVICE: return "CUDA error";
    case BLAST_ENOBASIS: return "basis not available";
    case BLAST_EBUSY: return "busy";
    default: return "unknown status";
    }
}

template <class T> static int dev_copy(T **dst, const std::vector<T> &src)
{
    if (cudaMalloc((void **)dst, sizeof(T) * src.size()) != cudaSuccess) { cudaGetLastError(); return BLAST_ENOMEM; }
    BL_CUDA(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return BLAST_OK;
}

static void plan_free_device(blast_plan *p)
{
    void *bufs[] = {p->d_chi, p->d_wchi, p->d_wR, p->d_kcheb_u, p->d_cos_tab, p->d_pref, p->d_env, p->d_ell,
                    p->T64, p->T32, p->Tsl, p->scT};
    for (void *b : bufs) if (b) cudaFree(b);
    p->d_chi = p->d_wchi = p->d_wR = p->d_kcheb_u = p->d_cos_tab = p->d_pref = p->d_env = nullptr;
    p->d_ell = nullptr;
    p->T64 = nullptr; p->T32 = nullptr; p->Tsl = nullptr; p->scT = nullptr;
    if (p->h_err) cudaFreeHost(p->h_err);
    p->h_err = p->d_err = nullptr;
    if (p->aux) cudaStreamDestroy(p->aux);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    p->aux = nullptr;
    p->ev_fork = p->ev_join = nullptr;
    p->ws.in.release(); p->ws.coef.release(); p->ws.wts.release();
    p->ws.ypart.release(); p->ws.cl.release(); p->ws.meta.release(); p->ws.tc.release(); p->ws.nl.release(); p->ws.ns.release();
}

extern "C" int blast_plan_create(const blast_plan_desc *d, blast_plan **out)
{
    if (!d || !out) return BLAST_EINVAL;
    *out = nullptr;
    if (d->n_ell < 1 || d->n_ell > BLAST_MAX_ELL || (!d->ell && !d->ell_real)) return BLAST_EINVAL;
    for (int e = 0; e < d->n_ell; e++) {
        const double l = d->ell_real ? d->ell_real[e] : (double)d->ell[e];
        if (!(l >= 2.0) || !(l <= 1e5)) return BLAST_EINVAL;
        if (e && !(l > (d->ell_real ? d->ell_real[e - 1] : (double)d->ell[e - 1]))) return BLAST_EINVAL;
    }
    if (d->n_chi < 4 || !(d->chi_min > 0) || !(d->chi_max > d->chi_min)) return BLAST_EINVAL;
    if (d->r_form != 0 && d->r_form != 1) return BLAST_EINVAL;
    if (d->n_R < 2 || d->n_R % 2 || d->n_R > 512) return BLAST_EINVAL;
    if (d->r_form == 0 && (!(d->R_min > 0) || !(d->R_min < 1.0) || !(d->R_max > 1.0))) return BLAST_EINVAL;
    if (d->n_cheb < 2 || d->n_cheb > 128 || !(d->k_min > 0) || !(d->k_max > d->k_min)) return BLAST_EINVAL;
    if (d->k_map < 0 || d->k_map > 1) return BLAST_EINVAL;
    int nq = d->n_kquad - 1;
    if (nq < 4 || (nq & (nq - 1)) || nq > (1 << 22)) return BLAST_EINVAL;
    if (d->max_clust < 0 || d->max_lens < 0 || d->max_clust + d->max_lens < 1 ||
        d->max_clust > BLAST_MAX_TRACERS / 2 || d->max_lens > BLAST_MAX_TRACERS / 2)
        return BLAST_EINVAL;

    blast_plan *p = new (std::nothrow) blast_plan();
    if (!p) return BLAST_ENOMEM;
    p->ell.resize(d->n_ell);
    for (int e = 0; e < d->n_ell; e++) {
        p->ell[e] = d->ell_real ? d->ell_real[e] : (double)d->ell[e];
        if (p->ell[e] != floor(p->ell[e])) p->real_ell = true;
    }
    p->L = d->n_ell; p->X = d->n_chi; p->Rn = d->n_R; p->Q = d->n_chi * d->n_R;
    p->N = d->n_cheb; p->Nk = d->n_kquad; p->kmap = d->k_map;
    p->chi_min = d->chi_min; p->chi_max = d->chi_max; p->R_min = d->R_min; p->R_max = d->R_max;
    p->k_min = d->k_min; p->k_max = d->k_max;
    p->max_clust = d->max_clust; p->max_lens = d->max_lens;
    p->r_form = d->r_form;
    // tracers per (type) list of partial sums: the B-side kind, or both kinds
    // for gs in the symmetrised form (K^A_i at R chi enters too)
    p->max_tr = d->max_clust > d->max_lens ? d->max_clust : d->max_lens;
    if (p->r_form == 1) p->max_tr = d->max_clust + d->max_lens;
    p->device = d->device;
    p->Kmma = (p->N + 15) / 16 * 16;
    p->Kst = p->Kmma > 64 ? p->Kmma : 64;

    // chi: uniform nodes, composite Simpson (+ 3/8 panel on the last three
    // intervals when the number of intervals is odd)
    const int X = p->X;
    const double h = (p->chi_max - p->chi_min) / (X - 1);
    p->chi.resize(X);
    p->wchi.assign(X, 0.0);
    for (int a = 0; a < X; a++) p->chi[a] = p->chi_min + (double)a * h;
    int simpson_end = (X % 2) ? X - 1 : X - 4;  // last node of the 1/3 part
    for (int a = 0; a <= simpson_end; a++) {
        double c = (a == 0 || a == simpson_end) ? 1.0 : ((a % 2) ? 4.0 : 2.0);
        p->wchi[a] += c * h / 3.0;
    }
    if (X % 2 == 0) {
        const double c38[4] = {1.0, 3.0, 3.0, 1.0};
        for (int i = 0; i < 4; i++) p->wchi[X - 4 + i] += c38[i] * 3.0 * h / 8.0;
    }

    std::vector<double> fx, fw;
    p->R.resize(p->Rn);
    p->wR.resize(p->Rn);
    const int hn = p->Rn / 2;
    if (p->r_form == 1) {
        // R in (0, 1] (App. A): the positive points of the (2 n_R + 1)-point
        // first-kind rule on [-1, 1], with its Fejer-1 weights: the even
        // extension of the R integrand, whose value at R = 0 (the middle node)
        // vanishes with j_l(0)
        fejer1(2 * p->Rn + 1, fx, fw);
        for (int i = 0; i < p->Rn; i++) {
            p->R[i] = fx[p->Rn + 1 + i];
            p->wR[i] = fw[p->Rn + 1 + i];
        }
        p->R_min = p->R[0];
        p->R_max = 1.0;
    }
    // R: two Fejer-1 panels meeting at R = 1
    if (p->r_form == 0) fejer1(p->Rn / 2, fx, fw);
    for (int i = 0; i < hn && p->r_form == 0; i++) {
        double h1 = 0.5 * (1.0 - p->R_min), h2 = 0.5 * (p->R_max - 1.0);
        p->R[i] = 0.5 * (p->R_min + 1.0) + h1 * fx[i];
        p->wR[i] = h1 * fw[i];
        p->R[hn + i] = 0.5 * (1.0 + p->R_max) + h2 * fx[i];
        p->wR[hn + i] = h2 * fw[i];
    }

    // Chebyshev nodes of the fit
    p->tcheb.resize(p->N);
    p->kcheb.resize(p->N);
    for (int j = 0; j < p->N; j++) {
        p->tcheb[j] = cos(kPi * (2.0 * j + 1.0) / (2.0 * p->N));
        p->kcheb[j] = map_x_to_k(p->kmap, p->tcheb[j], p->k_min, p->k_max);
    }

    // Clenshaw-Curtis rule in k
    std::vector<double> cx, cw;
    int rc = cc_weights(nq, cx, cw);
    if (rc) { delete p; return rc; }
    const double kc = 0.5 * (p->k_min + p->k_max), kh = 0.5 * (p->k_max - p->k_min);
    p->kq.resize(nq + 1);
    p->wq.resize(nq + 1);
    for (int m = 0; m <= nq; m++) { p->kq[m] = kc + kh * cx[m]; p->wq[m] = kh * cw[m]; }

    // grid hash (for basis files)
    uint64_t hsh = fnv1a(p->ell.data(), sizeof(double) * p->L);
    double dv[6] = {p->chi_min, p->chi_max, p->R_min, p->R_max, p->k_min, p->k_max};
    int iv[6] = {p->X, p->Rn, p->N, p->Nk, p->kmap, p->r_form};
    hsh = fnv1a(dv, sizeof dv, hsh);
    p->grid_hash = fnv1a(iv, sizeof iv, hsh);

    // device tables
    if (cudaSetDevice(p->device) != cudaSuccess) { cudaGetLastError(); delete p; return BLAST_EDEVICE; }
    std::vector<double> u(p->N), ct(4 * p->N), pref(3 * p->L);
    for (int j = 0; j < p->N; j++) u[j] = log(p->kcheb[j]);
    for (int q = 0; q < 4 * p->N; q++) ct[q] = cos(kPi * (double)q / (2.0 * p->N));
    for (int e = 0; e < p->L; e++) {
        double l = p->ell[e];
        double f = (l + 2.0) * (l + 1.0) * l * (l - 1.0);
        pref[e] = 2.0 / kPi;
        pref[p->L + e] = 2.0 / kPi * sqrt(f);
        pref[2 * p->L + e] = 2.0 / kPi * f;
    }
    if ((rc = dev_copy(&p->d_chi, p->chi)) || (rc = dev_copy(&p->d_wchi, p->wchi)) ||
        (rc = dev_copy(&p->d_wR, p->wR)) || (rc = dev_copy(&p->d_kcheb_u, u)) ||
        (rc = dev_copy(&p->d_cos_tab, ct)) || (rc = dev_copy(&p->d_pref, pref)) || (rc = dev_copy(&p->d_ell, p->ell)) ||
        (default_envelope(p, p->env), (rc = dev_copy(&p->d_env, p->env)))) {
        plan_free_device(p);
        delete p;
        return rc;
    }
    // error word the kernels' bounded waits write; host mapped so it can be
    // read without synchronising the stream
    if (cudaHostAlloc((void **)&p->h_err, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&p->d_err, p->h_err, 0) != cudaSuccess) {
        cudaGetLastError();
        plan_free_device(p);
        delete p;
        return BLAST_EDEVICE;
    }
    *p->h_err = 0;
    if (cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        plan_free_device(p);
        delete p;
        return BLAST_EDEVICE;
    }
    if ((rc = noalloc_prepare(p->device))) {
        plan_free_device(p);
        delete p;
        return rc;
    }
    *out = p;
    return BLAST_OK;
}

// Coefficient envelope of the tensor-core path.  The slices carry 40 bits
// relative to the largest coefficient of a cosmology; Chebyshev coefficients
// of a power spectrum fall by three or more decades with n, so the basis row n
// is scaled by a power of two s_n following that fall and the coefficients by
// 1 / s_n (both exact), which spends the 40 bits on every product a_n T~_n
// instead of on the largest a_n only.  The default s_n follows the
// coefficients of a generic linear power spectrum shape, P(k) ~ x / (1 + x^3),
// x = k / 0.02 h/Mpc, at the plan's Chebyshev nodes: their running maximum
// over n +- 4, rounded to a power of two and held at or above 2^-8, because
// tabulated spectra (spline interpolation, wiggles) keep coefficients of a
// few 1e-3 of the largest at high n, and an envelope below a cosmology's own
// coefficients moves its normalisation to high n and costs precision
// everywhere.  Any positive s_n gives the same sums in exact arithmetic; a
// poor one only costs accuracy.
void default_envelope(const blast_plan *p, std::vector<double> &env)
{
    const int N = p->N;
    std::vector<double> P(N), a(N);
    for (int j = 0; j < N; j++) {
        const double x = p->kcheb[j] / 0.02;
        P[j] = x / (1.0 + x * x * x);
    }
    for (int n = 0; n < N; n++) {
        double acc = 0.0;
        for (int j = 0; j < N; j++) acc += P[j] * cos(kPi * (double)n * (2.0 * j + 1.0) / (2.0 * N));
        a[n] = fabs((n == 0 ? 1.0 : 2.0) * acc / N);
    }
    double top = 0.0;
    env.assign(N, 0.0);
    for (int n = 0; n < N; n++) {
        for (int m = (n > 4 ? n - 4 : 0); m <= n + 4 && m < N; m++) env[n] = fmax(env[n], a[m]);
        top = fmax(top, env[n]);
    }
    for (int n = 0; n < N; n++) {
        double r = (top > 0.0 && env[n] > 0.0) ? env[n] / top : 1.0;
        int e = (int)lround(log2(r));
        env[n] = ldexp(1.0, e < -8 ? -8 : (e > 0 ? 0 : e));
    }
}

extern "C" int blast_set_coef_envelope(blast_plan *p, const double *env)
{
    if (!p) return BLAST_EINVAL;
    std::vector<double> e(p->N);
    if (env) {
        double top = 0.0;
        for (int n = 0; n < p->N; n++) {
            if (!(env[n] > 0.0) || std::isinf(env[n])) return BLAST_EINVAL;
            top = fmax(top, env[n]);
        }
        for (int n = 0; n < p->N; n++) {
            int ex = (int)lround(log2(env[n] / top));
            e[n] = ldexp(1.0, ex < -16 ? -16 : (ex > 0 ? 0 : ex));
        }
    } else {
        default_envelope(p, e);
    }
    BL_CUDA(cudaSetDevice(p->device));
    BL_CUDA(cudaMemcpy(p->d_env, e.data(), sizeof(double) * p->N, cudaMemcpyHostToDevice));
    p->env = e;
    if (p->havebf && p->Tsl) {  // rebuild the slice tables with the new envelope
        int rc = launch_basis_slices(p, nullptr);
        if (rc) return rc;
        BL_CUDA(cudaStreamSynchronize(nullptr));
    }
    return BLAST_OK;
}

extern "C" int blast_plan_destroy(blast_plan *p)
{
    if (!p) return BLAST_OK;
    cudaSetDevice(p->device);
    plan_free_device(p);
    delete p;
    return BLAST_OK;
}

extern "C" int blast_plan_nodes(const blast_plan *p, double *chi, double *R, double *k_cheb)
{
    if (!p) return BLAST_EINVAL;
    if (chi) memcpy(chi, p->chi.data(), sizeof(double) * p->X);
    if (R) memcpy(R, p->R.data(), sizeof(double) * p->Rn);
    if (k_cheb) memcpy(k_cheb, p->kcheb.data(), sizeof(double) * p->N);
    return BLAST_OK;
}

int plan_alloc_basis(blast_plan *p, unsigned mask)
{
    size_t n64 = (size_t)3 * p->L * p->N * p->Q;
    size_t ncol = (size_t)3 * p->L * p->Q;
    if (!p->T64) {
        if (cudaMalloc(&p->T64, n64 * sizeof(double)) != cudaSuccess) { cudaGetLastError(); p->T64 = nullptr; return BLAST_ENOMEM; }
    }
    if ((mask & BLAST_BASIS_FP32) && !p->T32) {
        if (cudaMalloc(&p->T32, n64 * sizeof(float)) != cudaSuccess) { cudaGetLastError(); p->T32 = nullptr; return BLAST_ENOMEM; }
    }
    if ((mask & BLAST_BASIS_BF16S) && tc_supported(p) && !p->Tsl) {
        if (cudaMalloc(&p->Tsl, ncol * p->Kst * 2 * BLAST_TC_SLICES) != cudaSuccess) { cudaGetLastError(); p->Tsl = nullptr; return BLAST_ENOMEM; }
        if (cudaMalloc(&p->scT, ncol / 32 * sizeof(float)) != cudaSuccess) { cudaGetLastError(); p->scT = nullptr; return BLAST_ENOMEM; }
    }
    return BLAST_OK;
}

extern "C" int blast_precompute_basis(blast_plan *p, unsigned mask, void *stream)
{
    if (!p) return BLAST_EINVAL;
    BL_CUDA(cudaSetDevice(p->device));
    int rc = plan_alloc_basis(p, mask);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    p->have64 = p->have32 = p->havebf = false;
    if ((rc = launch_basis(p, s))) return rc;
    p->have64 = true;
    if ((rc = launch_basis_convert(p, mask, s))) return rc;
    BL_CUDA(cudaStreamSynchronize(s));
    return BLAST_OK;
}

extern "C" int blast_basis_get(const blast_plan *p, double *dst, int mem_space, void *stream)
{
    if (!p || !dst) return BLAST_EINVAL;
    if (!p->have64) return BLAST_ENOBASIS;
    BL_CUDA(cudaSetDevice(p->device));
    size_t n = (size_t)3 * p->L * p->N * p->Q * sizeof(double);
    cudaStream_t s = (cudaStream_t)stream;
    BL_CUDA(cudaMemcpyAsync(dst, p->T64, n, mem_space ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    BL_CUDA(cudaStreamSynchronize(s));
    return BLAST_OK;
}

extern "C" int blast_basis_set(blast_plan *p, const double *src, int mem_space, unsigned mask, void *stream)
{
    if (!p || !src) return BLAST_EINVAL;
    BL_CUDA(cudaSetDevice(p->device));
    int rc = plan_alloc_basis(p, mask);
    if (rc) return rc;
    size_t n = (size_t)3 * p->L * p->N * p->Q * sizeof(double);
    cudaStream_t s = (cudaStream_t)stream;
    BL_CUDA(cudaMemcpyAsync(p->T64, src, n, mem_space ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    p->have64 = true;
    p->have32 = p->havebf = false;
    if ((rc = launch_basis_convert(p, mask, s))) return rc;
    BL_CUDA(cudaStreamSynchronize(s));
    return BLAST_OK;
}

struct BasisFileHeader {
    char magic[8];
    int32_t version, L, N, X, Rn, Nk, kmap, pad;
    uint64_t grid_hash, payload_hash;
};

extern "C" int blast_basis_save(const blast_plan *p, const char *path)
{
    if (!p || !path) return BLAST_EINVAL;
    if (!p->have64) return BLAST_ENOBASIS;
    size_t n = (size_t)3 * p->L * p->N * p->Q;
    std::vector<double> h(n);
    int rc = blast_basis_get(p, h.data(), 0, nullptr);
    if (rc) return rc;
    BasisFileHeader hd;
    memset(&hd, 0, sizeof hd);
    memcpy(hd.magic, "BLASTTB1", 8);
    hd.version = 1; hd.L = p->L; hd.N = p->N; hd.X = p->X; hd.Rn = p->Rn; hd.Nk = p->Nk; hd.kmap = p->kmap;
    hd.grid_hash = p->grid_hash;
    hd.payload_hash = fnv1a(h.data(), n * sizeof(double));
    FILE *f = fopen(path, "wb");
    if (!f) return BLAST_EINVAL;
    bool ok = fwrite(&hd, sizeof hd, 1, f) == 1 && fwrite(h.data(), sizeof(double), n, f) == n;
    ok = (fclose(f) == 0) && ok;
    return ok ? BLAST_OK : BLAST_EINVAL;
}

extern "C" int blast_basis_load(blast_plan *p, const char *path, unsigned mask)
{
    if (!p || !path) return BLAST_EINVAL;
    FILE *f = fopen(path, "rb");
    if (!f) return BLAST_EINVAL;
    BasisFileHeader hd;
    if (fread(&hd, sizeof hd, 1, f) != 1 || memcmp(hd.magic, "BLASTTB1", 8) || hd.version != 1 ||
        hd.grid_hash != p->grid_hash || hd.L != p->L || hd.N != p->N || hd.X != p->X || hd.Rn != p->Rn) {
        fclose(f);
        return BLAST_EINVAL;
    }
    size_t n = (size_t)3 * p->L * p->N * p->Q;
    std::vector<double> h(n);
    bool ok = fread(h.data(), sizeof(double), n, f) == n;
    fclose(f);
    if (!ok || fnv1a(h.data(), n * sizeof(double)) != hd.payload_hash) return BLAST_EINVAL;
    return blast_basis_set(p, h.data(), 0, mask, nullptr);
}
