// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/blast.h"

#define BLAST_MAX_ELL 128
#define BLAST_MAX_TRACERS 32
#define BLAST_TC_SLICES 5   // 8-bit fixed-point slices per operand on the tensor-core path

// Status helpers -------------------------------------------------------------
#define BL_CUDA(expr)                                                             \
    do {                                                                          \
        cudaError_t _e = (expr);                                                  \
        if (_e != cudaSuccess) {                                                  \
            blast_last_error(__FILE__, __LINE__, cudaGetErrorString(_e));         \
            cudaGetLastError(); /* a non-sticky error must not fail later calls */ \
            return BLAST_EDEVICE;                                                 \
        }                                                                         \
    } while (0)

void blast_last_error(const char *file, int line, const char *msg);

// Lets `func` launch with as much dynamic shared memory as the device allows a
// block beside the kernel's static shared memory.  Every caller writes the same
// value, so plans served from several host threads cannot race on the
// attribute (a per-launch size written by one thread could fall under the size
// another thread launches with).
template <class F>
inline cudaError_t allow_opt_in_smem(F *func, int device)
{
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, func)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

// Device buffer owned by the library ------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    int ensure(size_t nbytes);  // grow (never shrink); BLAST_OK / BLAST_ENOMEM
    void release();
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// Per-call work space: one request, or a batch of them ----------------------
struct Workspace {
    DevBuf in;      // staged request inputs (float64)
    DevBuf coef;    // a_n per request (fp64), and fp32 / bf16 split copies
    DevBuf wts;     // U (per chi node) and V (per chi-R node) weights
    DevBuf ypart;   // partial sums Y[b][t][e][a][j]
    DevBuf cl;      // device C before scatter to the caller
    DevBuf meta;    // per-request descriptors
    DevBuf tc;      // coefficient slices and scales of the tensor-core path
    DevBuf nl;      // non-linear spectra at the Limber points, staged from host requests
    DevBuf ns;      // per-node Chebyshev coefficients (and staged samples) of non-separable spectra
    std::vector<char> hmeta;
};

struct blast_plan {
    // description (ells copied)
    std::vector<double> ell;        // multipoles (integers, or real values: real_ell)
    bool real_ell = false;
    int L = 0, X = 0, Rn = 0, Q = 0, N = 0, Nk = 0, kmap = 0;
    int r_form = 0;  // 0: R in [R_min, R_max]; 1: symmetrised form on (0, 1]
    double chi_min = 0, chi_max = 0, R_min = 0, R_max = 0, k_min = 0, k_max = 0;
    int max_clust = 0, max_lens = 0, max_tr = 0, device = 0;

    // host grids
    std::vector<double> chi, wchi, R, wR, tcheb, kcheb;
    std::vector<double> kq, wq;  // Clenshaw-Curtis nodes / weights in k
    uint64_t grid_hash = 0;

    // device constant tables
    double *d_chi = nullptr, *d_wchi = nullptr, *d_wR = nullptr;
    double *d_kcheb_u = nullptr;   // ln k of each Chebyshev node
    double *d_cos_tab = nullptr;   // cos(pi p / 2N), p < 4N
    double *d_pref = nullptr;      // N_AB(l) [3][L]
    double *d_ell = nullptr;       // the plan's ells
    std::vector<double> env;       // power-of-two coefficient envelope s_n of the tensor-core path
    double *d_env = nullptr;

    // basis tables
    double *T64 = nullptr;          // [3][L][N][Q]
    float *T32 = nullptr;           // [3][L][N][Q]
    uint16_t *Tsl = nullptr;        // [S][3 L Q][Kst] bf16 slices (integer x 2^-8p), K-major (n fastest)
    float *scT = nullptr;           // [3 L Q / 32] 2^(eG - 16) per 32-column tile
    int Kmma = 0;                   // N rounded up to a multiple of 16 (the MMA's K)
    int Kst = 0;                    // stored K of the slice table: max(64, Kmma), zero padded
    bool have64 = false, have32 = false, havebf = false;
    int *d_err = nullptr;           // host-mapped error word written by bounded device waits
    int test_trip = -1;             // test hook of the tensor-core contraction (blast_test_trip_wait)
    int *h_err = nullptr;
    // side stream of a call: the Chebyshev fit runs there beside the weights
    // kernel (fork and join through the two events, in the caller's stream order)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    Workspace ws;

    // launch parameters of the tensor-core kernels (0 = built-in choice), set by blast_autotune
    struct {
        int grid = 0;            // persistent CTAs of the contraction
        int red_w = 0, red_ns = 0;  // chi-chunk warps and stages per warp of the reduction
        int nbt = 0;             // cosmology tiles of the batch size tuned for
    } tune;

    // per-kernel-class launch counts and (optional) event timing
    bool prof_on = false;
    long long launches[BLAST_K_CLASSES] = {0};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev[BLAST_K_CLASSES];
    double prof_ms[BLAST_K_CLASSES] = {0};
};

// Run one launcher under the plan's profiler: count it, and when timing is on
// bracket it with events on stream s.
template <class F> int prof_launch(blast_plan *p, int cls, cudaStream_t s, F &&fn)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (p->prof_on) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    int rc = fn();
    p->launches[cls]++;
    if (p->prof_on) {
        cudaEventRecord(b, s);
        p->prof_ev[cls].emplace_back(a, b);
    }
    return rc;
}

// Request descriptor on the device (one per cosmology of a call).
struct ReqDev {
    const double *kern_chi, *kern_Rchi, *growth_chi, *growth_Rchi, *k_tab, *p_tab;
    int n_clust, n_lens, n_ptab, status;
    double *a64;      // [N]
    float *a32;       // [N]
    double *U64, *V64;  // [ntr][X], [ntr][Q]
    float *U32, *V32;
    double *cl;       // [npairs][n_sel] device output
    double *spM;      // [n_ptab] spline second derivatives of ln P (ln k), written by the fit if set
    const double *pnl;  // [L][X] non-linear P at the Limber points (Limber paths), or null
    int n_sel;
    int e_out[BLAST_MAX_ELL];  // plan ell e -> output column, -1 if not selected
};

// Launchers (defined in the kernel translation units) ------------------------
int launch_basis(blast_plan *p, cudaStream_t s);
int launch_basis_convert(blast_plan *p, unsigned mask, cudaStream_t s);
int launch_fit(blast_plan *p, ReqDev *dreq, int nreq, cudaStream_t s);
int launch_weights(blast_plan *p, ReqDev *dreq, int nreq, int want32, cudaStream_t s, int want_v64 = 1);
int launch_contract(blast_plan *p, ReqDev *dreq, int nreq, int prec, const int *d_esel, int n_esel,
                    void *ypart, cudaStream_t s);
int launch_reduce(blast_plan *p, ReqDev *dreq, int nreq, int prec, const int *d_esel, int n_esel,
                  const void *ypart, cudaStream_t s);
int launch_contract_tc(blast_plan *p, ReqDev *dreq, int nreq, const int *d_esel, int n_esel,
                       void *ypart, cudaStream_t s);
int launch_reduce_tc(blast_plan *p, ReqDev *dreq, int nreq, const int *d_esel, int n_esel,
                     const void *ypart, cudaStream_t s);
int launch_basis_slices(blast_plan *p, cudaStream_t s);
// Limber terms (limber.cu): mode 0 writes C^Limber with the linear P of each
// request (extended adds the first-order correction), mode 1 writes it with
// the request's non-linear table, mode 2 adds C^Limber(P_nl) - C^Limber(P_lin).
int launch_limber(blast_plan *p, ReqDev *dreq, int nreq, const int *d_esel, int n_esel, int mode, int extended,
                  cudaStream_t s);
// Non-separable spectra (nonsep.cu): per-node coefficients c[n][q] from the
// samples Pq[q][j]; contraction and R sum into the separable FP64 path's partials.
int launch_fit_nodes(blast_plan *p, const double *Pq, double *c, cudaStream_t s);
int launch_contract_ns(blast_plan *p, const ReqDev *dreq, const double *c, const int *d_esel, int n_esel, double *Y,
                       cudaStream_t s);
bool tc_supported(const blast_plan *p);
size_t tc_y_bytes(const blast_plan *p, int n, int n_esel);  // R-tile partials of a tensor-core call
size_t tc_ws_total(const blast_plan *p, int n);  // coefficient slices, scales and chi weights of a call
int tc_reserve(blast_plan *p, int n);
// Staging of a batch: checks, ell union, work space, request descriptors on the
// device; with prep, also the fit and the weights (launch_prep).
int stage_batch(blast_plan *p, int n, const blast_request *reqs, int prec, double *const *outs, int out_mem_space,
                cudaStream_t s, ReqDev **dreq_out, int **d_esel, int *n_esel, std::vector<ReqDev> &hreq,
                std::vector<char> &direct_out, const double *const *pnl, bool prep);
int launch_prep(blast_plan *p, ReqDev *dreq, int n, int prec, cudaStream_t s);
// Steps (a) and (b) of a staged, prepared batch in the plan's work space.
int launch_cl_kernels(blast_plan *p, ReqDev *dreq, int n, int prec, const int *d_esel, int n_esel, cudaStream_t s);
// Work space for batches of up to nmax requests with device inputs and outputs,
// every ell and any precision, allocated now; *bytes = the plan's work space.
int plan_reserve(blast_plan *p, int nmax, size_t *bytes);

// Host helpers
int plan_alloc_basis(blast_plan *p, unsigned mask);
void default_envelope(const blast_plan *p, std::vector<double> &env);  // generic linear-P coefficient envelope
int request_check(const blast_plan *p, const blast_request *r);  // the checks of blast_cl
int request_n_sel(const blast_plan *p, const blast_request *r);  // ells selected by the mask
double host_now();
int noalloc_prepare(int dev);     // allocation-free path: scratch address and kernel code, per device
int preload_fp64_kernels();       // load the FP64 evaluation kernels' code (lazy module loading)
