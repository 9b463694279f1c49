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

// Status helpers -------------------------------------------------------------
#define BL_CUDA(expr)                                                             \
    do {                                                                          \
        cudaError_t _e = (expr);                                                  \
        if (_e != cudaSuccess) {                                                  \
            blast_last_error(__FILE__, __LINE__, cudaGetErrorString(_e));         \
            return BLAST_EDEVICE;                                                 \
        }                                                                         \
    } while (0)

void blast_last_error(const char *file, int line, const char *msg);

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
    std::vector<char> hmeta;
};

struct blast_plan {
    // description (ells copied)
    std::vector<int32_t> ell;
    int L = 0, X = 0, Rn = 0, Q = 0, N = 0, Nk = 0, kmap = 0;
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

    // basis tables
    double *T64 = nullptr;          // [3][L][N][Q]
    float *T32 = nullptr;           // [3][L][N][Q]
    uint16_t *Tbf_hi = nullptr;     // [3][L][Q][Nk16] bf16 high part, K-major (n fastest)
    uint16_t *Tbf_lo = nullptr;     // [3][L][Q][Nk16] bf16 low part (T - hi, rounded)
    int Nk16 = 0;                   // N rounded up to a multiple of 16 (zero padded)
    bool have64 = false, have32 = false, havebf = false;

    Workspace ws;
};

// Request descriptor on the device (one per cosmology of a call).
struct ReqDev {
    const double *kern_chi, *kern_Rchi, *growth_chi, *growth_Rchi, *k_tab, *p_tab;
    int n_clust, n_lens, n_ptab, status;
    double *a64;      // [N]
    float *a32;       // [N]
    double *U64, *V64;  // [ntr][X], [ntr][Q]
    float *U32, *V32;
    double *cl;       // [npairs][n_sel] device output
    int n_sel;
    int e_out[BLAST_MAX_ELL];  // plan ell e -> output column, -1 if not selected
};

// Launchers (defined in the kernel translation units) ------------------------
int launch_basis(blast_plan *p, cudaStream_t s);
int launch_basis_convert(blast_plan *p, unsigned mask, cudaStream_t s);
int launch_fit(blast_plan *p, ReqDev *dreq, int nreq, cudaStream_t s);
int launch_weights(blast_plan *p, ReqDev *dreq, int nreq, int want32, cudaStream_t s);
int launch_contract(blast_plan *p, ReqDev *dreq, int nreq, int prec, const int *d_esel, int n_esel,
                    void *ypart, cudaStream_t s);
int launch_reduce(blast_plan *p, ReqDev *dreq, int nreq, int prec, const int *d_esel, int n_esel,
                  const void *ypart, cudaStream_t s);
int launch_contract_tc(blast_plan *p, ReqDev *dreq, int nreq, const int *d_esel, int n_esel,
                       void *ypart, void *coef_bf, cudaStream_t s);

// Host helpers
int plan_alloc_basis(blast_plan *p, unsigned mask);
double host_now();
