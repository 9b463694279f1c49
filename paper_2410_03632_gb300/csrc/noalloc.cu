// blast_cl_noalloc: the FP64 evaluation of one cosmology (fit, weights,
// contraction, quadrature) with every piece of scratch memory taken from a
// fixed array compiled into the library instead of from cudaMalloc.
//
// Who needs it: callers that must not allocate device memory at evaluation
// time.  Examples are a host framework that has reserved the GPU's memory for
// its own pool allocator (a raw cudaMalloc behind its back can fail or
// fragment that pool) and latency-critical request loops, where cudaMalloc /
// cudaFree can synchronise the device and stall work on other streams.  The
// caller still owns and passes the inputs (device arrays) and the output.
//
// The scratch array lives in the device image: every GPU that loads the
// library holds BLAST_NOALLOC_SCRATCH_BYTES of it until the process exits.
// CUDA loads modules lazily, so the array (and the code of the kernels this
// path launches) is placed on a device the first time it is touched there;
// plan creation touches it (noalloc_prepare), so that memory is taken when a
// plan is made and never inside blast_cl_noalloc.
#include <cstring>
#include <mutex>

#include "blast_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[BLAST_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_dev[kMaxDevices] = {nullptr};  // device address of the array, per ordinal

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// Set-up, once per device and with that device current: the array's name is
// only a host-side stand-in, so its device address is looked up here.
int scratch_for_device(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return BLAST_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            blast_last_error(__FILE__, __LINE__, cudaGetErrorString(e));
            return BLAST_EDEVICE;
        }
        g_scratch_dev[dev] = static_cast<unsigned char *>(ptr);
    }
    *out = g_scratch_dev[dev];
    return BLAST_OK;
}

// The request descriptor and ell list travel as a kernel argument and are
// written into the scratch array on the stream: no host-to-device copy call.
struct NoallocDesc {
    ReqDev req;
    int esel[BLAST_MAX_ELL];
};

__global__ void k_put_desc(const NoallocDesc d, ReqDev *req_dst, int *esel_dst)
{
    const int *src = reinterpret_cast<const int *>(&d.req);
    int *dst = reinterpret_cast<int *>(req_dst);
    for (int i = threadIdx.x; i < (int)(sizeof(ReqDev) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    for (int i = threadIdx.x; i < BLAST_MAX_ELL; i += blockDim.x) esel_dst[i] = d.esel[i];
}

bool selected(const blast_request *r, int e)
{
    if (!r->ell_mask_lo && !r->ell_mask_hi) return true;
    return e < 64 ? ((r->ell_mask_lo >> e) & 1) : ((r->ell_mask_hi >> (e - 64)) & 1);
}

}  // namespace

// Set-up for one device, with that device current: look up the array's device
// address and load the code of every kernel the allocation-free path launches
// (module loading is lazy and would otherwise take device memory on the first
// call).  Called by blast_plan_create.
int noalloc_prepare(int dev)
{
    unsigned char *S = nullptr;
    int rc = scratch_for_device(dev, &S);
    if (rc) return rc;
    cudaFuncAttributes fa;
    BL_CUDA(cudaFuncGetAttributes(&fa, k_put_desc));
    return preload_fp64_kernels();
}

extern "C" int blast_cl_noalloc(blast_plan *p, const blast_request *r, double *cl_out, void *stream)
{
    if (!p || !r || !cl_out) return BLAST_EINVAL;
    if (r->mem_space != 1) return BLAST_EINVAL;  // device inputs only: nothing is staged
    // the checks of blast_cl: tracer counts, table size, ell mask within the plan
    int rc = request_check(p, r);
    if (rc) return rc;
    // the kernels load and store doubles through these pointers
    const void *ptrs[] = {r->kern_chi, r->kern_Rchi, r->growth_chi, r->growth_Rchi, r->k_tab, r->p_tab, cl_out};
    for (const void *q : ptrs)
        if (reinterpret_cast<uintptr_t>(q) % 8) return BLAST_EINVAL;

    // ells to evaluate and their output columns
    NoallocDesc nd;
    memset(&nd, 0, sizeof nd);
    ReqDev &h = nd.req;
    int *esel = nd.esel, n_esel = 0;
    for (int e = 0; e < BLAST_MAX_ELL; e++) h.e_out[e] = -1;
    for (int e = 0; e < p->L; e++)
        if (selected(r, e)) { h.e_out[e] = n_esel; esel[n_esel++] = e; }
    if (n_esel == 0) return BLAST_EINVAL;
    h.n_sel = n_esel;

    // scratch layout, every piece 256-byte aligned
    const int ntr = r->n_clust + r->n_lens;
    const size_t o_req = 0;
    const size_t o_esel = o_req + al256(sizeof(ReqDev));
    const size_t o_a64 = o_esel + al256(sizeof(int) * BLAST_MAX_ELL);
    const size_t o_a32 = o_a64 + al256(sizeof(double) * p->N);
    const size_t o_U = o_a32 + al256(sizeof(float) * p->N);
    const size_t o_V = o_U + al256(sizeof(double) * ntr * p->X);
    const size_t o_Y = o_V + al256(sizeof(double) * ntr * p->Q);
    const size_t end = o_Y + al256(sizeof(double) * 3 * n_esel * p->X * p->max_tr);
    if (end > BLAST_NOALLOC_SCRATCH_BYTES) {
        blast_last_error(__FILE__, __LINE__, "request needs more scratch than BLAST_NOALLOC_SCRATCH_BYTES");
        return BLAST_ENOMEM;
    }
    if (!p->have64) return BLAST_ENOBASIS;

    if (cudaSetDevice(p->device) != cudaSuccess) { cudaGetLastError(); return BLAST_EDEVICE; }
    unsigned char *S = nullptr;
    if ((rc = scratch_for_device(p->device, &S))) return rc;
    cudaStream_t s = (cudaStream_t)stream;

    h.kern_chi = r->kern_chi; h.kern_Rchi = r->kern_Rchi;
    h.growth_chi = r->growth_chi; h.growth_Rchi = r->growth_Rchi;
    h.k_tab = r->k_tab; h.p_tab = r->p_tab;
    h.n_clust = r->n_clust; h.n_lens = r->n_lens; h.n_ptab = r->n_ptab; h.status = 0;
    h.a64 = reinterpret_cast<double *>(S + o_a64);
    h.a32 = reinterpret_cast<float *>(S + o_a32);
    h.U64 = reinterpret_cast<double *>(S + o_U);
    h.V64 = reinterpret_cast<double *>(S + o_V);
    h.U32 = nullptr;  // the FP64 path writes no single-precision weights
    h.V32 = nullptr;
    h.cl = cl_out;
    ReqDev *dreq = reinterpret_cast<ReqDev *>(S + o_req);
    int *d_esel = reinterpret_cast<int *>(S + o_esel);
    // Every scratch byte a kernel reads below is written earlier in this call
    // on the same stream, so nothing needs clearing first.
    k_put_desc<<<1, 128, 0, s>>>(nd, dreq, d_esel);
    BL_CUDA(cudaGetLastError());
    if ((rc = launch_fit(p, dreq, 1, s))) return rc;
    if ((rc = launch_weights(p, dreq, 1, 0, s))) return rc;
    void *Y = S + o_Y;
    if ((rc = launch_contract(p, dreq, 1, BLAST_FP64, d_esel, n_esel, Y, s))) return rc;
    if ((rc = launch_reduce(p, dreq, 1, BLAST_FP64, d_esel, n_esel, Y, s))) return rc;
    return BLAST_OK;
}
