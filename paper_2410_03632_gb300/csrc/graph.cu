// Batch graphs: one blast_cl_batch call (device inputs and outputs) captured
// once into a CUDA graph and launched again and again with the same buffers.
// The request descriptors are staged and every buffer the kernels touch is
// allocated before the capture, in a work space the graph owns, so a launch
// is the kernels alone: fit and weights (forked onto the plan's side stream
// during the capture), coefficient slices, contraction and reduction.  The
// caller rewrites the contents of its input arrays between launches, e.g. the
// proposals of a sampler written into fixed device buffers.
#include <utility>

#include "blast_internal.h"

struct blast_graph {
    blast_plan *plan = nullptr;
    Workspace ws;  // the graph's work space, baked into its kernels
    cudaStream_t cs = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void graph_free(blast_graph *g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->cs) cudaStreamDestroy(g->cs);
    g->ws.in.release(); g->ws.coef.release(); g->ws.wts.release(); g->ws.ypart.release(); g->ws.cl.release();
    g->ws.meta.release(); g->ws.tc.release(); g->ws.nl.release(); g->ws.ns.release();
    delete g;
}

extern "C" int blast_graph_create(blast_plan *p, int n, const blast_request *reqs, int precision,
                                  double *const *outs, blast_graph **out)
{
    if (!p || n < 1 || !reqs || !outs || !out) return BLAST_EINVAL;
    *out = nullptr;
    if (precision < BLAST_FP64 || precision > BLAST_BF16S) return BLAST_EINVAL;
    for (int i = 0; i < n; i++) {
        if (reqs[i].mem_space != 1 || !outs[i] || reinterpret_cast<uintptr_t>(outs[i]) % 8) return BLAST_EINVAL;
        int rc = request_check(p, &reqs[i]);
        if (rc) return rc;
    }
    if (precision == BLAST_BF16S && !tc_supported(p)) return BLAST_EINVAL;
    if ((precision == BLAST_FP64 && !p->have64) || (precision == BLAST_FP32 && !p->have32) ||
        (precision == BLAST_BF16S && !p->havebf))
        return BLAST_ENOBASIS;
    if (*p->h_err) {
        *p->h_err = 0;
        return BLAST_ETIMEOUT;
    }
    BL_CUDA(cudaSetDevice(p->device));
    auto *g = new blast_graph;
    g->plan = p;
    if (cudaStreamCreateWithFlags(&g->cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        graph_free(g);
        return BLAST_EDEVICE;
    }
    // the graph's buffers stand in for the plan's during set-up and capture
    std::swap(p->ws, g->ws);
    const bool prof = p->prof_on;
    p->prof_on = false;  // no profiler events inside the graph
    std::vector<ReqDev> hreq;
    std::vector<char> direct_out;
    ReqDev *dreq = nullptr;
    int *d_esel = nullptr, n_esel = 0;
    int rc = plan_reserve(p, n, nullptr);
    if (!rc)
        rc = stage_batch(p, n, reqs, precision, outs, 1, g->cs, &dreq, &d_esel, &n_esel, hreq, direct_out, nullptr,
                         false);
    if (!rc && cudaStreamSynchronize(g->cs) != cudaSuccess) {  // the descriptors are on the device
        cudaGetLastError();
        rc = BLAST_EDEVICE;
    }
    if (!rc) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(g->cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            cudaGetLastError();
            rc = BLAST_EDEVICE;
        } else {
            rc = launch_prep(p, dreq, n, precision, g->cs);
            if (!rc) rc = launch_cl_kernels(p, dreq, n, precision, d_esel, n_esel, g->cs);
            const cudaError_t e = cudaStreamEndCapture(g->cs, &graph);  // always ends the capture
            if (!rc && e != cudaSuccess) rc = BLAST_EDEVICE;
            if (!rc && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) rc = BLAST_EDEVICE;
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
        }
    }
    p->prof_on = prof;
    std::swap(p->ws, g->ws);
    if (rc) {
        graph_free(g);
        return rc;
    }
    *out = g;
    return BLAST_OK;
}

extern "C" int blast_graph_launch(blast_graph *g, void *stream)
{
    if (!g) return BLAST_EINVAL;
    blast_plan *p = g->plan;
    if (*p->h_err) {  // a bounded device wait of an earlier launch or call gave up
        *p->h_err = 0;
        return BLAST_ETIMEOUT;
    }
    BL_CUDA(cudaSetDevice(p->device));
    BL_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return BLAST_OK;
}

extern "C" size_t blast_graph_reserved(const blast_graph *g)
{
    if (!g) return 0;
    const Workspace &w = g->ws;
    return w.in.bytes + w.coef.bytes + w.wts.bytes + w.ypart.bytes + w.cl.bytes + w.meta.bytes + w.tc.bytes +
           w.nl.bytes + w.ns.bytes;
}

extern "C" int blast_graph_destroy(blast_graph *g)
{
    if (!g) return BLAST_EINVAL;
    cudaSetDevice(g->plan->device);
    graph_free(g);
    return BLAST_OK;
}
