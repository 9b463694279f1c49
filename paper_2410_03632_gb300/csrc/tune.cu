// Autotuner of the tensor-core path's launch parameters: the number of
// persistent CTAs of the contraction (it sets how the (cosmology tile, tracer
// group, q tile) units fall on the SMs) and the reduction's chi-chunk warps
// and stages.  Each candidate runs the caller's representative batch a few
// times under the plan's kernel timer; the fastest stays in the plan.  A
// cache file keeps choices across processes, one line per key:
//   <GPU name>|L|X|n_R|N|max_clust|max_lens|cosmology tiles <TAB> grid W NS
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "blast_internal.h"

namespace {

std::string tune_key(const blast_plan *p, int nbt)
{
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) name = prop.name;
    for (char &c : name)
        if (c == '|' || c == '\t' || c == '\n') c = '_';
    char buf[256];
    snprintf(buf, sizeof buf, "|%d|%d|%d|%d|%d|%d|%d", p->L, p->X, p->Rn, p->N, p->max_clust, p->max_lens, nbt);
    return name + buf;
}

bool cache_lookup(const char *path, const std::string &key, int &grid, int &w, int &ns)
{
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof line, f)) {  // the last entry of a key wins
        char *tab = strchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        int g2, w2, n2;
        if (key == line && sscanf(tab + 1, "%d %d %d", &g2, &w2, &n2) == 3) {
            grid = g2; w = w2; ns = n2;
            found = true;
        }
    }
    fclose(f);
    return found;
}

// Summed device time of the contraction and the reduction over `reps` runs.
int time_batch(blast_plan *p, int n, const blast_request *reqs, double *const *outs, cudaStream_t s, int reps,
               double *ms)
{
    int rc = blast_profile_reset(p);
    if (rc) return rc;
    blast_profile_enable(p, 1);
    for (int r = 0; r < reps && !rc; r++) rc = blast_cl_batch(p, n, reqs, BLAST_BF16S, outs, 1, s);
    blast_profile_enable(p, 0);
    if (rc) return rc;
    double a = 0.0, b = 0.0;
    if ((rc = blast_profile_read(p, BLAST_K_CONTRACT_TC, &a, nullptr)) ||
        (rc = blast_profile_read(p, BLAST_K_REDUCE, &b, nullptr)))
        return rc;
    *ms = a + b;
    return blast_profile_reset(p);
}

}  // namespace

extern "C" int blast_autotune(blast_plan *p, int n, const blast_request *reqs, const char *cache_path, void *stream)
{
    if (!p || n < 1 || !reqs) return BLAST_EINVAL;
    if (!tc_supported(p)) return BLAST_EINVAL;
    if (!p->havebf) return BLAST_ENOBASIS;
    BL_CUDA(cudaSetDevice(p->device));
    const int nbt = (n + 127) / 128;
    const std::string key = tune_key(p, nbt);
    int grid = 0, w = 0, ns = 0;
    if (cache_path && cache_lookup(cache_path, key, grid, w, ns)) {
        p->tune.grid = grid; p->tune.red_w = w; p->tune.red_ns = ns; p->tune.nbt = nbt;
        return BLAST_OK;
    }
    // device outputs for the representative batch
    std::vector<double *> outs(n, nullptr);
    int rc = BLAST_OK;
    for (int i = 0; i < n && !rc; i++) {
        const size_t bytes = sizeof(double) * blast_npairs(reqs[i].n_clust, reqs[i].n_lens) * p->L;
        if (cudaMalloc(&outs[i], bytes) != cudaSuccess) { cudaGetLastError(); rc = BLAST_ENOMEM; }
    }
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    const int gmax = sms / nbt * nbt;
    // candidates: every SM and a few counts a cosmology tile below
    std::vector<int> grids;
    for (int k = 0; k < 6 && gmax - k * nbt >= nbt; k++) grids.push_back(gmax - k * nbt);
    const int Ws[3] = {2, 4, 8};
    double best = 1e300;
    int bg = 0, bw = 0, bns = 0;
    const auto saved = p->tune;
    if (!rc) {  // warm-up with the built-in choice (also checks the batch)
        p->tune.grid = p->tune.red_w = p->tune.red_ns = 0;
        double ms = 0.0;
        rc = time_batch(p, n, reqs, outs.data(), s, 1, &ms);
    }
    // the two kernels are independent: the CTA count first (built-in reduction),
    // then the reduction's shape with that count
    for (size_t gi = 0; gi < grids.size() && !rc; gi++) {
        p->tune.grid = grids[gi]; p->tune.red_w = p->tune.red_ns = 0;
        double ms = 0.0;
        rc = time_batch(p, n, reqs, outs.data(), s, 3, &ms);
        if (!rc && ms < best) { best = ms; bg = grids[gi]; }
    }
    best = 1e300;
    for (int wi = 0; wi < 3 && !rc; wi++) {
        for (int nsv = 1; nsv <= 4 && !rc; nsv++) {
            p->tune.grid = bg; p->tune.red_w = Ws[wi]; p->tune.red_ns = nsv;
            double ms = 0.0;
            rc = time_batch(p, n, reqs, outs.data(), s, 3, &ms);
            if (!rc && ms < best) { best = ms; bw = Ws[wi]; bns = nsv; }
        }
    }
    for (double *o : outs)
        if (o) cudaFree(o);
    if (rc) {
        p->tune = saved;
        return rc;
    }
    p->tune.grid = bg; p->tune.red_w = bw; p->tune.red_ns = bns; p->tune.nbt = nbt;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s\t%d %d %d\n", key.c_str(), bg, bw, bns);
            fclose(f);
        }
    }
    return BLAST_OK;
}

extern "C" int blast_tuned_params(const blast_plan *p, int *grid, int *red_warps, int *red_stages)
{
    if (!p) return BLAST_EINVAL;
    if (grid) *grid = p->tune.grid;
    if (red_warps) *red_warps = p->tune.red_w;
    if (red_stages) *red_stages = p->tune.red_ns;
    return BLAST_OK;
}
