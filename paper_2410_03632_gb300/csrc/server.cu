// Request server: continuous batching of C_l requests over resident plans.
//
// blast_submit copies a request's inputs into pinned host staging (the caller
// may free its arrays when the call returns), checks it, and admits it against
// a device-byte budget (blast_request_footprint of every admitted request not
// yet finished).  One worker thread per server forms batches: the oldest
// waiting request fixes (plan, precision) and every waiting request with the
// same pair joins, up to max_slots, in arrival order.  Requests that arrive
// while a batch runs wait for the next one.  A batch is one blast_cl_batch call
// on the plan's own stream; inputs and outputs stay in pinned host memory that
// the kernels read and write in place.  If a batch fails, its requests run one
// by one so a bad request fails alone.  blast_poll waits (bounded) for a
// ticket, copies its C_l out and retires it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "blast_internal.h"

namespace {

struct Job {
    uint64_t ticket = 0;
    int plan_idx = 0, prec = 0;
    blast_request req{};      // points into in[]
    double *in = nullptr;     // pinned: kern_chi | kern_Rchi | growth_chi | growth_Rchi | k_tab | p_tab
    size_t in_bytes = 0;
    double *out = nullptr;    // pinned: C[npairs][n_sel]
    size_t out_bytes = 0;
    size_t footprint = 0;
    int status = BLAST_ENOTREADY;
    bool done = false;
};

// Pinned host buffers, reused by size class (a pinned allocation costs far more
// than a request's evaluation).
class PinnedPool {
public:
    void *get(size_t bytes)
    {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = free_.lower_bound(bytes);
        if (it != free_.end() && it->first <= 2 * bytes + 4096) {
            void *p = it->second;
            size_[p] = it->first;
            free_.erase(it);
            return p;
        }
        void *p = nullptr;
        if (cudaHostAlloc(&p, bytes, cudaHostAllocPortable | cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        size_[p] = bytes;
        return p;
    }
    void put(void *p)
    {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu_);
        free_.emplace(size_[p], p);
    }
    ~PinnedPool()
    {
        for (auto &kv : size_) cudaFreeHost(kv.first);
    }

private:
    std::mutex mu_;
    std::multimap<size_t, void *> free_;
    std::unordered_map<void *, size_t> size_;
};

}  // namespace

struct blast_server {
    std::vector<blast_plan *> plans;
    std::vector<cudaStream_t> streams;  // one per plan, created on the plan's device
    size_t budget = 0, used = 0;
    int max_slots = 1;
    size_t max_pending = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> pending;
    std::unordered_map<uint64_t, Job *> jobs;  // admitted and not yet retired by poll
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    PinnedPool pool;
};

namespace {

void release(blast_server *s, Job *j)
{
    s->pool.put(j->in);
    s->pool.put(j->out);
    delete j;
}

int run_batch(blast_server *s, std::vector<Job *> &batch)
{
    const int pi = batch[0]->plan_idx, prec = batch[0]->prec;
    std::vector<blast_request> reqs;
    std::vector<double *> outs;
    for (Job *j : batch) {
        reqs.push_back(j->req);
        outs.push_back(j->out);
    }
    return blast_cl_batch(s->plans[pi], (int)batch.size(), reqs.data(), prec, outs.data(), 0, s->streams[pi]);
}

void worker_loop(blast_server *s)
{
    for (;;) {
        std::vector<Job *> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
            if (s->pending.empty()) return;  // stopping with nothing left
            const Job *head = s->pending.front();
            const int pi = head->plan_idx, prec = head->prec;
            for (auto it = s->pending.begin(); it != s->pending.end() && (int)batch.size() < s->max_slots;) {
                if ((*it)->plan_idx == pi && (*it)->prec == prec) {
                    batch.push_back(*it);
                    it = s->pending.erase(it);
                } else {
                    ++it;
                }
            }
        }
        std::vector<int> st(batch.size(), run_batch(s, batch));
        if (st[0] != BLAST_OK && batch.size() > 1) {  // isolate the request that failed
            for (size_t i = 0; i < batch.size(); i++) {
                std::vector<Job *> one{batch[i]};
                st[i] = run_batch(s, one);
            }
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (size_t i = 0; i < batch.size(); i++) {
                batch[i]->status = st[i];
                batch[i]->done = true;
                s->used -= batch[i]->footprint;
            }
        }
        s->cv_done.notify_all();
    }
}

}  // namespace

extern "C" int blast_server_create(blast_plan *const *plans, int n_plans, size_t hbm_budget, int max_slots,
                                   blast_server **out)
{
    if (!plans || n_plans < 1 || !out || max_slots < 1 || hbm_budget == 0) return BLAST_EINVAL;
    for (int i = 0; i < n_plans; i++)
        if (!plans[i]) return BLAST_EINVAL;
    auto *s = new blast_server;
    s->plans.assign(plans, plans + n_plans);
    s->budget = hbm_budget;
    s->max_slots = max_slots;
    s->max_pending = (size_t)16 * max_slots;
    for (int i = 0; i < n_plans; i++) {
        cudaStream_t st = nullptr;
        if (cudaSetDevice(plans[i]->device) != cudaSuccess ||
            cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return BLAST_EDEVICE;
        }
        s->streams.push_back(st);
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return BLAST_OK;
}

extern "C" int blast_submit(blast_server *s, int plan_idx, const blast_request *req, int precision, uint64_t *ticket)
{
    if (!s || !req || !ticket || plan_idx < 0 || plan_idx >= (int)s->plans.size()) return BLAST_EINVAL;
    if (precision < BLAST_FP64 || precision > BLAST_BF16S) return BLAST_EINVAL;
    blast_plan *p = s->plans[plan_idx];
    if (req->n_clust < 0 || req->n_lens < 0 || req->n_clust + req->n_lens < 1 || req->n_clust > p->max_clust ||
        req->n_lens > p->max_lens || req->n_ptab < 3 || req->n_ptab > 1 << 20 ||
        (req->mem_space != 0 && req->mem_space != 1))
        return BLAST_EINVAL;
    if (precision == BLAST_BF16S && !tc_supported(p)) return BLAST_EINVAL;
    if ((precision == BLAST_FP64 && !p->have64) || (precision == BLAST_FP32 && !p->have32) ||
        (precision == BLAST_BF16S && !p->havebf))
        return BLAST_ENOBASIS;
    if (!req->kern_chi || !req->kern_Rchi || !req->growth_chi || !req->growth_Rchi || !req->k_tab || !req->p_tab)
        return BLAST_EINVAL;

    // stage the inputs (host or device memory) into pinned host memory
    const int ntr = req->n_clust + req->n_lens;
    const size_t nkc = (size_t)ntr * p->X, nkr = (size_t)ntr * p->Q, npt = (size_t)req->n_ptab;
    auto *j = new Job;
    j->in_bytes = (nkc + nkr + p->X + p->Q + 2 * npt) * sizeof(double);
    j->in = static_cast<double *>(s->pool.get(j->in_bytes));
    if (!j->in) {
        delete j;
        return BLAST_ENOMEM;
    }
    double *d = j->in;
    const struct {
        const double *src;
        size_t n;
    } parts[6] = {{req->kern_chi, nkc}, {req->kern_Rchi, nkr}, {req->growth_chi, (size_t)p->X},
                  {req->growth_Rchi, (size_t)p->Q}, {req->k_tab, npt}, {req->p_tab, npt}};
    const double *dst[6];
    for (int k = 0; k < 6; k++) {
        if (req->mem_space == 0) {
            std::memcpy(d, parts[k].src, parts[k].n * sizeof(double));
        } else if (cudaMemcpy(d, parts[k].src, parts[k].n * sizeof(double), cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            release(s, j);
            return BLAST_EINVAL;
        }
        dst[k] = d;
        d += parts[k].n;
    }
    j->req = *req;
    j->req.kern_chi = dst[0];
    j->req.kern_Rchi = dst[1];
    j->req.growth_chi = dst[2];
    j->req.growth_Rchi = dst[3];
    j->req.k_tab = dst[4];
    j->req.p_tab = dst[5];
    j->req.mem_space = 0;
    int rc = request_check(p, &j->req);  // full check on the staged copy (P table included)
    if (rc) {
        release(s, j);
        return rc;
    }
    j->plan_idx = plan_idx;
    j->prec = precision;
    j->out_bytes = blast_npairs(req->n_clust, req->n_lens) * (size_t)request_n_sel(p, &j->req) * sizeof(double);
    j->out = static_cast<double *>(s->pool.get(std::max<size_t>(j->out_bytes, 8)));
    if (!j->out) {
        release(s, j);
        return BLAST_ENOMEM;
    }
    j->footprint = blast_request_footprint(p, &j->req);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (j->footprint > s->budget) {
            rc = BLAST_ENOMEM;  // could never be admitted
        } else if (s->used + j->footprint > s->budget || s->pending.size() >= s->max_pending) {
            rc = BLAST_EBUSY;
        } else {
            j->ticket = s->next_ticket++;
            s->used += j->footprint;
            s->jobs[j->ticket] = j;
            s->pending.push_back(j);
            *ticket = j->ticket;
        }
    }
    if (rc) {
        release(s, j);
        return rc;
    }
    s->cv_work.notify_one();
    return BLAST_OK;
}

extern "C" int blast_poll(blast_server *s, uint64_t ticket, double *cl_out, int *done, int64_t timeout_us)
{
    if (!s || !done) return BLAST_EINVAL;
    *done = 0;
    Job *j = nullptr;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return BLAST_EINVAL;
        j = it->second;
        auto ready = [&] { return j->done; };
        if (timeout_us < 0)
            s->cv_done.wait(lk, ready);
        else
            s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
        if (!j->done) return BLAST_ENOTREADY;
        s->jobs.erase(it);
    }
    *done = 1;
    int rc = j->status;
    if (rc == BLAST_OK && j->out_bytes) {
        if (!cl_out) {
            rc = BLAST_EINVAL;
        } else if (cudaMemcpy(cl_out, j->out, j->out_bytes, cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            rc = BLAST_EDEVICE;
        }
    }
    release(s, j);
    return rc;
}

extern "C" int blast_server_destroy(blast_server *s)
{
    if (!s) return BLAST_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();  // waiting requests are evaluated first
    for (auto &kv : s->jobs) release(s, kv.second);
    for (size_t i = 0; i < s->streams.size(); i++) {
        cudaSetDevice(s->plans[i]->device);
        cudaStreamDestroy(s->streams[i]);
    }
    delete s;
    return BLAST_OK;
}
