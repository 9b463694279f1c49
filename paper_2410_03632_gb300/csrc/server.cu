// Request server: continuous batching of C_l requests over resident plans.
//
// Each plan is a lane with its own worker thread, CUDA stream, reserved work
// space and ring of device slots, so the batches of different plans overlap on
// the GPU.  blast_submit copies a request's inputs into pinned host staging (the
// caller may free its arrays when the call returns), checks them, and admits the
// request when its plan's ring has a free slot (and the queue has room).  A
// lane's worker forms batches: the oldest waiting request of the plan fixes the
// precision and every waiting request of the plan with that precision joins, up
// to max_slots, in arrival order; requests that arrive while a batch runs wait
// for the next one.  A batch copies each request's inputs into its device slot,
// runs one blast_cl_batch with device inputs and outputs on the lane's stream,
// and copies the C_l back to pinned memory.  No device memory is allocated
// after blast_server_create: every buffer a batch touches was reserved there.
// If a batch fails, its requests run one by one so a bad request fails alone.
// blast_poll waits (bounded) for a ticket, copies its C_l out and retires it.
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
    int plan_idx = 0, prec = 0, slot = -1;
    blast_request req{};      // points into in[] (host copy) until the batch moves it to the slot
    double *in = nullptr;     // pinned: kern_chi | kern_Rchi | growth_chi | growth_Rchi | k_tab | p_tab
    size_t in_bytes = 0;
    double *out = nullptr;    // pinned: C[npairs][n_sel]
    size_t out_bytes = 0;
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

// One plan's share of the server: stream, worker and the device slot ring.
struct Lane {
    blast_plan *plan = nullptr;
    cudaStream_t stream = nullptr;
    std::thread worker;
    double *ring = nullptr;     // nslots x slot_doubles device doubles
    size_t slot_doubles = 0;    // inputs of the largest request, then its C_l
    size_t in_doubles = 0;
    std::vector<int> free_slots;
    size_t reserved = 0;        // device bytes: ring + the plan's reserved work space
};

}  // namespace

struct blast_server {
    std::vector<Lane> lanes;
    size_t budget = 0;
    int max_slots = 1;
    size_t max_pending = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> pending;
    std::unordered_map<uint64_t, Job *> jobs;  // admitted and not yet retired by poll
    uint64_t next_ticket = 1;
    bool stop = false;
    PinnedPool pool;
};

namespace {

void release(blast_server *s, Job *j)
{
    s->pool.put(j->in);
    s->pool.put(j->out);
    delete j;
}

// One batch of lane li: inputs into the jobs' device slots, one evaluation with
// device inputs and outputs on the lane's stream, C_l back to pinned memory.
int run_batch(blast_server *s, int li, std::vector<Job *> &batch)
{
    Lane &ln = s->lanes[li];
    blast_plan *p = ln.plan;
    const int prec = batch[0]->prec;
    std::vector<blast_request> reqs;
    std::vector<double *> outs;
    for (Job *j : batch) {
        double *slot = ln.ring + (size_t)j->slot * ln.slot_doubles;
        BL_CUDA(cudaMemcpyAsync(slot, j->in, j->in_bytes, cudaMemcpyHostToDevice, ln.stream));
        blast_request r = j->req;
        auto moved = [&](const double *hp) { return slot + (hp - j->in); };
        r.kern_chi = moved(j->req.kern_chi);
        r.kern_Rchi = moved(j->req.kern_Rchi);
        r.growth_chi = moved(j->req.growth_chi);
        r.growth_Rchi = moved(j->req.growth_Rchi);
        r.k_tab = moved(j->req.k_tab);
        r.p_tab = moved(j->req.p_tab);
        r.mem_space = 1;
        reqs.push_back(r);
        outs.push_back(slot + ln.in_doubles);
    }
    int rc = blast_cl_batch(p, (int)batch.size(), reqs.data(), prec, outs.data(), 1, ln.stream);
    if (rc == BLAST_OK)
        for (size_t i = 0; i < batch.size(); i++)
            if (batch[i]->out_bytes)
                BL_CUDA(cudaMemcpyAsync(batch[i]->out, outs[i], batch[i]->out_bytes, cudaMemcpyDeviceToHost,
                                        ln.stream));
    BL_CUDA(cudaStreamSynchronize(ln.stream));
    if (rc == BLAST_OK && *p->h_err) {  // a bounded device wait gave up
        *p->h_err = 0;
        rc = BLAST_ETIMEOUT;
    }
    return rc;
}

void worker_loop(blast_server *s, int li)
{
    cudaSetDevice(s->lanes[li].plan->device);
    for (;;) {
        std::vector<Job *> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto mine = [&] {
                for (Job *j : s->pending)
                    if (j->plan_idx == li) return true;
                return false;
            };
            s->cv_work.wait(lk, [&] { return s->stop || mine(); });
            if (!mine()) return;  // stopping with nothing left for this lane
            int prec = -1;
            for (auto it = s->pending.begin(); it != s->pending.end() && (int)batch.size() < s->max_slots;) {
                Job *j = *it;
                if (j->plan_idx == li && (prec < 0 || j->prec == prec)) {
                    prec = j->prec;
                    batch.push_back(j);
                    it = s->pending.erase(it);
                } else {
                    ++it;
                }
            }
        }
        std::vector<int> st(batch.size(), run_batch(s, li, batch));
        if (st[0] != BLAST_OK && batch.size() > 1) {  // isolate the request that failed
            for (size_t i = 0; i < batch.size(); i++) {
                std::vector<Job *> one{batch[i]};
                st[i] = run_batch(s, li, one);
            }
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (size_t i = 0; i < batch.size(); i++) {
                batch[i]->status = st[i];
                batch[i]->done = true;
                s->lanes[li].free_slots.push_back(batch[i]->slot);
                batch[i]->slot = -1;
            }
        }
        s->cv_done.notify_all();
    }
}

}  // namespace

static void free_lanes(blast_server *s)
{
    for (Lane &ln : s->lanes) {
        cudaSetDevice(ln.plan->device);
        if (ln.ring) cudaFree(ln.ring);
        if (ln.stream) cudaStreamDestroy(ln.stream);
        ln.ring = nullptr;
        ln.stream = nullptr;
    }
}

extern "C" int blast_server_create(blast_plan *const *plans, int n_plans, size_t hbm_budget, int max_slots,
                                   blast_server **out)
{
    if (!plans || n_plans < 1 || !out || max_slots < 1 || hbm_budget == 0) return BLAST_EINVAL;
    for (int i = 0; i < n_plans; i++) {
        if (!plans[i]) return BLAST_EINVAL;
        for (int k = 0; k < i; k++)
            if (plans[k] == plans[i]) return BLAST_EINVAL;  // a plan's work space serves one lane
    }
    auto *s = new blast_server;
    s->budget = hbm_budget;
    s->max_slots = max_slots;
    s->max_pending = (size_t)16 * max_slots;
    s->lanes.resize(n_plans);
    size_t total = 0;
    int rc = BLAST_OK;
    for (int i = 0; i < n_plans && !rc; i++) {
        Lane &ln = s->lanes[i];
        blast_plan *p = plans[i];
        ln.plan = p;
        const int ntr = p->max_clust + p->max_lens;
        ln.in_doubles = ((size_t)ntr * (p->X + p->Q) + p->X + p->Q + 2 * 1024 + 31) / 32 * 32;
        ln.slot_doubles = ln.in_doubles + ((size_t)blast_npairs(p->max_clust, p->max_lens) * p->L + 31) / 32 * 32;
        const int nslots = 2 * max_slots;  // one batch running, one forming
        size_t ws_bytes = 0;
        if (cudaSetDevice(p->device) != cudaSuccess ||
            cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            rc = BLAST_EDEVICE;
        } else if (cudaMalloc(&ln.ring, sizeof(double) * ln.slot_doubles * nslots) != cudaSuccess) {
            cudaGetLastError();
            ln.ring = nullptr;
            rc = BLAST_ENOMEM;
        } else if ((rc = plan_reserve(p, max_slots, &ws_bytes)) == BLAST_OK) {
            ln.reserved = sizeof(double) * ln.slot_doubles * nslots + ws_bytes;
            total += ln.reserved;
            for (int k = nslots - 1; k >= 0; k--) ln.free_slots.push_back(k);
        }
    }
    if (!rc && total > hbm_budget) rc = BLAST_ENOMEM;  // the reservation does not fit the budget
    if (rc) {
        free_lanes(s);
        delete s;
        return rc;
    }
    for (int i = 0; i < n_plans; i++) s->lanes[i].worker = std::thread(worker_loop, s, i);
    *out = s;
    return BLAST_OK;
}

extern "C" size_t blast_server_reserved(const blast_server *s)
{
    if (!s) return 0;
    size_t t = 0;
    for (const Lane &ln : s->lanes) t += ln.reserved;
    return t;
}

extern "C" int blast_submit(blast_server *s, int plan_idx, const blast_request *req, int precision, uint64_t *ticket)
{
    if (!s || !req || !ticket || plan_idx < 0 || plan_idx >= (int)s->lanes.size()) return BLAST_EINVAL;
    if (precision < BLAST_FP64 || precision > BLAST_BF16S) return BLAST_EINVAL;
    blast_plan *p = s->lanes[plan_idx].plan;
    if (req->n_clust < 0 || req->n_lens < 0 || req->n_clust + req->n_lens < 1 || req->n_clust > p->max_clust ||
        req->n_lens > p->max_lens || req->n_ptab < 3 || req->n_ptab > 1024 ||
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
    {
        // admission: a free device slot of the plan's ring (the reserved bytes)
        std::lock_guard<std::mutex> lk(s->mu);
        Lane &ln = s->lanes[plan_idx];
        if (ln.free_slots.empty() || s->pending.size() >= s->max_pending) {
            rc = BLAST_EBUSY;
        } else {
            j->slot = ln.free_slots.back();
            ln.free_slots.pop_back();
            j->ticket = s->next_ticket++;
            s->jobs[j->ticket] = j;
            s->pending.push_back(j);
            *ticket = j->ticket;
        }
    }
    if (rc) {
        release(s, j);
        return rc;
    }
    s->cv_work.notify_all();
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
    for (Lane &ln : s->lanes)
        if (ln.worker.joinable()) ln.worker.join();  // waiting requests are evaluated first
    for (auto &kv : s->jobs) release(s, kv.second);
    free_lanes(s);
    delete s;
    return BLAST_OK;
}
