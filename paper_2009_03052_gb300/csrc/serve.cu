// serve.cu -- a request loop over device-resident tables: continuous
// batching of sample and estimate requests on a pool of slots.
//
// Every slot is a host thread with its own CUDA stream.  Requests queue in
// arrival order; the first queued request is admitted as soon as a slot is
// idle and its device buffers fit the free device memory (and the caller's
// cap, if one was given), so requests that
// arrive while others run start at once on another slot and their kernels
// overlap on the device.  A request's results depend only on the tables,
// its seed and its sample indices, so they are the same alone or in a mix.
#include <chrono>
#include <condition_variable>
#include <algorithm>
#include <deque>
#include <map>
#include <thread>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    mc_request r{};
    size_t mem = 0;
    int state = 0;  // 0 queued, 1 running, 2 done
    mc_status status = MC_OK;
    std::string error;
    std::vector<uint32_t> nodes;
    std::vector<int32_t> classes;
    std::vector<double> est;
    std::vector<uint64_t> hits;
    Clock::time_point t_submit, t_start, t_done;
};

}  // namespace

struct mc_server {
    std::vector<const mc_tables *> tables;
    size_t budget = 0, in_use = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<int64_t> queue;
    std::map<int64_t, Request> reqs;
    int64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;  // one per slot, created and checked at creation
    ~mc_server()
    {
        for (cudaStream_t s : streams) cudaStreamDestroy(s);
    }
};

namespace mc {

int64_t bucket_count(int64_t n);

// Device bytes a request allocates while it runs (outputs, scratch, and any
// root or star index it creates on first use), from the request and the
// tables it reads: what admission charges it.
static size_t request_memory(const mc_tables *t, const mc_request &r)
{
    const int64_t n = t->g->n;
    const size_t scan = (size_t)((n + 4095) / 4096 + 1) * 16;            // scan tile sums
    const size_t index = (size_t)n * 16 + (size_t)(bucket_count(n) + 1) * 4 + scan + 64;  // prefix + buckets
    const size_t small = 4096;                                            // flags, counters
    if (r.kind == MC_REQ_SAMPLE) {
        size_t m = (size_t)std::max<int64_t>(r.count, 1) * ((size_t)r.h + 1) * 4 + small;
        if (r.unrooted_shape >= 0 || !t->prefix[r.h]) m += index;  // a shape's index is per call
        return m;
    }
    const mc_estimate_params &p = r.est;
    const int h = p.h;
    const int ncls = mc_num_classes(h);
    const size_t cls = (size_t)std::max(ncls, 1) * 8;
    size_t m = small + 3 * cls;                                           // histogram, sigma, estimates
    if (!t->prefix[h]) m += index;
    if (p.mode == MC_EST_AGS) {
        // a root index per treelet shape it samples from (at most all of
        // them), one shape-total pass, and the class ids and part table of
        // one launch (the current treelet's run and a short one per other)
        const int nu = mc_num_unrooted(h);
        const int64_t bmax = p.batch > 0 ? p.batch : (int64_t)1 << 22;
        const int64_t ahead = std::min<int64_t>(bmax, 4096);
        m += (size_t)std::max(nu, 1) * index + index + (size_t)(bmax + (int64_t)nu * ahead) * 4 +
             (size_t)nu * 128;
    }
    if (p.star_samples > 0 && !t->g->star_prefix[h]) m += index + cls;
    return m;
}

// Free device memory now (0 if the query fails).
static size_t free_device_memory()
{
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return free_b;
}

static void run_request(mc_server *sv, Request &q, cudaStream_t s)
{
    const mc_tables *t = sv->tables[q.r.table];
    if (q.r.kind == MC_REQ_SAMPLE) {
        const int64_t n = q.r.count;
        Arena out(true);  // stream-ordered device outputs, freed when the request is done
        out.stream = s;
        uint32_t *dn = out.get<uint32_t>((size_t)std::max<int64_t>(n, 1) * q.r.h);
        int32_t *dc = out.get<int32_t>((size_t)std::max<int64_t>(n, 1));
        mc_status st = mc_sample_range(t, q.r.h, q.r.unrooted_shape, q.r.node_lo, q.r.node_hi, q.r.seed,
                                       q.r.first_index, n, dn, nullptr, nullptr, dc, (void *)s);
        if (st != MC_OK) throw Error(st, mc_last_error());
        q.nodes.resize((size_t)n * q.r.h);
        q.classes.resize((size_t)n);
        if (n) {
            MC_CUDA(cudaMemcpyAsync(q.nodes.data(), dn, q.nodes.size() * 4, cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaMemcpyAsync(q.classes.data(), dc, q.classes.size() * 4, cudaMemcpyDeviceToHost, s));
        }
        MC_CUDA(cudaStreamSynchronize(s));
    } else {
        const int nc = mc_num_classes(q.r.est.h);
        if (nc < 0) throw Error(MC_E_INVALID, mc_last_error());
        q.est.assign((size_t)nc, 0.0);
        q.hits.assign((size_t)nc, 0);
        mc_status st = mc_estimate_counts(t, &q.r.est, q.est.data(), q.hits.data(), nullptr, (void *)s);
        if (st != MC_OK) throw Error(st, mc_last_error());
    }
}

// Admission of the head of the queue: it fits the caller's cap (if any)
// next to the running requests, and the device's free memory right now
// still holds it on top of what the running requests were charged (they
// may not have allocated it yet).  With nothing running it is admitted
// regardless: a request larger than the device then fails alone with
// MC_E_NOMEM.
static bool admissible(const mc_server *sv, size_t mem)
{
    if (sv->in_use == 0) return true;
    if (sv->budget && sv->in_use + mem > sv->budget) return false;
    const size_t free_b = free_device_memory();
    return free_b > sv->in_use && mem <= free_b - sv->in_use;
}

static void worker(mc_server *sv, cudaStream_t s)
{
    cudaSetDevice(sv->device);
    for (;;) {
        int64_t id = 0;
        {
            std::unique_lock<std::mutex> lock(sv->mu);
            // memory freed by others (not only by this server) admits a
            // waiting request at the next poll
            while (!sv->stop) {
                if (!sv->queue.empty() && admissible(sv, sv->reqs.at(sv->queue.front()).mem)) break;
                sv->cv.wait_for(lock, std::chrono::milliseconds(2));
            }
            if (sv->stop) break;
            id = sv->queue.front();
            sv->queue.pop_front();
            Request &q = sv->reqs.at(id);
            sv->in_use += q.mem;
            q.state = 1;
            q.t_start = Clock::now();
        }
        Request *qp;
        {
            std::lock_guard<std::mutex> lock(sv->mu);
            qp = &sv->reqs.at(id);
        }
        mc_status st = guarded([&] { run_request(sv, *qp, s); });
        {
            std::lock_guard<std::mutex> lock(sv->mu);
            qp->status = st;
            if (st != MC_OK) qp->error = mc_last_error();
            qp->state = 2;
            qp->t_done = Clock::now();
            sv->in_use -= qp->mem;
        }
        sv->cv.notify_all();
    }
}

}  // namespace mc

using namespace mc;

extern "C" mc_status mc_server_create(const mc_tables *const *tables, int n_tables, int slots, size_t memory_budget,
                                      mc_server **out)
{
    if (out) *out = nullptr;
    mc_server *sv = nullptr;
    mc_status st = guarded([&] {
        MC_REQUIRE(out && tables && n_tables >= 1 && slots >= 1 && slots <= 64, "bad server arguments");
        sv = new mc_server();
        for (int i = 0; i < n_tables; ++i) {
            MC_REQUIRE(tables[i], "NULL tables");
            sv->tables.push_back(tables[i]);
        }
        MC_CUDA(cudaGetDevice(&sv->device));
        sv->budget = memory_budget;
        for (int i = 0; i < slots; ++i) {
            cudaStream_t s = nullptr;
            MC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            sv->streams.push_back(s);
        }
        for (int i = 0; i < slots; ++i) sv->workers.emplace_back(worker, sv, sv->streams[i]);
    });
    if (st != MC_OK) {
        if (sv) {  // stop the workers started before the failure
            {
                std::lock_guard<std::mutex> lock(sv->mu);
                sv->stop = true;
            }
            sv->cv.notify_all();
            for (auto &w : sv->workers) w.join();
        }
        delete sv;
        return st;
    }
    *out = sv;
    return MC_OK;
}

extern "C" mc_status mc_server_submit(mc_server *sv, const mc_request *r, int64_t *id)
{
    return guarded([&] {
        MC_REQUIRE(sv && r && id, "NULL argument");
        MC_REQUIRE(r->table >= 0 && r->table < (int)sv->tables.size(), "table index out of range");
        const mc_tables *t = sv->tables[r->table];
        if (r->kind == MC_REQ_SAMPLE) {
            MC_REQUIRE(r->h >= 2 && r->h <= t->k && r->count >= 0, "bad sample request");
        } else {
            MC_REQUIRE(r->kind == MC_REQ_ESTIMATE, "unknown request kind");
            MC_REQUIRE(r->est.h >= 2 && r->est.h <= t->k, "bad estimate request");
        }
        const size_t mem = request_memory(t, *r);  // may build the class catalogue: outside the lock
        std::lock_guard<std::mutex> lock(sv->mu);
        const int64_t i = sv->next_id++;
        Request &q = sv->reqs[i];
        q.r = *r;
        q.mem = mem;
        q.t_submit = Clock::now();
        sv->queue.push_back(i);
        *id = i;
        sv->cv.notify_all();
    });
}

extern "C" mc_status mc_server_wait(mc_server *sv, int64_t id, uint32_t *nodes, int32_t *classes, double *est,
                                    uint64_t *hits, double *queue_us, double *latency_us)
{
    Request q;
    mc_status st = guarded([&] {
        MC_REQUIRE(sv, "server is NULL");
        std::unique_lock<std::mutex> lock(sv->mu);
        auto it = sv->reqs.find(id);
        MC_REQUIRE(it != sv->reqs.end(), "unknown request id");
        sv->cv.wait(lock, [&] { return sv->reqs.at(id).state == 2; });
        q = std::move(sv->reqs.at(id));
        sv->reqs.erase(id);
    });
    if (st != MC_OK) return st;
    if (q.status != MC_OK) {
        set_last_error(q.error);
        return q.status;
    }
    if (nodes && !q.nodes.empty()) std::copy(q.nodes.begin(), q.nodes.end(), nodes);
    if (classes && !q.classes.empty()) std::copy(q.classes.begin(), q.classes.end(), classes);
    if (est && !q.est.empty()) std::copy(q.est.begin(), q.est.end(), est);
    if (hits && !q.hits.empty()) std::copy(q.hits.begin(), q.hits.end(), hits);
    using us = std::chrono::duration<double, std::micro>;
    if (queue_us) *queue_us = us(q.t_start - q.t_submit).count();
    if (latency_us) *latency_us = us(q.t_done - q.t_submit).count();
    return MC_OK;
}

extern "C" void mc_server_free(mc_server *sv)
{
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    for (auto &w : sv->workers) w.join();
    delete sv;
}
