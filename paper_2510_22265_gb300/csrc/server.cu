// Serving loop of the GB300 EBCC library: continuous batching of compress and
// decompress requests with admission by an HBM budget.
//
// Requests are copied at submit time and queued FIFO.  Two worker threads, each
// with its own CUDA stream and device workspace, take the oldest requests that
// fit the budget (up to max_batch per group), run them, and complete their
// tickets; a request that arrives while groups are on the GPU is admitted as
// soon as budget and a worker free up, so the two streams keep the device
// busy with overlapping work.  Latency is measured from submit to completion.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string.h>
#include <thread>
#include <vector>
#include "ebcc_internal.cuh"

namespace {
using clk = std::chrono::steady_clock;

struct Job {
    uint64_t ticket;
    ebcc_request req;
    std::vector<uint8_t> in;   // copied field bytes or stream
    size_t footprint = 0;
    int state = 0;             // 0 queued, 1 running, 2 done
    ebcc_result res;
    clk::time_point t_submit, t_start;
};

}  // namespace

struct ebcc_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Job> jobs;
    uint64_t next = 1;
    size_t budget = 0, in_use = 0;
    int max_batch = 64;
    ebcc_params p;
    bool stop = false;
    int device = 0;
    std::vector<std::thread> workers;
};

namespace {

size_t footprint(const ebcc_request &r, const ebcc_params &p) {
    size_t n = r.ny * r.nx;
    if (r.kind == EBCC_REQ_COMPRESS) return ebcc_compress_footprint(r.ny, r.nx, p) + ebcc_max_stream_bytes(r.ny, r.nx);
    return n * 4 * 6 + r.stream_len + spiht_work_bytes(n) + (1 << 20);
}

void run_job(ebcc_server *s, Job &j, Arena &arena, cudaStream_t st) {
    ebcc_result &res = j.res;
    memset(&res, 0, sizeof(res));
    const size_t n = j.req.ny * j.req.nx;
    if (j.req.kind == EBCC_REQ_COMPRESS) {
        float *dx = nullptr;
        uint8_t *dout = nullptr;
        size_t cap = ebcc_max_stream_bytes(j.req.ny, j.req.nx), len = 0;
        int rc = EBCC_OK;
        if (cudaMalloc(&dx, n * 4) != cudaSuccess || cudaMalloc(&dout, cap) != cudaSuccess) rc = EBCC_ENOMEM;
        if (!rc && cudaMemcpyAsync(dx, j.in.data(), n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = EBCC_ECUDA;
        if (!rc)
            rc = ebcc_compress_arena(arena, dx, j.req.ny, j.req.nx, j.req.bound, j.req.bound_kind, s->p, dout, cap,
                                     &len, nullptr, st);
        if (!rc) {
            res.stream = (uint8_t *)malloc(len);
            if (!res.stream) rc = EBCC_ENOMEM;
            else if (cudaMemcpyAsync(res.stream, dout, len, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                     cudaStreamSynchronize(st) != cudaSuccess) rc = EBCC_ECUDA;
            res.stream_len = len;
        }
        if (rc && res.stream) { free(res.stream); res.stream = nullptr; res.stream_len = 0; }
        cudaFree(dx);
        cudaFree(dout);
        res.status = rc;
    } else {
        uint8_t *ds = nullptr;
        float *dout = nullptr;
        int rc = EBCC_OK;
        if (cudaMalloc(&ds, j.in.size() + 16) != cudaSuccess || cudaMalloc(&dout, n * 4) != cudaSuccess)
            rc = EBCC_ENOMEM;
        if (!rc && cudaMemcpyAsync(ds, j.in.data(), j.in.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
            rc = EBCC_ECUDA;
        if (!rc) rc = ebcc_decompress_arena(arena, ds, j.in.data(), j.in.size(), j.req.ny, j.req.nx, dout, st);
        if (!rc) {
            res.field = (float *)malloc(n * 4);
            if (!res.field) rc = EBCC_ENOMEM;
            else if (cudaMemcpyAsync(res.field, dout, n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                     cudaStreamSynchronize(st) != cudaSuccess) rc = EBCC_ECUDA;
        }
        if (rc && res.field) { free(res.field); res.field = nullptr; }
        cudaFree(ds);
        cudaFree(dout);
        res.status = rc;
    }
}

void worker(ebcc_server *s) {
    cudaSetDevice(s->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    Arena arena;
    for (;;) {
        std::vector<uint64_t> group;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                if (s->stop && s->queue.empty()) return true;
                return !s->queue.empty() && s->jobs[s->queue.front()].footprint + s->in_use <= s->budget;
            });
            if (s->queue.empty()) break;
            // admit the oldest requests that fit
            while (!s->queue.empty() && (int)group.size() < s->max_batch) {
                Job &j = s->jobs[s->queue.front()];
                if (s->in_use + j.footprint > s->budget) break;
                s->in_use += j.footprint;
                j.state = 1;
                j.t_start = clk::now();
                group.push_back(j.ticket);
                s->queue.pop_front();
            }
        }
        for (uint64_t t : group) {
            Job *jp;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                jp = &s->jobs[t];
            }
            run_job(s, *jp, arena, st);
            std::lock_guard<std::mutex> lk(s->mu);
            auto now = clk::now();
            jp->res.latency_s = std::chrono::duration<double>(now - jp->t_submit).count();
            jp->res.queue_s = std::chrono::duration<double>(jp->t_start - jp->t_submit).count();
            jp->state = 2;
            s->in_use -= jp->footprint;
            jp->in.clear();
            jp->in.shrink_to_fit();
            s->cv_done.notify_all();
            s->cv_work.notify_all();
        }
    }
    if (arena.base) cudaFree(arena.base);
    cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

int ebcc_server_create(size_t hbm_budget_bytes, int max_batch, const ebcc_params *p, ebcc_server **out) {
    if (!out || hbm_budget_bytes == 0 || max_batch < 0) return EBCC_EINVAL;
    ebcc_server *s = new (std::nothrow) ebcc_server();
    if (!s) return EBCC_ENOMEM;
    s->budget = hbm_budget_bytes;
    s->max_batch = max_batch ? max_batch : 64;
    if (p) s->p = *p; else ebcc_params_default(&s->p);
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return EBCC_ECUDA; }
    for (int k = 0; k < 2; k++) s->workers.emplace_back(worker, s);
    *out = s;
    return EBCC_OK;
}

int ebcc_server_submit(ebcc_server *s, const ebcc_request *r, uint64_t *ticket) {
    if (!s || !r || !ticket) return EBCC_EINVAL;
    if (r->ny == 0 || r->nx == 0 || r->ny * r->nx >= 0x7FFFFFFFull) return EBCC_EINVAL;
    if (r->kind != EBCC_REQ_COMPRESS && r->kind != EBCC_REQ_DECOMPRESS) return EBCC_EINVAL;
    if (r->kind == EBCC_REQ_COMPRESS && (!r->field || !(r->bound > 0))) return EBCC_EINVAL;
    if (r->kind == EBCC_REQ_DECOMPRESS && (!r->stream || r->stream_len < HDR_BYTES)) return EBCC_EINVAL;
    Job j;
    j.req = *r;
    j.footprint = footprint(*r, s->p);
    if (j.footprint > s->budget) return EBCC_EBUDGET;
    if (r->kind == EBCC_REQ_COMPRESS) {
        const uint8_t *b = (const uint8_t *)r->field;
        j.in.assign(b, b + r->ny * r->nx * 4);
    } else {
        j.in.assign(r->stream, r->stream + r->stream_len);
    }
    j.t_submit = clk::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return EBCC_EINVAL;
    j.ticket = s->next++;
    *ticket = j.ticket;
    s->jobs.emplace(j.ticket, std::move(j));
    s->queue.push_back(*ticket);
    s->cv_work.notify_one();
    return EBCC_OK;
}

int ebcc_server_poll(ebcc_server *s, uint64_t ticket, double timeout_s, ebcc_result *r) {
    if (!s || !r) return EBCC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return EBCC_EINVAL;
    if (it->second.state != 2 && timeout_s > 0) {
        s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                            [&] { return s->jobs.count(ticket) && s->jobs[ticket].state == 2; });
        it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return EBCC_EINVAL;
    }
    if (it->second.state != 2) return EBCC_ETIMEOUT;
    *r = it->second.res;
    s->jobs.erase(it);
    return EBCC_OK;
}

int ebcc_server_cancel(ebcc_server *s, uint64_t ticket) {
    if (!s) return EBCC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end() || it->second.state != 0) return EBCC_EINVAL;
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
        if (*q == ticket) { s->queue.erase(q); break; }
    s->jobs.erase(it);
    s->cv_work.notify_all();
    return EBCC_OK;
}

int ebcc_server_destroy(ebcc_server *s) {
    if (!s) return EBCC_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto &kv : s->jobs) {
        free(kv.second.res.stream);
        free(kv.second.res.field);
    }
    delete s;
    return EBCC_OK;
}

}  // extern "C"
