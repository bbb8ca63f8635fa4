// Serving loop of the GB300 EBCC library: continuous batching of compress and
// decompress requests with admission by an HBM budget.
//
// Requests are copied at submit time and queued FIFO.  Two worker threads, each
// with its own CUDA stream and engine (device workspace), take the oldest
// requests that fit the budget (up to max_batch per group) and run the group's
// compressions as one batch and its decompressions as another (every kernel
// covers all fields of the batch); a request that arrives while groups are on
// the GPU is admitted as soon as budget and a worker free up, so the two
// streams keep the device busy with overlapping work.  Latency is measured
// from submit to completion.
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
    if (r.kind == EBCC_REQ_COMPRESS) return ebcc_compress_footprint(r.ny, r.nx, p) + ebcc_max_stream_bytes(r.ny, r.nx) + n * 4;
    return n * 4 * 21 + r.stream_len + spiht_work_bytes(n) + (1 << 20);
}

// One admitted group: its compress requests run as one batch, its decompress
// requests as another, on this worker's stream and engine.
void run_group(ebcc_server *s, const std::vector<Job *> &jobs, EbccEngine *eng, cudaStream_t st) {
    std::vector<Job *> cj, dj;
    for (Job *j : jobs) {
        memset(&j->res, 0, sizeof(j->res));
        (j->req.kind == EBCC_REQ_COMPRESS ? cj : dj).push_back(j);
    }
    if (!cj.empty()) {
        const int n = (int)cj.size();
        std::vector<float *> dx(n, nullptr);
        std::vector<uint8_t *> dout(n, nullptr);
        std::vector<ebcc_field_desc> fd(n);
        std::vector<ebcc_out_desc> od(n);
        int rc = EBCC_OK;
        for (int k = 0; k < n && !rc; k++) {
            const ebcc_request &q = cj[k]->req;
            const size_t cap = ebcc_max_stream_bytes(q.ny, q.nx);
            if (cudaMalloc(&dx[k], q.ny * q.nx * 4) != cudaSuccess || cudaMalloc(&dout[k], cap) != cudaSuccess) {
                rc = EBCC_ENOMEM;
                break;
            }
            if (cudaMemcpyAsync(dx[k], cj[k]->in.data(), q.ny * q.nx * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
                rc = EBCC_ECUDA;
            fd[k] = ebcc_field_desc{dx[k], q.ny, q.nx, q.bound, q.bound_kind};
            memset(&od[k], 0, sizeof(od[k]));
            od[k].stream = dout[k];
            od[k].capacity = cap;
        }
        if (!rc) rc = engine_compress(eng, fd.data(), n, od.data(), s->p, st);
        for (int k = 0; k < n; k++) {
            ebcc_result &res = cj[k]->res;
            int r = rc ? rc : od[k].status;
            if (!r) {
                res.stream = (uint8_t *)malloc(od[k].len ? od[k].len : 1);
                if (!res.stream) r = EBCC_ENOMEM;
                else if (cudaMemcpyAsync(res.stream, dout[k], od[k].len, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                         cudaStreamSynchronize(st) != cudaSuccess) r = EBCC_ECUDA;
                res.stream_len = od[k].len;
            }
            if (r && res.stream) { free(res.stream); res.stream = nullptr; res.stream_len = 0; }
            res.status = r;
            cudaFree(dx[k]);
            cudaFree(dout[k]);
        }
    }
    if (!dj.empty()) {
        const int n = (int)dj.size();
        std::vector<uint8_t *> ds(n, nullptr);
        std::vector<float *> dout(n, nullptr);
        std::vector<ebcc_stream_desc> sd(n);
        std::vector<int> status(n, EBCC_OK);
        int rc = EBCC_OK;
        for (int k = 0; k < n && !rc; k++) {
            const ebcc_request &q = dj[k]->req;
            if (cudaMalloc(&ds[k], dj[k]->in.size() + 16) != cudaSuccess || cudaMalloc(&dout[k], q.ny * q.nx * 4) != cudaSuccess) {
                rc = EBCC_ENOMEM;
                break;
            }
            if (cudaMemcpyAsync(ds[k], dj[k]->in.data(), dj[k]->in.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
                rc = EBCC_ECUDA;
            sd[k] = ebcc_stream_desc{ds[k], dj[k]->in.size(), q.ny, q.nx};
        }
        if (!rc) rc = engine_decompress(eng, sd.data(), n, dout.data(), status.data(), st);
        for (int k = 0; k < n; k++) {
            ebcc_result &res = dj[k]->res;
            const ebcc_request &q = dj[k]->req;
            int r = rc ? rc : status[k];
            if (!r) {
                res.field = (float *)malloc(q.ny * q.nx * 4);
                if (!res.field) r = EBCC_ENOMEM;
                else if (cudaMemcpyAsync(res.field, dout[k], q.ny * q.nx * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                         cudaStreamSynchronize(st) != cudaSuccess) r = EBCC_ECUDA;
            }
            if (r && res.field) { free(res.field); res.field = nullptr; }
            res.status = r;
            cudaFree(ds[k]);
            cudaFree(dout[k]);
        }
    }
}

void worker(ebcc_server *s) {
    cudaSetDevice(s->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    EbccEngine *eng = engine_create();
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
        std::vector<Job *> jp;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (uint64_t t : group) jp.push_back(&s->jobs[t]);
        }
        if (eng) run_group(s, jp, eng, st);
        else
            for (Job *j : jp) { memset(&j->res, 0, sizeof(j->res)); j->res.status = EBCC_ENOMEM; }
        std::lock_guard<std::mutex> lk(s->mu);
        auto now = clk::now();
        for (Job *j : jp) {
            j->res.latency_s = std::chrono::duration<double>(now - j->t_submit).count();
            j->res.queue_s = std::chrono::duration<double>(j->t_start - j->t_submit).count();
            j->state = 2;
            s->in_use -= j->footprint;
            j->in.clear();
            j->in.shrink_to_fit();
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    engine_destroy(eng);
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
