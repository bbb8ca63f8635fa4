// Serving loop of the GB300 EBCC library: continuous batching of compress and
// decompress requests with admission by an HBM budget.
//
// Requests are copied at submit time and queued FIFO.  Four worker threads
// (EBCC_SERVER_WORKERS, 1..8), each with its own CUDA stream, batch engine
// and device buffers (kept and grown, never allocated per request), take the
// oldest requests that fit the budget (up to max_batch per group) and run the
// group's decompressions as one batch, publishing them at once, then its
// compressions as another (every kernel covers all fields of the batch).  A
// request that arrives while groups are on the GPU is admitted as soon as
// budget and a worker free up, so the streams keep the device busy with
// overlapping work: the latency-bound steps of one group (the MQ coders'
// longest chains, SPIHT's one CTA per field) leave room for the others'.  On
// 721 x 1440 requests four workers gave the lowest p99 (two: 77 ms, three:
// 57 ms, four: 50 ms, six: 63 ms at 75% of capacity).  Latency is measured
// from submit to completion.
//
// Intake: a group's request bytes enter the device through a request ring in
// page-locked host memory that the GPU reads directly.  The worker launches
// the intake kernel first; the kernel waits on the ring's doorbell -- a
// sequence number the host publishes after writing the group -- with a time
// limit, then copies every request into the worker's device buffers.  A wait
// that runs out ends the kernel with EBCC_ETIMEOUT in a status word the host
// reads, so nothing hangs and the context stays usable.  Results come back
// with one copy per request into page-locked staging and one synchronisation
// per group.
#include <atomic>
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

// one request's bytes: ring offset, device buffer offset, length (16-byte units)
struct IntakeJob {
    long long src, dst, n16;
};

__device__ __forceinline__ unsigned long long load_acquire_sys(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until *bell >= want (at most timeout_ns), then
// copies the jobs listed at the start of the ring into dst.  On a timeout the
// CTA copies nothing and sets *status = EBCC_ETIMEOUT.
__global__ void __launch_bounds__(256) intake_kernel(const uint8_t *ring, uint8_t *dst, int njobs,
                                                     const unsigned long long *bell, unsigned long long want,
                                                     unsigned long long timeout_ns, int *status) {
    __shared__ int go;
    if (threadIdx.x == 0) {
        const unsigned long long t0 = global_ns();
        int ok = 0;
        // the clock ends the wait; the poll count is a second limit in case it
        // does not advance (a poll takes well over 64 ns)
        const unsigned long long max_polls = timeout_ns / 64 + 4096;
        for (unsigned long long it = 0; it < max_polls; it++) {
            if (load_acquire_sys(bell) >= want) { ok = 1; break; }
            if (global_ns() - t0 > timeout_ns) break;
            __nanosleep(500);
        }
        if (!ok) atomicExch(status, EBCC_ETIMEOUT);
        go = ok;
    }
    __syncthreads();
    if (!go) return;
    const IntakeJob *jobs = (const IntakeJob *)ring;
    for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
        const IntakeJob jb = jobs[j];
        const uint4 *s = (const uint4 *)(ring + jb.src);
        uint4 *d = (uint4 *)(dst + jb.dst);
        for (long long k = threadIdx.x; k < jb.n16; k += blockDim.x) d[k] = s[k];
    }
}

// page-locked host memory the device reads (mapped), grown on demand
struct MappedBuf {
    uint8_t *host = nullptr, *dev = nullptr;
    size_t cap = 0;
    int grow(size_t need) {
        if (cap >= need) return EBCC_OK;
        if (host) cudaFreeHost(host);
        host = dev = nullptr;
        cap = 0;
        size_t c = need + need / 4 + 4096;
        if (cudaHostAlloc((void **)&host, c, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) return EBCC_ENOMEM;
        if (cudaHostGetDevicePointer((void **)&dev, host, 0) != cudaSuccess) return EBCC_ECUDA;
        cap = c;
        return EBCC_OK;
    }
    void release() {
        if (host) cudaFreeHost(host);
        host = dev = nullptr;
        cap = 0;
    }
};

// The request ring of one worker: the jobs table and the request bytes, the
// doorbell, and the kernel's status word.
struct Intake {
    MappedBuf ring, bell;
    int *status = nullptr;  // device
    unsigned long long seq = 0;
    int init() {
        RC(bell.grow(64));
        memset(bell.host, 0, 64);
        if (!status) CK(cudaMalloc(&status, sizeof(int)));
        return EBCC_OK;
    }
    void release() {
        ring.release();
        bell.release();
        if (status) cudaFree(status);
        status = nullptr;
    }
};

size_t up16(size_t v) { return (v + 15) & ~(size_t)15; }
size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// One intake round: the n byte ranges src[k] (host, len[k] bytes) land at
// dst + off[k] (device, 16-byte aligned).  The kernel is launched before the
// host writes the ring, so it waits on the doorbell; publish = 0 leaves the
// doorbell unset (the kernel's wait then runs out: a diagnostic).  Returns the
// kernel's status after a synchronise of st.
int intake_round(Intake &in, const std::vector<const uint8_t *> &src, const std::vector<size_t> &len,
                 const std::vector<size_t> &off, uint8_t *dst, double wait_s, int publish, cudaStream_t st) {
    const int n = (int)src.size();
    RC(in.init());
    size_t pos = up256((size_t)n * sizeof(IntakeJob));
    std::vector<IntakeJob> jobs(n);
    for (int k = 0; k < n; k++) {
        jobs[k] = IntakeJob{(long long)pos, (long long)off[k], (long long)(up16(len[k]) / 16)};
        pos += up256(len[k]);
    }
    RC(in.ring.grow(pos));
    CK(cudaMemsetAsync(in.status, 0, sizeof(int), st));
    const unsigned long long want = ++in.seq;
    const unsigned long long tns = (unsigned long long)(wait_s * 1e9);
    int grid = n < 1 ? 1 : (n > 304 ? 304 : n);
    PROF("intake_kernel", st, 0.0,
         intake_kernel<<<grid, 256, 0, st>>>(in.ring.dev, dst, n, (const unsigned long long *)in.bell.dev, want, tns,
                                             in.status));
    CK(cudaGetLastError());
    memcpy(in.ring.host, jobs.data(), (size_t)n * sizeof(IntakeJob));
    for (int k = 0; k < n; k++) memcpy(in.ring.host + jobs[k].src, src[k], len[k]);
    if (publish) {
        std::atomic_thread_fence(std::memory_order_seq_cst);
        reinterpret_cast<std::atomic<unsigned long long> *>(in.bell.host)->store(want, std::memory_order_release);
    }
    int status = EBCC_OK;
    CK(cudaMemcpyAsync(&status, in.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return status;
}

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
    double intake_wait_s = 2.0;
    std::vector<std::thread> workers;
};

namespace {

size_t footprint(const ebcc_request &r, const ebcc_params &p) {
    size_t n = r.ny * r.nx;
    if (r.kind == EBCC_REQ_COMPRESS) return ebcc_compress_footprint(r.ny, r.nx, p) + ebcc_max_stream_bytes(r.ny, r.nx) + n * 4;
    return n * 4 * 21 + r.stream_len + spiht_work_bytes(n) + (1 << 20);
}

// a worker's kept resources
struct WorkerRes {
    cudaStream_t st = nullptr;
    EbccEngine *eng = nullptr;
    Arena io;          // device: the group's inputs and outputs
    Intake in;
    uint8_t *back = nullptr;  // page-locked: results on their way back
    size_t back_cap = 0;
    int back_grow(size_t need) {
        if (back_cap >= need) return EBCC_OK;
        if (back) cudaFreeHost(back);
        back = nullptr;
        back_cap = 0;
        size_t c = need + need / 4 + 4096;
        if (cudaHostAlloc((void **)&back, c, cudaHostAllocDefault) != cudaSuccess) return EBCC_ENOMEM;
        back_cap = c;
        return EBCC_OK;
    }
};

void fail_all(const std::vector<Job *> &js, int rc) {
    for (Job *j : js) j->res.status = rc;
}

// the group's compressions as one batch
void run_compress(ebcc_server *s, const std::vector<Job *> &cj, WorkerRes &w) {
    const int n = (int)cj.size();
    std::vector<size_t> in_off(n), out_off(n), cap(n), len(n);
    std::vector<const uint8_t *> src(n);
    size_t pos = 0;
    for (int k = 0; k < n; k++) {
        const ebcc_request &q = cj[k]->req;
        in_off[k] = pos;
        len[k] = q.ny * q.nx * 4;
        src[k] = cj[k]->in.data();
        pos += up256(len[k]);
    }
    for (int k = 0; k < n; k++) {
        const ebcc_request &q = cj[k]->req;
        cap[k] = ebcc_max_stream_bytes(q.ny, q.nx);
        out_off[k] = pos;
        pos += up256(cap[k]);
    }
    int rc = arena_reserve(w.io, pos + 256);
    if (!rc) rc = intake_round(w.in, src, len, in_off, w.io.base, s->intake_wait_s, 1, w.st);
    if (rc) { fail_all(cj, rc); return; }
    std::vector<ebcc_field_desc> fd(n);
    std::vector<ebcc_out_desc> od(n);
    for (int k = 0; k < n; k++) {
        const ebcc_request &q = cj[k]->req;
        fd[k] = ebcc_field_desc{(const float *)(w.io.base + in_off[k]), q.ny, q.nx, q.bound, q.bound_kind};
        memset(&od[k], 0, sizeof(od[k]));
        od[k].stream = w.io.base + out_off[k];
        od[k].capacity = cap[k];
    }
    rc = engine_compress(w.eng, fd.data(), n, od.data(), s->p, w.st);
    if (rc) { fail_all(cj, rc); return; }
    // every stream back: one copy each into page-locked staging, one synchronise
    size_t tot = 0;
    std::vector<size_t> boff(n);
    for (int k = 0; k < n; k++) { boff[k] = tot; tot += od[k].status ? 0 : up16(od[k].len); }
    if ((rc = w.back_grow(tot + 16)) != EBCC_OK) { fail_all(cj, rc); return; }
    for (int k = 0; k < n && !rc; k++)
        if (!od[k].status && od[k].len &&
            cudaMemcpyAsync(w.back + boff[k], od[k].stream, od[k].len, cudaMemcpyDeviceToHost, w.st) != cudaSuccess)
            rc = EBCC_ECUDA;
    if (!rc && cudaStreamSynchronize(w.st) != cudaSuccess) rc = EBCC_ECUDA;
    for (int k = 0; k < n; k++) {
        ebcc_result &res = cj[k]->res;
        int r = rc ? rc : od[k].status;
        if (!r) {
            res.stream = (uint8_t *)malloc(od[k].len ? od[k].len : 1);
            if (!res.stream) r = EBCC_ENOMEM;
            else { memcpy(res.stream, w.back + boff[k], od[k].len); res.stream_len = od[k].len; }
        }
        res.status = r;
    }
}

// the group's decompressions as one batch
void run_decompress(ebcc_server *s, const std::vector<Job *> &dj, WorkerRes &w) {
    const int n = (int)dj.size();
    std::vector<size_t> in_off(n), out_off(n), len(n);
    std::vector<const uint8_t *> src(n);
    size_t pos = 0;
    for (int k = 0; k < n; k++) {
        in_off[k] = pos;
        len[k] = dj[k]->in.size();
        src[k] = dj[k]->in.data();
        pos += up256(len[k] + 16);
    }
    for (int k = 0; k < n; k++) {
        const ebcc_request &q = dj[k]->req;
        out_off[k] = pos;
        pos += up256(q.ny * q.nx * 4);
    }
    int rc = arena_reserve(w.io, pos + 256);
    if (!rc) rc = intake_round(w.in, src, len, in_off, w.io.base, s->intake_wait_s, 1, w.st);
    if (rc) { fail_all(dj, rc); return; }
    std::vector<ebcc_stream_desc> sd(n);
    std::vector<float *> dout(n);
    std::vector<int> status(n, EBCC_OK);
    for (int k = 0; k < n; k++) {
        const ebcc_request &q = dj[k]->req;
        sd[k] = ebcc_stream_desc{w.io.base + in_off[k], len[k], q.ny, q.nx};
        dout[k] = (float *)(w.io.base + out_off[k]);
    }
    rc = engine_decompress(w.eng, sd.data(), n, dout.data(), status.data(), w.st);
    if (rc) { fail_all(dj, rc); return; }
    size_t tot = 0;
    std::vector<size_t> boff(n);
    for (int k = 0; k < n; k++) {
        boff[k] = tot;
        tot += status[k] ? 0 : up16(dj[k]->req.ny * dj[k]->req.nx * 4);
    }
    if ((rc = w.back_grow(tot + 16)) != EBCC_OK) { fail_all(dj, rc); return; }
    for (int k = 0; k < n && !rc; k++)
        if (!status[k] && cudaMemcpyAsync(w.back + boff[k], dout[k], dj[k]->req.ny * dj[k]->req.nx * 4,
                                          cudaMemcpyDeviceToHost, w.st) != cudaSuccess)
            rc = EBCC_ECUDA;
    if (!rc && cudaStreamSynchronize(w.st) != cudaSuccess) rc = EBCC_ECUDA;
    for (int k = 0; k < n; k++) {
        ebcc_result &res = dj[k]->res;
        const size_t bytes = dj[k]->req.ny * dj[k]->req.nx * 4;
        int r = rc ? rc : status[k];
        if (!r) {
            res.field = (float *)malloc(bytes);
            if (!res.field) r = EBCC_ENOMEM;
            else memcpy(res.field, w.back + boff[k], bytes);
        }
        res.status = r;
    }
}

// publish finished jobs: latency, budget back, waiters woken
void finish(ebcc_server *s, const std::vector<Job *> &jp) {
    if (jp.empty()) return;
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

// a group's decompressions (short) run first and are published before its
// compressions run, so they do not wait for them
void run_group(ebcc_server *s, const std::vector<Job *> &jobs, WorkerRes &w) {
    std::vector<Job *> cj, dj;
    for (Job *j : jobs) {
        memset(&j->res, 0, sizeof(j->res));
        (j->req.kind == EBCC_REQ_COMPRESS ? cj : dj).push_back(j);
    }
    if (!dj.empty()) run_decompress(s, dj, w);
    finish(s, dj);
    if (!cj.empty()) run_compress(s, cj, w);
    finish(s, cj);
}

void worker(ebcc_server *s) {
    cudaSetDevice(s->device);
    WorkerRes w;
    const bool ok = cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking) == cudaSuccess;
    w.eng = ok ? engine_create() : nullptr;
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
        if (w.eng) {
            run_group(s, jp, w);
        } else {
            for (Job *j : jp) { memset(&j->res, 0, sizeof(j->res)); j->res.status = EBCC_ENOMEM; }
            finish(s, jp);
        }
    }
    engine_destroy(w.eng);
    if (w.io.base) cudaFree(w.io.base);
    w.in.release();
    if (w.back) cudaFreeHost(w.back);
    if (w.st) cudaStreamDestroy(w.st);
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
    // worker threads, each with its own stream and batch engine (EBCC_SERVER_WORKERS, 1..8; 4)
    int nw = 4;
    if (const char *v = getenv("EBCC_SERVER_WORKERS")) nw = atoi(v);
    if (nw < 1 || nw > 8) nw = 4;
    for (int k = 0; k < nw; k++) s->workers.emplace_back(worker, s);
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

int ebcc_intake_check(size_t bytes, double wait_s, int publish, void *stream) {
    if (bytes == 0 || bytes > ((size_t)1 << 30) || !(wait_s > 0) || wait_s > 60) return EBCC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Intake in;
    std::vector<uint8_t> data(bytes);
    for (size_t i = 0; i < bytes; i++) data[i] = (uint8_t)(i * 131 + 7);
    uint8_t *d = nullptr;
    CK(cudaMalloc(&d, up16(bytes) + 256));
    CK(cudaMemsetAsync(d, 0, up16(bytes) + 256, st));
    int rc = intake_round(in, {data.data()}, {bytes}, {0}, d, wait_s, publish, st);
    if (!rc) {  // the bytes arrived unchanged
        std::vector<uint8_t> back(bytes);
        if (cudaMemcpy(back.data(), d, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) rc = EBCC_ECUDA;
        else if (memcmp(back.data(), data.data(), bytes) != 0) rc = EBCC_ECORRUPT;
    }
    cudaFree(d);
    in.release();
    return rc;
}

}  // extern "C"
