// Host-buffer entry points of the C ABI: fields and streams in host memory.
//
// The library copies them through device buffers it keeps between calls
// (grown on demand, never freed per call), so a call allocates nothing once
// those have reached the size of the largest batch seen.  Host buffers that
// are page-locked (cudaHostAlloc, cudaHostRegister, torch pin_memory) and
// mapped into the device's address space are copied by one kernel per
// direction for the whole batch (the SMs read or write the host memory over
// the CPU-GPU link, every field's copy in flight at once); page-locked
// buffers without a device mapping by DMA directly; pageable buffers go
// through two pinned chunks, the CPU filling one while the DMA engine drains
// the other.  The computation is
// the device batch engine (Algorithm 1 on every field of the batch at once).
#include <string.h>
#include <algorithm>
#include <vector>
#include "ebcc_internal.cuh"

namespace {

constexpr size_t kChunk = (size_t)32 << 20;

struct HostIO {
    Arena in, out;                   // device copies of the inputs and of the outputs
    uint8_t *pin[2] = {nullptr, nullptr};
    cudaEvent_t free_ev[2];          // chunk b may be refilled once free_ev[b] has completed
    bool ready = false;
};
HostIO g_io;

int io_init() {
    if (g_io.ready) return EBCC_OK;
    for (int b = 0; b < 2; b++) {
        if (cudaHostAlloc((void **)&g_io.pin[b], kChunk, cudaHostAllocDefault) != cudaSuccess) return EBCC_ENOMEM;
        CK(cudaEventCreateWithFlags(&g_io.free_ev[b], cudaEventDisableTiming));
    }
    g_io.ready = true;
    return EBCC_OK;
}

bool host_pinned(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// the address under which the device reaches a page-locked host buffer
// (null for pageable memory, or where the device cannot map it)
void *host_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Copies between page-locked host buffers and device buffers done by one
// kernel for a whole batch: the SMs read (or write) the host memory through
// its device mapping, every copy of the batch in flight at once, instead of
// one copy-engine transfer per field.
struct CopyJob {
    const uint8_t *src;
    uint8_t *dst;
    unsigned long long n;
};

// grid.y = job; grid.x strides over the job in 16-byte pieces when both ends
// are 16-byte aligned (bytes past the last whole piece, or every byte of an
// unaligned job, one at a time)
__global__ void __launch_bounds__(256) copy_jobs(const CopyJob *__restrict__ jobs, int njobs) {
    const int j = blockIdx.y;
    if (j >= njobs) return;
    const CopyJob c = jobs[j];
    const bool vec = (((uintptr_t)c.src | (uintptr_t)c.dst) & 15) == 0;
    const unsigned long long nv = vec ? c.n / 16 : 0;
    const unsigned long long t0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
    const uint4 *s4 = (const uint4 *)c.src;
    uint4 *d4 = (uint4 *)c.dst;
    for (unsigned long long i = t0; i < nv; i += step) d4[i] = s4[i];
    for (unsigned long long i = nv * 16 + t0; i < c.n; i += step) c.dst[i] = c.src[i];
}

struct JobTable {
    Arena dev;
    std::vector<CopyJob> host;
};
JobTable g_jobs;

// run the queued jobs on st (one small upload of the table, one launch)
int run_jobs(cudaStream_t st) {
    const int n = (int)g_jobs.host.size();
    if (!n) return EBCC_OK;
    if (n > 65535) return EBCC_EINVAL;
    unsigned long long most = 0;
    for (const CopyJob &c : g_jobs.host) most = std::max(most, c.n);
    RC(arena_reserve(g_jobs.dev, sizeof(CopyJob) * (size_t)n + 256));
    CK(cudaMemcpyAsync(g_jobs.dev.base, g_jobs.host.data(), sizeof(CopyJob) * (size_t)n, cudaMemcpyHostToDevice, st));
    // enough CTAs per job that the whole batch fills the GPU a few times over
    unsigned long long gx = (most / 16 + 255) / 256;
    const unsigned long long want = std::max(1ull, 152ull * 8 / (unsigned long long)n);
    gx = std::min(std::max(gx, 1ull), std::max(want, 1ull) * 4);
    copy_jobs<<<dim3((unsigned)std::min(gx, 65535ull), (unsigned)n), 256, 0, st>>>((const CopyJob *)g_jobs.dev.base, n);
    CK(cudaGetLastError());
    g_jobs.host.clear();
    return EBCC_OK;
}

// host -> device, queued on st
int h2d(void *dst, const void *src, size_t n, cudaStream_t st) {
    if (!n) return EBCC_OK;
    if (host_pinned(src)) {
        CK(cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st));
        return EBCC_OK;
    }
    RC(io_init());
    for (size_t off = 0, k = 0; off < n; off += kChunk, k++) {
        const int b = (int)(k & 1);
        const size_t m = std::min(kChunk, n - off);
        CK(cudaEventSynchronize(g_io.free_ev[b]));
        memcpy(g_io.pin[b], (const uint8_t *)src + off, m);
        CK(cudaMemcpyAsync((uint8_t *)dst + off, g_io.pin[b], m, cudaMemcpyHostToDevice, st));
        CK(cudaEventRecord(g_io.free_ev[b], st));
    }
    return EBCC_OK;
}

// device -> host; synchronous for pageable destinations, queued on st for
// pinned ones (the caller synchronises st)
int d2h(void *dst, const void *src, size_t n, cudaStream_t st) {
    if (!n) return EBCC_OK;
    if (host_pinned(dst)) {
        CK(cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, st));
        return EBCC_OK;
    }
    RC(io_init());
    const size_t nk = (n + kChunk - 1) / kChunk;
    auto issue = [&](size_t k) -> int {
        const int b = (int)(k & 1);
        const size_t off = k * kChunk, m = std::min(kChunk, n - off);
        CK(cudaMemcpyAsync(g_io.pin[b], (const uint8_t *)src + off, m, cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(g_io.free_ev[b], st));
        return EBCC_OK;
    };
    RC(issue(0));
    for (size_t k = 0; k < nk; k++) {
        const int b = (int)(k & 1);
        if (k + 1 < nk) {
            // chunk k + 1 lands in the other buffer, whose previous contents
            // (chunk k - 1) were copied out in the last iteration
            RC(issue(k + 1));
        }
        CK(cudaEventSynchronize(g_io.free_ev[b]));
        const size_t off = k * kChunk, m = std::min(kChunk, n - off);
        memcpy((uint8_t *)dst + off, g_io.pin[b], m);
    }
    return EBCC_OK;
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// fields[i] and outs[i] hold host pointers; the batch runs on device copies
int compress_host_locked(const ebcc_field_desc *fields, int n, ebcc_out_desc *outs, const ebcc_params &p,
                         cudaStream_t st) {
    std::vector<size_t> in_off(n, 0), out_off(n, 0), cap(n, 0);
    size_t tin = 0, tout = 0;
    for (int i = 0; i < n; i++) {
        if (api_check_shape(fields[i].ny, fields[i].nx) || !fields[i].field || !outs[i].stream) continue;
        in_off[i] = tin;
        tin += up256(fields[i].ny * fields[i].nx * sizeof(float));
        cap[i] = std::min(outs[i].capacity, ebcc_max_stream_bytes(fields[i].ny, fields[i].nx));
        out_off[i] = tout;
        tout += up256(cap[i]);
    }
    RC(arena_reserve(g_io.in, tin + 256));
    RC(arena_reserve(g_io.out, tout + 256));
    std::vector<ebcc_field_desc> dfd(fields, fields + n);
    std::vector<ebcc_out_desc> dod(outs, outs + n);
    for (int i = 0; i < n; i++) {
        if (!cap[i] && (api_check_shape(fields[i].ny, fields[i].nx) || !fields[i].field || !outs[i].stream)) {
            dfd[i].field = nullptr;  // the engine reports EINVAL for it
            continue;
        }
        float *d = (float *)(g_io.in.base + in_off[i]);
        const size_t bytes = fields[i].ny * fields[i].nx * sizeof(float);
        if (const void *m = host_device_ptr(fields[i].field))
            g_jobs.host.push_back({(const uint8_t *)m, (uint8_t *)d, (unsigned long long)bytes});
        else
            RC(h2d(d, fields[i].field, bytes, st));
        dfd[i].field = d;
        dod[i].stream = g_io.out.base + out_off[i];
        dod[i].capacity = cap[i];
    }
    RC(run_jobs(st));
    const int rc = engine_compress(ebcc_api_engine(), dfd.data(), n, dod.data(), p, st);
    for (int i = 0; i < n; i++) {
        outs[i].status = dod[i].status;
        outs[i].stats = dod[i].stats;
        outs[i].len = dod[i].status ? 0 : dod[i].len;
        if (dod[i].status) continue;
        if (void *m = host_device_ptr(outs[i].stream))
            g_jobs.host.push_back({dod[i].stream, (uint8_t *)m, (unsigned long long)dod[i].len});
        else
            RC(d2h(outs[i].stream, dod[i].stream, dod[i].len, st));
    }
    RC(run_jobs(st));
    CK(cudaStreamSynchronize(st));
    return rc;
}

int decompress_host_locked(const ebcc_stream_desc *streams, int n, float **outs, int *status, cudaStream_t st) {
    std::vector<size_t> in_off(n, 0), out_off(n, 0);
    std::vector<char> ok(n, 0);
    size_t tin = 0, tout = 0;
    for (int i = 0; i < n; i++) {
        status[i] = EBCC_OK;
        if (!streams[i].stream || !outs[i] || api_check_shape(streams[i].ny, streams[i].nx)) {
            status[i] = EBCC_EINVAL;
            continue;
        }
        ok[i] = 1;
        in_off[i] = tin;
        tin += up256(streams[i].len + 16);
        out_off[i] = tout;
        tout += up256(streams[i].ny * streams[i].nx * sizeof(float));
    }
    RC(arena_reserve(g_io.in, tin + 256));
    RC(arena_reserve(g_io.out, tout + 256));
    std::vector<ebcc_stream_desc> dsd(streams, streams + n);
    std::vector<float *> dout(n, nullptr);
    std::vector<int> dst(n, EBCC_OK);
    for (int i = 0; i < n; i++) {
        if (!ok[i]) { dsd[i].stream = nullptr; continue; }
        uint8_t *d = g_io.in.base + in_off[i];
        if (const void *m = host_device_ptr(streams[i].stream))
            g_jobs.host.push_back({(const uint8_t *)m, d, (unsigned long long)streams[i].len});
        else
            RC(h2d(d, streams[i].stream, streams[i].len, st));
        dsd[i].stream = d;
        dout[i] = (float *)(g_io.out.base + out_off[i]);
    }
    RC(run_jobs(st));
    const int rc = engine_decompress(ebcc_api_engine(), dsd.data(), n, dout.data(), dst.data(), st);
    for (int i = 0; i < n; i++) {
        if (!ok[i]) continue;
        status[i] = dst[i];
        if (dst[i]) continue;
        const size_t bytes = streams[i].ny * streams[i].nx * sizeof(float);
        if (void *m = host_device_ptr(outs[i]))
            g_jobs.host.push_back({(const uint8_t *)dout[i], (uint8_t *)m, (unsigned long long)bytes});
        else
            RC(d2h(outs[i], dout[i], bytes, st));
    }
    RC(run_jobs(st));
    CK(cudaStreamSynchronize(st));
    return rc;
}

}  // namespace

extern "C" {

int ebcc_compress_batch(const ebcc_field_desc *fields, int n, ebcc_out_desc *outs, const ebcc_params *pp,
                        void *stream) {
    if (n < 0 || (n > 0 && (!fields || !outs))) return EBCC_EINVAL;
    ebcc_params p;
    if (pp) p = *pp; else ebcc_params_default(&p);
    RC(api_validate_params(p));
    std::lock_guard<std::mutex> lk(ebcc_api_mutex());
    if (!ebcc_api_engine()) return EBCC_ENOMEM;
    RC(compress_host_locked(fields, n, outs, p, (cudaStream_t)stream));
    for (int i = 0; i < n; i++)
        if (outs[i].status) return outs[i].status;
    return EBCC_OK;
}

int ebcc_decompress_batch(const ebcc_stream_desc *streams, int n, float **outs, void *stream) {
    if (n < 0 || (n > 0 && (!streams || !outs))) return EBCC_EINVAL;
    std::lock_guard<std::mutex> lk(ebcc_api_mutex());
    if (!ebcc_api_engine()) return EBCC_ENOMEM;
    std::vector<int> status(n, EBCC_OK);
    RC(decompress_host_locked(streams, n, outs, status.data(), (cudaStream_t)stream));
    for (int i = 0; i < n; i++)
        if (status[i]) return status[i];
    return EBCC_OK;
}

int ebcc_compress(const float *field, size_t ny, size_t nx, double bound, int bound_kind, const ebcc_params *pp,
                  uint8_t **out, size_t *out_len, ebcc_stats *stats) {
    if (!field || !out || !out_len) return EBCC_EINVAL;
    *out = nullptr;
    *out_len = 0;
    RC(api_check_shape(ny, nx));
    if (!(bound > 0) || !isfinite(bound) || (bound_kind != EBCC_BOUND_ABS && bound_kind != EBCC_BOUND_REL))
        return EBCC_EINVAL;
    const size_t cap = ebcc_max_stream_bytes(ny, nx);
    uint8_t *h = (uint8_t *)malloc(cap);
    if (!h) return EBCC_ENOMEM;
    ebcc_field_desc fd{field, ny, nx, bound, bound_kind};
    ebcc_out_desc od;
    memset(&od, 0, sizeof(od));
    od.stream = h;
    od.capacity = cap;
    const int rc = ebcc_compress_batch(&fd, 1, &od, pp, nullptr);
    if (rc) {
        free(h);
        return rc;
    }
    uint8_t *r = (uint8_t *)realloc(h, od.len ? od.len : 1);
    *out = r ? r : h;
    *out_len = od.len;
    if (stats) *stats = od.stats;
    return EBCC_OK;
}

int ebcc_decompress(const uint8_t *stream, size_t len, float *out, size_t ny, size_t nx) {
    if (!stream || !out) return EBCC_EINVAL;
    RC(api_check_shape(ny, nx));
    size_t hy = 0, hx = 0;
    RC(api_stream_shape(stream, len, &hy, &hx));
    if (hy != ny || hx != nx) return EBCC_EINVAL;
    ebcc_stream_desc sd{stream, len, ny, nx};
    return ebcc_decompress_batch(&sd, 1, &out, nullptr);
}

}  // extern "C"
