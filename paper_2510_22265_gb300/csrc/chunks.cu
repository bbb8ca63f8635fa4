// N-D front end of EBCC (Materials and Methods, first paragraph): a 4-D array
// (time, level, latitude, longitude) is split into chunks of one shape, each
// chunk is flattened to a 2-D field of (T*P*H, W) rows and compressed as a
// field of its own; the decompressor writes every chunk back in place.
//
// On the device: one gather kernel copies the chunks, flattened, into a
// library-owned buffer (every flattened row is a contiguous run of cW floats
// of the array, so a warp moves consecutive floats and rows are coalesced);
// the batch engine then compresses every chunk as one batch.  Decompression
// runs the batch decoder into the same buffer and one scatter kernel writes
// the chunks back.  Edge chunks (array extents that are not multiples of the
// chunk shape) are smaller.
#include <string.h>
#include <algorithm>
#include <vector>
#include "ebcc_internal.cuh"

namespace {

struct ChunkGrid {
    long long shape[4], chunk[4], n[4];
    long long count;
};

int make_grid(const size_t *shape, const size_t *chunk, ChunkGrid &g) {
    if (!shape || !chunk) return EBCC_EINVAL;
    g.count = 1;
    for (int d = 0; d < 4; d++) {
        if (shape[d] == 0 || chunk[d] == 0 || shape[d] > (1ull << 40)) return EBCC_EINVAL;
        g.shape[d] = (long long)shape[d];
        g.chunk[d] = (long long)std::min(chunk[d], shape[d]);
        g.n[d] = (g.shape[d] + g.chunk[d] - 1) / g.chunk[d];
        g.count *= g.n[d];
        if (g.count > (1ll << 24)) return EBCC_EINVAL;
    }
    return EBCC_OK;
}

// chunk k (row-major over the chunk grid): origin and extents
void chunk_box(const ChunkGrid &g, long long k, long long o[4], long long e[4]) {
    for (int d = 3; d >= 0; d--) {
        const long long c = k % g.n[d];
        k /= g.n[d];
        o[d] = c * g.chunk[d];
        e[d] = std::min(g.chunk[d], g.shape[d] - o[d]);
    }
}

// one flattened row of one chunk: array offset of its first float, offset in
// the flattened buffer, length
struct RowJob {
    long long src, dst;
    int len, pad;
};

// grid.x covers the row's floats, grid.y the rows (strided)
__global__ void __launch_bounds__(256) gather_rows(const float *__restrict__ a, float *__restrict__ buf,
                                                   const RowJob *__restrict__ rows, long long nrows, int to_buf) {
    for (long long r = blockIdx.y; r < nrows; r += gridDim.y) {
        const RowJob j = rows[r];
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < j.len; c += gridDim.x * blockDim.x) {
            if (to_buf) buf[j.dst + c] = a[j.src + c];
            else const_cast<float *>(a)[j.src + c] = buf[j.dst + c];
        }
    }
}

struct ChunkIO {
    Arena buf, jobs;
};
ChunkIO g_cio;

// rows of every chunk, and each chunk's offset and flattened shape
int plan(const ChunkGrid &g, std::vector<RowJob> &rows, std::vector<long long> &off, std::vector<long long> &fy,
         std::vector<long long> &fx) {
    rows.clear();
    off.assign(g.count, 0);
    fy.assign(g.count, 0);
    fx.assign(g.count, 0);
    long long pos = 0;
    for (long long k = 0; k < g.count; k++) {
        long long o[4], e[4];
        chunk_box(g, k, o, e);
        off[k] = pos;
        fy[k] = e[0] * e[1] * e[2];
        fx[k] = e[3];
        if (fy[k] > (1ll << 30) || fy[k] * fx[k] >= 0x7FFFFFFFll) return EBCC_EINVAL;
        long long r = 0;
        for (long long t = 0; t < e[0]; t++)
            for (long long p = 0; p < e[1]; p++)
                for (long long h = 0; h < e[2]; h++, r++) {
                    RowJob j;
                    j.src = (((o[0] + t) * g.shape[1] + o[1] + p) * g.shape[2] + o[2] + h) * g.shape[3] + o[3];
                    j.dst = pos + r * e[3];
                    j.len = (int)e[3];
                    j.pad = 0;
                    rows.push_back(j);
                }
        pos += (fy[k] * fx[k] + 63) / 64 * 64;  // 256-byte aligned fields
    }
    return EBCC_OK;
}

int move_rows(const float *a, const std::vector<RowJob> &rows, long long total, int to_buf, cudaStream_t st) {
    RC(arena_reserve(g_cio.jobs, rows.size() * sizeof(RowJob) + 256));
    CK(cudaMemcpyAsync(g_cio.jobs.base, rows.data(), rows.size() * sizeof(RowJob), cudaMemcpyHostToDevice, st));
    long long maxlen = 1;
    for (const RowJob &j : rows) maxlen = std::max<long long>(maxlen, j.len);
    dim3 grid((unsigned)std::min<long long>((maxlen + 255) / 256, 64),
              (unsigned)std::min<long long>((long long)rows.size(), 65535));
    const RowJob *jobs = (const RowJob *)g_cio.jobs.base;
    float *buf = (float *)g_cio.buf.base;
    if (to_buf)
        PROF("chunk_gather", st, 8.0 * (double)total, gather_rows<<<grid, 256, 0, st>>>(a, buf, jobs, (long long)rows.size(), 1));
    else
        PROF("chunk_scatter", st, 8.0 * (double)total, gather_rows<<<grid, 256, 0, st>>>(a, buf, jobs, (long long)rows.size(), 0));
    CK(cudaGetLastError());
    // the job table is read by this launch: keep it until the launch ran
    CK(cudaStreamSynchronize(st));
    return EBCC_OK;
}

}  // namespace

extern "C" {

long long ebcc_chunk_count(const size_t shape[4], const size_t chunk[4]) {
    ChunkGrid g;
    const int rc = make_grid(shape, chunk, g);
    return rc ? rc : g.count;
}

int ebcc_chunk_info(const size_t shape[4], const size_t chunk[4], long long k, size_t origin[4], size_t extent[4],
                    size_t *ny, size_t *nx) {
    ChunkGrid g;
    RC(make_grid(shape, chunk, g));
    if (k < 0 || k >= g.count) return EBCC_EINVAL;
    long long o[4], e[4];
    chunk_box(g, k, o, e);
    for (int d = 0; d < 4; d++) {
        if (origin) origin[d] = (size_t)o[d];
        if (extent) extent[d] = (size_t)e[d];
    }
    if (ny) *ny = (size_t)(e[0] * e[1] * e[2]);
    if (nx) *nx = (size_t)e[3];
    return EBCC_OK;
}

int ebcc_compress_chunks_dev(const float *array, const size_t shape[4], const size_t chunk[4], double bound,
                             int bound_kind, const ebcc_params *pp, ebcc_out_desc *outs, void *stream) {
    if (!array || !outs) return EBCC_EINVAL;
    ChunkGrid g;
    RC(make_grid(shape, chunk, g));
    ebcc_params p;
    if (pp) p = *pp; else ebcc_params_default(&p);
    RC(api_validate_params(p));
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<RowJob> rows;
    std::vector<long long> off, fy, fx;
    RC(plan(g, rows, off, fy, fx));
    const long long total = off.back() + (fy.back() * fx.back() + 63) / 64 * 64;
    std::lock_guard<std::mutex> lk(ebcc_api_mutex());
    if (!ebcc_api_engine()) return EBCC_ENOMEM;
    RC(arena_reserve(g_cio.buf, (size_t)total * sizeof(float) + 256));
    RC(move_rows(array, rows, total, 1, st));
    std::vector<ebcc_field_desc> fd(g.count);
    const float *base = (const float *)g_cio.buf.base;
    for (long long k = 0; k < g.count; k++)
        fd[k] = ebcc_field_desc{base + off[k], (size_t)fy[k], (size_t)fx[k], bound, bound_kind};
    RC(engine_compress(ebcc_api_engine(), fd.data(), (int)g.count, outs, p, st));
    for (long long k = 0; k < g.count; k++)
        if (outs[k].status) return outs[k].status;
    return EBCC_OK;
}

int ebcc_decompress_chunks_dev(const ebcc_stream_desc *streams, const size_t shape[4], const size_t chunk[4],
                               float *array, void *stream) {
    if (!array || !streams) return EBCC_EINVAL;
    ChunkGrid g;
    RC(make_grid(shape, chunk, g));
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<RowJob> rows;
    std::vector<long long> off, fy, fx;
    RC(plan(g, rows, off, fy, fx));
    for (long long k = 0; k < g.count; k++)
        if (streams[k].ny != (size_t)fy[k] || streams[k].nx != (size_t)fx[k]) return EBCC_EINVAL;
    const long long total = off.back() + (fy.back() * fx.back() + 63) / 64 * 64;
    std::lock_guard<std::mutex> lk(ebcc_api_mutex());
    if (!ebcc_api_engine()) return EBCC_ENOMEM;
    RC(arena_reserve(g_cio.buf, (size_t)total * sizeof(float) + 256));
    std::vector<float *> dst(g.count);
    for (long long k = 0; k < g.count; k++) dst[k] = (float *)g_cio.buf.base + off[k];
    std::vector<int> status(g.count, EBCC_OK);
    RC(engine_decompress(ebcc_api_engine(), streams, (int)g.count, dst.data(), status.data(), st));
    for (long long k = 0; k < g.count; k++)
        if (status[k]) return status[k];
    RC(move_rows(array, rows, total, 0, st));
    return EBCC_OK;
}

}  // extern "C"
