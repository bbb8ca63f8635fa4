// Code-block shape autotuner for batches of uneven fields.
//
// The code-block shape (cblk_w x cblk_h, recorded in every stream's header)
// sets how the base layer's tier-1 work is cut: 32 x 32 and smaller blocks run
// on the warp-per-block model + MQ kernels, larger ones on the serial-pass
// kernel; it also moves the rate-distortion points PCRD can pick, so the
// compression ratio depends on it a little.  Per grid class (field shape) the
// tuner compresses up to four probe fields of the class with each candidate
// shape (after one untimed warm-up call), timing each on the device with CUDA
// events, and keeps, among the candidates at most kSlowTol times slower than
// the fastest, the one with the shortest streams: throughput first, and a
// better ratio where it costs little time.  (Larger blocks give streams 1-7%
// shorter on ERA5-shaped fields but run 1.7-4.4 times slower at batch scale,
// so a ratio-first rule gave a tuned batch several times slower than the
// untuned one.)  Choices are cached per (ny, nx) for the life of the process.
// A batch call then compresses each group of fields that share a chosen shape
// as one batch.
#include <string.h>
#include <map>
#include <mutex>
#include <utility>
#include <vector>
#include "ebcc_internal.cuh"

namespace {

const int kCand[4][2] = {{32, 32}, {64, 64}, {32, 64}, {64, 32}};
constexpr double kSlowTol = 1.25;

std::mutex g_tune_mu;
std::map<std::pair<size_t, size_t>, int> g_choice;  // (ny, nx) -> candidate index

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// time every candidate on the probe fields; *best = the chosen candidate
int tune_class(EbccEngine *eng, const ebcc_field_desc *probe, int n, const ebcc_params &base, int *best,
               double *ms, long long *bytes, cudaStream_t st) {
    std::vector<uint8_t *> bufs(n, nullptr);
    std::vector<ebcc_out_desc> od(n);
    Arena out;
    size_t tot = 0;
    for (int i = 0; i < n; i++) tot += (ebcc_max_stream_bytes(probe[i].ny, probe[i].nx) + 255) & ~(size_t)255;
    RC(arena_reserve(out, tot + 256));
    Events ev;
    CK(cudaEventCreate(&ev.a));
    CK(cudaEventCreate(&ev.b));
    int rc = EBCC_OK;
    for (int c = 0; c < 4 && !rc; c++) {
        ebcc_params p = base;
        p.cblk_w = kCand[c][0];
        p.cblk_h = kCand[c][1];
        bytes[c] = -1;
        ms[c] = -1;
        for (int rep = 0; rep < 2 && !rc; rep++) {  // a warm-up call, then the timed one
            size_t off = 0;
            for (int i = 0; i < n; i++) {
                memset(&od[i], 0, sizeof(od[i]));
                od[i].stream = out.base + off;
                od[i].capacity = ebcc_max_stream_bytes(probe[i].ny, probe[i].nx);
                off += (od[i].capacity + 255) & ~(size_t)255;
            }
            if (rep == 1 && cudaEventRecord(ev.a, st) != cudaSuccess) rc = EBCC_ECUDA;
            if (!rc) rc = engine_compress(eng, probe, n, od.data(), p, st);
            if (!rc && rep == 1 && (cudaEventRecord(ev.b, st) != cudaSuccess || cudaEventSynchronize(ev.b) != cudaSuccess))
                rc = EBCC_ECUDA;
        }
        if (rc) break;
        long long b = 0;
        bool ok = true;
        for (int i = 0; i < n; i++) {
            if (od[i].status) ok = false;
            b += (long long)od[i].len;
        }
        if (!ok) continue;  // a shape that fails on this class is not a candidate
        float t = 0;
        CK(cudaEventElapsedTime(&t, ev.a, ev.b));
        ms[c] = t;
        bytes[c] = b;
    }
    if (out.base) cudaFree(out.base);
    if (rc) return rc;
    double fastest = -1;
    for (int c = 0; c < 4; c++)
        if (bytes[c] >= 0 && (fastest < 0 || ms[c] < fastest)) fastest = ms[c];
    if (fastest < 0) return EBCC_EINVAL;
    int pick = -1;
    for (int c = 0; c < 4; c++)
        if (bytes[c] >= 0 && ms[c] <= kSlowTol * fastest &&
            (pick < 0 || bytes[c] < bytes[pick] || (bytes[c] == bytes[pick] && ms[c] < ms[pick])))
            pick = c;
    *best = pick;
    return EBCC_OK;
}

}  // namespace

extern "C" {

int ebcc_autotune_cblk(const ebcc_field_desc *probe, int n, const ebcc_params *pp, int *cblk_w, int *cblk_h,
                       double *ms, long long *bytes, void *stream) {
    if (!probe || n <= 0 || !cblk_w || !cblk_h) return EBCC_EINVAL;
    for (int i = 0; i < n; i++)
        if (probe[i].ny != probe[0].ny || probe[i].nx != probe[0].nx || !probe[i].field) return EBCC_EINVAL;
    ebcc_params p;
    if (pp) p = *pp; else ebcc_params_default(&p);
    RC(api_validate_params(p));
    double m[4];
    long long b[4];
    int best = 0;
    {
        std::lock_guard<std::mutex> lk(ebcc_api_mutex());
        if (!ebcc_api_engine()) return EBCC_ENOMEM;
        RC(tune_class(ebcc_api_engine(), probe, n, p, &best, m, b, (cudaStream_t)stream));
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_choice[{probe[0].ny, probe[0].nx}] = best;
    }
    *cblk_w = kCand[best][0];
    *cblk_h = kCand[best][1];
    for (int c = 0; c < 4; c++) {
        if (ms) ms[c] = m[c];
        if (bytes) bytes[c] = b[c];
    }
    return EBCC_OK;
}

int ebcc_autotune_lookup(size_t ny, size_t nx, int *cblk_w, int *cblk_h) {
    if (!cblk_w || !cblk_h) return EBCC_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_choice.find({ny, nx});
    if (it == g_choice.end()) return EBCC_EINVAL;
    *cblk_w = kCand[it->second][0];
    *cblk_h = kCand[it->second][1];
    return EBCC_OK;
}

void ebcc_autotune_reset(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_choice.clear();
}

int ebcc_compress_batch_tuned_dev(const ebcc_field_desc *fields, int n, ebcc_out_desc *outs, const ebcc_params *pp,
                                  void *stream) {
    if (n < 0 || (n > 0 && (!fields || !outs))) return EBCC_EINVAL;
    ebcc_params p;
    if (pp) p = *pp; else ebcc_params_default(&p);
    RC(api_validate_params(p));
    cudaStream_t st = (cudaStream_t)stream;
    // grid classes in order of first appearance; tune the ones not cached yet
    std::vector<std::pair<size_t, size_t>> classes;
    std::map<std::pair<size_t, size_t>, std::vector<int>> members;
    for (int i = 0; i < n; i++) {
        auto key = std::make_pair(fields[i].ny, fields[i].nx);
        if (!members.count(key)) classes.push_back(key);
        members[key].push_back(i);
    }
    std::map<std::pair<size_t, size_t>, int> chosen;
    for (auto &k : classes) {
        int c = -1;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_choice.find(k);
            if (it != g_choice.end()) c = it->second;
        }
        if (c < 0 && api_check_shape(k.first, k.second) == EBCC_OK) {
            std::vector<ebcc_field_desc> probe;
            for (int i : members[k])
                if (probe.size() < 4 && fields[i].field && fields[i].bound > 0) probe.push_back(fields[i]);
            int w = 32, h = 32;
            if (!probe.empty() &&
                ebcc_autotune_cblk(probe.data(), (int)probe.size(), &p, &w, &h, nullptr, nullptr, stream) == EBCC_OK) {
                for (int q = 0; q < 4; q++)
                    if (kCand[q][0] == w && kCand[q][1] == h) c = q;
            }
        }
        chosen[k] = c < 0 ? 0 : c;
    }
    // one batch per chosen shape
    std::lock_guard<std::mutex> lk(ebcc_api_mutex());
    if (!ebcc_api_engine()) return EBCC_ENOMEM;
    for (int c = 0; c < 4; c++) {
        std::vector<int> idx;
        for (auto &k : classes)
            if (chosen[k] == c)
                for (int i : members[k]) idx.push_back(i);
        if (idx.empty()) continue;
        std::vector<ebcc_field_desc> fd;
        std::vector<ebcc_out_desc> od;
        for (int i : idx) { fd.push_back(fields[i]); od.push_back(outs[i]); }
        ebcc_params q = p;
        q.cblk_w = kCand[c][0];
        q.cblk_h = kCand[c][1];
        const int rc = engine_compress(ebcc_api_engine(), fd.data(), (int)fd.size(), od.data(), q, st);
        for (size_t j = 0; j < idx.size(); j++) outs[idx[j]] = od[j];
        if (rc) return rc;
    }
    for (int i = 0; i < n; i++)
        if (outs[i].status) return outs[i].status;
    return EBCC_OK;
}

}  // extern "C"
