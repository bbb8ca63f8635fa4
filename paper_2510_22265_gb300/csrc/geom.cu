// Host-side geometry of the GB300 EBCC library: effective wavelet levels,
// Mallat band layout, code-block partition, and the base-layer step sizes
// (T.800 Annex E form of 2^-P divided by each band's synthesis L2 norm; the
// norm of a 2-D band is the product of two 1-D synthesis-basis norms, each
// measured here by inverting a unit impulse with this library's own host 9/7
// lifting).  Also the status strings and parameter defaults of the C ABI.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <mutex>
#include "ebcc_internal.cuh"

static const double H_ALPHA = -1.586134342059924;
static const double H_BETA = -0.052980118572961;
static const double H_GAMMA = 0.882911075530934;
static const double H_DELTA = 0.443506852043971;
static const double H_KAPPA = 1.230174104914001;

static int ceil_sh(int n, int l) { return (int)(((long)n + (1L << l) - 1) >> l); }

int effective_levels(int ny, int nx, int levels) {
    int m = ny < nx ? ny : nx, L = 0;
    while (L < levels && L < EBCC_MAX_LEVELS && ceil_sh(m, L) >= 2) L++;
    return L;
}

// inverse 1-D lifting of a de-interleaved signal (low | high), symmetric ext.
static void inv1d(std::vector<double> &x, int n) {
    if (n < 2) return;
    std::vector<double> y(n);
    int nl = (n + 1) / 2;
    for (int i = 0; i < n; i++) y[i] = (i & 1) ? x[nl + i / 2] / H_KAPPA : x[i / 2] * H_KAPPA;
    auto at = [&](int i) {
        int p = 2 * (n - 1);
        i %= p;
        if (i < 0) i += p;
        if (i >= n) i = p - i;
        return y[i];
    };
    const double c[4] = {H_DELTA, H_GAMMA, H_BETA, H_ALPHA};
    for (int s = 0; s < 4; s++) {
        int par = (s & 1) ? 1 : 0;  // delta: even, gamma: odd, beta: even, alpha: odd
        for (int i = par; i < n; i += 2) y[i] -= c[s] * (at(i - 1) + at(i + 1));
    }
    for (int i = 0; i < n; i++) x[i] = y[i];
}

// L2 norm of the 1-D synthesis basis of level l, low (high = 0) or high (1)
static double norm1d(int l, int high) {
    int n = 64 << l;
    std::vector<double> x(n, 0.0);
    // position of a coefficient in the middle of the level-l band
    int len = n >> l;  // length of the level-l low band (n is a multiple of 2^l)
    int pos = high ? (len + len / 2) : (len / 2);
    x[pos] = 1.0;
    for (int k = l; k >= 1; k--) {
        int m = n >> (k - 1);
        std::vector<double> seg(x.begin(), x.begin() + m);
        inv1d(seg, m);
        for (int i = 0; i < m; i++) x[i] = seg[i];
    }
    double s = 0;
    for (double v : x) s += v * v;
    return sqrt(s);
}

static double norm_cache[EBCC_MAX_LEVELS + 1][2];
static std::once_flag norm_once;

static void fill_norms() {
    for (int l = 1; l <= EBCC_MAX_LEVELS; l++)
        for (int h = 0; h < 2; h++) norm_cache[l][h] = norm1d(l, h);
}

double band_step(int P, int level, int orient) {
    std::call_once(norm_once, fill_norms);
    double nrm = 1.0;
    if (level >= 1) {
        int hh = (orient == 1 || orient == 3), vh = (orient == 2 || orient == 3);
        nrm = norm_cache[level][hh] * norm_cache[level][vh];
    }
    double d = ldexp(1.0, -P) / nrm;
    int e = -(int)floor(log2(d));
    double f = ldexp(d, e);
    long m = lround((f - 1.0) * 2048.0);
    if (m >= 2048) { m = 0; e -= 1; }
    return ldexp(1.0 + m / 2048.0, -e);
}

int base_precision(double eps_n) {
    int P = (int)ceil(log2(1.0 / eps_n)) + 6;
    return P < 16 ? 16 : (P > 18 ? 18 : P);
}

void make_geom(FieldGeom *g, int ny, int nx, int levels, int cw, int ch, int P) {
    memset(g, 0, sizeof(*g));
    g->ny = ny; g->nx = nx; g->cw = cw; g->ch = ch; g->P = P;
    g->L = effective_levels(ny, nx, levels);
    for (int l = 0; l <= g->L; l++) { g->h[l] = ceil_sh(ny, l); g->w[l] = ceil_sh(nx, l); }
    int k = 0, L = g->L;
    auto add = [&](int x0, int y0, int w, int h, int level, int orient) {
        BandGeom &b = g->band[k++];
        b.x0 = x0; b.y0 = y0; b.w = w; b.h = h; b.level = level; b.orient = orient;
        b.delta = (float)band_step(P, level, orient);
    };
    add(0, 0, g->w[L], g->h[L], L, 0);
    for (int l = L; l >= 1; l--) {
        add(g->w[l], 0, g->w[l - 1] - g->w[l], g->h[l], l, 1);
        add(0, g->h[l], g->w[l], g->h[l - 1] - g->h[l], l, 2);
        add(g->w[l], g->h[l], g->w[l - 1] - g->w[l], g->h[l - 1] - g->h[l], l, 3);
    }
    g->nbands = k;
    int nb = 0;
    for (int b = 0; b < k; b++) {
        BandGeom &B = g->band[b];
        B.blk0 = nb;
        B.nbx = (B.w + cw - 1) / cw;
        B.nby = (B.h + ch - 1) / ch;
        nb += B.nbx * B.nby;
    }
    g->nblocks = nb;
}

int ebcc_debug_sync_enabled() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("EBCC_DEBUG_SYNC");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v;
}

int ebcc_stage_check(cudaStream_t st, const char *what, int line) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "ebcc: stage '%s' (line %d) failed: %s\n", what, line, cudaGetErrorString(e));
        return EBCC_ECUDA;
    }
    return EBCC_OK;
}

int ebcc_cuda_fail(cudaError_t e, const char *file, int line) {
    if (getenv("EBCC_DEBUG")) fprintf(stderr, "ebcc: CUDA error %s at %s:%d\n", cudaGetErrorString(e), file, line);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return EBCC_ENOMEM;
    }
    return EBCC_ECUDA;
}

extern "C" {

void ebcc_params_default(ebcc_params *p) {
    p->levels = 5;
    p->cblk_w = 32;
    p->cblk_h = 32;
    p->r0 = 20.0;
    p->q = 0.999;
    p->tol = 1e-3;
    p->spiht_guard_bits = 3;
}

const char *ebcc_strerror(int s) {
    switch (s) {
    case EBCC_OK: return "ok";
    case EBCC_EINVAL: return "invalid argument";
    case EBCC_ENONFINITE: return "non-finite value in field";
    case EBCC_ECORRUPT: return "corrupt or truncated stream";
    case EBCC_ENOMEM: return "out of memory";
    case EBCC_EBUDGET: return "request exceeds the HBM budget";
    case EBCC_ECAPACITY: return "buffer capacity exceeded";
    case EBCC_ETIMEOUT: return "timed out";
    case EBCC_ECUDA: return "CUDA runtime error";
    default: return "unknown status";
    }
}

void ebcc_free(void *p) { free(p); }

int ebcc_effective_levels(size_t ny, size_t nx, int levels) {
    if (ny == 0 || nx == 0 || ny > (1u << 30) || nx > (1u << 30) || levels < 0) return EBCC_EINVAL;
    return effective_levels((int)ny, (int)nx, levels);
}

double ebcc_band_step(int P, int level, int orient) {
    if (level < 0 || level > EBCC_MAX_LEVELS || orient < 0 || orient > 3) return 0.0;
    return band_step(P, level, orient);
}

}  // extern "C"

// ------------------------------------------------------------ kernel profiler
// When enabled, launch sites bracket their kernels with CUDA events recorded
// on the launching stream; durations are resolved when the table is read.
namespace {
struct ProfPending {
    int id;
    cudaEvent_t a, b;
    double bytes;
};
struct ProfEntry {
    const char *name;
    double ms = 0, bytes = 0;
    long long launches = 0;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfPending> g_prof_pending;
std::vector<ProfEntry> g_prof;

void prof_resolve_locked() {
    for (auto &p : g_prof_pending) {
        float ms = 0;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_prof[p.id].ms += ms;
            g_prof[p.id].bytes += p.bytes;
            g_prof[p.id].launches++;
        }
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_prof_pending.clear();
}
}  // namespace

int prof_id(const char *name) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (size_t i = 0; i < g_prof.size(); i++)
        if (strcmp(g_prof[i].name, name) == 0) return (int)i;
    ProfEntry e;
    e.name = name;
    g_prof.push_back(e);
    return (int)g_prof.size() - 1;
}

void *prof_begin(int id, cudaStream_t st) {
    if (!g_prof_on) return nullptr;
    ProfPending *p = new ProfPending{id, nullptr, nullptr, 0};
    cudaEventCreate(&p->a);
    cudaEventCreate(&p->b);
    cudaEventRecord(p->a, st);
    return p;
}

int prof_enabled() { return g_prof_on ? 1 : 0; }

void prof_add_bytes(const char *name, double bytes) {
    const int id = prof_id(name);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof[id].bytes += bytes;
}

void prof_end(void *tok, cudaStream_t st, double bytes) {
    if (!tok) return;
    ProfPending *p = (ProfPending *)tok;
    cudaEventRecord(p->b, st);
    p->bytes = bytes;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_pending.push_back(*p);
    delete p;
    if (g_prof_pending.size() > 20000) prof_resolve_locked();
}

extern "C" {

void ebcc_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!on) prof_resolve_locked();
    g_prof_on = on != 0;
}

void ebcc_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_resolve_locked();
    for (auto &e : g_prof) { e.ms = 0; e.bytes = 0; e.launches = 0; }
}

int ebcc_profile_count(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_resolve_locked();
    return (int)g_prof.size();
}

int ebcc_profile_get(int i, const char **name, double *total_ms, long long *launches, double *bytes) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_resolve_locked();
    if (i < 0 || i >= (int)g_prof.size()) return EBCC_EINVAL;
    if (name) *name = g_prof[i].name;
    if (total_ms) *total_ms = g_prof[i].ms;
    if (launches) *launches = g_prof[i].launches;
    if (bytes) *bytes = g_prof[i].bytes;
    return EBCC_OK;
}

}  // extern "C"
