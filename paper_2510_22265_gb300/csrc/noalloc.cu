// Forward DWT on a fixed device scratch that the library owns statically, for
// callers that must not allocate device memory per call.
//
// ebcc_dwt_fwd_dev allocates its two LL scratch regions with cudaMalloc and
// frees them with cudaFree, which synchronises the whole device.  A caller in
// a latency-critical loop that shares the GPU with work on other streams, or a
// process whose device memory is fully committed to its own pools (a server
// holding an HBM budget), cannot take that.  ebcc_dwt_fwd_static_dev runs the
// same kernels with the scratch carved from one file-scope __device__ array
// of EBCC_DWT_STATIC_SCRATCH_FLOATS floats instead.
#include <mutex>
#include "ebcc_internal.cuh"

namespace {

constexpr size_t kScratchFloats = EBCC_DWT_STATIC_SCRATCH_FLOATS;
// LL intermediates of the forward transform: level l writes its LL quarter
// into region (l odd ? 1 : 2) and level l + 1 reads exactly what was written,
// so no element has to start at zero
__device__ __align__(256) float g_dwt_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float *g_addr[kMaxDevices];  // address of g_dwt_scratch on each device, looked up once

int scratch_address(float **p) {
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return EBCC_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *a = nullptr;
        CK(cudaGetSymbolAddress(&a, g_dwt_scratch));
        g_addr[dev] = (float *)a;
    }
    *p = g_addr[dev];
    return EBCC_OK;
}

}  // namespace

extern "C" int ebcc_dwt_fwd_static_dev(const float *in, float *out, size_t ny, size_t nx, int levels,
                                       double norm_min, double norm_range, void *stream) {
    if (ny == 0 || nx == 0 || ny > (1u << 30) || nx > (1u << 30) || ny * nx >= 0x7FFFFFFFull) return EBCC_EINVAL;
    if (levels < 0 || !in || !out) return EBCC_EINVAL;
    // region 1 holds ceil(ny/2) rows of ceil(nx/2) floats, region 2 ceil(ny/4)
    // rows of ceil(nx/4), each row padded to a multiple of 4 floats, each
    // region with 16 floats of slack; region 2 starts 256-byte aligned
    const size_t n1 = dwt_scratch_floats(ny, nx, 1);
    const size_t n1a = (n1 + 63) / 64 * 64;
    const size_t n2 = dwt_scratch_floats(ny, nx, 2);
    if (n1a + n2 > kScratchFloats) return EBCC_ECAPACITY;
    float *s = nullptr;
    RC(scratch_address(&s));
    const int L = effective_levels((int)ny, (int)nx, levels);
    const double inv = norm_range > 0 ? 1.0 / norm_range : 0.0;
    return dwt_forward(in, out, s, s + n1a, (int)ny, (int)nx, L, norm_min, inv, (cudaStream_t)stream);
}
