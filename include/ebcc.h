/*
 * ebcc.h -- C ABI of the GB300 (sm_103a) EBCC library.
 *
 * EBCC (arxiv 2510.22265) compresses a 2-D float32 field with a pointwise
 * error bound: a JPEG2000 base layer whose compression ratio is found by a
 * feedback bisection so that a fraction q of the points meets the bound, then
 * a residual layer (wavelet + SPIHT) truncated by a second bisection at the
 * shortest prefix that meets the bound everywhere, with a fallback to the base
 * layer alone when that is shorter (Materials and Methods, Algorithm 1).
 *
 * Conventions for every call:
 *  - return 0 (EBCC_OK) or a negative EBCC_E* status; no call throws;
 *  - fields are row-major, nx contiguous (a (T*P*H, W) flattening of a chunk,
 *    Materials and Methods), float32;
 *  - "_dev" calls take device pointers owned by the caller and a cudaStream_t
 *    passed as void* (NULL = the legacy default stream); they are asynchronous
 *    unless stated otherwise, and their scalar outputs live in device memory;
 *  - host outputs allocated by the library are released with ebcc_free.
 */
#ifndef EBCC_H
#define EBCC_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define EBCC_OK 0
#define EBCC_EINVAL (-1)      /* bad dimensions, bound <= 0 or non-finite, bad kind or params */
#define EBCC_ENONFINITE (-2)  /* NaN or Inf in the field */
#define EBCC_ECORRUPT (-3)    /* stream: bad magic, version, lengths or truncation */
#define EBCC_ENOMEM (-4)      /* device or host allocation failed */
#define EBCC_EBUDGET (-5)     /* request does not fit the server's HBM budget */
#define EBCC_ECAPACITY (-6)   /* an output or internal buffer is too small */
#define EBCC_ETIMEOUT (-7)    /* a bounded device wait or poll gave up */
#define EBCC_ECUDA (-8)       /* a CUDA runtime call failed */

/* Bound kinds.  REL is the paper's range-relative bound (Benchmarks: the ratio
 * of the max absolute error to the data range of a chunk): eps = bound *
 * (max - min).  ABS is an absolute bound in the field's units. */
#define EBCC_BOUND_ABS 0
#define EBCC_BOUND_REL 1

/* Algorithm 1 inputs and the codec parameters the paper leaves implicit.
 * levels: wavelet levels (5); cblk_w / cblk_h: code-block size, powers of two
 * in [4, 64] (32 x 32); r0: initial base compression ratio (20); q: fraction of
 * points the base layer must bring within the bound (0.999); tol: bisection
 * tolerance on the ratio (1e-3, Algorithm 1); spiht_guard_bits: SPIHT step =
 * 2^(floor(log2 eps_n) - guard) (3). */
typedef struct {
    int levels;
    int cblk_w, cblk_h;
    double r0, q, tol;
    int spiht_guard_bits;
} ebcc_params;

/* Per-field diagnostics of one compression. */
typedef struct {
    double r_base, r_base1;      /* ratio kept by the q loop and by the q = 1 loop */
    int iters_base, iters_base1; /* enc_base evaluations of the two loops */
    int iters_trunc;             /* truncation bisection steps */
    int used_fallback;           /* 1 = base layer alone was shorter */
    int guard_bits, n_escape;    /* SPIHT guard bits used; escaped points */
    long long base_bytes, res_bytes, total_bytes, spiht_len_bytes;
    long long len_two, len_one;  /* two-layer and base-only stream lengths (0 = none; len_two is also 0
                                    when the base-only stream was proven shorter before the two-layer
                                    stream was finished) */
    double q_base;               /* q_A of the kept base encoding (a lower bound in the one case
                                    where that encoding missed q -- the r = 1 encoding kept after
                                    every ratio missed -- since a count stops once a miss is
                                    certain) */
} ebcc_stats;

/* Fill *p with the defaults listed above. */
void ebcc_params_default(ebcc_params *p);

/* Message for a status code (static storage). */
const char *ebcc_strerror(int status);

/* Release memory returned by the library. */
void ebcc_free(void *p);

/* Compress a host field (Algorithm 1).  field: ny*nx float32, row-major.
 * bound > 0 and finite; bound_kind EBCC_BOUND_ABS or EBCC_BOUND_REL; p may be
 * NULL (defaults).  On success *out is a library-allocated stream of *out_len
 * bytes (free with ebcc_free); stats may be NULL.  Host -> device copy,
 * device pipeline and device -> host copy happen inside; synchronous.
 * Errors: EINVAL, ENONFINITE, ENOMEM, ECAPACITY, ECUDA. */
int ebcc_compress(const float *field, size_t ny, size_t nx, double bound, int bound_kind,
                  const ebcc_params *p, uint8_t **out, size_t *out_len, ebcc_stats *stats);

/* Decompress a host stream into the caller's host buffer out (ny*nx float32);
 * ny, nx must match the stream.  Every point is within the stream's bound of
 * the original.  Synchronous.  Errors: EINVAL (shape), ECORRUPT, ENOMEM, ECUDA. */
int ebcc_decompress(const uint8_t *stream, size_t len, float *out, size_t ny, size_t nx);

/* Read dimensions and absolute bound from a stream header (host memory). */
int ebcc_stream_info(const uint8_t *stream, size_t len, size_t *ny, size_t *nx, double *bound_abs);

/* ----------------------------------------------------- batched device API */
/* One field of a batch: device pointer to ny*nx float32. */
typedef struct {
    const float *field;
    size_t ny, nx;
    double bound;
    int bound_kind;
} ebcc_field_desc;

/* Output of one field: caller-owned device buffer `stream` of `capacity`
 * bytes; the library writes the stream there and sets len, status, stats. */
typedef struct {
    uint8_t *stream;
    size_t capacity;
    size_t len;
    int status;
    ebcc_stats stats;
} ebcc_out_desc;

/* Compress n device fields of any sizes together: every step of Algorithm 1 is
 * one launch over all fields that take part in it, and the two feedback loops
 * are per-field state machines on the device that drop fields from the
 * launches as they finish (a batch of one field is the plain path).  Fields
 * whose workspace would exceed half the free device memory are split into
 * several batches.  Synchronises `stream` before returning (it reads the
 * per-field outcomes).  The return
 * value is EBCC_OK if every field succeeded, else the first failing status;
 * per-field status is in outs[i].status.  Stream capacity needed per field:
 * ebcc_max_stream_bytes(ny, nx). */
int ebcc_compress_batch_dev(const ebcc_field_desc *fields, int n, ebcc_out_desc *outs,
                            const ebcc_params *p, void *stream);

/* One stream of a decompression batch (device pointer). */
typedef struct {
    const uint8_t *stream;
    size_t len;
    size_t ny, nx;
} ebcc_stream_desc;

/* Decompress n device streams into caller-owned device buffers outs[i]
 * (ny*nx float32 each).  Synchronous on `stream`.  Errors: ECORRUPT, ENOMEM, ECUDA. */
int ebcc_decompress_batch_dev(const ebcc_stream_desc *streams, int n, float **outs, void *stream);

/* Upper bound of a stream's length for an ny x nx field. */
size_t ebcc_max_stream_bytes(size_t ny, size_t nx);

/* ----------------------------------------------------- code-block autotuner */
/* Code-block shape per grid class for batches of uneven fields.  The shape
 * (cblk_w x cblk_h, stored in each stream's header; the paper leaves it to the
 * JPEG 2000 codec) changes how the tier-1 work is cut and, slightly, which
 * rate-distortion points the base layer can choose.  ebcc_autotune_cblk
 * compresses the n probe fields (device, all of one shape) with each of
 * 32x32, 64x64, 32x64 and 64x32 (after an untimed warm-up call each), timing
 * them with CUDA events on `stream`, and picks, among the shapes at most 1.25
 * times slower than the fastest, the one with the shortest total stream
 * length (ties: the faster); the choice is cached for that (ny, nx) for the
 * life of the process.  ms[4] and bytes[4] (either may be
 * NULL) receive each candidate's time and total length (-1: the candidate
 * failed on these fields).  Synchronous.  Errors: EINVAL (no probe, mixed
 * shapes, bad params), ENOMEM, ECUDA.
 * ebcc_autotune_lookup: the cached shape of a grid class (EINVAL if none).
 * ebcc_autotune_reset: forget every cached choice.
 * ebcc_compress_batch_tuned_dev: ebcc_compress_batch_dev with the code-block
 * shape of each field's grid class taken from the cache, tuning (on up to 4
 * fields of the batch) the classes not cached yet; fields that share a shape
 * are compressed as one batch.  p's cblk_w / cblk_h are ignored. */
int ebcc_autotune_cblk(const ebcc_field_desc *probe, int n, const ebcc_params *p, int *cblk_w, int *cblk_h,
                       double *ms, long long *bytes, void *stream);
int ebcc_autotune_lookup(size_t ny, size_t nx, int *cblk_w, int *cblk_h);
void ebcc_autotune_reset(void);
int ebcc_compress_batch_tuned_dev(const ebcc_field_desc *fields, int n, ebcc_out_desc *outs, const ebcc_params *p,
                                  void *stream);

/* --------------------------------------------------- batched host-buffer API */
/* The batch calls above with every buffer in host memory (Algorithm 1 KwIn /
 * KwOut: the arrays in, the byte sequences out).  fields[i].field points to
 * ny*nx host float32; outs[i].stream is a caller-owned host buffer of
 * outs[i].capacity bytes that receives the stream (len, status and stats as
 * in ebcc_compress_batch_dev).  The library copies the fields to device
 * buffers it keeps between calls (grown to the largest batch seen, so a call
 * allocates nothing once they have that size), runs the device batch, and
 * copies every stream back.  Page-locked host buffers (cudaHostAlloc,
 * cudaHostRegister) that the device maps are copied by one kernel per
 * direction for the whole batch, reading or writing the host memory through
 * its device mapping; other page-locked buffers by DMA; pageable ones through
 * the library's pinned staging.  A caller's host buffers must not be written
 * (inputs) or read (outputs) by the host during the call.  `stream` is a cudaStream_t as void* (NULL = the
 * legacy default stream); the call is synchronous.  Return value as
 * ebcc_compress_batch_dev.  Errors: EINVAL, ENONFINITE, ENOMEM, ECAPACITY,
 * ECUDA (per field in outs[i].status). */
int ebcc_compress_batch(const ebcc_field_desc *fields, int n, ebcc_out_desc *outs, const ebcc_params *p,
                        void *stream);
/* Decompress n host streams into caller-owned host buffers outs[i] (ny*nx
 * float32 each), through the same device buffers.  Synchronous.  Errors:
 * EINVAL, ECORRUPT, ENOMEM, ECUDA (the first failing stream's status). */
int ebcc_decompress_batch(const ebcc_stream_desc *streams, int n, float **outs, void *stream);

/* ------------------------------------------------------- error statistics */
/* Statistics of a reconstruction x_hat of x (Benchmarks, error statistics:
 * SSIM against Baker's 0.99995 threshold, histograms of the compression
 * errors, RMSE), computed on the GPU.  With e = x_hat - x in FP64:
 * mean_err = mean e, rmse = sqrt(mean e^2), max_abs_err = max |e|; range =
 * max x - min x; ssim = the mean SSIM (Wang et al. 2004) of x and x_hat both
 * rescaled by x's min and range (dynamic range 1), 11 x 11 Gaussian window of
 * standard deviation 1.5, C1 = 0.01^2, C2 = 0.03^2, over the n_ssim windows
 * that lie inside the field (NaN when there are none: a side below 11, or a
 * constant x). */
typedef struct {
    long long n, n_ssim;
    double mean_err, rmse, max_abs_err, range, ssim;
} ebcc_error_stats;
/* x, x_hat: device ny*nx float32.  hist (device, nbins uint64, nbins <= 4096,
 * NULL when nbins = 0): counts of the errors in nbins equal bins over
 * [-eps, eps], point i in bin floor((e_i + eps) * (nbins / (2 eps))) clamped
 * to [0, nbins - 1], computed in FP64.  Synchronous on `stream` (the library
 * keeps its accumulators between calls).  Errors: EINVAL, ECUDA. */
int ebcc_error_stats_dev(const float *x, const float *x_hat, size_t ny, size_t nx, double eps, int nbins,
                         unsigned long long *hist, ebcc_error_stats *out, void *stream);

/* --------------------------------------------------- JPEG 2000 codestream */
/* The base layer of an EBCC stream rewritten as a JPEG 2000 Part 1
 * codestream (Materials and Methods: the base layer is a JPEG 2000 image; the
 * syntax is ITU-T T.800 Annex A markers and Annex B packets).  No coding pass
 * is re-encoded: each code-block's kept passes and MQ codeword are copied.
 * The codestream has one tile, one signed 16-bit component, one quality
 * layer, LRCP progression, one precinct per resolution, the stream's
 * code-block size, default code-block style and the 9/7 irreversible
 * transform with scalar expounded quantisation.  A sample s stands for
 * mn + s / 16384 * (mx - mn) of the field (the stream's minimum and maximum,
 * also written as text in a COM marker): band b's step is 16384 times the
 * base layer's normalised step, i.e. exponent epsilon_b = 2 + gain_b + e_b
 * (gain_b = 0, 1, 1, 2 for LL, HL, LH, HH) and the same 11-bit mantissa; the
 * guard bits are the fewest (at least 1) that give every block's bit-planes
 * room, and a block's zero bit-planes are G + epsilon_b - 1 - K.  The residual
 * layer and the escape list are not part of it.
 * stream/len: a host EBCC stream.  *out: a host buffer the library allocates
 * and the caller releases with ebcc_free; *out_len its length.  Host code only
 * (no device work, callable without a GPU).
 * Errors: EINVAL (NULL argument, or a constant field: no base layer),
 * ECORRUPT (malformed stream), ECAPACITY (a step exponent outside 0..31 or
 * more than 7 guard bits needed), ENOMEM. */
int ebcc_j2k_codestream(const uint8_t *stream, size_t len, uint8_t **out, size_t *out_len);

/* ------------------------------------------------------------- N-D chunks */
/* The N-D front end (Materials and Methods, first paragraph): a 4-D float32
 * array of shape[4] = (T, P, H, W) -- time, level, latitude, longitude --
 * row-major (W contiguous), is split into chunks of chunk[4] = (cT, cP, cH,
 * cW) (an extent that is not a multiple of the chunk leaves smaller chunks at
 * the end of that axis); each chunk is flattened to a 2-D field of
 * (cT*cP*cH) rows by cW columns and compressed as a field of its own, with
 * its own range-relative or absolute bound.  Chunks are numbered row-major
 * over the chunk grid (the W chunk index fastest).
 * ebcc_chunk_count: the number of chunks, or EINVAL (a zero extent, or more
 * than 2^24 chunks).
 * ebcc_chunk_info: chunk k's origin and extent in the array (either may be
 * NULL) and its flattened 2-D shape ny x nx. */
long long ebcc_chunk_count(const size_t shape[4], const size_t chunk[4]);
int ebcc_chunk_info(const size_t shape[4], const size_t chunk[4], long long k, size_t origin[4], size_t extent[4],
                    size_t *ny, size_t *nx);
/* Compress every chunk of the device array `array` as one batch: the chunks
 * are flattened on the device into a buffer the library owns (kept between
 * calls), with no host copy; outs[k] (ebcc_chunk_count entries, caller-owned
 * device buffers of at least ebcc_max_stream_bytes(ny, nx) bytes) receives
 * chunk k's stream, status and stats as in ebcc_compress_batch_dev.
 * Synchronises `stream`.  Errors: EINVAL, ENONFINITE, ENOMEM, ECAPACITY,
 * ECUDA (the first failing chunk's status). */
int ebcc_compress_chunks_dev(const float *array, const size_t shape[4], const size_t chunk[4], double bound,
                             int bound_kind, const ebcc_params *p, ebcc_out_desc *outs, void *stream);
/* Decompress the streams of every chunk (device, streams[k].ny / nx the
 * chunk's flattened shape) back into the device array of shape[4] (each chunk
 * written in place).  Synchronises `stream`.  Errors: EINVAL (a chunk's shape
 * does not match), ECORRUPT, ENOMEM, ECUDA. */
int ebcc_decompress_chunks_dev(const ebcc_stream_desc *streams, const size_t shape[4], const size_t chunk[4],
                               float *array, void *stream);

/* ---------------------------------------------------------------- serving */
/* A request loop with continuous batching: requests that arrive while others
 * are on the GPU are admitted as slots and memory free up (HBM budget); four
 * workers (EBCC_SERVER_WORKERS, 1..8), each with its own stream and device
 * buffers (kept between groups, no allocation per request), run admitted
 * groups as batches -- a group's decompressions first, their results
 * published before its compressions run -- so groups overlap on the device.  A group's requests enter the device through a
 * request ring in page-locked host memory, read by an intake kernel that
 * waits on the ring's doorbell for at most 2 s (EBCC_ETIMEOUT for the group's
 * requests if it runs out).  Thread-safe per handle. */
typedef struct ebcc_server ebcc_server;

#define EBCC_REQ_COMPRESS 0
#define EBCC_REQ_DECOMPRESS 1

/* A request.  Compress: host field (ny*nx float32), bound, bound_kind.
 * Decompress: host stream of stream_len bytes, ny, nx.  The library copies the
 * inputs at submit time. */
typedef struct {
    int kind;
    const float *field;
    const uint8_t *stream;
    size_t stream_len;
    size_t ny, nx;
    double bound;
    int bound_kind;
} ebcc_request;

/* Result of a finished request: status; for compress a library-allocated
 * stream (free with ebcc_free); for decompress a library-allocated field of
 * ny*nx floats (free with ebcc_free); times in seconds from submit. */
typedef struct {
    int status;
    uint8_t *stream;
    size_t stream_len;
    float *field;
    double latency_s, queue_s;
} ebcc_result;

/* Create a server that admits work while its device memory stays within
 * hbm_budget_bytes; max_batch fields per batch (0 = 64).  Errors: EINVAL, ENOMEM, ECUDA. */
int ebcc_server_create(size_t hbm_budget_bytes, int max_batch, const ebcc_params *p, ebcc_server **s);
/* Queue a request; returns its ticket.  EBUDGET if the request alone exceeds the budget. */
int ebcc_server_submit(ebcc_server *s, const ebcc_request *r, uint64_t *ticket);
/* Non-blocking: EBCC_OK and *r filled if finished, EBCC_ETIMEOUT if not yet
 * (after waiting up to timeout_s seconds), EINVAL for an unknown ticket. */
int ebcc_server_poll(ebcc_server *s, uint64_t ticket, double timeout_s, ebcc_result *r);
/* Cancel a request that is still queued (EINVAL if unknown or already running). */
int ebcc_server_cancel(ebcc_server *s, uint64_t ticket);
/* Drain and destroy. */
int ebcc_server_destroy(ebcc_server *s);
/* Diagnostic of the server's request intake (the device-side wait the
 * serving loop runs for every group): `bytes` bytes written into a request
 * ring of page-locked host memory are copied to the device by the intake
 * kernel, which waits for the ring's doorbell for at most wait_s seconds
 * (0 < wait_s <= 60).  publish = 1: the host rings the doorbell after writing
 * the ring, as the server does; returns EBCC_OK when the bytes arrived
 * unchanged (ECORRUPT otherwise).  publish = 0: nothing rings it, the wait
 * runs out and the call returns EBCC_ETIMEOUT, with the device still usable.
 * Synchronous on `stream`.  Errors: EINVAL, ENOMEM, ECUDA. */
int ebcc_intake_check(size_t bytes, double wait_s, int publish, void *stream);

/* ------------------------------------------------ hot-path step entry points
 * Each runs one step of the device pipeline on caller-owned device buffers,
 * asynchronously on `stream`.  They exist so that each kernel can be checked
 * on its own against the CPU oracle. */

/* Forward 9/7 lifting DWT (T.800 Annex F; Algorithm 1 "DWT"): in -> out, both
 * ny*nx float32, Mallat layout, `levels` levels (reduced so every level sees
 * at least 2 samples per axis).  If norm_range > 0 the input is first mapped
 * to (x - norm_min) / norm_range (Materials and Methods: min-max normalisation). */
int ebcc_dwt_fwd_dev(const float *in, float *out, size_t ny, size_t nx, int levels,
                     double norm_min, double norm_range, void *stream);
/* Same forward DWT without any device allocation (the paper has no
 * counterpart; this is a library-usage variant).  ebcc_dwt_fwd_dev takes its
 * two scratch regions from cudaMalloc and returns them with cudaFree, which
 * synchronises the whole device; callers that cannot take that -- a
 * latency-critical loop sharing the GPU with other streams, or a process whose
 * device memory is fully committed to its own pools -- call this one instead.
 * Its scratch is one static device array of EBCC_DWT_STATIC_SCRATCH_FLOATS
 * floats (8 MiB) per device, owned by the library; the call needs
 * ceil(ny/2) * r4(ceil(nx/2)) + 16 floats (rounded up to 64) plus
 * ceil(ny/4) * r4(ceil(nx/4)) + 16, r4 rounding up to a multiple of 4, i.e.
 * fields up to about 6.7 M points (1441 x 2880 fits), and returns
 * EBCC_ECAPACITY, touching nothing, beyond that.  Nothing in the scratch has
 * to start at zero.  The first call on a device looks up the array's address
 * (cudaGetSymbolAddress, with that device current) and may load the module,
 * so make it before any latency-critical region and before any stream
 * capture; the address is kept for the
 * life of the process, so the call must not be used after a cudaDeviceReset
 * of that device.  All calls on one device share the scratch: calls that
 * can overlap in time (different streams, or threads without ordering) race
 * on it and must be serialised by the caller.  Asynchronous on `stream`: the
 * caller synchronises before reading `out`.  Arguments and errors otherwise as
 * ebcc_dwt_fwd_dev. */
#define EBCC_DWT_STATIC_SCRATCH_FLOATS (2u * 1024u * 1024u)
int ebcc_dwt_fwd_static_dev(const float *in, float *out, size_t ny, size_t nx, int levels,
                            double norm_min, double norm_range, void *stream);
/* Inverse DWT (Algorithm 1 "IDWT"): in -> out, ny*nx float32. */
int ebcc_dwt_inv_dev(const float *in, float *out, size_t ny, size_t nx, int levels, void *stream);
/* Effective number of levels for a shape. */
int ebcc_effective_levels(size_t ny, size_t nx, int levels);

/* Dead-zone quantisation (T.800 Annex E) of Mallat-layout coefficients with the
 * base-layer steps for precision P: q[i] = sign * floor(|c| / delta_band). */
int ebcc_quantise_dev(const float *coef, int32_t *q, size_t ny, size_t nx, int levels, int P,
                      void *stream);
/* Base step size of a band (level 1..L, orient 0 LL, 1 HL, 2 LH, 3 HH): T.800
 * Annex E form 2^-eps (1 + mu/2048) of 2^-P / (synthesis norm). */
double ebcc_band_step(int P, int level, int orient);

/* EBCOT tier-1 (T.800 Annex D) of nblk code-blocks.  q: nblk blocks of w*h
 * int32 coefficients each (row-major, stride w), orient[k] per block.  Outputs
 * per block k: bytes at stream + k*cap (continuing MQ stream, cap bytes each),
 * K[k] bit-planes, npass[k] = 3K-2; per pass p (stride maxpass): pass_len
 * (bytes of the stream terminated after p), tail (flushed-tail bytes packed
 * little-endian), tail_len, dD (int64 distortion decrease in (step/2)^2 units);
 * D0[k]; spp[k*w*h + i] = 1 if coefficient i became significant in a
 * significance-propagation pass.  Errors: EINVAL, ECAPACITY (a block
 * overflowed cap or maxpass; reported after a synchronise). */
int ebcc_t1_encode_dev(const int32_t *q, const int32_t *orient, int nblk, int w, int h,
                       uint8_t *stream, int cap, int maxpass, int32_t *K, int32_t *npass,
                       int32_t *pass_len, uint32_t *tail, int32_t *tail_len, int64_t *dD,
                       int64_t *D0, uint8_t *spp, void *stream_);
/* Tier-1 decode of npass[k] passes of each block (bytes at stream + off[k],
 * len[k]): mag (known magnitude bits), plane (lowest known plane, -1 = zero),
 * neg. */
int ebcc_t1_decode_dev(const uint8_t *stream, const int64_t *off, const int32_t *len,
                       const int32_t *orient, const int32_t *K, const int32_t *npass, int nblk,
                       int w, int h, int32_t *mag, int8_t *plane, uint8_t *neg, void *stream_);

/* PCRD (rate allocation for Algorithm 1's ratio r): convex hulls of nblk
 * blocks from the tier-1 outputs (same layout), then the selection for a
 * byte budget: npass_out[k] passes per block (int32).  Synchronous. */
int ebcc_pcrd_dev(const int32_t *npass, const int32_t *pass_len, const int64_t *dD,
                  const int64_t *D0, int nblk, int maxpass, double budget, int32_t *npass_out,
                  void *stream);

/* SPIHT encoding (Said & Pearlman 1996; Algorithm 1 enc_SPIHT) of ny*nx int32
 * coefficients in Mallat layout with `levels` levels.  out: cap_bytes device
 * bytes; nbits_out (device int64) total bits; nmax_out (device int32) top
 * plane; sig_pos (device uint32 per coefficient, 0xFFFFFFFF = never
 * significant): bit offset of the coefficient's sign bit; lsp_idx (device
 * uint32 per coefficient): its place in the list of significant pixels;
 * refine_start (device int64[32]): bit offset of each plane's refinement pass.
 * Errors: EINVAL, ECAPACITY (after a synchronise). */
int ebcc_spiht_encode_dev(const int32_t *s, size_t ny, size_t nx, int levels, uint8_t *out,
                          size_t cap_bytes, int64_t *nbits_out, int32_t *nmax_out,
                          uint32_t *sig_pos, uint32_t *lsp_idx, int64_t *refine_start,
                          void *stream);
/* SPIHT decoding of the first nbits bits (Algorithm 1 dec_SPIHT): mag, plane
 * (-1 = not significant), neg per coefficient. */
int ebcc_spiht_decode_dev(const uint8_t *in, int64_t nbits, size_t ny, size_t nx, int levels,
                          int nmax, int32_t *mag, int8_t *plane, uint8_t *neg, void *stream);
/* Value implied by the first nbits bits, from the encoder trace, times
 * 2^step_exp: out[i] float32 (midpoint of the known interval). */
int ebcc_spiht_prefix_recon_dev(const int32_t *s, const uint32_t *sig_pos, const uint32_t *lsp_idx,
                                const int64_t *refine_start, int64_t nbits, size_t n, int step_exp,
                                float *out, void *stream);

/* Count points whose reconstruction meets the bound (Algorithm 1 q_A and the
 * max-error test): x original, an_hat normalised reconstruction (float32);
 * point i passes iff |x - (float)(mn + an_hat * range)| <= eps_abs - guard in
 * FP64.  *count_out (device int64) = passing points. */
int ebcc_count_within_dev(const float *x, const float *an_hat, size_t n, double mn, double range,
                          double eps_abs, double guard, int64_t *count_out, void *stream);

/* ------------------------------------------------------------- profiling
 * Kernel timing for measurement: while enabled, every kernel launch of the
 * library is bracketed by CUDA events recorded on its own stream.  Entries are
 * named after the kernel; total_ms is the summed device duration, bytes the
 * summed algorithmic bytes (minimum the kernel must move) of its launches. */
void ebcc_profile_enable(int on);
void ebcc_profile_reset(void);
int ebcc_profile_count(void);
int ebcc_profile_get(int i, const char **name, double *total_ms, long long *launches, double *bytes);

#ifdef __cplusplus
}
#endif
#endif
