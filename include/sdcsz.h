/*
 * sdcsz — SDC-resilient, error-bounded lossy compression of float32/float64 fields on one
 * NVIDIA GB300 (sm_103a).
 *
 * The library implements the independent-block SZ compressor with algorithm-based fault
 * tolerance of "SDC Resilient Error-bounded Lossy Compressor" (Li, Di, Zhao, Liang, Chen,
 * Cappello, arXiv 2010.03144): per-block Lorenzo or linear-regression prediction (Sec. 3.1),
 * linear-scaling quantization with an unpredictable-value fallback, one Huffman code for the
 * whole field with every block encoded on its own (Sec. 5.1), and the checks of Algorithm 1
 * (input checksums sum_in/isum_in, duplicated prediction and reconstruction, code checksums
 * sum_q/isum_q, reconstructed-data checksum sum_dc) and Algorithm 2 (block verification and
 * re-execution) fused into the GPU passes. The lossless Zstd stage of the paper is not part of
 * this library.
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are CUDA device pointers; h_* and plain struct pointers are host
 *    pointers. The caller owns every buffer; the library allocates no device memory.
 *  - `stream` is a cudaStream_t (passed as void* so this header needs no CUDA headers); all
 *    device work is enqueued on it. NULL means the legacy default stream.
 *  - Fields are dense, C order (last dimension fastest), dims[0] the slowest.
 *  - Return value 0 = success; a negative SDCSZ_E* code otherwise. Soft errors that were
 *    detected and corrected still return 0 and are counted in the report.
 *  - A call returns after enqueueing its work unless it has a host output to fill
 *    (`out_bytes`, `report`); then it synchronizes `stream` before returning. Errors found on
 *    the device (invalid error bound, capacity, corrupt stream, spin timeout) are returned only
 *    by calls that synchronize; the stream header and the per-block status record them too.
 *  - Calls on different streams must use different workspaces and outputs.
 */
#ifndef SDCSZ_H
#define SDCSZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SDCSZ_VERSION 1

/* Error codes. */
#define SDCSZ_OK 0
#define SDCSZ_EINVAL (-1)    /* bad argument: dims, block, bins, eb <= 0 / non-finite, ... */
#define SDCSZ_ECAPACITY (-2) /* output or workspace buffer too small */
#define SDCSZ_EFORMAT (-3)   /* not a valid sdcsz stream (magic, version, sizes, code table) */
#define SDCSZ_ESDC (-4)      /* >= 1 block failed verification twice (Alg. 2: "SDC in
                                compression"); the block status array names those blocks,
                                every other block is decompressed normally */
#define SDCSZ_ETIMEOUT (-5)  /* a bounded device wait gave up (never expected) */
#define SDCSZ_ECUDA (-6)     /* a CUDA runtime call failed */

typedef enum { SDCSZ_F32 = 0, SDCSZ_F64 = 1 } sdcsz_dtype;
typedef enum { SDCSZ_EB_ABS = 0, SDCSZ_EB_REL = 1 } sdcsz_eb_mode;
typedef enum { SDCSZ_PRED_AUTO = 0, SDCSZ_PRED_LORENZO = 1, SDCSZ_PRED_REGRESSION = 2 } sdcsz_predictor;

/*
 * The compression problem as the paper states it (Alg. 1 input: original data ori[] and
 * error bound e).
 *  ndim        1, 2 or 3.
 *  dtype       sdcsz_dtype.
 *  dims        dims[0..ndim-1], slowest first; each <= 2^40, product <= 2^40. A zero extent
 *              gives an empty field.
 *  block       block edge per dimension (Sec. 5.1 independent blocks), 0 = default
 *              (3D 6, 2D 12, 1D 128). Limits: 3D 2..16, 2D 2..64, 1D 2..4096, and at most
 *              4096 points per block. Edge blocks are cut to the field.
 *  eb_mode/eb  absolute bound, or value-range relative: eb_abs = eb * (max - min) over the
 *              finite values, rounded to dtype (falls back to eb when the range is 0).
 *  quant_bins  number of quantization bins, even, 2..65536; 0 = 65536.
 *  abft        1 = fault-tolerant mode (the paper's ftrsz), 0 = independent blocks without
 *              checks (rsz).
 *  predictor   sdcsz_predictor; AUTO selects per block by estimated error (Algorithm 1).
 */
typedef struct {
  uint32_t ndim;
  uint32_t dtype;
  uint64_t dims[3];
  uint32_t block[3];
  uint32_t eb_mode;
  double eb;
  uint32_t quant_bins;
  uint32_t abft;
  uint32_t predictor;
  /* bit 0 -- 0 = raw: regression coefficients and unpredictable values in sections of their
   * own, as stored values; 1 = compact: coefficients as integer multiples of eb/(16 B_a)
   * (slopes) and eb/16 (intercept), written as length-prefixed zigzag integers at the head of
   * the block's payload, and each unpredictable value right after its code 0 with only the
   * mantissa bits the bound needs (SZ's own encodings, kept block-local).
   * bit 1 -- the lossless stage that ends Algorithm 1 (Zstd in the paper): an order-0 rANS
   * coder over everything after the block tables (sum_dc, coefficients, unpredictable values,
   * payload) in 16 KiB chunks; the header and random-access tables stay as they are. Needs a
   * 16-byte aligned output (and stream, when decompressing) and a larger decompression
   * workspace (sdcsz_decompress_workspace_size_for); not available in batches. */
  uint32_t encoding;
} sdcsz_params;

/* Counters of one call (Algorithm 2 reports corrected errors and SDCs to the user). */
typedef struct {
  uint64_t blocks;
  uint64_t regression_blocks;
  uint64_t unpredictable_points;
  uint64_t compressed_bytes;
  uint64_t input_corrected;         /* input words repaired with sum_in/isum_in */
  uint64_t codes_corrected;         /* codes repaired with sum_q/isum_q */
  uint64_t dup_mismatch_corrected;  /* f_dup / dec_dup disagreed (Algorithm 1) */
  uint64_t decomp_reexec_corrected; /* blocks fixed by re-execution (Algorithm 2) */
  uint64_t uncorrectable_blocks;    /* detected, not correctable (outside the single-error model) */
  uint64_t bound_violations;        /* verify with an original: points with |x - x'| > eb */
  double eb_abs;                    /* the absolute bound used */
  double max_abs_err;               /* verify with an original: max |x - x'| over finite points */
} sdcsz_report;

/* Block status values written by decompress/verify. */
#define SDCSZ_BLOCK_OK 0
#define SDCSZ_BLOCK_CORRECTED 1     /* checksum mismatch fixed by re-execution */
#define SDCSZ_BLOCK_SDC 2           /* checksum mismatch twice: SDC in compression */
#define SDCSZ_BLOCK_BAD 3           /* undecodable block data */

/* Upper bound on the stream size for `p` (every point unpredictable with a 24-bit code). */
int sdcsz_compress_bound(const sdcsz_params* p, size_t* max_bytes);

/* Device workspace bytes needed by sdcsz_compress for `p` (codes, per-block checksums,
 * histogram, codebook, scan state). 256-byte aligned base required. */
int sdcsz_workspace_size(const sdcsz_params* p, size_t* bytes);

/* Device workspace bytes needed by sdcsz_decompress, sdcsz_verify and
 * sdcsz_decompress_region for any stream without the lossless stage (the least they accept). */
size_t sdcsz_decompress_workspace_size(void);

/* Device workspace bytes recommended to decompress, verify or take a region of the stream whose
 * first 128 bytes (the header) are at h_header in HOST memory; nbytes is the stream's size.
 * With the lossless stage this includes the stream without it. For 3D cube blocks of edge 16
 * (float32) or 10, 12, 16 (float64), sdcsz_decompress uses a two-pass decoder when the workspace
 * has this size: the blocks' codes (2 bytes a point), unpredictable values (one value a point)
 * and a few bytes a block; a workspace of at least sdcsz_decompress_workspace_size() bytes (plus
 * the lossless stage's part) but less than this decodes the same values with the one-pass
 * kernels, more slowly. SDCSZ_EFORMAT for a bad header. */
int sdcsz_decompress_workspace_size_for(const void* h_header, size_t nbytes, size_t* bytes);

/*
 * Compress one field (Alg. 1 without the Zstd stage).
 *  d_field     device pointer to the field (dtype, dims from p). Read only.
 *  d_out       device buffer of out_cap bytes for the stream (size it with
 *              sdcsz_compress_bound; a smaller buffer returns SDCSZ_ECAPACITY if it overflows).
 *  out_bytes   host, nullable: receives the stream size (synchronizes).
 *  d_ws        device workspace of ws_bytes >= sdcsz_workspace_size(p), 256-byte aligned.
 *  report      host, nullable: receives the counters (synchronizes).
 * The stream is self-describing: its header carries dims, dtype, block, bins, abft and eb.
 */
int sdcsz_compress(const void* d_field, const sdcsz_params* p, void* d_out, size_t out_cap, size_t* out_bytes,
                   void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream);

/*
 * Decompress a stream (Alg. 2): Huffman decoding and Lorenzo/regression reconstruction of
 * every block, then (abft streams) each block's checksum is compared with sum_dc and a
 * mismatching block is decompressed once more from its compressed bytes.
 *  d_stream/nbytes  device pointer to the stream and its length.
 *  d_field     device buffer of field_bytes >= points * sizeof(dtype).
 *  d_block_status   device, nullable: one SDCSZ_BLOCK_* byte per block.
 * Returns SDCSZ_ESDC when a block failed twice (when it synchronizes).
 */
int sdcsz_decompress(const void* d_stream, size_t nbytes, void* d_field, size_t field_bytes,
                     uint8_t* d_block_status, void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream);

/*
 * Verify a stream without writing a field: the decompression and checksum checks of Alg. 2.
 * With d_original (device, nullable) also checks every point against the bound
 * (|x - x'| <= eb_abs; non-finite points must match bit for bit) and reports max |x - x'|.
 */
int sdcsz_verify(const void* d_stream, size_t nbytes, const void* d_original, uint8_t* d_block_status,
                 void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream);

/*
 * Profiling variants: the same work as sdcsz_compress / sdcsz_decompress, with CUDA events
 * recorded on `stream` between the stages; the call synchronizes and writes the elapsed
 * milliseconds of each stage to stage_ms (host). Compression has 5 stages: buffer reset,
 * K1 preparation (range, sum_in/isum_in, regression, estimates), K2 prediction/quantization,
 * K3 Huffman code, K4 encoding (with the lossless stage, when on). Decompression has 1
 * stage: K5 (after undoing the lossless stage, when on).
 */
int sdcsz_compress_traced(const void* d_field, const sdcsz_params* p, void* d_out, size_t out_cap, size_t* out_bytes,
                          void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream, float* stage_ms);
int sdcsz_decompress_traced(const void* d_stream, size_t nbytes, void* d_field, size_t field_bytes,
                            uint8_t* d_block_status, void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream,
                            float* stage_ms);

/*
 * Deferred stage timing, for timing many calls without a host wait in each. Between
 * sdcsz_trace_begin and sdcsz_trace_end, every sdcsz_compress, sdcsz_decompress and
 * sdcsz_verify call (from any host thread) records CUDA events between its stages on its own
 * stream (the stages of the profiling variants above) and returns as it would untimed; the
 * events are created by sdcsz_trace_begin, so the calls create none.
 *  - sdcsz_trace_begin(max_calls): opens the recorder for up to max_calls calls (1 to 2^20;
 *    6 CUDA events each, on the current device). SDCSZ_EINVAL when max_calls is out of range
 *    or a recorder is already open; SDCSZ_ECUDA when the events cannot be created.
 *  - sdcsz_trace_end(kinds, stage_ms, cap_calls, n_calls): waits for the recorded events,
 *    writes per call, in call order, its kind to kinds[c] (host; 0 compress, 1 decompress,
 *    2 verify) and its stage milliseconds to stage_ms[5c .. 5c+4] (host; compression: reset,
 *    K1, K2, K3, K4; decompression and verification: K5 in the first, zeros after), and the
 *    number of calls to *n_calls (nullable); then closes the recorder and frees its events.
 *    Calls that returned an error before their last stage are left out. SDCSZ_EINVAL when no
 *    recorder is open; SDCSZ_ECAPACITY when calls were made beyond max_calls (those are not
 *    timed) or more calls were timed than cap_calls (the first cap_calls are written);
 *    SDCSZ_ECUDA when an event cannot be read. Call it after every call made while the
 *    recorder was open has returned.
 */
int sdcsz_trace_begin(size_t max_calls);
int sdcsz_trace_end(int32_t* kinds, float* stage_ms, size_t cap_calls, size_t* n_calls);

/*
 * Allocation-free compression. The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory when they compress: callbacks and
 * latency-critical serving loops that must not enter an allocator (a cudaMalloc can
 * synchronize the device and take milliseconds), and hosts whose device memory belongs to
 * another framework's pool, which the library must not grow or fragment. It runs the same
 * kernels as sdcsz_compress, with the workspace in a fixed 64 MiB device array that every GPU
 * loading this library holds until the process exits; it calls no allocator. Arguments as
 * for sdcsz_compress, without d_ws/ws_bytes.
 *  - Returns SDCSZ_ECAPACITY when sdcsz_workspace_size(p) exceeds 64 MiB: compare the two
 *    before calling. At the default block sizes that allows about 6.4 million float32 points
 *    (a 186^3 cube, a 2592^2 square) or about 4.7 million float64 points (168^3, 2172^2); the
 *    limit moves a little with the block size, and the lossless stage lowers it.
 *  - The first call on a device looks up the array's device address (with that device
 *    current) and keeps it for the life of the process; make that first call before any
 *    stream capture. Do not call this entry point after cudaDeviceReset in the same process:
 *    the kept address belongs to the context that the reset destroyed.
 *  - All calls share the array and it keeps the last call's contents (each call clears what
 *    must start at zero): calls whose GPU work overlaps (different streams, or different host
 *    threads) race and corrupt each other's output. Serialize them.
 */
int sdcsz_compress_noalloc(const void* d_field, const sdcsz_params* p, void* d_out, size_t out_cap,
                           size_t* out_bytes, sdcsz_report* report, void* stream);

/*
 * Random-access (region) decompression: only the blocks that intersect the box
 * [lo[a], hi[a]) (a < ndim, the field's axis order, element coordinates) are decoded and
 * verified (each block is independent, Sec. 5.1), and the box is written densely (C order,
 * its own shape) to d_out (out_bytes >= box points * element size). d_block_status (may be
 * NULL; else room for prod_a (floor((hi[a]-1)/B[a]) - floor(lo[a]/B[a]) + 1) bytes) receives
 * one status per intersecting block, in row-major order of the box's block range; the report
 * counts those blocks. lo and hi each hold ndim values; an empty or out-of-field box is
 * SDCSZ_EINVAL. Same return codes as sdcsz_decompress; the header
 * is read to the host first (one synchronisation).
 */
int sdcsz_decompress_region(const void* d_stream, size_t nbytes, const uint64_t* lo, const uint64_t* hi, void* d_out,
                            size_t out_bytes, uint8_t* d_block_status, void* d_ws, size_t ws_bytes,
                            sdcsz_report* report, void* stream);

/* Parse a stream header held in HOST memory (the first 128 bytes suffice for dims and
 * dtype; total_bytes is the full stream length). */
int sdcsz_read_header(const void* h_stream, size_t nbytes, sdcsz_params* out, uint64_t* total_bytes);

/* Static string for an error code. */
const char* sdcsz_strerror(int code);

/*
 * Batches (no counterpart in the paper, which compresses one field per call). A batch
 * compresses up to 64 fields of any shapes, dtypes and parameters with one persistent launch
 * per stage and kernel shape: the fields are rows of a device-side job table and the CTAs of
 * each launch pull (field, block range) items from a queue counter in the workspace. Each
 * field's stream is byte-identical to sdcsz_compress of that field with the same parameters.
 *
 *   sdcsz_batch_create       validate the items and plan the workspace (host only); the
 *                            item array is copied.
 *   sdcsz_batch_workspace_size  bytes of device workspace the batch needs (one buffer,
 *                            256-byte aligned, owned by the caller, reused by every run).
 *   sdcsz_batch_bind         bind the workspace, build the job table and copy it to the
 *                            device (waits for `stream`); drops any captured graph.
 *   sdcsz_batch_set_fields   point the batch at other field / output buffers (NULL arrays
 *                            keep the current ones); shapes and parameters stay. Waits for
 *                            `stream`, so no run may be in flight on another stream.
 *   sdcsz_batch_compress     enqueue the compression of every field on `stream`; no host
 *                            synchronisation and no allocation, so it may be captured.
 *   sdcsz_batch_capture      capture sdcsz_batch_compress into a CUDA graph owned by the
 *                            batch (`stream` must not be the legacy default stream).
 *   sdcsz_batch_launch       replay the captured graph on `stream` (or enqueue directly when
 *                            nothing was captured).
 *   sdcsz_batch_results      wait for `stream`, then per field the stream size (0 on error)
 *                            and the report; returns the first field's error, if any.
 *   sdcsz_batch_destroy      free the host-side plan (not the caller's device memory).
 * The workspace and outputs belong to one run at a time: runs of one batch on different
 * streams must not overlap.
 */
typedef struct sdcsz_batch_item {
  const void* d_field;
  sdcsz_params params;
  void* d_out;
  size_t out_cap;
} sdcsz_batch_item;

typedef struct sdcsz_batch sdcsz_batch;

int sdcsz_batch_create(const sdcsz_batch_item* items, uint32_t n, sdcsz_batch** out);
int sdcsz_batch_workspace_size(const sdcsz_batch* b, size_t* bytes);
int sdcsz_batch_bind(sdcsz_batch* b, void* d_ws, size_t ws_bytes, void* stream);
int sdcsz_batch_set_fields(sdcsz_batch* b, const void* const* d_fields, void* const* d_outs, const size_t* out_caps,
                           void* stream);
int sdcsz_batch_compress(sdcsz_batch* b, void* stream);
int sdcsz_batch_capture(sdcsz_batch* b, void* stream);
int sdcsz_batch_launch(sdcsz_batch* b, void* stream);
int sdcsz_batch_results(sdcsz_batch* b, size_t* out_bytes, sdcsz_report* reports, void* stream);
void sdcsz_batch_destroy(sdcsz_batch* b);

/*
 * Block-size autotuner (no counterpart in the paper, which fixes the block size by a
 * rate-distortion study, Sec. 6.2.1). Compresses the leading `sample_points` of d_field (whole
 * planes in 3D, rows in 2D; the shape, dtype and bound of *p) once per candidate edge (the
 * same edge on every axis, each a valid block of p's dimensionality), timing `3` runs with
 * CUDA events. results[c] receives the candidate's time, stream size, throughput and ratio;
 * *best the index of the fastest candidate whose stream is at most (1 + size_slack) times the
 * smallest. Allocates its scratch with cudaMallocAsync on `stream` and waits for it (a tuning
 * call, not for the hot path).
 */
typedef struct sdcsz_tune_result {
  uint32_t block;
  double ms;       /* mean compression time of the sample */
  uint64_t bytes;  /* stream size of the sample */
  double gbs;      /* sample bytes / ms */
  double ratio;    /* sample bytes / stream bytes */
} sdcsz_tune_result;

int sdcsz_autotune_block(const void* d_field, const sdcsz_params* p, const uint32_t* candidates, uint32_t n_cand,
                         uint64_t sample_points, double size_slack, void* stream, sdcsz_tune_result* results,
                         uint32_t* best);

/* Number of CUDA kernels the library has launched in this process so far (all devices, all
 * entry points). Instrumentation only; the paper has no counterpart. */
unsigned long long sdcsz_kernel_launches(void);

/*
 * Soft-error simulation for tests (the paper's evaluation mode A, Sec. 6.1.2, and the
 * transient errors of Sec. 6.4.3-6.4.4). One record flips one bit:
 *  SDCSZ_SITE_INPUT  index = global 32-bit word of the field (float64 = 2 words, low
 *                    first); flipped in the caller's field buffer after the input checksums
 *                    are taken. The flip stays in d_field after the call.
 *  SDCSZ_SITE_CODE   block, index = point in the block; the stored quantization code,
 *                    after its checksums are taken, before encoding.
 *  SDCSZ_SITE_COEF   block, index = coefficient; after predictor selection, before use.
 *  SDCSZ_SITE_PRED   block, index = point; the first evaluation of the prediction.
 *  SDCSZ_SITE_RECON  block, index = point; the first evaluation of the reconstruction.
 *  SDCSZ_SITE_DECOMP block, index = point; the reconstructed value in the first decompression.
 *  SDCSZ_SITE_REWALK block (index and bit unused); changes no value. A block of the
 *                    compile-time shapes walked without per-point voting is handled as if its
 *                    duplicate evaluations had disagreed: its codes are withdrawn from the
 *                    histogram and it is walked again with voting, which counts one
 *                    dup_mismatch_corrected. No effect with ABFT off, in blocks that also
 *                    have a PRED or RECON record (those are walked with voting from the
 *                    start) and in blocks of other shapes. The output equals the clean run's.
 * d_flips is a device array of n records sorted by (block, site, index).
 */
#define SDCSZ_SITE_INPUT 1
#define SDCSZ_SITE_CODE 2
#define SDCSZ_SITE_COEF 3
#define SDCSZ_SITE_PRED 4
#define SDCSZ_SITE_RECON 5
#define SDCSZ_SITE_DECOMP 6
#define SDCSZ_SITE_REWALK 7
typedef struct {
  uint32_t site;
  uint32_t bit;
  uint64_t block;
  uint64_t index;
} sdcsz_flip;

int sdcsz_debug_compress_flips(const void* d_field, const sdcsz_params* p, void* d_out, size_t out_cap,
                               size_t* out_bytes, void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream,
                               const sdcsz_flip* d_flips, size_t n_flips);
int sdcsz_debug_decompress_flips(const void* d_stream, size_t nbytes, void* d_field, size_t field_bytes,
                                 uint8_t* d_block_status, void* d_ws, size_t ws_bytes, sdcsz_report* report,
                                 void* stream, const sdcsz_flip* d_flips, size_t n_flips);

/*
 * Request server (no counterpart in the paper). One scheduler thread and `slots` CUDA
 * streams on the current device. Requests are admitted in arrival order as soon as a slot is
 * free and the device memory they need fits in `hbm_budget` (their workspace, plus the
 * output when d_out is NULL and the server provides it); admitted requests run concurrently,
 * and a slot goes to the next pending request the moment its work completes (continuous
 * batching, no batch boundaries). Each request runs the same kernels as the single-call
 * entry points, so its result is the same alone and in any mix.
 *   compress:   d_in = field (device), params; result = the stream (d_out, or server memory)
 *   decompress: d_in/in_bytes = stream (device); result = the field (d_out, or server memory)
 *   verify:     d_in/in_bytes = stream, d_original optional; result = report only
 * Caller buffers (d_in, d_out, d_original, d_flips) must stay valid until the request's
 * completion is polled. Server-provided results stay in device memory (and count against
 * the budget) until sdcsz_server_release(id). SITE_INPUT flips modify d_in, as with
 * sdcsz_debug_compress_flips. Completions carry the server-clock times (seconds) of submit,
 * admission and completion (observed by the scheduler), the status (an SDCSZ_E* code or
 * SDCSZ_OK; decompress/verify return SDCSZ_ESDC when a block failed twice) and the report.
 * sdcsz_server_destroy finishes every submitted request, then frees the server's memory.
 */
enum { SDCSZ_OP_COMPRESS = 1, SDCSZ_OP_DECOMPRESS = 2, SDCSZ_OP_VERIFY = 3 };

typedef struct sdcsz_server_config {
  uint64_t hbm_budget; /* bytes of device memory admitted requests may hold */
  uint32_t slots;      /* requests on the device at once (1..64) */
  uint32_t reserved;
} sdcsz_server_config;

typedef struct sdcsz_request {
  uint32_t op;
  uint32_t reserved;
  uint64_t id;               /* returned with the completion */
  const void* d_in;
  size_t in_bytes;           /* decompress / verify: stream length */
  sdcsz_params params;       /* compress */
  void* d_out;               /* NULL: the server provides the output */
  size_t out_cap;
  const void* d_original;    /* verify: optional */
  const sdcsz_flip* d_flips; /* optional soft-error records (sorted by block) */
  size_t n_flips;
} sdcsz_request;

typedef struct sdcsz_completion {
  uint64_t id;
  uint32_t op;
  int status;
  const void* d_result;
  size_t result_bytes;
  sdcsz_report report;
  double t_submit, t_admit, t_done;
} sdcsz_completion;

typedef struct sdcsz_server_stats {
  uint64_t pending, in_flight, admitted, completed, bytes_in_use, peak_bytes;
} sdcsz_server_stats;

typedef struct sdcsz_server sdcsz_server;

int sdcsz_server_create(const sdcsz_server_config* cfg, sdcsz_server** out);
int sdcsz_server_submit(sdcsz_server* s, const sdcsz_request* r);
int sdcsz_server_poll(sdcsz_server* s, sdcsz_completion* out, uint32_t max, uint32_t* n, uint32_t wait_us);
int sdcsz_server_release(sdcsz_server* s, uint64_t id);
int sdcsz_server_get_stats(sdcsz_server* s, sdcsz_server_stats* out);
void sdcsz_server_destroy(sdcsz_server* s);

/*
 * Sharded compression: one field split over several GPUs (ranks) into slabs of whole block rows
 * along its slowest axis (axis 0 of dims), written as the stream sdcsz_compress writes for the
 * whole field, byte for byte. Sec. 5.1 of the paper makes the blocks independent, so a slab's
 * blocks compress exactly as inside the field once the ranks agree on three field-wide values:
 * the value range (value-range relative bound, Fig. 2), the code histogram (one Huffman code,
 * Algorithm 1) and the running totals of payload bytes, unpredictable values and regression
 * blocks (where each block's data goes, Sec. 5.1). The stages run in this order on every rank,
 * with an exchange (a collective over the ranks, made by the caller) between them:
 *
 *  1. sdcsz_shard_prep: the slab's first pass (range, input checksums, regression,
 *     estimates). range_keys[2] (host) receive the slab's range in an order-preserving form.
 *       exchange: elementwise maximum of range_keys over the ranks.
 *  2. sdcsz_shard_predict(the field's range_keys): the field's bound, then prediction,
 *     quantization and the ABFT checks of the slab. counts[3] (host): the slab's regression
 *     blocks, unpredictable points, uncorrectable blocks; *d_hist (device, 65536 u64 inside the
 *     workspace): the slab's code histogram.
 *       exchange: sum of counts, and of the histograms in place.
 *  3. sdcsz_shard_encode(the field's counts): the Huffman code of the field's histogram (the
 *     same on every rank) and the slab's blocks encoded at the field's layout into d_out
 *     (header != 0 on exactly one rank: it also writes the header and the code table).
 *     totals[4] (host): the slab's payload bytes, unpredictable values (as encoded),
 *     regression blocks and uncorrectable blocks.
 *       exchange: the sum of totals over the ranks of the earlier slabs (prefix[3], the first
 *       three) and over all ranks (field_totals[4]).
 *  4. sdcsz_shard_assemble(prefix, field_totals): the slab's payload, unpredictable values,
 *     coefficients and random-access table entries at their places in d_out; the header rank
 *     also the field's totals. *out_bytes: the field's stream size; report: the slab's counters.
 *       exchange: the byte-wise sum of every rank's d_out over [0, out_bytes) is the stream (the
 *       ranks write disjoint bytes, except bitmap words of two slabs whose bits are disjoint).
 *
 * p_field: the whole field's parameters (raw or compact encoding; the lossless stage is
 * SDCSZ_EINVAL). The slab is block rows [slab_b0, slab_b1) of axis 0: planes
 * [slab_b0 * B, min(slab_b1 * B, dims[0])), B the block edge along axis 0, contiguous in C
 * order at d_slab. d_ws: sdcsz_shard_workspace_size bytes, 256-byte aligned, kept through the
 * four stages. d_out: out_cap >= sdcsz_compress_bound(p_field) bytes, zero when stage 3 starts.
 * Each stage synchronises the stream once to return its host values. Return codes as for
 * sdcsz_compress.
 */
int sdcsz_shard_workspace_size(const sdcsz_params* p_field, uint64_t slab_b0, uint64_t slab_b1, size_t* bytes);
int sdcsz_shard_prep(const void* d_slab, const sdcsz_params* p_field, uint64_t slab_b0, uint64_t slab_b1, void* d_ws,
                     size_t ws_bytes, uint64_t* range_keys, void* stream);
int sdcsz_shard_predict(const void* d_slab, const sdcsz_params* p_field, uint64_t slab_b0, uint64_t slab_b1,
                        void* d_ws, size_t ws_bytes, const uint64_t* field_range_keys, uint64_t* counts,
                        void** d_hist, void* stream);
int sdcsz_shard_encode(const sdcsz_params* p_field, uint64_t slab_b0, uint64_t slab_b1, void* d_ws, size_t ws_bytes,
                       const uint64_t* field_counts, int header, void* d_out, size_t out_cap, uint64_t* totals,
                       void* stream);
int sdcsz_shard_assemble(const sdcsz_params* p_field, uint64_t slab_b0, uint64_t slab_b1, void* d_ws,
                         size_t ws_bytes, const uint64_t* prefix, const uint64_t* field_totals, int header,
                         void* d_out, size_t out_cap, size_t* out_bytes, sdcsz_report* report, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SDCSZ_H */
