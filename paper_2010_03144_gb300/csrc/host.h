// Host-side helpers of the library shared by its translation units (entry points, batches,
// the request server). Not part of the C ABI.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include "sdcsz_internal.cuh"

namespace sdcsz {
inline namespace host {

// NVTX range around the host-side enqueue of one stage, so that a timeline profiler groups
// the stage's kernels under its name.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Byte offsets of the regions of a compression workspace.
struct WsPlan {
  size_t state, sum_in, isum_in, sum_q, isum_q, sum_dc, coef, est, pflag, flags, coefT, hist, codebook, gt, sort_keys,
      node_w, node_parent, codes, ustage, etmp, total;
  // lossless stage
  size_t raw, raw_cap, llw, llst, llsz, lltop, lloff, llhist, llcum;
};

// Worst-case size of a stream before the lossless stage.
uint64_t raw_stream_bound(const Geo& g);

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
int sm_count();
int make_geo(const sdcsz_params* p, Geo* g);
WsPlan plan_ws(const Geo& g);
Ws bind_ws(void* base, const WsPlan& p);
int map_error(unsigned int e);
// The State of a call to the host (synchronises the stream).
int read_state(const State* d_st, cudaStream_t s, State* h);
void fill_report(const State& h, uint64_t nb, sdcsz_report* r);
int parse_header(const uint8_t* s, uint64_t nbytes, Hdr* h, sdcsz_params* pout);

// Compression of one field on `stream`. With out_bytes and report both null it only
// enqueues work (no host synchronisation).
int compress_impl(const void* d_field, const sdcsz_params* p, void* d_out, size_t out_cap, size_t* out_bytes,
                  void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream, const sdcsz_flip* flips,
                  size_t n_flips, float* stage_ms = nullptr);

// Decompression (write) or verification of a stream whose header was already parsed to the
// host: clears the State at `st` and enqueues the decoder; no host synchronisation.
// A stream with the lossless stage is first decoded into `raw` (h.raw_total bytes, 16-byte
// aligned; unused otherwise).
int decode_enqueue(const void* d_stream, size_t nbytes, const Hdr& h, void* d_field, size_t field_bytes,
                   uint8_t* status, const void* d_orig, bool write, State* st, cudaStream_t s, const sdcsz_flip* flips,
                   size_t n_flips, uint8_t* raw = nullptr, uint8_t* wave = nullptr);

// Decompression workspace: the least (the State and the lossless stage's scratch) and the
// recommended (plus the two-pass decoder's buffers, for the shapes it serves).
size_t decode_ws_min(const Hdr& h);
size_t decode_ws_bytes(const Hdr& h);
int decompress_impl(const void* d_stream, size_t nbytes, void* d_field, size_t field_bytes, uint8_t* status,
                    const void* d_orig, bool write, void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream,
                    const sdcsz_flip* flips, size_t n_flips, float* stage_ms = nullptr);

}  // namespace host
}  // namespace sdcsz
