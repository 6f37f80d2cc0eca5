// Host entry points of libsdcsz (the C ABI declared in include/sdcsz.h).
//
// Compression enqueues K1 (k_prep) -> K2 (k_predict) -> K3 (k_codebook) -> K4 (k_encode) on
// the caller's stream with no host round trip; decompression and verification read the
// 128-byte stream header to the host, then enqueue K5 (k_decode). All device memory comes
// from the caller (stream, field, workspace).
#include <algorithm>
#include <cstring>
#include <atomic>
#include <mutex>

#include "sdcsz_internal.cuh"

namespace sdcsz {

namespace {

constexpr uint64_t kMaxPoints = 1ull << 40;

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (dev < 0 || dev >= 64) return 148;
  if (!cached[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 1;
  }
  return cached[dev];
}

}  // namespace

namespace {
std::atomic<unsigned long long> g_launches{0};
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

cudaStream_t side_stream() {
  static std::mutex mu;
  static cudaStream_t streams[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!streams[dev]) cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
  return streams[dev];
}

namespace {

// Validate parameters and fill the padded-3D geometry.
int make_geo(const sdcsz_params* p, Geo* g) {
  if (!p) return SDCSZ_EINVAL;
  if (p->ndim < 1 || p->ndim > 3 || p->dtype > 1 || p->eb_mode > 1 || p->abft > 1 || p->predictor > 2 ||
      p->reserved != 0)
    return SDCSZ_EINVAL;
  if (!(p->eb > 0.0) || !(p->eb < 1.0 / 0.0)) return SDCSZ_EINVAL;
  const uint32_t bins = p->quant_bins ? p->quant_bins : 65536u;
  if (bins < 2 || bins > 65536 || (bins & 1)) return SDCSZ_EINVAL;
  std::memset(g, 0, sizeof(*g));
  g->ndim = (int)p->ndim;
  g->dtype = (int)p->dtype;
  const int off = 3 - g->ndim;
  for (int a = 0; a < 3; ++a) {
    g->d[a] = 1;
    g->B[a] = 1;
    g->nbd[a] = 1;
  }
  const uint32_t def = g->ndim == 3 ? 6 : (g->ndim == 2 ? 12 : 128);
  const uint32_t maxb = g->ndim == 3 ? 16 : (g->ndim == 2 ? 64 : 4096);
  uint64_t N = 1, nb = 1, P = 1;
  for (int a = 0; a < g->ndim; ++a) {
    const uint64_t n = p->dims[a];
    const uint32_t b = p->block[a] ? p->block[a] : def;
    if (n > kMaxPoints || b < 2 || b > maxb) return SDCSZ_EINVAL;
    g->d[off + a] = n;
    g->B[off + a] = b;
    g->nbd[off + a] = (n + b - 1) / b;
    if (n && N > kMaxPoints / n) return SDCSZ_EINVAL;
    N *= n;
    nb *= g->nbd[off + a];
    P *= b;
  }
  if (P > 4096 || N > kMaxPoints) return SDCSZ_EINVAL;
  g->N = N;
  g->nb = nb;
  g->P = (uint32_t)P;
  g->bins = bins;
  g->R = bins / 2;
  g->abft = (int)p->abft;
  g->predictor = (int)p->predictor;
  g->eb_mode = (int)p->eb_mode;
  g->e = p->eb;
  return SDCSZ_OK;
}

struct WsPlan {
  size_t state, sum_in, isum_in, sum_q, isum_q, sum_dc, coef, est, pflag, flags, coefT, hist, codebook, lb, sort_keys,
      node_w, node_parent, codes, ustage, total;
};

WsPlan plan_ws(const Geo& g) {
  WsPlan w;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t r = o;
    o = align256(o + bytes);
    return r;
  };
  const size_t nb = g.nb, s = g.dtype ? 8 : 4;
  const size_t ngroups = (nb + kGroup - 1) / kGroup;
  const size_t slots = ((nb + 31) / 32) * 32 * (size_t)g.P;
  const size_t pair_slots = ((nb + 31) / 32) * 32 * (size_t)pairs_of(g.P);
  w.state = take(sizeof(State));
  w.sum_in = take(8 * nb);
  w.isum_in = take(8 * nb);
  w.sum_q = take(8 * nb);
  w.isum_q = take(8 * nb);
  w.sum_dc = take(8 * nb);
  w.coef = take(16 * nb);
  w.est = take(8 * nb);
  w.pflag = take(nb);
  w.flags = take(nb);
  w.coefT = take(4 * s * nb);
  w.hist = take(8 * 65536);
  w.codebook = take(4 * 65536);
  w.lb = take(sizeof(LookBack) * std::max<size_t>(ngroups, 1));
  w.sort_keys = take(8 * 65536);
  w.node_w = take(8 * 65536);
  w.node_parent = take(4 * 2 * 65536 + 2 * 65536);
  w.codes = take(4 * pair_slots);
  w.ustage = take(s * slots);
  w.total = o;
  return w;
}

Ws bind_ws(void* base, const WsPlan& p) {
  uint8_t* b = static_cast<uint8_t*>(base);
  Ws w;
  w.st = reinterpret_cast<State*>(b + p.state);
  w.sum_in = reinterpret_cast<unsigned long long*>(b + p.sum_in);
  w.isum_in = reinterpret_cast<unsigned long long*>(b + p.isum_in);
  w.sum_q = reinterpret_cast<unsigned long long*>(b + p.sum_q);
  w.isum_q = reinterpret_cast<unsigned long long*>(b + p.isum_q);
  w.sum_dc = reinterpret_cast<unsigned long long*>(b + p.sum_dc);
  w.coef = reinterpret_cast<float4*>(b + p.coef);
  w.est = reinterpret_cast<float2*>(b + p.est);
  w.pflag = b + p.pflag;
  w.flags = b + p.flags;
  w.coefT = b + p.coefT;
  w.hist = reinterpret_cast<unsigned long long*>(b + p.hist);
  w.codebook = reinterpret_cast<uint32_t*>(b + p.codebook);
  w.lb = reinterpret_cast<LookBack*>(b + p.lb);
  w.sort_keys = reinterpret_cast<unsigned long long*>(b + p.sort_keys);
  w.node_w = reinterpret_cast<unsigned long long*>(b + p.node_w);
  w.node_parent = reinterpret_cast<uint32_t*>(b + p.node_parent);
  w.codes = reinterpret_cast<uint16_t*>(b + p.codes);
  w.ustage = b + p.ustage;
  return w;
}

int map_error(unsigned int e) {
  if (e & ERR_TIMEOUT) return SDCSZ_ETIMEOUT;
  if (e & ERR_FORMAT) return SDCSZ_EFORMAT;
  if (e & ERR_CAPACITY) return SDCSZ_ECAPACITY;
  if (e & (ERR_EB | ERR_FIELD)) return SDCSZ_EINVAL;
  return SDCSZ_OK;
}

int read_state(const State* d_st, cudaStream_t s, State* h) {
  if (cudaMemcpyAsync(h, d_st, sizeof(State), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SDCSZ_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SDCSZ_ECUDA;
  return SDCSZ_OK;
}

void fill_report(const State& h, uint64_t nb, sdcsz_report* r) {
  std::memset(r, 0, sizeof(*r));
  r->blocks = nb;
  r->regression_blocks = h.n_reg;
  r->unpredictable_points = h.n_unpred;
  r->compressed_bytes = h.total_bytes;
  r->input_corrected = h.input_corrected;
  r->codes_corrected = h.codes_corrected;
  r->dup_mismatch_corrected = h.dup_fixed;
  r->decomp_reexec_corrected = h.reexec_corrected;
  r->uncorrectable_blocks = h.uncorrectable;
  r->bound_violations = h.bound_viol;
  r->eb_abs = h.eb;
  double me;
  std::memcpy(&me, &h.max_err_bits, 8);
  r->max_abs_err = me;
}

// Optional stage timing: CUDA events recorded on the caller's stream between the kernels.
struct Trace {
  float* ms;
  int n;
  cudaEvent_t ev[8];
  int used = 0;
  cudaStream_t s = nullptr;
  bool on() const { return ms != nullptr; }
  void start(cudaStream_t st) {
    if (!on()) return;
    s = st;
    for (int q = 0; q <= n && q < 8; ++q) cudaEventCreate(&ev[q]);
    cudaEventRecord(ev[0], s);
    used = 1;
  }
  void mark() {
    if (!on() || used > n) return;
    cudaEventRecord(ev[used], s);
    ++used;
  }
  void finish() {
    if (!on()) return;
    cudaEventSynchronize(ev[used - 1]);
    for (int q = 0; q < n; ++q) ms[q] = 0.0f;
    for (int q = 1; q < used; ++q) cudaEventElapsedTime(&ms[q - 1], ev[q - 1], ev[q]);
    for (int q = 0; q < used; ++q) cudaEventDestroy(ev[q]);
    used = 0;
  }
};

int compress_impl(const void* d_field, const sdcsz_params* p, void* d_out, size_t out_cap, size_t* out_bytes,
                  void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream, const sdcsz_flip* flips,
                  size_t n_flips, float* stage_ms = nullptr) {
  Geo g;
  int rc = make_geo(p, &g);
  if (rc) return rc;
  if ((!d_field && g.N) || !d_out || !d_ws) return SDCSZ_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_ws) & 255) return SDCSZ_EINVAL;
  if (n_flips > 0xffffffffu || (n_flips && !flips)) return SDCSZ_EINVAL;
  const WsPlan plan = plan_ws(g);
  if (ws_bytes < plan.total) return SDCSZ_ECAPACITY;
  if (out_cap < (size_t)kHeaderBytes) return SDCSZ_ECAPACITY;
  const Ws w = bind_ws(d_ws, plan);
  Launch L;
  L.stream = static_cast<cudaStream_t>(stream);
  L.sms = sm_count();
  const uint32_t nf = (uint32_t)n_flips;
  Trace tr;
  tr.ms = stage_ms;
  tr.n = 5;
  cudaGetLastError();
  tr.start(L.stream);
  if (cudaMemsetAsync(w.st, 0, sizeof(State), L.stream) != cudaSuccess) return SDCSZ_ECUDA;
  if (cudaMemsetAsync(w.hist, 0, 8 * (size_t)g.bins, L.stream) != cudaSuccess) return SDCSZ_ECUDA;
  const size_t ngroups = (g.nb + kGroup - 1) / kGroup;
  if (ngroups && cudaMemsetAsync(w.lb, 0, sizeof(LookBack) * ngroups, L.stream) != cudaSuccess) return SDCSZ_ECUDA;
  tr.mark();
  launch_prep(d_field, g, w, L);
  if (nf) launch_flip_input(const_cast<void*>(d_field), g, flips, nf, w, L);
  tr.mark();
  if (g.nb) launch_predict(d_field, g, w, flips, nf, L);
  if (nf) launch_flip_codes(g, w, flips, nf, L);
  tr.mark();
  launch_codebook(g, w, static_cast<uint8_t*>(d_out), out_cap, L);
  tr.mark();
  launch_encode(g, w, static_cast<uint8_t*>(d_out), out_cap, L);
  tr.mark();
  if (cudaGetLastError() != cudaSuccess) return SDCSZ_ECUDA;
  tr.finish();
  if (out_bytes || report) {
    State h;
    rc = read_state(w.st, L.stream, &h);
    if (rc) return rc;
    if (report) fill_report(h, g.nb, report);
    rc = map_error(h.error);
    if (rc) return rc;
    if (out_bytes) *out_bytes = (size_t)h.total_bytes;
  }
  return SDCSZ_OK;
}

// Host-side header parse (the same checks as the stream layout requires).
int parse_header(const uint8_t* s, uint64_t nbytes, Hdr* h, sdcsz_params* pout) {
  if (nbytes < (uint64_t)kHeaderBytes || std::memcmp(s, "SDSZ", 4) != 0) return SDCSZ_EFORMAT;
  uint16_t ver;
  std::memcpy(&ver, s + 4, 2);
  if (ver != SDCSZ_VERSION) return SDCSZ_EFORMAT;
  sdcsz_params p;
  std::memset(&p, 0, sizeof(p));
  p.dtype = s[6];
  p.ndim = s[7];
  if (p.ndim < 1 || p.ndim > 3 || p.dtype > 1) return SDCSZ_EFORMAT;
  for (uint32_t a = 0; a < 3; ++a) std::memcpy(&p.dims[a], s + 8 + 8 * a, 8);
  for (uint32_t a = 0; a < 3; ++a) std::memcpy(&p.block[a], s + 32 + 4 * a, 4);
  for (uint32_t a = 0; a < p.ndim; ++a)
    if (p.block[a] == 0) return SDCSZ_EFORMAT;
  std::memcpy(&p.quant_bins, s + 44, 4);
  if (p.quant_bins == 0) return SDCSZ_EFORMAT;
  p.abft = s[48];
  p.predictor = s[49];
  p.eb_mode = s[50];
  std::memcpy(&p.eb, s + 64, 8);
  if (!(p.eb > 0.0)) p.eb = 1.0;  // the user bound is informational for decoding
  Geo g;
  if (make_geo(&p, &g)) return SDCSZ_EFORMAT;
  uint32_t n_live;
  uint64_t nb, n_reg, n_unpred, payload, total;
  double eb;
  std::memcpy(&n_live, s + 52, 4);
  std::memcpy(&eb, s + 56, 8);
  std::memcpy(&nb, s + 72, 8);
  std::memcpy(&n_reg, s + 80, 8);
  std::memcpy(&n_unpred, s + 88, 8);
  std::memcpy(&payload, s + 96, 8);
  std::memcpy(&total, s + 104, 8);
  if (nb != g.nb || n_live > g.bins || n_reg > g.nb || n_unpred > g.N) return SDCSZ_EFORMAT;
  if (p.dtype == 0) {
    const float ebf = (float)eb;
    if ((double)ebf != eb) return SDCSZ_EFORMAT;
  }
  if (!(eb > 0.0) || !(eb < 1.0 / 0.0)) return SDCSZ_EFORMAT;
  const Layout L = make_layout(g, n_live, n_reg, n_unpred);
  if (payload > total || total != L.payload + payload || total > nbytes) return SDCSZ_EFORMAT;
  if (h) {
    h->g = g;
    h->L = L;
    h->n_live = n_live;
    h->n_reg = n_reg;
    h->n_unpred = n_unpred;
    h->payload_bytes = payload;
    h->total = total;
    h->eb = eb;
  }
  if (pout) *pout = p;
  return SDCSZ_OK;
}

int decompress_impl(const void* d_stream, size_t nbytes, void* d_field, size_t field_bytes, uint8_t* status,
                    const void* d_orig, bool write, void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream,
                    const sdcsz_flip* flips, size_t n_flips, float* stage_ms = nullptr) {
  if (!d_stream || !d_ws) return SDCSZ_EINVAL;
  if (nbytes < (size_t)kHeaderBytes) return SDCSZ_EFORMAT;
  if (ws_bytes < sdcsz_decompress_workspace_size()) return SDCSZ_ECAPACITY;
  if (reinterpret_cast<uintptr_t>(d_ws) & 255) return SDCSZ_EINVAL;
  if (n_flips > 0xffffffffu || (n_flips && !flips)) return SDCSZ_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t hb[kHeaderBytes];
  cudaGetLastError();
  if (cudaMemcpyAsync(hb, d_stream, kHeaderBytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return SDCSZ_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SDCSZ_ECUDA;
  Hdr h;
  int rc = parse_header(hb, nbytes, &h, nullptr);
  if (rc) return rc;
  const uint64_t need = h.g.N * (h.g.dtype ? 8 : 4);
  if (write && need && (!d_field || field_bytes < need)) return d_field ? SDCSZ_ECAPACITY : SDCSZ_EINVAL;
  State* st = static_cast<State*>(d_ws);
  if (cudaMemsetAsync(st, 0, sizeof(State), s) != cudaSuccess) return SDCSZ_ECUDA;
  Launch L;
  L.stream = s;
  L.sms = sm_count();
  Trace tr;
  tr.ms = stage_ms;
  tr.n = 1;
  tr.start(s);
  launch_decode(static_cast<const uint8_t*>(d_stream), nbytes, h, d_field, status, d_orig, st, write, flips,
                (uint32_t)n_flips, L);
  tr.mark();
  if (cudaGetLastError() != cudaSuccess) return SDCSZ_ECUDA;
  tr.finish();
  if (report) {
    State hs;
    rc = read_state(st, s, &hs);
    if (rc) return rc;
    hs.n_reg = h.n_reg;
    hs.n_unpred = h.n_unpred;
    hs.total_bytes = h.total;
    hs.eb = h.eb;
    fill_report(hs, h.g.nb, report);
    rc = map_error(hs.error);
    if (rc) return rc;
    if (hs.uncorrectable) return SDCSZ_ESDC;
  }
  return SDCSZ_OK;
}

}  // namespace

}  // namespace sdcsz

using namespace sdcsz;

extern "C" {

int sdcsz_compress_bound(const sdcsz_params* p, size_t* max_bytes) {
  Geo g;
  const int rc = make_geo(p, &g);
  if (rc) return rc;
  if (!max_bytes) return SDCSZ_EINVAL;
  const Layout L = make_layout(g, g.bins, g.nb, g.N);
  *max_bytes = (size_t)(L.payload + g.nb * (((uint64_t)g.P * kMaxLen + 7) / 8));
  return SDCSZ_OK;
}

int sdcsz_workspace_size(const sdcsz_params* p, size_t* bytes) {
  Geo g;
  const int rc = make_geo(p, &g);
  if (rc) return rc;
  if (!bytes) return SDCSZ_EINVAL;
  *bytes = plan_ws(g).total;
  return SDCSZ_OK;
}

size_t sdcsz_decompress_workspace_size(void) { return align256(sizeof(State)); }

int sdcsz_compress(const void* d_field, const sdcsz_params* p, void* d_out, size_t out_cap, size_t* out_bytes,
                   void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream) {
  return compress_impl(d_field, p, d_out, out_cap, out_bytes, d_ws, ws_bytes, report, stream, nullptr, 0);
}

int sdcsz_debug_compress_flips(const void* d_field, const sdcsz_params* p, void* d_out, size_t out_cap,
                               size_t* out_bytes, void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream,
                               const sdcsz_flip* d_flips, size_t n_flips) {
  return compress_impl(d_field, p, d_out, out_cap, out_bytes, d_ws, ws_bytes, report, stream, d_flips, n_flips);
}

int sdcsz_decompress(const void* d_stream, size_t nbytes, void* d_field, size_t field_bytes, uint8_t* d_block_status,
                     void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream) {
  return decompress_impl(d_stream, nbytes, d_field, field_bytes, d_block_status, nullptr, true, d_ws, ws_bytes,
                         report, stream, nullptr, 0);
}

int sdcsz_debug_decompress_flips(const void* d_stream, size_t nbytes, void* d_field, size_t field_bytes,
                                 uint8_t* d_block_status, void* d_ws, size_t ws_bytes, sdcsz_report* report,
                                 void* stream, const sdcsz_flip* d_flips, size_t n_flips) {
  return decompress_impl(d_stream, nbytes, d_field, field_bytes, d_block_status, nullptr, true, d_ws, ws_bytes,
                         report, stream, d_flips, n_flips);
}

int sdcsz_verify(const void* d_stream, size_t nbytes, const void* d_original, uint8_t* d_block_status, void* d_ws,
                 size_t ws_bytes, sdcsz_report* report, void* stream) {
  return decompress_impl(d_stream, nbytes, nullptr, 0, d_block_status, d_original, false, d_ws, ws_bytes, report,
                         stream, nullptr, 0);
}

int sdcsz_compress_traced(const void* d_field, const sdcsz_params* p, void* d_out, size_t out_cap, size_t* out_bytes,
                          void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream, float* stage_ms) {
  if (!stage_ms) return SDCSZ_EINVAL;
  return compress_impl(d_field, p, d_out, out_cap, out_bytes, d_ws, ws_bytes, report, stream, nullptr, 0, stage_ms);
}

int sdcsz_decompress_traced(const void* d_stream, size_t nbytes, void* d_field, size_t field_bytes,
                            uint8_t* d_block_status, void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream,
                            float* stage_ms) {
  if (!stage_ms) return SDCSZ_EINVAL;
  return decompress_impl(d_stream, nbytes, d_field, field_bytes, d_block_status, nullptr, true, d_ws, ws_bytes,
                         report, stream, nullptr, 0, stage_ms);
}

int sdcsz_read_header(const void* h_stream, size_t nbytes, sdcsz_params* out, uint64_t* total_bytes) {
  if (!h_stream) return SDCSZ_EINVAL;
  Hdr h;
  sdcsz_params p;
  // only the first 128 bytes are read; the total is checked against the caller's length
  const int rc = parse_header(static_cast<const uint8_t*>(h_stream), nbytes, &h, &p);
  if (rc) return rc;
  if (out) *out = p;
  if (total_bytes) *total_bytes = h.total;
  return SDCSZ_OK;
}

const char* sdcsz_strerror(int code) {
  switch (code) {
    case SDCSZ_OK: return "ok";
    case SDCSZ_EINVAL: return "invalid argument";
    case SDCSZ_ECAPACITY: return "buffer too small";
    case SDCSZ_EFORMAT: return "not a valid sdcsz stream";
    case SDCSZ_ESDC: return "silent data corruption detected and not correctable";
    case SDCSZ_ETIMEOUT: return "device wait timed out";
    case SDCSZ_ECUDA: return "CUDA runtime error";
    default: return "unknown error";
  }
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free compression
// Some callers cannot allocate device memory at the moment they compress: code running while
// a stream is being captured into a CUDA graph (allocation is not a capturable operation),
// callbacks and latency-critical serving loops that must not enter the allocator, and hosts
// whose device memory is owned by another framework's pool. For them, sdcsz_compress_noalloc
// runs the same kernels with the workspace placed in a fixed device array of this library.

namespace sdcsz {
namespace {

// Workspace of the allocation-free entry point. Every GPU that loads this library holds these
// 64 MiB until the process exits; all calls share them.
constexpr size_t kStaticScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// In host code `g_static_scratch` only names the symbol; its device address is looked up once
// per device (with that device current) and cached.
void* static_scratch_address() {
  static std::mutex mu;
  static void* addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) return nullptr;
    addr[dev] = p;
  }
  return addr[dev];
}

}  // namespace
}  // namespace sdcsz

extern "C" int sdcsz_compress_noalloc(const void* d_field, const sdcsz_params* p, void* d_out, size_t out_cap,
                                      size_t* out_bytes, sdcsz_report* report, void* stream) {
  Geo g;
  const int rc = make_geo(p, &g);
  if (rc) return rc;
  if (plan_ws(g).total > kStaticScratchBytes) return SDCSZ_ECAPACITY;  // field too large for the array
  void* ws = static_scratch_address();
  if (!ws) return SDCSZ_ECUDA;
  // the regions that must start at zero (state, histogram, look-back records) are cleared on
  // the stream by every call; everything else is written before it is read
  return compress_impl(d_field, p, d_out, out_cap, out_bytes, ws, kStaticScratchBytes, report, stream, nullptr, 0);
}

extern "C" unsigned long long sdcsz_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }
