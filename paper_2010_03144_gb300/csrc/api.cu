// Host entry points of libsdcsz (the C ABI declared in include/sdcsz.h).
//
// Compression enqueues K1 (k_prep) -> K2 (k_predict) -> K3 (k_codebook) -> K4 (k_encode) on
// the caller's stream with no host round trip; decompression and verification read the
// 128-byte stream header to the host, then enqueue K5 (k_decode). All device memory comes
// from the caller (stream, field, workspace).
#include <algorithm>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "host.h"

namespace sdcsz {

inline namespace host {

constexpr uint64_t kMaxPoints = 1ull << 40;


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

cudaStream_t side_stream(cudaStream_t main) {
  static std::mutex mu;
  static std::map<std::pair<int, cudaStream_t>, cudaStream_t> streams;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  cudaStream_t& s = streams[{dev, main}];
  if (!s && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
  return s;
}

namespace {
std::mutex g_occ_mu;
std::map<std::tuple<int, const void*, int, size_t>, int> g_occ;
std::map<std::pair<int, const void*>, size_t> g_smem;

void allow_smem_locked(int dev, const void* kern, size_t smem) {
  size_t& cur = g_smem[{dev, kern}];
  if (smem > cur && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess)
    cur = smem;
}
}  // namespace

void allow_smem(const void* kern, size_t smem) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_occ_mu);
  allow_smem_locked(dev, kern, smem);
}

int occupancy(const void* kern, int threads, size_t smem) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_occ_mu);
  allow_smem_locked(dev, kern, smem);
  const auto key = std::make_tuple(dev, kern, threads, smem);
  auto it = g_occ.find(key);
  if (it != g_occ.end()) return it->second;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess) occ = 1;
  occ = occ < 1 ? 1 : occ;
  g_occ[key] = occ;
  return occ;
}

inline namespace host {

// Validate parameters and fill the padded-3D geometry.
int make_geo(const sdcsz_params* p, Geo* g) {
  if (!p) return SDCSZ_EINVAL;
  if (p->ndim < 1 || p->ndim > 3 || p->dtype > 1 || p->eb_mode > 1 || p->abft > 1 || p->predictor > 2 ||
      p->encoding > 3)
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
  g->enc = (int)(p->encoding & 1);
  g->lossless = (int)((p->encoding >> 1) & 1);
  g->e = p->eb;
  geo_rcp(g);
  return SDCSZ_OK;
}

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
  // the State, the histogram and the group totals first, next to each other: one reset clears them
  w.state = take(sizeof(State));
  w.hist = take(8 * 65536);
  w.gt = take(8 * std::max<size_t>(group_total_words(ngroups), 1));
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
  w.codebook = take(4 * 65536);
  w.sort_keys = take(8 * 65536);
  w.node_w = take(8 * 65536);
  w.node_parent = take(4 * 2 * 65536 + 2 * 65536);
  w.codes = take(4 * pair_slots);
  w.ustage = take(s * slots);
  w.etmp = take(4 * encode_slot_words(g) * nb);
  w.raw = w.raw_cap = w.llw = w.llst = w.llsz = w.lltop = w.lloff = w.llhist = w.llcum = 0;
  if (g.lossless) {
    w.raw_cap = raw_stream_bound(g);
    const size_t chunks = (w.raw_cap + kLLChunk - 1) / kLLChunk;
    w.raw = take(w.raw_cap);
    w.llw = take(2 * (size_t)kLLChunk * chunks);
    w.llst = take(128 * chunks);
    w.llsz = take(4 * chunks);
    w.lltop = take(4 * chunks);
    w.lloff = take(8 * chunks);
    w.llhist = take(8 * 256);
    w.llcum = take(4 * 257);
  }
  w.total = o;
  return w;
}

uint64_t raw_stream_bound(const Geo& g) {
  const Layout L = make_layout(g, g.bins, g.nb, g.N);
  return L.payload + g.nb * 4 * encode_slot_words(g);
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
  w.gt = reinterpret_cast<unsigned long long*>(b + p.gt);
  w.sort_keys = reinterpret_cast<unsigned long long*>(b + p.sort_keys);
  w.node_w = reinterpret_cast<unsigned long long*>(b + p.node_w);
  w.node_parent = reinterpret_cast<uint32_t*>(b + p.node_parent);
  w.codes = reinterpret_cast<uint16_t*>(b + p.codes);
  w.ustage = b + p.ustage;
  w.etmp = reinterpret_cast<uint32_t*>(b + p.etmp);
  w.raw = p.raw_cap ? b + p.raw : nullptr;
  w.raw_cap = p.raw_cap;
  w.llw = reinterpret_cast<uint16_t*>(b + p.llw);
  w.llst = reinterpret_cast<uint32_t*>(b + p.llst);
  w.llsz = reinterpret_cast<uint32_t*>(b + p.llsz);
  w.lltop = reinterpret_cast<uint32_t*>(b + p.lltop);
  w.lloff = reinterpret_cast<unsigned long long*>(b + p.lloff);
  w.llhist = reinterpret_cast<unsigned long long*>(b + p.llhist);
  w.llcum = reinterpret_cast<uint32_t*>(b + p.llcum);
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

// Deferred stage timing: while a recorder is open, every compression, decompression and
// verification records CUDA events between its stages on its own stream, in events created
// when the recorder opened, and returns without waiting for them; sdcsz_trace_end waits once
// and converts them to milliseconds.
constexpr int kTraceEvents = 6;  // one before the first stage and one after each of up to 5
struct Recorder {
  std::mutex mu;
  bool open = false;
  std::vector<cudaEvent_t> ev;  // cap * kTraceEvents
  std::vector<int32_t> kind;    // per call: 0 compress, 1 decompress, 2 verify
  std::vector<int32_t> marks;   // per call: events recorded when the call finished (0: unfinished)
  size_t cap = 0, used = 0, dropped = 0;
};
Recorder& recorder() {
  static Recorder r;
  return r;
}

// Stage timing of one call: synchronous (stage_ms given) or into the open recorder.
struct Trace {
  float* ms;
  int n;
  cudaEvent_t ev[8];
  cudaEvent_t* e = nullptr;
  int used = 0;
  long slot = -1;
  cudaStream_t s = nullptr;
  bool on() const { return e != nullptr; }
  void start(cudaStream_t st, int kind) {
    s = st;
    used = 0;
    if (ms) {
      for (int q = 0; q <= n && q < 8; ++q) cudaEventCreate(&ev[q]);
      e = ev;
    } else {
      Recorder& r = recorder();
      std::lock_guard<std::mutex> lk(r.mu);
      if (!r.open) return;
      if (r.used == r.cap) {
        ++r.dropped;
        return;
      }
      slot = (long)r.used++;
      r.kind[slot] = kind;
      r.marks[slot] = 0;
      e = &r.ev[(size_t)slot * kTraceEvents];
    }
    cudaEventRecord(e[0], s);
    used = 1;
  }
  void mark() {
    if (!on() || used > n) return;
    cudaEventRecord(e[used], s);
    ++used;
  }
  void finish() {
    if (!on()) return;
    if (!ms) {
      Recorder& r = recorder();
      std::lock_guard<std::mutex> lk(r.mu);
      r.marks[slot] = used;
      e = nullptr;
      return;
    }
    cudaEventSynchronize(ev[used - 1]);
    for (int q = 0; q < n; ++q) ms[q] = 0.0f;
    for (int q = 1; q < used; ++q) cudaEventElapsedTime(&ms[q - 1], ev[q - 1], ev[q]);
    for (int q = 0; q <= n && q < 8; ++q) cudaEventDestroy(ev[q]);
    used = 0;
    e = nullptr;
  }
};

int compress_impl(const void* d_field, const sdcsz_params* p, void* d_out, size_t out_cap, size_t* out_bytes,
                  void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream, const sdcsz_flip* flips,
                  size_t n_flips, float* stage_ms) {
  Geo g;
  int rc = make_geo(p, &g);
  if (rc) return rc;
  if ((!d_field && g.N) || !d_out || !d_ws) return SDCSZ_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_ws) & 255) return SDCSZ_EINVAL;
  if (n_flips > 0xffffffffu || (n_flips && !flips)) return SDCSZ_EINVAL;
  const WsPlan plan = plan_ws(g);
  if (ws_bytes < plan.total) return SDCSZ_ECAPACITY;
  if (out_cap < (size_t)kHeaderBytes) return SDCSZ_ECAPACITY;
  if (g.lossless && (reinterpret_cast<uintptr_t>(d_out) & 15)) return SDCSZ_EINVAL;
  const Ws w = bind_ws(d_ws, plan);
  // with the lossless stage the stream is first assembled in the workspace
  uint8_t* kout = g.lossless ? w.raw : static_cast<uint8_t*>(d_out);
  const uint64_t kcap = g.lossless ? w.raw_cap : out_cap;
  Launch L;
  L.stream = static_cast<cudaStream_t>(stream);
  L.sms = sm_count();
  const uint32_t nf = (uint32_t)n_flips;
  Trace tr;
  tr.ms = stage_ms;
  tr.n = 5;
  cudaGetLastError();
  tr.start(L.stream, 0);
  {  // State, histogram and group totals, adjacent in the workspace (plan_ws)
    const size_t ngroups = (g.nb + kGroup - 1) / kGroup;
    const uint8_t* end = reinterpret_cast<const uint8_t*>(w.gt) + 8 * group_total_words(ngroups);
    if (cudaMemsetAsync(w.st, 0, (size_t)(end - reinterpret_cast<const uint8_t*>(w.st)), L.stream) != cudaSuccess)
      return SDCSZ_ECUDA;
  }
  tr.mark();
  {
    NvtxRange r("sdcsz prep (range, checksums, regression, estimates)");
    launch_prep(d_field, g, w, L);
    if (nf) launch_flip_input(const_cast<void*>(d_field), g, flips, nf, w, L);
  }
  tr.mark();
  {
    NvtxRange r("sdcsz predict (prediction, quantization, checks)");
    if (g.nb) launch_predict(d_field, g, w, flips, nf, L);
    if (nf) launch_flip_codes(g, w, flips, nf, L);
  }
  tr.mark();
  {
    NvtxRange r("sdcsz codebook");
    launch_codebook(g, w, kout, kcap, L);
  }
  tr.mark();
  {
    NvtxRange r("sdcsz encode");
    launch_encode(d_field, g, w, kout, kcap, L);
  }
  if (g.lossless) {
    NvtxRange r("sdcsz lossless stage");
    launch_ll_pack(g, w, static_cast<uint8_t*>(d_out), out_cap, L);
  }
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
  p.encoding = s[51];
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
  uint64_t raw_total = total;
  if (g.lossless) std::memcpy(&raw_total, s + 120, 8);
  if (payload > raw_total || raw_total != L.payload + payload || total > nbytes) return SDCSZ_EFORMAT;
  if (g.lossless && ll_data(L.sumdc, ll_chunks(L.sumdc, raw_total)) > total) return SDCSZ_EFORMAT;
  if (h) {
    h->g = g;
    h->L = L;
    h->n_live = n_live;
    h->n_reg = n_reg;
    h->n_unpred = n_unpred;
    h->payload_bytes = payload;
    h->total = total;
    h->raw_total = raw_total;
    h->eb = eb;
    if (p.dtype == 0) {
      const float ebf = (float)eb;
      uint32_t u;
      std::memcpy(&u, &ebf, 4);
      h->texp = (int)((u >> 23) & 0xffu) - 127;
    } else {
      uint64_t u;
      std::memcpy(&u, &eb, 8);
      h->texp = (int)((u >> 52) & 0x7ffu) - 1023;
    }
    const CoefSteps cs = coef_steps(g, eb);
    for (int a = 0; a < 4; ++a) h->cstep[a] = cs.step[a];
  }
  if (pout) *pout = p;
  return SDCSZ_OK;
}

int decode_enqueue(const void* d_stream, size_t nbytes, const Hdr& h, void* d_field, size_t field_bytes,
                   uint8_t* status, const void* d_orig, bool write, State* st, cudaStream_t s, const sdcsz_flip* flips,
                   size_t n_flips, uint8_t* raw, uint8_t* wave) {
  const uint64_t need = h.g.N * (h.g.dtype ? 8 : 4);
  if (write && need && (!d_field || field_bytes < need)) return d_field ? SDCSZ_ECAPACITY : SDCSZ_EINVAL;
  if (n_flips > 0xffffffffu || (n_flips && !flips)) return SDCSZ_EINVAL;
  if (h.g.lossless && (!raw || (reinterpret_cast<uintptr_t>(raw) & 15) ||
                       (reinterpret_cast<uintptr_t>(d_stream) & 15)))
    return SDCSZ_EINVAL;
  if (cudaMemsetAsync(st, 0, sizeof(State), s) != cudaSuccess) return SDCSZ_ECUDA;
  Launch L;
  L.stream = s;
  L.sms = sm_count();
  const uint8_t* src = static_cast<const uint8_t*>(d_stream);
  uint64_t n = nbytes;
  if (h.g.lossless) {  // Algorithm 2's first step: undo the lossless stage into `raw`
    launch_ll_unpack(src, nbytes, h, raw, st, L);
    src = raw;
    n = h.raw_total;
  }
  launch_decode(src, n, h, d_field, status, d_orig, st, write, flips, (uint32_t)n_flips, L, wave);
  return SDCSZ_OK;
}

// Decompression workspace: the State, then (lossless stage) the stream without the stage, then
// (recommended size) the two-pass decoder's buffers.
size_t decode_ws_min(const Hdr& h) { return align256(sizeof(State)) + (h.g.lossless ? align256(h.raw_total) : 0); }
size_t decode_ws_bytes(const Hdr& h) { return decode_ws_min(h) + wave_decode_ws_bytes(h.g); }

int decompress_impl(const void* d_stream, size_t nbytes, void* d_field, size_t field_bytes, uint8_t* status,
                    const void* d_orig, bool write, void* d_ws, size_t ws_bytes, sdcsz_report* report, void* stream,
                    const sdcsz_flip* flips, size_t n_flips, float* stage_ms) {
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
  if (ws_bytes < decode_ws_min(h)) return SDCSZ_ECAPACITY;
  State* st = static_cast<State*>(d_ws);
  uint8_t* raw = static_cast<uint8_t*>(d_ws) + align256(sizeof(State));
  // the two-pass decoder of large cube blocks when the workspace holds its buffers
  uint8_t* wave = (wave_decode_ws_bytes(h.g) && ws_bytes >= decode_ws_bytes(h))
                      ? static_cast<uint8_t*>(d_ws) + decode_ws_min(h)
                      : nullptr;
  Trace tr;
  tr.ms = stage_ms;
  tr.n = 1;
  tr.start(s, write ? 1 : 2);
  {
    NvtxRange r(write ? "sdcsz decode" : "sdcsz verify");
    rc = decode_enqueue(d_stream, nbytes, h, d_field, field_bytes, status, d_orig, write, st, s, flips, n_flips, raw,
                        wave);
  }
  if (rc) return rc;
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
  uint64_t b = raw_stream_bound(g);
  if (g.lossless) {  // up to 2 bytes per coded byte, the tables and each chunk's states
    const Layout L = make_layout(g, g.bins, g.nb, g.N);
    const uint64_t n = b - L.sumdc, nch = ll_chunks(L.sumdc, b);
    b = ll_data(L.sumdc, nch) + 2 * n + nch * 132;
  }
  *max_bytes = (size_t)b;
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

int sdcsz_decompress_workspace_size_for(const void* h_header, size_t nbytes, size_t* bytes) {
  if (!h_header || !bytes) return SDCSZ_EINVAL;
  Hdr h;
  const int rc = parse_header(static_cast<const uint8_t*>(h_header), nbytes, &h, nullptr);
  if (rc) return rc;
  *bytes = decode_ws_bytes(h);
  return SDCSZ_OK;
}

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

int sdcsz_trace_begin(size_t max_calls) {
  if (max_calls == 0 || max_calls > (1u << 20)) return SDCSZ_EINVAL;
  Recorder& r = recorder();
  std::lock_guard<std::mutex> lk(r.mu);
  if (r.open) return SDCSZ_EINVAL;
  r.ev.assign(max_calls * kTraceEvents, nullptr);
  for (size_t q = 0; q < r.ev.size(); ++q)
    if (cudaEventCreate(&r.ev[q]) != cudaSuccess) {
      for (size_t k = 0; k < q; ++k) cudaEventDestroy(r.ev[k]);
      r.ev.clear();
      return SDCSZ_ECUDA;
    }
  r.kind.assign(max_calls, 0);
  r.marks.assign(max_calls, 0);
  r.cap = max_calls;
  r.used = 0;
  r.dropped = 0;
  r.open = true;
  return SDCSZ_OK;
}

int sdcsz_trace_end(int32_t* kinds, float* stage_ms, size_t cap_calls, size_t* n_calls) {
  Recorder& r = recorder();
  std::lock_guard<std::mutex> lk(r.mu);
  if (!r.open) return SDCSZ_EINVAL;
  int rc = SDCSZ_OK;
  size_t n = 0;
  for (size_t c = 0; c < r.used; ++c) {
    const int m = r.marks[c];
    if (m < 2) continue;  // a call that returned an error before its last stage
    if (n < cap_calls && kinds && stage_ms) {
      cudaEvent_t* e = &r.ev[c * kTraceEvents];
      if (cudaEventSynchronize(e[m - 1]) != cudaSuccess) rc = SDCSZ_ECUDA;
      float* o = stage_ms + n * (kTraceEvents - 1);
      for (int q = 0; q < kTraceEvents - 1; ++q) o[q] = 0.0f;
      for (int q = 1; q < m && rc == SDCSZ_OK; ++q)
        if (cudaEventElapsedTime(&o[q - 1], e[q - 1], e[q]) != cudaSuccess) rc = SDCSZ_ECUDA;
      kinds[n] = r.kind[c];
    }
    ++n;
  }
  for (cudaEvent_t ev : r.ev) cudaEventDestroy(ev);
  r.ev.clear();
  r.open = false;
  if (n_calls) *n_calls = n;
  if (rc == SDCSZ_OK && (r.dropped || n > cap_calls || ((!kinds || !stage_ms) && n))) rc = SDCSZ_ECAPACITY;
  return rc;
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
// Some callers cannot allocate device memory at the moment they compress: callbacks and
// latency-critical serving loops that must not enter the allocator (cudaMalloc can
// synchronize the device), and hosts whose device memory is owned by another framework's
// pool. For them, sdcsz_compress_noalloc runs the same kernels with the workspace placed in a
// fixed device array of this library.

namespace sdcsz {
namespace {

// Workspace of the allocation-free entry point. Every GPU that loads this library holds these
// 64 MiB until the process exits; all calls share them.
constexpr size_t kStaticScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// In host code `g_static_scratch` only names the symbol; its device address is looked up once
// per device (with that device current) and cached for the life of the process (a
// cudaDeviceReset invalidates it; the header tells callers not to use the entry point after one).
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

extern "C" int sdcsz_decompress_region(const void* d_stream, size_t nbytes, const uint64_t* lo, const uint64_t* hi,
                                       void* d_out, size_t out_bytes, uint8_t* d_block_status, void* d_ws,
                                       size_t ws_bytes, sdcsz_report* report, void* stream) {
  using namespace sdcsz;
  if (!d_stream || !d_ws || !lo || !hi) return SDCSZ_EINVAL;
  if (nbytes < (size_t)kHeaderBytes) return SDCSZ_EFORMAT;
  if (ws_bytes < sdcsz_decompress_workspace_size()) return SDCSZ_ECAPACITY;
  if (reinterpret_cast<uintptr_t>(d_ws) & 255) return SDCSZ_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t hb[kHeaderBytes];
  cudaGetLastError();
  if (cudaMemcpyAsync(hb, d_stream, kHeaderBytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return SDCSZ_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SDCSZ_ECUDA;
  Hdr h;
  int rc = parse_header(hb, nbytes, &h, nullptr);
  if (rc) return rc;
  if (ws_bytes < decode_ws_min(h)) return SDCSZ_ECAPACITY;
  if (h.g.lossless && (reinterpret_cast<uintptr_t>(d_stream) & 15)) return SDCSZ_EINVAL;
  // the box in padded 3D coordinates
  uint64_t lo3[3] = {0, 0, 0}, hi3[3] = {1, 1, 1}, pts = 1, nblk = 1;
  const int off = 3 - h.g.ndim;
  for (int a = 0; a < h.g.ndim; ++a) {
    if (lo[a] >= hi[a] || hi[a] > h.g.d[off + a]) return SDCSZ_EINVAL;
    lo3[off + a] = lo[a];
    hi3[off + a] = hi[a];
    pts *= hi[a] - lo[a];
    nblk *= (hi[a] - 1) / h.g.B[off + a] - lo[a] / h.g.B[off + a] + 1;
  }
  if (!d_out || out_bytes < pts * (h.g.dtype ? 8 : 4)) return d_out ? SDCSZ_ECAPACITY : SDCSZ_EINVAL;
  State* st = static_cast<State*>(d_ws);
  if (cudaMemsetAsync(st, 0, sizeof(State), s) != cudaSuccess) return SDCSZ_ECUDA;
  Launch L;
  L.stream = s;
  L.sms = sm_count();
  {
    NvtxRange r("sdcsz decode region");
    const uint8_t* src = static_cast<const uint8_t*>(d_stream);
    uint64_t n = nbytes;
    if (h.g.lossless) {  // the whole stage is undone (its chunks do not follow block boundaries)
      uint8_t* raw = static_cast<uint8_t*>(d_ws) + align256(sizeof(State));
      launch_ll_unpack(src, nbytes, h, raw, st, L);
      src = raw;
      n = h.raw_total;
    }
    launch_region(src, n, h, d_out, lo3, hi3, d_block_status, st, L);
  }
  if (cudaGetLastError() != cudaSuccess) return SDCSZ_ECUDA;
  if (report) {
    State hs;
    rc = read_state(st, s, &hs);
    if (rc) return rc;
    hs.n_reg = h.n_reg;
    hs.n_unpred = h.n_unpred;
    hs.total_bytes = h.total;
    hs.eb = h.eb;
    fill_report(hs, nblk, report);
    rc = map_error(hs.error);
    if (rc) return rc;
    if (hs.uncorrectable) return SDCSZ_ESDC;
  }
  return SDCSZ_OK;
}

extern "C" int sdcsz_compress_noalloc(const void* d_field, const sdcsz_params* p, void* d_out, size_t out_cap,
                                      size_t* out_bytes, sdcsz_report* report, void* stream) {
  Geo g;
  const int rc = make_geo(p, &g);
  if (rc) return rc;
  if (plan_ws(g).total > kStaticScratchBytes) return SDCSZ_ECAPACITY;  // field too large for the array
  void* ws = static_scratch_address();
  if (!ws) return SDCSZ_ECUDA;
  // the regions that must start at zero (state, histogram, group totals) are cleared on
  // the stream by every call; everything else is written before it is read
  return compress_impl(d_field, p, d_out, out_cap, out_bytes, ws, kStaticScratchBytes, report, stream, nullptr, 0);
}

extern "C" unsigned long long sdcsz_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------- batches
// A batch holds the plan of one set of fields: each field's geometry and workspace slice, the
// device job table, and the launches of each stage (one per kernel shape, each a persistent
// grid pulling items from its own queue counter). Compression of the whole batch is a fixed
// sequence of launches on one stream (edge-block launches forked to a batch-owned side
// stream and joined), with no host synchronisation, so it can be captured into a CUDA graph
// and replayed; the kernels read fields, outputs and workspaces from the job table, so a
// replay after sdcsz_batch_set_fields works on new buffers of the same shapes.
namespace sdcsz {
namespace {

__global__ void k_batch_reset(const Job* __restrict__ jobs, unsigned long long* heads, uint32_t nheads) {
  const Job& jb = jobs[blockIdx.x];
  const uint64_t ngroups = (jb.g.nb + kGroup - 1) / kGroup;
  const uint64_t nst = sizeof(State) / 8, nh = jb.g.bins, nl = group_total_words(ngroups);
  unsigned long long* st = reinterpret_cast<unsigned long long*>(jb.w.st);
  unsigned long long* gt = jb.w.gt;
  for (uint64_t q = (uint64_t)blockIdx.y * blockDim.x + threadIdx.x; q < nst + nh + nl;
       q += (uint64_t)gridDim.y * blockDim.x) {
    if (q < nst) st[q] = 0ull;
    else if (q < nst + nh) jb.w.hist[q - nst] = 0ull;
    else gt[q - nst - nh] = 0ull;
  }
  if (blockIdx.x == 0 && blockIdx.y == 0)
    for (uint32_t q = threadIdx.x; q < nheads; q += blockDim.x) heads[q] = 0ull;
}

enum BatchKind { BK_PREP_FAST, BK_PREP_GENERIC, BK_PREDICT_FAST, BK_PREDICT_GENERIC, BK_ENCODE_BLOCKS, BK_ENCODE };

struct BatchLaunch {
  BatchKind kind;
  int dtype, ndim;
  uint32_t B;
  bool abft;
  bool enc;  // compact encoding (the fast predict kernels are instantiated per encoding)
  uint32_t threads;
  size_t smem;
  std::vector<uint32_t> jobs;
  std::vector<uint64_t> items;
  BatchArgs args;
};

uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

}  // namespace
}  // namespace sdcsz

struct sdcsz_batch {
  std::vector<sdcsz_batch_item> items;
  std::vector<sdcsz::Geo> geo;
  std::vector<sdcsz::WsPlan> plan;
  std::vector<size_t> ws_off;
  std::vector<sdcsz::BatchLaunch> launches;
  size_t heads_off = 0, table_off = 0, total = 0;
  void* d_ws = nullptr;
  sdcsz::Job* h_table = nullptr;  // pinned host copy of the job table
  sdcsz::Job* d_table = nullptr;
  unsigned long long* d_heads = nullptr;
  int device = -1;
  cudaStream_t side = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaGraphExec_t exec = nullptr;
};

namespace sdcsz {
namespace {

void batch_release(sdcsz_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto& e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->h_table) cudaFreeHost(b->h_table);
  b->exec = nullptr;
  b->side = nullptr;
  b->h_table = nullptr;
  for (auto& e : b->ev) e = nullptr;
}

// The job table entries that depend on the caller's buffers.
void batch_fill_jobs(sdcsz_batch* b) {
  for (size_t j = 0; j < b->items.size(); ++j) {
    Job& jb = b->h_table[j];
    const Geo& g = b->geo[j];
    const size_t s = g.dtype ? 8 : 4;
    jb.field = b->items[j].d_field;
    jb.out = static_cast<uint8_t*>(b->items[j].d_out);
    jb.cap = b->items[j].out_cap;
    jb.vec2 = (g.B[2] % 2 == 0) && (g.d[2] % 2 == 0) && (reinterpret_cast<uintptr_t>(jb.field) % (2 * s) == 0);
  }
}

// Group the jobs into launches (one per stage and kernel shape) and number their items.
void batch_plan_launches(sdcsz_batch* b) {
  b->launches.clear();
  auto add = [&](BatchKind kind, int dtype, int ndim, uint32_t B, bool abft, uint32_t threads, size_t smem,
                 uint32_t j, uint64_t items, bool enc = false) {
    if (!items) return;
    for (auto& L : b->launches)
      if (L.kind == kind && L.dtype == dtype && L.ndim == ndim && L.B == B && L.abft == abft && L.enc == enc) {
        L.jobs.push_back(j);
        L.items.push_back(items);
        L.threads = std::min(L.threads, threads);
        L.smem = std::max(L.smem, smem);
        return;
      }
    BatchLaunch L;
    L.kind = kind;
    L.dtype = dtype;
    L.ndim = ndim;
    L.B = B;
    L.abft = abft;
    L.enc = enc;
    L.threads = threads;
    L.smem = smem;
    L.jobs.push_back(j);
    L.items.push_back(items);
    b->launches.push_back(L);
  };
  for (uint32_t j = 0; j < (uint32_t)b->geo.size(); ++j) {
    const Geo& g = b->geo[j];
    const Job& jb = b->h_table[j];
    const size_t s = g.dtype ? 8 : 4;
    const uint32_t slots = walker_slots(g.ndim, g.B);
    if (jb.fast) {
      add(BK_PREP_FAST, g.dtype, g.ndim, g.B[2], false, 128, 0, j, ceil_div(g.nb, 128));
      // wavefront shapes: items are groups of full blocks, then groups of edge blocks
      const uint64_t wg = wave_groups(g);
      add(BK_PREDICT_FAST, g.dtype, g.ndim, g.B[2], g.abft != 0, 128, 0, j, wg ? wg : ceil_div(g.nb, 128),
          g.enc != 0);
    }
    add(BK_PREP_GENERIC, g.dtype, g.ndim, 0, false, 128, g.predictor == 0 ? (size_t)slots * 128 * 4 : 0, j,
        ceil_div(jb.gcount, 128));
    uint32_t threads = 128;
    while (threads > 32 && (size_t)slots * s * threads > 160 * 1024) threads >>= 1;
    add(BK_PREDICT_GENERIC, g.dtype, g.ndim, 0, g.abft != 0, threads, 0, j, 1);  // items set below
    add(BK_ENCODE_BLOCKS, g.dtype, 0, 0, g.abft != 0, 128, 0, j, ceil_div(g.nb, 128));
    add(BK_ENCODE, g.dtype, 0, 0, false, 256, 0, j, ceil_div(g.nb, kGroup));
  }
  // generic predict: threads are the class minimum, so the items follow it
  for (auto& L : b->launches) {
    if (L.kind != BK_PREDICT_GENERIC) continue;
    size_t per = 0;
    std::vector<uint32_t> jobs;
    std::vector<uint64_t> items;
    for (uint32_t j : L.jobs) {
      const Geo& g = b->geo[j];
      // the wavefront kernel predicts the edge blocks of its shapes too
      const uint64_t n = (b->h_table[j].fast && wave_groups(g)) ? 0 : ceil_div(b->h_table[j].gcount, L.threads);
      if (!n) continue;
      per = std::max(per, (size_t)walker_slots(g.ndim, g.B) * (g.dtype ? 8 : 4));
      jobs.push_back(j);
      items.push_back(n);
    }
    L.jobs = jobs;
    L.items = items;
    L.smem = per * L.threads;
  }
  b->launches.erase(std::remove_if(b->launches.begin(), b->launches.end(),
                                   [](const BatchLaunch& L) { return L.jobs.empty(); }),
                    b->launches.end());
  for (size_t q = 0; q < b->launches.size(); ++q) {
    BatchLaunch& L = b->launches[q];
    std::memset(&L.args, 0, sizeof(L.args));
    L.args.jobs = b->d_table;
    L.args.head = b->d_heads + q;
    L.args.n = (uint32_t)L.jobs.size();
    uint64_t acc = 0;
    for (size_t t = 0; t < L.jobs.size(); ++t) {
      L.args.idx[t] = L.jobs[t];
      L.args.start[t] = acc;
      acc += L.items[t];
    }
    L.args.start[L.jobs.size()] = acc;
  }
}

// Enqueue the whole batch on `s` (no host synchronisation).
int batch_enqueue(sdcsz_batch* b, cudaStream_t s) {
  NvtxRange r("sdcsz batch compress");
  Launch L;
  L.stream = s;
  L.sms = sm_count();
  Launch Ls = L;
  Ls.stream = b->side;
  const uint32_t n = (uint32_t)b->items.size();
  cudaGetLastError();
  k_batch_reset<<<dim3(n, 16), 256, 0, s>>>(b->d_table, b->d_heads, (uint32_t)kMaxQueues);
  note_launch();
  auto stage = [&](BatchKind fast_kind, BatchKind gen_kind, int e) {
    cudaEventRecord(b->ev[e], s);
    cudaStreamWaitEvent(b->side, b->ev[e], 0);
    for (auto& Q : b->launches) {
      if (Q.kind == gen_kind) {
        if (gen_kind == BK_PREP_GENERIC) batch_prep_generic(Q.dtype, Q.ndim, Q.args, Q.smem, Ls);
        else batch_predict_generic(Q.dtype, Q.ndim, Q.abft, Q.args, Q.threads, Q.smem, Ls);
      }
    }
    for (auto& Q : b->launches) {
      if (Q.kind == fast_kind) {
        if (fast_kind == BK_PREP_FAST) batch_prep_fast(Q.dtype, Q.ndim, Q.B, Q.args, L);
        else batch_predict_fast(Q.dtype, Q.ndim, Q.B, Q.abft, Q.enc, Q.args, L);
      }
    }
    cudaEventRecord(b->ev[e + 1], b->side);
    cudaStreamWaitEvent(s, b->ev[e + 1], 0);
  };
  stage(BK_PREP_FAST, BK_PREP_GENERIC, 0);
  batch_bound(b->d_table, n, L);
  stage(BK_PREDICT_FAST, BK_PREDICT_GENERIC, 2);
  batch_codebook(b->d_table, n, L);
  for (auto& Q : b->launches)
    if (Q.kind == BK_ENCODE_BLOCKS) batch_encode_blocks(Q.dtype, Q.abft, Q.args, L);
  for (auto& Q : b->launches)
    if (Q.kind == BK_ENCODE) batch_encode_assemble(Q.dtype, Q.args, L);
  return cudaGetLastError() == cudaSuccess ? SDCSZ_OK : SDCSZ_ECUDA;
}

}  // namespace
}  // namespace sdcsz

extern "C" {

int sdcsz_batch_create(const sdcsz_batch_item* items, uint32_t n, sdcsz_batch** out) {
  using namespace sdcsz;
  if (!out || !items || n == 0 || n > (uint32_t)kMaxBatch) return SDCSZ_EINVAL;
  *out = nullptr;
  sdcsz_batch* b = new sdcsz_batch();
  b->items.assign(items, items + n);
  size_t o = 0;
  b->heads_off = o;
  o = align256(o + 8 * kMaxQueues);
  b->table_off = o;
  o = align256(o + sizeof(Job) * n);
  for (uint32_t j = 0; j < n; ++j) {
    Geo g;
    const int rc = make_geo(&items[j].params, &g);
    if (rc || g.lossless) {  // the lossless stage runs per field (sdcsz_compress), not in batches
      delete b;
      return rc ? rc : SDCSZ_EINVAL;
    }
    b->geo.push_back(g);
    b->plan.push_back(plan_ws(g));
    b->ws_off.push_back(o);
    o = align256(o + b->plan.back().total);
  }
  b->total = o;
  *out = b;
  return SDCSZ_OK;
}

int sdcsz_batch_workspace_size(const sdcsz_batch* b, size_t* bytes) {
  if (!b || !bytes) return SDCSZ_EINVAL;
  *bytes = b->total;
  return SDCSZ_OK;
}

int sdcsz_batch_bind(sdcsz_batch* b, void* d_ws, size_t ws_bytes, void* stream) {
  using namespace sdcsz;
  if (!b || !d_ws || ws_bytes < b->total || (reinterpret_cast<uintptr_t>(d_ws) & 255)) return SDCSZ_EINVAL;
  const uint32_t n = (uint32_t)b->items.size();
  for (uint32_t j = 0; j < n; ++j) {
    const sdcsz_batch_item& it = b->items[j];
    if ((!it.d_field && b->geo[j].N) || !it.d_out || it.out_cap < (size_t)kHeaderBytes) return SDCSZ_EINVAL;
  }
  batch_release(b);
  if (cudaGetDevice(&b->device) != cudaSuccess) return SDCSZ_ECUDA;
  if (cudaMallocHost(&b->h_table, sizeof(Job) * n) != cudaSuccess) return SDCSZ_ECUDA;
  if (cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess) return SDCSZ_ECUDA;
  for (auto& e : b->ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return SDCSZ_ECUDA;
  uint8_t* base = static_cast<uint8_t*>(d_ws);
  b->d_ws = d_ws;
  b->d_heads = reinterpret_cast<unsigned long long*>(base + b->heads_off);
  b->d_table = reinterpret_cast<Job*>(base + b->table_off);
  std::memset(b->h_table, 0, sizeof(Job) * n);
  for (uint32_t j = 0; j < n; ++j) {
    Job& jb = b->h_table[j];
    jb.g = b->geo[j];
    jb.w = bind_ws(base + b->ws_off[j], b->plan[j]);
    jb.fast = prep_has_fast(jb.g) ? 1 : 0;
    jb.gcount = jb.fast ? edge_count(jb.g) : jb.g.nb;
  }
  batch_fill_jobs(b);
  batch_plan_launches(b);
  if (b->launches.size() > (size_t)kMaxQueues) return SDCSZ_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(b->d_table, b->h_table, sizeof(Job) * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return SDCSZ_ECUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? SDCSZ_OK : SDCSZ_ECUDA;
}

int sdcsz_batch_set_fields(sdcsz_batch* b, const void* const* d_fields, void* const* d_outs, const size_t* out_caps,
                           void* stream) {
  using namespace sdcsz;
  if (!b || !b->h_table) return SDCSZ_EINVAL;
  const uint32_t n = (uint32_t)b->items.size();
  for (uint32_t j = 0; j < n; ++j) {
    if (d_fields) {
      if (!d_fields[j] && b->geo[j].N) return SDCSZ_EINVAL;
      b->items[j].d_field = d_fields[j];
    }
    if (d_outs) {
      if (!d_outs[j]) return SDCSZ_EINVAL;
      b->items[j].d_out = d_outs[j];
    }
    if (out_caps) {
      if (out_caps[j] < (size_t)kHeaderBytes) return SDCSZ_EINVAL;
      b->items[j].out_cap = out_caps[j];
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the pinned table may still be in flight from an earlier update
  if (cudaStreamSynchronize(s) != cudaSuccess) return SDCSZ_ECUDA;
  batch_fill_jobs(b);
  if (cudaMemcpyAsync(b->d_table, b->h_table, sizeof(Job) * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return SDCSZ_ECUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? SDCSZ_OK : SDCSZ_ECUDA;
}

int sdcsz_batch_compress(sdcsz_batch* b, void* stream) {
  if (!b || !b->h_table) return SDCSZ_EINVAL;
  return sdcsz::batch_enqueue(b, static_cast<cudaStream_t>(stream));
}

int sdcsz_batch_capture(sdcsz_batch* b, void* stream) {
  if (!b || !b->h_table || !stream) return SDCSZ_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SDCSZ_ECUDA;
  const int rc = sdcsz::batch_enqueue(b, s);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (rc || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc ? rc : SDCSZ_ECUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    b->exec = nullptr;
    return SDCSZ_ECUDA;
  }
  return SDCSZ_OK;
}

int sdcsz_batch_launch(sdcsz_batch* b, void* stream) {
  if (!b || !b->h_table) return SDCSZ_EINVAL;
  if (!b->exec) return sdcsz::batch_enqueue(b, static_cast<cudaStream_t>(stream));
  return cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? SDCSZ_OK : SDCSZ_ECUDA;
}

int sdcsz_batch_results(sdcsz_batch* b, size_t* out_bytes, sdcsz_report* reports, void* stream) {
  using namespace sdcsz;
  if (!b || !b->h_table) return SDCSZ_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t n = (uint32_t)b->items.size();
  int first = SDCSZ_OK;
  std::vector<State> h(n);
  for (uint32_t j = 0; j < n; ++j)
    if (cudaMemcpyAsync(&h[j], b->h_table[j].w.st, sizeof(State), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return SDCSZ_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SDCSZ_ECUDA;
  for (uint32_t j = 0; j < n; ++j) {
    const int rc = map_error(h[j].error);
    if (reports) fill_report(h[j], b->geo[j].nb, &reports[j]);
    if (out_bytes) out_bytes[j] = rc ? 0 : (size_t)h[j].total_bytes;
    if (rc && !first) first = rc;
  }
  return first;
}

void sdcsz_batch_destroy(sdcsz_batch* b) {
  if (!b) return;
  sdcsz::batch_release(b);
  delete b;
}

}  // extern "C"

// ---------------------------------------------------------------- block-size autotuner
// Compresses a leading slab of the field (contiguous, so no copy) with each candidate block
// edge and times it with CUDA events; the choice is the fastest candidate whose compressed
// size is within `size_slack` of the smallest. At a fixed error bound the compressed size is
// the rate side of the paper's rate-distortion block-size study (Sec. 6.2.1): the slack bounds
// the rate given up for speed.
extern "C" int sdcsz_autotune_block(const void* d_field, const sdcsz_params* p, const uint32_t* candidates,
                                    uint32_t n_cand, uint64_t sample_points, double size_slack, void* stream,
                                    sdcsz_tune_result* results, uint32_t* best) {
  using namespace sdcsz;
  Geo g;
  int rc = make_geo(p, &g);
  if (rc) return rc;
  if (!d_field || !candidates || !n_cand || !results || !best || !(size_slack >= 0.0 && size_slack < 1e6))
    return SDCSZ_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the sample: whole planes (3D), rows (2D) or a prefix (1D) up to sample_points
  sdcsz_params q = *p;
  const uint64_t inner = g.ndim == 1 ? 1 : (g.ndim == 2 ? g.d[2] : g.d[1] * g.d[2]);
  const uint64_t outer = g.ndim == 1 ? g.d[2] : (g.ndim == 2 ? g.d[1] : g.d[0]);
  uint64_t take = std::max<uint64_t>(1, sample_points / std::max<uint64_t>(inner, 1));
  take = std::min(take, outer);
  q.dims[0] = take;
  std::vector<sdcsz_params> cp(n_cand, q);
  size_t ws_max = 0, out_max = 0;
  for (uint32_t c = 0; c < n_cand; ++c) {
    for (uint32_t a = 0; a < q.ndim; ++a) cp[c].block[a] = candidates[c];
    Geo gc;
    rc = make_geo(&cp[c], &gc);
    if (rc) return rc;
    size_t cap = 0;
    if ((rc = sdcsz_compress_bound(&cp[c], &cap))) return rc;
    ws_max = std::max(ws_max, plan_ws(gc).total);
    out_max = std::max(out_max, cap);
  }
  void *ws = nullptr, *out = nullptr;
  if (cudaMallocAsync(&ws, ws_max, s) != cudaSuccess) return SDCSZ_ECUDA;
  if (cudaMallocAsync(&out, out_max, s) != cudaSuccess) {
    cudaFreeAsync(ws, s);
    return SDCSZ_ECUDA;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  uint64_t smallest = ~0ull;
  const int reps = 3;
  for (uint32_t c = 0; c < n_cand && !rc; ++c) {
    size_t nbytes = 0;
    rc = compress_impl(d_field, &cp[c], out, out_max, &nbytes, ws, ws_max, nullptr, stream, nullptr, 0);
    if (rc) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && !rc; ++r)
      rc = compress_impl(d_field, &cp[c], out, out_max, nullptr, ws, ws_max, nullptr, stream, nullptr, 0);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = SDCSZ_ECUDA;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double in_bytes = (double)take * inner * (p->dtype ? 8.0 : 4.0);
    results[c].block = candidates[c];
    results[c].ms = ms / reps;
    results[c].bytes = nbytes;
    results[c].gbs = in_bytes / (results[c].ms * 1e-3) / 1e9;
    results[c].ratio = nbytes ? in_bytes / (double)nbytes : 0.0;
    smallest = std::min<uint64_t>(smallest, nbytes);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(ws, s);
  cudaFreeAsync(out, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = SDCSZ_ECUDA;
  if (rc) return rc;
  uint32_t pick = 0;
  bool have = false;
  for (uint32_t c = 0; c < n_cand; ++c) {
    if ((double)results[c].bytes > (1.0 + size_slack) * (double)smallest) continue;
    if (!have || results[c].gbs > results[pick].gbs) {
      pick = c;
      have = true;
    }
  }
  *best = pick;
  return SDCSZ_OK;
}
